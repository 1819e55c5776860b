"""GPU: fused multi-field sweeps (several stencils in one pass, the coupled
system u_k <- u_k + sum_j A[k][j] L(u_j)) against the FP64 oracle, bit for bit
against independent heat sweeps when A = a I, and across every compiled variant.
Tolerance: 1e-5 max-norm relative (FP32 storage), as for the heat sweeps."""
import json

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
A3 = np.array([[0.030, 0.012, -0.004],
               [0.007, 0.025, 0.009],
               [0.002, -0.006, 0.020]])
A4 = np.array([[0.020, 0.005, 0.000, 0.003],
               [0.004, 0.025, 0.006, 0.000],
               [0.000, 0.002, 0.018, 0.004],
               [0.001, 0.000, 0.003, 0.022]])


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_system(dims, so, A, seeds, **kw):
    from paper_2404_02218_gb300.grid import System
    s = System(dims, so, A, **kw)
    u = [synthetic.uniform_field(sd, tuple(reversed(dims))) for sd in seeds]
    for k, f in enumerate(u):
        s.set_field(k, "u", f)
    return s, u


@pytest.mark.parametrize("so", [2, 4, 8])
def test_diagonal_system_equals_heat_sweeps_bitwise(torch_cuda, so):
    from paper_2404_02218_gb300.grid import Grid
    dims = (70, 45, 33)
    a = float(np.float32(0.8 * synthetic.heat_a_max(3, so)))
    s, u = make_system(dims, so, a * np.eye(3), (11, 12, 13))
    s.run(7)
    for k in range(3):
        g = Grid(3, dims, so, "heat", dt=a, temporal_block=1)
        g.set_field("u", u[k])
        g.run(7)
        np.testing.assert_array_equal(s.get_field(k, "u"), g.get_field("u"))
        g.close()


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("A", [A3, A3[:2, :2], A4], ids=["nf3", "nf2", "nf4"])
@pytest.mark.parametrize("dims", [(130, 37, 21), (9, 5, 3)])
def test_coupled_system_matches_oracle(torch_cuda, so, A, dims):
    nf = A.shape[0]
    seeds = tuple(range(20, 20 + nf))
    s, u = make_system(dims, so, A, seeds)
    s.run(6)
    ref = oracle.system_run(u, so, A.astype(np.float32).astype(np.float64), 6)
    for k in range(nf):
        assert oracle.max_rel_error(s.get_field(k, "u"), ref[k]) <= TOL_F32, k


def test_every_system_variant_bitwise(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    dims = (140, 30, 19)
    for so in (2, 4, 8):
        s, u = make_system(dims, so, A3, (31, 32, 33))
        s.run(4)
        want = [s.get_field(k, "u") for k in range(3)]
        variants = [i for i in range(N.stencil_variant_count())
                    if (lambda v: v["nf"] == 3 and v["R"] == so // 2)(json.loads(N.stencil_variant_info(i)))]
        assert variants
        for v in variants:
            for zc, sched in ((0, 1), (3, 1), (3, 0)):
                t, _ = make_system(dims, so, A3, (31, 32, 33))
                t.set_schedule(sched)
                t.set_plan(v, 0, zc, 0)
                t.run(4)
                for k in range(3):
                    np.testing.assert_array_equal(t.get_field(k, "u"), want[k],
                                                  err_msg=f"variant {v} zc {zc} schedule {sched}")
                t.close()
        s.close()


def test_split_runs_graphs_and_reductions(torch_cuda):
    dims = (64, 40, 30)
    s1, u = make_system(dims, 4, A3, (41, 42, 43))
    s1.run(3)
    s1.run(5)
    s2, _ = make_system(dims, 4, A3, (41, 42, 43), use_graph=False)
    s2.run(8)
    for k in range(3):
        a, b = s1.get_field(k, "u"), s2.get_field(k, "u")
        np.testing.assert_array_equal(a, b)
        assert s1.reduce("l2sq", k) == pytest.approx(float(np.sum(a * a)), rel=1e-12)


def test_system_validation(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import System
    with pytest.raises(N.GbstError) as e:
        System((16, 16, 16), 4, 0.5 * np.eye(3))  # |1 + lambda a| > 1
    assert e.value.status == N.GBST_EUNSTABLE
    with pytest.raises(N.GbstError) as e:
        System((16, 16, 16), 4, 0.01 * np.eye(5))
    assert e.value.status == N.GBST_EINVAL
    s = System((16, 16, 16), 4, 0.5 * np.eye(3), allow_unstable=True)
    assert json.loads(s.describe())["nf"] == 3
