"""GPU: temporally blocked heat sweeps (two forward-Euler steps per pass).

A blocked run must give the same bits as the same number of single steps: the
step-1 field is recomputed on overlapped tiles with the single-step kernel's
per-point arithmetic, and its points outside the domain are zero like the ghost
cells of a stored field.  Checked for every compiled blocked variant, several
z-chunkings, odd step counts (the last step runs alone), ragged and tiny grids,
against the FP64 oracle, and on single-device decompositions, where the ghost
regions are 2r deep and a three-phase exchange (faces and the edges two steps
reach) precedes every two-step launch.
"""
import json

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def tb_variants(so):
    from paper_2404_02218_gb300 import native as N
    out = []
    for i in range(N.stencil_variant_count()):
        v = json.loads(N.stencil_variant_info(i))
        if v["tb"] == 2 and v["R"] == so // 2:
            out.append(i)
    return out


def heat(dims, so, temporal_block, **kw):
    from paper_2404_02218_gb300.grid import Grid
    a = float(np.float32(0.8 * synthetic.heat_a_max(3, so)))
    return Grid(3, dims, so, "heat", dt=a, temporal_block=temporal_block, **kw), a


def single_steps(dims, so, u0, nsteps):
    g, _ = heat(dims, so, 1)
    g.set_field("u", u0)
    g.run(nsteps)
    out = g.get_field("u")
    g.close()
    return out


@pytest.mark.parametrize("so", [2, 4])
def test_blocked_variants_exist(so):
    assert tb_variants(so)


@pytest.mark.parametrize("so", [2, 4])
@pytest.mark.parametrize("dims", [(130, 70, 19), (257, 33, 40), (128, 16, 9), (5, 3, 2), (1, 1, 1)])
def test_blocked_equals_single_steps_bitwise(torch_cuda, so, dims):
    u0 = synthetic.uniform_field(21, tuple(reversed(dims)))
    want = {n: single_steps(dims, so, u0, n) for n in (1, 2, 5)}
    g, _ = heat(dims, so, 2)
    for v in tb_variants(so):
        for zc, sched in ((0, 1), (1, 1), (3, 1), (3, 0)):
            g.set_schedule(sched)
            for n in (1, 2, 5):
                g.set_field("u", u0)
                g.set_plan(v, 0, zc, 0)
                assert json.loads(g.describe())["tb"] == 2
                g.run(n)
                np.testing.assert_array_equal(g.get_field("u"), want[n],
                                              err_msg=f"variant {v} zchunks {zc} schedule {sched} n {n}")
    g.close()


@pytest.mark.parametrize("so", [2, 4])
def test_blocked_matches_oracle(torch_cuda, so):
    dims = (150, 90, 40)
    u0 = synthetic.uniform_field(22, tuple(reversed(dims)))
    g, a = heat(dims, so, 2)
    assert json.loads(g.describe())["tb"] == 2
    g.set_field("u", u0)
    g.run(9)
    ref = oracle.heat_run(u0, so, a, 9)
    assert oracle.max_rel_error(g.get_field("u"), ref) <= TOL_F32


def test_blocked_split_runs_and_graphs(torch_cuda):
    """run(3) + run(4) with graphs == run(7) without graphs == 7 single steps."""
    dims = (140, 60, 30)
    so = 2
    u0 = synthetic.uniform_field(23, tuple(reversed(dims)))
    want = single_steps(dims, so, u0, 7)
    g, _ = heat(dims, so, 2)
    g.set_field("u", u0)
    g.run(3)
    g.run(4)
    assert g.step == 7
    np.testing.assert_array_equal(g.get_field("u"), want)
    h, _ = heat(dims, so, 2, use_graph=False)
    h.set_field("u", u0)
    h.run(7)
    np.testing.assert_array_equal(h.get_field("u"), want)


def test_blocking_off_and_unsupported_cases_use_single_steps(torch_cuda):
    dims = (64, 40, 24)
    g, _ = heat(dims, 2, 1)
    assert json.loads(g.describe())["tb"] == 1
    rep = g.tune(reps=1)
    assert all(c["tb"] == 1 for c in rep["candidates"])
    # order 8 has no blocked variants (two 9-plane queues do not fit the register file)
    d, _ = heat(dims, 8, 2, decomp=(2, 1, 1))
    assert json.loads(d.describe())["tb"] == 1
    # subdomains thinner than 2r along a split axis: single steps (on the deep-ghost layout),
    # still the undecomposed bits
    thin = (10, 12, 9)
    t, _ = heat(thin, 4, 2, decomp=(4, 1, 1))
    assert json.loads(t.describe())["tb"] == 1
    u0 = synthetic.uniform_field(28, tuple(reversed(thin)))
    t.set_field("u", u0)
    t.run(3)
    np.testing.assert_array_equal(t.get_field("u"), single_steps(thin, 4, u0, 3))
    # BF16 storage: not blocked
    b, _ = heat(dims, 2, 2, storage="bf16")
    assert json.loads(b.describe())["tb"] == 1


def test_autotuner_considers_blocking(torch_cuda):
    dims = (256, 128, 64)
    g, _ = heat(dims, 4, 0)
    u0 = synthetic.uniform_field(24, tuple(reversed(dims)))
    g.set_field("u", u0)
    rep = g.tune(reps=2)
    assert {c["tb"] for c in rep["candidates"]} == {1, 2}
    np.testing.assert_array_equal(g.get_field("u"), u0)
    want = single_steps(dims, 4, u0, 6)
    g.run(6)
    np.testing.assert_array_equal(g.get_field("u"), want)


@pytest.mark.parametrize("so", [2, 4])
@pytest.mark.parametrize("decomp,dims", [((2, 2, 2), (68, 50, 44)), ((3, 2, 1), (130, 37, 29)),
                                         ((1, 1, 4), (40, 33, 50)), ((2, 1, 1), (1040, 20, 12))])
def test_blocked_decomposed_equals_single_steps_bitwise(torch_cuda, so, decomp, dims):
    """Two steps per launch across subdomain exchanges give the undecomposed single steps'
    bits (ragged splits; (2, 1, 1) of 1040 points: wide rows, 128-byte x ghosts)."""
    u0 = synthetic.uniform_field(25, tuple(reversed(dims)))
    want = {n: single_steps(dims, so, u0, n) for n in (1, 2, 5)}
    g, _ = heat(dims, so, 2, decomp=decomp)
    assert json.loads(g.describe())["tb"] == 2
    for n in (1, 2, 5):
        g.set_field("u", u0)
        g.run(n)
        np.testing.assert_array_equal(g.get_field("u"), want[n], err_msg=f"n {n}")
    g.close()


@pytest.mark.parametrize("so", [2, 4])
def test_blocked_decomposed_every_variant_bitwise(torch_cuda, so):
    dims = (70, 45, 36)
    u0 = synthetic.uniform_field(26, tuple(reversed(dims)))
    want = single_steps(dims, so, u0, 5)
    g, _ = heat(dims, so, 2, decomp=(2, 2, 2))
    for v in tb_variants(so):
        for zc, sched in ((0, 1), (3, 0)):
            g.set_schedule(sched)
            g.set_field("u", u0)
            g.set_plan(v, 0, zc, 0)
            assert json.loads(g.describe())["tb"] == 2
            g.run(5)
            np.testing.assert_array_equal(g.get_field("u"), want, err_msg=f"variant {v} zchunks {zc} schedule {sched}")
    g.close()


def test_decomposed_single_step_plans_on_deep_ghosts(torch_cuda):
    """A decomposed grid keeps 2r-deep ghosts for blocking; its single-step plans (r-deep
    face exchange) give the same bits too, and the tuner considers both."""
    dims = (96, 40, 30)
    so = 2
    u0 = synthetic.uniform_field(27, tuple(reversed(dims)))
    want = single_steps(dims, so, u0, 4)
    g, _ = heat(dims, so, 0, decomp=(2, 2, 1))
    g.set_field("u", u0)
    rep = g.tune(reps=1)
    assert {c["tb"] for c in rep["candidates"]} == {1, 2}
    for tb in (1, 2):
        v = next(c["variant"] for c in rep["candidates"] if c["tb"] == tb)
        g.set_field("u", u0)
        g.set_plan(v, 0, 0, 0)
        g.run(4)
        np.testing.assert_array_equal(g.get_field("u"), want, err_msg=f"tb {tb}")
    g.close()
