"""GPU: halo exchange overlapped with the sweep (decomposition mode and the
periodic wrap).

With the overlap on, each step copies the exchanged faces on a second stream
while the work units whose TMA boxes read no exchanged ghost cell sweep; the
remaining units sweep after the copies.  The result must be the same bits as
the plain order (copies, then one sweep) and as the undecomposed grid, for
heat and wave, 2D and 3D, every order, every compiled 3D heat variant, with
and without captured graphs; the plan reports the split.
"""
import json

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def heat(dims, so, overlap, **kw):
    from paper_2404_02218_gb300.grid import Grid
    a = float(np.float32(0.8 * synthetic.heat_a_max(len(dims), so)))
    g = Grid(len(dims), dims, so, "heat", dt=a, **kw)
    g.set_overlap(overlap)
    return g


def run_heat(dims, so, nsteps, overlap, seed=71, splits=(), zchunks=0, **kw):
    u0 = synthetic.uniform_field(seed, tuple(reversed(dims)))
    g = heat(dims, so, overlap, **kw)
    if zchunks:  # z-chunks whose planes stay clear of an exchanged z face
        g.set_plan(-1, 0, zchunks, 0)
    g.set_field("u", u0)
    for n in splits:
        g.run(n)
    g.run(nsteps)
    plan = json.loads(g.describe())
    out = g.get_field("u", np.float32)
    g.close()
    return out, plan


@pytest.mark.parametrize("so", [2, 4, 8])
@pytest.mark.parametrize("decomp", [(2, 2, 2), (2, 1, 3), (1, 2, 1)])
def test_decomposed_overlap_bitwise(torch_cuda, so, decomp):
    # subdomains of at least 150 points in x: each has a 128-wide tile clear of its exchanged x face
    dims = (300, 70, 66)
    want, _ = run_heat(dims, so, 8, 0)
    off, p_off = run_heat(dims, so, 5, 0, decomp=decomp, zchunks=3, splits=(2, 1))
    on, p_on = run_heat(dims, so, 5, 1, decomp=decomp, zchunks=3, splits=(2, 1))
    assert p_off["overlap"] == 0 and p_on["overlap"] == 1
    assert 0 < p_on["interior_units"] < p_on["units"]
    np.testing.assert_array_equal(off, want)
    np.testing.assert_array_equal(on, want)


def test_overlap_without_graphs_and_2d(torch_cuda):
    dims3 = (300, 66, 30)
    a, pa = run_heat(dims3, 4, 7, 1, decomp=(2, 2, 1), use_graph=False)
    b, _ = run_heat(dims3, 4, 7, 0, decomp=(2, 2, 1), use_graph=False)
    assert pa["overlap"] == 1
    np.testing.assert_array_equal(a, b)
    dims2 = (300, 140)
    c, pc = run_heat(dims2, 8, 6, 1, decomp=(2, 2))
    d, _ = run_heat(dims2, 8, 6, 0)
    assert pc["overlap"] == 1
    np.testing.assert_array_equal(c, d)


def test_every_heat_variant_decomposed_with_overlap(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    dims = (300, 40, 24)
    want, _ = run_heat(dims, 4, 4, 0)
    u0 = synthetic.uniform_field(71, tuple(reversed(dims)))
    g = heat(dims, 4, 1, decomp=(2, 1, 2))
    variants = [i for i in range(N.stencil_variant_count())
                if (lambda v: (v["R"], v["eq"], v["storage"], v["has_z"], v["tb"], v["nf"]) == (2, 0, 0, 1, 1, 1))(
                    json.loads(N.stencil_variant_info(i)))]
    assert variants
    for v in variants:
        for zc in (2, 3):
            g.set_plan(v, 0, zc, 0)
            g.set_field("u", u0)
            g.run(4)
            assert json.loads(g.describe())["overlap"] == 1
            np.testing.assert_array_equal(g.get_field("u", np.float32), want, err_msg=f"variant {v} zc {zc}")
    g.close()


def test_periodic_overlap_matches_oracle(torch_cuda):
    dims = (300, 40, 36)
    so = 4
    a = float(np.float32(0.8 * synthetic.heat_a_max(3, so)))
    u0 = synthetic.uniform_field(72, tuple(reversed(dims)))
    on, p_on = run_heat(dims, so, 6, 1, seed=72, bc="periodic", zchunks=4)
    off, _ = run_heat(dims, so, 6, 0, seed=72, bc="periodic", zchunks=4)
    assert p_on["overlap"] == 1
    np.testing.assert_array_equal(on, off)
    ref = oracle.heat_run(u0, so, a, 6, bc=oracle.BC_PERIODIC)
    assert oracle.max_rel_error(on, ref) <= 1e-5


def test_wave_decomposed_overlap_bitwise(torch_cuda):
    from paper_2404_02218_gb300.grid import Grid
    dims = (300, 50, 44)
    h = 10.0
    speeds = synthetic.five_layer_speeds()
    c = synthetic.layered_velocity(tuple(reversed(dims)), speeds)
    dt = 0.5 * synthetic.wave_courant_max(3, 8) * h / max(speeds)
    out = []
    for decomp, overlap in (((1, 1, 1), 0), ((2, 1, 2), 0), ((2, 1, 2), 1)):
        g = Grid(3, dims, 8, "wave", h=h, dt=dt, decomp=decomp)
        g.set_overlap(overlap)
        g.set_plan(-1, 0, 2, 0)
        if decomp != (1, 1, 1):
            assert json.loads(g.describe())["overlap"] == overlap
        g.set_field("vel", c)
        g.set_source((60, 20, 30), 10.0, 0.1, 1.0)
        g.run(12)
        out.append((g.get_field("u", np.float32), g.get_field("u_prev", np.float32)))
        g.close()
    for u, p in out[1:]:
        np.testing.assert_array_equal(u, out[0][0])
        np.testing.assert_array_equal(p, out[0][1])


def test_overlap_validation(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    g = heat((300, 32, 16), 2, -1, decomp=(2, 1, 1))
    assert json.loads(g.describe())["overlap"] == 0  # the default: off on one device
    g.set_overlap(1)
    assert json.loads(g.describe())["overlap"] == 1
    for bad in (2, -2):
        with pytest.raises(N.GbstError) as e:
            g.set_overlap(bad)
        assert e.value.status == N.GBST_EINVAL
    g.close()
    u = heat((64, 32, 16), 2, 1)  # nothing to exchange: no split
    assert json.loads(u.describe())["overlap"] == 0
    # the autotuner keeps a plan that can split when the overlap is on
    t = heat((300, 64, 48), 4, 1, decomp=(2, 1, 2))
    t.set_field("u", synthetic.uniform_field(73, (48, 64, 300)))
    rep = t.tune(reps=1)
    assert rep["candidates"] and json.loads(t.describe())["overlap"] == 1
    t.close()
