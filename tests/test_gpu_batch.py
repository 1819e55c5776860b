"""GPU: batched grids and persistent launches.

* every member of a batch matches its own FP64 oracle run (FP32 tolerance);
* a batch gives the same bits as the same grids run as separate handles;
* a persistent launch (one cooperative kernel with grid-wide barriers between
  steps) gives the same bits as one launch per step;
* a grid barrier that can never complete (a test hook adds arrivals nobody
  makes) expires after its bounded wait and is reported as GBST_ETIMEOUT; the
  GPU context stays usable.
"""
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


def small_cases(count=5, so=4):
    """Like the batched configuration, at sizes the oracle runs in seconds."""
    cases = synthetic.batch_wave_cases(count=count, seed=14, lo=20, hi=44, so=so, nsteps=60)
    return cases


def make_batch(cases, so, **kw):
    from paper_2404_02218_gb300.grid import Batch
    members = [dict(dims=c.dims, h=c.h, dt=c.dt) for c in cases]
    b = Batch(3, members, so, "wave", **kw)
    for i, c in enumerate(cases):
        b.set_field(i, "vel", c.velocity())
        b.set_source(i, c.src, c.f0, c.t0, c.amp)
    return b


def test_batch_members_match_oracle(torch_cuda):
    so = 4
    cases = small_cases(so=so)
    b = make_batch(cases, so)
    b.run(60)
    for i, c in enumerate(cases):
        kap = oracle.kappa_from_velocity(c.velocity(), c.dt, c.h)
        z = np.zeros(kap.shape)
        _, C = oracle.wave_run(z, z, kap, so, 60, src=c.src, f0=c.f0, t0=c.t0, amp=c.amp, dt=c.dt, h=c.h)
        got = b.get_field(i, "u")
        assert np.max(np.abs(C)) > 0
        assert oracle.max_rel_error(got, C) <= TOL_F32, i


def test_batch_equals_separate_grids_bitwise(torch_cuda):
    from paper_2404_02218_gb300.grid import Grid
    so = 8
    cases = small_cases(so=so)
    b = make_batch(cases, so)
    b.run(37)
    for i, c in enumerate(cases):
        g = Grid(3, c.dims, so, "wave", h=c.h, dt=c.dt)
        g.set_field("vel", c.velocity())
        g.set_source(c.src, c.f0, c.t0, c.amp)
        g.run(37)
        np.testing.assert_array_equal(b.get_field(i, "u"), g.get_field("u"))
        g.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_persistent_equals_per_step_bitwise(torch_cuda, use_graph):
    so = 4
    cases = small_cases(so=so)
    a = make_batch(cases, so, use_graph=use_graph)
    a.run(23)
    a.run(18)
    p = make_batch(cases, so, use_graph=use_graph)
    p.set_persistent(True)
    p.run(23)
    p.run(18)
    for i in range(len(cases)):
        np.testing.assert_array_equal(p.get_field(i, "u"), a.get_field(i, "u"))
        np.testing.assert_array_equal(p.get_field(i, "u_prev"), a.get_field(i, "u_prev"))


def test_persistent_heat_single_grid(torch_cuda):
    from paper_2404_02218_gb300.grid import Grid
    dims = (90, 70, 50)
    so = 8
    a = float(np.float32(0.8 * synthetic.heat_a_max(3, so)))
    u0 = synthetic.uniform_field(3, tuple(reversed(dims)))
    g1 = Grid(3, dims, so, "heat", dt=a)
    g1.set_field("u", u0)
    g1.run(15)
    g2 = Grid(3, dims, so, "heat", dt=a)
    g2.set_persistent(True)
    g2.set_field("u", u0)
    g2.run(15)
    np.testing.assert_array_equal(g2.get_field("u"), g1.get_field("u"))
    ref = oracle.heat_run(u0, so, a, 15)
    assert oracle.max_rel_error(g2.get_field("u"), ref) <= TOL_F32


def test_batch_reductions(torch_cuda):
    so = 4
    cases = small_cases(so=so)
    b = make_batch(cases, so)
    b.run(30)
    total = 0.0
    for i in range(len(cases)):
        u = b.get_field(i, "u")
        s = b.reduce("l2sq", i)
        assert s == pytest.approx(float(np.sum(u * u)), rel=1e-12)
        total += s
    assert b.reduce("l2sq") == pytest.approx(total, rel=1e-12)


def test_batch_autotune(torch_cuda):
    cases = small_cases(so=4)
    b = make_batch(cases, 4)
    b.run(5)
    u = b.get_field(2, "u")
    rep = b.tune(reps=2)
    assert rep["candidates"]
    np.testing.assert_array_equal(b.get_field(2, "u"), u)


def test_grid_barrier_timeout_is_reported(torch_cuda):
    """A barrier that can never complete expires (bounded wait) -> GBST_ETIMEOUT."""
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid
    dims = (64, 48, 40)
    so = 4
    a = float(np.float32(0.5 * synthetic.heat_a_max(3, so)))
    g = Grid(3, dims, so, "heat", dt=a)
    g.set_persistent(True)
    N.stencil_debug_barrier_extra(g.h, 1)
    g.run(3)
    with pytest.raises(N.GbstError) as e:
        g.sync()
    assert e.value.status == N.GBST_ETIMEOUT
    with pytest.raises(N.GbstError):  # the handle stays poisoned
        g.run(1)
    g.close()
    # the context is still usable
    g2 = Grid(3, dims, so, "heat", dt=a)
    u0 = synthetic.uniform_field(4, tuple(reversed(dims)))
    g2.set_field("u", u0)
    g2.run(2)
    assert oracle.max_rel_error(g2.get_field("u"), oracle.heat_run(u0, so, a, 2)) <= TOL_F32
