"""Accuracy over the configured run lengths, against the FP64 oracle (GPU).

The acoustic-wave configuration (order 8, five layers, Ricker 10 Hz, 500 steps)
runs whole on a 192^3 grid, where the oracle finishes in seconds, in FP32 and in
BF16 storage; the 1024^3 heat configuration runs its 50 steps per order and is
compared on output boxes whose exact values the oracle computes from their
dependency cones (oracle/cones.py).  Tolerances are the stated ones: max
relative error 1e-5 for FP32 storage and 2e-2 for BF16 storage.
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle.cones import heat_on_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def wave192_oracle():
    case = synthetic.wave3d(192)
    c = case.velocity()
    kap = oracle.kappa_from_velocity(c, case.dt, case.h)
    z = np.zeros(c.shape)
    _, ref = oracle.wave_run(z, z, kap, case.so, case.nsteps, src=case.src, f0=case.f0, t0=case.t0,
                             amp=case.amp, dt=case.dt, h=case.h)
    return case, c, kap, ref


BF16_DIVERGES = ("BF16 storage of the leapfrog state (round to nearest even on every store, FP32 "
                 "arithmetic) does not stay within 2e-2 over 500 steps: every rounding of u^{n+1} "
                 "perturbs the three-level recurrence, and its low-wavenumber part grows with each later "
                 "step.  A plain CPU emulation of the same scheme gives max rel 0.024 after 100 steps, "
                 "0.27 after 300 and 4.7 after 500 on 96^3; the GPU run measures 11.9 here")


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5),
                                         pytest.param("bf16", 2e-2, marks=pytest.mark.xfail(
                                             strict=True, reason=BF16_DIVERGES))])
def test_wave3d_so8_500_steps_whole_grid(torch_cuda, wave192_oracle, storage, tol):
    from paper_2404_02218_gb300.grid import Grid
    case, c, kap, ref = wave192_oracle
    g = Grid(3, case.dims, case.so, "wave", h=case.h, dt=case.dt, storage=storage)
    g.set_field("vel", c)
    g.set_source(case.src, case.f0, case.t0, case.amp)
    g.tune(reps=1)
    g.set_field("u", np.zeros(c.shape, np.float32))
    g.set_field("u_prev", np.zeros(c.shape, np.float32))
    g.step = 0
    g.run(case.nsteps)
    got = g.get_field("u")
    e0 = g.reduce("energy")
    g.close()
    err = oracle.max_rel_error(got, ref)
    l2 = oracle.rel_l2_error(got, ref)
    print(f"wave 192^3 order 8, {case.nsteps} steps, {storage}: max rel {err:.3e}, rel L2 {l2:.3e}, energy {e0:.6e}")
    assert np.all(np.isfinite(got))
    assert err <= tol
    assert l2 <= tol


def _boxes(n, edge=16):
    m = n // 2 - edge // 2
    return [((m, m, m), (m + edge, m + edge, m + edge)),          # interior
            ((0, 0, 0), (edge // 2, edge // 2, edge)),             # corner (x seam of 16-wide tiles)
            ((n - 4, m, 120), (n, m + 8, 136))]                    # far face, across a 128-wide tile seam


@pytest.mark.parametrize("so", [2, 4, 8])
def test_heat3d_1024_50_steps_cone_boxes(torch_cuda, so):
    torch = torch_cuda
    from paper_2404_02218_gb300.grid import Grid
    case = synthetic.heat3d(1024, so)
    dims = case.dims
    shape = tuple(reversed(dims))
    u0 = synthetic.uniform_field_torch(case.seed, shape, "cuda")
    g = Grid(3, dims, so, "heat", h=1.0, dt=case.a, alpha=1.0)
    g.set_field("u", u0)
    g.tune(reps=1)  # the benchmark's plan
    g.set_field("u", u0)
    g.run(case.nsteps)
    out = torch.empty_like(u0)
    g.get_field("u", out=out)
    g.close()
    del u0
    worst = 0.0
    for lo, hi in _boxes(1024):
        ref = heat_on_box(lambda l, h: synthetic.uniform_box(case.seed, shape, l, h), shape, lo, hi, so, case.a,
                          case.nsteps)
        got = out[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]].cpu().numpy().astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - ref))))
    # max |u| <= 1 under a stable heat step from U[0,1): the absolute bound is a relative one
    print(f"heat 1024^3 order {so}, {case.nsteps} steps: max abs error on the boxes {worst:.3e}")
    assert worst <= 1e-5


@pytest.fixture(scope="module")
def batch64_errors(torch_cuda):
    """The 64-grid batch over its configured 300 steps in one persistent launch: max relative
    error of the three smallest members (96-127 points per axis), whole, against the oracle."""
    from paper_2404_02218_gb300.grid import Batch
    cases = synthetic.batch_wave_cases()
    b = Batch(3, [dict(dims=c.dims, h=c.h, dt=c.dt) for c in cases], 4, "wave")
    for i, c in enumerate(cases):
        b.set_field(i, "vel", c.velocity())
        b.set_source(i, c.src, c.f0, c.t0, c.amp)
    b.set_persistent(True)
    b.run(cases[0].nsteps)
    order = np.argsort([int(np.prod(c.dims)) for c in cases])
    errs = {}
    for i in order[:3]:
        c = cases[int(i)]
        kap = oracle.kappa_from_velocity(c.velocity(), c.dt, c.h)
        z = np.zeros(kap.shape)
        _, ref = oracle.wave_run(z, z, kap, 4, c.nsteps, src=c.src, f0=c.f0, t0=c.t0, amp=c.amp, dt=c.dt, h=c.h)
        got = b.get_field(int(i), "u")
        assert np.all(np.isfinite(got))
        errs[int(i)] = oracle.max_rel_error(got, ref)
        print(f"batch member {int(i)} {c.dims}, {c.nsteps} steps: max rel {errs[int(i)]:.3e}")
    b.close()
    return cases[0].nsteps, errs


def test_batch64_300_steps_within_fp32_rounding_bound(batch64_errors):
    """Bound from the arithmetic: each leapfrog step rounds u^{n+1} a few times (the sum of
    the star, 2u - u^{n-1}, the fused multiply-add), at most 4 roundings of 2^-24 relative
    to max |u|, and the scheme carries every rounding error forward undamped, so the error
    after n steps stays below n * 4 * 2^-24 of the field's maximum."""
    nsteps, errs = batch64_errors
    bound = nsteps * 4 * 2.0 ** -24
    assert max(errs.values()) <= bound, (errs, bound)


def test_batch64_300_steps_within_1e5(batch64_errors):
    """The stated FP32 tolerance over the configured 300 steps.  It holds because the sweep
    takes the star's weights as integers over a common denominator (exact in FP32, so the
    star of a constant is exactly zero): with the weights rounded to FP32 the zeroth moment
    of the star was off by about 1e-8, a spurious term the leapfrog carries coherently,
    and one member measured 1.07e-5."""
    _, errs = batch64_errors
    assert max(errs.values()) <= 1e-5, errs
