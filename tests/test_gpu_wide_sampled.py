"""Parity at the measured sizes, in the benchmark's launch configuration, on
sampled outputs the oracle computes one by one.

After k steps a point depends only on the input within k*r cells of it (the
star stencil's dependency cone), so the oracle advances the sub-box
[p - k r, p + k r] (clipped at the true boundary, where the zero halo is the
real one) and its centre value is exact.  Samples cover corners, edges, faces,
tile seams and seeded interior points.
"""
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


def sample_points(dims, seed, n_random=24):
    nx, ny, nz = dims
    pts = set()
    for x in (0, 1, nx // 2, nx - 2, nx - 1):
        for y in (0, ny - 1, 63, 64):
            for z in (0, nz - 1, nz // 3):
                pts.add((x, y, z))
    for x in (31, 32, 63, 64, 127, 128):  # tile seams of the common tile widths
        pts.add((x, ny // 2, nz // 2))
    u = synthetic.uniform_ints(seed, 0, min(dims) - 1, 3 * n_random).reshape(n_random, 3)
    for p in u:
        pts.add((int(p[0]) % nx, int(p[1]) % ny, int(p[2]) % nz))
    return sorted(pts)


def sub_box(dims, p, reach):
    lo = [max(0, p[a] - reach) for a in range(3)]
    hi = [min(dims[a], p[a] + reach + 1) for a in range(3)]
    return lo, hi


@pytest.mark.parametrize("so,tb", [(2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (2, 0), (4, 0), (8, 0)])
def test_heat3d_1024_sampled(torch_cuda, so, tb):
    """tb = 1: single steps (default plan); tb = 2: the temporally blocked kernel
    (3 steps = one two-step launch and one single-step launch); tb = 0: the plan the
    autotuner picks, as in the benchmark."""
    torch = torch_cuda
    import json
    from paper_2404_02218_gb300.grid import Grid
    case = synthetic.heat3d(1024, so)
    k = 3
    dims = case.dims
    u0 = synthetic.uniform_field_torch(case.seed, tuple(reversed(dims)), "cuda")
    g = Grid(3, dims, so, "heat", h=1.0, dt=case.a, alpha=1.0, temporal_block=tb)
    if tb:
        assert json.loads(g.describe())["tb"] == tb
    else:
        g.set_field("u", u0)
        g.tune(reps=1)
    g.set_field("u", u0)
    g.run(k)
    out = torch.empty_like(u0)
    g.get_field("u", out=out)
    g.close()
    reach = k * (so // 2)
    worst = 0.0
    for p in sample_points(dims, so):
        lo, hi = sub_box(dims, p, reach)
        sub = u0[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].cpu().numpy().astype(np.float64)
        ref = oracle.heat_run(sub, so, case.a, k)[p[2] - lo[2], p[1] - lo[1], p[0] - lo[0]]
        got = float(out[p[2], p[1], p[0]].item())
        worst = max(worst, abs(got - ref))
    # max |u| <= 1 for the U[0,1) initial field under a stable heat step
    assert worst <= 1e-5


def test_wave3d_768_so8_sampled(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300.grid import Grid
    case = synthetic.wave3d()
    so, k = case.so, 4
    dims = case.dims
    shape = tuple(reversed(dims))
    g = Grid(3, dims, so, "wave", h=case.h, dt=case.dt)
    c = synthetic.layered_velocity(shape, case.speeds)
    g.set_field("vel", c)
    g.tune(reps=1)  # the benchmark's plan
    u0 = synthetic.uniform_field_torch(31, shape, "cuda") - 0.5
    up = synthetic.uniform_field_torch(32, shape, "cuda") - 0.5
    g.set_field("u", u0)
    g.set_field("u_prev", up)
    g.set_source(case.src, case.f0, case.t0, 1000.0)
    g.run(k)
    out = torch.empty_like(u0)
    g.get_field("u", out=out)
    g.close()
    kap = oracle.kappa_from_velocity(c, case.dt, case.h)
    reach = k * (so // 2)
    pts = sample_points(dims, 7) + [tuple(case.src)]
    worst = 0.0
    for p in pts:
        lo, hi = sub_box(dims, p, reach)
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        su = u0[sl].cpu().numpy().astype(np.float64)
        sp = up[sl].cpu().numpy().astype(np.float64)
        sk = np.ascontiguousarray(kap[sl])
        src = case.src
        inside = all(lo[a] <= src[a] < hi[a] for a in range(3))
        P, C = oracle.wave_run(sp, su, sk, so, k, src=tuple(src[a] - lo[a] for a in range(3)) if inside else None,
                               f0=case.f0, t0=case.t0, amp=1000.0, dt=case.dt, h=case.h)
        ref = C[p[2] - lo[2], p[1] - lo[1], p[0] - lo[0]]
        got = float(out[p[2], p[1], p[0]].item())
        worst = max(worst, abs(got - ref))
    # |u| stays O(1) over four steps; the bound is relative to max |u0| = 0.5
    assert worst <= 1e-5 * 0.5 * 4


def sample_points_2d(dims, seed, n_random=24):
    nx, ny = dims
    pts = set()
    for x in (0, 1, nx // 2, nx - 2, nx - 1, 31, 32, 127, 128):
        for y in (0, 1, ny // 2, ny - 1, 63, 64):
            pts.add((x, y))
    u = synthetic.uniform_ints(seed, 0, min(dims) - 1, 2 * n_random).reshape(n_random, 2)
    for p in u:
        pts.add((int(p[0]) % nx, int(p[1]) % ny))
    return sorted(pts)


@pytest.mark.parametrize("so", [2, 4, 8])
def test_heat2d_16384_sampled(torch_cuda, so):
    """The paper's large 2D size (Section 6.1), U[0,1) input, a = 0.8 of the limit."""
    torch = torch_cuda
    from paper_2404_02218_gb300.grid import Grid
    n, k = 16384, 4
    a = float(np.float32(0.8 * synthetic.heat_a_max(2, so)))
    u0 = synthetic.uniform_field_torch(7, (n, n), "cuda")
    g = Grid(2, (n, n), so, "heat", h=1.0, dt=a, alpha=1.0)
    g.set_field("u", u0)
    g.tune(reps=1)  # the benchmark's plan
    g.set_field("u", u0)
    g.run(k)
    out = torch.empty_like(u0)
    g.get_field("u", out=out)
    g.close()
    reach = k * (so // 2)
    worst = 0.0
    for p in sample_points_2d((n, n), so):
        lo = [max(0, p[i] - reach) for i in range(2)]
        hi = [min(n, p[i] + reach + 1) for i in range(2)]
        sub = u0[lo[1]:hi[1], lo[0]:hi[0]].cpu().numpy().astype(np.float64)
        ref = oracle.heat_run(sub, so, a, k)[p[1] - lo[1], p[0] - lo[0]]
        worst = max(worst, abs(float(out[p[1], p[0]].item()) - ref))
    assert worst <= 1e-5


def test_wave3d_768_so8_bf16_sampled(torch_cuda):
    """The 768^3 order-8 wave in BF16 storage, as the benchmark runs it (2e-2 of max |u|:
    BF16 rounding of the inputs and of every stored step)."""
    torch = torch_cuda
    from paper_2404_02218_gb300.grid import Grid
    case = synthetic.wave3d()
    so, k = case.so, 4
    dims = case.dims
    shape = tuple(reversed(dims))
    g = Grid(3, dims, so, "wave", h=case.h, dt=case.dt, storage="bf16")
    c = synthetic.layered_velocity(shape, case.speeds)
    g.set_field("vel", c)
    g.tune(reps=1)  # the benchmark's plan
    u0 = synthetic.uniform_field_torch(33, shape, "cuda") - 0.5
    up = synthetic.uniform_field_torch(34, shape, "cuda") - 0.5
    g.set_field("u", u0)
    g.set_field("u_prev", up)
    g.run(k)
    out = torch.empty_like(u0)
    g.get_field("u", out=out)
    g.close()
    kap = oracle.kappa_from_velocity(c, case.dt, case.h)
    reach = k * (so // 2)
    worst = 0.0
    for p in sample_points(dims, 9):
        lo, hi = sub_box(dims, p, reach)
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        P, C = oracle.wave_run(up[sl].cpu().numpy().astype(np.float64), u0[sl].cpu().numpy().astype(np.float64),
                               np.ascontiguousarray(kap[sl]), so, k)
        ref = C[p[2] - lo[2], p[1] - lo[1], p[0] - lo[0]]
        worst = max(worst, abs(float(out[p[2], p[1], p[0]].item()) - ref))
    assert worst <= 2e-2 * 0.5 * 4


def test_batch64_full_configuration(torch_cuda):
    """The 64-grid batch as benchmarked (sizes U[96, 256], order 4, one persistent
    launch): the three smallest members and the largest, after 20 steps, in full
    against the oracle."""
    from paper_2404_02218_gb300.grid import Batch
    cases = synthetic.batch_wave_cases()
    k = 20
    b = Batch(3, [dict(dims=c.dims, h=c.h, dt=c.dt) for c in cases], 4, "wave")
    for i, c in enumerate(cases):
        b.set_field(i, "vel", c.velocity())
        b.set_source(i, c.src, c.f0, c.t0, c.amp)
    b.set_persistent(True)
    b.run(k)
    vol = [int(np.prod(c.dims)) for c in cases]
    order = np.argsort(vol)
    for i in order[:3]:
        c = cases[i]
        kap = oracle.kappa_from_velocity(c.velocity(), c.dt, c.h)
        z = np.zeros(kap.shape)
        _, C = oracle.wave_run(z, z, kap, 4, k, src=c.src, f0=c.f0, t0=c.t0, amp=c.amp, dt=c.dt, h=c.h)
        got = b.get_field(int(i), "u")
        assert np.max(np.abs(C)) > 0
        assert oracle.max_rel_error(got, C) <= 1e-5, int(i)
    i = int(order[-1])
    c = cases[i]
    got = b.get_field(i, "u")
    kap = oracle.kappa_from_velocity(c.velocity(), c.dt, c.h)
    z = np.zeros(kap.shape)
    _, C = oracle.wave_run(z, z, kap, 4, k, src=c.src, f0=c.f0, t0=c.t0, amp=c.amp, dt=c.dt, h=c.h)
    assert oracle.max_rel_error(got, C) <= 1e-5
