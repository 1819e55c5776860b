"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test ties the oracle to something other than itself: exact rational
weights from the moment conditions, discrete Fourier eigenvalues, invariants,
a dense-matrix brute force built independently, and the worked dmp.swap
example printed in the paper (Section 4.2).  A plausible slip in the oracle --
a dropped axis, a wrong sign, a swapped time level, a mis-placed source, an
off-by-one ghost -- fails at least one of these.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic
from oracle import brute
from oracle.weights import central_weights, symbol, symbol_max

SOS = (2, 4, 8)


# ---------------------------------------------------------------- weights ---

def test_weights_textbook_values():
    # Central second-derivative weights (Fornberg, Math. Comp. 51, 1988, Table 1).
    assert central_weights(2) == [Fraction(-2), Fraction(1)]
    assert central_weights(4) == [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)]
    assert central_weights(8) == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                                  Fraction(8, 315), Fraction(-1, 560)]


@pytest.mark.parametrize("so", SOS)
def test_weights_differentiate_polynomials_exactly(so):
    w = central_weights(so)
    r = so // 2
    for x0 in (Fraction(0), Fraction(3), Fraction(-7, 2)):
        for k in range(0, so + 2):
            got = sum(w[abs(m)] * (x0 + m) ** k for m in range(-r, r + 1))
            want = k * (k - 1) * x0 ** (k - 2) if k >= 2 else 0
            assert got == want, (so, k)
        # accuracy is exactly `so`: degree so+2 is no longer differentiated exactly
        k = so + 2
        got = sum(w[abs(m)] * Fraction(m) ** k for m in range(-r, r + 1))
        assert got != 0
    assert sum(w[abs(m)] for m in range(-r, r + 1)) == 0


@pytest.mark.parametrize("so,den,ints", [(2, 1, [-2, 1]), (4, 12, [-30, 16, -1]),
                                         (8, 5040, [-14350, 8064, -1008, 128, -9])])
def test_weights_over_their_common_denominator(so, den, ints):
    """The sweeps apply the central weights as integers over their least common
    denominator (exact in FP32); rounded one by one to FP32 instead, the weights of the
    3D star no longer sum to zero, so the star of a constant is not exactly zero."""
    w = central_weights(so)
    assert math.lcm(*(x.denominator for x in w)) == den
    assert [x * den for x in w] == [Fraction(v) for v in ints]
    r = so // 2
    # the 3D star of the constant 1 as the sweeps evaluate it in FP32: s = ndim * w0, then
    # s = fma(w_m, 6, s) per offset (the FP64 sum below is exact, so it rounds once, as an FMA)
    def star_of_one(wc, wm):
        s = np.float32(wc)
        for m in range(1, r + 1):
            s = np.float32(np.float64(s) + np.float64(wm[m]) * 6.0)
        return s
    assert star_of_one(np.float32(3 * ints[0]), [np.float32(v) for v in ints]) == 0
    if so > 2:
        assert star_of_one(np.float32(3 * float(w[0])), [np.float32(float(x)) for x in w]) != 0


@pytest.mark.parametrize("so", SOS)
def test_symbol_max_matches_recipe(so):
    S = symbol_max(central_weights(so))
    assert float(S) == pytest.approx(synthetic.SYMBOL_MAX[so], rel=0, abs=1e-15)
    # the maximum of |lambda| is attained at theta = pi
    ws = central_weights(so)
    th = np.linspace(0, math.pi, 2001)
    assert max(abs(symbol(ws, t)) for t in th) <= float(S) + 1e-12


# ------------------------------------------------------------ heat sweeps ---

def _mode(shape_zyx, ks, periodic=True):
    """Separable cosine mode prod_a cos(2 pi k_a i_a / N_a + phase_a)."""
    grids = np.meshgrid(*[np.arange(n) for n in shape_zyx], indexing="ij")
    out = np.ones(shape_zyx)
    thetas = []
    for a, (g, n, k) in enumerate(zip(grids, shape_zyx, ks)):
        th = 2 * math.pi * k / n
        thetas.append(th)
        out = out * np.cos(th * g + 0.3 * (a + 1))
    return out, thetas


@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape,ks", [((16, 12), (3, 2)), ((10, 12, 8), (1, 5, 3))])
def test_heat_periodic_fourier_mode_decay(orc, so, shape, ks):
    w = central_weights(so)
    u0, thetas = _mode(shape, ks)
    a = 0.7 * synthetic.heat_a_max(len(shape), so)
    g = 1.0 + a * sum(symbol(w, t) for t in thetas)
    n = 13
    u = orc.heat_run(u0, so, a, n, bc=orc.BC_PERIODIC)
    np.testing.assert_allclose(u, (g ** n) * u0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(17,), (9, 11), (6, 7, 5)])
def test_heat_dirichlet_sine_eigenvector_so2(orc, shape):
    if len(shape) == 1:
        pytest.skip("1D is not a library mode")
    ks = [1 + (i % 3) for i in range(len(shape))]
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    u0 = np.ones(shape)
    lam = 0.0
    for g, n, k in zip(grids, shape, ks):
        th = math.pi * k / (n + 1)
        u0 = u0 * np.sin(th * (g + 1))
        lam += -2.0 + 2.0 * math.cos(th)
    a = 0.2 if len(shape) == 2 else 0.15
    n = 20
    u = orc.heat_run(u0, 2, a, n, bc=orc.BC_ZERO)
    np.testing.assert_allclose(u, (1 + a * lam) ** n * u0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("so", SOS)
def test_constant_field(orc, so):
    r = so // 2
    shape = (20, 18, 22)
    c = np.full(shape, 0.75)
    a = 0.8 * synthetic.heat_a_max(3, so)
    # periodic: L(1) = 0 exactly, the field never changes
    np.testing.assert_array_equal(orc.heat_run(c, so, a, 5, bc=orc.BC_PERIODIC), c)
    # Dirichlet: after n steps the boundary influence reaches r*n cells
    n = 2
    u = orc.heat_run(c, so, a, n, bc=orc.BC_ZERO)
    m = r * n
    inner = u[m:-m, m:-m, m:-m]
    np.testing.assert_array_equal(inner, 0.75)
    assert np.all(u[:m] < 0.75) or np.any(u[:m] != 0.75)


@pytest.mark.parametrize("so", SOS)
def test_heat_periodic_invariants(orc, so):
    u0 = synthetic.uniform_field(7, (10, 11, 12)).astype(np.float64)
    a = 0.8 * synthetic.heat_a_max(3, so)
    prev = u0
    for _ in range(6):
        u = orc.heat_run(prev, so, a, 1, bc=orc.BC_PERIODIC)
        assert np.sum(u) == pytest.approx(np.sum(prev), rel=1e-13)
        assert np.linalg.norm(u) <= np.linalg.norm(prev) * (1 + 1e-14)
        prev = u


def test_heat_maximum_principle_so2(orc):
    u0 = synthetic.uniform_field(8, (12, 13, 14)).astype(np.float64)
    a = 1.0 / 6.0  # = 1/(2D) in 3D
    u = orc.heat_run(u0, 2, a, 10, bc=orc.BC_ZERO)
    assert u.min() >= 0.0 and u.max() <= u0.max()


@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape", [(6, 7), (5, 4, 6), (9, 3)])
@pytest.mark.parametrize("periodic", [False, True])
def test_heat_brute_force(orc, so, shape, periodic):
    if periodic and min(shape) < so // 2:
        pytest.skip("periodic ghosts need N >= r")
    u0 = synthetic.uniform_field(11, shape).astype(np.float64)
    w = [float(x) for x in central_weights(so)]
    a = 0.9 * synthetic.heat_a_max(len(shape), so)
    ref = brute.heat_brute(u0, w, a, 7, periodic)
    got = orc.heat_run(u0, so, a, 7, bc=orc.BC_PERIODIC if periodic else orc.BC_ZERO)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


# ------------------------------------------------------------ wave sweeps ---

@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape,ks", [((16, 12), (3, 1)), ((10, 12, 8), (2, 1, 3))])
def test_wave_periodic_mode_oscillates(orc, so, shape, ks):
    w = central_weights(so)
    mode, thetas = _mode(shape, ks)
    nd = len(shape)
    kap = (0.6 * synthetic.wave_courant_max(nd, so)) ** 2
    lam = sum(symbol(w, t) for t in thetas)
    cw = 1.0 + kap * lam / 2.0  # cos(omega dt)
    assert -1 < cw < 1
    om = math.acos(cw)
    n = 40
    P, C = orc.wave_run(cw * mode, mode, np.full(shape, kap), so, n, bc=orc.BC_PERIODIC)
    np.testing.assert_allclose(C, math.cos(n * om) * mode, rtol=0, atol=1e-11)
    np.testing.assert_allclose(P, math.cos((n - 1) * om) * mode, rtol=0, atol=1e-11)


@pytest.mark.parametrize("so", SOS)
def test_wave_energy_conserved_variable_speed(orc, so):
    shape = (12, 10, 14)  # (nz, ny, nx)
    c = synthetic.layered_velocity(shape, synthetic.five_layer_speeds()).astype(np.float64)
    h = 10.0
    dt = 0.5 * synthetic.wave_courant_max(3, so) * h / 4500.0
    kap = orc.kappa_from_velocity(c, dt, h)
    u0 = synthetic.uniform_field(21, shape).astype(np.float64) - 0.5
    um = synthetic.uniform_field(22, shape).astype(np.float64) * 0.1 + 0.9 * u0
    E0 = orc.energy(u0, um, kap, so)
    assert E0 > 0
    P, C = um, u0
    for _ in range(5):
        P, C = orc.wave_run(P, C, kap, so, 10)
        assert orc.energy(C, P, kap, so) == pytest.approx(E0, rel=1e-11)


def test_wave_energy_detects_instability(orc):
    shape = (8, 9, 10)
    so = 4
    kap = np.full(shape, (1.2 * synthetic.wave_courant_max(3, so)) ** 2)
    u0 = synthetic.uniform_field(5, shape).astype(np.float64) - 0.5
    P, C = orc.wave_run(u0, u0, kap, so, 60)
    assert not np.isfinite(np.abs(C).max()) or np.abs(C).max() > 1e3


@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape", [(6, 5), (4, 5, 6)])
def test_wave_brute_force_with_source(orc, so, shape):
    u0 = synthetic.uniform_field(31, shape).astype(np.float64) - 0.5
    um = synthetic.uniform_field(32, shape).astype(np.float64) - 0.5
    c = 1500.0 + 3000.0 * synthetic.uniform_field(33, shape).astype(np.float64)
    h, nd = 10.0, len(shape)
    dt = 0.5 * synthetic.wave_courant_max(nd, so) * h / c.max()
    kap = orc.kappa_from_velocity(c, dt, h)
    src_xyz = tuple(reversed([s // 2 for s in shape]))
    src_zyx = tuple(reversed(src_xyz))
    flat = int(np.ravel_multi_index(src_zyx, shape))
    f0, t0, amp, step0, n = 15.0, 0.05, 2.0, 3, 9
    vals = [amp * kap.reshape(-1)[flat] * h * h * orc.ricker((step0 + s) * dt, f0, t0)
            for s in range(n)]
    refP, refC = brute.wave_brute(um, u0, kap, [float(x) for x in central_weights(so)], n,
                                  src_flat=flat, src_values=vals)
    P, C = orc.wave_run(um, u0, kap, so, n, step0=step0, src=src_xyz, f0=f0, t0=t0, amp=amp,
                        dt=dt, h=h)
    np.testing.assert_allclose(C, refC, rtol=0, atol=1e-11)
    np.testing.assert_allclose(P, refP, rtol=0, atol=1e-11)


def test_ricker_closed_form(orc):
    f0, t0 = 10.0, 0.1
    assert orc.ricker(t0, f0, t0) == 1.0
    tz = 1.0 / (math.pi * f0 * math.sqrt(2.0))  # zeros of 1 - 2 (pi f0 t)^2
    assert abs(orc.ricker(t0 + tz, f0, t0)) < 1e-15
    assert abs(orc.ricker(t0 - tz, f0, t0)) < 1e-15
    tm = math.sqrt(1.5) / (math.pi * f0)  # minima, value -2 e^{-3/2}
    assert orc.ricker(t0 + tm, f0, t0) == pytest.approx(-2.0 * math.exp(-1.5), rel=1e-14)
    for dt_ in (0.01, 0.033):
        assert orc.ricker(t0 + dt_, f0, t0) == orc.ricker(t0 - dt_, f0, t0)


# --------------------------------------------------- decomposition (dmp) ---

def test_swap_exchanges_match_paper_example():
    """Section 4.2 listing: memref 108x108, halo 4, exchanges along dim 1."""
    from oracle import exchanges_for, Exchange
    ex = exchanges_for((100, 100), (4, 4), grid=(1, 3), coord=(0, 1))
    assert ex == [
        Exchange(at=(4, 0), size=(100, 4), source_offset=(0, 4), to=(0, -1)),
        Exchange(at=(4, 104), size=(100, 4), source_offset=(0, -4), to=(0, 1)),
    ]
    # a corner rank of a 2x2 grid has one neighbour per dimension
    ex = exchanges_for((100, 100), (4, 4), grid=(2, 2), coord=(0, 0))
    assert ex == [
        Exchange(at=(104, 4), size=(4, 100), source_offset=(-4, 0), to=(1, 0)),
        Exchange(at=(4, 104), size=(100, 4), source_offset=(0, -4), to=(0, 1)),
    ]


def test_decompose_extents():
    from oracle import decompose_extents
    assert decompose_extents(10, 3) == [4, 3, 3]
    assert decompose_extents(1024, 2) == [512, 512]
    assert sum(decompose_extents(1001, 7)) == 1001


@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape,decomp", [((12, 14, 16), (2, 2, 2)), ((11, 9, 13), (3, 2, 2)),
                                          ((20, 22), (2, 3, 1))])
def test_decomposed_heat_equals_global(orc, so, shape, decomp):
    u0 = synthetic.uniform_field(41, shape).astype(np.float64)
    a = 0.8 * synthetic.heat_a_max(len(shape), so)
    ref = orc.heat_run(u0, so, a, 6)
    got = orc.decomposed_heat_run(u0, so, a, 6, decomp)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("so", SOS)
@pytest.mark.parametrize("shape,decomp", [((12, 14, 16), (2, 2, 2)), ((11, 9, 13), (3, 2, 2)),
                                          ((20, 22), (2, 3, 1))])
@pytest.mark.parametrize("nsteps", (5, 6))
def test_decomposed_two_step_heat_equals_global(orc, so, shape, decomp, nsteps):
    """Two steps per exchange: halos 2r deep and the phased exchange that carries the edge
    regions; the step-1 values in the halos equal the neighbours' own, so the result is the
    global run's, in FP64 bit for bit (odd counts end with one step).  Subdomains are at
    least 2r wide where the shapes allow it."""
    r = so // 2
    if any(n // p < 2 * r for n, p in zip(reversed(shape), decomp)):
        pytest.skip("a subdomain thinner than 2r")
    u0 = synthetic.uniform_field(42, shape).astype(np.float64)
    a = 0.8 * synthetic.heat_a_max(len(shape), so)
    ref = orc.heat_run(u0, so, a, nsteps)
    got = orc.decomposed_heat_run_two_step(u0, so, a, nsteps, decomp)
    np.testing.assert_array_equal(got, ref)


def test_two_step_exchange_without_edges_differs(orc):
    """The edge regions matter: with faces only (each phase over the interior of the other
    axes) two steps differ from the global run near the subdomain corners."""
    from oracle import decomp as dm
    shape, so, decomp = (12, 14, 16), 2, (2, 2, 2)
    u0 = synthetic.uniform_field(43, shape).astype(np.float64)
    a = 0.8 * synthetic.heat_a_max(3, so)
    ref = orc.heat_run(u0, so, a, 2)
    saved = dm.deep_swap

    def faces_only(D, bufs):
        # a deep exchange whose phases never span the earlier phases' halos
        h = D.r
        for d in reversed(range(D.nd)):
            sends = {}
            for c in D.coords:
                ls = D.local_shape(c)
                for direction in (-1, 1):
                    nb = c[d] + direction
                    if nb < 0 or nb >= D.grid[d]:
                        continue
                    src = [slice(h, h + ls[e]) if e != d else
                           slice(h if direction < 0 else ls[e], (h if direction < 0 else ls[e]) + h)
                           for e in range(D.nd)]
                    sends[(c, direction)] = bufs[c][tuple(src)].copy()
            for c in D.coords:
                ls = D.local_shape(c)
                for direction in (-1, 1):
                    nb = c[d] + direction
                    if nb < 0 or nb >= D.grid[d]:
                        continue
                    dst = [slice(h, h + ls[e]) if e != d else
                           slice(0 if direction < 0 else h + ls[e], (0 if direction < 0 else h + ls[e]) + h)
                           for e in range(D.nd)]
                    ncoord = tuple(ci + (direction if e == d else 0) for e, ci in enumerate(c))
                    bufs[c][tuple(dst)] = sends[(ncoord, -direction)]

    dm.deep_swap = faces_only
    try:
        got = orc.decomposed_heat_run_two_step(u0, so, a, 2, decomp)
    finally:
        dm.deep_swap = saved
    assert np.max(np.abs(got - ref)) > 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("so", (2, 8))
def test_decomposed_wave_equals_global(orc, so):
    shape = (10, 12, 14)
    u0 = synthetic.uniform_field(51, shape).astype(np.float64)
    um = synthetic.uniform_field(52, shape).astype(np.float64)
    kap = np.full(shape, 0.1) + 0.05 * synthetic.uniform_field(53, shape).astype(np.float64)
    rp, rc = orc.wave_run(um, u0, kap, so, 5)
    gp, gc = orc.decomposed_wave_run(um, u0, kap, so, 5, (2, 2, 2))
    np.testing.assert_array_equal(gc, rc)
    np.testing.assert_array_equal(gp, rp)


# ---------------------------------------------------------------------------
# Adjoint of the leapfrog step (used to train a closure through rollouts) and
# the dependency-cone sampling of long heat runs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("so,shape", [(2, (5, 4, 6)), (4, (4, 6, 5)), (8, (3, 9, 7))])
def test_wave_adjoint_is_the_transpose_of_the_step_matrix(orc, so, shape):
    """The adjoint equals T^T applied to the cotangents, T the dense block step matrix
    [[2I + K L, -I], [I, 0]] built independently of the loop code."""
    from oracle.brute import laplacian_matrix
    rng = np.random.default_rng(so)
    kap = rng.uniform(0.01, 0.3, shape)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    L = laplacian_matrix(shape, orc.central_weights_f64(so))
    K = np.diag(kap.reshape(-1))
    n = L.shape[0]
    T = np.block([[2.0 * np.eye(n) + K @ L, -np.eye(n)], [np.eye(n), np.zeros((n, n))]])
    want = T.T @ np.concatenate([a.reshape(-1), b.reshape(-1)])
    cur, prev = orc.wave_step_adjoint(a, b, kap, so)
    assert np.allclose(cur.reshape(-1), want[:n], rtol=1e-13, atol=1e-13)
    assert np.allclose(prev.reshape(-1), want[n:], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("so", [2, 4, 8])
def test_wave_adjoint_dot_product(orc, so):
    """<step(x), y> = <x, step^T(y)> on a grid too large for the dense matrix."""
    rng = np.random.default_rng(10 + so)
    shape = (13, 17, 19)
    kap = rng.uniform(0.01, 0.3, shape)
    u, up, a, b = (rng.standard_normal(shape) for _ in range(4))
    n1, n0 = orc.wave_step(u, up, kap, so)
    cur, prev = orc.wave_step_adjoint(a, b, kap, so)
    lhs = np.sum(n1 * a) + np.sum(n0 * b)
    rhs = np.sum(u * cur) + np.sum(up * prev)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.sqrt(np.sum(n1 * n1) * np.sum(a * a)))


@pytest.mark.parametrize("so", [2, 4, 8])
def test_cone_boxes_equal_the_whole_grid_run(orc, so):
    from oracle.cones import heat_on_box
    dims = (30, 28, 33)
    a = 0.8 * synthetic.heat_a_max(3, so)
    full = orc.heat_run(synthetic.uniform_field(2, dims), so, a, 6)
    for lo, hi in (((10, 11, 12), (14, 16, 15)), ((0, 0, 0), (4, 5, 6)), ((26, 0, 29), (30, 28, 33))):
        got = heat_on_box(lambda l, h: synthetic.uniform_box(2, dims, l, h), dims, lo, hi, so, a, 6)
        assert np.array_equal(got, full[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
