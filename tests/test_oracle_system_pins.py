"""CPU pins of the oracle's coupled multi-field system (several stencils fused
into one sweep: u_k <- u_k + sum_j A[k][j] L(u_j)).

Pinned against what the mathematics fixes:
* A = a I is nf independent heat equations (the heat oracle, itself pinned);
* periodic Fourier modes: with u_j = c_j * mode, one step maps the amplitude
  vector c to (I + lambda A) c, lambda the stencil's symbol summed over axes;
* a symmetric A = Q diag(mu) Q^T decouples: the fields Q^T u evolve as heat
  equations with a = mu_i;
* brute force: the dense operator I + A (x) L on tiny grids.
A dropped coupling term, a transposed A or a wrong field index fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import brute
from oracle.weights import central_weights, symbol

A3 = np.array([[0.030, 0.012, -0.004],
               [0.007, 0.025, 0.009],
               [0.002, -0.006, 0.020]])  # not symmetric: catches a transposed A


def fields(shape, seeds):
    return [synthetic.uniform_field(s, shape).astype(np.float64) for s in seeds]


@pytest.mark.parametrize("so", [2, 4, 8])
def test_diagonal_coupling_is_independent_heat(so):
    shape = (7, 6, 9)
    u = fields(shape, (1, 2, 3))
    a = 0.6 * synthetic.heat_a_max(3, so)
    got = oracle.system_run(u, so, a * np.eye(3), 6)
    for k in range(3):
        np.testing.assert_array_equal(got[k], oracle.heat_run(u[k], so, a, 6))


@pytest.mark.parametrize("so", [2, 4])
def test_periodic_fourier_mode_amplitudes(so):
    shape, ks = (10, 12, 8), (1, 5, 3)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    mode = np.ones(shape)
    lam = 0.0
    w = central_weights(so)
    for a_, (g, n, k) in enumerate(zip(grids, shape, ks)):
        th = 2 * math.pi * k / n
        mode = mode * np.cos(th * g + 0.3 * (a_ + 1))
        lam += symbol(w, th)
    c = np.array([1.0, -0.5, 0.25])
    n = 9
    got = oracle.system_run([ci * mode for ci in c], so, A3, n, bc=oracle.BC_PERIODIC)
    want = np.linalg.matrix_power(np.eye(3) + lam * A3, n) @ c
    for k in range(3):
        np.testing.assert_allclose(got[k], want[k] * mode, rtol=0, atol=1e-12)


def test_symmetric_coupling_decouples_into_heat_modes():
    so = 4
    shape = (6, 8, 7)
    S = 0.5 * (A3 + A3.T) + 0.02 * np.eye(3)
    mu, Q = np.linalg.eigh(S)
    assert (mu > 0).all()
    u = fields(shape, (4, 5, 6))
    got = oracle.system_run(u, so, S, 5)
    for i in range(3):
        v0 = sum(Q[k, i] * u[k] for k in range(3))
        v = sum(Q[k, i] * got[k] for k in range(3))
        np.testing.assert_allclose(v, oracle.heat_run(v0, so, mu[i], 5), rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape", [(3, 4, 3), (5, 4)])
def test_brute_force_dense_operator(shape):
    so = 4
    w = central_weights(so)
    L = brute.laplacian_matrix(shape, [float(x) for x in w])
    npts = L.shape[0]
    M = np.eye(3 * npts) + np.kron(A3, L)
    u = fields(shape, (7, 8, 9))
    v = np.concatenate([f.reshape(-1) for f in u])
    n = 4
    for _ in range(n):
        v = M @ v
    got = oracle.system_run(u, so, A3, n)
    for k in range(3):
        np.testing.assert_allclose(got[k].reshape(-1), v[k * npts:(k + 1) * npts], rtol=0, atol=1e-13)
