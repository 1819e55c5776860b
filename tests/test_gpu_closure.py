"""GPU: the learned closure's forward pass, gradients and optimiser against the
FP64 oracle, its coupling to the wave solver, and what training gains.

Tolerances: the GPU network stores weights and activations in BF16 (8-bit
mantissa, relative rounding 2^-9) and accumulates in FP32, so its output and
its gradients are compared with the FP64 oracle by relative L2 error <= 3e-2
(three BF16 layers, each adding a few 2^-9 roundings).  Adam runs in FP32 on
the GPU's own gradients and is compared at 1e-5.
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import closure as ocl

pytestmark = pytest.mark.gpu

TOL_NET = 3e-2


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make_inputs(torch, dims, seed):
    shape = tuple(reversed(dims))
    up = synthetic.uniform_field(seed, shape) - np.float32(0.5)
    un = synthetic.uniform_field(seed + 1, shape) - np.float32(0.5)
    cn = (np.float32(0.3) + np.float32(0.7) * synthetic.uniform_field(seed + 2, shape)).astype(np.float32)
    ref = up + np.float32(0.05) * (synthetic.uniform_field(seed + 3, shape) - np.float32(0.5))
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (up, un, cn, ref)]
    return (up, un, cn, ref), t


def oracle_params(seed=9, w3_gain=10.0):
    p = ocl.init_params(4, 16, seed)
    p["w3"] = p["w3"] * w3_gain
    p["b3"] = p["b3"] + 0.05
    return p


def closure_inputs(s, up, un, cn):
    """x = s (u+, u^n, c_n^2 u+, c_n^2 u^n): the closure's input definition."""
    up, un, c2 = (np.asarray(v, dtype=np.float64) for v in (up, un, np.asarray(cn, np.float64) ** 2))
    return np.stack([s * up, s * un, s * c2 * up, s * c2 * un])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims", [(20, 18, 16), (35, 9, 7)])
def test_forward_matches_oracle(torch_cuda, dims):
    from paper_2404_02218_gb300.closure import Closure, flatten_params
    s = 2.0
    (up, un, cn, _), (tu, tn, tc, _) = make_inputs(torch_cuda, dims, 40)
    p = oracle_params()
    cl = Closure(int(np.prod(dims)), s)
    cl.set_params(flatten_params(p))
    corr = cl.forward(tu, tn, tc).cpu().numpy()
    x = closure_inputs(s, up, un, cn)
    o, _ = ocl.forward(x, p)
    assert rel(corr * s, o[0]) <= TOL_NET
    cl.close()


def test_tcgen05_and_mma_sync_convolutions_agree(torch_cuda):
    """The tcgen05 (tensor memory) and mma.sync convolutions compute the same network, with the
    last layer on the tensor cores in tap-split form (impl 0), on the CUDA cores (impl 2) or
    on the tensor cores like the hidden layers (impl 3)."""
    from paper_2404_02218_gb300.closure import Closure, flatten_params
    dims = (300, 21, 40)  # several 128-point rows, a ragged row end, two z chunks
    s = 2.0
    (up, un, cn, _), (tu, tn, tc, _) = make_inputs(torch_cuda, dims, 45)
    p = oracle_params()
    cl = Closure(int(np.prod(dims)), s)
    cl.set_params(flatten_params(p))
    a = cl.forward(tu, tn, tc).cpu().numpy()
    cl.set_conv_impl(1)
    b = cl.forward(tu, tn, tc).cpu().numpy()
    cl.set_conv_impl(2)
    c = cl.forward(tu, tn, tc).cpu().numpy()
    cl.set_conv_impl(3)
    d = cl.forward(tu, tn, tc).cpu().numpy()
    assert np.abs(b).max() > 0
    # FP32 sums of the same BF16 products in another order; a few BF16 roundings of
    # intermediate activations may differ by one unit
    assert rel(a, b) <= 2e-3
    assert rel(c, b) <= 2e-3
    assert rel(d, b) <= 2e-3
    o, _ = ocl.forward(closure_inputs(s, up, un, cn), p)
    assert rel(a * s, o[0]) <= TOL_NET
    cl.close()


@pytest.mark.parametrize("impl", [0, 1, 2, 3])
def test_loss_and_gradients_match_oracle_all_impls(torch_cuda, impl):
    from paper_2404_02218_gb300.closure import Closure, flatten_params, unflatten_params
    dims = (140, 12, 9)
    s = 2.0
    (up, un, cn, ref), (tu, tn, tc, tr) = make_inputs(torch_cuda, dims, 52)
    p = oracle_params()
    cl = Closure(int(np.prod(dims)), s)
    cl.set_conv_impl(impl)
    cl.set_params(flatten_params(p))
    loss = cl.loss_grad(tu, tn, tc, tr)
    g = unflatten_params(cl.get_grads())
    x = closure_inputs(s, up, un, cn)
    target = (s * (ref.astype(np.float64) - up))[None]
    L, gref = ocl.loss_and_grads(x, target, p)
    assert loss == pytest.approx(L, rel=TOL_NET)
    for k in ocl.PARAM_ORDER:
        assert rel(g[k], gref[k]) <= TOL_NET, k
    cl.close()


def test_loss_and_gradients_match_oracle(torch_cuda):
    from paper_2404_02218_gb300.closure import Closure, flatten_params, unflatten_params
    dims = (24, 20, 12)
    s = 2.0
    (up, un, cn, ref), (tu, tn, tc, tr) = make_inputs(torch_cuda, dims, 50)
    p = oracle_params()
    cl = Closure(int(np.prod(dims)), s)
    cl.set_params(flatten_params(p))
    loss = cl.loss_grad(tu, tn, tc, tr)
    g = unflatten_params(cl.get_grads())
    x = closure_inputs(s, up, un, cn)
    target = (s * (ref.astype(np.float64) - up))[None]
    L, gref = ocl.loss_and_grads(x, target, p)
    assert loss == pytest.approx(L, rel=TOL_NET)
    for k in ocl.PARAM_ORDER:
        assert rel(g[k], gref[k]) <= TOL_NET, k
    cl.close()


def test_adam_step_matches_oracle(torch_cuda):
    from paper_2404_02218_gb300.closure import Closure, flatten_params, unflatten_params
    dims = (16, 16, 8)
    (_, _, _, _), (tu, tn, tc, tr) = make_inputs(torch_cuda, dims, 60)
    p = oracle_params()
    cl = Closure(int(np.prod(dims)), 1.0)
    cl.set_params(flatten_params(p))
    p0 = unflatten_params(cl.get_params())
    cl.loss_grad(tu, tn, tc, tr)
    g = unflatten_params(cl.get_grads())
    cl.adam_step(1e-3)
    p1 = unflatten_params(cl.get_params())
    ref = {k: v.copy() for k, v in p0.items()}
    ocl.adam_step(ref, g, {}, 1e-3, 1)
    for k in ocl.PARAM_ORDER:
        np.testing.assert_allclose(p1[k], ref[k], rtol=1e-5, atol=1e-9)
    cl.close()


def test_strided_read_is_injection(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid
    dims = (34, 30, 22)
    g = Grid(3, dims, 4, "heat", dt=0.01)
    u0 = synthetic.uniform_field(70, tuple(reversed(dims)))
    g.set_field("u", u0)
    out = torch.empty((11, 15, 17), dtype=torch.float32, device="cuda")
    N.stencil_get_field_strided(g.h, N.GBST_U, out.data_ptr(), 2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), u0[::2, ::2, ::2])


def test_attached_closure_adds_its_correction(torch_cuda):
    """run(1) with a closure == plain run(1) + closure(u+, u^n, c_norm), bit for bit."""
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.closure import Closure, flatten_params, C_REF
    from paper_2404_02218_gb300.grid import Grid
    dims = (40, 36, 24)
    shape = tuple(reversed(dims))
    so, h = 4, 20.0
    c = synthetic.layered_velocity(shape, synthetic.five_layer_speeds())
    dt = 0.5 * synthetic.wave_courant_max(3, so) * h / 4500.0
    u0 = synthetic.uniform_field(80, shape) - np.float32(0.5)
    um = synthetic.uniform_field(81, shape) - np.float32(0.5)
    cl = Closure(int(np.prod(dims)), 3.0)
    cl.set_params(flatten_params(oracle_params()))

    def grid():
        g = Grid(3, dims, so, "wave", h=h, dt=dt, stream=cl.stream)
        g.set_field("vel", c)
        g.set_field("u", u0)
        g.set_field("u_prev", um)
        return g

    plain = grid()
    plain.run(1)
    up = torch.empty(shape, dtype=torch.float32, device="cuda")
    plain.get_field("u", out=up)
    un = torch.from_numpy(u0).cuda()
    cn = torch.from_numpy((c / np.float32(C_REF)).astype(np.float32)).cuda()
    corr = cl.forward(up, un, cn)
    want = (up + corr).cpu().numpy()
    g = grid()
    N.stencil_attach_closure(g.h, cl.h, C_REF)
    g.run(1)
    got = g.get_field("u", np.float32)
    # c_norm is computed on the device from kappa (sqrt), so allow its last-bit difference
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-6 * float(np.abs(want).max()))


def test_training_reduces_coarse_error(torch_cuda):
    """Train on small fine/coarse pairs and measure what the closure gains.

    Fine 192^3 (h = 10 m) and coarse 96^3 (h = 20 m) grids of seeded layered
    models, 100 coarse steps; four training seeds, a disjoint test seed.  The
    gain is err(plain coarse) / err(closure-corrected coarse), both relative L2
    against the restricted fine solution at the last step.
    """
    from paper_2404_02218_gb300.closure import PairConfig, evaluate, new_closure, train
    cfg = PairConfig(nc=96, steps=100)
    cl = new_closure(cfg, cfg.nc ** 3)
    losses = train(cl, seeds=(10, 11, 12, 13), cfg=cfg, lr=2e-3, epochs=20)
    assert len(losses) > 1000 and np.isfinite(losses).all()
    res = evaluate(cl, 99, cfg, checkpoints=(25, 50, 75))
    print("closure result:", res)
    assert np.isfinite(res["rel_l2_closure"])
    assert res["gain"] > 1.0


def test_gelu_within_its_stated_bound(torch_cuda):
    """The hidden layers' activation (Abramowitz & Stegun 7.1.26 form of Phi) against the
    exact GELU in FP64 on a dense grid, the signed zeros and large magnitudes."""
    from math import erf
    from paper_2404_02218_gb300 import native as N
    torch = torch_cuda
    xs = np.concatenate([np.linspace(-14.0, 14.0, 1_000_001), [0.0, -0.0, 40.0, -40.0, 1e-30, -1e-30]])
    x = torch.from_numpy(xs.astype(np.float32)).cuda()
    y = torch.empty_like(x)
    N.closure_gelu(x.data_ptr(), y.data_ptr(), x.numel())
    torch.cuda.synchronize()
    xf = xs.astype(np.float32).astype(np.float64)
    exact = xf * 0.5 * (1.0 + np.vectorize(erf)(xf / np.sqrt(2.0)))
    err = np.abs(y.double().cpu().numpy() - exact)
    assert np.all(err <= 1.8e-7 * np.maximum(1.0, np.abs(xf)))
    # n = 0 is a no-op; in place works
    N.closure_gelu(x.data_ptr(), x.data_ptr(), 0)
    N.closure_gelu(x.data_ptr(), x.data_ptr(), x.numel())
    torch.cuda.synchronize()
    assert torch.equal(x, y)
