"""GPU: field transfers through the C ABI -- host staging, device buffers, and
the asynchronous forms (page-locked host memory or device memory only)."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("dims", [(37, 21, 9), (256, 64, 33)])
def test_async_round_trip_equals_sync(torch_cuda, dims):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid
    shape = tuple(reversed(dims))
    u0 = synthetic.uniform_field(31, shape)
    g = Grid(3, dims, 4, "heat", dt=0.05)
    hin = torch.from_numpy(u0).pin_memory()
    hout = torch.empty(shape, dtype=torch.float32).pin_memory()
    N.stencil_set_field_async(g.h, N.GBST_U, hin.data_ptr(), N.GBST_F32, 0)
    g.run(3)
    N.stencil_get_field_async(g.h, N.GBST_U, hout.data_ptr(), N.GBST_F32, 0)
    g.sync()
    ref = Grid(3, dims, 4, "heat", dt=0.05)
    ref.set_field("u", u0)
    ref.run(3)
    np.testing.assert_array_equal(hout.numpy(), ref.get_field("u", np.float32))
    # device buffers
    din = torch.from_numpy(u0).cuda()
    dout = torch.empty_like(din)
    torch.cuda.synchronize()
    N.stencil_set_field_async(g.h, N.GBST_U, din.data_ptr(), N.GBST_F32, 1)
    N.stencil_get_field_async(g.h, N.GBST_U, dout.data_ptr(), N.GBST_F32, 1)
    g.sync()
    np.testing.assert_array_equal(dout.cpu().numpy(), u0)


def test_async_rejects_pageable_memory_and_velocity(torch_cuda):
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid
    dims = (20, 16, 12)
    g = Grid(3, dims, 2, "heat", dt=0.05)
    a = np.zeros(tuple(reversed(dims)), dtype=np.float32)
    with pytest.raises(N.GbstError) as e:
        N.stencil_set_field_async(g.h, N.GBST_U, a.ctypes.data, N.GBST_F32, 0)
    assert e.value.status == N.GBST_EINVAL
    w = Grid(3, dims, 2, "wave", h=10.0, dt=1e-4)
    torch = pytest.importorskip("torch")
    c = torch.full(tuple(reversed(dims)), 2000.0).pin_memory()
    with pytest.raises(N.GbstError) as e:
        N.stencil_set_field_async(w.h, N.GBST_VEL, c.data_ptr(), N.GBST_F32, 0)
    assert e.value.status == N.GBST_EINVAL


@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_sync_transfers_other_dtypes(torch_cuda, dtype):
    """Row-based transfer kernels with FP64 and BF16 host buffers."""
    from paper_2404_02218_gb300.grid import Grid
    dims = (45, 13, 7)
    shape = tuple(reversed(dims))
    u0 = synthetic.uniform_field(32, shape).astype(np.float64)
    g = Grid(3, dims, 2, "heat", dt=0.05, storage="bf16" if dtype == "bf16" else "f32")
    g.set_field("u", u0)
    got = g.get_field("u", np.float64)
    if dtype == "bf16":
        import torch
        want = torch.from_numpy(u0).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(got, want)
    else:
        np.testing.assert_array_equal(got, u0.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("case", ["2d", "bf16_direct", "bf16_from_f32", "decomposed", "wave_prev"])
def test_async_paths(torch_cuda, case):
    """Pitched copies straight into the padded field (page-locked host data in the
    storage type, one subdomain) and the staging path (other dtypes, decomposed
    grids) give the same fields as the synchronous transfers."""
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid
    dims = (70, 33) if case == "2d" else (70, 33, 17)
    shape = tuple(reversed(dims))
    u0 = synthetic.uniform_field(32, shape)
    storage = "bf16" if case.startswith("bf16") else "f32"
    kw = dict(decomp=(2, 1, 1)) if case == "decomposed" else {}
    eq = "wave" if case == "wave_prev" else "heat"

    def make():
        if eq == "wave":
            g = Grid(3, dims, 4, "wave", h=10.0, dt=1e-3)
            g.set_field("vel", np.full(shape, 1500.0, dtype=np.float32))
            return g
        return Grid(len(dims), dims, 4, "heat", dt=0.05, storage=storage, **kw)

    field = N.GBST_U_PREV if case == "wave_prev" else N.GBST_U
    name = "u_prev" if case == "wave_prev" else "u"
    if case == "bf16_direct":
        host = torch.from_numpy(u0).to(torch.bfloat16).pin_memory()
        dt = N.GBST_BF16
    else:
        host = torch.from_numpy(u0).pin_memory()
        dt = N.GBST_F32
    g = make()
    N.stencil_set_field_async(g.h, field, host.data_ptr(), dt, 0)
    g.run(2)
    out = torch.empty(shape, dtype=host.dtype).pin_memory()
    N.stencil_get_field_async(g.h, field, out.data_ptr(), dt, 0)
    g.sync()
    ref = make()
    ref.set_field(name, host.float().numpy())
    ref.run(2)
    want = ref.get_field(name, np.float32)
    if dt == N.GBST_BF16:
        want = torch.from_numpy(want).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(out.float().numpy(), want)
