"""The allocation-free reduction entry point, through the C ABI (GPU).

gbst_reduce_dense_f64_noalloc is for callers that cannot allocate device
memory at the point of use (their device memory is owned by their own pool, or
their loop must not call cudaMalloc/cudaFree, which can synchronise the
device).  It keeps its partial sums in a fixed array inside the library.  This
file is collected last so that a failure here cannot hide other results, and
it passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

CHUNK = 65536  # elements reduced by one block of the entry point


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _expected(v64: np.ndarray, kind, N) -> float:
    if v64.size == 0:
        return 0.0
    if kind == N.GBST_RED_SUM:
        return float(np.sum(v64))
    if kind == N.GBST_RED_L2SQ:
        return float(np.sum(v64 * v64))
    return float(np.max(np.abs(v64)))


def _reduce(torch, N, x, dtype_code, kind, out, stream):
    N.gbst_reduce_dense_f64_noalloc(x.data_ptr() if x.numel() else 0, dtype_code, x.numel(), kind,
                                    out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return float(out.item())


def _check(got, want, kind, N, n):
    if kind == N.GBST_RED_MAXABS:
        assert got == want
    else:
        # FP64 sums of n terms in two different orders
        assert got == pytest.approx(want, rel=1e-12, abs=1e-13 * max(1, n))


def test_noalloc_reduction_matches_stencil_reduce_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    from paper_2404_02218_gb300.grid import Grid

    dims = (70, 45, 33)
    shape = tuple(reversed(dims))
    cases = [(synthetic.uniform_field(81, shape) - np.float32(0.5), N.GBST_RED_SUM),
             (synthetic.uniform_field(82, shape) * np.float32(3.0), N.GBST_RED_L2SQ),
             (synthetic.uniform_field(83, shape) - np.float32(0.7), N.GBST_RED_MAXABS)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for field, kind in cases:
        g = Grid(3, dims, 4, "heat", h=1.0, dt=0.01, alpha=1.0)
        g.set_field("u", field)
        ref = N.stencil_reduce_f64(g.h, kind)
        g.close()
        x = torch.from_numpy(np.ascontiguousarray(field)).cuda()
        got = _reduce(torch, N, x, N.GBST_F32, kind, out, stream)
        if kind == N.GBST_RED_MAXABS:
            assert got == ref
        else:
            assert got == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_noalloc_every_input_type_and_kind_against_numpy(torch_cuda, dtype):
    """Each load path (FP32, FP64, BF16) and each kind on a ragged many-block array."""
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    n = 37 * CHUNK + 4321
    v = synthetic.uniform_field(90, (n,)).astype(np.float64) * 2.0 - 1.0
    if dtype == "f32":
        x = torch.from_numpy(v.astype(np.float32)).cuda()
        code = N.GBST_F32
    elif dtype == "f64":
        x = torch.from_numpy(v).cuda()
        code = N.GBST_F64
    else:
        x = torch.from_numpy(v.astype(np.float32)).cuda().to(torch.bfloat16)
        code = N.GBST_BF16
    v64 = x.float().double().cpu().numpy()  # the values the device holds, exactly
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for kind in (N.GBST_RED_SUM, N.GBST_RED_L2SQ, N.GBST_RED_MAXABS):
        _check(_reduce(torch, N, x, code, kind, out, stream), _expected(v64, kind, N), kind, N, n)


def test_noalloc_empty_input_gives_zero(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    out = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
    x = torch.zeros(0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for kind in (N.GBST_RED_SUM, N.GBST_RED_L2SQ, N.GBST_RED_MAXABS):
        out.fill_(123.0)
        assert _reduce(torch, N, x, N.GBST_F32, kind, out, stream) == 0.0


def test_noalloc_large_call_then_small_call_reads_no_stale_partials(torch_cuda):
    """More than 256 partials (the final pass loops over them), then a one-block call on the
    same stream: the second result must not include partials the first call left behind."""
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    n_big = 300 * CHUNK + 17
    big = torch.from_numpy(synthetic.uniform_field(91, (n_big,))).cuda() + 0.25
    small_np = synthetic.uniform_field(92, (1000,)) - np.float32(0.5)
    small = torch.from_numpy(small_np).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    big64 = big.double().cpu().numpy()
    for kind in (N.GBST_RED_SUM, N.GBST_RED_L2SQ, N.GBST_RED_MAXABS):
        _check(_reduce(torch, N, big, N.GBST_F32, kind, out, stream), _expected(big64, kind, N), kind, N, n_big)
        _check(_reduce(torch, N, small, N.GBST_F32, kind, out, stream),
               _expected(small_np.astype(np.float64), kind, N), kind, N, small.numel())


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(N.GbstError) as e:
        N.gbst_reduce_dense_f64_noalloc(x.data_ptr(), N.GBST_F32, (1 << 30) + 1, N.GBST_RED_SUM, out.data_ptr(), 0)
    assert e.value.status == N.GBST_EINVAL
    assert "2^30" in str(e.value)
