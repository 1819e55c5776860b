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


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


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
        N.gbst_reduce_dense_f64_noalloc(x.data_ptr(), N.GBST_F32, x.numel(), kind, out.data_ptr(),
                                        stream.cuda_stream)
        torch.cuda.synchronize()
        got = float(out.item())
        if kind == N.GBST_RED_MAXABS:
            assert got == ref
        else:
            assert got == pytest.approx(ref, rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2404_02218_gb300 import native as N
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(N.GbstError) as e:
        N.gbst_reduce_dense_f64_noalloc(x.data_ptr(), N.GBST_F32, (1 << 30) + 1, N.GBST_RED_SUM, out.data_ptr(), 0)
    assert e.value.status == N.GBST_EINVAL
    assert "2^30" in str(e.value)
