"""Convenience wrapper of one stencil handle, with PyTorch supplying device memory and streams.

PyTorch is plumbing here: its caching allocator backs the library's device
allocations (through the ``gbst_allocator`` hook) and its streams order the
work.  Every step of the computation runs in ``libgbstencil.so``.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import native as N

_EQ = {"heat": N.GBST_HEAT, "wave": N.GBST_WAVE}
_BC = {"zero": N.GBST_BC_ZERO, "periodic": N.GBST_BC_PERIODIC}
_ST = {"f32": N.GBST_F32, "bf16": N.GBST_BF16}
_KER = {"auto": N.GBST_KERNEL_AUTO, "stream": N.GBST_KERNEL_STREAM, "simple": N.GBST_KERNEL_SIMPLE}
_FIELD = {"u": N.GBST_U, "u_prev": N.GBST_U_PREV, "vel": N.GBST_VEL}
_RED = {"sum": N.GBST_RED_SUM, "l2sq": N.GBST_RED_L2SQ, "maxabs": N.GBST_RED_MAXABS,
        "energy": N.GBST_RED_ENERGY}


def _np_dtype_code(dt) -> int:
    dt = np.dtype(dt)
    if dt == np.float32:
        return N.GBST_F32
    if dt == np.float64:
        return N.GBST_F64
    raise TypeError(f"unsupported dtype {dt}")


def _torch_dtype_code(t) -> int:
    import torch
    return {torch.float32: N.GBST_F32, torch.float64: N.GBST_F64, torch.bfloat16: N.GBST_BF16}[t.dtype]


class TorchAllocator:
    """gbst_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device: int):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(size, stream, ctx):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(size), self.device, int(stream or 0))
            except Exception:  # out of memory -> NULL, the library reports ENOMEM
                return None

        def _release(ptr, size, stream, ctx):
            if ptr:
                self._torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc = N.ALLOC_FN(_alloc)
        self._release = N.RELEASE_FN(_release)
        self.struct = N.gbst_allocator(self._alloc, self._release, None)


class Grid:
    """One heat or wave grid (see ``stencil_create`` in include/gbstencil.h)."""

    def __init__(self, ndim: int, dims: Sequence[int], space_order: int, eq: str = "heat", *,
                 bc: str = "zero", storage: str = "f32", h: float = 1.0, dt: float = 1.0,
                 alpha: float = 1.0, coeffs=None, decomp=(1, 1, 1), allow_unstable: bool = False,
                 kernel: str = "auto", tile: int = 0, use_graph: bool = True, stream=None,
                 torch_allocator: bool = True, temporal_block: int = 0):
        import torch
        self._torch = torch
        self.ndim = ndim
        self.dims = tuple(int(d) for d in dims)[:ndim]
        self.eq = eq
        self.storage = storage
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        d = N.gbst_desc()
        d.ndim = ndim
        full = list(self.dims) + [1] * (3 - ndim)
        for i in range(3):
            d.dims[i] = full[i]
        d.space_order = space_order
        d.eq = _EQ[eq]
        d.bc = _BC[bc]
        d.storage = _ST[storage]
        d.h, d.dt, d.alpha = float(h), float(dt), float(alpha)
        self._coeffs = None
        if coeffs is not None:
            self._coeffs = (ctypes.c_double * len(coeffs))(*[float(c) for c in coeffs])
            d.coeffs = self._coeffs
        dec = list(decomp) + [1] * (3 - len(decomp))
        for i in range(3):
            d.decomp[i] = int(dec[i])
        d.allow_unstable = int(allow_unstable)
        d.kernel = _KER[kernel]
        d.tile = int(tile)
        d.use_graph = int(use_graph)
        d.temporal_block = int(temporal_block)
        d.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self._alloc = TorchAllocator(dev) if torch_allocator else None
        d.allocator = ctypes.pointer(self._alloc.struct) if self._alloc else None
        self._desc = d
        self.h = N.stencil_create(d)

    # -- shape helpers -------------------------------------------------------
    @property
    def shape(self):
        """numpy/torch shape of a dense field: (nz, ny, nx) or (ny, nx)."""
        return tuple(reversed(self.dims))

    def _prep_torch(self, t):
        self.stream.wait_stream(self._torch.cuda.current_stream())
        return t

    def set_field(self, field: str, data):
        f = _FIELD[field]
        if isinstance(data, np.ndarray):
            a = np.ascontiguousarray(data)
            assert a.shape == self.shape, (a.shape, self.shape)
            N.stencil_set_field(self.h, f, a.ctypes.data, _np_dtype_code(a.dtype), False)
        else:
            t = data.contiguous()
            assert tuple(t.shape) == self.shape
            if t.is_cuda:
                self._prep_torch(t)
            N.stencil_set_field(self.h, f, t.data_ptr(), _torch_dtype_code(t), t.is_cuda)

    def get_field(self, field: str = "u", dtype=np.float64, out=None):
        f = _FIELD[field]
        if out is None:
            out = np.empty(self.shape, dtype=dtype)
        if isinstance(out, np.ndarray):
            N.stencil_get_field(self.h, f, out.ctypes.data, _np_dtype_code(out.dtype), False)
        else:
            self._prep_torch(out)
            N.stencil_get_field(self.h, f, out.data_ptr(), _torch_dtype_code(out), out.is_cuda)
        return out

    def set_source(self, idx, f0: float, t0: float, amp: float = 1.0):
        N.stencil_set_source(self.h, idx, f0, t0, amp)

    def run(self, nsteps: int):
        N.stencil_run(self.h, nsteps)

    def sync(self):
        N.stencil_sync(self.h)

    def reduce(self, kind: str) -> float:
        return N.stencil_reduce_f64(self.h, _RED[kind])

    @property
    def step(self) -> int:
        return N.stencil_get_step(self.h)

    @step.setter
    def step(self, v: int):
        N.stencil_set_step(self.h, v)

    def describe(self) -> str:
        return N.stencil_describe(self.h)

    def set_plan(self, variant: int = -1, txt: int = 0, zchunks: int = 0, ctas: int = 0):
        N.stencil_set_plan(self.h, variant, txt, zchunks, ctas)

    def set_schedule(self, dynamic: int = -1):
        """Static (0), dynamic (1) or default (-1) work-unit assignment."""
        N.stencil_set_schedule(self.h, dynamic)

    def set_overlap(self, enable: int = -1):
        """Halo exchange overlapped with the sweep: on (1), off (0) or default (-1)."""
        N.stencil_set_overlap(self.h, enable)

    def tune(self, reps: int = 5) -> dict:
        import json
        return json.loads(N.stencil_tune(self.h, reps))

    def set_profile(self, on: bool):
        N.stencil_set_profile(self.h, on)

    def set_persistent(self, on: bool):
        N.stencil_set_persistent(self.h, on)

    def last_kernel_time(self):
        return N.stencil_last_kernel_time(self.h)

    def close(self):
        if getattr(self, "h", None):
            N.stencil_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent grids advanced together (see ``stencil_batch_create``).

    ``members`` is a list of dicts with keys ``dims`` and optionally ``h``,
    ``dt``, ``alpha``; the remaining settings are shared.
    """

    def __init__(self, ndim: int, members, space_order: int, eq: str = "wave", *, storage: str = "f32",
                 kernel: str = "auto", tile: int = 0, use_graph: bool = True, stream=None,
                 torch_allocator: bool = True, allow_unstable: bool = False):
        import torch
        self._torch = torch
        self.ndim = ndim
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._alloc = TorchAllocator(dev) if torch_allocator else None
        self.dims = []
        descs = []
        for m in members:
            d = N.gbst_desc()
            d.ndim = ndim
            dims = tuple(int(x) for x in m["dims"])[:ndim]
            self.dims.append(dims)
            full = list(dims) + [1] * (3 - ndim)
            for i in range(3):
                d.dims[i] = full[i]
                d.decomp[i] = 1
            d.space_order = space_order
            d.eq = _EQ[eq]
            d.bc = N.GBST_BC_ZERO
            d.storage = _ST[storage]
            d.h = float(m.get("h", 1.0))
            d.dt = float(m.get("dt", 1.0))
            d.alpha = float(m.get("alpha", 1.0))
            d.allow_unstable = int(allow_unstable)
            d.kernel = _KER[kernel]
            d.tile = int(tile)
            d.use_graph = int(use_graph)
            d.stream = ctypes.c_void_p(self.stream.cuda_stream)
            d.allocator = ctypes.pointer(self._alloc.struct) if self._alloc else None
            descs.append(d)
        self._descs = descs
        self.h = N.stencil_batch_create(descs)

    def __len__(self):
        return len(self.dims)

    def shape(self, i: int):
        return tuple(reversed(self.dims[i]))

    def set_field(self, i: int, field: str, data):
        f = _FIELD[field]
        if isinstance(data, np.ndarray):
            a = np.ascontiguousarray(data)
            assert a.shape == self.shape(i), (a.shape, self.shape(i))
            N.stencil_batch_set_field(self.h, i, f, a.ctypes.data, _np_dtype_code(a.dtype), False)
        else:
            t = data.contiguous()
            if t.is_cuda:
                self.stream.wait_stream(self._torch.cuda.current_stream())
            N.stencil_batch_set_field(self.h, i, f, t.data_ptr(), _torch_dtype_code(t), t.is_cuda)

    def get_field(self, i: int, field: str = "u", dtype=np.float64):
        out = np.empty(self.shape(i), dtype=dtype)
        N.stencil_batch_get_field(self.h, i, _FIELD[field], out.ctypes.data, _np_dtype_code(out.dtype), False)
        return out

    def set_source(self, i: int, idx, f0: float, t0: float, amp: float = 1.0):
        N.stencil_batch_set_source(self.h, i, idx, f0, t0, amp)

    def run(self, nsteps: int):
        N.stencil_run(self.h, nsteps)

    def sync(self):
        N.stencil_sync(self.h)

    def reduce(self, kind: str, grid: int = -1) -> float:
        return N.stencil_batch_reduce_f64(self.h, grid, _RED[kind])

    def set_persistent(self, on: bool):
        N.stencil_set_persistent(self.h, on)

    def set_plan(self, variant: int = -1, txt: int = 0, zchunks: int = 0, ctas: int = 0):
        N.stencil_set_plan(self.h, variant, txt, zchunks, ctas)

    def set_schedule(self, dynamic: int = -1):
        """Static (0), dynamic (1) or default (-1) work-unit assignment."""
        N.stencil_set_schedule(self.h, dynamic)

    def set_overlap(self, enable: int = -1):
        """Halo exchange overlapped with the sweep: on (1), off (0) or default (-1)."""
        N.stencil_set_overlap(self.h, enable)

    def tune(self, reps: int = 5) -> dict:
        import json
        return json.loads(N.stencil_tune(self.h, reps))

    def describe(self) -> str:
        return N.stencil_describe(self.h)

    def set_profile(self, on: bool):
        N.stencil_set_profile(self.h, on)

    def last_kernel_time(self):
        return N.stencil_last_kernel_time(self.h)

    @property
    def step(self) -> int:
        return N.stencil_get_step(self.h)

    def close(self):
        if getattr(self, "h", None):
            N.stencil_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System(Batch):
    """A coupled system of fields on one 3D grid advanced by fused multi-field
    sweeps (see ``stencil_system_create``): u_k <- u_k + sum_j A[k][j] L(u_j).
    Field k is batch member k."""

    def __init__(self, dims: Sequence[int], space_order: int, coupling, *, kernel: str = "auto", tile: int = 0,
                 use_graph: bool = True, stream=None, torch_allocator: bool = True, allow_unstable: bool = False):
        import torch
        self._torch = torch
        self.ndim = 3
        A = np.asarray(coupling, dtype=np.float64)
        nf = A.shape[0]
        assert A.shape == (nf, nf)
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._alloc = TorchAllocator(dev) if torch_allocator else None
        dims = tuple(int(x) for x in dims)
        self.dims = [dims] * nf
        d = N.gbst_desc()
        d.ndim = 3
        for i in range(3):
            d.dims[i] = dims[i]
            d.decomp[i] = 1
        d.space_order = space_order
        d.eq = N.GBST_HEAT
        d.bc = N.GBST_BC_ZERO
        d.storage = N.GBST_F32
        d.h = d.dt = d.alpha = 1.0
        d.allow_unstable = int(allow_unstable)
        d.kernel = _KER[kernel]
        d.tile = int(tile)
        d.use_graph = int(use_graph)
        d.stream = ctypes.c_void_p(self.stream.cuda_stream)
        d.allocator = ctypes.pointer(self._alloc.struct) if self._alloc else None
        self._descs = [d]
        self.coupling = A
        self.h = N.stencil_system_create(d, nf, A.reshape(-1))
