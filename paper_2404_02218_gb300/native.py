"""ctypes binding of ``libgbstencil.so`` -- argument marshalling only.

Every function here has the name of the C entry point it wraps (see
``include/gbstencil.h``) and raises :class:`GbstError` on a non-zero status.
All computation runs in the CUDA library; there is no fallback: if the library
cannot be built or loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

# ---- constants (mirror include/gbstencil.h) --------------------------------
GBST_OK, GBST_EINVAL, GBST_ENOMEM, GBST_ECUDA, GBST_ETIMEOUT, GBST_EUNSTABLE, GBST_ESTATE, GBST_ENOTSUP = \
    0, -1, -2, -3, -4, -5, -6, -7
GBST_HEAT, GBST_WAVE = 0, 1
GBST_BC_ZERO, GBST_BC_PERIODIC = 0, 1
GBST_F32, GBST_BF16, GBST_F64 = 0, 1, 2
GBST_U, GBST_U_PREV, GBST_VEL = 0, 1, 2
GBST_RED_SUM, GBST_RED_L2SQ, GBST_RED_MAXABS, GBST_RED_ENERGY = 0, 1, 2, 3
GBST_KERNEL_AUTO, GBST_KERNEL_STREAM, GBST_KERNEL_SIMPLE = 0, 1, 2

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EUNSTABLE",
                -6: "ESTATE", -7: "ENOTSUP"}


class GbstError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class gbst_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


class gbst_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("dims", ctypes.c_int64 * 3),
        ("space_order", ctypes.c_int),
        ("eq", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("h", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("coeffs", ctypes.POINTER(ctypes.c_double)),
        ("decomp", ctypes.c_int * 3),
        ("allow_unstable", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("tile", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("allocator", ctypes.POINTER(gbst_allocator)),
        ("temporal_block", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Build (if needed) and load the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            H = ctypes.c_void_p
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            sig = {
                "gbst_version": ([], i32),
                "stencil_last_error": ([], ctypes.c_char_p),
                "stencil_fd_weights": ([i32, ctypes.POINTER(dbl)], i32),
                "stencil_create": ([ctypes.POINTER(gbst_desc), ctypes.POINTER(H)], i32),
                "stencil_set_field": ([H, i32, vp, i32, i32], i32),
                "stencil_get_field": ([H, i32, vp, i32, i32], i32),
                "stencil_set_source": ([H, ctypes.POINTER(i64), dbl, dbl, dbl], i32),
                "stencil_run": ([H, i64], i32),
                "stencil_sync": ([H], i32),
                "stencil_get_step": ([H, ctypes.POINTER(i64)], i32),
                "stencil_set_step": ([H, i64], i32),
                "stencil_reduce_f64": ([H, i32, ctypes.POINTER(dbl)], i32),
                "stencil_describe": ([H, ctypes.c_char_p, ctypes.c_size_t], i32),
                "stencil_destroy": ([H], i32),
                "stencil_set_profile": ([H, i32], i32),
                "stencil_last_kernel_time": ([H, ctypes.POINTER(dbl), ctypes.POINTER(i64)], i32),
                "stencil_set_plan": ([H, i32, i32, i32, i32], i32),
                "stencil_set_schedule": ([H, i32], i32),
                "stencil_set_overlap": ([H, i32], i32),
                "stencil_tune": ([H, i32, ctypes.c_char_p, ctypes.c_size_t], i32),
                "stencil_variant_count": ([], i32),
                "stencil_variant_info": ([i32, ctypes.c_char_p, ctypes.c_size_t], i32),
                "gbst_reduce_dense_f64_noalloc": ([vp, i32, i64, i32, vp, vp], i32),
                "stencil_wave_adjoint_dense": ([i32, i64, i64, i64, vp, vp, vp, vp, vp], i32),
                "closure_set_features": ([H, i32, ctypes.POINTER(dbl), i32], i32),
                "closure_set_trainable": ([H, vp, i64], i32),
                "closure_feature_values": ([H, vp, vp, vp, i64, i64, i64, vp], i32),
                "closure_backward": ([H, vp, vp, vp, i64, i64, i64, vp, vp, vp, i32], i32),
                "stencil_closure_rollout_grad": ([H, vp, vp, i64, ctypes.POINTER(vp), i32, ctypes.POINTER(dbl)],
                                                 i32),
                "stencil_batch_create": ([ctypes.POINTER(gbst_desc), i32, ctypes.POINTER(H)], i32),
                "stencil_batch_size": ([H, ctypes.POINTER(i32)], i32),
                "stencil_system_create": ([ctypes.POINTER(gbst_desc), i32, ctypes.POINTER(dbl), ctypes.POINTER(H)],
                                          i32),
                "stencil_batch_set_field": ([H, i32, i32, vp, i32, i32], i32),
                "stencil_batch_get_field": ([H, i32, i32, vp, i32, i32], i32),
                "stencil_batch_set_source": ([H, i32, ctypes.POINTER(i64), dbl, dbl, dbl], i32),
                "stencil_batch_reduce_f64": ([H, i32, i32, ctypes.POINTER(dbl)], i32),
                "stencil_set_persistent": ([H, i32], i32),
                "stencil_debug_barrier_extra": ([H, ctypes.c_uint], i32),
                "closure_create": ([i32, i32, i64, dbl, vp, ctypes.POINTER(gbst_allocator), ctypes.POINTER(H)], i32),
                "closure_destroy": ([H], i32),
                "closure_param_count": ([H, ctypes.POINTER(i64)], i32),
                "closure_set_params": ([H, vp, i64], i32),
                "closure_get_params": ([H, vp, i64], i32),
                "closure_get_grads": ([H, vp, i64], i32),
                "closure_forward": ([H, vp, vp, vp, i64, i64, i64, vp], i32),
                "closure_gelu": ([vp, vp, i64, vp], i32),
                "closure_loss_grad": ([H, vp, vp, vp, vp, i64, i64, i64, ctypes.POINTER(dbl)], i32),
                "closure_adam_step": ([H, dbl], i32),
                "closure_set_out_scale": ([H, dbl], i32),
                "closure_freeze_biases": ([H, i32], i32),
                "closure_set_conv_impl": ([H, i32], i32),
                "closure_set_loss_weight": ([H, dbl], i32),
                "stencil_attach_closure": ([H, H, dbl], i32),
                "stencil_get_field_strided": ([H, i32, vp, i32], i32),
                "stencil_set_field_async": ([H, i32, vp, i32, i32], i32),
                "stencil_get_field_async": ([H, i32, vp, i32, i32], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(status: int, func: str):
    if status != GBST_OK:
        msg = lib().stencil_last_error()
        raise GbstError(status, func, msg.decode() if msg else "")


def last_error() -> str:
    return lib().stencil_last_error().decode()


def gbst_version() -> int:
    return lib().gbst_version()


def stencil_fd_weights(space_order: int) -> list[float]:
    r = space_order // 2
    out = (ctypes.c_double * (r + 1))()
    _check(lib().stencil_fd_weights(space_order, out), "stencil_fd_weights")
    return list(out)


def stencil_create(desc: gbst_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().stencil_create(ctypes.byref(desc), ctypes.byref(h)), "stencil_create")
    return h


def stencil_set_field(h, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_set_field(h, field, ctypes.c_void_p(ptr), dtype, int(on_device)), "stencil_set_field")


def stencil_get_field(h, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_get_field(h, field, ctypes.c_void_p(ptr), dtype, int(on_device)), "stencil_get_field")


def stencil_set_field_async(h, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_set_field_async(h, field, ctypes.c_void_p(ptr), dtype, int(on_device)),
           "stencil_set_field_async")


def stencil_get_field_async(h, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_get_field_async(h, field, ctypes.c_void_p(ptr), dtype, int(on_device)),
           "stencil_get_field_async")


def stencil_set_source(h, idx, f0: float, t0: float, amp: float):
    arr = (ctypes.c_int64 * 3)(*(list(idx) + [0] * (3 - len(idx))))
    _check(lib().stencil_set_source(h, arr, float(f0), float(t0), float(amp)), "stencil_set_source")


def stencil_run(h, nsteps: int):
    _check(lib().stencil_run(h, int(nsteps)), "stencil_run")


def stencil_sync(h):
    _check(lib().stencil_sync(h), "stencil_sync")


def stencil_get_step(h) -> int:
    v = ctypes.c_int64()
    _check(lib().stencil_get_step(h, ctypes.byref(v)), "stencil_get_step")
    return v.value


def stencil_set_step(h, step: int):
    _check(lib().stencil_set_step(h, int(step)), "stencil_set_step")


def stencil_reduce_f64(h, kind: int) -> float:
    v = ctypes.c_double()
    _check(lib().stencil_reduce_f64(h, kind, ctypes.byref(v)), "stencil_reduce_f64")
    return v.value


def stencil_describe(h) -> str:
    buf = ctypes.create_string_buffer(1024)
    _check(lib().stencil_describe(h, buf, 1024), "stencil_describe")
    return buf.value.decode()


def stencil_destroy(h):
    _check(lib().stencil_destroy(h), "stencil_destroy")


def stencil_set_profile(h, enable: bool):
    _check(lib().stencil_set_profile(h, int(enable)), "stencil_set_profile")


def stencil_last_kernel_time(h):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().stencil_last_kernel_time(h, ctypes.byref(ms), ctypes.byref(n)), "stencil_last_kernel_time")
    return ms.value, n.value


def stencil_set_plan(h, variant: int = -1, txt: int = 0, zchunks: int = 0, ctas: int = 0):
    _check(lib().stencil_set_plan(h, variant, txt, zchunks, ctas), "stencil_set_plan")


def stencil_set_schedule(h, dynamic: int = -1):
    _check(lib().stencil_set_schedule(h, dynamic), "stencil_set_schedule")


def stencil_set_overlap(h, enable: int = -1):
    _check(lib().stencil_set_overlap(h, enable), "stencil_set_overlap")


def stencil_tune(h, reps: int = 5) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().stencil_tune(h, reps, buf, 1 << 16), "stencil_tune")
    return buf.value.decode()


def stencil_variant_count() -> int:
    return lib().stencil_variant_count()


def stencil_variant_info(i: int) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(lib().stencil_variant_info(i, buf, 512), "stencil_variant_info")
    return buf.value.decode()


def gbst_reduce_dense_f64_noalloc(x_ptr: int, dtype: int, n: int, kind: int, out_ptr: int, stream: int = 0):
    """Allocation-free FP64 reduction of a dense device array (result written to out_ptr on the device)."""
    _check(lib().gbst_reduce_dense_f64_noalloc(ctypes.c_void_p(x_ptr), dtype, int(n), kind,
                                               ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)),
           "gbst_reduce_dense_f64_noalloc")


def stencil_wave_adjoint_dense(space_order: int, dims, kappa_ptr: int, lam_next_ptr: int, lam_cur_ptr: int,
                               lam_prev_ptr: int = 0, stream: int = 0):
    """Transpose of one leapfrog step on dense device arrays (dims = (nx, ny, nz))."""
    nx, ny, nz = (int(v) for v in dims)
    _check(lib().stencil_wave_adjoint_dense(space_order, nx, ny, nz, ctypes.c_void_p(kappa_ptr),
                                            ctypes.c_void_p(lam_next_ptr), ctypes.c_void_p(lam_cur_ptr),
                                            ctypes.c_void_p(lam_prev_ptr or None), ctypes.c_void_p(stream)),
           "stencil_wave_adjoint_dense")


def closure_set_trainable(c, mask=None):
    """mask: uint8 numpy array of the parameter count (non-zero trains), or None for all."""
    if mask is None:
        _check(lib().closure_set_trainable(c, None, 0), "closure_set_trainable")
        return
    import numpy as _np
    m = _np.ascontiguousarray(mask, dtype=_np.uint8)
    _check(lib().closure_set_trainable(c, ctypes.c_void_p(m.ctypes.data), m.size), "closure_set_trainable")


def closure_set_features(c, space_order: int, scales):
    arr = (ctypes.c_double * 8)(*[float(v) for v in scales])
    _check(lib().closure_set_features(c, space_order, arr, 8), "closure_set_features")


def closure_feature_values(c, up_ptr: int, un_ptr: int, cn_ptr: int, dims, out_ptr: int):
    nx, ny, nz = (int(v) for v in dims)
    _check(lib().closure_feature_values(c, ctypes.c_void_p(up_ptr), ctypes.c_void_p(un_ptr), ctypes.c_void_p(cn_ptr),
                                        nx, ny, nz, ctypes.c_void_p(out_ptr)), "closure_feature_values")


def closure_backward(c, up_ptr: int, un_ptr: int, cn_ptr: int, dims, grad_corr_ptr: int, grad_up_ptr: int,
                     grad_un_ptr: int, accumulate: bool = False):
    nx, ny, nz = (int(v) for v in dims)
    _check(lib().closure_backward(c, ctypes.c_void_p(up_ptr), ctypes.c_void_p(un_ptr), ctypes.c_void_p(cn_ptr),
                                  nx, ny, nz, ctypes.c_void_p(grad_corr_ptr), ctypes.c_void_p(grad_up_ptr),
                                  ctypes.c_void_p(grad_un_ptr), int(bool(accumulate))), "closure_backward")


def stencil_closure_rollout_grad(h, u_cur_ptr: int, u_prev_ptr: int, step0: int, ref_ptrs) -> float:
    """Rollout loss of the attached closure and its parameter gradient (kept in the closure)."""
    arr = (ctypes.c_void_p * len(ref_ptrs))(*[ctypes.c_void_p(p) for p in ref_ptrs])
    out = ctypes.c_double(0.0)
    _check(lib().stencil_closure_rollout_grad(h, ctypes.c_void_p(u_cur_ptr), ctypes.c_void_p(u_prev_ptr), int(step0),
                                              arr, len(ref_ptrs), ctypes.byref(out)),
           "stencil_closure_rollout_grad")
    return out.value


def stencil_batch_create(descs) -> ctypes.c_void_p:
    arr = (gbst_desc * len(descs))(*descs)
    h = ctypes.c_void_p()
    _check(lib().stencil_batch_create(arr, len(descs), ctypes.byref(h)), "stencil_batch_create")
    return h


def stencil_system_create(desc: gbst_desc, nfields: int, coupling):
    h = ctypes.c_void_p()
    arr = (ctypes.c_double * (nfields * nfields))(*[float(x) for x in coupling])
    _check(lib().stencil_system_create(ctypes.byref(desc), int(nfields), arr, ctypes.byref(h)),
           "stencil_system_create")
    return h


def stencil_batch_size(h) -> int:
    n = ctypes.c_int()
    _check(lib().stencil_batch_size(h, ctypes.byref(n)), "stencil_batch_size")
    return n.value


def stencil_batch_set_field(h, grid: int, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_batch_set_field(h, grid, field, ctypes.c_void_p(ptr), dtype, int(on_device)),
           "stencil_batch_set_field")


def stencil_batch_get_field(h, grid: int, field: int, ptr: int, dtype: int, on_device: bool):
    _check(lib().stencil_batch_get_field(h, grid, field, ctypes.c_void_p(ptr), dtype, int(on_device)),
           "stencil_batch_get_field")


def stencil_batch_set_source(h, grid: int, idx, f0: float, t0: float, amp: float):
    arr = (ctypes.c_int64 * 3)(*(list(idx) + [0] * (3 - len(idx))))
    _check(lib().stencil_batch_set_source(h, grid, arr, float(f0), float(t0), float(amp)),
           "stencil_batch_set_source")


def stencil_batch_reduce_f64(h, grid: int, kind: int) -> float:
    v = ctypes.c_double()
    _check(lib().stencil_batch_reduce_f64(h, grid, kind, ctypes.byref(v)), "stencil_batch_reduce_f64")
    return v.value


def stencil_set_persistent(h, enable: bool):
    _check(lib().stencil_set_persistent(h, int(enable)), "stencil_set_persistent")


def stencil_debug_barrier_extra(h, extra: int):
    _check(lib().stencil_debug_barrier_extra(h, int(extra)), "stencil_debug_barrier_extra")


def closure_create(cin: int, hidden: int, max_points: int, in_scale: float, stream: int = 0, allocator=None):
    h = ctypes.c_void_p()
    _check(lib().closure_create(cin, hidden, int(max_points), float(in_scale), ctypes.c_void_p(stream),
                                ctypes.pointer(allocator) if allocator is not None else None, ctypes.byref(h)),
           "closure_create")
    return h


def closure_destroy(c):
    _check(lib().closure_destroy(c), "closure_destroy")


def closure_param_count(c) -> int:
    n = ctypes.c_int64()
    _check(lib().closure_param_count(c, ctypes.byref(n)), "closure_param_count")
    return n.value


def closure_set_params(c, host_ptr: int, n: int):
    _check(lib().closure_set_params(c, ctypes.c_void_p(host_ptr), int(n)), "closure_set_params")


def closure_get_params(c, host_ptr: int, n: int):
    _check(lib().closure_get_params(c, ctypes.c_void_p(host_ptr), int(n)), "closure_get_params")


def closure_get_grads(c, host_ptr: int, n: int):
    _check(lib().closure_get_grads(c, ctypes.c_void_p(host_ptr), int(n)), "closure_get_grads")


def closure_gelu(x_ptr: int, y_ptr: int, n: int, stream: int = 0):
    _check(lib().closure_gelu(ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(n), ctypes.c_void_p(stream)),
           "closure_gelu")


def closure_forward(c, up: int, un: int, cn: int, dims, corr: int):
    nx, ny, nz = dims
    _check(lib().closure_forward(c, ctypes.c_void_p(up), ctypes.c_void_p(un), ctypes.c_void_p(cn), nx, ny, nz,
                                 ctypes.c_void_p(corr)), "closure_forward")


def closure_loss_grad(c, up: int, un: int, cn: int, ref: int, dims) -> float:
    nx, ny, nz = dims
    v = ctypes.c_double()
    _check(lib().closure_loss_grad(c, ctypes.c_void_p(up), ctypes.c_void_p(un), ctypes.c_void_p(cn),
                                   ctypes.c_void_p(ref), nx, ny, nz, ctypes.byref(v)), "closure_loss_grad")
    return v.value


def closure_adam_step(c, lr: float):
    _check(lib().closure_adam_step(c, float(lr)), "closure_adam_step")


def closure_set_conv_impl(c, impl: int):
    _check(lib().closure_set_conv_impl(c, int(impl)), "closure_set_conv_impl")


def stencil_attach_closure(h, c, c_ref: float):
    _check(lib().stencil_attach_closure(h, c, float(c_ref)), "stencil_attach_closure")


def stencil_get_field_strided(h, field: int, dst_ptr: int, stride: int):
    _check(lib().stencil_get_field_strided(h, field, ctypes.c_void_p(dst_ptr), int(stride)),
           "stencil_get_field_strided")


def closure_set_out_scale(c, v: float):
    _check(lib().closure_set_out_scale(c, float(v)), "closure_set_out_scale")


def closure_freeze_biases(c, freeze: bool):
    _check(lib().closure_freeze_biases(c, int(freeze)), "closure_freeze_biases")


def closure_set_loss_weight(c, w: float):
    _check(lib().closure_set_loss_weight(c, float(w)), "closure_set_loss_weight")
