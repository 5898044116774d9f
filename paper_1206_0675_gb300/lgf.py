"""ctypes binding of the lgf C-ABI (include/lgf.h).

Argument marshalling only: every step of the gauge-fixing path runs in the
CUDA kernels of ``liblgf.so``.  There is no CPU fallback; loading fails with
a clear error when the library has not been built.

Two layers:

* module-level functions with the C names (``lgf_create``, ``lgf_set_links``,
  ...) that take and return plain integers / pointers, and
* ``Lattice``, a small owner object that marshals numpy arrays (host) and
  torch CUDA tensors (device) into those calls.

Host arrays are complex128 of shape ``(4, Lt, Lz, Ly, Lx, 3, 3)`` for links
and ``(Lt, Lz, Ly, Lx, 3, 3)`` for site fields, i.e. the library's FP64 user
layout ``[mu][t][z][y][x][row][col][re, im]``.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgf.so")

LGF_OK, LGF_E_ARG, LGF_E_NOMEM, LGF_E_CUDA, LGF_E_STATE, LGF_E_NONFINITE, LGF_E_NOTCONV, LGF_E_TIMEOUT, \
    LGF_E_UNSUPPORTED = range(9)
LGF_FP64, LGF_FP32, LGF_MIXED = 0, 1, 2
LGF_STORE18, LGF_STORE12, LGF_TRACK_G, LGF_LEARNED, LGF_PLAIN_SD, LGF_EXACT_EXP = 0, 1, 2, 4, 8, 16
LGF_FFT_2D2D, LGF_FFT_1D4, LGF_FFT_3D1D = 0, 1, 2
LGF_TRACE_FP64, LGF_TRACE_LEARNED, LGF_TRACE_REDO, LGF_TRACE_REPAIRED = 1, 2, 4, 8
LGF_MLP_NPARAM = 8961
MLP_NBUCKET = 40
MLP_NSTAT = 7
LGF_HOST, LGF_DEVICE = 0, 1

_c_int_p = ctypes.POINTER(ctypes.c_int32)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)

# lgf_allocator: void* alloc(size_t, void* stream, void* ctx); void free(void*, size_t, void* stream, void* ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class LgfAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]

# (name, restype, argtypes) for every entry point of include/lgf.h
SIGNATURES = [
    ("lgf_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    ("lgf_create_with_allocator", ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_int, ctypes.c_uint32,
                                                 ctypes.c_void_p, ctypes.POINTER(LgfAllocator),
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    ("lgf_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("lgf_set_links", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_get_links", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("lgf_measure", ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, _c_dbl_p]),
    ("lgf_fix", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_double, _c_int_p,
                               _c_dbl_p, _c_dbl_p]),
    ("lgf_set_learned_theta", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("lgf_or_sweep", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32]),
    ("lgf_or_fix", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                  _c_int_p, _c_dbl_p, _c_dbl_p]),
    ("lgf_get_transform", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_get_gauge", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_get_divergence", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_set_trace", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_set_trace_ex", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_set_defect_bound", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    ("lgf_get_link_defect", ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, _c_int_p]),
    ("lgf_fft4", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int]),
    ("lgf_get_phase", ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    ("lgf_set_timing", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_set_switch_theta", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("lgf_set_fft_decomposition", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    ("lgf_set_fused_update", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_get_timing", ctypes.c_int, [ctypes.c_void_p, _c_dbl_p, ctypes.c_int32, _c_int_p]),
    ("lgf_measure_static", ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    ("lgf_load_preconditioner", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]),
    ("lgf_get_fallbacks", ctypes.c_int, [ctypes.c_void_p, _c_int_p]),
    ("lgf_set_mode_log", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("lgf_get_mode_log", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    ("lgf_mlp_eval", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    ("lgf_mlp_loss_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_void_p, _c_dbl_p, ctypes.c_void_p]),
    ("lgf_mlp_train", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                     ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    ("lgf_mlp_to_bf16", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("lgf_batch_create", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                        ctypes.c_uint32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("lgf_batch_destroy", ctypes.c_int, [ctypes.c_void_p]),
    ("lgf_batch_set_links", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_batch_get_links", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    ("lgf_batch_fix", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("lgf_batch_describe", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    ("lgf_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lgf_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("lgf_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
]

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblgf.so (once).  Raises RuntimeError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1206_0675_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LgfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        lib = load_library()
        msg = f"{where}: {lib.lgf_status_string(status).decode()}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)
        self.status = status


# --- thin C-name wrappers ---------------------------------------------------

def lgf_create(extents, prec: int, flags: int, stream: int = 0) -> int:
    lib = load_library()
    ext = (ctypes.c_int32 * 4)(*[int(e) for e in extents])
    h = ctypes.c_void_p()
    st = lib.lgf_create(ext, int(prec), ctypes.c_uint32(flags), ctypes.c_void_p(stream or None), ctypes.byref(h))
    if st != LGF_OK:
        raise LgfError(st, "lgf_create")
    return h.value


def lgf_create_with_allocator(extents, prec: int, flags: int, stream: int, allocator) -> int:
    """allocator: an LgfAllocator (kept alive by the caller for the handle's lifetime) or None."""
    lib = load_library()
    ext = (ctypes.c_int32 * 4)(*[int(e) for e in extents])
    h = ctypes.c_void_p()
    st = lib.lgf_create_with_allocator(ext, int(prec), ctypes.c_uint32(flags), ctypes.c_void_p(stream or None),
                                       ctypes.byref(allocator) if allocator is not None else None, ctypes.byref(h))
    if st != LGF_OK:
        raise LgfError(st, "lgf_create_with_allocator")
    return h.value


def torch_allocator():
    """An LgfAllocator that takes the handle's device memory from PyTorch's
    caching allocator (torch.cuda.caching_allocator_alloc / _delete), so
    that it is counted and reused with the rest of the process's tensors."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return LgfAllocator(ALLOC_FN(_alloc), FREE_FN(_free), None)


def _check(h, st, where, allow=()):
    if st != LGF_OK and st not in allow:
        detail = load_library().lgf_last_error(ctypes.c_void_p(h)).decode(errors="replace")
        raise LgfError(st, where, detail)
    return st


def lgf_destroy(h: int) -> None:
    load_library().lgf_destroy(ctypes.c_void_p(h))


def lgf_set_links(h: int, ptr: int, where: int) -> None:
    _check(h, load_library().lgf_set_links(ctypes.c_void_p(h), ctypes.c_void_p(ptr), where), "lgf_set_links")


def lgf_get_links(h: int, ptr: int, where: int) -> None:
    _check(h, load_library().lgf_get_links(ctypes.c_void_p(h), ctypes.c_void_p(ptr), where), "lgf_get_links")


def lgf_step(h: int, alpha: float) -> None:
    _check(h, load_library().lgf_step(ctypes.c_void_p(h), float(alpha)), "lgf_step")


def lgf_measure(h: int) -> tuple[float, float]:
    F, th = ctypes.c_double(), ctypes.c_double()
    _check(h, load_library().lgf_measure(ctypes.c_void_p(h), ctypes.byref(F), ctypes.byref(th)), "lgf_measure")
    return F.value, th.value


def lgf_fix(h: int, theta_tol: float, max_iter: int, alpha: float) -> tuple[int, float, float, int]:
    """Returns (iters, F, theta, status); status is LGF_OK or LGF_E_NOTCONV."""
    it, F, th = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    st = load_library().lgf_fix(ctypes.c_void_p(h), float(theta_tol), int(max_iter), float(alpha), ctypes.byref(it),
                                ctypes.byref(F), ctypes.byref(th))
    _check(h, st, "lgf_fix", allow=(LGF_E_NOTCONV,))
    return it.value, F.value, th.value, st


def lgf_set_learned_theta(h: int, theta: float) -> None:
    _check(h, load_library().lgf_set_learned_theta(ctypes.c_void_p(h), float(theta)), "lgf_set_learned_theta")


def lgf_or_sweep(h: int, omega: float, nsweeps: int) -> None:
    _check(h, load_library().lgf_or_sweep(ctypes.c_void_p(h), float(omega), int(nsweeps)), "lgf_or_sweep")


def lgf_or_fix(h: int, theta_tol: float, max_sweeps: int, omega: float,
               check_every: int) -> tuple[int, float, float, int]:
    """Returns (sweeps, F, theta, status); status is LGF_OK or LGF_E_NOTCONV."""
    n, F, th = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    st = load_library().lgf_or_fix(ctypes.c_void_p(h), float(theta_tol), int(max_sweeps), float(omega),
                                   int(check_every), ctypes.byref(n), ctypes.byref(F), ctypes.byref(th))
    _check(h, st, "lgf_or_fix", allow=(LGF_E_NOTCONV,))
    return n.value, F.value, th.value, st


def lgf_get_transform(h: int, ptr: int, where: int) -> None:
    _check(h, load_library().lgf_get_transform(ctypes.c_void_p(h), ctypes.c_void_p(ptr), where),
           "lgf_get_transform")


def lgf_get_gauge(h: int, ptr: int, where: int) -> None:
    _check(h, load_library().lgf_get_gauge(ctypes.c_void_p(h), ctypes.c_void_p(ptr), where), "lgf_get_gauge")


def lgf_get_divergence(h: int, ptr: int, where: int) -> None:
    _check(h, load_library().lgf_get_divergence(ctypes.c_void_p(h), ctypes.c_void_p(ptr), where),
           "lgf_get_divergence")


def lgf_set_trace(h: int, f_ptr: int, t_ptr: int, cap: int) -> None:
    _check(h, load_library().lgf_set_trace(ctypes.c_void_p(h), ctypes.c_void_p(f_ptr), ctypes.c_void_p(t_ptr),
                                           int(cap)), "lgf_set_trace")


def lgf_set_trace_ex(h: int, f_ptr: int, t_ptr: int, flags_ptr: int, defect_ptr: int, cap: int) -> None:
    _check(h, load_library().lgf_set_trace_ex(ctypes.c_void_p(h), ctypes.c_void_p(f_ptr), ctypes.c_void_p(t_ptr),
                                              ctypes.c_void_p(flags_ptr or None), ctypes.c_void_p(defect_ptr or None),
                                              int(cap)), "lgf_set_trace_ex")


def lgf_set_defect_bound(h: int, bound_fp64: float, bound_fp32: float) -> None:
    _check(h, load_library().lgf_set_defect_bound(ctypes.c_void_p(h), float(bound_fp64), float(bound_fp32)),
           "lgf_set_defect_bound")


def lgf_get_link_defect(h: int) -> tuple[float, int]:
    d, n = ctypes.c_double(), ctypes.c_int32()
    _check(h, load_library().lgf_get_link_defect(ctypes.c_void_p(h), ctypes.byref(d), ctypes.byref(n)),
           "lgf_get_link_defect")
    return d.value, n.value


def lgf_fft4(h: int, ptr: int, nfields: int, sign: int, where: int) -> None:
    _check(h, load_library().lgf_fft4(ctypes.c_void_p(h), ctypes.c_void_p(ptr), int(nfields), int(sign), where),
           "lgf_fft4")


def lgf_get_phase(h: int) -> int:
    b = ctypes.c_int32()
    _check(h, load_library().lgf_get_phase(ctypes.c_void_p(h), ctypes.byref(b)), "lgf_get_phase")
    return b.value


def lgf_set_timing(h: int, enable: bool) -> None:
    _check(h, load_library().lgf_set_timing(ctypes.c_void_p(h), 1 if enable else 0), "lgf_set_timing")


def lgf_get_timing(h: int) -> tuple[list[float], int]:
    ms = (ctypes.c_double * 5)()
    n = ctypes.c_int32()
    _check(h, load_library().lgf_get_timing(ctypes.c_void_p(h), ms, 5, ctypes.byref(n)), "lgf_get_timing")
    return list(ms), n.value


LGF_STATIC_MAX_SITES = 16777216


def lgf_load_preconditioner(h: int, ptr: int, n: int, where: int) -> None:
    _check(h, load_library().lgf_load_preconditioner(ctypes.c_void_p(h), ctypes.c_void_p(ptr), n, where),
           "lgf_load_preconditioner")


def lgf_get_fallbacks(h: int) -> int:
    n = ctypes.c_int32()
    _check(h, load_library().lgf_get_fallbacks(ctypes.c_void_p(h), ctypes.byref(n)), "lgf_get_fallbacks")
    return n.value


def lgf_set_mode_log(h: int, enable: bool) -> None:
    _check(h, load_library().lgf_set_mode_log(ctypes.c_void_p(h), 1 if enable else 0), "lgf_set_mode_log")


def lgf_get_mode_log(h: int, ptr: int, n: int) -> None:
    _check(h, load_library().lgf_get_mode_log(ctypes.c_void_p(h), ctypes.c_void_p(ptr), n), "lgf_get_mode_log")


def _stat(st: int, where: str) -> None:
    if st != LGF_OK:
        raise LgfError(st, where)


def lgf_mlp_eval(p_ptr: int, x_ptr: int, n: int, m_ptr: int, stream: int = 0) -> None:
    _stat(load_library().lgf_mlp_eval(ctypes.c_void_p(p_ptr), ctypes.c_void_p(x_ptr), n, ctypes.c_void_p(m_ptr),
                                      ctypes.c_void_p(stream or None)), "lgf_mlp_eval")


def lgf_mlp_loss_grad(p_ptr, x_ptr, y_ptr, w_ptr, n, g_ptr, stream=0) -> float:
    loss = ctypes.c_double()
    _stat(load_library().lgf_mlp_loss_grad(*(ctypes.c_void_p(v) for v in (p_ptr, x_ptr, y_ptr, w_ptr)), n,
                                           ctypes.c_void_p(g_ptr), ctypes.byref(loss),
                                           ctypes.c_void_p(stream or None)), "lgf_mlp_loss_grad")
    return loss.value


def lgf_mlp_train(p_ptr, adam_ptr, x_ptr, y_ptr, w_ptr, n, batch, steps, lr, seed, t0=0, stream=0) -> np.ndarray:
    hist = np.zeros(max(steps, 1))
    _stat(load_library().lgf_mlp_train(*(ctypes.c_void_p(v) for v in (p_ptr, adam_ptr, x_ptr, y_ptr, w_ptr)), n,
                                       batch, steps, ctypes.c_float(lr), ctypes.c_uint64(seed), t0,
                                       hist.ctypes.data, ctypes.c_void_p(stream or None)), "lgf_mlp_train")
    return hist[:steps]


def lgf_mlp_to_bf16(p_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _stat(load_library().lgf_mlp_to_bf16(ctypes.c_void_p(p_ptr), ctypes.c_void_p(out_ptr),
                                         ctypes.c_void_p(stream or None)), "lgf_mlp_to_bf16")


def lgf_measure_static(extents, u_ptr: int, d_ptr: int, f_theta_ptr: int, stream: int = 0) -> int:
    """Allocation-free measurement (device pointers only); returns the lgf_status code."""
    ext = (ctypes.c_int32 * 4)(*[int(e) for e in extents])
    return load_library().lgf_measure_static(ext, ctypes.c_void_p(u_ptr or None), ctypes.c_void_p(d_ptr or None),
                                             ctypes.c_void_p(f_theta_ptr or None), ctypes.c_void_p(stream or None))


class Batch:
    """Many configurations fixed together (lgf_batch_*); links as complex128 host arrays."""

    def __init__(self, extents_list, stream: int | None = None):
        lib = load_library()
        self.extents = [tuple(int(e) for e in ext) for ext in extents_list]
        flat = (ctypes.c_int32 * (4 * len(self.extents)))(*[e for ext in self.extents for e in ext])
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        h = ctypes.c_void_p()
        st = lib.lgf_batch_create(len(self.extents), flat, LGF_FP64, 0, ctypes.c_void_p(stream or None),
                                  ctypes.byref(h))
        if st != LGF_OK:
            raise LgfError(st, "lgf_batch_create")
        self.handle = h.value

    def _check(self, st, where, allow=()):
        if st != LGF_OK and st not in allow:
            raise LgfError(st, where, load_library().lgf_batch_last_error(ctypes.c_void_p(self.handle)).decode())
        return st

    def close(self):
        if getattr(self, "handle", None):
            load_library().lgf_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _shape(self, i):
        lx, ly, lz, lt = self.extents[i]
        return (4, lt, lz, ly, lx, 3, 3)

    def set_links(self, i: int, U) -> None:
        if _is_torch_cuda(U):
            self._check(load_library().lgf_batch_set_links(ctypes.c_void_p(self.handle), i,
                                                           ctypes.c_void_p(U.data_ptr()), LGF_DEVICE),
                        "lgf_batch_set_links")
            return
        a = _host_buffer(U, self._shape(i))
        self._check(load_library().lgf_batch_set_links(ctypes.c_void_p(self.handle), i, ctypes.c_void_p(a.ctypes.data),
                                                       LGF_HOST), "lgf_batch_set_links")

    def get_links(self, i: int) -> np.ndarray:
        a = np.empty(self._shape(i), dtype=np.complex128)
        self._check(load_library().lgf_batch_get_links(ctypes.c_void_p(self.handle), i, ctypes.c_void_p(a.ctypes.data),
                                                       LGF_HOST), "lgf_batch_get_links")
        return a

    def fix(self, theta_tol: float = 1e-14, max_iter: int = 20000, alpha: float = 0.08):
        """Returns (iters, F, theta, all_converged) with per-configuration arrays."""
        n = len(self.extents)
        it = np.zeros(n, dtype=np.int32)
        F = np.zeros(n)
        th = np.zeros(n)
        st = load_library().lgf_batch_fix(ctypes.c_void_p(self.handle), float(theta_tol), int(max_iter), float(alpha),
                                          ctypes.c_void_p(it.ctypes.data), ctypes.c_void_p(F.ctypes.data),
                                          ctypes.c_void_p(th.ctypes.data))
        self._check(st, "lgf_batch_fix", allow=(LGF_E_NOTCONV,))
        return it, F, th, st == LGF_OK

    def describe(self):
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(load_library().lgf_batch_describe(ctypes.c_void_p(self.handle), buf, len(buf)),
                    "lgf_batch_describe")
        return json.loads(buf.value.decode())


# --- marshalling helpers ----------------------------------------------------

_PREC = {"fp64": LGF_FP64, "fp32": LGF_FP32, "mixed": LGF_MIXED}


def _host_buffer(arr: np.ndarray, shape) -> np.ndarray:
    a = np.ascontiguousarray(arr, dtype=np.complex128)
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _is_torch_cpu(x) -> bool:
    return type(x).__module__.startswith("torch") and not getattr(x, "is_cuda", True)


def _torch_host_ptr(t, nbytes: int) -> int:
    """Pointer of a contiguous CPU torch tensor (e.g. pinned) holding nbytes of FP64 data."""
    if not t.is_contiguous() or t.numel() * t.element_size() != nbytes:
        raise ValueError(f"host tensor must be contiguous with {nbytes} bytes")
    return t.data_ptr()


class Lattice:
    """One lattice configuration on the GPU (owns an lgf handle)."""

    def __init__(self, extents, precision: str = "fp64", store12: bool = False, track_G: bool = False,
                 plain_sd: bool = False, learned: bool = False, exact_exp: bool = False,
                 stream: int | None = None, allocator=None):
        """allocator: None (CUDA's stream-ordered allocator), "torch" (PyTorch's
        caching allocator) or an LgfAllocator."""
        self.extents = tuple(int(e) for e in extents)
        lx, ly, lz, lt = self.extents
        self.link_shape = (4, lt, lz, ly, lx, 3, 3)
        self.site_shape = (lt, lz, ly, lx, 3, 3)
        self.nclass = int(np.prod([e // 2 + 1 for e in self.extents]))
        flags = ((LGF_STORE12 if store12 else 0) | (LGF_TRACK_G if track_G else 0) | (LGF_PLAIN_SD if plain_sd else 0)
                 | (LGF_LEARNED if learned else 0) | (LGF_EXACT_EXP if exact_exp else 0))
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        if allocator is None:
            self._allocator = None
            self.handle = lgf_create(self.extents, _PREC[precision], flags, stream)
        else:
            self._allocator = torch_allocator() if allocator == "torch" else allocator
            self.handle = lgf_create_with_allocator(self.extents, _PREC[precision], flags, stream, self._allocator)
        self._trace = None

    def close(self):
        if getattr(self, "handle", None):
            lgf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # links -------------------------------------------------------------------
    def set_links(self, U) -> None:
        """U: complex128 numpy array (host) or a CUDA torch tensor (complex128 or float64 [...,2])."""
        if _is_torch_cuda(U):
            if not U.is_contiguous():
                raise ValueError("device links must be contiguous")
            lgf_set_links(self.handle, U.data_ptr(), LGF_DEVICE)
        elif _is_torch_cpu(U):
            nbytes = 16 * int(np.prod(self.link_shape))
            lgf_set_links(self.handle, _torch_host_ptr(U, nbytes), LGF_HOST)
        else:
            a = _host_buffer(U, self.link_shape)
            lgf_set_links(self.handle, a.ctypes.data, LGF_HOST)

    def get_links(self, out=None):
        if out is not None and _is_torch_cuda(out):
            lgf_get_links(self.handle, out.data_ptr(), LGF_DEVICE)
            return out
        a = np.empty(self.link_shape, dtype=np.complex128) if out is None else out
        lgf_get_links(self.handle, a.ctypes.data, LGF_HOST)
        return a

    def _site_out(self, fn, out):
        if out is not None and _is_torch_cuda(out):
            fn(self.handle, out.data_ptr(), LGF_DEVICE)
            return out
        a = np.empty(self.site_shape, dtype=np.complex128) if out is None else out
        fn(self.handle, a.ctypes.data, LGF_HOST)
        return a

    def get_transform(self, out=None):
        return self._site_out(lgf_get_transform, out)

    def get_gauge(self, out=None):
        return self._site_out(lgf_get_gauge, out)

    def get_divergence(self, out=None):
        return self._site_out(lgf_get_divergence, out)

    # algorithm ---------------------------------------------------------------
    def step(self, alpha: float = 0.08) -> None:
        lgf_step(self.handle, alpha)

    def measure(self) -> tuple[float, float]:
        return lgf_measure(self.handle)

    def fix(self, theta_tol: float = 1e-15, max_iter: int = 10000, alpha: float = 0.08):
        """Returns (iters, F, theta, converged)."""
        it, F, th, st = lgf_fix(self.handle, theta_tol, max_iter, alpha)
        return it, F, th, st == LGF_OK

    def set_learned_theta(self, theta: float) -> None:
        """Apply the learned multiplier only to steps from links with theta below this level."""
        lgf_set_learned_theta(self.handle, theta)

    def or_sweep(self, omega: float = 1.7, nsweeps: int = 1) -> None:
        """nsweeps overrelaxation sweeps (even colour, then odd), then a measurement."""
        lgf_or_sweep(self.handle, omega, nsweeps)

    def or_fix(self, theta_tol: float = 1e-15, max_sweeps: int = 100000, omega: float = 1.7, check_every: int = 1):
        """Overrelaxation gauge fixing; returns (sweeps, F, theta, converged)."""
        n, F, th, st = lgf_or_fix(self.handle, theta_tol, max_sweeps, omega, check_every)
        return n, F, th, st == LGF_OK

    def set_trace(self, cap: int, flags: bool = False):
        """Record F and theta of every measurement of the next fix(); returns the (F, theta) arrays, or
        with flags=True (F, theta, trace flags, sampled link defect)."""
        if cap <= 0:
            lgf_set_trace(self.handle, 0, 0, 0)
            self._trace = None
            return None
        Fh = np.zeros(cap)
        Th = np.zeros(cap)
        if flags:
            Fl = np.zeros(cap, dtype=np.int32)
            Dh = np.zeros(cap)
            lgf_set_trace_ex(self.handle, Fh.ctypes.data, Th.ctypes.data, Fl.ctypes.data, Dh.ctypes.data, cap)
            self._trace = (Fh, Th, Fl, Dh)
        else:
            lgf_set_trace(self.handle, Fh.ctypes.data, Th.ctypes.data, cap)
            self._trace = (Fh, Th)
        return self._trace

    def set_defect_bound(self, bound_fp64: float = 1e-10, bound_fp32: float = 1e-4) -> None:
        lgf_set_defect_bound(self.handle, bound_fp64, bound_fp32)

    def link_defect(self) -> tuple[float, int]:
        """(sampled link defect of the last measurement, reunitarisations in the last fix)."""
        return lgf_get_link_defect(self.handle)

    def fft4(self, data: np.ndarray, sign: int = -1) -> np.ndarray:
        """The library's 4D DFT of 4 complex fields, shape (4, Lt, Lz, Ly, Lx), host arrays."""
        lx, ly, lz, lt = self.extents
        a = _host_buffer(data, (4, lt, lz, ly, lx)).copy()
        lgf_fft4(self.handle, a.ctypes.data, 4, sign, LGF_HOST)
        return a

    def set_switch_theta(self, theta: float) -> None:
        """Theta below which a mixed-precision fix switches to FP64 (1e-10 ... 1e-6)."""
        _check(self.handle, load_library().lgf_set_switch_theta(ctypes.c_void_p(self.handle), float(theta)),
               "lgf_set_switch_theta")

    def set_fft_decomposition(self, decomposition: str) -> None:
        """Decomposition of the 4D transform of every following step: "2d2d" (default), "1d4" or "3d1d"."""
        code = {"2d2d": LGF_FFT_2D2D, "1d4": LGF_FFT_1D4, "3d1d": LGF_FFT_3D1D}[decomposition]
        _check(self.handle, load_library().lgf_set_fft_decomposition(ctypes.c_void_p(self.handle), code),
               "lgf_set_fft_decomposition")

    def set_fused_update(self, enable: bool) -> None:
        """FP32 phase: update and measurement as one kernel (default) or as two."""
        _check(self.handle, load_library().lgf_set_fused_update(ctypes.c_void_p(self.handle), int(bool(enable))),
               "lgf_set_fused_update")

    def autotune(self) -> dict:
        """Time every tile plan and decomposition of the transform, keep the fastest; returns the report."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _check(self.handle, load_library().lgf_autotune(ctypes.c_void_p(self.handle), buf, len(buf)),
               "lgf_autotune")
        return json.loads(buf.value.decode())

    def set_timing(self, enable: bool = True) -> None:
        lgf_set_timing(self.handle, enable)

    def get_timing(self) -> tuple[list[float], int]:
        """Mean ms per step of [pass A, pass B, pass C+g, update, measure] and the step count
        (for 1D x 4 / 3D + 1D: forward passes, filter pass, inverse passes + g; a fused FP32
        update + measurement is reported under update)."""
        return lgf_get_timing(self.handle)

    def load_preconditioner(self, weights_bf16) -> None:
        """weights_bf16: uint16 numpy array (host) or CUDA tensor (int16/uint16/bfloat16) of 8961 values."""
        if _is_torch_cuda(weights_bf16):
            lgf_load_preconditioner(self.handle, weights_bf16.data_ptr(), LGF_MLP_NPARAM, LGF_DEVICE)
        else:
            w = np.ascontiguousarray(weights_bf16, dtype=np.uint16)
            if w.size != LGF_MLP_NPARAM:
                raise ValueError(f"expected {LGF_MLP_NPARAM} BF16 parameters")
            lgf_load_preconditioner(self.handle, w.ctypes.data, LGF_MLP_NPARAM, LGF_HOST)

    def fallbacks(self) -> int:
        return lgf_get_fallbacks(self.handle)

    def set_mode_log(self, enable: bool = True) -> None:
        lgf_set_mode_log(self.handle, enable)

    def get_mode_log(self) -> np.ndarray:
        """Sums [bucket][class][5] = (Re<D^_{k+1}, D^_k>, |D^_k|^2, count, iter_frac, rate)."""
        out = np.zeros((MLP_NBUCKET, self.nclass, MLP_NSTAT))
        lgf_get_mode_log(self.handle, out.ctypes.data, out.size)
        return out

    @property
    def phase(self) -> int:
        return lgf_get_phase(self.handle)
