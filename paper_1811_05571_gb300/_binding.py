"""ctypes binding of libadmm.so: one Python function per C-ABI entry point.

Argument marshalling only: buffers (torch tensors, numpy arrays or raw
integer addresses) become pointers, sizes become int64, the stream becomes a
cudaStream_t.  Every numerical step runs inside the CUDA library; nothing here
computes.  A non-zero status raises ``AdmmError`` carrying the library's
message.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

ADMM_OK, ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA, ADMM_ENOTPD = 0, 1, 2, 3, 4
ADMM_ENONFINITE, ADMM_ETIMEOUT, ADMM_EUNSUPPORTED, ADMM_EDIVERGED = 5, 6, 7, 8
ADMM_C64, ADMM_C128 = 0, 1
ADMM_OPT_TIMEOUT_NS, ADMM_OPT_HIST_CAP, ADMM_OPT_BARRIER_EXTRA, ADMM_OPT_TRACE_ITERS = 1, 2, 3, 4
ADMM_OPT_L2_KEEP_BYTES, ADMM_OPT_H_FP16, ADMM_OPT_L2_PREFETCH_BYTES, ADMM_OPT_RECORD_ITERS = 5, 6, 7, 8
ADMM_OPT_DIR_FACTOR_PASS = 9
ADMM_FORM_LEMMA, ADMM_FORM_DIRECT, ADMM_FORM_AUTO = 0, 1, 2
ABI_VERSION = 5


class AdmmInfo(ctypes.Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("ld", c_int64),
                ("row_blocks", c_int32), ("col_blocks", c_int32),
                ("lambda_", c_double), ("rho", c_double), ("kappa", c_double),
                ("iterations", c_int64), ("ctas", c_int32), ("rows_per_stage", c_int32),
                ("stages", c_int32), ("slab_cols", c_int32), ("smem_bytes", c_int32),
                ("num_sms", c_int32), ("h_bytes", c_int64), ("factor_bytes", c_int64),
                ("state_bytes", c_int64), ("setup_gram_ms", c_double),
                ("setup_factor_ms", c_double), ("h_fp16", c_int32), ("h16_ready", c_int32),
                ("h16_bytes", c_int64), ("l2_keep_bytes", c_int64), ("factor_form", c_int32),
                ("reserved", c_int32)]

    def as_dict(self) -> dict:
        return {name.rstrip("_"): getattr(self, name) for name, _ in self._fields_}


class AdmmPlan(ctypes.Structure):
    _fields_ = [("ctas", c_int32), ("slab_cols", c_int32), ("chunks", c_int32),
                ("box_cols", c_int32), ("boxes_per_row", c_int32), ("rows_per_stage", c_int32),
                ("stages", c_int32), ("smem_bytes", c_int32), ("max_blocks_per_slab", c_int32),
                ("ld", c_int64), ("groups", c_int32), ("reserved", c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class AdmmBatchInfo(ctypes.Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("batch", c_int32), ("row_blocks", c_int32),
                ("col_blocks", c_int32), ("splits", c_int32), ("iterations", c_int64),
                ("tensor_flops", c_double), ("method_flops", c_double), ("state_bytes", c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class AdmmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


# name -> (restype, argtypes)
SIGNATURES = {
    "admm_abi_version": (c_int32, []),
    "admm_strerror": (ctypes.c_char_p, [c_int32]),
    "admm_last_error": (ctypes.c_char_p, [c_void_p]),
    "admm_partition": (c_int32, [c_int64, c_int32, ctypes.POINTER(c_int64)]),
    "admm_comm_elements": (c_int32, [c_int64, c_int64, c_int32, c_int32, ctypes.POINTER(c_double)]),
    "admm_plan": (c_int32, [c_int64, c_int64, c_int32, c_int32, c_int32, c_int32,
                            ctypes.POINTER(AdmmPlan), ctypes.POINTER(c_int32)]),
    "admm_setup": (c_int32, [ctypes.POINTER(c_void_p), c_void_p, c_void_p, c_int64, c_int64,
                             c_int32, c_int32, c_double, c_double, c_int32, c_void_p]),
    "admm_setup_form": (c_int32, [ctypes.POINTER(c_void_p), c_void_p, c_void_p, c_int64, c_int64,
                                  c_int32, c_int32, c_double, c_double, c_int32, c_int32, c_void_p]),
    "admm_iterate": (c_int32, [c_void_p, c_int32, c_void_p]),
    "admm_solve": (c_int32, [c_void_p, c_int32, c_double, c_double, ctypes.POINTER(c_int32),
                             c_void_p]),
    "admm_get_v": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_get_u": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_get_residuals": (c_int32, [c_void_p, ctypes.POINTER(c_double), c_int32,
                                     ctypes.POINTER(c_int32), c_void_p]),
    "admm_set_g": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "admm_set_lambda": (c_int32, [c_void_p, c_double]),
    "admm_set_rho": (c_int32, [c_void_p, c_double, c_void_p]),
    "admm_reset": (c_int32, [c_void_p, c_void_p]),
    "admm_get_state": (c_int32, [c_void_p, ctypes.POINTER(c_int64), c_void_p, c_void_p, c_void_p,
                                 c_void_p]),
    "admm_set_state": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "admm_get_info": (c_int32, [c_void_p, ctypes.POINTER(AdmmInfo)]),
    "admm_set_option": (c_int32, [c_void_p, c_int32, c_int64]),
    "admm_get_trace": (c_int32, [c_void_p, ctypes.POINTER(c_int64), c_int32,
                                 ctypes.POINTER(c_int32), c_void_p]),
    "admm_status": (c_int32, [c_void_p, c_void_p]),
    "admm_tune": (c_int32, [c_void_p, c_void_p]),
    "admm_group_setup": (c_int32, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_int32, c_void_p]),
    "admm_group_iterate": (c_int32, [c_void_p, c_int32, c_void_p]),
    "admm_group_info": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32), c_int32]),
    "admm_group_launches": (c_int32, [c_void_p]),
    "admm_group_uses_graph": (c_int32, [c_void_p]),
    "admm_group_last_error": (ctypes.c_char_p, [c_void_p]),
    "admm_group_destroy": (None, [c_void_p]),
    "admm_backward": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                c_void_p]),
    "admm_destroy": (None, [c_void_p]),
    "admm_shard_enable": (c_int32, [c_void_p, c_int32, c_void_p]),
    "admm_shard_ghat_sum": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_shard_set_exchange": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_shard_ustep": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_shard_vstep": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(c_double), c_void_p]),
    "admm_solve_small_noalloc": (c_int32, [c_void_p, c_void_p, c_int64, c_int64, c_int32, c_int32,
                                           c_double, c_double, c_int32, c_void_p, c_void_p]),
    "admm_batch_setup": (c_int32, [ctypes.POINTER(c_void_p), c_void_p, c_int64, c_int64, c_int32, c_int32,
                                   c_int32, ctypes.POINTER(c_double), c_double, c_int32, c_void_p]),
    "admm_batch_set_g": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_batch_iterate": (c_int32, [c_void_p, c_int32, c_void_p]),
    "admm_batch_get_v": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "admm_batch_get_residuals": (c_int32, [c_void_p, ctypes.POINTER(c_double), c_void_p]),
    "admm_batch_reset": (c_int32, [c_void_p, c_void_p]),
    "admm_batch_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "admm_batch_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "admm_batch_status": (c_int32, [c_void_p, c_void_p]),
    "admm_batch_record": (c_int32, [c_void_p, c_int32]),
    "admm_batch_set_lambda": (c_int32, [c_void_p, ctypes.POINTER(c_double)]),
    "admm_batch_set_rho": (c_int32, [c_void_p, c_double, c_void_p]),
    "admm_batch_tune": (c_int32, [c_void_p, c_void_p]),
    "admm_batch_backward": (c_int32, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                                      ctypes.POINTER(c_double), c_void_p]),
    "admm_batch_get_info": (c_int32, [c_void_p, ctypes.POINTER(AdmmBatchInfo)]),
    "admm_batch_last_error": (ctypes.c_char_p, [c_void_p]),
    "admm_batch_destroy": (None, [c_void_p]),
}

_LIB = None


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load the in-tree libadmm.so (building it first when a source changed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libadmm.so is missing at {_build.LIB}; run paper_1811_05571_gb300.build")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def library_path() -> str:
    return _build.LIB


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x) -> int | None:
    """Address of a buffer: torch tensor / numpy array (contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):           # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):             # numpy.ndarray
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)            # torch.cuda.Stream


def _check(status: int, handle=None) -> None:
    if status != ADMM_OK:
        lib = load(False)
        msg = lib.admm_last_error(handle)
        raise AdmmError(status, (msg or lib.admm_strerror(status)).decode())


# ---------------------------------------------------------------------------
# one function per entry point
# ---------------------------------------------------------------------------

def admm_abi_version() -> int:
    return load().admm_abi_version()


def admm_strerror(status: int) -> str:
    return load().admm_strerror(status).decode()


def admm_comm_elements(m: int, n: int, row_blocks: int, col_blocks: int) -> dict:
    out = (c_double * 3)()
    _check(load().admm_comm_elements(m, n, row_blocks, col_blocks, out))
    return {"consensus": out[0], "sectioning": out[1], "cs": out[2]}


def admm_partition(total: int, parts: int) -> list[int]:
    off = (c_int64 * (parts + 1))()
    _check(load().admm_partition(total, parts, off))
    return list(off)


def admm_plan(m: int, n: int, row_blocks: int, col_blocks: int, num_sms: int = 152,
              smem_limit: int = 232448):
    """Plan of the iteration kernel and, per CTA, (slab begin, slab end, first
    owned column, one past the last owned column)."""
    plan = AdmmPlan()
    cols = (c_int32 * (4 * num_sms))()
    _check(load().admm_plan(m, n, row_blocks, col_blocks, num_sms, smem_limit, ctypes.byref(plan),
                            cols))
    flat = list(cols)[: 4 * plan.ctas]
    return plan.as_dict(), [tuple(flat[4 * c: 4 * c + 4]) for c in range(plan.ctas)]


def admm_setup(H, g, m: int, n: int, row_blocks: int, col_blocks: int, lam: float, rho: float,
               h_dtype: int = ADMM_C64, stream=None) -> int:
    h = c_void_p()
    _check(load().admm_setup(ctypes.byref(h), _ptr(H), _ptr(g), m, n, row_blocks, col_blocks,
                             lam, rho, h_dtype, _stream(stream)))
    return h.value


def admm_setup_form(H, g, m: int, n: int, row_blocks: int, col_blocks: int, lam: float, rho: float,
                    h_dtype: int = ADMM_C64, form: int = ADMM_FORM_LEMMA, stream=None) -> int:
    h = c_void_p()
    _check(load().admm_setup_form(ctypes.byref(h), _ptr(H), _ptr(g), m, n, row_blocks, col_blocks,
                                  lam, rho, h_dtype, form, _stream(stream)))
    return h.value


def admm_iterate(h: int, iters: int, stream=None) -> None:
    _check(load().admm_iterate(h, iters, _stream(stream)), h)


def admm_solve(h: int, max_iter: int, eps_abs: float, eps_rel: float, stream=None) -> int:
    done = c_int32(0)
    _check(load().admm_solve(h, max_iter, eps_abs, eps_rel, ctypes.byref(done), _stream(stream)), h)
    return done.value


def admm_get_v(h: int, v, stream=None) -> None:
    _check(load().admm_get_v(h, _ptr(v), _stream(stream)), h)


def admm_get_u(h: int, u, stream=None) -> None:
    _check(load().admm_get_u(h, _ptr(u), _stream(stream)), h)


def admm_get_residuals(h: int, cap: int, stream=None):
    import numpy as np
    out = np.zeros((max(cap, 1), 5), dtype=np.float64)
    count = c_int32(0)
    _check(load().admm_get_residuals(h, out.ctypes.data_as(ctypes.POINTER(c_double)), cap,
                                     ctypes.byref(count), _stream(stream)), h)
    return out[: count.value]


def admm_set_g(h: int, g, h_dtype: int = ADMM_C64, stream=None) -> None:
    _check(load().admm_set_g(h, _ptr(g), h_dtype, _stream(stream)), h)


def admm_set_lambda(h: int, lam: float) -> None:
    _check(load().admm_set_lambda(h, lam), h)


def admm_set_rho(h: int, rho: float, stream=None) -> None:
    _check(load().admm_set_rho(h, rho, _stream(stream)), h)


def admm_reset(h: int, stream=None) -> None:
    _check(load().admm_reset(h, _stream(stream)), h)


def admm_get_state(h: int, v=None, s=None, ghat=None, stream=None) -> int:
    k = c_int64(0)
    _check(load().admm_get_state(h, ctypes.byref(k), _ptr(v), _ptr(s), _ptr(ghat),
                                 _stream(stream)), h)
    return k.value


def admm_set_state(h: int, k: int, v, s, ghat=None, stream=None) -> None:
    _check(load().admm_set_state(h, k, _ptr(v), _ptr(s), _ptr(ghat), _stream(stream)), h)


def admm_get_info(h: int) -> dict:
    info = AdmmInfo()
    _check(load().admm_get_info(h, ctypes.byref(info)), h)
    return info.as_dict()


def admm_set_option(h: int, option: int, value: int) -> None:
    _check(load().admm_set_option(h, option, value), h)


def admm_get_trace(h: int, cap: int, stream=None):
    """(2, k, 8) int64 phase stamps of CTA 0 and the last CTA (see include/admm.h)."""
    import numpy as np
    out = np.zeros((2, max(cap, 1), 8), dtype=np.int64)
    count = c_int32(0)
    _check(load().admm_get_trace(h, out.ctypes.data_as(ctypes.POINTER(c_int64)), cap,
                                 ctypes.byref(count), _stream(stream)), h)
    k = count.value
    flat = out.reshape(-1)[: 2 * k * 8]
    return flat.reshape(2, k, 8)


def admm_status(h: int, stream=None) -> int:
    return load().admm_status(h, _stream(stream))


def admm_destroy(h: int) -> None:
    if h:
        load().admm_destroy(h)


def admm_shard_enable(h: int, row_blocks_total: int, stream=None) -> None:
    _check(load().admm_shard_enable(h, row_blocks_total, _stream(stream)), h)


def admm_shard_ghat_sum(h: int, t_local, stream=None) -> None:
    _check(load().admm_shard_ghat_sum(h, _ptr(t_local), _stream(stream)), h)


def admm_shard_set_exchange(h: int, t_global, stream=None) -> None:
    _check(load().admm_shard_set_exchange(h, _ptr(t_global), _stream(stream)), h)


def admm_shard_ustep(h: int, sum_out, stream=None) -> None:
    _check(load().admm_shard_ustep(h, _ptr(sum_out), _stream(stream)), h)


def admm_shard_vstep(h: int, sum_global, stream=None):
    import numpy as np
    rec = (c_double * 5)()
    _check(load().admm_shard_vstep(h, _ptr(sum_global), rec, _stream(stream)), h)
    return np.array(rec[:], dtype=np.float64)


def admm_solve_small_noalloc(H, g, m: int, n: int, row_blocks: int, col_blocks: int, lam: float,
                             rho: float, iters: int, v_out, stream=None) -> None:
    """Allocation-free solve of a small problem into the caller's v_out (see include/admm.h).

    H, g and v_out must be CUDA tensors: the call uses them in place."""
    import torch
    for name, t in (("H", H), ("g", g), ("v_out", v_out)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise TypeError(f"admm_solve_small_noalloc: {name} must be a CUDA tensor")
    _check(load().admm_solve_small_noalloc(_ptr(H), _ptr(g), m, n, row_blocks, col_blocks, lam, rho,
                                           iters, _ptr(v_out), _stream(stream)))


# ---------------------------------------------------------------------------
# batched shared-H solver
# ---------------------------------------------------------------------------

def _bcheck(status: int, handle=None) -> None:
    if status != ADMM_OK:
        lib = load(False)
        msg = lib.admm_batch_last_error(handle)
        raise AdmmError(status, (msg or lib.admm_strerror(status)).decode())


def admm_batch_setup(H, m: int, n: int, row_blocks: int, col_blocks: int, batch: int, lam, rho: float,
                     dtype: int, stream=None) -> int:
    out = c_void_p()
    lam = [float(x) for x in lam]
    lam_arr = (c_double * max(1, len(lam)))(*lam)
    _bcheck(load().admm_batch_setup(ctypes.byref(out), _ptr(H), m, n, row_blocks, col_blocks, batch, lam_arr,
                                    rho, dtype, _stream(stream)))
    return out.value


def admm_batch_set_g(h: int, G, stream=None) -> None:
    _bcheck(load().admm_batch_set_g(h, _ptr(G), _stream(stream)), h)


def admm_batch_iterate(h: int, iters: int, stream=None) -> None:
    _bcheck(load().admm_batch_iterate(h, iters, _stream(stream)), h)


def admm_batch_get_v(h: int, V, stream=None) -> None:
    _bcheck(load().admm_batch_get_v(h, _ptr(V), _stream(stream)), h)


def admm_batch_get_residuals(h: int, batch: int, stream=None):
    import numpy as np
    out = (c_double * (2 * batch))()
    _bcheck(load().admm_batch_get_residuals(h, out, _stream(stream)), h)
    return np.array(out[:], dtype=np.float64).reshape(batch, 2)


def admm_batch_reset(h: int, stream=None) -> None:
    _bcheck(load().admm_batch_reset(h, _stream(stream)), h)


def admm_batch_forward(h: int, X, Y, stream=None) -> None:
    _bcheck(load().admm_batch_forward(h, _ptr(X), _ptr(Y), _stream(stream)), h)


def admm_batch_adjoint(h: int, Y, X, stream=None) -> None:
    _bcheck(load().admm_batch_adjoint(h, _ptr(Y), _ptr(X), _stream(stream)), h)


def admm_batch_status(h: int, stream=None) -> int:
    return load().admm_batch_status(h, _stream(stream))


def admm_batch_get_info(h: int) -> dict:
    info = AdmmBatchInfo()
    _bcheck(load().admm_batch_get_info(h, ctypes.byref(info)), h)
    return info.as_dict()


def admm_batch_destroy(h: int) -> None:
    if h:
        load().admm_batch_destroy(h)


def admm_batch_record(h: int, iters: int) -> None:
    _bcheck(load().admm_batch_record(h, iters), h)


def admm_batch_set_lambda(h: int, lam) -> None:
    arr = (c_double * len(lam))(*[float(x) for x in lam])
    _bcheck(load().admm_batch_set_lambda(h, arr), h)


def admm_batch_set_rho(h: int, rho: float, stream=None) -> None:
    _bcheck(load().admm_batch_set_rho(h, float(rho), _stream(stream)), h)


def admm_batch_backward(h: int, batch: int, dV, dG, stream=None):
    import numpy as np
    dl = (c_double * batch)()
    dr = (c_double * batch)()
    _bcheck(load().admm_batch_backward(h, _ptr(dV), _ptr(dG), dl, dr, _stream(stream)), h)
    return np.array(dl[:]), np.array(dr[:])


def admm_batch_tune(h: int, stream=None) -> None:
    _bcheck(load().admm_batch_tune(h, _stream(stream)), h)


def admm_tune(h: int, stream=None) -> None:
    _check(load().admm_tune(h, _stream(stream)), h)


def admm_backward(h: int, grad_v, grad_g, stream=None):
    gl, gr = c_double(), c_double()
    _check(load().admm_backward(h, _ptr(grad_v), _ptr(grad_g), ctypes.byref(gl), ctypes.byref(gr),
                                _stream(stream)), h)
    return gl.value, gr.value


def _gcheck(status: int, handle=None) -> None:
    if status != ADMM_OK:
        lib = load(False)
        msg = lib.admm_group_last_error(handle)
        raise AdmmError(status, (msg or lib.admm_strerror(status)).decode())


def admm_group_setup(handles, stream=None) -> int:
    out = c_void_p()
    arr = (c_void_p * len(handles))(*handles)
    _gcheck(load().admm_group_setup(ctypes.byref(out), arr, len(handles), _stream(stream)))
    return out.value


def admm_group_iterate(g: int, iters: int, stream=None) -> None:
    _gcheck(load().admm_group_iterate(g, iters, _stream(stream)), g)


def admm_group_info(g: int, count: int):
    waves = c_int32()
    ctas = (c_int32 * max(1, count))()
    _gcheck(load().admm_group_info(g, ctypes.byref(waves), ctas, count), g)
    return waves.value, list(ctas[:count])


def admm_group_launches(g: int) -> int:
    return int(load().admm_group_launches(g))


def admm_group_uses_graph(g: int) -> int:
    return int(load().admm_group_uses_graph(g))


def admm_group_destroy(g: int) -> None:
    if g:
        load().admm_group_destroy(g)

