"""ctypes binding of libsymnmf (include/symnmf.h), same names as the C ABI.

Argument marshalling only: pointers may be given as integers or as torch
tensors (their ``data_ptr()``), structures mirror the C structs field by
field, and a negative status becomes a ``SymNMFError``.  Every step of the
solver runs in the library's CUDA kernels; if the library is missing this
module raises at import time instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsymnmf.so")

F32, BF16, FP8E4M3 = 0, 1, 2
ADAGRAD, RMSPROP, PIECEWISE_ADAGRAD, ROW_SVRG, BLOCK_SVRG_ADAPTGROW, ADMM = 0, 1, 2, 3, 4, 5
OK, CONVERGED = 0, 1
ERR_INVALID, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = (
    -1, -2, -3, -4, -5, -6, -7)
BUF_H, BUF_ACC, BUF_MOM, BUF_SNAPSHOT, BUF_GRAD = 0, 1, 2, 3, 4


class symnmf_hparams(C.Structure):
    _fields_ = [("method", C.c_int32), ("check_interval", C.c_int32), ("warmup", C.c_int32),
                ("snapshot_period", C.c_int32), ("block_rows", C.c_int32),
                ("reserved0", C.c_int32), ("eta", C.c_double), ("eps", C.c_double),
                ("alpha", C.c_double), ("mu", C.c_double), ("c", C.c_double),
                ("c_r", C.c_double), ("row_frac", C.c_double), ("phi0", C.c_double),
                ("tau_E", C.c_double), ("tau_g", C.c_double), ("tau_stag", C.c_double),
                ("growth_kkt_mult", C.c_double), ("seed", C.c_uint64), ("rho", C.c_double)]


class symnmf_ctrl(C.Structure):
    _fields_ = [("t", C.c_int64), ("E0", C.c_double), ("E_prev", C.c_double),
                ("phi", C.c_double), ("sumA_post", C.c_double), ("E_at_reset", C.c_double),
                ("have_prev", C.c_int32), ("stag_count", C.c_int32), ("resets", C.c_int32),
                ("resets_enabled", C.c_int32), ("cooldown", C.c_int32),
                ("converged", C.c_int32)]


class symnmf_record(C.Structure):
    _fields_ = [("t", C.c_int64), ("f", C.c_double), ("E", C.c_double), ("kkt", C.c_double),
                ("stag_ratio", C.c_double), ("phi", C.c_double), ("sumA", C.c_double),
                ("full", C.c_int32), ("check", C.c_int32), ("reset", C.c_int32),
                ("converged", C.c_int32), ("nonfinite", C.c_int32), ("reserved", C.c_int32),
                ("median_g2", C.c_double)]


class symnmf_stats(C.Structure):
    _fields_ = [("iter", C.c_int64), ("last_check", C.c_int64), ("f", C.c_double),
                ("E", C.c_double), ("kkt", C.c_double), ("stag_ratio", C.c_double),
                ("phi", C.c_double), ("converged", C.c_int32), ("resets", C.c_int32)]


class symnmf_kmeans_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("changed", C.c_int64),
                ("J", C.c_double), ("J_prev", C.c_double)]


class SymNMFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsymnmf.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "symnmf_create": [vp, i64, i32, i32, P(vp)],
        "symnmf_create_ld": [vp, i64, i64, i32, i32, P(vp)],
        "symnmf_destroy": [vp],
        "symnmf_set_stream": [vp, vp],
        "symnmf_set_tile_scales": [vp, vp, i64],
        "symnmf_set_norm": [vp, dbl],
        "symnmf_set_matrix": [vp, vp, i64, vp, i64],
        "symnmf_set_restarts": [vp, i32],
        "symnmf_get_restart_stats": [vp, i32, P(dbl), P(dbl), P(i32)],
        "symnmf_get_restart_ctrl": [vp, i32, P(i32), P(i32), P(i32), P(dbl)],
        "symnmf_solve_host": [vp, vp, i64, vp, i64, dbl, vp, P(symnmf_hparams), i32, vp,
                              P(symnmf_stats)],
        "symnmf_selftest_wait_timeout": [dbl],
        "symnmf_objective_noalloc": [vp, i64, i64, i32, vp, i64, vp, i32, dbl, vp, vp],
        "symnmf_objective_noalloc_check": [i64, i64, i32, i32, i64, i32, P(C.c_size_t)],
        "symnmf_quantize_fp8": [vp, i32, i64, i64, i64, vp, i64, vp, i64, vp, vp],
        "symnmf_get_norm": [vp, P(dbl)],
        "symnmf_set_impl": [vp, i32],
        "symnmf_get_impl": [vp, P(i32)],
        "symnmf_set_H": [vp, vp],
        "symnmf_get_H": [vp, vp],
        "symnmf_get_buffer": [vp, i32, vp],
        "symnmf_set_buffer": [vp, i32, vp],
        "symnmf_get_ctrl": [vp, P(symnmf_ctrl)],
        "symnmf_set_ctrl": [vp, P(symnmf_ctrl)],
        "symnmf_grad": [vp, vp],
        "symnmf_objective": [vp, P(dbl), P(dbl)],
        "symnmf_hparams_default": [i32, P(symnmf_hparams)],
        "symnmf_step": [vp, P(symnmf_hparams), i32, P(symnmf_stats)],
        "symnmf_spkmeans": [vp, vp, vp, i32, dbl, P(dbl), P(symnmf_kmeans_stats)],
        "symnmf_build_dependence": [vp, i64, i64, i64, i32, i32, vp, i64, vp, i64, vp, vp],
        "symnmf_batch_step": [P(vp), i32, P(symnmf_hparams), i32, P(symnmf_stats)],
        "symnmf_get_trace": [vp, P(symnmf_record), i64, P(i64)],
        "symnmf_set_profiling": [vp, i32],
        "symnmf_set_ctas": [vp, i32],
        "symnmf_get_ctas": [vp, P(i32)],
        "symnmf_batch_autotune": [P(vp), i32, P(symnmf_hparams), i32, P(i32)],
        "symnmf_get_profile": [vp, P(dbl), P(i64), P(dbl), P(i64)],
        "symnmf_state_bytes": [vp, P(C.c_size_t)],
        "symnmf_get_state": [vp, vp, C.c_size_t],
        "symnmf_set_state": [vp, vp, C.c_size_t],
        "symnmf_last_error": [vp],
        "symnmf_status_string": [i32],
        "symnmf_splitmix64": [u64, u64],
        "symnmf_sample_blocks": [u64, i64, i32, i64, i64, P(i64)],
        "symnmf_controller_check": [P(symnmf_ctrl), P(symnmf_hparams), i64, i64, dbl, dbl, dbl,
                                    dbl, P(i32), P(dbl)],
        "symnmf_window_update": [vp, vp, i64, i64, i32, vp, i64, vp, i64],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.symnmf_destroy.restype = None
    lib.symnmf_last_error.restype = C.c_char_p
    lib.symnmf_status_string.restype = C.c_char_p
    lib.symnmf_splitmix64.restype = C.c_uint64
    return lib


LIB = _load()
DECLARED = [
    "symnmf_create", "symnmf_create_ld", "symnmf_destroy", "symnmf_set_stream",
    "symnmf_set_tile_scales", "symnmf_quantize_fp8", "symnmf_set_norm", "symnmf_get_norm", "symnmf_set_impl",
    "symnmf_get_impl", "symnmf_set_H", "symnmf_get_H", "symnmf_get_buffer", "symnmf_set_buffer",
    "symnmf_get_ctrl", "symnmf_set_ctrl", "symnmf_grad", "symnmf_objective",
    "symnmf_hparams_default", "symnmf_step", "symnmf_batch_step", "symnmf_get_trace",
    "symnmf_set_profiling", "symnmf_get_profile", "symnmf_set_ctas", "symnmf_get_ctas",
    "symnmf_batch_autotune",
    "symnmf_state_bytes", "symnmf_get_state", "symnmf_set_state", "symnmf_last_error",
    "symnmf_status_string", "symnmf_splitmix64", "symnmf_sample_blocks",
    "symnmf_controller_check", "symnmf_objective_noalloc", "symnmf_objective_noalloc_check",
    "symnmf_spkmeans",
    "symnmf_build_dependence", "symnmf_set_matrix", "symnmf_set_restarts",
    "symnmf_get_restart_stats", "symnmf_selftest_wait_timeout", "symnmf_window_update",
    "symnmf_get_restart_ctrl", "symnmf_solve_host",
]

NOALLOC_SCRATCH_BYTES = 8 << 20


def noalloc_scratch_need(n, k):
    """Scratch bytes symnmf_objective_noalloc needs for n rows and rank k."""
    kp = 8 if k <= 8 else 16 if k <= 16 else 32 if k <= 32 else 64
    nt = -(-n // 128)
    return (nt * 64 + 255) // 256 * 256 + nt * kp * kp * 4


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(status, h=None):
    if status < 0:
        msg = LIB.symnmf_last_error(h).decode() if h else ""
        raise SymNMFError(status, msg or LIB.symnmf_status_string(status).decode())
    return status


def symnmf_status_string(status):
    return LIB.symnmf_status_string(status).decode()


def symnmf_last_error(h):
    return LIB.symnmf_last_error(h).decode()


def symnmf_create(S, n, k, dtype):
    h = C.c_void_p()
    _check(LIB.symnmf_create(_ptr(S), n, k, dtype, C.byref(h)))
    return h


def symnmf_create_ld(S, n, lds, k, dtype):
    h = C.c_void_p()
    _check(LIB.symnmf_create_ld(_ptr(S), n, lds, k, dtype, C.byref(h)))
    return h


def symnmf_destroy(h):
    LIB.symnmf_destroy(h)


def symnmf_set_stream(h, stream):
    """stream: a torch.cuda.Stream, an int handle, or None."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(LIB.symnmf_set_stream(h, s), h)


def symnmf_set_tile_scales(h, scales, ld_scales):
    return _check(LIB.symnmf_set_tile_scales(h, _ptr(scales), ld_scales), h)


def symnmf_quantize_fp8(src, src_dtype, rows, cols, ld_src, q, ldq, scales, ld_scales,
                        tile_sumsq=None, stream=None):
    """Per-tile power-of-two scaled E4M3 codes of src (device tensors)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(LIB.symnmf_quantize_fp8(_ptr(src), src_dtype, rows, cols, ld_src, _ptr(q), ldq,
                                          _ptr(scales), ld_scales, _ptr(tile_sumsq), s))


def symnmf_objective_noalloc(S, n, lds, dtype, scales, ld_scales, H, k, normS2, f, stream=None):
    """f (device double) = normS2 - 2 tr(H^T S H) + ||H^T H||^2 with no allocation."""
    s = getattr(stream, "cuda_stream", stream)
    st = LIB.symnmf_objective_noalloc(_ptr(S), n, lds, dtype, _ptr(scales), ld_scales, _ptr(H), k,
                                      float(normS2), _ptr(f), s)
    if st == ERR_UNSUPPORTED:
        raise SymNMFError(st, "n=%d, k=%d needs %d bytes of scratch, above the fixed %d"
                          % (n, k, noalloc_scratch_need(n, k), NOALLOC_SCRATCH_BYTES))
    return _check(st)


def symnmf_objective_noalloc_check(n, lds, dtype, have_scales, ld_scales, k):
    """(status, scratch bytes) of symnmf_objective_noalloc for these sizes,
    computed on the host without any CUDA call."""
    need = C.c_size_t()
    st = LIB.symnmf_objective_noalloc_check(n, lds, dtype, int(bool(have_scales)), ld_scales, k,
                                            C.byref(need))
    return st, need.value


def symnmf_build_dependence(Y, T, n, ldy, center, out_dtype, S, lds, scales=None, ld_scales=0,
                            normS2=None, stream=None):
    """S = |D^-1/2 Y^T Y D^-1/2| (centred columns for the correlation)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(LIB.symnmf_build_dependence(_ptr(Y), T, n, ldy, int(center), out_dtype, _ptr(S),
                                              lds, _ptr(scales), ld_scales, _ptr(normS2), s))


def symnmf_spkmeans(h, labels0, labels, max_iter, tol=1e-4, trace=True):
    """Spherical K-means (Lloyd) on the rows of S with K = the handle's k;
    labels0 / labels are device int32 tensors of n.  Returns (stats, J per
    iteration)."""
    st = symnmf_kmeans_stats()
    Jt = (C.c_double * max(1, max_iter))() if trace else None
    _check(LIB.symnmf_spkmeans(h, _ptr(labels0), _ptr(labels), max_iter, float(tol), Jt,
                               C.byref(st)), h)
    return st, (list(Jt)[:st.iters] if trace else None)


def symnmf_set_restarts(h, restarts):
    """Run the k columns of H as `restarts` independent blocks (one S stream)."""
    return _check(LIB.symnmf_set_restarts(h, restarts), h)


def symnmf_get_restart_stats(h, count):
    """Per-restart (E, kkt, converged) lists at the last check."""
    E = (C.c_double * count)()
    kkt = (C.c_double * count)()
    cv = (C.c_int32 * count)()
    _check(LIB.symnmf_get_restart_stats(h, count, E, kkt, cv), h)
    return list(E), list(kkt), list(cv)


def symnmf_get_restart_ctrl(h, count):
    """Per-restart Piecewise reset state: (resets, resets_enabled, cooldown,
    sumA_post) lists."""
    rs = (C.c_int32 * count)()
    en = (C.c_int32 * count)()
    cd = (C.c_int32 * count)()
    sp = (C.c_double * count)()
    _check(LIB.symnmf_get_restart_ctrl(h, count, rs, en, cd, sp), h)
    return list(rs), list(en), list(cd), list(sp)


def symnmf_set_matrix(h, S, lds, scales=None, ld_scales=0):
    """Rebind the handle to another S of the same n (warm start: H kept)."""
    return _check(LIB.symnmf_set_matrix(h, _ptr(S), lds, _ptr(scales), ld_scales), h)


def symnmf_window_update(h, Y, T, ldy, center, S, lds, scales=None, ld_scales=0):
    """Next rolling window in one call: build the window's dependence matrix
    into S (the handle's storage type), rebind the handle to it with H as
    the warm start and ||S||^2 from the build."""
    return _check(LIB.symnmf_window_update(h, _ptr(Y), T, ldy, int(center), _ptr(S), lds,
                                           _ptr(scales), ld_scales), h)


def symnmf_set_norm(h, normS2):
    return _check(LIB.symnmf_set_norm(h, float(normS2)), h)


def symnmf_get_norm(h):
    v = C.c_double()
    _check(LIB.symnmf_get_norm(h, C.byref(v)), h)
    return v.value


def symnmf_set_impl(h, impl):
    return _check(LIB.symnmf_set_impl(h, impl), h)


def symnmf_get_impl(h):
    v = C.c_int32()
    _check(LIB.symnmf_get_impl(h, C.byref(v)), h)
    return v.value


def symnmf_set_H(h, H):
    return _check(LIB.symnmf_set_H(h, _ptr(H)), h)


def symnmf_get_H(h, H):
    return _check(LIB.symnmf_get_H(h, _ptr(H)), h)


def symnmf_get_buffer(h, which, dst):
    return _check(LIB.symnmf_get_buffer(h, which, _ptr(dst)), h)


def symnmf_set_buffer(h, which, src):
    return _check(LIB.symnmf_set_buffer(h, which, _ptr(src)), h)


def symnmf_get_ctrl(h):
    c = symnmf_ctrl()
    _check(LIB.symnmf_get_ctrl(h, C.byref(c)), h)
    return c


def symnmf_set_ctrl(h, c):
    return _check(LIB.symnmf_set_ctrl(h, C.byref(c)), h)


def symnmf_grad(h, G):
    return _check(LIB.symnmf_grad(h, _ptr(G)), h)


def symnmf_objective(h):
    f, E = C.c_double(), C.c_double()
    _check(LIB.symnmf_objective(h, C.byref(f), C.byref(E)), h)
    return f.value, E.value


def symnmf_hparams_default(method, **overrides):
    hp = symnmf_hparams()
    _check(LIB.symnmf_hparams_default(method, C.byref(hp)))
    for k_, v in overrides.items():
        setattr(hp, k_, v)
    return hp


def symnmf_step(h, hp, iters):
    st = symnmf_stats()
    status = _check(LIB.symnmf_step(h, C.byref(hp), iters, C.byref(st)), h)
    return status, st


def symnmf_solve_host(h, S_host, lds_host, H0_host, hp, iters, H_out, scales_host=None,
                      ld_scales_host=0, normS2=float("nan")):
    """One solve from host memory (CPU tensors, pinned for asynchronous
    copies): S and H_0 in, the final H out; returns (status, stats)."""
    st = symnmf_stats()
    status = _check(LIB.symnmf_solve_host(h, _ptr(S_host), lds_host, _ptr(scales_host),
                                          ld_scales_host, normS2, _ptr(H0_host), C.byref(hp),
                                          iters, _ptr(H_out), C.byref(st)), h)
    return status, st


def symnmf_batch_step(hs, hps, iters):
    n = len(hs)
    harr = (C.c_void_p * n)(*[x.value if isinstance(x, C.c_void_p) else x for x in hs])
    parr = (symnmf_hparams * n)(*hps)
    sarr = (symnmf_stats * n)()
    status = _check(LIB.symnmf_batch_step(harr, n, parr, iters, sarr))
    return status, list(sarr)


def symnmf_get_trace(h, max_records=None):
    cnt = C.c_int64()
    _check(LIB.symnmf_get_trace(h, None, 0, C.byref(cnt)), h)
    m = cnt.value if max_records is None else min(max_records, cnt.value)
    arr = (symnmf_record * max(1, m))()
    _check(LIB.symnmf_get_trace(h, arr, m, C.byref(cnt)), h)
    return list(arr)[:m]


def symnmf_set_ctas(h, ctas):
    return _check(LIB.symnmf_set_ctas(h, ctas), h)


def symnmf_get_ctas(h):
    v = C.c_int32()
    _check(LIB.symnmf_get_ctas(h, C.byref(v)), h)
    return v.value


def symnmf_batch_autotune(hs, hps, iters):
    """Chosen CTA caps (list) after autotuning the batch (advances the solves)."""
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    hp_arr = (symnmf_hparams * len(hs))(*hps)
    out = (C.c_int32 * len(hs))()
    _check(LIB.symnmf_batch_autotune(arr, len(hs), hp_arr, iters, out))
    return list(out)


def symnmf_set_profiling(h, enable):
    return _check(LIB.symnmf_set_profiling(h, int(bool(enable))), h)


def symnmf_get_profile(h):
    """(product ms, product launches, S bytes streamed, kernels launched)."""
    ms, n, b, kl = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
    _check(LIB.symnmf_get_profile(h, C.byref(ms), C.byref(n), C.byref(b), C.byref(kl)), h)
    return ms.value, n.value, b.value, kl.value


def symnmf_state_bytes(h):
    v = C.c_size_t()
    _check(LIB.symnmf_state_bytes(h, C.byref(v)), h)
    return v.value


def symnmf_get_state(h):
    nb = symnmf_state_bytes(h)
    buf = (C.c_char * nb)()
    _check(LIB.symnmf_get_state(h, buf, nb), h)
    return bytes(buf)


def symnmf_set_state(h, blob):
    buf = (C.c_char * len(blob)).from_buffer_copy(blob)
    return _check(LIB.symnmf_set_state(h, buf, len(blob)), h)


def symnmf_splitmix64(state, index):
    return int(LIB.symnmf_splitmix64(state, index))


def symnmf_sample_blocks(seed, t, stream, nb, m):
    out = (C.c_int64 * max(1, min(m, nb)))()
    _check(LIB.symnmf_sample_blocks(seed, t, stream, nb, m, out))
    return list(out)[:min(m, nb)]


def symnmf_controller_check(ctrl, hp, n, t, E, kkt, sumA, median_g2):
    dec = (C.c_int32 * 3)()
    ratio = C.c_double()
    _check(LIB.symnmf_controller_check(C.byref(ctrl), C.byref(hp), n, t, E, kkt, sumA,
                                       median_g2, dec, C.byref(ratio)))
    return {"converged": bool(dec[0]), "reset": bool(dec[1]), "grow": bool(dec[2]),
            "stag_ratio": ratio.value}
