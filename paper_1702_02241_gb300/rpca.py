"""Thin ctypes binding of librpca.so (include/rpca.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  Device buffers may be passed as integers (raw device pointers) or as torch CUDA
tensors (their ``data_ptr()`` is used; the caller keeps them alive).  Matrices are
column-major: a torch tensor of shape (n, m), contiguous, holds an m x n column-major matrix.

If the shared library is missing this module raises at load time; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librpca.so")

RPCA_OK, RPCA_EINVAL, RPCA_ENOMEM, RPCA_ECUDA = 0, -1, -2, -3
RPCA_ENOTCONV, RPCA_ETIMEOUT, RPCA_EUNSUPPORTED = -4, -5, -6
STATUS_NAMES = {0: "RPCA_OK", -1: "RPCA_EINVAL", -2: "RPCA_ENOMEM", -3: "RPCA_ECUDA", -4: "RPCA_ENOTCONV",
                -5: "RPCA_ETIMEOUT", -6: "RPCA_EUNSUPPORTED"}
RPCA_F32, RPCA_BF16, RPCA_FP8E4M3 = 0, 1, 2
RPCA_INIT_SKETCH, RPCA_INIT_RANDOM, RPCA_INIT_LEARNED, RPCA_INIT_USER = 0, 1, 2, 3


class rpca_options(C.Structure):
    _fields_ = [("lbfgs_mem", C.c_int), ("max_iter", C.c_int), ("cert_tol", C.c_double),
                ("cert_every", C.c_int), ("init", C.c_int), ("seed", C.c_uint64), ("x_dtype", C.c_int),
                ("refine_fp32", C.c_int), ("timeout_s", C.c_double), ("gtol", C.c_double),
                ("sketch_oversample", C.c_int), ("sketch_power", C.c_int), ("ls_noise", C.c_double),
                ("autotune", C.c_int)]


class rpca_cert(C.Structure):
    _fields_ = [("cert", C.c_double), ("cert_rel", C.c_double), ("t1", C.c_double), ("t2", C.c_double),
                ("t3", C.c_double), ("t4", C.c_double), ("normL_F", C.c_double), ("F", C.c_double),
                ("F_bound", C.c_double), ("gap_bound", C.c_double), ("rank_r", C.c_int),
                ("krylov_steps", C.c_int), ("sigma1_perp", C.c_double), ("F_trunc", C.c_double),
                ("trunc_rel", C.c_double)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}

    def certified(self, tol):
        return self.cert_rel <= tol and self.trunc_rel <= tol


class rpca_fw_result(C.Structure):
    _fields_ = [("F", C.c_double), ("t", C.c_double), ("gap", C.c_double), ("sigma1", C.c_double),
                ("iters", C.c_int), ("seconds", C.c_double)]


class rpca_convex_result(C.Structure):
    _fields_ = [("F", C.c_double), ("phi", C.c_double), ("nuclear", C.c_double), ("rel_change", C.c_double),
                ("iters", C.c_int), ("rank", C.c_int), ("truncated", C.c_int), ("seconds", C.c_double),
                ("ms_pass", C.c_double), ("ms_rsvd", C.c_double), ("ms_tsqr", C.c_double),
                ("ms_recon", C.c_double)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rpca_aicc_result(C.Structure):
    _fields_ = [("aicc", C.c_double), ("loglik", C.c_double), ("dof", C.c_double), ("rank", C.c_int),
                ("nuclear", C.c_double), ("s_l1", C.c_double), ("nnz_s", C.c_int64), ("resid2", C.c_double),
                ("x2", C.c_double), ("count", C.c_int64)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rpca_result(C.Structure):
    _fields_ = [("F", C.c_double), ("iters", C.c_int), ("evals", C.c_int), ("cert_evals", C.c_int),
                ("seconds", C.c_double), ("cert", rpca_cert), ("status", C.c_int), ("ms_init", C.c_double),
                ("ms_iter", C.c_double), ("ms_cert", C.c_double), ("init_used", C.c_int)]


_lib = None


def lib():
    """Load librpca.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1702_02241_gb300.build` "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    L.rpca_default_options.argtypes = [C.POINTER(rpca_options)]
    L.rpca_default_options.restype = None
    L.rpca_create.argtypes = [C.POINTER(P), I64, I64, P, I64, P, I64, I, D, D, C.POINTER(rpca_options), P]
    L.rpca_create.restype = I
    L.rpca_fg.argtypes = [P, P, P, C.POINTER(C.c_double), P, P]
    L.rpca_fg.restype = I
    L.rpca_apply.argtypes = [P, P, P, I, P, P, P, P]
    L.rpca_apply.restype = I
    L.rpca_init_sketch.argtypes = [P, P, P, P]
    L.rpca_init_sketch.restype = I
    L.rpca_solve.argtypes = [P, P, P, C.POINTER(rpca_result)]
    L.rpca_solve.restype = I
    L.rpca_certificate.argtypes = [P, P, P, C.POINTER(rpca_cert)]
    L.rpca_certificate.restype = I
    L.rpca_destroy.argtypes = [P]
    L.rpca_destroy.restype = None
    L.rpca_release_memory.argtypes = []
    L.rpca_release_memory.restype = C.c_size_t
    L.rpca_last_error.argtypes = [P]
    L.rpca_last_error.restype = C.c_char_p
    L.rpca_plan_info.argtypes = [P, I, C.POINTER(C.c_int64)]
    L.rpca_plan_info.restype = I
    L.rpca_plan_kernel.argtypes = [P, I, C.POINTER(C.c_int64)]
    L.rpca_plan_kernel.restype = I
    L.rpca_profile.argtypes = [P, I]
    L.rpca_profile.restype = I
    L.rpca_profile_read.argtypes = [P, C.POINTER(C.c_double)]
    L.rpca_profile_read.restype = I
    L.rpca_solve_log.argtypes = [P, C.POINTER(C.c_double), I, C.POINTER(C.c_int)]
    L.rpca_solve_log.restype = I
    L.rpca_solve_trials.argtypes = [P, C.POINTER(C.c_double), I, C.POINTER(C.c_int)]
    L.rpca_solve_trials.restype = I
    L.rpca_x_storage.argtypes = [P, C.POINTER(C.c_int), C.c_void_p, C.c_int64, C.c_void_p]
    L.rpca_x_storage.restype = I
    L.rpca_create_batch.argtypes = [C.POINTER(P), I, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(rpca_options), P]
    L.rpca_create_batch.restype = I
    L.rpca_solve_batch.argtypes = [P, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(rpca_result)]
    L.rpca_solve_batch.restype = I
    L.rpca_batch_context.argtypes = [P, I]
    L.rpca_batch_context.restype = P
    L.rpca_batch_size.argtypes = [P]
    L.rpca_batch_size.restype = I
    L.rpca_batch_driver.argtypes = [P]
    L.rpca_batch_driver.restype = I
    L.rpca_batch_last_error.argtypes = [P]
    L.rpca_batch_last_error.restype = C.c_char_p
    L.rpca_destroy_batch.argtypes = [P]
    L.rpca_destroy_batch.restype = None
    L.rpca_fg_noalloc.argtypes = [I64, I64, P, I64, I, D, D, P, P, C.POINTER(C.c_double), P, P, P]
    L.rpca_fg_noalloc.restype = I
    L.rpca_version.argtypes = []
    L.rpca_version.restype = C.c_char_p
    L.rpca_perp_direction.argtypes = [P, P, P, C.POINTER(C.c_double)]
    L.rpca_perp_direction.restype = I
    L.rpca_perp_directions.argtypes = [P, I, P, I64, P, I64, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.rpca_perp_directions.restype = I
    L.rpca_aicc.argtypes = [P, P, P, C.POINTER(rpca_aicc_result)]
    L.rpca_aicc.restype = I
    L.rpca_fw_solve.argtypes = [P, P, I64, I, D, I, C.POINTER(C.c_double), C.POINTER(rpca_fw_result)]
    L.rpca_fw_solve.restype = I
    L.rpca_tsqr.argtypes = [P, P, I64, I64, I, P, I64, P]
    L.rpca_tsqr.restype = I
    L.rpca_convex_solve.argtypes = [P, P, I64, I, I, P, I, D, I, C.POINTER(C.c_double),
                                    C.POINTER(rpca_convex_result)]
    L.rpca_convex_solve.restype = I
    L.rpca_solve_grow.argtypes = [P, P, P, I, C.POINTER(rpca_result), C.POINTER(C.c_int)]
    L.rpca_solve_grow.restype = I
    FP = C.POINTER(C.c_float)
    L.rpca_ws_nparam.argtypes = []
    L.rpca_ws_nparam.restype = I
    L.rpca_ws_create.argtypes = [C.POINTER(P), FP, P]
    L.rpca_ws_create.restype = I
    L.rpca_ws_set_params.argtypes = [P, FP]
    L.rpca_ws_set_params.restype = I
    L.rpca_ws_get_params.argtypes = [P, FP, FP]
    L.rpca_ws_get_params.restype = I
    L.rpca_ws_predict.argtypes = [P, P, I, P]
    L.rpca_ws_predict.restype = I
    L.rpca_ws_train_step.argtypes = [P, P, P, P, I, C.c_float, FP]
    L.rpca_ws_train_step.restype = I
    L.rpca_ws_last_error.argtypes = [P]
    L.rpca_ws_last_error.restype = C.c_char_p
    L.rpca_ws_destroy.argtypes = [P]
    L.rpca_ws_destroy.restype = None
    L.rpca_set_warm_start.argtypes = [P, P]
    L.rpca_set_warm_start.restype = I
    L.rpca_sketch_spectrum.argtypes = [P, FP, C.POINTER(C.c_int)]
    L.rpca_sketch_spectrum.restype = I
    L.rpca_ws_sample.argtypes = [P, P, P, P, P, P, P]
    L.rpca_ws_sample.restype = I
    L.rpca_gen_planted.argtypes = [I64, I64, I, D, D, C.c_uint64, C.c_uint32, P, I64, P, P]
    L.rpca_gen_planted.restype = I
    L.rpca_philox4x32_10.argtypes = [P, I64, C.POINTER(C.c_uint32), C.c_uint64, P]
    L.rpca_philox4x32_10.restype = I
    L.rpca_fg_rows.argtypes = [P, P, P, C.POINTER(C.c_double), P, P]
    L.rpca_fg_rows.restype = I
    L.rpca_fg_rows_finish.argtypes = [P, P, P, D, C.POINTER(C.c_double), P]
    L.rpca_fg_rows_finish.restype = I
    L.rpca_inject_fault.argtypes = [P, I, I]
    L.rpca_inject_fault.restype = I
    _lib = L
    return L


EXPORTED = ["rpca_default_options", "rpca_create", "rpca_fg", "rpca_apply", "rpca_init_sketch", "rpca_solve",
            "rpca_certificate", "rpca_destroy", "rpca_release_memory", "rpca_last_error", "rpca_version", "rpca_plan_info", "rpca_plan_kernel",
            "rpca_profile", "rpca_profile_read", "rpca_solve_log", "rpca_solve_trials", "rpca_x_storage", "rpca_fg_noalloc", "rpca_create_batch",
            "rpca_solve_batch", "rpca_batch_context", "rpca_batch_size", "rpca_batch_driver", "rpca_batch_last_error",
            "rpca_destroy_batch", "rpca_ws_nparam", "rpca_ws_create", "rpca_ws_set_params", "rpca_ws_get_params",
            "rpca_ws_predict", "rpca_ws_train_step", "rpca_ws_last_error", "rpca_ws_destroy",
            "rpca_set_warm_start", "rpca_sketch_spectrum", "rpca_ws_sample", "rpca_gen_planted",
            "rpca_philox4x32_10", "rpca_perp_direction", "rpca_perp_directions",
            "rpca_solve_grow", "rpca_fw_solve", "rpca_aicc", "rpca_tsqr", "rpca_convex_solve",
            "rpca_inject_fault", "rpca_fg_rows", "rpca_fg_rows_finish"]


class RpcaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(st, ctx):
    if st != RPCA_OK:
        raise RpcaError(st, rpca_last_error(ctx))
    return st


def rpca_default_options() -> rpca_options:
    o = rpca_options()
    lib().rpca_default_options(C.byref(o))
    return o


def rpca_last_error(ctx=None) -> str:
    r = lib().rpca_last_error(ctx)
    return r.decode() if r else ""


def rpca_version() -> str:
    return lib().rpca_version().decode()


def rpca_create(m, n, X, ldx, mask, ldmask, k, lam_L, lam_S, opt=None, stream=None):
    """Returns an opaque context handle (int).  X / mask: device pointers or torch tensors."""
    h = C.c_void_p()
    st = lib().rpca_create(C.byref(h), m, n, _ptr(X), ldx, _ptr(mask), ldmask, k, float(lam_L),
                           float(lam_S) if not math.isinf(lam_S) else float("inf"),
                           C.byref(opt) if opt is not None else None, stream)
    _check(st, None)
    return h.value


def rpca_fg(ctx, U, V, gU, gV, want_f=True):
    f = C.c_double(float("nan"))
    st = lib().rpca_fg(ctx, _ptr(U), _ptr(V), C.byref(f) if want_f else None, _ptr(gU), _ptr(gV))
    _check(st, ctx)
    return f.value


def rpca_fg_rows(ctx, U, V, gU, PV, want_f=True):
    """This row shard's terms of F and the gradient; returns f_part (see include/rpca.h)."""
    f = C.c_double(float("nan"))
    _check(lib().rpca_fg_rows(ctx, _ptr(U), _ptr(V), C.byref(f) if want_f else None, _ptr(gU), _ptr(PV)), ctx)
    return f.value


def rpca_fg_rows_finish(ctx, V, PV_sum, f_sum, gV):
    """gV = PV_sum + lam_L V; returns f = f_sum + lam_L/2 ||V||^2."""
    f = C.c_double(float("nan"))
    _check(lib().rpca_fg_rows_finish(ctx, _ptr(V), _ptr(PV_sum), float(f_sum), C.byref(f), _ptr(gV)), ctx)
    return f.value


RPCA_FAULT_FG_STARVE, RPCA_FAULT_ALLOC = 1, 2


def rpca_inject_fault(ctx, kind, count):
    """Failure injection for tests (see include/rpca.h): starve the next fused launches of
    ctx, or fail the next device allocations of context set-up."""
    _check(lib().rpca_inject_fault(ctx, kind, count), ctx)


def rpca_fg_noalloc(m, n, X, ldx, k, lam_L, lam_S, U, V, gU, gV, stream=None):
    """Evaluation without a context and without allocation; returns f."""
    f = C.c_double(float("nan"))
    st = lib().rpca_fg_noalloc(m, n, _ptr(X), ldx, k, float(lam_L), float(lam_S), _ptr(U), _ptr(V), C.byref(f),
                               _ptr(gU), _ptr(gV), stream)
    _check(st, None)
    return f.value


def rpca_apply(ctx, U, V, b, Bv, Bu, DBv, DtBu):
    _check(lib().rpca_apply(ctx, _ptr(U), _ptr(V), b, _ptr(Bv), _ptr(Bu), _ptr(DBv), _ptr(DtBu)), ctx)


def rpca_init_sketch(ctx, Omega, U, V):
    _check(lib().rpca_init_sketch(ctx, _ptr(Omega), _ptr(U), _ptr(V)), ctx)


def rpca_solve(ctx, U, V, check=True) -> rpca_result:
    res = rpca_result()
    st = lib().rpca_solve(ctx, _ptr(U), _ptr(V), C.byref(res))
    if check and st not in (RPCA_OK, RPCA_ENOTCONV):
        _check(st, ctx)
    res.status = st
    return res


def rpca_certificate(ctx, U, V) -> rpca_cert:
    out = rpca_cert()
    _check(lib().rpca_certificate(ctx, _ptr(U), _ptr(V), C.byref(out)), ctx)
    return out


def rpca_plan_info(ctx, which=0) -> dict:
    out = (C.c_int64 * 9)()
    _check(lib().rpca_plan_info(ctx, which, out), ctx)
    keys = ["R", "warps", "row_blocks", "col_splits", "cols_per_cta", "threads", "smem", "ctas_per_sm", "stages"]
    return dict(zip(keys, list(out)))


def rpca_plan_kernel(ctx, which=0) -> dict:
    out = (C.c_int64 * 2)()
    _check(lib().rpca_plan_kernel(ctx, which, out), ctx)
    return {"kernel": {0: "cuda-core", 1: "tensor-core", 2: "gemm", 3: "tcgen05"}[int(out[0])], "npass": int(out[1])}


def rpca_profile(ctx, enable=True):
    _check(lib().rpca_profile(ctx, 1 if enable else 0), ctx)


def rpca_profile_read(ctx) -> dict:
    out = (C.c_double * 6)()
    _check(lib().rpca_profile_read(ctx, out), ctx)
    keys = ["fg_launches", "fg_ms", "finalize_launches", "finalize_ms", "kernel_launches", "graph_launches"]
    return dict(zip(keys, list(out)))


def rpca_solve_log(ctx, max_rows=256):
    """Rows {iteration, F, ||grad||, step, trials, outcome, pairs} of the last solve."""
    out = (C.c_double * (7 * max_rows))()
    rows = C.c_int(0)
    _check(lib().rpca_solve_log(ctx, out, max_rows, C.byref(rows)), ctx)
    return [list(out[7 * i:7 * i + 7]) for i in range(rows.value)]


def rpca_solve_trials(ctx, max_rows=256):
    """Rows {iteration, a, f(a) - f(0), phi'(a)/|phi'(0)|, ||g(a)||^2, phase, trial} of the last solve."""
    out = (C.c_double * (7 * max_rows))()
    rows = C.c_int(0)
    _check(lib().rpca_solve_trials(ctx, out, max_rows, C.byref(rows)), ctx)
    return [list(out[7 * i:7 * i + 7]) for i in range(rows.value)]


def rpca_x_storage(ctx, m, n):
    """(dtype, stored elements as a numpy (m, n) array of uint16/uint8 or None, scales or None)."""
    import numpy as np
    dt = C.c_int(0)
    _check(lib().rpca_x_storage(ctx, C.byref(dt), None, 0, None), ctx)
    if dt.value == RPCA_F32:
        return dt.value, None, None
    buf = np.zeros((n, m), np.uint16 if dt.value == RPCA_BF16 else np.uint8)
    sc = np.zeros(n, np.float32)
    _check(lib().rpca_x_storage(ctx, C.byref(dt), buf.ctypes.data_as(C.c_void_p), m,
                                sc.ctypes.data_as(C.c_void_p) if dt.value == RPCA_FP8E4M3 else None), ctx)
    return dt.value, buf.T, (sc if dt.value == RPCA_FP8E4M3 else None)


def rpca_create_batch(Xs, lds, ks, lam_Ls, lam_Ss, opt=None, stream=None):
    """Xs: device tensors (n_i, ld_i) holding column-major m_i x n_i X_i; returns the batch handle."""
    cnt = len(Xs)
    ms = (C.c_int64 * cnt)(*[int(m) for m, _ in lds])
    ns = (C.c_int64 * cnt)(*[int(X.shape[0]) for X in Xs])
    ldx = (C.c_int64 * cnt)(*[int(ld) for _, ld in lds])
    ptr = (C.c_void_p * cnt)(*[X.data_ptr() for X in Xs])
    kk = (C.c_int * cnt)(*[int(k) for k in ks])
    lL = (C.c_double * cnt)(*[float(v) for v in lam_Ls])
    lS = (C.c_double * cnt)(*[float(v) for v in lam_Ss])
    out = C.c_void_p()
    st = lib().rpca_create_batch(C.byref(out), cnt, ms, ns, ptr, ldx, kk, lL, lS,
                                 C.byref(opt) if opt is not None else None, stream)
    if st != RPCA_OK:
        raise RpcaError(st, lib().rpca_batch_last_error(None).decode())
    return out


def rpca_solve_batch(b, Us, Vs):
    """Solves the batch; Us, Vs: device (k_i, m_i) / (k_i, n_i) tensors.  Returns (status, results)."""
    cnt = len(Us)
    pu = (C.c_void_p * cnt)(*[U.data_ptr() for U in Us])
    pv = (C.c_void_p * cnt)(*[V.data_ptr() for V in Vs])
    res = (rpca_result * cnt)()
    st = lib().rpca_solve_batch(b, pu, pv, res)
    if st not in (RPCA_OK, RPCA_ENOTCONV):
        raise RpcaError(st, lib().rpca_batch_last_error(b).decode())
    return st, list(res)


def rpca_batch_context(b, i):
    """Instance i's context (owned by the batch)."""
    return lib().rpca_batch_context(b, i)


def rpca_batch_size(b):
    return lib().rpca_batch_size(b)


RPCA_DRIVER_THREADS, RPCA_DRIVER_ROUNDS, RPCA_DRIVER_GROUPED = 0, 1, 2


def rpca_batch_driver(b):
    """The driver of the batch's last solve (RPCA_DRIVER_*), -1 before the first."""
    return lib().rpca_batch_driver(b)


def rpca_batch_last_error(b=None):
    return lib().rpca_batch_last_error(b).decode()


def rpca_destroy_batch(b):
    lib().rpca_destroy_batch(b)


def rpca_destroy(ctx):
    lib().rpca_destroy(ctx)


def rpca_release_memory() -> int:
    """Returns the memory the library keeps from destroyed contexts; the bytes released."""
    return int(lib().rpca_release_memory())


# ---- Learned warm start -------------------------------------------------------------------


class WsError(RuntimeError):
    pass


def _ws_check(st, w):
    if st != RPCA_OK:
        raise RpcaError(st, rpca_ws_last_error(w))
    return st


def _floats(a, n):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} floats, got {a.size}")
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def rpca_ws_nparam():
    return lib().rpca_ws_nparam()


def rpca_ws_create(theta, stream=None):
    """A model from the packed float32 parameters theta (host array)."""
    keep, ptr = _floats(theta, rpca_ws_nparam())
    w = C.c_void_p()
    _ws_check(lib().rpca_ws_create(C.byref(w), ptr, stream), None)
    return w.value


def rpca_ws_set_params(w, theta):
    keep, ptr = _floats(theta, rpca_ws_nparam())
    _ws_check(lib().rpca_ws_set_params(w, ptr), w)


def rpca_ws_get_params(w):
    """(theta, grad of the last training step) as host float32 arrays."""
    import numpy as np
    n = rpca_ws_nparam()
    th = np.zeros(n, np.float32)
    gr = np.zeros(n, np.float32)
    _ws_check(lib().rpca_ws_get_params(w, th.ctypes.data_as(C.POINTER(C.c_float)),
                                       gr.ctypes.data_as(C.POINTER(C.c_float))), w)
    return th, gr


def rpca_ws_predict(w, X, B, W):
    _ws_check(lib().rpca_ws_predict(w, _ptr(X), B, _ptr(W)), w)


def rpca_ws_train_step(w, X, T, K, B, lr, want_loss=True):
    """One Adam step; returns the batch loss before the step (None unless want_loss: reading
    it synchronises)."""
    loss = C.c_float(0.0)
    _ws_check(lib().rpca_ws_train_step(w, _ptr(X), _ptr(T), _ptr(K), B, lr,
                                       C.byref(loss) if want_loss else None), w)
    return loss.value if want_loss else None


def offset(T, elements):
    """Device address of element `elements` of a contiguous torch tensor (no copy)."""
    return T.data_ptr() + elements * T.element_size()


def rpca_ws_last_error(w):
    return lib().rpca_ws_last_error(w).decode()


def rpca_ws_destroy(w):
    lib().rpca_ws_destroy(w)


def rpca_set_warm_start(ctx, w):
    _check(lib().rpca_set_warm_start(ctx, w), ctx)


def rpca_sketch_spectrum(ctx):
    import numpy as np
    s = np.zeros(32, np.float32)
    l = C.c_int(0)
    _check(lib().rpca_sketch_spectrum(ctx, s.ctypes.data_as(C.POINTER(C.c_float)), C.byref(l)), ctx)
    return s[:l.value].copy()


def rpca_ws_sample(ctx, Us, Vs, U, V, x, wstar):
    _check(lib().rpca_ws_sample(ctx, _ptr(Us), _ptr(Vs), _ptr(U), _ptr(V), _ptr(x), _ptr(wstar)), ctx)


def rpca_gen_planted(m, n, rank, p_outlier, noise_std, seed, instance, X, ldx, L0=None, stream=None):
    _check(lib().rpca_gen_planted(m, n, rank, p_outlier, noise_std, seed, instance, _ptr(X), ldx, _ptr(L0),
                                  stream), None)


def rpca_philox4x32_10(out, count, ctr, key, stream=None):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    _check(lib().rpca_philox4x32_10(_ptr(out), count, c, key, stream), None)


def rpca_perp_direction(ctx, u, v):
    """Writes the unit top singular pair of P_U1perp D P_V1perp (last full certificate) into the
    device buffers u (m) and v (n); returns sigma_1."""
    s1 = C.c_double(0.0)
    _check(lib().rpca_perp_direction(ctx, _ptr(u), _ptr(v), C.byref(s1)), ctx)
    return s1.value


def rpca_solve_grow(ctx, U, V, kmax):
    """Solve with dynamic rank increase; U, V: device (kmax, m) / (kmax, n) tensors.  Returns
    (result, final rank)."""
    r = rpca_result()
    k = C.c_int(0)
    st = lib().rpca_solve_grow(ctx, _ptr(U), _ptr(V), kmax, C.byref(r), C.byref(k))
    if st not in (RPCA_OK, RPCA_ENOTCONV):
        raise RpcaError(st, rpca_last_error(ctx))
    return r, k.value


def rpca_perp_directions(ctx, qmax, U, ldu, V, ldv):
    """The leading pairs of P_U1perp D P_V1perp into device buffers; returns the singular values."""
    sig = (C.c_double * 16)()
    q = C.c_int(0)
    _check(lib().rpca_perp_directions(ctx, qmax, _ptr(U), ldu, _ptr(V), ldv, sig, C.byref(q)), ctx)
    return list(sig)[:q.value]


def rpca_fw_solve(ctx, L, ldl, max_iter, gap_tol=0.0, power_iters=2, want_log=True):
    """Frank-Wolfe with marginalization on the dense device iterate L (torch (n, ldl)).
    Returns (rpca_fw_result, log rows [F, gap, sigma_1, eta] or None)."""
    r = rpca_fw_result()
    log = (C.c_double * (4 * max(1, max_iter)))() if want_log else None
    _check(lib().rpca_fw_solve(ctx, _ptr(L), ldl, max_iter, gap_tol, power_iters, log, C.byref(r)), ctx)
    rows = [list(log[4 * i:4 * i + 4]) for i in range(r.iters)] if want_log else None
    return r, rows


def rpca_tsqr(ctx, A, lda, rows, l, Q, ldq, R=None):
    """TSQR of the device matrix A (rows x l) into Q (rows x l) and R (l x l, or None)."""
    _check(lib().rpca_tsqr(ctx, _ptr(A), lda, rows, l, _ptr(Q), ldq, _ptr(R) if R is not None else None), ctx)


def rpca_convex_solve(ctx, L, ldl, l, Omega0, max_iter, tol=0.0, power_iters=1, profile=False, want_log=True):
    """The Sec. 6.1 convex baseline (FISTA with a TSQR-based rSVD prox) into the device iterate L.
    Returns (rpca_convex_result, log rows [F, rel_change, rank, s_l] for k = 0..iters, or None)."""
    r = rpca_convex_result()
    log = (C.c_double * (4 * (max_iter + 1)))() if want_log else None
    _check(lib().rpca_convex_solve(ctx, _ptr(L), ldl, l, power_iters, _ptr(Omega0), max_iter, tol,
                                   1 if profile else 0, log, C.byref(r)), ctx)
    rows = [list(log[4 * i:4 * i + 4]) for i in range(r.iters + 1)] if want_log else None
    return r, rows


def rpca_aicc(ctx, U, V):
    """AIC_c of the solution (U, V) (device factors); returns an rpca_aicc_result."""
    r = rpca_aicc_result()
    _check(lib().rpca_aicc(ctx, _ptr(U), _ptr(V), C.byref(r)), ctx)
    return r
