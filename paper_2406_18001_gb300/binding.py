"""ctypes binding of libdcd_gb300.so (include/dcd_gb300.h).

Argument marshalling only: every step of the solvers runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library cannot be built or
loaded, every call raises.  Device arrays are torch CUDA tensors; host arrays
(DCD_FLAG_HOST_IO) are numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- enums ---
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTCONV, EINTERNAL, ENOTSPD, EUNSUPPORTED = range(9)
DENSE, CSR = 0, 1
F64, F32, BF16, FP8E4M3 = 0, 1, 2, 3
LINEAR, POLY, RBF = 0, 1, 2
PREC_FP64, PREC_TF32, PREC_BF16, PREC_FP8, PREC_BF16X3, PREC_TF32X3, PREC_REFRESH, PREC_FP16 = 0, 1, 2, 3, 4, 5, 6, 7
FLAG_GRAD_VALID, FLAG_HOST_IO, FLAG_PHASE_TIMERS, FLAG_NO_GRAPH, FLAG_REFRESH = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_LITERAL = 0x20
FLAG_CSR_FULL_PASS = 0x40
FLAG_NO_DEFER = 0x80

PREC_NAMES = {"fp64": PREC_FP64, "tf32": PREC_TF32, "bf16": PREC_BF16, "fp8": PREC_FP8, "bf16x3": PREC_BF16X3,
              "tf32x3": PREC_TF32X3, "refresh": PREC_REFRESH, "fp16": PREC_FP16}


class Matrix(C.Structure):
    _fields_ = [("fmt", C.c_int32), ("dtype", C.c_int32), ("m", C.c_int64), ("n", C.c_int64), ("ld", C.c_int64),
                ("values", C.c_void_p), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("row_scale", C.c_void_p)]


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("degree", C.c_int32), ("gamma", C.c_double), ("coef0", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("s", C.c_int32), ("b", C.c_int32), ("max_iters", C.c_int64), ("seed", C.c_uint64),
                ("start_iter", C.c_uint64), ("tol", C.c_double), ("check_every", C.c_int32),
                ("prec", C.c_int32), ("flags", C.c_int32), ("reserved", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters_done", C.c_int64), ("outer_steps", C.c_int64), ("converged", C.c_int32),
                ("gpu_launches_per_step", C.c_int32), ("final_metric", C.c_double), ("primal", C.c_double),
                ("dual", C.c_double), ("ms_total", C.c_double), ("ms_setup", C.c_double),
                ("ms_sample", C.c_double), ("ms_gram", C.c_double), ("ms_recur", C.c_double),
                ("ms_block", C.c_double), ("ms_update", C.c_double), ("ms_check", C.c_double),
                ("refreshes", C.c_int64), ("ms_refresh", C.c_double), ("s_used", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KrrProblem(C.Structure):
    _fields_ = [("A", Matrix), ("y", C.c_void_p), ("k", Kernel), ("lam", C.c_double), ("b", C.c_int32),
                ("s", C.c_int32), ("max_iters", C.c_int64), ("seed", C.c_uint64), ("alpha", C.c_void_p),
                ("grad", C.c_void_p)]


class BatchOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("streams", C.c_int32), ("rounds_per_graph", C.c_int32),
                ("check_every", C.c_int32), ("tol", C.c_double), ("flags", C.c_int32), ("reserved", C.c_int32)]


EXPORTS = ["dcd_svm_solve", "bdcd_krr_solve", "bdcd_krr_solve_batched", "dcd_krr_autotune_s",
           "dcd_svm_plan_create", "bdcd_krr_plan_create", "dcd_plan_run",
           "dcd_plan_enqueue", "dcd_plan_destroy", "dcd_status_string", "dcd_sample_indices", "dcd_kernel_block",
           "dcd_kernel_block_apply", "dcd_kernel_block_static", "dcd_quantize_e4m3", "dcd_selftest_bounded_wait",
           "dcd_inject_alloc_failures", "dcd_shard_contribute", "dcd_shard_assemble", "dcd_bdcd_recurrence",
           "dcd_dcd_recurrence", "dcd_kernel_block_apply_points", "dcd_shard_update"]

_lock = threading.Lock()
_lib = None


class DcdError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}")


def lib():
    """Load (building first if needed) the CUDA library.  Raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        try:  # make sure the CUDA runtime PyTorch uses is the one resolved
            import torch  # noqa: F401
        except Exception:
            pass
        L = C.CDLL(path)
        P, i32, i64, u64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        M, K, O, S = C.POINTER(Matrix), C.POINTER(Kernel), C.POINTER(Opts), C.POINTER(Stats)
        sigs = {
            "dcd_svm_solve": (i32, [M, P, K, i32, d, O, P, P, S, P]),
            "bdcd_krr_solve": (i32, [M, P, K, d, O, P, P, S, P]),
            "dcd_svm_plan_create": (i32, [M, P, K, i32, d, O, P, P, P, C.POINTER(C.c_void_p)]),
            "bdcd_krr_plan_create": (i32, [M, P, K, d, O, P, P, P, C.POINTER(C.c_void_p)]),
            "dcd_plan_run": (i32, [P, i64, S]),
            "dcd_plan_enqueue": (i32, [P, i64, C.POINTER(C.c_int64)]),
            "bdcd_krr_solve_batched": (i32, [C.POINTER(KrrProblem), i32, C.POINTER(BatchOpts), S, P]),
            "dcd_krr_autotune_s": (i32, [M, P, K, d, i32, i32, C.POINTER(C.c_int32), P]),
            "dcd_plan_destroy": (i32, [P]),
            "dcd_status_string": (C.c_char_p, [i32]),
            "dcd_sample_indices": (i32, [i32, u64, i64, i32, u64, i64, P, P]),
            "dcd_kernel_block": (i32, [M, K, i32, P, i64, P, i64, P, i64, P]),
            "dcd_kernel_block_apply": (i32, [M, K, i32, P, i64, P, P, P, P]),
            "dcd_kernel_block_static": (i32, [M, K, i32, P, i64, P, i64, P, i64, P]),
            "dcd_quantize_e4m3": (i32, [M, P, i64, P, P]),
            "dcd_selftest_bounded_wait": (i32, [i64, P]),
            "dcd_inject_alloc_failures": (i32, [i32]),
            "dcd_shard_contribute": (i32, [M, i64, i64, P, i64, P, P, P, P, P]),
            "dcd_shard_assemble": (i32, [P, i32, P, i64, i64, P, P, P, P, P, P]),
            "dcd_bdcd_recurrence": (i32, [P, i32, i64, P, i64, i32, d, d, P, P, P, P]),
            "dcd_dcd_recurrence": (i32, [P, i32, i64, P, i64, P, P, P, i32, d, P, P, P]),
            "dcd_kernel_block_apply_points": (i32, [M, i64, M, P, K, i32, P, P, P, P]),
            "dcd_shard_update": (i32, [P, P, i64, d, i64, i64, P, P, P]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def status_string(s: int) -> str:
    return lib().dcd_status_string(int(s)).decode()


def kernel(kind, gamma=1.0, coef0=0.0, degree=2) -> Kernel:
    if isinstance(kind, str):
        kind = {"linear": LINEAR, "poly": POLY, "rbf": RBF}[kind]
    return Kernel(int(kind), int(degree), float(gamma), float(coef0))


def _prec(p):
    return PREC_NAMES[p] if isinstance(p, str) else int(p)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class Csr:
    """A CSR matrix for the library: int64 row_ptr[m+1], int32 col_idx[nnz],
    float32 / float64 values (torch tensors on one device, or numpy arrays
    with DCD_FLAG_HOST_IO)."""

    def __init__(self, row_ptr, col_idx, values, n):
        self.row_ptr, self.col_idx, self.values, self.n = row_ptr, col_idx, values, int(n)
        self.m = int(row_ptr.shape[0]) - 1

    @property
    def shape(self):
        return (self.m, self.n)

    @property
    def device(self):
        return self.values.device

    def matrix(self) -> Matrix:
        import numpy as _np
        v = self.values
        if isinstance(v, _np.ndarray):
            dt = {_np.dtype(_np.float64): F64, _np.dtype(_np.float32): F32}[v.dtype]
        else:
            import torch
            dt = {torch.float64: F64, torch.float32: F32}[v.dtype]
        return Matrix(CSR, dt, self.m, self.n, 0, _ptr(v), _ptr(self.row_ptr), _ptr(self.col_idx), None)


class Fp8:
    """FP8 storage of a dense matrix: e4m3 codes (uint8, m x n row-major, a
    torch tensor on the device or a numpy array with DCD_FLAG_HOST_IO) and
    one float32 scale per row; row i stands for scale[i] * value(codes[i])."""

    def __init__(self, codes, scale):
        self.codes, self.scale = codes, scale
        if codes.shape[0] != scale.shape[0]:
            raise ValueError("one scale per row")

    @property
    def shape(self):
        return tuple(self.codes.shape)

    @property
    def device(self):
        return self.codes.device

    def matrix(self) -> Matrix:
        q = self.codes
        if isinstance(q, np.ndarray):
            assert q.dtype == np.uint8 and q.flags.c_contiguous and self.scale.dtype == np.float32
            ld = q.shape[1]
        else:
            import torch
            assert q.dtype == torch.uint8 and q.dim() == 2 and q.stride(1) == 1
            assert self.scale.dtype == torch.float32 and self.scale.is_contiguous()
            ld = q.stride(0)
        return Matrix(DENSE, FP8E4M3, q.shape[0], q.shape[1], ld, _ptr(q), None, None, _ptr(self.scale))


def quantize_e4m3(A, stream=None) -> Fp8:
    """Per-row FP8 storage of a dense device matrix (dcd_quantize_e4m3)."""
    import torch
    m, n = A.shape
    q = torch.empty((m, n), dtype=torch.uint8, device=A.device)
    sc = torch.empty(m, dtype=torch.float32, device=A.device)
    Am = dense_matrix(A)
    _check(lib().dcd_quantize_e4m3(C.byref(Am), _ptr(q), n, _ptr(sc), _stream(stream)), "dcd_quantize_e4m3",
           allow_notconv=False)
    return Fp8(q, sc)


def dense_matrix(A) -> Matrix:
    """Describe a row-major 2-D torch tensor (device) or numpy array (host),
    a Csr or an Fp8."""
    if isinstance(A, (Csr, Fp8)):
        return A.matrix()
    if isinstance(A, np.ndarray):
        dt = {np.dtype(np.float64): F64, np.dtype(np.float32): F32}[A.dtype]
        assert A.flags.c_contiguous
        return Matrix(DENSE, dt, A.shape[0], A.shape[1], A.shape[1], A.ctypes.data, None, None, None)
    import torch
    dt = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[A.dtype]
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major tensor")
    return Matrix(DENSE, dt, A.shape[0], A.shape[1], A.stride(0), A.data_ptr(), None, None, None)


def _opts(s, b, H, seed, start_iter, tol, check_every, prec, flags):
    return Opts(int(s), int(b), int(H), int(seed) & (2**64 - 1), int(start_iter), float(tol), int(check_every),
                _prec(prec), int(flags), 0)


def _check(rc, what, allow_notconv=True):
    if rc == OK or (allow_notconv and rc == ENOTCONV):
        return rc
    raise DcdError(rc, what)


def svm_solve(A, y, k, loss, C_, s, H, seed=0, prec="fp64", alpha=None, grad=None, tol=0.0, check_every=0,
              start_iter=0, flags=0, stream=None):
    """s-step DCD for K-SVM (Algorithm 2).  A, y, alpha, grad on the device
    (torch) or, with FLAG_HOST_IO, on the host (numpy).  alpha is updated in
    place (alpha_0 -> alpha_H); returns (alpha, grad, stats, status)."""
    host = bool(flags & FLAG_HOST_IO)
    m = A.shape[0]
    if alpha is None:
        alpha = np.zeros(m) if host else _zeros(m, A)
    if grad is None:
        grad = np.empty(m) if host else _empty(m, A)
    Am = dense_matrix(A)
    o = _opts(s, 1, H, seed, start_iter, tol, check_every, prec, flags)
    st = Stats()
    rc = lib().dcd_svm_solve(C.byref(Am), _ptr(y), C.byref(k), int(loss), float(C_), C.byref(o), _ptr(alpha),
                             _ptr(grad), C.byref(st), None if host and stream is None else _stream(stream))
    _check(rc, "dcd_svm_solve")
    return alpha, grad, st.as_dict(), rc


def krr_solve(A, y, k, lam, b, s, H, seed=0, prec="fp64", alpha=None, grad=None, tol=0.0, check_every=0,
              start_iter=0, flags=0, stream=None):
    """s-step BDCD for K-RR (Algorithm 4); same conventions as svm_solve."""
    host = bool(flags & FLAG_HOST_IO)
    m = A.shape[0]
    if alpha is None:
        alpha = np.zeros(m) if host else _zeros(m, A)
    if grad is None:
        grad = np.empty(m) if host else _empty(m, A)
    Am = dense_matrix(A)
    o = _opts(s, b, H, seed, start_iter, tol, check_every, prec, flags)
    st = Stats()
    rc = lib().bdcd_krr_solve(C.byref(Am), _ptr(y), C.byref(k), float(lam), C.byref(o), _ptr(alpha), _ptr(grad),
                              C.byref(st), None if host and stream is None else _stream(stream))
    _check(rc, "bdcd_krr_solve")
    return alpha, grad, st.as_dict(), rc


class Plan:
    """A persistent solve (dcd_*_plan_create / dcd_plan_run / dcd_plan_destroy).

    Keeps references to the arrays it was created with, which the library
    reads and updates until close()."""

    def __init__(self, problem, A, y, k, param, b, s, H, seed=0, prec="fp64", alpha=None, grad=None, tol=0.0,
                 check_every=0, start_iter=0, flags=0, stream=None, loss=1):
        host = bool(flags & FLAG_HOST_IO)
        m = A.shape[0]
        self.A, self.y = A, y
        self.alpha = alpha if alpha is not None else (np.zeros(m) if host else _zeros(m, A))
        self.grad = grad if grad is not None else (np.empty(m) if host else _empty(m, A))
        self._Am = dense_matrix(A)
        self._k = k
        self._o = _opts(s, b if problem == 1 else 1, H, seed, start_iter, tol, check_every, prec, flags)
        self._h = C.c_void_p()
        strm = None if host and stream is None else _stream(stream)
        if problem == 0:
            rc = lib().dcd_svm_plan_create(C.byref(self._Am), _ptr(y), C.byref(k), int(loss), float(param),
                                           C.byref(self._o), _ptr(self.alpha), _ptr(self.grad), strm,
                                           C.byref(self._h))
        else:
            rc = lib().bdcd_krr_plan_create(C.byref(self._Am), _ptr(y), C.byref(k), float(param), C.byref(self._o),
                                            _ptr(self.alpha), _ptr(self.grad), strm, C.byref(self._h))
        _check(rc, "plan_create", allow_notconv=False)

    def run(self, max_outer_steps=-1):
        st = Stats()
        rc = lib().dcd_plan_run(self._h, int(max_outer_steps), C.byref(st))
        _check(rc, "dcd_plan_run")
        return st.as_dict(), rc

    def enqueue(self, outer_steps):
        """Enqueue outer steps without synchronising; returns how many were enqueued."""
        n = C.c_int64()
        rc = lib().dcd_plan_enqueue(self._h, int(outer_steps), C.byref(n))
        _check(rc, "dcd_plan_enqueue", allow_notconv=False)
        return int(n.value)

    def close(self):
        if self._h:
            rc = lib().dcd_plan_destroy(self._h)
            self._h = C.c_void_p()
            _check(rc, "dcd_plan_destroy", allow_notconv=False)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _zeros(m, like):
    import torch
    return torch.zeros(m, dtype=torch.float64, device=like.device)


def _empty(m, like):
    import torch
    return torch.empty(m, dtype=torch.float64, device=like.device)


def sample_indices(method, seed, m, b, first, count, device="cuda"):
    import torch
    n = count * (b if method == 1 else 1)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=device)
    rc = lib().dcd_sample_indices(int(method), int(seed), int(m), int(b), int(first), int(count), _ptr(out),
                                  _stream(None))
    _check(rc, "dcd_sample_indices", allow_notconv=False)
    return out[:n]


def kernel_block(A, k, prec, cols, rows=None, nrows=None):
    import torch
    ncols = cols.numel()
    nr = rows.numel() if rows is not None else (A.shape[0] if nrows is None else nrows)
    p = _prec(prec)
    out = torch.empty((nr, ncols), dtype=torch.float64 if p == PREC_FP64 else torch.float32, device=A.device)
    Am = dense_matrix(A)
    rc = lib().dcd_kernel_block(C.byref(Am), C.byref(k), p, _ptr(rows), nr, _ptr(cols), ncols, _ptr(out), ncols,
                                _stream(None))
    _check(rc, "dcd_kernel_block", allow_notconv=False)
    return out


def kernel_block_static(A, k, prec, cols, rows=None, nrows=None, out=None):
    """dcd_kernel_block_static: the kernel block with the library's static
    scratch array instead of any device allocation (for callers that cannot
    allocate).  `out` may be given to avoid allocating it here as well."""
    import torch
    ncols = cols.numel()
    nr = rows.numel() if rows is not None else (A.shape[0] if nrows is None else nrows)
    p = _prec(prec)
    if out is None:
        out = torch.empty((nr, ncols), dtype=torch.float64 if p == PREC_FP64 else torch.float32, device=A.device)
    Am = dense_matrix(A)
    rc = lib().dcd_kernel_block_static(C.byref(Am), C.byref(k), p, _ptr(rows), nr, _ptr(cols), ncols, _ptr(out),
                                       ncols, _stream(None))
    _check(rc, "dcd_kernel_block_static", allow_notconv=False)
    return out


def kernel_block_apply(A, k, prec, cols, w, g, rowscale=None):
    Am = dense_matrix(A)
    rc = lib().dcd_kernel_block_apply(C.byref(Am), C.byref(k), _prec(prec), _ptr(cols), cols.numel(), _ptr(w),
                                      _ptr(rowscale), _ptr(g), _stream(None))
    _check(rc, "dcd_kernel_block_apply", allow_notconv=False)
    return g


def kernel_block_apply_points(A, row_id0, P, col_ids, k, prec, w, g, rowscale=None):
    """dcd_kernel_block_apply_points: g[i] += rowscale[i] sum_c K(a_i, p_c) w[c]
    with the column points the rows of P; ids row_id0 + i and col_ids[c]
    decide the own-sample rule (col_ids None: no row matches)."""
    Am, Pm = dense_matrix(A), dense_matrix(P)
    rc = lib().dcd_kernel_block_apply_points(C.byref(Am), int(row_id0), C.byref(Pm), _ptr(col_ids), C.byref(k),
                                             _prec(prec), _ptr(w), _ptr(rowscale), _ptr(g), _stream(None))
    _check(rc, "dcd_kernel_block_apply_points", allow_notconv=False)
    return g


def shard_contribute(A, row0, m, S, g, alpha, y, buf):
    """dcd_shard_contribute: this rank's contribution of the sampled rows it
    holds (rows row0 .. row0 + A.shape[0] - 1 of m) into buf (cnt x (n + 4))."""
    Am = dense_matrix(A)
    rc = lib().dcd_shard_contribute(C.byref(Am), int(row0), int(m), _ptr(S), S.numel(), _ptr(g), _ptr(alpha),
                                    _ptr(y), _ptr(buf), _stream(None))
    _check(rc, "dcd_shard_contribute", allow_notconv=False)
    return buf


def shard_assemble(bufs, nranks, S, n, A_S, g_S, alpha_S, y_S=None, first_pos=None):
    """dcd_shard_assemble: A_S, g_S, alpha_S (and y_S, first_pos) from the
    all-gathered contributions (nranks buffers one after another)."""
    rc = lib().dcd_shard_assemble(_ptr(bufs), int(nranks), _ptr(S), S.numel(), int(n), _ptr(A_S), _ptr(g_S),
                                  _ptr(alpha_S), _ptr(y_S), _ptr(first_pos), _stream(None))
    _check(rc, "dcd_shard_assemble", allow_notconv=False)


def bdcd_recurrence(Kss, S, b, lam, mdiag, g_S, delta, w=None):
    """dcd_bdcd_recurrence on a (cnt x cnt) sampled kernel block (FP64 or FP32)."""
    import torch
    f64 = 1 if Kss.dtype == torch.float64 else 0
    cnt = S.numel()
    rc = lib().dcd_bdcd_recurrence(_ptr(Kss), f64, Kss.stride(0), _ptr(S), cnt // int(b), int(b), float(lam),
                                   float(mdiag), _ptr(g_S), _ptr(delta), _ptr(w), _stream(None))
    _check(rc, "dcd_bdcd_recurrence", allow_notconv=False)


def dcd_recurrence(Kss, S, y_S, alpha_S, g_S, loss, C_, theta, w=None):
    """dcd_dcd_recurrence on a (cnt x cnt) sampled kernel block (FP64 or FP32)."""
    import torch
    f64 = 1 if Kss.dtype == torch.float64 else 0
    rc = lib().dcd_dcd_recurrence(_ptr(Kss), f64, Kss.stride(0), _ptr(S), S.numel(), _ptr(y_S), _ptr(alpha_S),
                                  _ptr(g_S), int(loss), float(C_), _ptr(theta), _ptr(w), _stream(None))
    _check(rc, "dcd_dcd_recurrence", allow_notconv=False)


def shard_update(S, delta, diag, row0, alpha, g):
    """dcd_shard_update: alpha / g update of the rows row0 .. row0 + len(alpha) - 1."""
    rc = lib().dcd_shard_update(_ptr(S), _ptr(delta), S.numel(), float(diag), int(row0), alpha.numel(), _ptr(alpha),
                                _ptr(g), _stream(None))
    _check(rc, "dcd_shard_update", allow_notconv=False)


def selftest_bounded_wait(limit_ns, stream=None):
    """dcd_selftest_bounded_wait: the status (DCD_ETIMEOUT expected), not raised."""
    return int(lib().dcd_selftest_bounded_wait(int(limit_ns), _stream(stream)))


def inject_alloc_failures(count):
    """dcd_inject_alloc_failures: the next `count` device allocations fail (DCD_ENOMEM)."""
    _check(lib().dcd_inject_alloc_failures(int(count)), "dcd_inject_alloc_failures", allow_notconv=False)


def krr_solve_batched(problems, prec="bf16x3", tol=0.0, check_every=0, streams=0, rounds_per_graph=0, flags=0,
                      stream=None):
    """Batched K-RR (bdcd_krr_solve_batched).  problems: list of dicts with
    A (device tensor or Csr), y, k (Kernel), lam, b, s (<= 0: autotuned), H,
    seed, and optional alpha / grad (device tensors; zeros / fresh if
    absent).  Returns (alphas, grads, stats list, rc)."""
    n = len(problems)
    arr = (KrrProblem * n)()
    keep = []
    alphas, grads = [], []
    for i, p in enumerate(problems):
        A = p["A"]
        m = A.shape[0]
        al = p.get("alpha")
        if al is None:
            al = _zeros(m, A)
        gr = p.get("grad")
        if gr is None:
            gr = _empty(m, A)
        alphas.append(al)
        grads.append(gr)
        keep.append((A, p["y"]))
        arr[i] = KrrProblem(dense_matrix(A), _ptr(p["y"]), p["k"], float(p["lam"]), int(p["b"]), int(p.get("s", 0)),
                            int(p["H"]), int(p.get("seed", 0)), _ptr(al), _ptr(gr))
    bo = BatchOpts(_prec(prec), int(streams), int(rounds_per_graph), int(check_every), float(tol), int(flags), 0)
    st = (Stats * n)()
    rc = lib().bdcd_krr_solve_batched(arr, n, C.byref(bo), st, _stream(stream))
    _check(rc, "bdcd_krr_solve_batched")
    return alphas, grads, [x.as_dict() for x in st], rc


def krr_autotune_s(A, y, k, lam, b, prec="bf16x3", stream=None):
    Am = dense_matrix(A)
    out = C.c_int32()
    rc = lib().dcd_krr_autotune_s(C.byref(Am), _ptr(y), C.byref(k), float(lam), int(b), _prec(prec), C.byref(out),
                                  _stream(stream))
    _check(rc, "dcd_krr_autotune_s", allow_notconv=False)
    return int(out.value)
