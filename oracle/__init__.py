"""FP64 CPU oracle for s-step DCD / BDCD (arXiv 2406.18001, Algorithms 1-4).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The arithmetic lives in ``dcd_oracle.c`` (plain C, IEEE double, no blocking);
this module compiles it with gcc on first use and marshals numpy arrays.
Parity status per routine (pins live in tests/test_oracle_pins.py):
  kernel_eval / kernel_block   pinned: scipy distances, integer poly, K_ii = 1
  sample_dcd / sample_bdcd     pinned: published SplitMix64 test vector,
                               uniformity, distinctness
  dcd_svm (Alg. 1)             pinned: closed-form 1-D box QP, brute-force
                               optimum for tiny m, KKT and duality gap -> 0
  sstep_dcd_svm (Alg. 2)       pinned: equals Alg. 1 iterates (paper Sec. 3.2)
  bdcd_krr (Alg. 3)            pinned: numpy dense solve, b = m one-step exact,
                               K = I closed form
  sstep_bdcd_krr (Alg. 4)      pinned: equals Alg. 3 iterates (paper Sec. 3.4)
  svm_objectives / gradients   pinned: linear-kernel primal from w = A^T(y*alpha)
  krr_closed_form              pinned: numpy.linalg.solve
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dcd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdcd_oracle.so")
_lock = threading.Lock()
_lib = None

LINEAR, POLY, RBF = 0, 1, 2


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("degree", C.c_int32), ("gamma", C.c_double), ("coef0", C.c_double)]


def kernel(kind, gamma=1.0, coef0=0.0, degree=2) -> Kernel:
    if isinstance(kind, str):
        kind = {"linear": LINEAR, "poly": POLY, "rbf": RBF}[kind]
    return Kernel(int(kind), int(degree), float(gamma), float(coef0))


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libdcd_oracle.so (gcc, -O2)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    d, i64, u64, i32 = C.c_double, C.c_int64, C.c_uint64, C.c_int32
    P = C.c_void_p
    K = C.POINTER(Kernel)
    sig = {
        "orc_splitmix64": (u64, [u64, u64]),
        "orc_draw": (u64, [u64, u64, u64]),
        "orc_dcd_index": (i64, [u64, i64, u64]),
        "orc_bdcd_block": (None, [u64, i64, i32, u64, P]),
        "orc_sample_dcd": (None, [u64, i64, u64, i64, P]),
        "orc_sample_bdcd": (None, [u64, i64, i32, u64, i64, P]),
        "orc_kernel_eval": (d, [K, P, P, i64]),
        "orc_kernel_block": (None, [K, P, i64, i64, i64, P, i64, P, i64, P]),
        "orc_dcd_svm": (C.c_int, [P, i64, i64, i64, P, K, i32, d, i64, u64, u64, P]),
        "orc_sstep_dcd_svm": (C.c_int, [P, i64, i64, i64, P, K, i32, d, i32, i64, u64, u64, P]),
        "orc_bdcd_krr": (C.c_int, [P, i64, i64, i64, P, K, d, i32, i64, u64, u64, P]),
        "orc_sstep_bdcd_krr": (C.c_int, [P, i64, i64, i64, P, K, d, i32, i32, i64, u64, u64, P]),
        "orc_svm_gradient": (C.c_int, [P, i64, i64, i64, P, K, i32, d, P, P]),
        "orc_svm_objectives": (C.c_int, [P, i64, i64, i64, P, K, i32, d, P, P]),
        "orc_krr_gradient": (C.c_int, [P, i64, i64, i64, P, K, d, P, P]),
        "orc_krr_objective": (d, [P, i64, i64, i64, P, K, d, P]),
        "orc_krr_closed_form": (C.c_int, [P, i64, i64, i64, P, K, d, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _K(k):
    return C.byref(k)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ------------------------------------------------------------------ RNG ---
def splitmix64(state, k) -> int:
    """Output number k >= 1 of the SplitMix64 sequence started from `state`."""
    return int(_load().orc_splitmix64(state, k))


def draw(seed, stream, ctr) -> int:
    return int(_load().orc_draw(seed, stream, ctr))


def sample_dcd(seed, m, first, count) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    _load().orc_sample_dcd(seed, m, first, count, _ptr(out))
    return out


def sample_bdcd(seed, m, b, first_block, nblocks) -> np.ndarray:
    out = np.empty(nblocks * b, dtype=np.int64)
    _load().orc_sample_bdcd(seed, m, b, first_block, nblocks, _ptr(out))
    return out.reshape(nblocks, b)


# -------------------------------------------------------------- kernels ---
def kernel_eval(k, a, b) -> float:
    a, b = _f64(a), _f64(b)
    return float(_load().orc_kernel_eval(_K(k), _ptr(a), _ptr(b), a.shape[0]))


def kernel_block(k, A, cols, rows=None) -> np.ndarray:
    A = _f64(A)
    m, n = A.shape
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = m if r is None else r.shape[0]
    out = np.empty((nr, cols.shape[0]))
    _load().orc_kernel_block(_K(k), _ptr(A), m, n, n, None if r is None else _ptr(r), nr,
                             _ptr(cols), cols.shape[0], _ptr(out))
    return out


# ----------------------------------------------------------- algorithms ---
def dcd_svm(A, y, k, loss, C_, H, seed=0, first=0, alpha0=None) -> np.ndarray:
    """Algorithm 1 (DCD for K-SVM-L1 / -L2)."""
    A, y = _f64(A), _f64(y)
    m, n = A.shape
    al = np.zeros(m) if alpha0 is None else _f64(alpha0).copy()
    _check(_load().orc_dcd_svm(_ptr(A), m, n, n, _ptr(y), _K(k), loss, C_, H, seed, first, _ptr(al)), "dcd_svm")
    return al


def sstep_dcd_svm(A, y, k, loss, C_, s, H, seed=0, first=0, alpha0=None) -> np.ndarray:
    """Algorithm 2 (s-step DCD for K-SVM)."""
    A, y = _f64(A), _f64(y)
    m, n = A.shape
    al = np.zeros(m) if alpha0 is None else _f64(alpha0).copy()
    _check(_load().orc_sstep_dcd_svm(_ptr(A), m, n, n, _ptr(y), _K(k), loss, C_, s, H, seed, first, _ptr(al)),
           "sstep_dcd_svm")
    return al


def bdcd_krr(A, y, k, lam, b, H, seed=0, first_block=0, alpha0=None) -> np.ndarray:
    """Algorithm 3 (BDCD for K-RR)."""
    A, y = _f64(A), _f64(y)
    m, n = A.shape
    al = np.zeros(m) if alpha0 is None else _f64(alpha0).copy()
    _check(_load().orc_bdcd_krr(_ptr(A), m, n, n, _ptr(y), _K(k), lam, b, H, seed, first_block, _ptr(al)),
           "bdcd_krr")
    return al


def sstep_bdcd_krr(A, y, k, lam, b, s, H, seed=0, first_block=0, alpha0=None) -> np.ndarray:
    """Algorithm 4 (s-step BDCD for K-RR)."""
    A, y = _f64(A), _f64(y)
    m, n = A.shape
    al = np.zeros(m) if alpha0 is None else _f64(alpha0).copy()
    _check(_load().orc_sstep_bdcd_krr(_ptr(A), m, n, n, _ptr(y), _K(k), lam, b, s, H, seed, first_block,
                                      _ptr(al)), "sstep_bdcd_krr")
    return al


def svm_gradient(A, y, k, loss, C_, alpha) -> np.ndarray:
    A, y, al = _f64(A), _f64(y), _f64(alpha)
    m, n = A.shape
    g = np.empty(m)
    _check(_load().orc_svm_gradient(_ptr(A), m, n, n, _ptr(y), _K(k), loss, C_, _ptr(al), _ptr(g)), "svm_gradient")
    return g


def svm_objectives(A, y, k, loss, C_, alpha) -> dict:
    A, y, al = _f64(A), _f64(y), _f64(alpha)
    m, n = A.shape
    out = np.empty(4)
    _check(_load().orc_svm_objectives(_ptr(A), m, n, n, _ptr(y), _K(k), loss, C_, _ptr(al), _ptr(out)),
           "svm_objectives")
    return {"primal": out[0], "dual": out[1], "gap": out[2], "kkt": out[3]}


def krr_gradient(A, y, k, lam, alpha) -> np.ndarray:
    A, y, al = _f64(A), _f64(y), _f64(alpha)
    m, n = A.shape
    g = np.empty(m)
    _check(_load().orc_krr_gradient(_ptr(A), m, n, n, _ptr(y), _K(k), lam, _ptr(al), _ptr(g)), "krr_gradient")
    return g


def krr_objective(A, y, k, lam, alpha) -> float:
    A, y, al = _f64(A), _f64(y), _f64(alpha)
    m, n = A.shape
    return float(_load().orc_krr_objective(_ptr(A), m, n, n, _ptr(y), _K(k), lam, _ptr(al)))


def krr_closed_form(A, y, k, lam) -> np.ndarray:
    A, y = _f64(A), _f64(y)
    m, n = A.shape
    al = np.empty(m)
    _check(_load().orc_krr_closed_form(_ptr(A), m, n, n, _ptr(y), _K(k), lam, _ptr(al)), "krr_closed_form")
    return al
