"""Python binding of libkot (the C ABI in include/kot.h): argument marshalling only.

Arrays are passed as raw pointers.  With the default ``host_pointers=False`` every array must be
a contiguous float64 CUDA tensor on the context's device (torch is used for device memory
only); with ``host_pointers=True`` contiguous float64 NumPy arrays (or CPU tensors) are passed
and the library copies them in and out.  Every computation happens inside libkot; if the shared
library is missing this module raises on import of ``lib()``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkot.so")

# kot_status
OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_NOT_PD, ERR_NO_CONVERGENCE, ERR_NONFINITE, \
    ERR_TIMEOUT, ERR_STATE, ERR_TOO_LARGE = range(10)
STATUS_NAMES = ["OK", "INVALID", "CUDA", "OOM", "NOT_PD", "NO_CONVERGENCE", "NONFINITE",
                "TIMEOUT", "STATE", "TOO_LARGE"]
FP64, MIXED = 0, 1


class Options(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("precision", C.c_int),
                ("host_pointers", C.c_int), ("max_iter", C.c_int), ("cg_max_iter", C.c_int),
                ("tau", C.c_double), ("kappa", C.c_double), ("alpha1", C.c_double),
                ("alpha2", C.c_double), ("beta0", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("theta0", C.c_double), ("theta_min", C.c_double),
                ("theta_max", C.c_double), ("eg_step", C.c_double), ("jitter", C.c_double),
                ("jitter_max", C.c_double), ("use_eg", C.c_int), ("record_history", C.c_int),
                ("eig_ctas", C.c_int), ("mixed_switch", C.c_double),
                ("batch_workers", C.c_int), ("eig_refine", C.c_int), ("schur_solver", C.c_int),
                ("gram_fp32", C.c_int), ("tc_min_flops", C.c_double)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("ssn_accepted", C.c_int),
                ("eg_taken", C.c_int), ("cg_total", C.c_int), ("residual", C.c_double),
                ("r1_norm", C.c_double), ("r2_norm", C.c_double), ("objective", C.c_double),
                ("ot_hat", C.c_double), ("eps", C.c_double), ("seconds", C.c_double),
                ("eig_calls", C.c_int), ("eig_sweeps", C.c_int), ("eig_refined", C.c_int),
                ("eig_refine_steps", C.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int), ("l", C.c_int), ("X", C.c_void_p),
                ("Y", C.c_void_p), ("Xf", C.c_void_p), ("Yf", C.c_void_p),
                ("sigma", C.c_double), ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("tol", C.c_double), ("gamma_out", C.c_void_p)]


EXPORTS = ["kot_default_options", "kot_create", "kot_destroy", "kot_last_error",
           "kot_build_features", "kot_set_features", "kot_get_features", "kot_residual",
           "kot_newton_direction", "kot_ssn_solve", "kot_get_history", "kot_batch_solve",
           "kot_profile", "kot_profile_read", "kot_launch_count",
           "kot_embedding_sqnorm_noalloc", "kot_dense_product", "kot_get_trace", "kot_eig_sym",
           "kot_eg_solve", "kot_potentials", "kot_profile_every", "kot_autotune", "kot_wait_probe",
           "kot_bootstrap_solve"]

KERNEL_CLASSES = ["gemm_f64", "jacobi_f64", "reserved", "embed", "pair_sums", "gram",
                  "cholesky", "gemm_tc", "eig_refine", "gemm_oz", "oz_aux", "schur_matvec"]


class KernelStats(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double), ("exec_flops", C.c_double)]

_lib = None


def lib() -> C.CDLL:
    """Load libkot.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"libkot.so not built at {LIB_PATH}; run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "kot_default_options": (i, [C.POINTER(Options)]),
        "kot_create": (i, [C.POINTER(vp), C.POINTER(Options)]),
        "kot_destroy": (i, [vp]),
        "kot_last_error": (C.c_char_p, [vp]),
        "kot_build_features": (i, [vp, i, i, vp, vp, i, vp, vp, d, d, d]),
        "kot_set_features": (i, [vp, i, vp, vp, d, vp, d, d]),
        "kot_get_features": (i, [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "kot_residual": (i, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "kot_newton_direction": (i, [vp, vp, vp, d, d, vp, vp, C.POINTER(i)]),
        "kot_ssn_solve": (i, [vp, d, vp, vp, vp, vp, C.POINTER(Result)]),
        "kot_get_history": (i, [vp, vp, i, C.POINTER(i)]),
        "kot_batch_solve": (i, [vp, i, C.POINTER(Problem), C.POINTER(Result)]),
        "kot_bootstrap_solve": (i, [vp, i, i, vp, vp, d, vp, C.POINTER(Result)]),
        "kot_profile": (i, [vp, i]),
        "kot_profile_every": (i, [vp, i]),
        "kot_autotune": (i, [vp, i, vp]),
        "kot_wait_probe": (i, [vp, C.c_longlong]),
        "kot_profile_read": (i, [vp, i, C.POINTER(KernelStats)]),
        "kot_launch_count": (i, [C.POINTER(C.c_longlong)]),
        "kot_dense_product": (i, [vp, i, i, i, d, vp, i, i, vp, i, i, d, vp, i, i]),
        "kot_get_trace": (i, [vp, vp, i, C.POINTER(i)]),
        "kot_eig_sym": (i, [vp, i, vp, vp, vp, vp, C.POINTER(i)]),
        "kot_eg_solve": (i, [vp, d, vp, vp, vp, vp, C.POINTER(Result)]),
        "kot_potentials": (i, [vp, i, i, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class KotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def default_options(**kw) -> Options:
    o = Options()
    lib().kot_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(a) -> int | None:
    """Raw pointer of a contiguous float64 torch tensor or NumPy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def launch_count() -> int:
    n = C.c_longlong(0)
    lib().kot_launch_count(C.byref(n))
    return n.value


class Context:
    """Owns one kot_ctx.  ``opts`` fields follow kot_options."""

    def __init__(self, **opts):
        self.opt = default_options(**opts)
        h = C.c_void_p()
        s = lib().kot_create(C.byref(h), C.byref(self.opt))
        if s != OK:
            raise KotError(s, "kot_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().kot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self) -> str:
        return lib().kot_last_error(self.h).decode()

    def _check(self, s: int, ok=(OK,)):
        if s not in ok:
            raise KotError(s, self.last_error())
        return s

    # -- entry points, same names as the C ABI ------------------------------------------
    def build_features(self, X, Y, Xf, Yf, sigma, lambda1, lambda2):
        n, d = X.shape
        l = Xf.shape[0]
        return self._check(lib().kot_build_features(self.h, d, n, _ptr(X), _ptr(Y), l, _ptr(Xf),
                                                    _ptr(Yf), sigma, lambda1, lambda2))

    def set_features(self, Q, z, q2, R, lambda1, lambda2):
        return self._check(lib().kot_set_features(self.h, Q.shape[0], _ptr(Q), _ptr(z), q2,
                                                  _ptr(R), lambda1, lambda2))

    def get_features(self, Q=None, K=None, R=None, z=None, w_mu=None, w_nu=None, c=None,
                     q2=None, eps=None):
        return self._check(lib().kot_get_features(self.h, _ptr(Q), _ptr(K), _ptr(R), _ptr(z),
                                                  _ptr(w_mu), _ptr(w_nu), _ptr(c), _ptr(q2),
                                                  _ptr(eps)))

    def residual(self, gamma, X, r1=None, r2=None, proj=None, sig=None, norms=None):
        return self._check(lib().kot_residual(self.h, _ptr(gamma), _ptr(X), _ptr(r1), _ptr(r2),
                                              _ptr(proj), _ptr(sig), _ptr(norms)))

    def newton_direction(self, gamma, X, mu, dgamma, dX, cg_tol_abs=0.0) -> int:
        it = C.c_int(0)
        self._check(lib().kot_newton_direction(self.h, _ptr(gamma), _ptr(X), mu, cg_tol_abs,
                                               _ptr(dgamma), _ptr(dX), C.byref(it)))
        return it.value

    def ssn_solve(self, tol, gamma_out, X_out=None, gamma0=None, X0=None,
                  allow_no_convergence=False) -> Result:
        r = Result()
        ok = (OK, ERR_NO_CONVERGENCE) if allow_no_convergence else (OK,)
        self._check(lib().kot_ssn_solve(self.h, tol, _ptr(gamma_out), _ptr(X_out), _ptr(gamma0),
                                        _ptr(X0), C.byref(r)), ok)
        return r

    def eg_solve(self, tol, gamma_out, X_out=None, gamma0=None, X0=None,
                 allow_no_convergence=False) -> Result:
        """Pure extragradient (App. F) through kot_eg_solve."""
        r = Result()
        ok = (OK, ERR_NO_CONVERGENCE) if allow_no_convergence else (OK,)
        self._check(lib().kot_eg_solve(self.h, tol, _ptr(gamma_out), _ptr(X_out), _ptr(gamma0),
                                       _ptr(X0), C.byref(r)), ok)
        return r

    def potentials(self, side, m, points, gamma, u=None, grad=None, tmap=None):
        """u (side 0) or v (side 1), its gradient and the map x - grad at m points."""
        return self._check(lib().kot_potentials(self.h, side, m, _ptr(points), _ptr(gamma), _ptr(u),
                                                _ptr(grad), _ptr(tmap)))

    def dense_product(self, M, N, K, alpha, A, lda, transA, B, ldb, transB, beta, Cm, ldc,
                      pieces=3):
        return self._check(lib().kot_dense_product(self.h, M, N, K, alpha, _ptr(A), lda, transA,
                                                   _ptr(B), ldb, transB, beta, _ptr(Cm), ldc,
                                                   pieces))

    def eig_sym(self, l, Z, warm, P, sig):
        """Z = P diag(sig) P^T (sig ascending), refined from `warm` if given.  Returns
        (Jacobi sweeps, refinement steps) of the call."""
        info = (C.c_int * 2)()
        self._check(lib().kot_eig_sym(self.h, l, _ptr(Z), _ptr(warm), _ptr(P), _ptr(sig), info))
        return info[0], info[1]

    def profile(self, mask: int):
        return self._check(lib().kot_profile(self.h, mask))

    def autotune(self, l: int):
        """Tune the emulated product's tile widths and split counts and the Jacobi CTA count and
        threads per CTA for size l; returns (splits 3 slices, splits 6 slices, Jacobi CTAs,
        width 3 slices, width 6 slices, Jacobi threads)."""
        out = (C.c_int * 6)()
        self._check(lib().kot_autotune(self.h, l, out))
        return tuple(out)

    def wait_probe(self, polls: int) -> int:
        """Run the bounded-wait failure probe; returns its status (ERR_TIMEOUT expected)."""
        return lib().kot_wait_probe(self.h, polls)

    def profile_every(self, every: int):
        return self._check(lib().kot_profile_every(self.h, every))

    def profile_read(self, cls: int) -> KernelStats:
        st = KernelStats()
        self._check(lib().kot_profile_read(self.h, cls, C.byref(st)))
        return st

    def trace(self, cap=100000) -> np.ndarray:
        """Per-iteration rows (||R||, mu, CG steps, theta, direction kind) of the last solve."""
        buf = np.zeros(5 * cap)
        cnt = C.c_int(0)
        self._check(lib().kot_get_trace(self.h, buf.ctypes.data, cap, C.byref(cnt)))
        return buf[:5 * cnt.value].reshape(-1, 5).copy()

    def history(self, cap=100000) -> np.ndarray:
        buf = np.zeros(cap)
        cnt = C.c_int(0)
        self._check(lib().kot_get_history(self.h, buf.ctypes.data, cap, C.byref(cnt)))
        return buf[:cnt.value].copy()

    def bootstrap_solve(self, Xs, Ys, tol, gammas, allow_no_convergence=True):
        """Resamples Xs, Ys (B x n x d) sharing the filling points of the last build_features;
        gammas: B x l output.  Returns the B results."""
        B, n = Xs.shape[0], Xs.shape[1]
        res = (Result * B)()
        s = lib().kot_bootstrap_solve(self.h, B, n, _ptr(Xs), _ptr(Ys), tol, _ptr(gammas), res)
        ok = (OK, ERR_NO_CONVERGENCE) if allow_no_convergence else (OK,)
        self._check(s, ok)
        return list(res)

    def batch_solve(self, problems, gammas, allow_no_convergence=True):
        """problems: list of objects with X, Y, Xf, Yf (arrays), sigma, lambda1, lambda2, tol."""
        B = len(problems)
        arr = (Problem * B)()
        for i, (p, g) in enumerate(zip(problems, gammas)):
            arr[i] = Problem(p.X.shape[1], p.X.shape[0], p.Xf.shape[0], _ptr(p.X), _ptr(p.Y),
                             _ptr(p.Xf), _ptr(p.Yf), p.sigma, p.lambda1, p.lambda2, p.tol, _ptr(g))
        res = (Result * B)()
        s = lib().kot_batch_solve(self.h, B, arr, res)
        ok = (OK, ERR_NO_CONVERGENCE) if allow_no_convergence else (OK,)
        self._check(s, ok)
        return list(res)


@dataclass
class DeviceProblem:
    """A workloads.Problem moved to device tensors (float64)."""
    X: object
    Y: object
    Xf: object
    Yf: object
    sigma: float
    lambda1: float
    lambda2: float
    tol: float

    @staticmethod
    def from_problem(p, device="cuda"):
        import torch
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=device)
        return DeviceProblem(t(p.X), t(p.Y), t(p.Xf), t(p.Yf), p.sigma, p.lambda1, p.lambda2,
                             p.tol)
