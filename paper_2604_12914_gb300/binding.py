"""Thin ctypes binding of libcclr (include/cclr.h): argument marshalling only.

Every computation runs in the CUDA library.  Arrays may be numpy (host; the context is
created with device_ptrs=0) or CUDA torch tensors (device_ptrs=1, used on the given
stream).  Complex arrays are complex128 (interleaved re/im doubles).  If the shared
library is missing or cannot be loaded, every entry point raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcclr.so")

CCLR_OK, CCLR_EINVAL, CCLR_ENOMEM, CCLR_ENOCONV, CCLR_EDEVICE, CCLR_ETIMEOUT, CCLR_EUNSUPPORTED = range(7)
CCLR_FP64, CCLR_C64_TF32, CCLR_C64_3XTF32, CCLR_C64_FP32, CCLR_BF16X3 = range(5)
PREC = {"fp64": CCLR_FP64, "tf32": CCLR_C64_TF32, "3xtf32": CCLR_C64_3XTF32, "fp32": CCLR_C64_FP32,
        "bf16x3": CCLR_BF16X3}

EXPORTS = ["cc_lr_init", "cc_lr_sigma", "cc_lr_sigma_T", "cc_lr_sigma_packed", "cc_lr_xi", "cc_lr_solve_x", "cc_lr_solve",
           "cc_lr_solve_damped", "cc_lr_solve_left", "cc_lr_solve_alpha_tol", "cc_lr_eta",
           "cc_lr_lambda", "cc_lr_get_t", "cc_lr_ccsd_residual", "cc_lr_ccsd", "cc_lr_set_precision", "cc_lr_set_refinement", "cc_lr_set_graphs",
           "cc_lr_graph_stats", "cc_lr_ladder_tuning", "cc_lr_set_ladder_storage", "cc_lr_set_solver",
           "cc_lr_last_timings", "cc_lr_memory", "cc_lr_set_autotune", "cc_lr_gemm_tuning",
           "cc_lr_free", "cc_lr_strerror", "cc_lr_last_error", "cc_lr_launch_count"]


class CclrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libcclr status {status}: {msg}")
        self.status = status


class cclr_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("sigma_calls", ctypes.c_int),
                ("refinements", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("time_solve_ms", ctypes.c_double),
                ("time_lambda_ms", ctypes.c_double), ("time_alpha_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libcclr.so (raises if absent: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libcclr.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    sig = {
        "cc_lr_init": [ctypes.POINTER(ctypes.c_void_p), I, I, I, P, P, P, P, P, P, P, I, S, I, P],
        "cc_lr_sigma": [P, I, P, P, P, P],
        "cc_lr_sigma_T": [P, I, P, P, P, P],
        "cc_lr_sigma_packed": [P, I, I, P, P],
        "cc_lr_xi": [P, I, P, P],
        "cc_lr_solve_x": [P, D, I, D, I, P, P, ctypes.POINTER(cclr_stats)],
        "cc_lr_solve": [P, I, P, I, P, D, I, P, ctypes.POINTER(cclr_stats)],
        "cc_lr_solve_damped": [P, I, P, D, I, P, D, I, P, ctypes.POINTER(cclr_stats)],
        "cc_lr_solve_left": [P, I, P, I, P, D, I, P, ctypes.POINTER(cclr_stats)],
        "cc_lr_eta": [P, I, D, P, P],
        "cc_lr_solve_alpha_tol": [P, I, P, I, P, D, I, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(cclr_stats)],
        "cc_lr_lambda": [P, D, P, P],
        "cc_lr_get_t": [P, P, P],
        "cc_lr_ccsd_residual": [P, I, P, P, P, P, P],
        "cc_lr_ccsd": [P, I, D, I, I, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)],
        "cc_lr_set_precision": [P, I],
        "cc_lr_set_solver": [P, I, I, I],
        "cc_lr_set_refinement": [P, I],
        "cc_lr_set_graphs": [P, I],
        "cc_lr_set_ladder_storage": [P, I],
        "cc_lr_graph_stats": [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "cc_lr_ladder_tuning": [P, I, ctypes.POINTER(ctypes.c_int), I, P, P, ctypes.POINTER(ctypes.c_int)],
        "cc_lr_last_timings": [P, P, I],
        "cc_lr_memory": [P, ctypes.POINTER(S), ctypes.POINTER(S), ctypes.POINTER(S)],
        "cc_lr_set_autotune": [P, I],
        "cc_lr_gemm_tuning": [P, I, ctypes.POINTER(ctypes.c_int), P],
        "cc_lr_free": [P],
        "cc_lr_strerror": [I],
        "cc_lr_last_error": [],
        "cc_lr_launch_count": [],
        "cc_lr_selftest_gemm": [I, I, I, I, ctypes.c_uint, P],
        "cc_lr_selftest_gemm_noalloc": [I, I, I, I, ctypes.c_uint, P],
        "cc_lr_bench_gemm": [I, I, I, I, I, P],
        "cc_lr_bench_hbm": [I, I, I, P, I],
        "cc_lr_selftest_timeout": [I, ctypes.POINTER(ctypes.c_int)],
        "cc_lr_selftest_precond": [I, D, D, ctypes.c_uint, ctypes.POINTER(ctypes.c_double)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.cc_lr_free.restype = None
    lib.cc_lr_strerror.restype = ctypes.c_char_p
    lib.cc_lr_last_error.restype = ctypes.c_char_p
    lib.cc_lr_launch_count.restype = ctypes.c_ulonglong
    _lib = lib
    return lib


def _check(status, allow=()):
    if status != CCLR_OK and status not in allow:
        msg = load().cc_lr_last_error().decode()
        raise CclrError(status, msg)
    return status


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    # torch tensor: the library reads raw memory, so lazy conjugate / negative views and
    # non-contiguous strides are refused rather than silently misread
    if a.is_conj() or a.is_neg() or not a.is_contiguous():
        raise ValueError("pass a contiguous tensor without lazy conj/neg bits (use resolve_conj())")
    return a.data_ptr()


def _c128(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.complex128)


class Context:
    """Owning wrapper around a cclr_ctx (host numpy arrays unless device=True)."""

    def __init__(self, o, v, naux, eps, L, mu, t1=None, t2=None, lam1=None, lam2=None,
                 prec="fp64", hbm_budget=0, device=False, stream=None):
        lib = load()
        self.o, self.v, self.naux = o, v, naux
        self.device = device
        if device:
            arrs = [eps, L, mu, t1, t2, lam1, lam2]
            self._keep = arrs
            ptrs = [_ptr(a) for a in arrs]
        else:
            eps = np.ascontiguousarray(eps, dtype=np.float64)
            arrs = [eps, _c128(L), _c128(mu), _c128(t1), _c128(t2), _c128(lam1), _c128(lam2)]
            self._keep = arrs
            ptrs = [_ptr(a) for a in arrs]
        h = ctypes.c_void_p()
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        _check(lib.cc_lr_init(ctypes.byref(h), o, v, naux, *ptrs, p, int(hbm_budget),
                              1 if device else 0, stream))
        self._h = h
        self._keep = None

    # -- helpers
    def _out(self, shape):
        if self.device:
            import torch
            return torch.empty(shape, dtype=torch.complex128, device="cuda")
        return np.empty(shape, dtype=np.complex128)

    def _in(self, a):
        return a if self.device else _c128(a)

    def close(self):
        if getattr(self, "_h", None):
            load().cc_lr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points
    def cc_lr_sigma(self, x1, x2, transpose=False):
        o, v = self.o, self.v
        x1, x2 = self._in(x1), self._in(x2)
        batched = x1.ndim == 3
        nr = x1.shape[0] if batched else 1
        s1 = self._out(tuple(x1.shape))
        s2 = self._out(tuple(x2.shape))
        fn = load().cc_lr_sigma_T if transpose else load().cc_lr_sigma
        _check(fn(self._h, nr, _ptr(x1), _ptr(x2), _ptr(s1), _ptr(s2)))
        return s1, s2

    def sigma_into(self, x1, x2, s1, s2, nrhs=1, transpose=False):
        """sigma (or sigma^T) of caller-owned arrays (host or device memory), no allocation."""
        fn = load().cc_lr_sigma_T if transpose else load().cc_lr_sigma
        _check(fn(self._h, nrhs, _ptr(x1), _ptr(x2), _ptr(s1), _ptr(s2)))

    def n_packed(self):
        """Length of one packed unique-amplitude vector: o v + o(o-1)/2 v(v-1)/2."""
        o, v = self.o, self.v
        return o * v + (o * (o - 1) // 2) * (v * (v - 1) // 2)

    def sigma_packed(self, x, s, nrhs=1, transpose=False):
        """sigma (or sigma^T) of nrhs packed vectors, device arrays [nrhs][n_packed] complex128."""
        _check(load().cc_lr_sigma_packed(self._h, nrhs, 1 if transpose else 0, _ptr(x), _ptr(s)))

    def cc_lr_sigma_T(self, y1, y2):
        return self.cc_lr_sigma(y1, y2, transpose=True)

    def cc_lr_xi(self, comp):
        o, v = self.o, self.v
        x1 = self._out((o, v))
        x2 = self._out((o, o, v, v))
        _check(load().cc_lr_xi(self._h, comp, _ptr(x1), _ptr(x2)))
        return x1, x2

    def cc_lr_solve_x(self, omega, comp, tol=1e-10, diis_depth=8, allow_noconv=False):
        o, v = self.o, self.v
        x1 = self._out((o, v))
        x2 = self._out((o, o, v, v))
        st = cclr_stats()
        _check(load().cc_lr_solve_x(self._h, float(omega), comp, float(tol), diis_depth,
                                    _ptr(x1), _ptr(x2), ctypes.byref(st)),
               allow=(CCLR_ENOCONV,) if allow_noconv else ())
        return x1, x2, st.as_dict()

    def cc_lr_solve(self, omegas, comps=(0, 1, 2), tol=1e-10, diis_depth=8, allow_noconv=False, gamma=0.0):
        """alpha[w][a][b] at omega_w (+ i gamma when gamma > 0: damped response)."""
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        cp = np.ascontiguousarray(comps, dtype=np.int32)
        out = np.zeros((len(om), len(cp), len(cp)), dtype=np.complex128)
        st = cclr_stats()
        if gamma:
            call = load().cc_lr_solve_damped(self._h, len(om), _ptr(om), float(gamma), len(cp), _ptr(cp),
                                             float(tol), diis_depth, _ptr(out), ctypes.byref(st))
        else:
            call = load().cc_lr_solve(self._h, len(om), _ptr(om), len(cp), _ptr(cp), float(tol),
                                      diis_depth, _ptr(out), ctypes.byref(st))
        status = _check(call, allow=(CCLR_ENOCONV,) if allow_noconv else ())
        d = st.as_dict()
        d["status"] = status
        return out, d

    def cc_lr_solve_left(self, omegas, comps=(0, 1, 2), tol=1e-10, diis_depth=8, allow_noconv=False):
        """alpha[w][a][b] by the left-hand (Y) route."""
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        cp = np.ascontiguousarray(comps, dtype=np.int32)
        out = np.zeros((len(om), len(cp), len(cp)), dtype=np.complex128)
        st = cclr_stats()
        status = _check(load().cc_lr_solve_left(self._h, len(om), _ptr(om), len(cp), _ptr(cp), float(tol), diis_depth,
                                                _ptr(out), ctypes.byref(st)),
                        allow=(CCLR_ENOCONV,) if allow_noconv else ())
        d = st.as_dict()
        d["status"] = status
        return out, d

    def cc_lr_solve_alpha_tol(self, omegas, comps=(0, 1, 2), tol_alpha=1e-5, diis_depth=8, allow_noconv=False):
        """(alpha[w][a][b], a-posteriori |delta alpha| estimate, stats): solves tightened until the
        left- and right-route alphas agree within tol_alpha (a.u.)."""
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        cp = np.ascontiguousarray(comps, dtype=np.int32)
        out = np.zeros((len(om), len(cp), len(cp)), dtype=np.complex128)
        err = ctypes.c_double(0.0)
        st = cclr_stats()
        status = _check(load().cc_lr_solve_alpha_tol(self._h, len(om), _ptr(om), len(cp), _ptr(cp), float(tol_alpha),
                                                     diis_depth, _ptr(out), ctypes.byref(err), ctypes.byref(st)),
                        allow=(CCLR_ENOCONV,) if allow_noconv else ())
        d = st.as_dict()
        d["status"] = status
        return out, err.value, d

    def cc_lr_eta(self, comp, tol=1e-10):
        o, v = self.o, self.v
        e1 = self._out((o, v))
        e2 = self._out((o, o, v, v))
        _check(load().cc_lr_eta(self._h, comp, float(tol), _ptr(e1), _ptr(e2)))
        return e1, e2

    def cc_lr_lambda(self, tol=1e-10):
        o, v = self.o, self.v
        l1 = self._out((o, v))
        l2 = self._out((o, o, v, v))
        _check(load().cc_lr_lambda(self._h, float(tol), _ptr(l1), _ptr(l2)))
        return l1, l2

    def cc_lr_get_t(self):
        o, v = self.o, self.v
        t1 = self._out((o, v))
        t2 = self._out((o, o, v, v))
        _check(load().cc_lr_get_t(self._h, _ptr(t1), _ptr(t2)))
        return t1, t2

    def cc_lr_ccsd_residual(self, t1, t2, prec=-1):
        """Omega(T) (r1, r2) and the correlation energy E(T) at the given amplitudes."""
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        t1, t2 = self._in(t1), self._in(t2)
        r1 = self._out(tuple(t1.shape))
        r2 = self._out(tuple(t2.shape))
        e = np.zeros(2)
        _check(load().cc_lr_ccsd_residual(self._h, p, _ptr(t1), _ptr(t2), _ptr(r1), _ptr(r2), e.ctypes.data))
        return r1, r2, complex(e[0], e[1])

    def cc_lr_ccsd(self, tol=1e-9, max_iterations=60, diis_depth=8, prec=-1, allow_noconv=False):
        """Solve the ground-state CCSD equations from the context's amplitudes; the context then
        holds the converged T.  Returns (energy, residual norm, iterations)."""
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        e = np.zeros(2)
        rn = ctypes.c_double(0.0)
        its = ctypes.c_int(0)
        _check(load().cc_lr_ccsd(self._h, p, float(tol), int(max_iterations), int(diis_depth), e.ctypes.data,
                                 ctypes.byref(rn), ctypes.byref(its)),
               allow=(CCLR_ENOCONV,) if allow_noconv else ())
        return complex(e[0], e[1]), rn.value, its.value

    def cc_lr_set_precision(self, prec):
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        _check(load().cc_lr_set_precision(self._h, p))

    def cc_lr_set_graphs(self, on=True):
        """Capture repeated sigma products in CUDA graphs and replay them."""
        _check(load().cc_lr_set_graphs(self._h, 1 if on else 0))

    def cc_lr_graph_stats(self):
        """(graph captures, graph launches) so far."""
        c, l = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().cc_lr_graph_stats(self._h, ctypes.byref(c), ctypes.byref(l)))
        return c.value, l.value

    def cc_lr_set_ladder_storage(self, store=True):
        """Ablation: keep the packed <ab||ef>~ once formed (see include/cclr.h)."""
        _check(load().cc_lr_set_ladder_storage(self._h, 1 if store else 0))

    def cc_lr_ladder_tuning(self, prec="tf32"):
        """(group size in use, [(candidate, ms), ...]) of the pp-ladder autotuner."""
        ga, n = ctypes.c_int(0), ctypes.c_int(0)
        cand = np.zeros(8, dtype=np.int32)
        ms = np.zeros(8, dtype=np.float64)
        _check(load().cc_lr_ladder_tuning(self._h, PREC[prec], ctypes.byref(ga), 8, _ptr(cand), _ptr(ms),
                                          ctypes.byref(n)))
        return ga.value, [(int(cand[k]), float(ms[k])) for k in range(min(n.value, 8))]

    def cc_lr_set_refinement(self, prec="fp64"):
        """Arithmetic of the refinement residuals and F X stencils: "fp64" or "3xtf32"."""
        _check(load().cc_lr_set_refinement(self._h, PREC[prec] if isinstance(prec, str) else int(prec)))

    def cc_lr_set_solver(self, method="gmres", subspace=30, max_iterations=0):
        m = {"gmres": 1, "diis": 0, "block": 2}[method] if isinstance(method, str) else int(method)
        _check(load().cc_lr_set_solver(self._h, m, int(subspace), int(max_iterations)))

    def cc_lr_set_autotune(self, on=True):
        _check(load().cc_lr_set_autotune(self._h, 1 if on else 0))

    def cc_lr_gemm_tuning(self):
        """List of dicts: every tuned GEMM shape of this device and its chosen configuration."""
        n = ctypes.c_int(0)
        _check(load().cc_lr_gemm_tuning(self._h, 0, ctypes.byref(n), None))
        cap = max(1, n.value)
        rec = np.zeros((cap, 10), dtype=np.float64)
        _check(load().cc_lr_gemm_tuning(self._h, cap, ctypes.byref(n), _ptr(rec)))
        keys = ["kind", "M", "N", "K", "BN", "splits", "band", "ms_best", "ms_rule", "tried"]
        return [dict(zip(keys, map(float, rec[k]))) for k in range(min(n.value, cap))]

    def cc_lr_memory(self):
        """(bytes held, peak bytes held, budget) of this context's device memory."""
        a, b, c = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_size_t(0)
        _check(load().cc_lr_memory(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def cc_lr_last_timings(self):
        """[ladder, everything else, total, ladder formation GEMMs] of the last product (ms), and
        [4] the number of products the last multi-vector call was split into."""
        out = np.zeros(5, dtype=np.float64)
        _check(load().cc_lr_last_timings(self._h, _ptr(out), 5))
        return out


def cc_lr_selftest_gemm(M, N, K, mode, seed=1):
    """(tensor-core error, FP32 CUDA-core error) of a random complex64 GEMM vs FP64."""
    err = np.zeros(2, dtype=np.float64)
    _check(load().cc_lr_selftest_gemm(M, N, K, mode, seed, _ptr(err)))
    return float(err[0]), float(err[1])


def cc_lr_selftest_gemm_noalloc(M, N, K, mode, seed=1):
    """cc_lr_selftest_gemm computed in the library's fixed device array (no allocation)."""
    err = np.zeros(2, dtype=np.float64)
    _check(load().cc_lr_selftest_gemm_noalloc(M, N, K, mode, seed, _ptr(err)))
    return float(err[0]), float(err[1])


def cc_lr_bench_gemm(M, N, K, mode, reps=5):
    """(ms per GEMM, TFLOP/s) of the tensor-core complex GEMM path alone."""
    out = np.zeros(2, dtype=np.float64)
    _check(load().cc_lr_bench_gemm(M, N, K, mode, reps, _ptr(out)))
    return float(out[0]), float(out[1])


HBM_KERNELS = ["antisym_apply", "antisym_project", "unpack_doubles", "pack_doubles", "vec_precond", "vec_dot",
               "vec_axpy", "unpack_sig"]


def cc_lr_bench_hbm(o, v, reps=5):
    """{kernel: (ms per launch, algorithmic bytes per launch)} of the HBM-bound kernels at o, v."""
    out = np.zeros(16, dtype=np.float64)
    _check(load().cc_lr_bench_hbm(o, v, reps, _ptr(out), 8))
    return {k: (float(out[2 * i]), float(out[2 * i + 1])) for i, k in enumerate(HBM_KERNELS)}


def cc_lr_selftest_timeout(timeout_us=1000):
    """(status, device flag) of the bounded-wait give-up self-test."""
    flag = ctypes.c_int(0)
    st = load().cc_lr_selftest_timeout(int(timeout_us), ctypes.byref(flag))
    return st, flag.value


def cc_lr_selftest_precond(n=1 << 20, omega=0.0, omega_im=0.0, seed=1):
    """Max relative error of the device preconditioner against host FP64 division."""
    err = ctypes.c_double(0.0)
    _check(load().cc_lr_selftest_precond(int(n), float(omega), float(omega_im), int(seed), ctypes.byref(err)))
    return err.value


def cc_lr_launch_count() -> int:
    return int(load().cc_lr_launch_count())


def cc_lr_strerror(status: int) -> str:
    return load().cc_lr_strerror(status).decode()
