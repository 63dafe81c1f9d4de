"""Thin ctypes binding of libmeg.so (include/meg.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
library.  Objective data and streams come from PyTorch (device tensors,
``torch.cuda.current_stream().cuda_stream``).  Loading fails loudly when
the library has not been built or cannot be opened.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmeg.so")

MEG_OK, MEG_ERR_INVALID_ARG, MEG_ERR_OOM, MEG_ERR_CUDA, MEG_ERR_NUMERIC, MEG_ERR_NOT_CONVERGED, \
    MEG_ERR_TIMEOUT, MEG_ERR_STATE = range(8)
MEG_FP64, MEG_FP32, MEG_MIXED_BF16 = 0, 1, 2
MEG_DENSE_QUAD, MEG_CSR_QUAD, MEG_MEAS_STOCH, MEG_LINEAR, MEG_BILINEAR = 0, 1, 2, 3, 4
MEG_EIG_SUBSPACE, MEG_EIG_BLOCK_KRYLOV = 0, 1
PRECISION = {"fp64": MEG_FP64, "fp32": MEG_FP32, "bf16": MEG_MIXED_BF16}
# slots of the small state (csrc/meg_dev.cuh, SmallSlot)
SM_T, SM_EPS, SM_S, SM_LOGS, SM_SHIFT, SM_C0, SM_ALPHA, SM_GNORM, SM_FEST, SM_CERT, SM_HOLDS, \
    SM_FIRST_HOLD, SM_STATUS, SM_TRD, SM_FROD2, SM_LAST_T, SM_LSE, SM_RSS, SM_RESID_BOUND, SM_ETA, \
    SM_JSWEEPS, SM_F1 = range(22)
SM_MU, SM_DCOEF, SM_SIGMA = 32, 64, 96
SM_TOTAL = 128 + 13 * 1024 + 32


class meg_options(C.Structure):
    _fields_ = [("n", C.c_int), ("r", C.c_int), ("p", C.c_int), ("q", C.c_int),
                ("precision", C.c_int), ("eta", C.c_double), ("eps_a", C.c_double),
                ("eps_c", C.c_double), ("eps_pow", C.c_double), ("max_iters", C.c_int),
                ("tol", C.c_double), ("seed", C.c_uint64), ("stream", C.c_void_p), ("eigensolver", C.c_int)]


class meg_objective_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("dense", C.c_void_p), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("nnz", C.c_int64),
                ("A", C.c_void_p), ("y", C.c_void_p), ("m", C.c_int64), ("L", C.c_int),
                ("B", C.c_void_p), ("tau", C.c_double), ("mrank", C.c_int)]


class meg_autotune_options(C.Structure):
    _fields_ = [("q_max", C.c_int), ("p_cand", C.c_void_p), ("n_p", C.c_int), ("pilot_iters", C.c_int),
                ("horizon", C.c_int), ("tol_x", C.c_double), ("krylov", C.c_int)]


class meg_server_options(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("max_active", C.c_int), ("check_every", C.c_int),
                ("meas_check_every", C.c_int)]


class meg_request(C.Structure):
    _fields_ = [("opt", meg_options), ("kind", C.c_int), ("data", C.c_void_p), ("y", C.c_void_p),
                ("m", C.c_int64), ("L", C.c_int), ("warm_start_products", C.c_int), ("V0", C.c_void_p),
                ("lam0", C.c_void_p), ("fstar", C.c_double), ("tol", C.c_double), ("max_iters", C.c_int),
                ("out_V", C.c_void_p), ("out_mu", C.c_void_p), ("out_s", C.c_void_p)]


class meg_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int), ("iters", C.c_int), ("f1", C.c_double),
                ("f", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class MegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


_lib: Optional[C.CDLL] = None
_P = C.POINTER
_exiting = False


def _mark_exit():
    # objects still alive at interpreter exit are released by the process
    # exit itself; their destructors must not call into a CUDA runtime that
    # may already be shut down
    global _exiting
    _exiting = True


import atexit  # noqa: E402

atexit.register(_mark_exit)


def load(path: str = LIB_PATH) -> C.CDLL:
    """Open libmeg.so and declare its entry points (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmeg.so not built ({path}); run paper_2012_10469_gb300.build.build()")
    lib = C.CDLL(path)
    H = C.c_void_p
    sig = {
        "meg_create": (C.c_int, [_P(meg_options), _P(C.c_double), _P(C.c_double), _P(H)]),
        "meg_set_objective": (C.c_int, [H, _P(meg_objective_desc)]),
        "meg_warm_start": (C.c_int, [H, C.c_int]),
        "meg_refine_subspace": (C.c_int, [H, C.c_int]),
        "meg_trace_exp_estimate": (C.c_int, [H, _P(C.c_double), C.c_int, _P(C.c_double)]),
        "meg_step": (C.c_int, [H, C.c_int]),
        "meg_solve": (C.c_int, [H, C.c_double, C.c_int, _P(C.c_int)]),
        "meg_set_fstar": (C.c_int, [H, C.c_double]),
        "meg_certificate": (C.c_int, [H, _P(C.c_double), _P(C.c_int), _P(C.c_int)]),
        "meg_get_iterate": (C.c_int, [H, _P(C.c_double), _P(C.c_double), _P(C.c_double)]),
        "meg_get_ritz": (C.c_int, [H, _P(C.c_double), _P(C.c_int)]),
        "meg_objective": (C.c_int, [H, _P(C.c_double)]),
        "meg_destroy": (C.c_int, [H]),
        "meg_last_error": (C.c_char_p, []),
        "meg_group_create": (C.c_int, [_P(H), C.c_int, C.c_void_p, _P(H)]),
        "meg_group_step": (C.c_int, [H, C.c_int]),
        "meg_group_destroy": (C.c_int, [H]),
        "meg_footprint": (C.c_int64, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
        "meg_group_time_product": (C.c_int, [H, C.c_int, _P(C.c_float)]),
        "meg_group_kernels_per_step": (C.c_int, [H]),
        "meg_group_time_chain": (C.c_int, [H, C.c_int, _P(C.c_float)]),
        "meg_objective_dense_noalloc": (C.c_int, [C.c_void_p, _P(C.c_double), C.c_double, C.c_int, C.c_int,
                                                  C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
        "meg_group_launch": (C.c_int, [H, C.c_int]),
        "meg_autotune": (C.c_int, [_P(meg_options), _P(meg_objective_desc), _P(C.c_double), _P(C.c_double),
                                   _P(meg_autotune_options), _P(C.c_int), _P(C.c_int), _P(C.c_double),
                                   _P(C.c_int)]),
        "meg_warm_start_many": (C.c_int, [_P(H), C.c_int, C.c_int, C.c_void_p, _P(C.c_double)]),
        "meg_group_objective": (C.c_int, [H, _P(C.c_double)]),
        "meg_server_create": (C.c_int, [_P(meg_server_options), _P(H)]),
        "meg_server_submit": (C.c_int, [H, _P(meg_request), _P(C.c_uint64)]),
        "meg_server_poll": (C.c_int, [H, _P(meg_result), C.c_int, _P(C.c_int), C.c_int]),
        "meg_server_counts": (C.c_int, [H, _P(C.c_int64), _P(C.c_int64)]),
        "meg_server_tick_counts": (C.c_int, [H, _P(C.c_int64), _P(C.c_int64)]),
        "meg_server_now": (C.c_double, [H]),
        "meg_server_destroy": (C.c_int, [H]),
        "meg_state_size": (C.c_int64, [H]),
        "meg_get_state": (C.c_int, [H, C.c_void_p, C.c_int64]),
        "meg_set_state": (C.c_int, [H, C.c_void_p, C.c_int64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared by include/meg.h (parsed from the header)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "meg.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:meg_status|const char\*|int64_t|int|double)\s+(meg_\w+)\s*\(", text, re.M)))


def _check(status: int, what: str):
    if status != MEG_OK:
        msg = _lib.meg_last_error().decode() if _lib is not None else ""
        raise MegError(status, f"{what}: {msg}")


def _dptr(x) -> Optional[int]:
    if x is None:
        return None
    return int(x.data_ptr())


def _f64p(a: np.ndarray):
    return a.ctypes.data_as(_P(C.c_double))


def meg_last_error() -> str:
    return load().meg_last_error().decode()


def meg_footprint(n, r, p, precision, kind) -> int:
    return int(load().meg_footprint(n, r, p, precision, kind))


class Solve:
    """One solve (meg_handle) with the C ABI's calls as methods."""

    def __init__(self, n: int, r: int, p: int = 4, q: int = 2, precision: int = MEG_FP64,
                 eta: float = 1.0, eps=(0.8, 10.0, 2.0), seed: int = 1, V0=None, lam0=None,
                 stream=None, max_iters: int = 1000, tol: float = 1e-6, eigensolver: int = MEG_EIG_SUBSPACE):
        lib = load()
        self.n, self.r, self.k = n, r, r + p
        self.precision = precision
        self._keep = []
        opt = meg_options(n=n, r=r, p=p, q=q, precision=precision, eta=eta, eps_a=eps[0], eps_c=eps[1],
                          eps_pow=eps[2], max_iters=max_iters, tol=tol, seed=seed,
                          stream=None if stream is None else int(stream), eigensolver=eigensolver)
        h = C.c_void_p()
        if V0 is not None:
            V0 = np.ascontiguousarray(V0, dtype=np.float64)
            lam0 = np.ascontiguousarray(lam0, dtype=np.float64)
            st = lib.meg_create(C.byref(opt), _f64p(V0), _f64p(lam0), C.byref(h))
        else:
            st = lib.meg_create(C.byref(opt), None, None, C.byref(h))
        _check(st, "meg_create")
        self.h = h

    # -- objective
    def meg_set_objective(self, kind, dense=None, rowptr=None, col=None, val=None, A=None, y=None, L=0,
                          B=None, tau=1.0, mrank=1):
        """Tensors are borrowed (kept alive by this object)."""
        self._keep = [t for t in (dense, rowptr, col, val, A, y, B) if t is not None]
        d = meg_objective_desc(kind=kind, dense=_dptr(dense), rowptr=_dptr(rowptr), col=_dptr(col),
                               val=_dptr(val), nnz=0 if col is None else int(col.numel()),
                               A=_dptr(A), y=_dptr(y), m=0 if A is None else int(A.shape[0]) // max(1, mrank),
                               L=L, B=_dptr(B), tau=float(tau), mrank=int(mrank))
        _check(load().meg_set_objective(self.h, C.byref(d)), "meg_set_objective")

    def meg_warm_start(self, products: int = 40):
        _check(load().meg_warm_start(self.h, products), "meg_warm_start")

    def meg_trace_exp_estimate(self, U, steps: int) -> float:
        """Tr exp(M_t) by Hutchinson over the columns of U (n x k) with Lanczos quadrature."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = C.c_double()
        _check(load().meg_trace_exp_estimate(self.h, _f64p(U), steps, C.byref(out)), "meg_trace_exp_estimate")
        return out.value

    def meg_refine_subspace(self, products: int):
        _check(load().meg_refine_subspace(self.h, products), "meg_refine_subspace")

    def meg_step(self, nsteps: int = 1):
        _check(load().meg_step(self.h, nsteps), "meg_step")

    def meg_solve(self, tol: float, max_iters: int):
        it = C.c_int(0)
        st = load().meg_solve(self.h, tol, max_iters, C.byref(it))
        if st not in (MEG_OK, MEG_ERR_NOT_CONVERGED):
            _check(st, "meg_solve")
        return it.value, st == MEG_OK

    def meg_set_fstar(self, fstar: float):
        _check(load().meg_set_fstar(self.h, fstar), "meg_set_fstar")

    def meg_certificate(self):
        c, holds, first = C.c_double(), C.c_int(), C.c_int()
        _check(load().meg_certificate(self.h, C.byref(c), C.byref(holds), C.byref(first)), "meg_certificate")
        return c.value, bool(holds.value), first.value

    def meg_get_iterate(self):
        V = np.empty((self.n, self.r), dtype=np.float64)
        mu = np.empty(self.r, dtype=np.float64)
        s = C.c_double()
        _check(load().meg_get_iterate(self.h, _f64p(V), _f64p(mu), C.byref(s)), "meg_get_iterate")
        return V, mu, s.value

    def meg_get_ritz(self):
        sig = np.empty(self.k, dtype=np.float64)
        t = C.c_int()
        _check(load().meg_get_ritz(self.h, _f64p(sig), C.byref(t)), "meg_get_ritz")
        return sig, t.value

    def meg_objective(self) -> float:
        f = C.c_double()
        _check(load().meg_objective(self.h, C.byref(f)), "meg_objective")
        return f.value

    def meg_get_state(self) -> bytes:
        lib = load()
        nb = int(lib.meg_state_size(self.h))
        buf = C.create_string_buffer(nb)
        _check(lib.meg_get_state(self.h, buf, nb), "meg_get_state")
        return buf.raw

    def meg_set_state(self, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        _check(load().meg_set_state(self.h, buf, len(state)), "meg_set_state")

    def small_state(self) -> np.ndarray:
        """The float64 small state (scalars, mu, Ritz values, k x k blocks)."""
        st = self.meg_get_state()
        return np.frombuffer(st, dtype=np.float64, count=SM_TOTAL, offset=64).copy()

    def meg_destroy(self):
        if getattr(self, "h", None):
            load().meg_destroy(self.h)
            self.h = None

    def __del__(self):
        if _exiting:
            return
        try:
            self.meg_destroy()
        except Exception:
            pass


class Group:
    """Several solves stepped with grouped kernels (meg_group)."""

    def __init__(self, solves, stream=None):
        lib = load()
        self.solves = list(solves)
        arr = (C.c_void_p * len(self.solves))(*[s.h for s in self.solves])
        g = C.c_void_p()
        _check(lib.meg_group_create(arr, len(self.solves), None if stream is None else int(stream),
                                    C.byref(g)), "meg_group_create")
        self.g = g

    def meg_group_step(self, nsteps: int = 1):
        _check(load().meg_group_step(self.g, nsteps), "meg_group_step")

    def meg_group_time_product(self, reps: int = 20) -> float:
        ms = C.c_float()
        _check(load().meg_group_time_product(self.g, reps, C.byref(ms)), "meg_group_time_product")
        return ms.value

    def meg_group_time_chain(self, reps: int = 20) -> list:
        """Warm microseconds of each kernel after an intermediate product:
        [combine, its island, orth1, its island, orth2, its island]."""
        us = (C.c_float * 6)()
        _check(load().meg_group_time_chain(self.g, reps, us), "meg_group_time_chain")
        return [float(v) for v in us]

    def meg_group_kernels_per_step(self) -> int:
        return int(load().meg_group_kernels_per_step(self.g))

    def meg_group_launch(self, nsteps: int = 1):
        _check(load().meg_group_launch(self.g, nsteps), "meg_group_launch")

    def meg_group_objective(self) -> np.ndarray:
        f = np.empty(len(self.solves), dtype=np.float64)
        _check(load().meg_group_objective(self.g, _f64p(f)), "meg_group_objective")
        return f

    def meg_group_destroy(self):
        if getattr(self, "g", None):
            load().meg_group_destroy(self.g)
            self.g = None

    def __del__(self):
        if _exiting:
            return
        try:
            self.meg_group_destroy()
        except Exception:
            pass


def meg_autotune(n, r, precision, kind, V0, lam0, dense=None, A=None, y=None, L=0, rowptr=None, col=None,
                 val=None, eta=1.0, eps=(0.8, 10.0, 2.0), seed=1, q_max=4, p_cand=None, pilot_iters=20,
                 horizon=500, tol_x=1e-5, stream=None, krylov=False):
    """(p, q, distance to the reference, met_target, eigensolver) for one problem; device
    tensors as in Solve.meg_set_objective.  krylov: also try the block Krylov eigensolver."""
    lib = load()
    opt = meg_options(n=n, r=r, p=1, q=1, precision=precision, eta=eta, eps_a=eps[0], eps_c=eps[1],
                      eps_pow=eps[2], max_iters=horizon, tol=1e-6, seed=seed,
                      stream=None if stream is None else int(stream))
    d = meg_objective_desc(kind=kind, dense=_dptr(dense), rowptr=_dptr(rowptr), col=_dptr(col), val=_dptr(val),
                           nnz=0 if col is None else int(col.numel()), A=_dptr(A), y=_dptr(y),
                           m=0 if A is None else int(A.shape[0]), L=L)
    pc = None
    if p_cand is not None:
        pc = np.ascontiguousarray(p_cand, dtype=np.int32)
    ao = meg_autotune_options(q_max=q_max, p_cand=None if pc is None else pc.ctypes.data,
                              n_p=0 if pc is None else len(pc), pilot_iters=pilot_iters, horizon=horizon, tol_x=tol_x,
                              krylov=1 if krylov else 0)
    V0 = np.ascontiguousarray(V0, dtype=np.float64)
    lam0 = np.ascontiguousarray(lam0, dtype=np.float64)
    p, q, e, eig = C.c_int(), C.c_int(), C.c_double(), C.c_int()
    st = lib.meg_autotune(C.byref(opt), C.byref(d), _f64p(V0), _f64p(lam0), C.byref(ao), C.byref(p), C.byref(q),
                          C.byref(e), C.byref(eig))
    if st not in (MEG_OK, MEG_ERR_NOT_CONVERGED):
        _check(st, "meg_autotune")
    return p.value, q.value, e.value, st == MEG_OK, eig.value


def meg_warm_start_many(solves, products: int = 40, stream=None) -> np.ndarray:
    """Warm-start several solves together; returns f(X_1) of each."""
    arr = (C.c_void_p * len(solves))(*[s.h for s in solves])
    f1 = np.empty(len(solves), dtype=np.float64)
    _check(load().meg_warm_start_many(arr, len(solves), products, None if stream is None else int(stream),
                                      _f64p(f1)), "meg_warm_start_many")
    return f1


class Server:
    """Continuous-batching request loop (meg_server).  Host arrays of a
    request are kept alive here until its result has been polled."""

    def __init__(self, hbm_budget: int, max_active: int = 256, check_every: int = 10,
                 meas_check_every: int = 50):
        lib = load()
        opt = meg_server_options(hbm_budget=int(hbm_budget), max_active=max_active, check_every=check_every,
                                 meas_check_every=meas_check_every)
        h = C.c_void_p()
        _check(lib.meg_server_create(C.byref(opt), C.byref(h)), "meg_server_create")
        self.h = h
        self._live = {}

    def meg_server_submit(self, kind: int, n: int, r: int, data: np.ndarray, p: int = 4, q: int = 2,
                          precision: int = MEG_FP64, eta: float = 1.0, eps=(0.8, 10.0, 2.0), seed: int = 1,
                          y: Optional[np.ndarray] = None, L: int = 0, warm_start_products: int = 40,
                          V0=None, lam0=None, fstar: float = float("nan"), tol: float = 1e-6,
                          max_iters: int = 5000, eigensolver: int = MEG_EIG_SUBSPACE) -> int:
        """data: host array (dense n x n, or A m x n) in the precision's storage
        type (float64, float32, or uint16 bfloat16 bits); y: float64 (m)."""
        data = np.ascontiguousarray(data)
        keep = [data]
        opt = meg_options(n=n, r=r, p=p, q=q, precision=precision, eta=eta, eps_a=eps[0], eps_c=eps[1],
                          eps_pow=eps[2], max_iters=max_iters, tol=tol, seed=seed, stream=None,
                          eigensolver=eigensolver)
        outV = np.zeros((n, r), dtype=np.float64)
        outmu = np.zeros(r, dtype=np.float64)
        outs = np.zeros(1, dtype=np.float64)
        keep += [outV, outmu, outs]
        rq = meg_request(opt=opt, kind=kind, data=data.ctypes.data, y=None, m=0, L=L,
                         warm_start_products=warm_start_products, V0=None, lam0=None, fstar=fstar, tol=tol,
                         max_iters=max_iters, out_V=outV.ctypes.data, out_mu=outmu.ctypes.data,
                         out_s=outs.ctypes.data)
        if y is not None:
            y = np.ascontiguousarray(y, dtype=np.float64)
            keep.append(y)
            rq.y = y.ctypes.data
            rq.m = int(data.shape[0])
        if V0 is not None:
            V0 = np.ascontiguousarray(V0, dtype=np.float64)
            lam0 = np.ascontiguousarray(lam0, dtype=np.float64)
            keep += [V0, lam0]
            rq.V0, rq.lam0 = V0.ctypes.data, lam0.ctypes.data
        rid = C.c_uint64()
        _check(load().meg_server_submit(self.h, C.byref(rq), C.byref(rid)), "meg_server_submit")
        self._live[rid.value] = (keep, outV, outmu, outs)
        return rid.value

    def meg_server_poll(self, max_out: int = 256, timeout_ms: int = 0):
        """Finished requests: list of (meg_result fields as a dict, V, mu, s)."""
        buf = (meg_result * max_out)()
        cnt = C.c_int()
        _check(load().meg_server_poll(self.h, buf, max_out, C.byref(cnt), timeout_ms), "meg_server_poll")
        out = []
        for i in range(cnt.value):
            r = buf[i]
            rec = {f: getattr(r, f) for f, _ in meg_result._fields_}
            _, V, mu, s = self._live.pop(r.id)
            out.append((rec, V, mu, float(s[0])))
        return out

    def meg_server_counts(self):
        a, b = C.c_int64(), C.c_int64()
        _check(load().meg_server_counts(self.h, C.byref(a), C.byref(b)), "meg_server_counts")
        return a.value, b.value

    def meg_server_tick_counts(self):
        a, b = C.c_int64(), C.c_int64()
        _check(load().meg_server_tick_counts(self.h, C.byref(a), C.byref(b)), "meg_server_tick_counts")
        return a.value, b.value

    def meg_server_now(self) -> float:
        return float(load().meg_server_now(self.h))

    def meg_server_destroy(self):
        if getattr(self, "h", None):
            load().meg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        if _exiting:
            return
        try:
            self.meg_server_destroy()
        except Exception:
            pass
