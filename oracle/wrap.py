"""ctypes marshalling for the C oracle (``hc_oracle.c``).  Test infrastructure only.

Every function takes numpy arrays in the oracle's point-major layout and returns numpy
arrays; no arithmetic of the method happens in Python.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.c")
_SO = os.path.join(_HERE, "_build", "libhc_oracle.so")
_lock = threading.Lock()
_lib = None

# status codes (the oracle's own numbering, mirrored by the library's header)
STATUS = {0: "OK", 1: "NOCONV", 2: "SINGULAR", 3: "MIN_STEP", 4: "MAX_STEPS",
          5: "DIVERGED", 6: "NONFINITE"}

_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc.  Contraction of a*b+c into an FMA is switched off:
    the oracle's error-free transformations are the split-based (Dekker) ones."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fno-unsafe-math-optimizations", "-fPIC", "-shared", "-o", tmp, _SRC,
               "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class TrackOpts(ct.Structure):
    """Options of the oracle tracker (Alg. 3.1 readings; defaults match the library's)."""
    _fields_ = [("lambda0", ct.c_double), ("lambda_min", ct.c_double),
                ("lambda_max", ct.c_double), ("grow", ct.c_double), ("shrink", ct.c_double),
                ("eps", ct.c_double), ("eps_x", ct.c_double), ("eps_end", ct.c_double),
                ("eps_end_x", ct.c_double), ("div_bound", ct.c_double),
                ("max_it", ct.c_int32), ("end_it", ct.c_int32), ("grow_after", ct.c_int32),
                ("max_steps", ct.c_int32), ("predictor", ct.c_int32), ("lu_mode", ct.c_int32),
                ("max_refine", ct.c_int32), ("log_cap", ct.c_int32)]


class _Stats(ct.Structure):
    _fields_ = [("n_succ", ct.c_int64), ("n_corr", ct.c_int64), ("newton_its", ct.c_int64),
                ("min_step", ct.c_double), ("avg_step", ct.c_double), ("t_end", ct.c_double),
                ("res_end", ct.c_double), ("status", ct.c_int32), ("end_its", ct.c_int32)]


class PathState(ct.Structure):
    """The oracle's state of a path between corrector stages (or_state in hc_oracle.c);
    phase 0 starts the path at t = 0, 1 tracking, 2 end game pending, 3 done."""
    _fields_ = [("t", ct.c_double), ("tp", ct.c_double), ("tpp", ct.c_double),
                ("lam", ct.c_double), ("min_step", ct.c_double), ("sum_step", ct.c_double),
                ("res_end", ct.c_double), ("n_succ", ct.c_int64), ("n_corr", ct.c_int64),
                ("newton_its", ct.c_int64), ("nhist", ct.c_int32), ("consec", ct.c_int32),
                ("status", ct.c_int32), ("phase", ct.c_int32), ("end_its", ct.c_int32),
                ("pad", ct.c_int32)]


class _StepLog(ct.Structure):
    _fields_ = [("t", ct.c_double), ("lam", ct.c_double), ("res_first", ct.c_double),
                ("res_last", ct.c_double), ("pc_dist", ct.c_double), ("iters", ct.c_int32),
                ("accepted", ct.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ct.CDLL(so)
            d, i, p = ct.c_double, ct.c_int, ct.c_void_p
            for name in ("or_r_add", "or_r_mul", "or_r_div", "or_c_mul", "or_c_div"):
                fn = getattr(L, name)
                fn.argtypes = [i, _F64P, _F64P, _F64P]
                fn.restype = i
            L.or_validate.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P]
            L.or_validate.restype = i
            L.or_degrees.argtypes = [i, _I32P, _I32P, _I32P, _I32P]
            L.or_degrees.restype = i
            L.or_eval.argtypes = [i, i, i, i, _I32P, _I32P, _I32P, _I32P, _F64P, i, _F64P, d,
                                  _F64P, _F64P, p, ct.POINTER(ct.c_long)]
            L.or_eval.restype = i
            L.or_eval_threads.argtypes = [i, i, i, _I32P, _I32P, _I32P, _I32P, _F64P, i, _F64P,
                                          d, _F64P, _F64P, p, i]
            L.or_eval_threads.restype = i
            L.or_solve.argtypes = [i, i, _F64P, _F64P, _F64P]
            L.or_solve.restype = i
            L.or_newton_step.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P, _F64P, i, d, _F64P,
                                         _F64P, i, i, _F64P,
                                         np.ctypeslib.ndpointer(dtype=np.int32),
                                         np.ctypeslib.ndpointer(dtype=np.int32)]
            L.or_newton_step.restype = i
            L.or_newton_threads.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P, _F64P, i, d, _F64P,
                                            _F64P, i, i, _F64P,
                                            np.ctypeslib.ndpointer(dtype=np.int32),
                                            np.ctypeslib.ndpointer(dtype=np.int32), i]
            L.or_newton_threads.restype = i
            L.or_track.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P, _F64P, _F64P, _F64P,
                                   ct.POINTER(TrackOpts), _F64P, ct.POINTER(_Stats), p,
                                   ct.POINTER(ct.c_int32)]
            L.or_track.restype = i
            L.or_track_replay.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P, _F64P, _F64P, _F64P,
                                          ct.POINTER(TrackOpts), _F64P, i, _F64P,
                                          ct.POINTER(ct.c_int32), ct.POINTER(_Stats)]
            L.or_track_replay.restype = i
            L.or_track_resume.argtypes = [i, i, _I32P, _I32P, _I32P, _I32P, _F64P, _F64P,
                                          ct.POINTER(TrackOpts), ct.POINTER(PathState), _F64P,
                                          _F64P, _F64P, ct.c_int64, ct.POINTER(_Stats), p,
                                          ct.POINTER(ct.c_int32)]
            L.or_track_resume.restype = i
            L.or_predict.argtypes = [i, i, i, i, d, d, d, d, _F64P, _F64P, _F64P, _F64P]
            L.or_predict.restype = i
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _binop(name, L, a, b, width):
    out = np.zeros(width, dtype=np.float64)
    rc = getattr(lib(), name)(L, _f64(a, width), _f64(b, width), out)
    if rc != 0:
        raise ValueError(f"{name} failed ({rc})")
    return out


def r_add(L, a, b):
    return _binop("or_r_add", L, a, b, L)


def r_mul(L, a, b):
    return _binop("or_r_mul", L, a, b, L)


def r_div(L, a, b):
    return _binop("or_r_div", L, a, b, L)


def c_mul(L, a, b):
    return _binop("or_c_mul", L, a, b, 2 * L).reshape(2, L)


def c_div(L, a, b):
    return _binop("or_c_div", L, a, b, 2 * L).reshape(2, L)


def _sysargs(sysd):
    return (np.ascontiguousarray(sysd["mon_ptr"], dtype=np.int32),
            np.ascontiguousarray(sysd["var_ptr"], dtype=np.int32),
            np.ascontiguousarray(sysd["var_idx"], dtype=np.int32),
            np.ascontiguousarray(sysd["var_exp"], dtype=np.int32))


def validate(sysd) -> int:
    return lib().or_validate(sysd["n"], sysd["npoly"], *_sysargs(sysd))


def degrees(sysd) -> np.ndarray:
    mp, vp, vi, ve = _sysargs(sysd)
    deg = np.zeros(sysd["npoly"], dtype=np.int32)
    lib().or_degrees(sysd["npoly"], mp, vp, ve, deg)
    return deg


def evaluate(sysd, coef, x, t=-1.0, gamma=(1.0, 0.0), mode=1, jac=True):
    """f (and J) at the points x[npts][n][2][L]; t < 0 evaluates f, t >= 0 the homotopy.
    Returns (f, J or None, number of multiplications spent on the omega products)."""
    L = coef.shape[-1]
    n, npoly = sysd["n"], sysd["npoly"]
    x = _f64(x)
    npts = x.shape[0]
    f = np.zeros((npts, npoly, 2, L))
    J = np.zeros((npts, npoly, n, 2, L)) if jac else None
    cnt = ct.c_long(0)
    rc = lib().or_eval(L, mode, n, npoly, *_sysargs(sysd), _f64(coef), npts, x, float(t),
                       _f64(gamma), f, J.ctypes.data_as(ct.c_void_p) if jac else None,
                       ct.byref(cnt))
    if rc != 0:
        raise ValueError(f"or_eval failed ({rc})")
    return f, J, cnt.value


def evaluate_threads(sysd, coef, x, t=-1.0, gamma=(1.0, 0.0), nthreads=None):
    """Same as evaluate(mode=1, jac=True) split over POSIX threads (CPU baseline)."""
    L = coef.shape[-1]
    n, npoly = sysd["n"], sysd["npoly"]
    x = _f64(x)
    npts = x.shape[0]
    f = np.zeros((npts, npoly, 2, L))
    J = np.zeros((npts, npoly, n, 2, L))
    nthreads = nthreads or os.cpu_count() or 1
    rc = lib().or_eval_threads(L, n, npoly, *_sysargs(sysd), _f64(coef), npts, x, float(t),
                               _f64(gamma), f, J.ctypes.data_as(ct.c_void_p), nthreads)
    if rc != 0:
        raise ValueError(f"or_eval_threads failed ({rc})")
    return f, J


def solve(A, b):
    """Gaussian elimination with partial pivoting (Sec. 4).  A[n][n][2][L], b[n][2][L]."""
    A = _f64(A)
    b = _f64(b)
    n, L = A.shape[0], A.shape[-1]
    x = np.zeros((n, 2, L))
    rc = lib().or_solve(L, n, A, b, x)
    if rc < 0:
        raise ValueError("or_solve failed")
    return x, rc


def newton_step(sysd, coef, x, t, gamma, lu_mode=0, max_refine=4):
    """One Newton iteration per point (Alg. 4.1 loop body).  Returns
    (x_new, res_norm (pre-update), status, refinement sweeps)."""
    L = coef.shape[-1]
    x = _f64(x).copy()
    npts = x.shape[0]
    res = np.zeros(npts)
    st = np.zeros(npts, dtype=np.int32)
    sw = np.zeros(npts, dtype=np.int32)
    rc = lib().or_newton_step(L, sysd["n"], *_sysargs(sysd), _f64(coef), npts, float(t),
                              _f64(gamma), x, lu_mode, max_refine, res, st, sw)
    if rc != 0:
        raise ValueError(f"or_newton_step failed ({rc})")
    return x, res, st, sw


def newton_threads(sysd, coef, x, t, gamma, lu_mode=0, max_refine=4, nthreads=None):
    """newton_step split over POSIX threads (CPU baseline)."""
    L = coef.shape[-1]
    x = _f64(x).copy()
    npts = x.shape[0]
    res = np.zeros(npts)
    st = np.zeros(npts, dtype=np.int32)
    sw = np.zeros(npts, dtype=np.int32)
    nthreads = nthreads or os.cpu_count() or 1
    rc = lib().or_newton_threads(L, sysd["n"], *_sysargs(sysd), _f64(coef), npts, float(t),
                                 _f64(gamma), x, lu_mode, max_refine, res, st, sw, nthreads)
    if rc != 0:
        raise ValueError(f"or_newton_threads failed ({rc})")
    return x, res, st, sw


@dataclass
class TrackResult:
    x: np.ndarray
    status: int
    n_succ: int
    n_corr: int
    newton_its: int
    min_step: float
    avg_step: float
    t_end: float
    res_end: float
    end_its: int
    log: np.ndarray | None


def track(sysd, coef, x0, gamma, opts: TrackOpts, log_cap=0):
    """Track one path of h(x,t) = gamma (1-t) g(x) + t f(x) from x0 (Alg. 3.1)."""
    L = coef.shape[-1]
    n = sysd["n"]
    x1 = np.zeros((n, 2, L))
    st = _Stats()
    o = TrackOpts()
    ct.pointer(o)[0] = opts
    o.log_cap = int(log_cap)
    logbuf = (_StepLog * max(1, log_cap))()
    nl = ct.c_int32(0)
    rc = lib().or_track(L, n, *_sysargs(sysd), _f64(coef), _f64(gamma), _f64(x0),
                        ct.byref(o), x1, ct.byref(st), ct.cast(logbuf, ct.c_void_p),
                        ct.byref(nl))
    if rc != 0:
        raise ValueError(f"or_track failed ({rc})")
    log = _log_array(logbuf, nl.value) if log_cap else None
    return TrackResult(x1, st.status, st.n_succ, st.n_corr, st.newton_its, st.min_step,
                       st.avg_step, st.t_end, st.res_end, st.end_its, log)


def _log_array(logbuf, count):
    return np.array([(r.t, r.lam, r.res_first, r.res_last, r.pc_dist, r.iters, r.accepted)
                     for r in logbuf[:count]],
                    dtype=[("t", "f8"), ("lam", "f8"), ("res_first", "f8"), ("res_last", "f8"),
                           ("pc_dist", "f8"), ("iters", "i4"), ("accepted", "i4")])


def track_resume(sysd, coef, gamma, opts: TrackOpts, state: PathState, z, zp, zpp, max_stages,
                 log_cap=0):
    """At most max_stages corrector stages of one path from `state` (phase 0: start at
    t = 0 from z), then the end game if t = 1 is reached.  z, zp, zpp: [n][2][L], the
    current point and the two accepted points before it.  Returns (new state, z, zp, zpp,
    statistics dict, log or None); the arguments are not modified."""
    L = coef.shape[-1]
    n = sysd["n"]
    st = PathState()
    ct.pointer(st)[0] = state
    zz, zzp, zzpp = (_f64(v, (n, 2, L)).copy() for v in (z, zp, zpp))
    stats = _Stats()
    o = TrackOpts()
    ct.pointer(o)[0] = opts
    o.log_cap = int(log_cap)
    logbuf = (_StepLog * max(1, log_cap))()
    nl = ct.c_int32(0)
    rc = lib().or_track_resume(L, n, *_sysargs(sysd), _f64(coef), _f64(gamma), ct.byref(o),
                               ct.byref(st), zz, zzp, zzpp, int(max_stages), ct.byref(stats),
                               ct.cast(logbuf, ct.c_void_p), ct.byref(nl))
    if rc != 0:
        raise ValueError(f"or_track_resume failed ({rc})")
    sd = {k: getattr(stats, k) for k, _ in _Stats._fields_}
    return st, zz, zzp, zzpp, sd, (_log_array(logbuf, nl.value) if log_cap else None)


def predict(L, predictor, nhist, t, tp, tpp, t1, z, zp, zpp):
    """The tracker's predictor (Alg. 3.1; Sec. 5 quadratic) at t1 from the accepted points
    z (at t), zp (at tp), zpp (at tpp), each [n][2][L]; nhist of them exist.
    predictor 0 secant, 1 quadratic."""
    z = _f64(z)
    n = z.shape[0]
    out = np.zeros((n, 2, L))
    rc = lib().or_predict(L, n, int(predictor), int(nhist), float(t), float(tp), float(tpp),
                          float(t1), _f64(z, (n, 2, L)), _f64(zp, (n, 2, L)), _f64(zpp, (n, 2, L)),
                          out)
    if rc != 0:
        raise ValueError(f"or_predict failed ({rc})")
    return out


def track_replay(sysd, coef, x0, gamma, opts: TrackOpts, tseq):
    """Follow the accepted parameter values tseq with the tracker's predictor and
    corrector (and the end game).  Returns (end point, status, index of the first
    rejected stage or -1)."""
    L = coef.shape[-1]
    n = sysd["n"]
    x1 = np.zeros((n, 2, L))
    st = _Stats()
    fail = ct.c_int32(-1)
    t = np.ascontiguousarray(tseq, dtype=np.float64)
    rc = lib().or_track_replay(L, n, *_sysargs(sysd), _f64(coef), _f64(gamma), _f64(x0),
                               ct.byref(opts), t, len(t), x1, ct.byref(fail), ct.byref(st))
    if rc != 0:
        raise ValueError(f"or_track_replay failed ({rc})")
    return x1, st.status, fail.value
