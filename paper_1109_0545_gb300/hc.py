"""Thin ctypes binding of ``libhc.so`` (declared in ``include/hc.h``).

The functions carry the C names and only marshal arguments: device buffers are torch
CUDA tensors (or raw integer pointers), streams are torch streams.  Every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing, :func:`load` raises.

Layout helpers convert complex numpy arrays to and from the library's
structure-of-arrays layout ``[2][L][rows...][npts]`` (re limbs, im limbs; point index
fastest).
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

HC_SUCCESS, HC_EINVAL, HC_ENOMEM, HC_ECUDA, HC_ENOTIMPL, HC_ETIMEOUT = 0, -1, -2, -3, -4, -5
HC_OK, HC_NOCONV, HC_SINGULAR, HC_MIN_STEP, HC_MAX_STEPS, HC_DIVERGED, HC_NONFINITE = range(7)
STATUS_NAMES = {0: "OK", 1: "NOCONV", 2: "SINGULAR", 3: "MIN_STEP", 4: "MAX_STEPS",
                5: "DIVERGED", 6: "NONFINITE"}
HC_LU_NATIVE, HC_LU_FP64_REFINE = 0, 1

_lock = threading.Lock()
_lib = None


class TrackOpts(ct.Structure):
    """hc_track_opts (include/hc.h)."""
    _fields_ = [("lambda0", ct.c_double), ("lambda_min", ct.c_double),
                ("lambda_max", ct.c_double), ("grow", ct.c_double), ("shrink", ct.c_double),
                ("eps", ct.c_double), ("eps_x", ct.c_double), ("eps_end", ct.c_double),
                ("eps_end_x", ct.c_double), ("div_bound", ct.c_double),
                ("max_it", ct.c_int32), ("end_it", ct.c_int32), ("grow_after", ct.c_int32),
                ("max_steps", ct.c_int32), ("predictor", ct.c_int32), ("lu_mode", ct.c_int32),
                ("max_refine", ct.c_int32), ("mode", ct.c_int32), ("graph_steps", ct.c_int32),
                ("reserved", ct.c_int32), ("proposer", ct.c_void_p), ("proposer_margin", ct.c_double),
                ("explore", ct.c_double), ("explore_seed", ct.c_uint64)]


class PathStats(ct.Structure):
    """hc_path_stats (include/hc.h)."""
    _fields_ = [("n_succ", ct.c_int64), ("n_corr", ct.c_int64), ("newton_its", ct.c_int64),
                ("min_step", ct.c_double), ("avg_step", ct.c_double), ("t_end", ct.c_double),
                ("res_end", ct.c_double), ("status", ct.c_int32), ("end_its", ct.c_int32)]


class PathState(ct.Structure):
    """hc_path_state (include/hc.h): a path's state between calls of hc_track_resume."""
    _fields_ = [("t", ct.c_double), ("tp", ct.c_double), ("tpp", ct.c_double),
                ("lambda_", ct.c_double), ("minstep", ct.c_double), ("sumstep", ct.c_double),
                ("res_end", ct.c_double), ("pad", ct.c_double), ("n_succ", ct.c_int64),
                ("n_corr", ct.c_int64), ("nits", ct.c_int64), ("nhist", ct.c_int32),
                ("consec", ct.c_int32), ("status", ct.c_int32), ("phase", ct.c_int32),
                ("end_its", ct.c_int32), ("pad2", ct.c_int32), ("hl", ct.c_double * 3),
                ("hr", ct.c_double * 3), ("pcd", ct.c_double), ("cond", ct.c_double),
                ("hi", ct.c_int32 * 3), ("pad3", ct.c_int32), ("lam_plain", ct.c_double),
                ("pid", ct.c_int64)]


STEP_RECORD_DTYPE = np.dtype([("t", "f8"), ("lam", "f8"), ("res_first", "f8"), ("res_last", "f8"),
                              ("pc_dist", "f8"), ("cond_log10", "f8"), ("iters", "i4"),
                              ("accepted", "i4")])
HC_PRED_SECANT, HC_PRED_QUADRATIC, HC_PRED_TANGENT = 0, 1, 2
HC_EVAL_AUTO, HC_EVAL_PER_TERM, HC_EVAL_SHARED = 0, 1, 2
HC_TRACK_PERSISTENT, HC_TRACK_GRAPH, HC_TRACK_GRID = 0, 1, 2


class HCError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with code {code}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libhc.so (building it first if allowed).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libhc.so not built at {path}")
            _build.build()
        L = ct.CDLL(path)
        vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
        i32p = ct.POINTER(ct.c_int32)
        L.hc_system_load.argtypes = [ct.POINTER(vp), i, i, i32p, i32p, i32p, i32p,
                                     ct.POINTER(ct.c_double), i, ct.POINTER(ct.c_double)]
        L.hc_system_load.restype = i
        L.hc_system_free.argtypes = [vp]
        L.hc_system_free.restype = None
        L.hc_system_info.argtypes = [vp] + [ct.POINTER(ct.c_int)] * 7
        L.hc_system_info.restype = i
        L.hc_eval_jac.argtypes = [vp, i, d, vp, vp, vp, vp]
        L.hc_eval_jac.restype = i
        L.hc_newton_step.argtypes = [vp, i, d, vp, i, i, vp, vp, vp, vp]
        L.hc_newton_step.restype = i
        L.hc_last_error.argtypes = []
        L.hc_last_error.restype = ct.c_char_p
        L.hc_probe_fp64_peak.argtypes = [ct.POINTER(ct.c_double)]
        L.hc_probe_fp64_peak.restype = i
        L.hc_set_tiles.argtypes = [i, i]
        L.hc_set_tiles.restype = i
        L.hc_track_opts_default.argtypes = [ct.POINTER(TrackOpts)]
        L.hc_track_opts_default.restype = None
        L.hc_track_path.argtypes = [ct.POINTER(vp), i, vp, vp, ct.POINTER(TrackOpts),
                                    ct.POINTER(PathStats), vp, i, vp]
        L.hc_track_path.restype = i
        L.hc_track_resume.argtypes = [ct.POINTER(vp), i, vp, vp, ct.POINTER(PathState), i,
                                      ct.POINTER(TrackOpts), ct.POINTER(PathStats), vp, i, vp]
        L.hc_track_resume.restype = i
        L.hc_set_track_tiles.argtypes = [i, i, i, i]
        L.hc_set_track_tiles.restype = i
        L.hc_get_track_tiles.argtypes = [ct.POINTER(ct.c_int)] * 4
        L.hc_get_track_tiles.restype = i
        f = ct.c_float
        L.hc_mlp_grad.argtypes = [vp, i, vp, vp, vp, f, vp, vp, vp]
        L.hc_mlp_grad.restype = i
        L.hc_mlp_adamw.argtypes = [vp, vp, vp, vp, i, f, f, f, f, f, vp]
        L.hc_mlp_adamw.restype = i
        L.hc_mlp_forward.argtypes = [vp, i, vp, vp, vp]
        L.hc_mlp_forward.restype = i
        L.hc_system_set_eval_mode.argtypes = [vp, i]
        L.hc_system_set_eval_mode.restype = i
        L.hc_system_eval_mode.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
        L.hc_system_eval_mode.restype = i
        L.hc_eval_jac_noalloc.argtypes = [vp, i, d, vp, vp, vp, vp]
        L.hc_eval_jac_noalloc.restype = i
        L.hc_prof_enable.argtypes = [i]
        L.hc_prof_enable.restype = i
        L.hc_prof_read.argtypes = [ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)]
        L.hc_prof_read.restype = i
        _lib = L
        return L


def hc_last_error() -> str:
    return load().hc_last_error().decode()


def _check(fn: str, rc: int) -> int:
    if rc != HC_SUCCESS:
        raise HCError(fn, rc, hc_last_error())
    return rc


def _ptr(a) -> int | None:
    """Device pointer of a torch tensor (or an int pointer / None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ct.POINTER(ct.c_int32))


class System:
    """An uploaded system (hc_system_load); frees itself (hc_system_free)."""

    def __init__(self, handle, n, npoly, prec):
        self.handle = handle
        self.n, self.npoly, self.prec = n, npoly, prec

    def info(self) -> dict:
        vals = [ct.c_int() for _ in range(7)]
        _check("hc_system_info", load().hc_system_info(self.handle, *[ct.byref(v) for v in vals]))
        keys = ("n", "npoly", "nmon", "nvar", "prec", "max_exp", "max_deg")
        return {k: v.value for k, v in zip(keys, vals)}

    def set_eval_mode(self, mode: int) -> None:
        """hc_system_set_eval_mode: HC_EVAL_AUTO, HC_EVAL_PER_TERM or HC_EVAL_SHARED."""
        _check("hc_system_set_eval_mode", load().hc_system_set_eval_mode(self.handle, int(mode)))

    def eval_mode(self) -> tuple[int, float, float]:
        """hc_system_eval_mode: (scheme in use, FP64 per point per term, FP64 per point shared)."""
        a, b = ct.c_double(), ct.c_double()
        r = load().hc_system_eval_mode(self.handle, ct.byref(a), ct.byref(b))
        if r < 0:
            _check("hc_system_eval_mode", r)
        return r, a.value, b.value

    def free(self):
        if self.handle:
            load().hc_system_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hc_system_load(n, npoly, mon_ptr, var_ptr, var_idx, var_exp, coef, prec, gamma) -> System:
    """coef: float64 [nmon][2][L]; gamma: (re, im)."""
    L = load()
    mp, mpp = _i32(mon_ptr)
    vp, vpp = _i32(var_ptr)
    vi, vip = _i32(var_idx if len(var_idx) else np.zeros(1, np.int32))
    ve, vep = _i32(var_exp if len(var_exp) else np.ones(1, np.int32))
    c = np.ascontiguousarray(coef, dtype=np.float64)
    g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(2))
    h = ct.c_void_p()
    _check("hc_system_load", L.hc_system_load(
        ct.byref(h), int(n), int(npoly), mpp, vpp, vip, vep,
        c.ctypes.data_as(ct.POINTER(ct.c_double)), int(prec),
        g.ctypes.data_as(ct.POINTER(ct.c_double))))
    return System(h.value, int(n), int(npoly), int(prec))


def system_from(s, prec: int, gamma: complex) -> System:
    """Load a :class:`paper_1109_0545_gb300.synth.System`."""
    return hc_system_load(s.n, s.npoly, s.mon_ptr, s.var_ptr, s.var_idx, s.var_exp,
                          s.coef_limbs(prec), prec, (gamma.real, gamma.imag))


def hc_eval_jac(sys: System, npts: int, t: float, x, f, J=None, stream=None) -> None:
    _check("hc_eval_jac", load().hc_eval_jac(sys.handle, int(npts), float(t), _ptr(x), _ptr(f),
                                             _ptr(J), _stream(stream)))


def hc_eval_jac_noalloc(sys: System, npts: int, t: float, x, f, J=None, stream=None) -> None:
    """hc_eval_jac with the library's fixed 32 MiB device workspace: allocates nothing."""
    _check("hc_eval_jac_noalloc", load().hc_eval_jac_noalloc(
        sys.handle, int(npts), float(t), _ptr(x), _ptr(f), _ptr(J), _stream(stream)))


def hc_newton_step(sys: System, npts: int, t: float, x, lu_mode: int, max_refine: int,
                   res_norm, status, sweeps=None, stream=None) -> None:
    _check("hc_newton_step", load().hc_newton_step(
        sys.handle, int(npts), float(t), _ptr(x), int(lu_mode), int(max_refine), _ptr(res_norm),
        _ptr(status), _ptr(sweeps), _stream(stream)))


def hc_track_opts_default(**over) -> TrackOpts:
    o = TrackOpts()
    load().hc_track_opts_default(ct.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def hc_track_path(systems, x0, x1, opts: TrackOpts, log=None, log_cap: int = 0,
                  stream=None) -> list[dict]:
    """Track one path per system (a system may repeat).  x0/x1: device buffers packed
    path after path ([2][L][n_p] each); log: device buffer of hc_step_record."""
    handles = (ct.c_void_p * len(systems))(*[s.handle for s in systems])
    stats = (PathStats * len(systems))()
    _check("hc_track_path", load().hc_track_path(handles, len(systems), _ptr(x0), _ptr(x1),
                                                 ct.byref(opts), stats, _ptr(log), int(log_cap),
                                                 _stream(stream)))
    keys = [f[0] for f in PathStats._fields_]
    return [{k: getattr(st, k) for k in keys} for st in stats]


def new_states(npaths: int):
    """npaths zeroed hc_path_state records: phase 0, start at t = 0 from x."""
    return (PathState * npaths)()


def hc_track_resume(systems, x, hist, states, max_stages: int, opts: TrackOpts, log=None,
                    log_cap: int = 0, stream=None) -> list[dict]:
    """Advance each path by at most max_stages corrector stages from its state (updated
    in place, a ctypes array of PathState from new_states); x, hist: device buffers in
    the packings of hc_track_resume (x as pack_paths, hist 3 vectors per path)."""
    handles = (ct.c_void_p * len(systems))(*[s.handle for s in systems])
    stats = (PathStats * len(systems))()
    _check("hc_track_resume", load().hc_track_resume(handles, len(systems), _ptr(x), _ptr(hist), states,
                                                     int(max_stages), ct.byref(opts), stats, _ptr(log),
                                                     int(log_cap), _stream(stream)))
    keys = [f[0] for f in PathStats._fields_]
    return [{k: getattr(st, k) for k in keys} for st in stats]


def pack_hist(prev: list[np.ndarray], prev2: list[np.ndarray], L: int) -> np.ndarray:
    """The hist packing of hc_track_resume from per-path previous points (limbs [n][2][L]
    each); the tangent slot is zero."""
    out = []
    for a, b in zip(prev, prev2):
        n = a.shape[0]
        out += [pack_paths([a]), pack_paths([b]), np.zeros(2 * L * n)]
    return np.concatenate(out)


def unpack_hist(buf: np.ndarray, dims: list[int], L: int):
    """Inverse of pack_hist: lists of previous and second previous points (limbs)."""
    prev, prev2, o = [], [], 0
    for n in dims:
        w = 2 * L * n
        prev += unpack_paths(buf[o:o + w], [n], L)
        prev2 += unpack_paths(buf[o + w:o + 2 * w], [n], L)
        o += 3 * w
    return prev, prev2


def pack_paths(points: list[np.ndarray]) -> np.ndarray:
    """Start points (each limbs [n_p][2][L]) -> the packed layout of hc_track_path."""
    return np.concatenate([np.ascontiguousarray(np.transpose(p, (1, 2, 0))).ravel() for p in points])


def unpack_paths(buf: np.ndarray, dims: list[int], L: int) -> list[np.ndarray]:
    """Inverse of pack_paths: list of limbs [n_p][2][L]."""
    out, o = [], 0
    for n in dims:
        out.append(np.ascontiguousarray(np.transpose(buf[o:o + 2 * L * n].reshape(2, L, n), (2, 0, 1))))
        o += 2 * L * n
    return out


HC_MLP_IN, HC_MLP_NPARAM = 12, 5057


def hc_mlp_grad(params, nrec, feat, target, accepted, kappa, grad, loss=None, stream=None):
    _check("hc_mlp_grad", load().hc_mlp_grad(_ptr(params), int(nrec), _ptr(feat), _ptr(target),
                                             _ptr(accepted), float(kappa), _ptr(grad), _ptr(loss),
                                             _stream(stream)))


def hc_mlp_adamw(params, m1, m2, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4,
                 stream=None):
    _check("hc_mlp_adamw", load().hc_mlp_adamw(_ptr(params), _ptr(m1), _ptr(m2), _ptr(grad),
                                               int(step), float(lr), float(beta1), float(beta2),
                                               float(eps), float(wd), _stream(stream)))


def hc_mlp_forward(params, nrec, feat, out, stream=None):
    _check("hc_mlp_forward", load().hc_mlp_forward(_ptr(params), int(nrec), _ptr(feat), _ptr(out),
                                                   _stream(stream)))


def hc_probe_fp64_peak() -> float:
    v = ct.c_double()
    _check("hc_probe_fp64_peak", load().hc_probe_fp64_peak(ct.byref(v)))
    return v.value


def hc_set_tiles(rows_per_task: int, blocks_per_sm: int) -> None:
    _check("hc_set_tiles", load().hc_set_tiles(int(rows_per_task), int(blocks_per_sm)))


def hc_set_track_tiles(threads_per_block: int = 0, blocks_per_sm: int = 0, factors: int = 0,
                       grid_chunk: int = 0) -> None:
    """Execution shape of the tracker for later calls (0 = automatic): threads per path
    block (64, 128, 256; 512 in double and double-double), path blocks per SM, FP64 factors
    in shared (0, 1) or global (2) memory, and the whole-GPU engine's chunk length."""
    _check("hc_set_track_tiles", load().hc_set_track_tiles(int(threads_per_block), int(blocks_per_sm),
                                                           int(factors), int(grid_chunk)))


def hc_get_track_tiles() -> dict:
    v = [ct.c_int() for _ in range(4)]
    _check("hc_get_track_tiles", load().hc_get_track_tiles(*[ct.byref(x) for x in v]))
    return dict(zip(("threads_per_block", "blocks_per_sm", "factors", "grid_chunk"), (x.value for x in v)))


def hc_prof_enable(on: bool) -> None:
    _check("hc_prof_enable", load().hc_prof_enable(1 if on else 0))


def hc_prof_read() -> tuple[float, int]:
    ms, n = ct.c_double(), ct.c_int()
    _check("hc_prof_read", load().hc_prof_read(ct.byref(ms), ct.byref(n)))
    return ms.value, n.value


# ----------------------------------------------------------------------------- layouts
def to_soa(z: np.ndarray, L: int, limbs: np.ndarray | None = None) -> np.ndarray:
    """complex [npts][rows...] (leading limbs) or limbs [npts][rows...][2][L] ->
    float64 [2][L][rows...][npts]."""
    if limbs is None:
        z = np.asarray(z, dtype=np.complex128)
        limbs = np.zeros(z.shape + (2, L))
        limbs[..., 0, 0] = z.real
        limbs[..., 1, 0] = z.imag
    nd = limbs.ndim
    # [npts, rows..., 2, L] -> [2, L, rows..., npts]
    perm = (nd - 2, nd - 1) + tuple(range(1, nd - 2)) + (0,)
    return np.ascontiguousarray(np.transpose(limbs, perm))


def from_soa(a: np.ndarray) -> np.ndarray:
    """float64 [2][L][rows...][npts] -> limbs [npts][rows...][2][L]."""
    nd = a.ndim
    perm = (nd - 1,) + tuple(range(2, nd - 1)) + (0, 1)
    return np.ascontiguousarray(np.transpose(a, perm))
