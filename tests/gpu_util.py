"""Shared set-up of the GPU parity tests: systems and points from the seeded generator,
uploaded through the library's binding; oracle values from ``oracle``."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1109_0545_gb300 import hc, synth


def torch_cuda():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_eval(torch, s, gamma, L, pts_limbs, t, jac=True, mode=None):
    """Evaluate on the GPU (evaluation scheme `mode`, default the library's choice);
    returns (f, J) as limbs [npts][rows][(n)][2][L]."""
    sysh = hc.system_from(s, L, gamma)
    if mode is not None:
        sysh.set_eval_mode(mode)
    npts = pts_limbs.shape[0]
    x = dev(torch, hc.to_soa(None, L, pts_limbs))
    f = torch.zeros((2, L, s.npoly, npts), dtype=torch.float64, device="cuda")
    J = torch.zeros((2, L, s.npoly, s.n, npts), dtype=torch.float64, device="cuda") if jac else None
    hc.hc_eval_jac(sysh, npts, t, x, f, J)
    torch.cuda.synchronize()
    fo = hc.from_soa(f.cpu().numpy())
    Jo = hc.from_soa(J.cpu().numpy()) if jac else None
    sysh.free()
    return fo, Jo


def oracle_eval(s, gamma, L, pts_limbs, t, jac=True, threads=True):
    g = np.array([gamma.real, gamma.imag])
    if threads and jac:
        return oracle.evaluate_threads(s.as_dict(), s.coef_limbs(L), pts_limbs, t, g)
    f, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), pts_limbs, t, g, mode=1, jac=jac)
    return f, J


def gpu_newton(torch, s, gamma, L, pts_limbs, t, lu_mode, max_refine=4, mode=None):
    sysh = hc.system_from(s, L, gamma)
    if mode is not None:
        sysh.set_eval_mode(mode)
    npts = pts_limbs.shape[0]
    x = dev(torch, hc.to_soa(None, L, pts_limbs))
    res = torch.zeros(npts, dtype=torch.float64, device="cuda")
    st = torch.full((npts,), -1, dtype=torch.int32, device="cuda")
    sw = torch.full((npts,), -1, dtype=torch.int32, device="cuda")
    hc.hc_newton_step(sysh, npts, t, x, lu_mode, max_refine, res, st, sw)
    torch.cuda.synchronize()
    out = (hc.from_soa(x.cpu().numpy()), res.cpu().numpy(), st.cpu().numpy(), sw.cpu().numpy())
    sysh.free()
    return out


def limbs_of(pts, L):
    return synth.limbs(pts, L)
