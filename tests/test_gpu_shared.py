"""The shared-monomial evaluation scheme (HC_EVAL_SHARED) against the oracle: a system
with a common support (all polynomials on one set of monomials, the shape behind Table 1)
and general sparse systems, values and Jacobians of f and of the homotopy, in complex
double / DD / QD, several 32-point tiles with a ragged tail; the Newton step on it; and the
load-time choice of the scheme."""
import numpy as np
import pytest

from helpers import TOL, digits, rel_err_per_point
from gpu_util import gpu_eval, gpu_newton, limbs_of, oracle_eval, torch_cuda
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("t", [-1.0, 0.6])
def test_common_support_matches_oracle_in_both_schemes(L, t):
    torch = torch_cuda()
    s, gamma = synth.common_support_system(11, n=8, nuniq=20, dmax=12)
    rng = np.random.default_rng(500 + L)
    pts = limbs_of(synth.torus_points(rng, 70, 8), L)
    fo, Jo = oracle_eval(s, gamma, L, pts, t)
    for mode in (hc.HC_EVAL_SHARED, hc.HC_EVAL_PER_TERM):
        f, J = gpu_eval(torch, s, gamma, L, pts, t, mode=mode)
        ef, eJ = rel_err_per_point(f, fo), rel_err_per_point(J, Jo)
        print(f"L={L} t={t} mode={mode}: f {digits(ef):.1f} digits, J {digits(eJ):.1f} digits")
        assert np.all(ef <= TOL[L]) and np.all(eJ <= TOL[L])


@pytest.mark.parametrize("L", [2, 4])
def test_shared_scheme_on_a_general_system_with_constants(L):
    """Every structure the per-term kernel handles: constants, k = 1, repeated monomials
    within a polynomial, values only."""
    torch = torch_cuda()
    rng = np.random.default_rng(510)
    s = synth.random_system(rng, 7, (3, 9), (1, 4), (1, 4), const_term=True)
    gamma = synth.unit_complex(rng)
    pts = limbs_of(synth.torus_points(rng, 45, 7), L)
    for jac in (True, False):
        fo, Jo = oracle_eval(s, gamma, L, pts, 0.3, jac=jac)
        f, J = gpu_eval(torch, s, gamma, L, pts, 0.3, jac=jac, mode=hc.HC_EVAL_SHARED)
        assert np.all(rel_err_per_point(f, fo) <= TOL[L])
        if jac:
            assert np.all(rel_err_per_point(J, Jo) <= TOL[L])


def test_newton_step_with_shared_scheme_matches_oracle():
    torch = torch_cuda()
    s, gamma = synth.common_support_system(12, n=10, nuniq=30, dmax=10)
    rng = np.random.default_rng(520)
    pts = limbs_of(synth.torus_points(rng, 40, 10), 2)
    x, res, st, sw = gpu_newton(torch, s, gamma, 2, pts, 0.5, hc.HC_LU_FP64_REFINE, max_refine=6,
                                mode=hc.HC_EVAL_SHARED)
    xo, reso, sto, swo = oracle.newton_step(s.as_dict(), s.coef_limbs(2), pts, 0.5,
                                            np.array([gamma.real, gamma.imag]), hc.HC_LU_FP64_REFINE, 6)
    assert np.array_equal(st, sto)
    assert np.allclose(res, reso, rtol=1e-12, atol=0)
    assert np.all(rel_err_per_point(x, xo) <= TOL[2])


def test_scheme_choice_at_load():
    torch_cuda()
    s, g = synth.common_support_system(1)            # 40 x 200 shared monomials
    h = hc.system_from(s, 2, g)
    mode, ops_term, ops_shared = h.eval_mode()
    assert mode == hc.HC_EVAL_SHARED and ops_shared < 0.5 * ops_term
    h.set_eval_mode(hc.HC_EVAL_PER_TERM)
    assert h.eval_mode()[0] == hc.HC_EVAL_PER_TERM
    h.set_eval_mode(hc.HC_EVAL_AUTO)
    assert h.eval_mode()[0] == hc.HC_EVAL_SHARED
    with pytest.raises(hc.HCError):
        h.set_eval_mode(7)
    h.free()
    s2, _, g2 = synth.eval_throughput(2, npts=32)      # distinct monomials: per term
    h2 = hc.system_from(s2, 2, g2)
    assert h2.eval_mode()[0] == hc.HC_EVAL_PER_TERM
    h2.free()


def test_shared_scheme_edge_cases():
    """A monomial repeated inside one polynomial and across polynomials, a polynomial that is
    only a constant, k = 1 and k = 32 monomials, exponent 64, a ragged tile, and npts = 0."""
    torch = torch_cuda()
    n = 32
    # poly 0: x0^3 x5, x0^3 x5 again, constant; poly 1: constant only;
    # poly 2: all 32 variables, x0^3 x5 (shared with poly 0), x31^64
    idx = [0, 5, 0, 5] + list(range(32)) + [0, 5, 31]
    ex = [3, 1, 3, 1] + [1] * 16 + [2] * 16 + [3, 1, 64]
    var_ptr = [0, 2, 4, 4, 4, 36, 38, 39]
    s = synth.System(n=n, npoly=3, mon_ptr=np.array([0, 3, 4, 7], np.int32),
                     var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                     var_exp=np.array(ex, np.int32), coef=np.exp(1j * np.arange(7.0)))
    rng = np.random.default_rng(530)
    gamma = synth.unit_complex(rng)
    for L in (2, 4):
        pts = limbs_of(synth.torus_points(rng, 37, n), L)
        fo, Jo = oracle_eval(s, gamma, L, pts, -1.0)
        f, J = gpu_eval(torch, s, gamma, L, pts, -1.0, mode=hc.HC_EVAL_SHARED)
        assert np.all(rel_err_per_point(f, fo) <= TOL[L])
        assert np.all(rel_err_per_point(J, Jo) <= TOL[L])
    h = hc.system_from(s, 2, gamma)
    h.set_eval_mode(hc.HC_EVAL_SHARED)
    x = torch.zeros((2, 2, n, 1), dtype=torch.float64, device="cuda")
    f = torch.full((2, 2, 3, 1), 7.0, dtype=torch.float64, device="cuda")
    hc.hc_eval_jac(h, 0, -1.0, x, f, None)    # npts = 0: nothing is written
    torch.cuda.synchronize()
    assert torch.all(f == 7.0)
    h.free()


def test_table1_system_full_size_sampled():
    """Table 1's common-support system (40 x 40, 200 shared monomials, degree up to 80) at
    8,192 points, the benchmark's launch (five row groups per 32-point tile): both schemes
    agree at every point within the DD tolerance, and the oracle checks 6 sampled points
    (first and last, and in different tiles)."""
    torch = torch_cuda()
    s, gamma = synth.common_support_system(1)
    rng = np.random.default_rng(540)
    npts = 8192
    pts = synth.torus_points(rng, npts, s.n)
    out = {}
    for mode in (hc.HC_EVAL_SHARED, hc.HC_EVAL_PER_TERM):
        sysh = hc.system_from(s, 2, gamma)
        sysh.set_eval_mode(mode)
        x = torch.from_numpy(hc.to_soa(pts, 2)).cuda()
        f = torch.empty((2, 2, s.npoly, npts), dtype=torch.float64, device="cuda")
        J = torch.empty((2, 2, s.npoly, s.n, npts), dtype=torch.float64, device="cuda")
        hc.hc_eval_jac(sysh, npts, 0.5, x, f, J)
        torch.cuda.synchronize()
        out[mode] = (f.cpu().numpy(), J.cpu().numpy())
        sysh.free()
    fa, Ja = (hc.from_soa(v) for v in out[hc.HC_EVAL_SHARED])
    fb, Jb = (hc.from_soa(v) for v in out[hc.HC_EVAL_PER_TERM])
    assert np.all(rel_err_per_point(fa, fb) <= TOL[2]) and np.all(rel_err_per_point(Ja, Jb) <= TOL[2])
    sample = np.array([0, 31, 32, 4099, 8000, 8191])
    fo, Jo = oracle_eval(s, gamma, 2, limbs_of(pts[sample], 2), 0.5)
    ef, eJ = rel_err_per_point(fa[sample], fo), rel_err_per_point(Ja[sample], Jo)
    print(f"Table 1 system, 8,192 points: f {digits(ef):.1f} digits, J {digits(eJ):.1f} digits")
    assert np.all(ef <= TOL[2]) and np.all(eJ <= TOL[2])
