"""hc_newton_step against the oracle: one Newton iteration of Alg. 4.1 per point, with
the native elimination and with the FP64 LU + refinement, in double / DD / QD."""
import numpy as np
import pytest

from helpers import TOL, digits, rel_err_per_point
from gpu_util import gpu_newton, limbs_of, torch_cuda
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


def oracle_newton(s, gamma, L, pts, t, lu_mode, max_refine=4):
    return oracle.newton_step(s.as_dict(), s.coef_limbs(L), pts, t,
                              np.array([gamma.real, gamma.imag]), lu_mode, max_refine)


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("lu_mode", [hc.HC_LU_NATIVE, hc.HC_LU_FP64_REFINE])
def test_newton_step_matches_oracle(L, lu_mode):
    torch = torch_cuda()
    rng = np.random.default_rng(300 + L)
    s = synth.random_system(rng, 6, (4, 8), (1, 4), (1, 3))
    gamma = synth.unit_complex(rng)
    pts = limbs_of(synth.torus_points(rng, 70, 6), L)
    x, res, st, sw = gpu_newton(torch, s, gamma, L, pts, 0.42, lu_mode, max_refine=6)
    xo, reso, sto, swo = oracle_newton(s, gamma, L, pts, 0.42, lu_mode, max_refine=6)
    assert np.array_equal(st, sto)
    assert np.allclose(res, reso, rtol=1e-12, atol=0)
    e = rel_err_per_point(x, xo)
    print(f"L={L} lu_mode={lu_mode}: x {digits(e):.1f} digits, sweeps {np.bincount(sw)}")
    assert np.all(e <= TOL[L])
    if lu_mode == hc.HC_LU_NATIVE:
        assert np.all(sw == 0)
    else:
        assert np.all((sw >= 1) & (sw <= 6))


@pytest.mark.parametrize("L", [2, 4])
def test_mixed_and_native_agree(L):
    """FP64 LU + refinement converges to the native solve within the tolerance."""
    torch = torch_cuda()
    s, pts, gamma = synth.eval_throughput(2, npts=96)
    p = limbs_of(pts, L)
    a = gpu_newton(torch, s, gamma, L, p, 0.5, hc.HC_LU_NATIVE)
    b = gpu_newton(torch, s, gamma, L, p, 0.5, hc.HC_LU_FP64_REFINE, max_refine=8)
    assert np.all(a[2] == hc.HC_OK) and np.all(b[2] == hc.HC_OK)
    e = rel_err_per_point(b[0], a[0])
    print(f"L={L}: mixed vs native {digits(e):.1f} digits, sweeps {np.bincount(b[3])}")
    assert np.all(e <= TOL[L])


def test_singular_jacobian_leaves_point_unchanged():
    """f = (x0 x1, x0 x1) has a rank-deficient Jacobian everywhere: SINGULAR, x kept."""
    torch = torch_cuda()
    s = synth.System(n=2, npoly=2, mon_ptr=np.array([0, 1, 2], np.int32),
                     var_ptr=np.array([0, 2, 4], np.int32),
                     var_idx=np.array([0, 1, 0, 1], np.int32),
                     var_exp=np.array([1, 1, 1, 1], np.int32), coef=np.array([1.0 + 0j, 1.0 + 0j]))
    pts = limbs_of(np.zeros((5, 2), dtype=complex), 2)
    x, res, st, _ = gpu_newton(torch, s, 1 + 0j, 2, pts, -1.0, hc.HC_LU_NATIVE)
    assert np.all(st == hc.HC_SINGULAR) and np.array_equal(x, pts)
    _, _, sto, _ = oracle_newton(s, 1 + 0j, 2, pts, -1.0, 0)
    assert np.all(sto == 2)
    x, res, st, _ = gpu_newton(torch, s, 1 + 0j, 2, pts, -1.0, hc.HC_LU_FP64_REFINE)
    assert np.all(st == hc.HC_SINGULAR) and np.array_equal(x, pts)


def test_nonfinite_point_reported():
    torch = torch_cuda()
    s, gamma = synth.single_path_dd(1)
    pts = limbs_of(np.ones((3, 8), dtype=complex), 2)
    pts[1, 3, 0, 0] = np.inf
    x, res, st, _ = gpu_newton(torch, s, gamma, 2, pts, 0.2, hc.HC_LU_NATIVE)
    assert st[1] == hc.HC_NONFINITE and st[0] == hc.HC_OK and st[2] == hc.HC_OK
    assert np.array_equal(x[1], pts[1])


def test_newton_full_size_sampled():
    """All 65,536 points of the eval-throughput workload, one Newton step each, both
    linear solvers in DD; 8 sampled points checked against the oracle."""
    torch = torch_cuda()
    s, pts, gamma = synth.eval_throughput(2)
    npts = pts.shape[0]
    sample = np.array([0, 77, 8191, 16384, 32767, 49152, 65500, 65535])
    po = limbs_of(pts[sample], 2)
    for lu in (hc.HC_LU_NATIVE, hc.HC_LU_FP64_REFINE):
        sysh = hc.system_from(s, 2, gamma)
        x = torch.from_numpy(hc.to_soa(pts, 2)).cuda()
        res = torch.zeros(npts, dtype=torch.float64, device="cuda")
        st = torch.zeros(npts, dtype=torch.int32, device="cuda")
        sw = torch.zeros(npts, dtype=torch.int32, device="cuda")
        hc.hc_newton_step(sysh, npts, 0.25, x, lu, 6, res, st, sw)
        torch.cuda.synchronize()
        xs = hc.from_soa(x[..., sample].cpu().numpy())
        xo, reso, sto, _ = oracle_newton(s, gamma, 2, po, 0.25, lu, 6)
        assert np.array_equal(st[sample].cpu().numpy(), sto)
        assert np.allclose(res[sample].cpu().numpy(), reso, rtol=1e-12)
        e = rel_err_per_point(xs, xo)
        print(f"lu={lu}: {digits(e):.1f} digits; sweeps {np.bincount(sw.cpu().numpy())}")
        assert np.all(e <= TOL[2])
        sysh.free()
