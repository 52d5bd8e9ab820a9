"""hc_eval_jac against the oracle: values and full Jacobians, of f and of the homotopy,
in complex double / double-double / quad-double, element by element (normwise per
point within 1e-13 / 1e-28 / 1e-58), at sizes spanning several 32-point tiles with a
ragged tail, at the full eval-throughput size on sampled points, and on edge cases."""
import numpy as np
import pytest

from helpers import TOL, digits, rel_err_per_point
from gpu_util import gpu_eval, limbs_of, oracle_eval, torch_cuda
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("t", [-1.0, 0.37, 1.0])
def test_eval_small_system_several_tiles(L, t):
    torch = torch_cuda()
    rng = np.random.default_rng(200 + L)
    s = synth.random_system(rng, 7, (3, 9), (1, 5), (1, 4), const_term=True)
    gamma = synth.unit_complex(rng)
    pts = limbs_of(synth.torus_points(rng, 75, 7), L)   # 2 full tiles + 11
    f, J = gpu_eval(torch, s, gamma, L, pts, t)
    fo, Jo = oracle_eval(s, gamma, L, pts, t)
    ef, eJ = rel_err_per_point(f, fo), rel_err_per_point(J, Jo)
    print(f"L={L} t={t}: f {digits(ef):.1f} digits, J {digits(eJ):.1f} digits")
    assert np.all(ef <= TOL[L]) and np.all(eJ <= TOL[L])


@pytest.mark.parametrize("L", [2, 4])
def test_values_only_matches_with_jacobian_run(L):
    torch = torch_cuda()
    rng = np.random.default_rng(210)
    s = synth.random_system(rng, 6, 8, (2, 4), (1, 3))
    gamma = synth.unit_complex(rng)
    pts = limbs_of(synth.torus_points(rng, 40, 6), L)
    f1, _ = gpu_eval(torch, s, gamma, L, pts, 0.5, jac=False)
    fo, _ = oracle_eval(s, gamma, L, pts, 0.5, jac=False)
    assert np.all(rel_err_per_point(f1, fo) <= TOL[L])


def test_start_point_bit_exact():
    """At t = 0 and x = (1..1): h = 0 exactly and J = diag(gamma d_i) exactly, the same
    bits as the oracle (a unique, exactly representable result)."""
    torch = torch_cuda()
    s, gamma = synth.single_path_dd(1)
    for L in (1, 2, 4):
        pts = limbs_of(np.ones((33, 8), dtype=complex), L)
        f, J = gpu_eval(torch, s, gamma, L, pts, 0.0)
        fo, Jo = oracle_eval(s, gamma, L, pts[:1], 0.0)
        assert np.all(f == 0.0)
        assert np.array_equal(J, np.broadcast_to(Jo, J.shape))


def test_single_path_system_all_t():
    """The n = 8 single-path system (12 monomials + constant, k = 3) along the path."""
    torch = torch_cuda()
    s, gamma = synth.single_path_dd(1)
    rng = np.random.default_rng(220)
    pts = limbs_of(1.5 * synth.torus_points(rng, 64, 8), 2)
    for t in (0.0, 0.01, 0.5, 0.999, 1.0):
        f, J = gpu_eval(torch, s, gamma, 2, pts, t)
        fo, Jo = oracle_eval(s, gamma, 2, pts, t)
        assert np.all(rel_err_per_point(f, fo) <= TOL[2])
        assert np.all(rel_err_per_point(J, Jo) <= TOL[2])


def test_edge_monomials():
    """Constant-only polynomial, k = 1 monomials, the largest k (32), exponent 64."""
    torch = torch_cuda()
    n = 32
    var_ptr = [0, 0, 1, 33, 35, 35]
    idx = [5] + list(range(32)) + [0, 31]
    ex = [64] + [1] * 16 + [2] * 16 + [3, 1]
    s = synth.System(n=n, npoly=3, mon_ptr=np.array([0, 1, 3, 5], np.int32),
                     var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                     var_exp=np.array(ex, np.int32),
                     coef=np.exp(1j * np.arange(5.0)))
    rng = np.random.default_rng(230)
    for L in (1, 2, 4):
        pts = limbs_of(synth.torus_points(rng, 35, n), L)
        f, J = gpu_eval(torch, s, 1 + 0j, L, pts, -1.0)
        fo, Jo = oracle_eval(s, 1 + 0j, L, pts, -1.0)
        assert np.all(rel_err_per_point(f, fo) <= TOL[L])
        assert np.all(rel_err_per_point(J, Jo) <= TOL[L])


def test_zero_points_is_a_noop():
    torch = torch_cuda()
    s, gamma = synth.single_path_dd(1)
    sysh = hc.system_from(s, 2, gamma)
    hc.hc_eval_jac(sysh, 0, 0.5, None, None, None)
    sysh.free()


def test_deterministic():
    torch = torch_cuda()
    s, pts, gamma = synth.eval_throughput(2, npts=300)
    p = limbs_of(pts, 2)
    a = gpu_eval(torch, s, gamma, 2, p, 0.3)
    b = gpu_eval(torch, s, gamma, 2, p, 0.3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("L", [2, 4])
def test_eval_throughput_workload_full_size_sampled(L):
    """n = 32, 32 x 128 monomials, k = 6, exponents 1..4, all 65,536 torus points on
    the GPU in one call; the oracle checks 12 sampled points (first, last, spread)."""
    torch = torch_cuda()
    s, pts, gamma = synth.eval_throughput(2)
    npts = pts.shape[0]
    sysh = hc.system_from(s, L, gamma)
    x = torch.from_numpy(hc.to_soa(pts, L)).cuda()
    f = torch.empty((2, L, 32, npts), dtype=torch.float64, device="cuda")
    J = torch.empty((2, L, 32, 32, npts), dtype=torch.float64, device="cuda")
    hc.hc_eval_jac(sysh, npts, 0.61, x, f, J)
    torch.cuda.synchronize()
    sample = np.array([0, 1, 31, 32, 4097, 20000, 33333, 40000, 50001, 65503, 65534, 65535])
    fs = hc.from_soa(f[..., sample].cpu().numpy())
    Js = hc.from_soa(J[..., sample].cpu().numpy())
    fo, Jo = oracle_eval(s, gamma, L, limbs_of(pts[sample], L), 0.61)
    ef, eJ = rel_err_per_point(fs, fo), rel_err_per_point(Js, Jo)
    print(f"L={L} full size: f {digits(ef):.1f} digits, J {digits(eJ):.1f} digits")
    assert np.all(ef <= TOL[L]) and np.all(eJ <= TOL[L])
    sysh.free()


def _rows_subsystem(s, rows):
    """The polynomials `rows` of s as a system of its own (same n)."""
    mon_ptr, var_ptr, idx, ex, coef = [0], [0], [], [], []
    for i in rows:
        for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
            q0, q1 = s.var_ptr[m], s.var_ptr[m + 1]
            idx.extend(s.var_idx[q0:q1])
            ex.extend(s.var_exp[q0:q1])
            var_ptr.append(var_ptr[-1] + q1 - q0)
            coef.append(s.coef[m])
        mon_ptr.append(len(coef))
    return synth.System(n=s.n, npoly=len(rows), mon_ptr=np.array(mon_ptr, np.int32),
                        var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                        var_exp=np.array(ex, np.int32), coef=np.array(coef))


def test_large_qd_workload_sampled_rows():
    """n = 96, 96 x 1024 monomials, k = 12, exponents 1..5, complex QD: the full system
    on the GPU at 40 points; the oracle evaluates rows 0, 50 and 95 at 2 points."""
    torch = torch_cuda()
    s, gamma = synth.large_path_qd(4)
    rng = np.random.default_rng(240)
    pts = limbs_of(synth.torus_points(rng, 40, s.n), 4)
    f, J = gpu_eval(torch, s, gamma, 4, pts, -1.0)
    rows = [0, 50, 95]
    sub = _rows_subsystem(s, rows)
    sample = [0, 39]
    fo, Jo = oracle_eval(sub, gamma, 4, pts[sample], -1.0)
    ef = rel_err_per_point(f[sample][:, rows], fo)
    eJ = rel_err_per_point(J[sample][:, rows], Jo)
    print(f"large QD: f {digits(ef):.1f} digits, J {digits(eJ):.1f} digits")
    assert np.all(ef <= TOL[4]) and np.all(eJ <= TOL[4])


def test_autotuned_tiles_give_identical_results():
    """Every tile shape computes the same bits (a point's arithmetic does not depend on
    how the work is cut), and the tuner returns one of the candidates."""
    torch = torch_cuda()
    from paper_1109_0545_gb300 import autotune
    s, pts, gamma = synth.eval_throughput(2, npts=2000)
    sysh = hc.system_from(s, 2, gamma)
    x = torch.from_numpy(hc.to_soa(pts, 2)).cuda()
    f = torch.zeros((2, 2, 32, 2000), dtype=torch.float64, device="cuda")
    J = torch.zeros((2, 2, 32, 32, 2000), dtype=torch.float64, device="cuda")
    ref = None
    for r, b in [(0, 0), (1, 2), (3, 3), (8, 6), (32, 1)]:
        hc.hc_set_tiles(r, b)
        hc.hc_eval_jac(sysh, 2000, 0.3, x, f, J)
        torch.cuda.synchronize()
        got = (f.cpu().numpy().copy(), J.cpu().numpy().copy())
        if ref is None:
            ref = got
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    best = autotune.tune_eval(sysh, x, f, J, 2000, 0.3, reps=1, use_cache=False)
    assert (best["rows_per_task"], best["blocks_per_sm"]) in [(r, b) for r in autotune.ROWS for b in autotune.BLOCKS]
    hc.hc_set_tiles(0, 0)
    sysh.free()
