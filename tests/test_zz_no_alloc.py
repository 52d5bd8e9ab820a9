"""hc_eval_jac_noalloc, the evaluation entry point for callers that cannot allocate device
memory (their memory belongs to their own pool allocator, or a cudaMalloc's implicit
synchronisation is not acceptable where they call).  It must give the results of
hc_eval_jac, call after call, from its fixed workspace, and refuse work that does not fit.

This file is collected last on purpose: a run that stops at the first failure has run
every other test before this one.  It also passes alone in a fresh process.
"""
import numpy as np
import pytest

from helpers import TOL, rel_err_per_point
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(torch, fn, sysh, s, L, pts, t):
    npts = pts.shape[0]
    x = torch.from_numpy(hc.to_soa(pts, L)).cuda()
    f = torch.full((2, L, s.npoly, npts), np.nan, dtype=torch.float64, device="cuda")
    J = torch.full((2, L, s.npoly, s.n, npts), np.nan, dtype=torch.float64, device="cuda")
    fn(sysh, npts, t, x, f, J)
    torch.cuda.synchronize()
    return hc.from_soa(f.cpu().numpy()), hc.from_soa(J.cpu().numpy())


@pytest.mark.parametrize("L", [1, 2, 4])
def test_noalloc_matches_eval_jac_on_two_calls_in_a_row(L):
    torch = _torch()
    s, pts, gamma = synth.eval_throughput(2, npts=3000)
    sysh = hc.system_from(s, L, gamma)
    # two consecutive calls on different point sets and t; each is checked against the
    # allocating entry point on the same inputs
    cases = [(pts[:3000], 0.3), (synth.torus_points(np.random.default_rng(77), 1111, s.n), -1.0)]
    for p, t in cases:
        got_f, got_J = _run(torch, hc.hc_eval_jac_noalloc, sysh, s, L, p, t)
        ref_f, ref_J = _run(torch, hc.hc_eval_jac, sysh, s, L, p, t)
        assert np.all(rel_err_per_point(got_f, ref_f) <= TOL[L])
        assert np.all(rel_err_per_point(got_J, ref_J) <= TOL[L])
    sysh.free()


def test_noalloc_shared_monomial_scheme_on_two_calls_in_a_row():
    """The shared-monomial scheme (a common support: Table 1's 40 x 40 system with 200
    monomials of degree up to 80, whose power table takes about 100 KB per DD point)."""
    torch = _torch()
    s, gamma = synth.common_support_system(1)
    sysh = hc.system_from(s, 2, gamma)
    sysh.set_eval_mode(hc.HC_EVAL_SHARED)
    rng = np.random.default_rng(78)
    for npts, t in ((300, 0.7), (57, -1.0)):
        p = synth.torus_points(rng, npts, s.n)
        got_f, got_J = _run(torch, hc.hc_eval_jac_noalloc, sysh, s, 2, p, t)
        ref_f, ref_J = _run(torch, hc.hc_eval_jac, sysh, s, 2, p, t)
        assert np.all(rel_err_per_point(got_f, ref_f) <= TOL[2])
        assert np.all(rel_err_per_point(got_J, ref_J) <= TOL[2])
    sysh.free()


def test_noalloc_without_a_power_table():
    """Exponents at most 2 need no workspace at all: any number of points is accepted."""
    torch = _torch()
    rng = np.random.default_rng(79)
    s = synth.random_system(rng, 6, 10, (1, 4), (1, 2), const_term=True)
    gamma = synth.unit_complex(rng)
    sysh = hc.system_from(s, 2, gamma)
    for npts, t in ((70000, 0.2), (33, 0.9)):
        p = synth.torus_points(rng, npts, s.n)
        got_f, got_J = _run(torch, hc.hc_eval_jac_noalloc, sysh, s, 2, p, t)
        ref_f, ref_J = _run(torch, hc.hc_eval_jac, sysh, s, 2, p, t)
        assert np.all(rel_err_per_point(got_f, ref_f) <= TOL[2])
        assert np.all(rel_err_per_point(got_J, ref_J) <= TOL[2])
    sysh.free()


def test_noalloc_rejects_work_beyond_its_workspace():
    torch = _torch()
    s, pts, gamma = synth.eval_throughput(2, npts=16)
    sysh = hc.system_from(s, 2, gamma)
    # n = 32, exponents up to 4, DD: 2048 bytes of power table per point -> 16,384 points fit
    big = 16385
    x = torch.zeros((2, 2, s.n, big), dtype=torch.float64, device="cuda")
    f = torch.zeros((2, 2, s.npoly, big), dtype=torch.float64, device="cuda")
    with pytest.raises(hc.HCError) as e:
        hc.hc_eval_jac_noalloc(sysh, big, 0.5, x, f, None)
    assert e.value.code == hc.HC_EINVAL and "at most 16384 points" in str(e.value)
    sysh.free()
