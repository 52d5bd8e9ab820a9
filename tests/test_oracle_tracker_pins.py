"""Pins of the oracle's tracker parts against facts other than the oracle itself.

* The predictor of Alg. 3.1 (secant) and of Sec. 5 (quadratic) against exact rational
  interpolation: on a path x(t) that is a polynomial of degree 1 (secant) or 2
  (quadratic) in t, the predicted point is x(t') itself.  At dyadic t values whose
  Lagrange weights are exact in double the agreement is exact; elsewhere it is within
  the rounding of the weights.  A swapped weight, a wrong sign or the wrong previous
  point misses by O(1).
* The tracker driven on constructed homotopies whose solution path is exactly linear
  (one unknown) or has a linear and a quadratic coordinate (two unknowns): from the
  third accepted point on, the quadratic predictor lands on the path to the rounding of
  its weights, the secant predictor does so only on the linear path, and the end point
  is the closed-form solution at t = 1.
* The homotopy gamma (1-t) g + t f and its Jacobian at 0 < t < 1 against mpmath at 400
  bits, at t whose 1 - t is not a double (a 1 - t rounded to one limb fails).
* Replay and resume: replaying the accepted t values of a tracked path reproduces its end
  point bit for bit; resuming it in chunks of stages reproduces the one-call run.
* The tracker on a decoupled system of three unknowns (f_i = x_i^{d_i} - c_i, degrees 2, 3
  and 4): each coordinate of the path is a d_i-th root continued along t in closed form,
  and every accepted point, at the t the tracker records, lies on it (mpmath at 200 bits).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_1109_0545_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def fr_limbs(v):
    return sum(Fr(float(x)) for x in v)


def to_limbs(z: complex, L: int) -> np.ndarray:
    out = np.zeros((2, L))
    out[0, 0], out[1, 0] = z.real, z.imag
    return out


def cfr(c):
    return fr_limbs(c[0]), fr_limbs(c[1])


def lagrange(ts, vs, t1):
    """Exact value at t1 of the interpolating polynomial through (ts[i], vs[i]) (Fractions)."""
    total = Fr(0)
    for i, (ti, vi) in enumerate(zip(ts, vs)):
        w = Fr(1)
        for j, tj in enumerate(ts):
            if j != i:
                w *= (Fr(t1) - Fr(tj)) / (Fr(ti) - Fr(tj))
        total += w * vi
    return total


def poly_path(rng, n, degree):
    """Coefficients of x_j(t) = a_j + b_j t (+ c_j t^2), dyadic complex numbers."""
    def dy():
        return complex(int(rng.integers(-64, 65)) / 16.0, int(rng.integers(-64, 65)) / 16.0)
    return [[dy() for _ in range(degree + 1)] for _ in range(n)]


def eval_path(coefs, t):
    """Exact (Fraction re, im) values of the path at t."""
    out = []
    for cs in coefs:
        re = sum(Fr(c.real) * Fr(t) ** k for k, c in enumerate(cs))
        im = sum(Fr(c.imag) * Fr(t) ** k for k, c in enumerate(cs))
        out.append((re, im))
    return out


def as_limbs(vals, L):
    """Exact Fraction values (exactly representable in double here) -> [n][2][L]."""
    out = np.zeros((len(vals), 2, L))
    for j, (re, im) in enumerate(vals):
        out[j, 0, 0], out[j, 1, 0] = float(re), float(im)
        assert Fr(out[j, 0, 0]) == re and Fr(out[j, 1, 0]) == im
    return out


# t_pp, t_p, t, t' with Lagrange weights that are exact in double (equal or doubling steps)
DYADIC_T = [(0.0, 0.25, 0.5, 0.75), (0.0, 0.125, 0.25, 0.5), (0.375, 0.5, 0.625, 0.75),
            (0.5, 0.5625, 0.625, 0.75), (0.25, 0.3125, 0.375, 0.4375)]


@pytest.mark.parametrize("L", [2, 4])
def test_quadratic_predictor_is_exact_on_a_parabola(L):
    rng = np.random.default_rng(900 + L)
    for tpp, tp, t, t1 in DYADIC_T:
        coefs = poly_path(rng, 3, 2)
        pts = [eval_path(coefs, s) for s in (t, tp, tpp)]
        zh = oracle.predict(L, 1, 3, t, tp, tpp, t1, *[as_limbs(v, L) for v in pts])
        want = eval_path(coefs, t1)
        for j in range(3):
            assert cfr(zh[j]) == want[j], (tpp, tp, t, t1, j)


@pytest.mark.parametrize("L", [2, 4])
def test_secant_predictor_is_exact_on_a_line_and_linear_on_a_parabola(L):
    rng = np.random.default_rng(910 + L)
    for tpp, tp, t, t1 in DYADIC_T:
        line = poly_path(rng, 3, 1)
        pts = [as_limbs(eval_path(line, s), L) for s in (t, tp, tpp)]
        zh = oracle.predict(L, 0, 3, t, tp, tpp, t1, *pts)
        for j, v in enumerate(eval_path(line, t1)):
            assert cfr(zh[j]) == v
        # on a parabola the secant step is the line through the last two points, not the
        # parabola: its value is the exact linear extrapolation
        par = poly_path(rng, 3, 2)
        vals = [eval_path(par, s) for s in (t, tp)]
        zh = oracle.predict(L, 0, 3, t, tp, tpp, t1, as_limbs(vals[0], L), as_limbs(vals[1], L),
                            as_limbs(vals[1], L))
        for j in range(3):
            want = tuple(lagrange([t, tp], [vals[0][j][c], vals[1][j][c]], t1) for c in (0, 1))
            assert cfr(zh[j]) == want
        # the quadratic predictor with fewer than three points falls back to the secant
        zq = oracle.predict(L, 1, 2, t, tp, tpp, t1, as_limbs(vals[0], L), as_limbs(vals[1], L),
                            as_limbs(vals[1], L))
        assert np.array_equal(zq, zh)
        # zeroth order with one point
        z0 = oracle.predict(L, 0, 1, t, tp, tpp, t1, as_limbs(vals[0], L), as_limbs(vals[1], L),
                            as_limbs(vals[1], L))
        assert np.array_equal(z0, as_limbs(vals[0], L))


def test_predictors_within_weight_rounding_at_arbitrary_t():
    """Non-dyadic t: the quadratic prediction of a parabola, and the secant prediction of
    a line, are within the rounding of the double weights (a few 1e-16 relative)."""
    rng = np.random.default_rng(920)
    for _ in range(50):
        tpp = float(rng.uniform(0, 0.5))
        tp = tpp + float(rng.uniform(1e-3, 0.05))
        t = tp + float(rng.uniform(1e-3, 0.05))
        t1 = t + float(rng.uniform(1e-3, 0.08))
        for pred, deg in ((1, 2), (0, 1)):
            coefs = [[complex(*rng.normal(size=2)) for _ in range(deg + 1)] for _ in range(2)]
            vals = [eval_path(coefs, s) for s in (t, tp, tpp)]
            pts = [np.array([to_limbs(complex(float(re), float(im)), 2) for re, im in v]) for v in vals]
            # the points as stored (rounded to double) define the interpolant exactly
            stored = [[cfr(p[j]) for j in range(2)] for p in pts]
            zh = oracle.predict(2, pred, 3, t, tp, tpp, t1, *pts)
            ts = [t, tp, tpp][:deg + 1]
            for j in range(2):
                for c in (0, 1):
                    want = lagrange(ts, [stored[k][j][c] for k in range(deg + 1)], t1)
                    scale = max(abs(float(stored[k][j][c])) for k in range(deg + 1)) + 1
                    assert abs(float(cfr(zh[j])[c] - want)) <= 64 * 2.0 ** -53 * scale * 20


def linear_path_system(gamma: complex, c: complex, a: complex | None = None, b: complex = 0):
    """f_1 = gamma x_1 + c (and f_2 = gamma x_2 + a x_1 + b): all degrees 1, so
    h = gamma (1-t)(x - 1) + t f has the exact path x_1(t) = 1 - t (1 + c/gamma) and
    x_2(t) = (1 - t) - t (a x_1(t) + b)/gamma, linear and quadratic in t."""
    if a is None:
        return synth.System(n=1, npoly=1, mon_ptr=np.array([0, 2], np.int32),
                            var_ptr=np.array([0, 1, 1], np.int32), var_idx=np.array([0], np.int32),
                            var_exp=np.array([1], np.int32), coef=np.array([gamma, c]))
    return synth.System(n=2, npoly=2, mon_ptr=np.array([0, 2, 5], np.int32),
                        var_ptr=np.array([0, 1, 1, 2, 3, 3], np.int32),
                        var_idx=np.array([0, 1, 0], np.int32), var_exp=np.array([1, 1, 1], np.int32),
                        coef=np.array([gamma, c, gamma, a, b]))


def track_opts(**kw):
    o = oracle.TrackOpts(lambda0=0.01, lambda_min=1e-12, lambda_max=0.08, grow=2.0, shrink=0.5,
                         eps=1e-26, eps_x=1e-8, eps_end=1e-26, eps_end_x=1e-26, div_bound=1e6,
                         max_it=3, end_it=8, grow_after=3, max_steps=100000, predictor=0,
                         lu_mode=1, max_refine=4)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def exact_end(gamma, c, a=None, b=0):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    G, Cc = mpmath.mpc(gamma.real, gamma.imag), mpmath.mpc(c.real, c.imag)
    x1 = -Cc / G
    if a is None:
        return [x1]
    A, B = mpmath.mpc(a.real, a.imag), mpmath.mpc(b.real, b.imag)
    return [x1, -(A * x1 + B) / G]


@pytest.mark.parametrize("L", [2, 4])
def test_tracker_follows_exact_polynomial_paths(L):
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(930 + L)
    gamma, c, a, b = (synth.unit_complex(rng) for _ in range(4))
    tol = {2: 1e-28, 4: 1e-58}[L]
    eps = {2: 1e-26, 4: 1e-58}[L]
    g = np.array([gamma.real, gamma.imag])
    cases = [(linear_path_system(gamma, c), exact_end(gamma, c)),
             (linear_path_system(gamma, c, a, b), exact_end(gamma, c, a, b))]
    firsts = {}
    for idx, (s, end) in enumerate(cases):
        for pred in (0, 1):
            r = oracle.track(s.as_dict(), s.coef_limbs(L), synth.limbs(np.ones(s.n), L), g,
                             track_opts(predictor=pred, eps=eps, eps_end=eps, eps_end_x=eps), log_cap=1000)
            assert oracle.STATUS[r.status] == "OK"
            assert np.all(r.log["accepted"] == 1)
            for j in range(s.n):
                got = mpmath.mpc(sum(mpmath.mpf(float(v)) for v in r.x[j, 0]),
                                 sum(mpmath.mpf(float(v)) for v in r.x[j, 1]))
                assert abs(got - end[j]) <= tol * abs(end[j])
            firsts[(idx, pred)] = r.log["res_first"]
    # the residual of the predicted point: stage k has k accepted points before it
    lin_sec, lin_quad = firsts[(0, 0)], firsts[(0, 1)]
    quad_sec, quad_quad = firsts[(1, 0)], firsts[(1, 1)]
    assert lin_sec[0] > 1e-5                 # zeroth order on the first stage
    assert np.max(lin_sec[1:]) < 1e-12       # secant: exact on a line
    assert np.max(lin_quad[2:]) < 1e-12      # quadratic: exact on a line
    assert np.max(quad_quad[2:]) < 1e-12     # quadratic: exact on a parabola
    assert np.min(quad_sec[2:]) > 1e-7       # secant: second-order error on the parabola


def test_homotopy_between_0_and_1_matches_mpmath():
    """h = gamma (1-t)(x^d - 1) + t f and dh/dx at 0 < t < 1, DD within 1e-30 and QD within
    1e-60 of mpmath at 400 bits.  The t values are chosen so that 1 - t needs two limbs."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    rng = np.random.default_rng(940)
    s = synth.random_system(rng, 3, 5, (1, 3), (1, 4), const_term=True)
    gamma = synth.unit_complex(rng)
    xs = synth.torus_points(rng, 2, 3) * 1.1
    deg = oracle.degrees(s.as_dict())
    # below 1/2, t with low mantissa bits set has a 1 - t that is not a double (its two-sum
    # error is nonzero); above 1/2, 1 - t is exact
    ts = [0.1 + 2.0 ** -52, float(np.nextafter(0.37, 1.0)), 0.013, 0.61, 0.999]
    assert sum(Fr(1) - Fr(t) != Fr(1.0 - t) for t in ts) == 3
    for t in ts:
        for L, tol in ((2, 1e-30), (4, 1e-60)):
            h, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), synth.limbs(xs, L), t,
                                      np.array([gamma.real, gamma.imag]), mode=1)
            G = mpmath.mpc(gamma.real, gamma.imag)
            T = mpmath.mpf(t)
            for p in range(2):
                X = [mpmath.mpc(float(z.real), float(z.imag)) for z in xs[p]]
                for i in range(s.npoly):
                    fi = mpmath.mpc(0)
                    Ji = [mpmath.mpc(0)] * s.n
                    for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
                        term = mpmath.mpc(float(s.coef[m].real), float(s.coef[m].imag))
                        vs = list(range(s.var_ptr[m], s.var_ptr[m + 1]))
                        for q in vs:
                            term *= X[s.var_idx[q]] ** int(s.var_exp[q])
                        fi += term
                        for q in vs:
                            Ji[s.var_idx[q]] += term * int(s.var_exp[q]) / X[s.var_idx[q]]
                    d = int(deg[i])
                    hi_ = G * (1 - T) * (X[i] ** d - 1) + T * fi
                    got = mpmath.mpc(sum(mpmath.mpf(float(a)) for a in h[p, i, 0]),
                                     sum(mpmath.mpf(float(a)) for a in h[p, i, 1]))
                    assert abs(got - hi_) <= tol * max(1, abs(hi_)), (t, L, p, i)
                    for j in range(s.n):
                        want = T * Ji[j] + (G * (1 - T) * d * X[i] ** (d - 1) if i == j else 0)
                        gj = mpmath.mpc(sum(mpmath.mpf(float(a)) for a in J[p, i, j, 0]),
                                        sum(mpmath.mpf(float(a)) for a in J[p, i, j, 1]))
                        assert abs(gj - want) <= tol * max(1, abs(want)), (t, L, p, i, j)


def _regular(seed, n):
    rng = np.random.default_rng(seed)
    return synth.regular_system(rng, n, 4, (1, min(2, n)), (1, 2), lead=3), synth.unit_complex(rng)


@pytest.mark.parametrize("pred", [0, 1])
def test_replay_of_the_accepted_steps_reproduces_the_path_bitwise(pred):
    for seed in (950, 951):
        s, gamma = _regular(seed, 3)
        g = np.array([gamma.real, gamma.imag])
        o = track_opts(predictor=pred)
        x0 = synth.limbs(np.ones(s.n), 2)
        r = oracle.track(s.as_dict(), s.coef_limbs(2), x0, g, o, log_cap=100000)
        assert oracle.STATUS[r.status] == "OK"
        lg = r.log
        acc = np.nonzero(lg["accepted"] == 1)[0]
        assert len(acc) < len(lg)          # the path has rejected stages to skip
        tseq = [lg["t"][k + 1] if k + 1 < len(lg) else 1.0 for k in acc]
        x1, status, fail = oracle.track_replay(s.as_dict(), s.coef_limbs(2), x0, g, o, tseq)
        assert fail == -1 and status == 0
        assert np.array_equal(x1, r.x)


def test_resume_in_chunks_equals_one_call():
    s, gamma = _regular(960, 3)
    g = np.array([gamma.real, gamma.imag])
    o = track_opts(predictor=1)
    x0 = synth.limbs(np.ones(s.n), 2)
    r = oracle.track(s.as_dict(), s.coef_limbs(2), x0, g, o, log_cap=100000)
    st = oracle.PathState()
    z, zp, zpp = x0, np.zeros_like(x0), np.zeros_like(x0)
    logs = []
    for _ in range(1000):
        st, z, zp, zpp, stats, lg = oracle.track_resume(s.as_dict(), s.coef_limbs(2), g, o, st, z, zp, zpp, 7,
                                                        log_cap=7)
        logs.append(lg)
        assert len(lg) <= 7
        if st.phase == 3:
            break
    assert st.phase == 3
    assert np.array_equal(z, r.x)
    assert (stats["status"], stats["n_succ"], stats["n_corr"], stats["newton_its"], stats["end_its"]) == \
        (r.status, r.n_succ, r.n_corr, r.newton_its, r.end_its)
    assert stats["t_end"] == r.t_end and stats["res_end"] == r.res_end
    assert np.array_equal(np.concatenate(logs), r.log)


def decoupled_system(c, d):
    """f_i = x_i^{d_i} - c_i, i = 0..n-1: the homotopy decouples, and coordinate i of the
    path solves x^{d_i} = (gamma (1-t) + t c_i) / (gamma (1-t) + t)."""
    n = len(c)
    coef, idx, ex, var_ptr = [], [], [], [0]
    for i in range(n):
        coef += [1.0, -c[i]]
        idx.append(i)
        ex.append(d[i])
        var_ptr += [var_ptr[-1] + 1, var_ptr[-1] + 1]
    return synth.System(n=n, npoly=n, mon_ptr=np.arange(0, 2 * n + 1, 2, dtype=np.int32),
                        var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                        var_exp=np.array(ex, np.int32), coef=np.array(coef, dtype=complex))


def exact_branch(gamma, c, d, ts, mpmath):
    """x(t) along ts (increasing, from 0) for x^d = w(t), continued from x(0) = 1 in
    substeps of at most 1e-3, each time taking the d-th root nearest the previous point."""
    G, C = mpmath.mpc(gamma.real, gamma.imag), mpmath.mpc(c.real, c.imag)
    x, t0, out = mpmath.mpc(1), mpmath.mpf(0), []
    for t in ts:
        T = mpmath.mpf(t)
        m = max(1, int(mpmath.ceil((T - t0) / mpmath.mpf("1e-3"))))
        for k in range(1, m + 1):
            s = t0 + (T - t0) * k / m
            w = (G * (1 - s) + s * C) / (G * (1 - s) + s)
            r0 = mpmath.root(w, d)
            roots = [r0 * mpmath.exp(2j * mpmath.pi * q / d) for q in range(d)]
            x = min(roots, key=lambda r: abs(r - x))
        t0 = T
        out.append(x)
    return out


@pytest.mark.parametrize("L", [2, 4])
def test_tracker_points_lie_on_the_exact_path_of_a_decoupled_system(L):
    """n = 3, degrees 2, 3, 4: every accepted point of the oracle's tracker, at the t it
    records, equals the exact path point (each coordinate a continued d-th root, mpmath at
    200 bits) to the corrector's accuracy, and the end point equals the root reached at
    t = 1 within the tolerance of the precision."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(970 + L)
    d = [2, 3, 4]
    c = [synth.unit_complex(rng) for _ in d]
    gamma = synth.unit_complex(rng)
    s = decoupled_system(c, d)
    g = np.array([gamma.real, gamma.imag])
    eps = {2: 1e-26, 4: 1e-58}[L]
    o = track_opts(predictor=1, eps=eps, eps_end=eps, eps_end_x=eps)
    st = oracle.PathState()
    z = synth.limbs(np.ones(s.n), L)
    zp, zpp = np.zeros_like(z), np.zeros_like(z)
    ts, pts = [], []
    for _ in range(5000):
        before = st.n_succ
        st, z, zp, zpp, _, _ = oracle.track_resume(s.as_dict(), s.coef_limbs(L), g, o, st, z, zp, zpp, 1)
        if st.phase == 3:
            break
        if st.n_succ > before:
            ts.append(st.t)
            pts.append(z.copy())
    assert oracle.STATUS[st.status] == "OK" and len(ts) > 10
    ts.append(1.0)
    pts.append(z.copy())
    for i in range(s.n):
        exact = exact_branch(gamma, c[i], d[i], ts, mpmath)
        for k, (t, p) in enumerate(zip(ts, pts)):
            got = mpmath.mpc(sum(mpmath.mpf(float(v)) for v in p[i, 0]), sum(mpmath.mpf(float(v)) for v in p[i, 1]))
            tol = 1e-12 if k < len(ts) - 1 else {2: 1e-28, 4: 1e-58}[L]
            assert abs(got - exact[k]) <= tol * max(1, abs(exact[k])), (i, k, t, float(abs(got - exact[k])))
