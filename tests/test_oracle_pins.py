"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle routine to an independent fact: exact rational arithmetic
(fractions / sympy), a library derivative (sympy.diff), high-precision evaluation
(mpmath at 400 bits), a finite difference, a closed form (the roots of the start
system), library polynomial roots (numpy.roots refined by mpmath.polyroots), or an
invariant of the step-size control.  They are chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_1109_0545_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def fr_limbs(v):
    return sum(Fr(float(x)) for x in v)


def fr_c(c):  # c[2][L] -> (re, im) Fractions
    return fr_limbs(c[0]), fr_limbs(c[1])


def rand_limbs(rng, L, scale_exp=20):
    a = np.zeros(L)
    a[0] = rng.normal() * 2.0 ** int(rng.integers(-scale_exp, scale_exp))
    for j in range(1, L):
        a[j] = a[j - 1] * 2.0 ** -53 * rng.uniform(-1, 1)
    return a


# ---------------------------------------------------------------------- arithmetic (Sec. 1-2)
@pytest.mark.parametrize("L", [1, 2, 4])
def test_real_ops_within_bound_of_exact(L):
    """add/mul/div of L-limb reals are within 2^(-52L) of the exact rational result."""
    rng = np.random.default_rng(10 + L)
    bound = 2.0 ** (-52 * L)
    for _ in range(200):
        a, b = rand_limbs(rng, L), rand_limbs(rng, L)
        A, B = fr_limbs(a), fr_limbs(b)
        for op, ex in ((oracle.r_add, A + B), (oracle.r_mul, A * B), (oracle.r_div, A / B)):
            out = op(L, a, b)
            if ex != 0:
                assert abs(fr_limbs(out) - ex) <= bound * abs(ex)


@pytest.mark.parametrize("L", [2, 4])
def test_cancellation_is_exact(L):
    """(1 + tiny) - 1 keeps the tiny part exactly: a double-only sum would lose it."""
    a = np.zeros(L)
    b = np.zeros(L)
    a[0], a[1] = 1.0, 2.0 ** -70
    b[0] = -1.0
    out = oracle.r_add(L, a, b)
    assert fr_limbs(out) == Fr(2) ** -70


@pytest.mark.parametrize("L", [1, 2, 4])
def test_complex_mul_div_within_bound(L):
    rng = np.random.default_rng(20 + L)
    bound = 4 * 2.0 ** (-52 * L)
    for _ in range(100):
        a = np.stack([rand_limbs(rng, L, 5), rand_limbs(rng, L, 5)])
        b = np.stack([rand_limbs(rng, L, 5), rand_limbs(rng, L, 5)])
        ar, ai = fr_c(a)
        br, bi = fr_c(b)
        pr, pi = ar * br - ai * bi, ar * bi + ai * br
        den = br * br + bi * bi
        qr, qi = (ar * br + ai * bi) / den, (ai * br - ar * bi) / den
        for out, (er, ei) in ((oracle.c_mul(L, a, b), (pr, pi)), (oracle.c_div(L, a, b), (qr, qi))):
            orr, oi = fr_c(out)
            mag = max(abs(er), abs(ei))
            assert abs(orr - er) <= bound * mag and abs(oi - ei) <= bound * mag


# ---------------------------------------------------------------------- evaluation (Sec. 6)
def tiny_integer_system(rng, n, mons, k, exps, const=False):
    s = synth.random_system(rng, n, mons, k, exps, const_term=const)
    s.coef = rng.integers(-7, 8, size=s.nmon) + 1j * rng.integers(-7, 8, size=s.nmon)
    return s


def sympy_f_and_J(s, xs):
    """f and J of the system at rational complex points by sympy: exact expansion of the
    definition and sympy.diff for the derivatives."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols(f"x0:{s.n}")
    F = []
    for i in range(s.npoly):
        expr = 0
        for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
            term = sp.Integer(int(s.coef[m].real)) + sp.I * sp.Integer(int(s.coef[m].imag))
            for q in range(s.var_ptr[m], s.var_ptr[m + 1]):
                term = term * X[s.var_idx[q]] ** int(s.var_exp[q])
            expr = expr + term
        F.append(expr)
    sub = {X[j]: sp.Rational(Fr(xs[j].real).numerator, Fr(xs[j].real).denominator)
           + sp.I * sp.Rational(Fr(xs[j].imag).numerator, Fr(xs[j].imag).denominator)
           for j in range(s.n)}
    fv = [sp.expand(e.subs(sub)) for e in F]
    Jv = [[sp.expand(sp.diff(e, X[j]).subs(sub)) for j in range(s.n)] for e in F]
    return fv, Jv


def sp_to_fr(v):
    import sympy as sp
    re, im = sp.re(v), sp.im(v)
    return Fr(int(sp.numer(re)), int(sp.denom(re))), Fr(int(sp.numer(im)), int(sp.denom(im)))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("L", [2, 4])
def test_eval_exact_on_dyadic_points(mode, L):
    """Integer coefficients at dyadic points: the DD/QD result equals the exact value
    (sympy expansion and sympy.diff), because every intermediate fits in the limbs."""
    rng = np.random.default_rng(30 + L + 10 * mode)
    s = tiny_integer_system(rng, 3, 4, (1, 3), (1, 3), const=True)
    xs = (rng.integers(-8, 9, size=3) + 1j * rng.integers(-8, 9, size=3)) / 4.0
    f, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), synth.limbs(xs[None, :], L),
                              mode=mode)
    fv, Jv = sympy_f_and_J(s, xs)
    for i in range(s.npoly):
        assert fr_c(f[0, i]) == sp_to_fr(fv[i])
        for j in range(s.n):
            assert fr_c(J[0, i, j]) == sp_to_fr(Jv[i][j]), (i, j)


def test_eval_matches_mpmath_at_400_bits():
    """Unit-circle coefficients at torus points: DD within 1e-30, QD within 1e-60 of an
    mpmath evaluation at 400 bits (normwise over f and over J)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    rng = np.random.default_rng(40)
    s = synth.random_system(rng, 4, 6, 3, (1, 4), const_term=True)
    xs = synth.torus_points(rng, 2, 4)
    for L, tol in ((2, 1e-30), (4, 1e-60)):
        f, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), synth.limbs(xs, L), mode=1)
        for p in range(2):
            X = [mpmath.mpc(float(z.real), float(z.imag)) for z in xs[p]]
            for i in range(s.npoly):
                fi = mpmath.mpc(0)
                Ji = [mpmath.mpc(0)] * s.n
                for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
                    c = mpmath.mpc(float(s.coef[m].real), float(s.coef[m].imag))
                    vs = list(range(s.var_ptr[m], s.var_ptr[m + 1]))
                    term = c
                    for q in vs:
                        term *= X[s.var_idx[q]] ** int(s.var_exp[q])
                    fi += term
                    for q in vs:
                        j = s.var_idx[q]
                        Ji[j] += term * int(s.var_exp[q]) / X[j]
                got = mpmath.mpc(*[mpmath.mpf(float(a)) for a in f[p, i, 0]][:1]) * 0
                gr = sum(mpmath.mpf(float(a)) for a in f[p, i, 0])
                gi = sum(mpmath.mpf(float(a)) for a in f[p, i, 1])
                got = mpmath.mpc(gr, gi)
                assert abs(got - fi) <= tol * max(1, abs(fi))
                for j in range(s.n):
                    gr = sum(mpmath.mpf(float(a)) for a in J[p, i, j, 0])
                    gi = sum(mpmath.mpf(float(a)) for a in J[p, i, j, 1])
                    assert abs(mpmath.mpc(gr, gi) - Ji[j]) <= tol * max(1, abs(Ji[j]))


def test_jacobian_matches_central_difference_in_qd():
    """dF/dx_j against (f(x + h e_j) - f(x - h e_j)) / 2h with h = 2^-66 in QD: the
    truncation error is O(h^2) ~ 1e-40, so a wrong derivative term shows at once."""
    rng = np.random.default_rng(50)
    s = synth.random_system(rng, 3, 5, (1, 3), (1, 4), const_term=True)
    L = 4
    x = synth.torus_points(rng, 1, 3)[0]
    h = 2.0 ** -66
    base = synth.limbs(x[None, :], L)
    _, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), base, mode=1)
    for j in range(3):
        xp = base.copy()
        xm = base.copy()
        # x_j +/- h exactly: h sits far below the leading limb, in the second limb
        xp[0, j, 0, 1] = h
        xm[0, j, 0, 1] = -h
        fp, _, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), xp, mode=1, jac=False)
        fm, _, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), xm, mode=1, jac=False)
        for i in range(3):
            dr = (fr_limbs(fp[0, i, 0]) - fr_limbs(fm[0, i, 0])) / (2 * Fr(h))
            di = (fr_limbs(fp[0, i, 1]) - fr_limbs(fm[0, i, 1])) / (2 * Fr(h))
            jr, ji = fr_c(J[0, i, j])
            assert abs(float(dr - jr)) < 1e-35 and abs(float(di - ji)) < 1e-35


@pytest.mark.parametrize("k", list(range(1, 13)))
def test_speelpenning_multiplication_count(k):
    """Sec. 6: all omega_m of a k-variable monomial in 3k-6 multiplications (k >= 2;
    none for k = 1)."""
    n = 12
    s = synth.System(n=n, npoly=1, mon_ptr=np.array([0, 1], np.int32),
                     var_ptr=np.array([0, k], np.int32),
                     var_idx=np.arange(k, dtype=np.int32),
                     var_exp=np.full(k, 2, np.int32), coef=np.array([1.0 + 0j]))
    x = synth.limbs(synth.torus_points(np.random.default_rng(k), 1, n), 2)
    _, _, cnt = oracle.evaluate(s.as_dict(), s.coef_limbs(2), x, mode=1)
    assert cnt == max(3 * k - 6, 0)


def test_ad_scheme_agrees_with_plain_definition():
    rng = np.random.default_rng(60)
    s = synth.random_system(rng, 6, 10, (1, 6), (1, 4), const_term=True)
    xs = synth.torus_points(rng, 3, 6)
    for L, tol in ((1, 1e-13), (2, 1e-29), (4, 1e-59)):
        c = s.coef_limbs(L)
        f0, J0, _ = oracle.evaluate(s.as_dict(), c, synth.limbs(xs, L), mode=0)
        f1, J1, _ = oracle.evaluate(s.as_dict(), c, synth.limbs(xs, L), mode=1)
        for a, b in ((f0, f1), (J0, J1)):
            va = a.sum(axis=-1)  # leading + lower limbs, approximately (for the norm only)
            vb = b.sum(axis=-1)
            assert np.max(np.abs(va - vb)) <= tol * np.max(np.abs(va)) + 1e-300


# ---------------------------------------------------------------------- homotopy (Sec. 3, 7)
@pytest.mark.parametrize("L", [1, 2, 4])
def test_start_point_is_exact_root_of_start_system(L):
    """At t = 0, h = gamma (x^d - 1) vanishes exactly at x = (1..1) and the Jacobian is
    exactly diag(gamma d_i) (in double, L = 1, gamma d_i is rounded once)."""
    if L == 1:
        pytest.skip("gamma * d_i is not exact in one limb")
    s, gamma = synth.single_path_dd(1)
    deg = oracle.degrees(s.as_dict())
    f, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), synth.limbs(np.ones((1, 8)), L),
                              t=0.0, gamma=np.array([gamma.real, gamma.imag]))
    assert np.all(f == 0.0)
    for i in range(8):
        for j in range(8):
            if i == j:
                # the limbs hold gamma * d_i exactly (d_i * gamma needs < 106 bits)
                assert fr_limbs(J[0, i, i, 0]) == Fr(gamma.real) * int(deg[i])
                assert fr_limbs(J[0, i, i, 1]) == Fr(gamma.imag) * int(deg[i])
            else:
                assert np.all(J[0, i, j] == 0.0)


def test_start_roots_of_unity():
    """Every x with x_i = exp(2 pi i j_i / d_i) is a root of the start system: h(x, 0) is
    at rounding level in QD."""
    s, gamma = synth.single_path_dd(1)
    deg = oracle.degrees(s.as_dict())
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 300
    rng = np.random.default_rng(70)
    L = 4
    x = np.zeros((1, 8, 2, L))
    for i in range(8):
        jj = int(rng.integers(0, deg[i]))
        z = mpmath.exp(2j * mpmath.pi * jj / int(deg[i]))
        for part, v in ((0, z.real), (1, z.imag)):
            rem = v
            for limb in range(L):
                x[0, i, part, limb] = float(rem)
                rem -= mpmath.mpf(x[0, i, part, limb])
    f, _, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), x, t=0.0,
                              gamma=np.array([gamma.real, gamma.imag]))
    assert np.max(np.abs(f[..., 0])) < 1e-60


def test_degrees_are_max_total_degree():
    s, _ = synth.single_path_dd(1)
    deg = oracle.degrees(s.as_dict())
    for i in range(8):
        best = 0
        for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
            best = max(best, int(s.var_exp[s.var_ptr[m]:s.var_ptr[m + 1]].sum()))
        assert deg[i] == best


# ---------------------------------------------------------------------- linear solve (Sec. 4)
def exact_complex_solve(A, b):
    """Gauss-Jordan over Q(i) with Fractions: independent exact reference."""
    n = len(A)
    M = [[A[i][j] for j in range(n)] + [b[i]] for i in range(n)]

    def mul(x, y):
        return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])

    def div(x, y):
        d = y[0] * y[0] + y[1] * y[1]
        return ((x[0] * y[0] + x[1] * y[1]) / d, (x[1] * y[0] - x[0] * y[1]) / d)

    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != (0, 0))
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i == k:
                continue
            l = div(M[i][k], M[k][k])
            M[i] = [(M[i][j][0] - mul(l, M[k][j])[0], M[i][j][1] - mul(l, M[k][j])[1])
                    for j in range(n + 1)]
    return [div(M[i][n], M[i][i]) for i in range(n)]


@pytest.mark.parametrize("L", [1, 2, 4])
@pytest.mark.parametrize("n", [1, 2, 5])
def test_solve_matches_exact_rational_elimination(L, n):
    rng = np.random.default_rng(80 + n)
    Ai = rng.integers(-9, 10, size=(n, n)) + 1j * rng.integers(-9, 10, size=(n, n))
    bi = rng.integers(-9, 10, size=n) + 1j * rng.integers(-9, 10, size=n)
    if abs(np.linalg.det(Ai)) < 1e-6:
        Ai += np.eye(n) * 20
    A = synth.limbs(Ai, L)
    b = synth.limbs(bi, L)
    x, rc = oracle.solve(A, b)
    assert rc == 0
    ex = exact_complex_solve([[(Fr(int(v.real)), Fr(int(v.imag))) for v in row] for row in Ai],
                             [(Fr(int(v.real)), Fr(int(v.imag))) for v in bi])
    cond = np.linalg.cond(Ai)
    tol = {1: 1e-15, 2: 1e-31, 4: 1e-62}[L] * 10 * cond * n
    scale = max(max(abs(float(e[0])), abs(float(e[1]))) for e in ex)
    for i in range(n):
        er, ei = fr_c(x[i])
        assert abs(float(er - ex[i][0])) <= tol * scale
        assert abs(float(ei - ex[i][1])) <= tol * scale


def test_solve_reports_singular():
    A = synth.limbs(np.array([[1, 2], [2, 4]], dtype=complex), 2)
    b = synth.limbs(np.array([1, 1], dtype=complex), 2)
    _, rc = oracle.solve(A, b)
    assert rc == 1


def test_partial_pivoting_picks_largest_modulus():
    """A zero leading entry needs the row swap; without pivoting the solve would divide
    by zero.  The exact solution of [[0,1],[1,0]] x = (a, b) is (b, a)."""
    A = synth.limbs(np.array([[0, 1], [1, 0]], dtype=complex), 2)
    b = synth.limbs(np.array([3 + 1j, -2 + 5j]), 2)
    x, rc = oracle.solve(A, b)
    assert rc == 0
    assert x[0, 0, 0] == -2 and x[0, 1, 0] == 5 and x[1, 0, 0] == 3 and x[1, 1, 0] == 1


# ---------------------------------------------------------------------- Newton (Alg. 4.1)
def univariate(seed, d):
    rng = np.random.default_rng(seed)
    # f(x) = sum_{e=0..d} c_e x^e, one polynomial in one unknown
    var_ptr = [0]
    idx, ex = [], []
    for e in range(d, -1, -1):
        if e > 0:
            idx.append(0)
            ex.append(e)
            var_ptr.append(var_ptr[-1] + 1)
        else:
            var_ptr.append(var_ptr[-1])
    th = rng.uniform(0, 2 * np.pi, size=d + 1)
    s = synth.System(n=1, npoly=1, mon_ptr=np.array([0, d + 1], np.int32),
                     var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                     var_exp=np.array(ex, np.int32), coef=np.cos(th) + 1j * np.sin(th))
    return s, synth.unit_complex(rng)


def roots_refined(s, digits=80):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = digits
    d = int(s.var_exp[0])
    coeffs = [mpmath.mpc(float(c.real), float(c.imag)) for c in s.coef]  # degree d .. 0
    return mpmath.polyroots(coeffs, maxsteps=200, extraprec=400)


def default_opts(**kw):
    o = oracle.TrackOpts(lambda0=0.01, lambda_min=1e-12, lambda_max=0.08, grow=2.0, shrink=0.5,
                         eps=1e-26, eps_x=1e-8, eps_end=1e-26, eps_end_x=1e-26, div_bound=1e6,
                         max_it=3, end_it=8, grow_after=3, max_steps=100000, predictor=0,
                         lu_mode=0, max_refine=4)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("lu_mode", [0, 1])
def test_newton_converges_quadratically_to_polynomial_root(lu_mode):
    """Newton on a univariate polynomial from a point 1e-3 away from a root (mpmath
    polyroots): the error squares at every step until DD rounding."""
    mpmath = pytest.importorskip("mpmath")
    s, g = univariate(90, 5)
    r = roots_refined(s)[0]
    L = 2
    x = synth.limbs(np.array([[complex(r) * (1 + 1e-3)]]), L)
    errs = []
    for _ in range(4):
        x, res, st, _ = oracle.newton_step(s.as_dict(), s.coef_limbs(L), x, -1.0, np.array([1.0, 0.0]),
                                           lu_mode=lu_mode)
        assert st[0] == 0
        xr = mpmath.mpc(sum(mpmath.mpf(float(v)) for v in x[0, 0, 0]),
                        sum(mpmath.mpf(float(v)) for v in x[0, 0, 1]))
        errs.append(float(abs(xr - r) / abs(r)))
    assert errs[0] < 1e-5 and errs[1] < 1e-10 and errs[2] < 1e-20 and errs[3] < 1e-30


def test_mixed_solve_matches_native_solve():
    rng = np.random.default_rng(95)
    s = synth.random_system(rng, 5, 6, (1, 4), (1, 3))
    g = synth.unit_complex(rng)
    x = synth.limbs(synth.torus_points(rng, 3, 5), 2)
    ga = np.array([g.real, g.imag])
    a, ra, sa, _ = oracle.newton_step(s.as_dict(), s.coef_limbs(2), x, 0.4, ga, lu_mode=0)
    b, rb, sb, sw = oracle.newton_step(s.as_dict(), s.coef_limbs(2), x, 0.4, ga, lu_mode=1,
                                       max_refine=6)
    assert np.all(sa == 0) and np.all(sb == 0)
    assert np.all(ra == rb)
    va, vb = a.sum(-1), b.sum(-1)
    assert np.max(np.abs(va - vb)) < 1e-28 * np.max(np.abs(va))
    assert np.all(sw >= 1)


# ---------------------------------------------------------------------- tracker (Alg. 3.1)
@pytest.mark.parametrize("seed", [100, 101, 102])
def test_univariate_track_ends_at_a_root(seed):
    """n = 1: the total-degree homotopy has no path to infinity, so the path from x = 1
    ends at a root of f; the end point equals an mpmath polyroots root to 1e-28."""
    mpmath = pytest.importorskip("mpmath")
    s, g = univariate(seed, 6)
    L = 2
    r = oracle.track(s.as_dict(), s.coef_limbs(L), synth.limbs(np.ones(1), L),
                     np.array([g.real, g.imag]), default_opts())
    assert oracle.STATUS[r.status] == "OK"
    xr = mpmath.mpc(sum(mpmath.mpf(float(v)) for v in r.x[0, 0]),
                    sum(mpmath.mpf(float(v)) for v in r.x[0, 1]))
    best = min(float(abs(xr - z) / abs(z)) for z in roots_refined(s))
    assert best < 1e-28


def test_track_step_sizes_follow_the_halving_rule():
    """Tables 2-3 invariants: every accepted step except a clipped last one is
    lambda0 * 2^j, and the accepted steps add up to the path length 1."""
    s, g = univariate(103, 5)
    r = oracle.track(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(1), 2),
                     np.array([g.real, g.imag]), default_opts(), log_cap=100000)
    acc = r.log[r.log["accepted"] == 1]
    lam = acc["lam"][:-1]
    j = np.log2(lam / 0.01)
    # t + lambda rounds in double, so the realised step is lambda0 2^j up to that rounding
    assert np.max(np.abs(j - np.round(j))) < 1e-9
    assert abs(acc["lam"].sum() - 1.0) < 1e-12
    assert abs(r.n_succ * r.avg_step - 1.0) < 1e-12
    assert r.n_succ == len(acc) and r.n_corr == len(r.log)


def _linear_system(A, b):
    """f_i = sum_j A_ij x_j - b_i as a sparse system (every x_j a monomial of degree 1)."""
    n = A.shape[0]
    mon_ptr, var_ptr, idx, ex, coef = [0], [0], [], [], []
    for i in range(n):
        for j in range(n):
            idx.append(j)
            ex.append(1)
            var_ptr.append(var_ptr[-1] + 1)
            coef.append(A[i, j])
        var_ptr.append(var_ptr[-1])
        coef.append(-b[i])
        mon_ptr.append(len(coef))
    return synth.System(n=n, npoly=n, mon_ptr=np.array(mon_ptr, np.int32), var_ptr=np.array(var_ptr, np.int32),
                        var_idx=np.array(idx, np.int32), var_exp=np.array(ex, np.int32),
                        coef=np.array(coef, dtype=complex))


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("log_cond", [6, 12])
def test_refined_solve_of_an_ill_conditioned_system_reaches_the_working_precision(L, log_cond):
    """One Newton step from 0 on a linear system f = A x - b is x = A^-1 b.  With A
    conditioned to 10^6 or 10^12, the FP64 LU gains only 10 or 4 digits a refinement sweep;
    the mixed solve (and its stop rule: a correction that does not shrink is not applied)
    must still reach the exact solution (mpmath at 400 bits) to within cond x the precision,
    as the native elimination in the working precision does."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    rng = np.random.default_rng(990 + L + log_cond)
    n = 4
    q1, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    q2, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    A = q1 @ np.diag(np.logspace(0, -log_cond, n)) @ q2
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    s = _linear_system(A, b)
    Am = mpmath.matrix([[mpmath.mpc(A[i, j].real, A[i, j].imag) for j in range(n)] for i in range(n)])
    bm = mpmath.matrix([mpmath.mpc(v.real, v.imag) for v in b])
    xm = mpmath.lu_solve(Am, bm)
    xnorm = max(abs(xm[i]) for i in range(n))
    x0 = np.zeros((1, n, 2, L))
    bound = 100 * 10.0 ** log_cond * 2.0 ** (-52 * L)
    for lu_mode, refine in ((0, 1), (1, 64)):
        x1, _, st, sw = oracle.newton_step(s.as_dict(), s.coef_limbs(L), x0, -1.0, np.array([1.0, 0.0]),
                                           lu_mode, refine)
        assert st[0] == 0
        got = [mpmath.mpc(sum(mpmath.mpf(float(v)) for v in x1[0, i, 0]),
                          sum(mpmath.mpf(float(v)) for v in x1[0, i, 1])) for i in range(n)]
        err = max(abs(got[i] - xm[i]) for i in range(n)) / xnorm
        assert err <= bound, (lu_mode, L, log_cond, float(err), int(sw[0]))
        if lu_mode == 1:
            assert 1 <= sw[0] < 64   # the refinement stopped by itself


def test_paths_of_a_system_without_finite_roots_do_not_end_ok():
    """f_1 = x_1 x_2 - 1, f_2 = x_1 x_2 - 2 has no finite root, while the total-degree start
    system has 4: every path from a start root goes to infinity, so none may end as OK;
    each stops as DIVERGED (|x| above the bound) or MIN_STEP (the step collapsed near the
    end), with |x| far above its start."""
    s = synth.System(n=2, npoly=2, mon_ptr=np.array([0, 2, 4], np.int32),
                     var_ptr=np.array([0, 2, 2, 4, 4], np.int32), var_idx=np.array([0, 1, 0, 1], np.int32),
                     var_exp=np.array([1, 1, 1, 1], np.int32), coef=np.array([1, -1, 1, -2], dtype=complex))
    g = synth.unit_complex(np.random.default_rng(1010))
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            x0 = synth.limbs(np.array([a, b], dtype=complex), 2)
            r = oracle.track(s.as_dict(), s.coef_limbs(2), x0, np.array([g.real, g.imag]), default_opts())
            assert oracle.STATUS[r.status] in ("DIVERGED", "MIN_STEP"), (a, b, oracle.STATUS[r.status])
            xmax = max(abs(complex(r.x[j, 0, 0], r.x[j, 1, 0])) for j in range(2))
            assert xmax > 10.0, (a, b, xmax)


def test_eval_at_high_degree_matches_mpmath():
    """The shapes the parity tests need the oracle for at high degree: 8 rows of Table 1's
    common-support system (degree up to 80, up to 32 variables a monomial) and monomials
    of exponent 64, at torus points: DD and QD within 1e-28 / 1e-58 of mpmath at 400 bits,
    normwise over a point's values and over its Jacobian."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 400
    full, _ = synth.common_support_system(1)
    rows = list(range(8))
    mon_ptr, var_ptr, idx, ex, coef = [0], [0], [], [], []
    for i in rows:
        for m in range(full.mon_ptr[i], full.mon_ptr[i + 1]):
            q0, q1 = full.var_ptr[m], full.var_ptr[m + 1]
            idx.extend(full.var_idx[q0:q1])
            ex.extend(full.var_exp[q0:q1])
            var_ptr.append(var_ptr[-1] + q1 - q0)
            coef.append(full.coef[m])
        mon_ptr.append(len(coef))
    # and one row of exponent-64 monomials
    for vs in ([0, 5], [31], [3, 7, 11]):
        idx.extend(vs)
        ex.extend([64] * len(vs))
        var_ptr.append(var_ptr[-1] + len(vs))
        coef.append(np.exp(1j * len(vs)))
    mon_ptr.append(len(coef))
    s = synth.System(n=full.n, npoly=len(rows) + 1, mon_ptr=np.array(mon_ptr, np.int32),
                     var_ptr=np.array(var_ptr, np.int32), var_idx=np.array(idx, np.int32),
                     var_exp=np.array(ex, np.int32), coef=np.array(coef))
    assert int(s.var_exp.max()) == 64 and max(np.diff(s.var_ptr)) >= 20
    xs = synth.torus_points(np.random.default_rng(1020), 2, s.n)
    for L, tol in ((2, 1e-28), (4, 1e-58)):
        f, J, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(L), synth.limbs(xs, L), mode=1)
        for p in range(2):
            X = [mpmath.mpc(float(z.real), float(z.imag)) for z in xs[p]]
            fe, Je = [], []
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
                fe.append(fi)
                Je.append(Ji)

            def val(a):
                return mpmath.mpc(sum(mpmath.mpf(float(v)) for v in a[0]), sum(mpmath.mpf(float(v)) for v in a[1]))
            fscale = max(abs(v) for v in fe)
            jscale = max(abs(v) for row in Je for v in row)
            assert max(abs(val(f[p, i]) - fe[i]) for i in range(s.npoly)) <= tol * fscale
            assert max(abs(val(J[p, i, j]) - Je[i][j]) for i in range(s.npoly) for j in range(s.n)) <= tol * jscale
