/*
 * hc_oracle.c -- plain, slow CPU oracle for the hot path of the multithreaded path
 * tracker of Verschelde & Yoffe, "Quality Up in Polynomial Homotopy Continuation by
 * Multithreaded Path Tracking" (2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library.  The product library never links it,
 * and this file shares no code, header, table or helper with the CUDA path.
 *
 * Arithmetic.  A real number is held as L doubles (L = 1 double, 2 double-double,
 * 4 quad-double; Sec. 1 and Sec. 2 of the paper use double doubles and quad doubles).
 * Every elementary operation is carried out EXACTLY on floating-point expansions
 * (Shewchuk's expansion arithmetic: Knuth's two-sum, Dekker's split-based two-product,
 * no fused multiply-add; this file must be compiled with -ffp-contract=off) and the exact
 * result is rounded ONCE to L limbs by compressing the expansion and keeping its L
 * largest components.  The rounding error of each operation is therefore below
 * about 2^(-52 L) of the result, independent of how the GPU path forms its
 * error-free transforms.
 *
 * What is computed (each routine cites the passage it follows):
 *   - polynomial values and all partial derivatives, by the plain definition
 *     (or_eval mode 0) and by the common-factor / Speelpenning scheme of Sec. 6
 *     (or_eval mode 1, with a multiplication counter for the 3k-6 claim);
 *   - the homotopy h(x,t) = gamma (1-t) g(x) + t f(x), g_i = x_i^{d_i} - 1, with t a
 *     parameter, not a variable (Sec. 7, Table 6 caption);
 *   - Gaussian elimination with partial pivoting on [A b] and back substitution (Sec. 4);
 *   - one Newton step (Alg. 4.1), native or FP64 LU with L-limb refinement;
 *   - the path tracker loop of Alg. 3.1 with a secant or quadratic (Sec. 5) predictor,
 *     from t = 0 (or_track), from a saved state for a bounded number of stages
 *     (or_track_resume), or along a given sequence of accepted t (or_track_replay); the
 *     three share one implementation of each stage's steps.
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_tracker_pins.py) tie each routine to
 * exact rationals, sympy, mpmath or closed forms: the predictors to exact polynomial
 * interpolation, the tracker to homotopies whose paths are exactly linear or quadratic
 * in t and to decoupled systems whose paths are continued roots in closed form, the
 * homotopy at 0 < t < 1 to mpmath.  Parity unpinned: the exact stage-by-stage
 * trajectory (which steps are accepted) of or_track on a general coupled system with
 * n > 1.  Only its invariants (steps on the lambda0 2^-j lattice, accepted steps adding
 * up to 1), its univariate end points, the constructed and decoupled paths and the
 * start-system roots are pinned.
 *
 * Readings of the paper where it is silent or garbled are stated at each routine.
 * Layout of every array here is point-major, array-of-structures:
 *   x[p][j][2][L], f[p][i][2][L], J[p][i][j][2][L], coef[m][2][L] (re limbs, im limbs).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXL 4
#define OR_XLEN 512 /* scratch length of an expansion */

/* ------------------------------------------------------------------------------------
 * Error-free transformations (Knuth two-sum, Dekker fast-two-sum, split, two-product).
 * ---------------------------------------------------------------------------------- */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

static void fast_two_sum(double a, double b, double *s, double *e)
{
    /* requires |a| >= |b| or a == 0 */
    double x = a + b;
    *s = x;
    *e = b - (x - a);
}

static void split(double a, double *hi, double *lo)
{
    const double c = 134217729.0; /* 2^27 + 1 */
    double t = c * a;
    double h = t - (t - a);
    *hi = h;
    *lo = a - h;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    double err1 = x - ah * bh;
    double err2 = err1 - al * bh;
    double err3 = err2 - ah * bl;
    *p = x;
    *e = al * bl - err3;
}

/* ------------------------------------------------------------------------------------
 * Expansions: arrays of doubles, nonoverlapping, increasing magnitude (Shewchuk 1997).
 * ---------------------------------------------------------------------------------- */

/* h = e + b exactly (Grow-Expansion); zero components are dropped. */
static int grow(int m, const double *e, double b, double *h)
{
    double q = b;
    int k = 0;
    for (int i = 0; i < m; i++) {
        double s, err;
        two_sum(q, e[i], &s, &err);
        q = s;
        if (err != 0.0) h[k++] = err;
    }
    if (q != 0.0 || k == 0) h[k++] = q;
    return k;
}

/* h = e + f exactly (Expansion-Sum by repeated growth). */
static int esum(int m, const double *e, int n, const double *f, double *h)
{
    double a[OR_XLEN], b[OR_XLEN];
    int len = m;
    memcpy(a, e, sizeof(double) * (size_t)m);
    for (int i = 0; i < n; i++) {
        len = grow(len, a, f[i], b);
        memcpy(a, b, sizeof(double) * (size_t)len);
    }
    memcpy(h, a, sizeof(double) * (size_t)len);
    return len;
}

/* h = e * b exactly (Scale-Expansion). */
static int escale(int m, const double *e, double b, double *h)
{
    double out[OR_XLEN];
    int k = 0;
    double q, lo;
    if (m == 0) { h[0] = 0.0; return 1; }
    two_prod(e[0], b, &q, &lo);
    if (lo != 0.0) out[k++] = lo;
    for (int i = 1; i < m; i++) {
        double tp, tl, s, err;
        two_prod(e[i], b, &tp, &tl);
        two_sum(q, tl, &s, &err);
        if (err != 0.0) out[k++] = err;
        fast_two_sum(tp, s, &q, &err);
        if (err != 0.0) out[k++] = err;
    }
    if (q != 0.0 || k == 0) out[k++] = q;
    memcpy(h, out, sizeof(double) * (size_t)k);
    return k;
}

/* Compress: same value, nonadjacent components, largest component approximates the sum. */
static int compress(int m, const double *e, double *h)
{
    double g[OR_XLEN];
    if (m == 0) { h[0] = 0.0; return 1; }
    int bottom = m - 1;
    double q = e[m - 1];
    for (int i = m - 2; i >= 0; i--) {
        double s, lo;
        fast_two_sum(q, e[i], &s, &lo);
        if (lo != 0.0) {
            g[bottom--] = s;
            q = lo;
        } else {
            q = s;
        }
    }
    g[bottom] = q;
    int top = 0;
    for (int i = bottom + 1; i < m; i++) {
        double s, lo;
        fast_two_sum(g[i], q, &s, &lo);
        if (lo != 0.0) h[top++] = lo;
        q = s;
    }
    h[top] = q;
    return top + 1;
}

/* ------------------------------------------------------------------------------------
 * L-limb reals.  v[0] is the leading limb; the limbs are nonoverlapping.
 * ---------------------------------------------------------------------------------- */
typedef struct { double v[OR_MAXL]; } R;
typedef struct { R re, im; } C;

/* The expansion of an L-limb value, formed exactly even if the limbs overlap. */
static int r_exp(int L, const R *a, double *h)
{
    double t[OR_XLEN];
    int m = 0;
    for (int j = L - 1; j >= 0; j--) {
        if (a->v[j] == 0.0) continue;
        m = grow(m, t, a->v[j], h);
        memcpy(t, h, sizeof(double) * (size_t)m);
    }
    if (m == 0) { h[0] = 0.0; return 1; }
    memcpy(h, t, sizeof(double) * (size_t)m);
    return m;
}

/* Round an exact expansion to L limbs: compress, keep the L largest components. */
static R r_round(int L, int m, const double *e)
{
    double h[OR_XLEN];
    R r;
    memset(&r, 0, sizeof r);
    int n = compress(m, e, h);
    for (int j = 0; j < L && n - 1 - j >= 0; j++) r.v[j] = h[n - 1 - j];
    return r;
}

static R r_from_d(double d)
{
    R r;
    memset(&r, 0, sizeof r);
    r.v[0] = d;
    return r;
}

/* exact product of two expansions */
static int emul(int m, const double *e, int n, const double *f, double *h)
{
    double acc[OR_XLEN], part[OR_XLEN], tmp[OR_XLEN];
    int len = 1;
    acc[0] = 0.0;
    for (int j = 0; j < n; j++) {
        int pl = escale(m, e, f[j], part);
        len = esum(len, acc, pl, part, tmp);
        len = compress(len, tmp, acc);
    }
    memcpy(h, acc, sizeof(double) * (size_t)len);
    return len;
}

static void eneg(int m, double *e)
{
    for (int i = 0; i < m; i++) e[i] = -e[i];
}

static R r_add(int L, R a, R b)
{
    double ea[OR_XLEN], eb[OR_XLEN], h[OR_XLEN];
    int ma = r_exp(L, &a, ea), mb = r_exp(L, &b, eb);
    return r_round(L, esum(ma, ea, mb, eb, h), h);
}

static R r_neg(int L, R a)
{
    for (int j = 0; j < L; j++) a.v[j] = -a.v[j];
    return a;
}

static R r_mul(int L, R a, R b)
{
    double ea[OR_XLEN], eb[OR_XLEN], h[OR_XLEN];
    int ma = r_exp(L, &a, ea), mb = r_exp(L, &b, eb);
    return r_round(L, emul(ma, ea, mb, eb, h), h);
}

/* num / den for exact expansions: long division with exact remainders, one rounding. */
static R e_div(int L, int mn, const double *num, int md, const double *den)
{
    double r[OR_XLEN], t[OR_XLEN], dd[OR_XLEN], q[OR_XLEN], part[OR_XLEN];
    int mr = compress(mn, num, r);
    int mdd = compress(md, den, dd);
    double dtop = dd[mdd - 1];
    int mq = 1;
    q[0] = 0.0;
    for (int it = 0; it < L + 2; it++) {
        double rtop = r[mr - 1];
        if (rtop == 0.0) break;
        double qj = rtop / dtop;
        mq = grow(mq, q, qj, t);
        memcpy(q, t, sizeof(double) * (size_t)mq);
        int pl = escale(mdd, dd, -qj, part);
        int ml = esum(mr, r, pl, part, t);
        mr = compress(ml, t, r);
    }
    return r_round(L, mq, q);
}

static R r_div(int L, R a, R b)
{
    double ea[OR_XLEN], eb[OR_XLEN];
    int ma = r_exp(L, &a, ea), mb = r_exp(L, &b, eb);
    return e_div(L, ma, ea, mb, eb);
}

/* ---- complex ---- */
static C c_zero(void)
{
    C z;
    memset(&z, 0, sizeof z);
    return z;
}

static C c_from(double re, double im)
{
    C z = c_zero();
    z.re.v[0] = re;
    z.im.v[0] = im;
    return z;
}

static C c_add(int L, C a, C b)
{
    C z;
    z.re = r_add(L, a.re, b.re);
    z.im = r_add(L, a.im, b.im);
    return z;
}

static C c_sub(int L, C a, C b)
{
    C z;
    z.re = r_add(L, a.re, r_neg(L, b.re));
    z.im = r_add(L, a.im, r_neg(L, b.im));
    return z;
}

/* exact expansion of a.re*b.re - a.im*b.im (sgn=-1) or a.re*b.im + a.im*b.re */
static int e_dot2(int L, R a1, R b1, R a2, R b2, double sgn, double *h)
{
    double e1[OR_XLEN], e2[OR_XLEN], f1[OR_XLEN], f2[OR_XLEN], p1[OR_XLEN], p2[OR_XLEN];
    int m1 = r_exp(L, &a1, e1), n1 = r_exp(L, &b1, f1);
    int m2 = r_exp(L, &a2, e2), n2 = r_exp(L, &b2, f2);
    int l1 = emul(m1, e1, n1, f1, p1);
    int l2 = emul(m2, e2, n2, f2, p2);
    if (sgn < 0) eneg(l2, p2);
    return esum(l1, p1, l2, p2, h);
}

/* complex product, each component rounded once from its exact value */
static C c_mul(int L, C a, C b)
{
    double h[OR_XLEN];
    C z;
    int m = e_dot2(L, a.re, b.re, a.im, b.im, -1.0, h);
    z.re = r_round(L, m, h);
    m = e_dot2(L, a.re, b.im, a.im, b.re, 1.0, h);
    z.im = r_round(L, m, h);
    return z;
}

/* complex times an L-limb real */
static C c_mul_r(int L, C a, R s)
{
    C z;
    z.re = r_mul(L, a.re, s);
    z.im = r_mul(L, a.im, s);
    return z;
}

/* a - l*b with one rounding per component (the elimination update of Sec. 4) */
static C c_fnma(int L, C a, C l, C b)
{
    double h[OR_XLEN], ea[OR_XLEN], t[OR_XLEN];
    C z;
    int m = e_dot2(L, l.re, b.re, l.im, b.im, -1.0, h);
    eneg(m, h);
    int ma = r_exp(L, &a.re, ea);
    int mt = esum(ma, ea, m, h, t);
    z.re = r_round(L, mt, t);
    m = e_dot2(L, l.re, b.im, l.im, b.re, 1.0, h);
    eneg(m, h);
    ma = r_exp(L, &a.im, ea);
    mt = esum(ma, ea, m, h, t);
    z.im = r_round(L, mt, t);
    return z;
}

/* a / b = a conj(b) / |b|^2, numerator and denominator exact, one rounding per part */
static C c_div(int L, C a, C b)
{
    double num[OR_XLEN], den[OR_XLEN];
    C z;
    int md = e_dot2(L, b.re, b.re, b.im, b.im, 1.0, den);
    /* re: a.re*b.re + a.im*b.im ; im: a.im*b.re - a.re*b.im */
    int mn = e_dot2(L, a.re, b.re, a.im, b.im, 1.0, num);
    z.re = e_div(L, mn, num, md, den);
    mn = e_dot2(L, a.im, b.re, a.re, b.im, -1.0, num);
    z.im = e_div(L, mn, num, md, den);
    return z;
}

/* leading-limb squared modulus in plain double: the pivot and norm measure */
static double c_abs2_lead(C a)
{
    double r = a.re.v[0], i = a.im.v[0];
    return r * r + i * i;
}

static C c_load(int L, const double *p)
{
    C z = c_zero();
    for (int j = 0; j < L; j++) {
        z.re.v[j] = p[j];
        z.im.v[j] = p[L + j];
    }
    return z;
}

static void c_store(int L, C z, double *p)
{
    for (int j = 0; j < L; j++) {
        p[j] = z.re.v[j];
        p[L + j] = z.im.v[j];
    }
}

static int valid_L(int L) { return L == 1 || L == 2 || L == 4; }

/* ------------------------------------------------------------------------------------
 * Exported arithmetic primitives (for pin tests against exact rationals).
 * Inputs/outputs: L limbs each, leading limb first.
 * ---------------------------------------------------------------------------------- */
int or_r_add(int L, const double *a, const double *b, double *out)
{
    if (!valid_L(L)) return -1;
    R x, y;
    memset(&x, 0, sizeof x);
    memset(&y, 0, sizeof y);
    for (int j = 0; j < L; j++) { x.v[j] = a[j]; y.v[j] = b[j]; }
    R z = r_add(L, x, y);
    for (int j = 0; j < L; j++) out[j] = z.v[j];
    return 0;
}

int or_r_mul(int L, const double *a, const double *b, double *out)
{
    if (!valid_L(L)) return -1;
    R x, y;
    memset(&x, 0, sizeof x);
    memset(&y, 0, sizeof y);
    for (int j = 0; j < L; j++) { x.v[j] = a[j]; y.v[j] = b[j]; }
    R z = r_mul(L, x, y);
    for (int j = 0; j < L; j++) out[j] = z.v[j];
    return 0;
}

int or_r_div(int L, const double *a, const double *b, double *out)
{
    if (!valid_L(L)) return -1;
    R x, y;
    memset(&x, 0, sizeof x);
    memset(&y, 0, sizeof y);
    for (int j = 0; j < L; j++) { x.v[j] = a[j]; y.v[j] = b[j]; }
    R z = r_div(L, x, y);
    for (int j = 0; j < L; j++) out[j] = z.v[j];
    return 0;
}

/* complex ops: a, b, out are [2][L] (re limbs, im limbs) */
int or_c_mul(int L, const double *a, const double *b, double *out)
{
    if (!valid_L(L)) return -1;
    c_store(L, c_mul(L, c_load(L, a), c_load(L, b)), out);
    return 0;
}

int or_c_div(int L, const double *a, const double *b, double *out)
{
    if (!valid_L(L)) return -1;
    c_store(L, c_div(L, c_load(L, a), c_load(L, b)), out);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * System description (as handed to the oracle; the same CSR the library's loader takes):
 *   polynomial i owns monomials mon_ptr[i] .. mon_ptr[i+1]-1;
 *   monomial m owns variables var_ptr[m] .. var_ptr[m+1]-1, indices var_idx[], exponents
 *   var_exp[]; k = var_ptr[m+1]-var_ptr[m] = 0 is a constant term.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int n, npoly;
    const int32_t *mon_ptr, *var_ptr, *var_idx, *var_exp;
    const double *coef; /* [nmon][2][L] */
} sysdesc;

/* Check the normalised form of Sec. 6: indices strictly increasing in [0,n), exps >= 1. */
int or_validate(int n, int npoly, const int32_t *mon_ptr, const int32_t *var_ptr,
                const int32_t *var_idx, const int32_t *var_exp)
{
    if (n < 1 || npoly < 1) return -1;
    if (mon_ptr[0] != 0) return -2;
    for (int i = 0; i < npoly; i++)
        if (mon_ptr[i + 1] < mon_ptr[i]) return -3;
    int nmon = mon_ptr[npoly];
    if (var_ptr[0] != 0) return -4;
    for (int m = 0; m < nmon; m++) {
        if (var_ptr[m + 1] < var_ptr[m]) return -5;
        for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++) {
            if (var_idx[q] < 0 || var_idx[q] >= n) return -6;
            if (var_exp[q] < 1) return -7;
            if (q > var_ptr[m] && var_idx[q] <= var_idx[q - 1]) return -8;
        }
        if (var_ptr[m + 1] - var_ptr[m] > 63) return -9;
    }
    return 0;
}

/* d_i = the largest total degree of a monomial of f_i (the degree of the start system). */
int or_degrees(int npoly, const int32_t *mon_ptr, const int32_t *var_ptr,
               const int32_t *var_exp, int32_t *deg)
{
    for (int i = 0; i < npoly; i++) {
        int32_t d = 0;
        for (int m = mon_ptr[i]; m < mon_ptr[i + 1]; m++) {
            int32_t s = 0;
            for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++) s += var_exp[q];
            if (s > d) d = s;
        }
        deg[i] = d;
    }
    return 0;
}

/* c * a for a small positive integer a, rounded once */
static C c_mul_int(int L, C c, int a)
{
    return c_mul_r(L, c, r_from_d((double)a));
}

/* x^e by repeated multiplication, x^0 = 1 (Sec. 6 reading: powers by x^p = x^(p-1) x) */
static C c_pow(int L, C x, int e)
{
    C r = c_from(1.0, 0.0);
    for (int p = 0; p < e; p++) r = (p == 0) ? x : c_mul(L, r, x);
    return r;
}

/*
 * Evaluate f (and J = df/dx) at one point by the PLAIN DEFINITION:
 *   f_i = sum_mon c * prod_j x_{i_j}^{a_j},
 *   df_i/dx_l = sum_{mon containing l} (c a_l) x^{a - e_l},
 * every power by repeated multiplication, no shared factors.
 */
static void eval_plain_point(int L, const sysdesc *s, const C *x, C *f, C *J)
{
    int n = s->n;
    for (int i = 0; i < s->npoly; i++) {
        C fi = c_zero();
        C *Ji = J ? J + (size_t)i * n : NULL;
        if (Ji)
            for (int j = 0; j < n; j++) Ji[j] = c_zero();
        for (int m = s->mon_ptr[i]; m < s->mon_ptr[i + 1]; m++) {
            C c = c_load(L, s->coef + (size_t)m * 2 * L);
            int q0 = s->var_ptr[m], q1 = s->var_ptr[m + 1];
            C term = c;
            for (int q = q0; q < q1; q++)
                for (int e = 0; e < s->var_exp[q]; e++) term = c_mul(L, term, x[s->var_idx[q]]);
            fi = c_add(L, fi, term);
            if (!Ji) continue;
            for (int qm = q0; qm < q1; qm++) {
                C d = c_mul_int(L, c, s->var_exp[qm]);
                for (int q = q0; q < q1; q++) {
                    int e = s->var_exp[q] - (q == qm ? 1 : 0);
                    for (int r = 0; r < e; r++) d = c_mul(L, d, x[s->var_idx[q]]);
                }
                Ji[s->var_idx[qm]] = c_add(L, Ji[s->var_idx[qm]], d);
            }
        }
        f[i] = fi;
    }
}

/*
 * Evaluate f and J at one point by the algorithmic-differentiation scheme of Sec. 6.
 * For a normalised monomial x_{i1}^{a1} ... x_{ik}^{ak}:
 *   1. common factor CF = prod_j x_{ij}^{aj-1} (from a per-point power table built by
 *      repeated multiplication);
 *   2. prefix products psi_m = psi_{m-1} x_{im}, psi_1 = x_{i1}, m = 1..k-1;
 *      suffix products phi_m = phi_{m-1} x_{i(k-m+1)}, phi_1 = x_{ik}, m = 1..k-1;
 *      Speelpenning products omega_m = prod_{j != m} x_{ij}:
 *        omega_1 = phi_{k-1}, omega_k = psi_{k-1}, omega_m = psi_{m-1} phi_{k-m}.
 *      The printed indices (omega_1 = psi_{k-1}, omega_k = phi_{k-1},
 *      omega_m = psi_{m-1} phi_{k-m+2}) contradict the definition of omega_m; this
 *      routine follows the definition.  These take 3k-6 multiplications for k >= 2;
 *      *nmul_omega accumulates that count.
 *   3. the partial monomials D_m = CF omega_m = x^{a - e_m};
 *   4. the monomial itself, D_1 x_{i1}.
 * Coefficient_Product (Alg. 4.1) then adds c * value into f_i and (c a_m) D_m into
 * J_{i,im}; the factor a_m is applied here, with the coefficient.
 */
static void eval_ad_point(int L, const sysdesc *s, const C *x, C *f, C *J, long *nmul_omega,
                          C *pw, int emax)
{
    int n = s->n;
    /* power table pw[j*emax + p] = x_j^p, p = 0..emax-1 */
    for (int j = 0; j < n; j++) {
        pw[(size_t)j * emax] = c_from(1.0, 0.0);
        for (int p = 1; p < emax; p++)
            pw[(size_t)j * emax + p] = (p == 1) ? x[j] : c_mul(L, pw[(size_t)j * emax + p - 1], x[j]);
    }
    C psi[64], phi[64], om[64], D[64];
    for (int i = 0; i < s->npoly; i++) {
        C fi = c_zero();
        C *Ji = J ? J + (size_t)i * n : NULL;
        if (Ji)
            for (int j = 0; j < n; j++) Ji[j] = c_zero();
        for (int m = s->mon_ptr[i]; m < s->mon_ptr[i + 1]; m++) {
            C c = c_load(L, s->coef + (size_t)m * 2 * L);
            int q0 = s->var_ptr[m], k = s->var_ptr[m + 1] - q0;
            const int32_t *id = s->var_idx + q0, *ex = s->var_exp + q0;
            if (k == 0) {
                fi = c_add(L, fi, c);
                continue;
            }
            /* 1. common factor */
            C cf = c_from(1.0, 0.0);
            int have = 0;
            for (int j = 0; j < k; j++) {
                if (ex[j] < 2) continue;
                C pj = pw[(size_t)id[j] * emax + ex[j] - 1];
                cf = have ? c_mul(L, cf, pj) : pj;
                have = 1;
            }
            /* 2. Speelpenning products (index 1..k in the paper -> 0..k-1 here) */
            if (k == 1) {
                om[0] = c_from(1.0, 0.0);
            } else {
                psi[1] = x[id[0]];
                for (int mm = 2; mm <= k - 1; mm++) {
                    psi[mm] = c_mul(L, psi[mm - 1], x[id[mm - 1]]);
                    (*nmul_omega)++;
                }
                phi[1] = x[id[k - 1]];
                for (int mm = 2; mm <= k - 1; mm++) {
                    phi[mm] = c_mul(L, phi[mm - 1], x[id[k - mm]]);
                    (*nmul_omega)++;
                }
                om[0] = phi[k - 1];
                om[k - 1] = psi[k - 1];
                for (int mm = 2; mm <= k - 1; mm++) {
                    om[mm - 1] = c_mul(L, psi[mm - 1], phi[k - mm]);
                    (*nmul_omega)++;
                }
            }
            /* 3. partial monomials */
            for (int j = 0; j < k; j++) D[j] = have ? c_mul(L, cf, om[j]) : om[j];
            /* 4. the monomial */
            C val = c_mul(L, D[0], x[id[0]]);
            /* Coefficient_Product */
            fi = c_add(L, fi, c_mul(L, c, val));
            if (Ji)
                for (int j = 0; j < k; j++)
                    Ji[id[j]] = c_add(L, Ji[id[j]], c_mul(L, c_mul_int(L, c, ex[j]), D[j]));
        }
        f[i] = fi;
    }
}

/*
 * Homotopy assembly with t a parameter (Sec. 7, Table 6 caption):
 *   h_i = gamma (1-t) (x_i^{d_i} - 1) + t f_i,
 *   dh_i/dx_j = t J_ij + [i == j] gamma (1-t) d_i x_i^{d_i - 1}.
 * 1-t is formed exactly and rounded to L limbs.  Requires npoly == n.
 */
static void homotopy_point(int L, int n, const int32_t *deg, double t, C gamma, const C *x,
                           C *f, C *J)
{
    double s, e;
    two_sum(1.0, -t, &s, &e);
    double ex[2] = {e, s}; /* increasing magnitude */
    R omt = (e != 0.0) ? r_round(L, 2, ex) : r_round(L, 1, ex + 1);
    C gs = c_mul_r(L, gamma, omt);
    R tr = r_from_d(t);
    for (int i = 0; i < n; i++) {
        C xd1 = c_pow(L, x[i], deg[i] - 1);
        C xd = c_mul(L, xd1, x[i]);
        C g = c_sub(L, xd, c_from(1.0, 0.0));
        f[i] = c_add(L, c_mul(L, gs, g), c_mul_r(L, f[i], tr));
        if (J) {
            for (int j = 0; j < n; j++) J[(size_t)i * n + j] = c_mul_r(L, J[(size_t)i * n + j], tr);
            C dg = c_mul_int(L, xd1, deg[i]);
            J[(size_t)i * n + i] = c_add(L, J[(size_t)i * n + i], c_mul(L, gs, dg));
        }
    }
}

static int max_exp(const sysdesc *s)
{
    int e = 1;
    int nmon = s->mon_ptr[s->npoly];
    for (int q = 0; q < s->var_ptr[nmon]; q++)
        if (s->var_exp[q] > e) e = s->var_exp[q];
    return e;
}

/* evaluate at one point: f (npoly) and optionally J (npoly x n); t < 0 means f itself */
static void eval_point(int L, const sysdesc *s, const int32_t *deg, int mode, double t,
                       C gamma, const C *x, C *f, C *J, long *nmul)
{
    if (mode == 1) {
        int emax = max_exp(s);
        C *pw = (C *)malloc(sizeof(C) * (size_t)s->n * (size_t)emax);
        eval_ad_point(L, s, x, f, J, nmul, pw, emax);
        free(pw);
    } else {
        eval_plain_point(L, s, x, f, J);
    }
    if (t >= 0.0) homotopy_point(L, s->n, deg, t, gamma, x, f, J);
}

/*
 * or_eval: values and Jacobians of f (t < 0) or of h(., t) (t >= 0) at npts points.
 * mode 0: plain definition; mode 1: Sec. 6 scheme (nmul_omega gets the count of
 * multiplications spent on the Speelpenning products omega_m, summed over points).
 * x[npts][n][2][L] -> f[npts][npoly][2][L], J[npts][npoly][n][2][L] (J may be NULL).
 */
int or_eval(int L, int mode, int n, int npoly, const int32_t *mon_ptr, const int32_t *var_ptr,
            const int32_t *var_idx, const int32_t *var_exp, const double *coef, int npts,
            const double *x, double t, const double *gamma, double *f, double *J,
            long *nmul_omega)
{
    if (!valid_L(L)) return -1;
    if (or_validate(n, npoly, mon_ptr, var_ptr, var_idx, var_exp) != 0) return -2;
    if (t >= 0.0 && npoly != n) return -3;
    if (n > 1024) return -4;
    sysdesc s = {n, npoly, mon_ptr, var_ptr, var_idx, var_exp, coef};
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)npoly);
    or_degrees(npoly, mon_ptr, var_ptr, var_exp, deg);
    C gam = c_from(gamma ? gamma[0] : 1.0, gamma ? gamma[1] : 0.0);
    C *xv = (C *)malloc(sizeof(C) * (size_t)n);
    C *fv = (C *)malloc(sizeof(C) * (size_t)npoly);
    C *Jv = J ? (C *)malloc(sizeof(C) * (size_t)npoly * (size_t)n) : NULL;
    long cnt = 0;
    for (int p = 0; p < npts; p++) {
        for (int j = 0; j < n; j++) xv[j] = c_load(L, x + ((size_t)p * n + j) * 2 * L);
        eval_point(L, &s, deg, mode, t, gam, xv, fv, Jv, &cnt);
        for (int i = 0; i < npoly; i++) c_store(L, fv[i], f + ((size_t)p * npoly + i) * 2 * L);
        if (J)
            for (size_t q = 0; q < (size_t)npoly * n; q++)
                c_store(L, Jv[q], J + ((size_t)p * npoly * n + q) * 2 * L);
    }
    if (nmul_omega) *nmul_omega = cnt;
    free(deg);
    free(xv);
    free(fv);
    free(Jv);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Linear solve of Sec. 4: Gaussian elimination with partial pivoting on the augmented
 * matrix [A b], then back substitution.  The pivot is the entry of largest modulus in
 * the current column, measured as re^2 + im^2 of the leading limbs in plain double;
 * ties go to the lowest row.  Returns 0, or 1 if a pivot is exactly zero (singular).
 * ---------------------------------------------------------------------------------- */
static int ge_solve(int L, int n, C *M /* n x (n+1), row-major, destroyed */, C *z)
{
    int w = n + 1;
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = c_abs2_lead(M[(size_t)k * w + k]);
        for (int i = k + 1; i < n; i++) {
            double v = c_abs2_lead(M[(size_t)i * w + k]);
            if (v > best) { best = v; p = i; }
        }
        if (!(best > 0.0)) return 1;
        if (p != k)
            for (int j = 0; j < w; j++) {
                C tmp = M[(size_t)k * w + j];
                M[(size_t)k * w + j] = M[(size_t)p * w + j];
                M[(size_t)p * w + j] = tmp;
            }
        for (int i = k + 1; i < n; i++) {
            C l = c_div(L, M[(size_t)i * w + k], M[(size_t)k * w + k]);
            for (int j = k + 1; j < w; j++)
                M[(size_t)i * w + j] = c_fnma(L, M[(size_t)i * w + j], l, M[(size_t)k * w + j]);
            M[(size_t)i * w + k] = c_zero();
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        C s = M[(size_t)i * w + n];
        for (int j = i + 1; j < n; j++) s = c_fnma(L, s, M[(size_t)i * w + j], z[j]);
        z[i] = c_div(L, s, M[(size_t)i * w + i]);
    }
    return 0;
}

/* exported: A[n][n][2][L], b[n][2][L] -> x[n][2][L]; returns 0 ok, 1 singular */
int or_solve(int L, int n, const double *A, const double *b, double *x)
{
    if (!valid_L(L) || n < 1) return -1;
    C *M = (C *)malloc(sizeof(C) * (size_t)n * (size_t)(n + 1));
    C *z = (C *)malloc(sizeof(C) * (size_t)n);
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) M[(size_t)i * (n + 1) + j] = c_load(L, A + ((size_t)i * n + j) * 2 * L);
        M[(size_t)i * (n + 1) + n] = c_load(L, b + (size_t)i * 2 * L);
    }
    int rc = ge_solve(L, n, M, z);
    if (rc == 0)
        for (int i = 0; i < n; i++) c_store(L, z[i], x + (size_t)i * 2 * L);
    free(M);
    free(z);
    return rc;
}

/*
 * Mixed-precision solve: factor the leading limbs of A in plain double (the same
 * elimination, L = 1), then refine in L-limb arithmetic:
 *   dz_0 = LU^{-1} b_lead;  r = b - A dz;  dz += LU^{-1} r_lead;
 * Stop after max_refine sweeps, or once the correction is below 2^(-53 L) of
 * max(||x||, ||dz||) (x + dz is formed next, so that is the working precision of the
 * update).  A correction no smaller than the previous one (the residual is at its
 * rounding floor, or the double factors cannot reduce it) stops the refinement and is
 * not added.  Returns 0/1 as ge_solve; *sweeps receives the number of refinement sweeps.
 */
static int mixed_solve(int L, int n, const C *A, const C *b, C *z, int max_refine,
                       double xnorm, int *sweeps)
{
    int w = n + 1;
    C *M = (C *)malloc(sizeof(C) * (size_t)n * (size_t)w);
    C *d = (C *)malloc(sizeof(C) * (size_t)n);
    C *r = (C *)malloc(sizeof(C) * (size_t)n);
    int rc = 0;
    double tol = ldexp(1.0, -53 * L), prev = INFINITY;
    *sweeps = 0;
    /* the first solve and every correction solve use the double LU; a plain-double
       re-elimination of [A_lead r_lead] is the same arithmetic as reusing the factors */
    for (int it = 0; it <= max_refine; it++) {
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++) {
                C a = A[(size_t)i * n + j];
                M[(size_t)i * w + j] = c_from(a.re.v[0], a.im.v[0]);
            }
            C rhs;
            if (it == 0) {
                rhs = b[i];
            } else {
                /* r_i = b_i - sum_j A_ij z_j in L-limb arithmetic */
                C s = b[i];
                for (int j = 0; j < n; j++) s = c_fnma(L, s, A[(size_t)i * n + j], z[j]);
                rhs = s;
                r[i] = s;
            }
            M[(size_t)i * w + n] = c_from(rhs.re.v[0], rhs.im.v[0]);
        }
        rc = ge_solve(1, n, M, d);
        if (rc) break;
        if (it == 0) {
            for (int i = 0; i < n; i++) {
                z[i] = c_zero();
                z[i].re.v[0] = d[i].re.v[0];
                z[i].im.v[0] = d[i].im.v[0];
            }
            continue;
        }
        double dn = 0.0, zn = 0.0;
        for (int i = 0; i < n; i++) {
            double v = sqrt(c_abs2_lead(d[i]));
            if (v > dn) dn = v;
        }
        *sweeps = it;
        /* a correction no smaller than the previous one (the residual is at its rounding
           floor, or the double factors cannot reduce it) ends the refinement unapplied */
        if (dn >= prev) break;
        for (int i = 0; i < n; i++) {
            z[i] = c_add(L, z[i], c_from(d[i].re.v[0], d[i].im.v[0]));
            double v = sqrt(c_abs2_lead(z[i]));
            if (v > zn) zn = v;
        }
        if (dn <= tol * (xnorm > zn ? xnorm : zn)) break;
        prev = dn;
    }
    free(M);
    free(d);
    free(r);
    return rc;
}

/* ------------------------------------------------------------------------------------
 * Newton step (Alg. 4.1, one pass of its loop body):
 *   evaluate h and its Jacobian at z, ||h||_inf (max over i of |h_i| from the leading
 *   limbs), solve J dz = -h, z := z + dz.
 * lu_mode 0: native L-limb elimination; 1: FP64 LU with L-limb refinement.
 * ---------------------------------------------------------------------------------- */
enum { OR_OK = 0, OR_NOCONV = 1, OR_SINGULAR = 2, OR_MIN_STEP = 3, OR_MAX_STEPS = 4,
       OR_DIVERGED = 5, OR_NONFINITE = 6 };

static double cnorm_inf_lead(int n, const C *z);

static int newton_once(int L, const sysdesc *s, const int32_t *deg, double t, C gamma, C *z,
                       int lu_mode, int max_refine, double *res, int *sweeps, C *fv, C *Jv,
                       C *M, C *dz, double *dzn, double *zn)
{
    int n = s->n;
    long cnt = 0;
    eval_point(L, s, deg, 1, t, gamma, z, fv, Jv, &cnt);
    double r2 = 0.0;
    int finite = 1;
    for (int i = 0; i < n; i++) {
        double v = c_abs2_lead(fv[i]);
        if (!isfinite(v)) finite = 0;
        if (v > r2) r2 = v;
    }
    *res = sqrt(r2);
    if (!finite) return OR_NONFINITE;
    int rc;
    *sweeps = 0;
    if (lu_mode == 0) {
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++) M[(size_t)i * (n + 1) + j] = Jv[(size_t)i * n + j];
            C b = fv[i];
            b.re = r_neg(L, b.re);
            b.im = r_neg(L, b.im);
            M[(size_t)i * (n + 1) + n] = b;
        }
        rc = ge_solve(L, n, M, dz);
    } else {
        C *b = (C *)malloc(sizeof(C) * (size_t)n);
        for (int i = 0; i < n; i++) {
            b[i] = fv[i];
            b[i].re = r_neg(L, b[i].re);
            b[i].im = r_neg(L, b[i].im);
        }
        rc = mixed_solve(L, n, Jv, b, dz, max_refine, cnorm_inf_lead(n, z), sweeps);
        free(b);
    }
    if (rc) return OR_SINGULAR;
    for (int i = 0; i < n; i++) z[i] = c_add(L, z[i], dz[i]);
    if (dzn) *dzn = cnorm_inf_lead(n, dz);
    if (zn) *zn = cnorm_inf_lead(n, z);
    for (int i = 0; i < n; i++)
        if (!isfinite(z[i].re.v[0]) || !isfinite(z[i].im.v[0])) return OR_NONFINITE;
    return OR_OK;
}

/* exported batch Newton step over npts points; x[npts][n][2][L] in/out */
int or_newton_step(int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
                   const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                   int npts, double t, const double *gamma, double *x, int lu_mode,
                   int max_refine, double *res_norm, int32_t *status, int32_t *sweeps)
{
    if (!valid_L(L)) return -1;
    if (or_validate(n, n, mon_ptr, var_ptr, var_idx, var_exp) != 0) return -2;
    sysdesc s = {n, n, mon_ptr, var_ptr, var_idx, var_exp, coef};
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_degrees(n, mon_ptr, var_ptr, var_exp, deg);
    C gam = c_from(gamma[0], gamma[1]);
    C *z = (C *)malloc(sizeof(C) * (size_t)n);
    C *fv = (C *)malloc(sizeof(C) * (size_t)n);
    C *Jv = (C *)malloc(sizeof(C) * (size_t)n * (size_t)n);
    C *M = (C *)malloc(sizeof(C) * (size_t)n * (size_t)(n + 1));
    C *dz = (C *)malloc(sizeof(C) * (size_t)n);
    for (int p = 0; p < npts; p++) {
        for (int j = 0; j < n; j++) z[j] = c_load(L, x + ((size_t)p * n + j) * 2 * L);
        double res;
        int sw;
        int st = newton_once(L, &s, deg, t, gam, z, lu_mode, max_refine, &res, &sw, fv, Jv, M, dz,
                             NULL, NULL);
        if (res_norm) res_norm[p] = res;
        if (status) status[p] = st;
        if (sweeps) sweeps[p] = sw;
        if (st == OR_OK)
            for (int j = 0; j < n; j++) c_store(L, z[j], x + ((size_t)p * n + j) * 2 * L);
    }
    free(deg);
    free(z);
    free(fv);
    free(Jv);
    free(M);
    free(dz);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Path tracker (Alg. 3.1) around the Newton corrector (Alg. 4.1).
 *
 * Readings (the paper gives no constants and no predictor formula for Alg. 3.1):
 *  - t = 0, z = start solution, lambda = lambda0;
 *  - while t < 1 and not stop: predict at t' = min(t + lambda, 1); run Newton at t'
 *    (Alg. 4.1: evaluate, residual of the evaluated z, solve, update; repeat while not
 *    converged and iterations < max_it).  The paper names neither the norm nor the
 *    tolerance; converged := ||h(z,t')||_inf <= eps  or  ||dz||_inf <= eps_x max(1,
 *    ||z||_inf) for the update just applied (norms from the leading limbs, in double).
 *    The second test keeps the criterion meaningful when ||z|| grows along a path
 *    that diverges, where an absolute residual test can no longer be met;
 *  - success: accept (t', z), shift the history; after grow_after consecutive successes
 *    lambda := min(grow * lambda, lambda_max);
 *    failure: step back to the last accepted (t, z), lambda := shrink * lambda;
 *  - stop if lambda < lambda_min (status MIN_STEP) or the number of corrector stages
 *    reaches max_steps (MAX_STEPS); ||z||_inf > div_bound is DIVERGED;
 *  - fail := (t < 1)  (Alg. 3.1 prints "fail := not stop", which contradicts its own
 *    comment "failure if stopped with t < 1");
 *  - at t = 1, up to end_it further Newton iterations on h(., 1) = f until converged
 *    with the tolerances eps_end, eps_end_x.
 * Predictors: 0 secant (linear through the last two accepted points; zeroth order when
 * there is only one), 1 quadratic (Sec. 5: per coordinate, the parabola through the
 * last three accepted points, evaluated at t'; lower order while fewer exist).
 *
 * The loop is split into the steps the three drivers share: or_track (from t = 0 to the
 * end), or_track_resume (at most a given number of stages from a saved state) and
 * or_track_replay (along a given sequence of accepted t values).
 * ---------------------------------------------------------------------------------- */
typedef struct {
    double lambda0, lambda_min, lambda_max, grow, shrink;
    double eps, eps_x, eps_end, eps_end_x, div_bound;
    int32_t max_it, end_it, grow_after, max_steps, predictor, lu_mode, max_refine, log_cap;
} or_opts;

typedef struct {
    int64_t n_succ, n_corr, newton_its;
    double min_step, avg_step, t_end, res_end;
    int32_t status, end_its;
} or_stats;

/* per corrector-stage log record (what the learned step proposer trains on) */
typedef struct {
    double t, lambda, res_first, res_last, pc_dist;
    int32_t iters, accepted;
} or_steplog;

/* The state of a path between corrector stages: the current point's t and the two
 * accepted values before it, the next step, the step controller's counters and the
 * statistics of Tables 2-3.  phase: 1 tracking, 2 at t = 1 with the end game to run,
 * 3 done.  The points themselves (z, z_prev, z_prev2) are held by the caller. */
typedef struct {
    double t, tp, tpp, lambda, min_step, sum_step, res_end;
    int64_t n_succ, n_corr, newton_its;
    int32_t nhist, consec, status, phase, end_its, pad;
} or_state;

static double cnorm_inf_lead(int n, const C *z)
{
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        double v = c_abs2_lead(z[i]);
        if (!(v <= m)) m = v; /* propagates NaN */
    }
    return sqrt(m);
}

static void state_init(or_state *st, const or_opts *o)
{
    memset(st, 0, sizeof *st);
    st->lambda = o->lambda0;
    st->min_step = INFINITY;
    st->res_end = -1.0;
    st->nhist = 1;
    st->status = OR_OK;
    st->phase = 1;
}

/* Predictor (Alg. 3.1 "predict"; Sec. 5 for the quadratic one): the predicted point zh
 * at t1 from the accepted points z (at t), zp (at tp) and zpp (at tpp), of which the
 * first nhist exist.  Quadratic: the Lagrange form of the parabola through the three,
 * its weights w0, w1, w2 formed in double; secant: z + (z - zp) (t1 - t) / (t - tp);
 * zeroth order: z.  Each product of a point with a double weight is rounded once. */
static void predict(int L, int n, int predictor, int nhist, double t, double tp, double tpp,
                    double t1, const C *z, const C *zp, const C *zpp, C *zh)
{
    if (predictor == 1 && nhist >= 3) {
        double w0 = ((t1 - tp) * (t1 - t)) / ((tpp - tp) * (tpp - t));
        double w1 = ((t1 - tpp) * (t1 - t)) / ((tp - tpp) * (tp - t));
        double w2 = ((t1 - tpp) * (t1 - tp)) / ((t - tpp) * (t - tp));
        for (int j = 0; j < n; j++) {
            C a = c_mul_r(L, zpp[j], r_from_d(w0));
            C b = c_mul_r(L, zp[j], r_from_d(w1));
            C c = c_mul_r(L, z[j], r_from_d(w2));
            zh[j] = c_add(L, c_add(L, a, b), c);
        }
    } else if (nhist >= 2) {
        double r = (t1 - t) / (t - tp);
        for (int j = 0; j < n; j++)
            zh[j] = c_add(L, z[j], c_mul_r(L, c_sub(L, z[j], zp[j]), r_from_d(r)));
    } else {
        memcpy(zh, z, sizeof(C) * (size_t)n);
    }
}

/* exported predictor: points are [n][2][L]; returns -1 on a bad argument */
int or_predict(int L, int n, int predictor, int nhist, double t, double tp, double tpp,
               double t1, const double *z, const double *zp, const double *zpp, double *zh)
{
    if (!valid_L(L) || n < 1 || nhist < 1 || nhist > 3) return -1;
    C *buf = (C *)malloc(sizeof(C) * (size_t)n * 4);
    C *a = buf, *b = buf + n, *c = buf + 2 * (size_t)n, *out = buf + 3 * (size_t)n;
    for (int j = 0; j < n; j++) {
        a[j] = c_load(L, z + (size_t)j * 2 * L);
        b[j] = c_load(L, zp + (size_t)j * 2 * L);
        c[j] = c_load(L, zpp + (size_t)j * 2 * L);
    }
    predict(L, n, predictor, nhist, t, tp, tpp, t1, a, b, c, out);
    for (int j = 0; j < n; j++) c_store(L, out[j], zh + (size_t)j * 2 * L);
    free(buf);
    return 0;
}

/* scratch of one path */
typedef struct {
    C *zh, *fv, *Jv, *M, *dz;
} or_work;

static void work_alloc(or_work *w, int n)
{
    size_t nc = (size_t)n;
    w->zh = (C *)malloc(sizeof(C) * nc);
    w->fv = (C *)malloc(sizeof(C) * nc);
    w->Jv = (C *)malloc(sizeof(C) * nc * nc);
    w->M = (C *)malloc(sizeof(C) * nc * (nc + 1));
    w->dz = (C *)malloc(sizeof(C) * nc);
}

static void work_free(or_work *w)
{
    free(w->zh); free(w->fv); free(w->Jv); free(w->M); free(w->dz);
}

/* Corrector (Alg. 4.1) at t1 on zh in place: at most max_it Newton iterations until
 * ||h||_inf <= eps or the update just applied has ||dz||_inf <= eps_x max(1, ||z||_inf).
 * Returns the status of the last iteration; *its, *conv, *res (residual of the last
 * iterate evaluated) and *res_first (of the first) as outputs. */
static int correct(int L, const sysdesc *s, const int32_t *deg, C gam, const or_opts *o,
                   double t1, int max_it, double eps, double eps_x, or_work *w, int *its,
                   int *conv, double *res, double *res_first)
{
    int nst = OR_OK;
    *its = 0;
    *conv = 0;
    *res = 1.0;
    *res_first = -1.0;
    while (!*conv && *its < max_it) {
        int sw;
        double dzn = 0.0, zn = 0.0;
        nst = newton_once(L, s, deg, t1, gam, w->zh, o->lu_mode, o->max_refine, res, &sw, w->fv,
                          w->Jv, w->M, w->dz, &dzn, &zn);
        if (*res_first < 0) *res_first = *res;
        (*its)++;
        if (nst != OR_OK) break;
        *conv = (*res <= eps) || (dzn <= eps_x * (zn > 1.0 ? zn : 1.0));
    }
    return nst;
}

/* Accept the corrected point zh at t1: shift the history (z -> zp -> zpp), t's, counts. */
static void accept_point(or_state *st, int n, C *z, C *zp, C *zpp, const C *zh, double t1)
{
    size_t b = sizeof(C) * (size_t)n;
    double h = t1 - st->t;
    memcpy(zpp, zp, b);
    memcpy(zp, z, b);
    memcpy(z, zh, b);
    st->tpp = st->tp;
    st->tp = st->t;
    st->t = t1;
    if (st->nhist < 3) st->nhist++;
    st->n_succ++;
    st->sum_step += h;
    if (h < st->min_step) st->min_step = h;
}

/* End game at t = 1: up to end_it Newton iterations on f; phase 2 -> 3. */
static void end_game(int L, const sysdesc *s, const int32_t *deg, C gam, const or_opts *o,
                     or_state *st, C *z, or_work *w)
{
    int n = s->n, its, conv;
    double res, res_first;
    memcpy(w->zh, z, sizeof(C) * (size_t)n);
    int nst = correct(L, s, deg, gam, o, 1.0, o->end_it, o->eps_end, o->eps_end_x, w, &its, &conv,
                      &res, &res_first);
    /* every iteration that ran moved z (an iteration that failed left zh unchanged) */
    memcpy(z, w->zh, sizeof(C) * (size_t)n);
    st->end_its += its;
    st->res_end = res;
    if (nst != OR_OK) st->status = nst;
    else if (!conv) st->status = OR_NOCONV;
    st->phase = 3;
}

/* One corrector stage of Alg. 3.1 from state st (phase 1): predict, correct, accept or
 * step back, step-size control, stop tests; the log record if asked for. */
static void stage(int L, const sysdesc *s, const int32_t *deg, C gam, const or_opts *o,
                  or_state *st, C *z, C *zp, C *zpp, or_work *w, or_steplog *log, int log_cap,
                  int32_t *nl)
{
    int n = s->n;
    double t1 = st->t + st->lambda;
    if (t1 > 1.0) t1 = 1.0;
    double h = t1 - st->t;
    predict(L, n, o->predictor, st->nhist, st->t, st->tp, st->tpp, t1, z, zp, zpp, w->zh);
    int its, conv;
    double res, res_first;
    int nst = correct(L, s, deg, gam, o, t1, o->max_it, o->eps, o->eps_x, w, &its, &conv, &res,
                      &res_first);
    st->newton_its += its;
    st->n_corr++;
    int ok = (nst == OR_OK) && conv, stop = 0;
    double znorm = cnorm_inf_lead(n, w->zh);
    if (ok && !(znorm <= o->div_bound)) {
        ok = 0;
        st->status = isfinite(znorm) ? OR_DIVERGED : OR_NONFINITE;
        stop = 1;
    }
    if (log && *nl < log_cap) {
        /* the distance between the predicted and the corrected point is not logged */
        or_steplog *rec = &log[(*nl)++];
        rec->t = st->t;
        rec->lambda = h;
        rec->res_first = res_first;
        rec->res_last = res;
        rec->iters = its;
        rec->accepted = ok;
        rec->pc_dist = -1.0;
    }
    if (ok) {
        accept_point(st, n, z, zp, zpp, w->zh, t1);
        st->consec++;
        if (st->consec >= o->grow_after) {
            st->lambda = st->lambda * o->grow;
            if (st->lambda > o->lambda_max) st->lambda = o->lambda_max;
            st->consec = 0;
        }
    } else if (!stop) {
        st->consec = 0;
        st->lambda = st->lambda * o->shrink;
        if (st->lambda < o->lambda_min) { stop = 1; st->status = OR_MIN_STEP; }
    }
    if (!stop && st->t < 1.0 && st->n_corr >= o->max_steps) { stop = 1; st->status = OR_MAX_STEPS; }
    if (stop) st->phase = 3;
    else if (st->t >= 1.0) st->phase = 2;
}

/* At most max_stages corrector stages from st, then the end game if t = 1 was reached. */
static void run_stages(int L, const sysdesc *s, const int32_t *deg, C gam, const or_opts *o,
                       or_state *st, C *z, C *zp, C *zpp, int64_t max_stages, or_steplog *log,
                       int32_t *nl)
{
    or_work w;
    work_alloc(&w, s->n);
    for (int64_t k = 0; st->phase == 1 && k < max_stages; k++)
        stage(L, s, deg, gam, o, st, z, zp, zpp, &w, log, o->log_cap, nl);
    if (st->phase == 2) end_game(L, s, deg, gam, o, st, z, &w);
    work_free(&w);
}

static void stats_of(const or_state *st, or_stats *out)
{
    out->n_succ = st->n_succ;
    out->n_corr = st->n_corr;
    out->newton_its = st->newton_its;
    out->min_step = st->n_succ ? st->min_step : 0.0;
    out->avg_step = st->n_succ ? st->sum_step / (double)st->n_succ : 0.0;
    out->t_end = st->t;
    out->res_end = st->res_end;
    out->status = st->status;
    out->end_its = st->end_its;
}

typedef struct {
    sysdesc s;
    int32_t *deg;
    C gam, *z, *zp, *zpp;
} or_path;

static int path_open(or_path *p, int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
                     const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                     const double *gamma)
{
    if (!valid_L(L)) return -1;
    if (or_validate(n, n, mon_ptr, var_ptr, var_idx, var_exp) != 0) return -2;
    sysdesc s = {n, n, mon_ptr, var_ptr, var_idx, var_exp, coef};
    p->s = s;
    p->deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_degrees(n, mon_ptr, var_ptr, var_exp, p->deg);
    p->gam = c_from(gamma[0], gamma[1]);
    p->z = (C *)calloc((size_t)n, sizeof(C));
    p->zp = (C *)calloc((size_t)n, sizeof(C));
    p->zpp = (C *)calloc((size_t)n, sizeof(C));
    return 0;
}

static void path_close(or_path *p)
{
    free(p->deg); free(p->z); free(p->zp); free(p->zpp);
}

static void load_vec(int L, int n, const double *src, C *dst)
{
    for (int j = 0; j < n; j++) dst[j] = c_load(L, src + (size_t)j * 2 * L);
}

static void store_vec(int L, int n, const C *src, double *dst)
{
    for (int j = 0; j < n; j++) c_store(L, src[j], dst + (size_t)j * 2 * L);
}

/* or_track: one path from x0 at t = 0 to its end (Alg. 3.1).  x0, x1 are [n][2][L]; x1
 * gets the last accepted point (the end point if the status is OK). */
int or_track(int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
             const int32_t *var_idx, const int32_t *var_exp, const double *coef,
             const double *gamma, const double *x0, const or_opts *o, double *x1,
             or_stats *st, or_steplog *log, int32_t *nlog)
{
    or_path p;
    int rc = path_open(&p, L, n, mon_ptr, var_ptr, var_idx, var_exp, coef, gamma);
    if (rc) return rc;
    or_state s;
    state_init(&s, o);
    load_vec(L, n, x0, p.z);
    int32_t nl = 0;
    run_stages(L, &p.s, p.deg, p.gam, o, &s, p.z, p.zp, p.zpp, INT64_MAX, log, &nl);
    store_vec(L, n, p.z, x1);
    if (st) stats_of(&s, st);
    if (nlog) *nlog = nl;
    path_close(&p);
    return 0;
}

/* or_track_resume: at most max_stages corrector stages of one path from a saved state
 * (then the end game if t = 1 is reached), the state saved again.  state->phase == 0
 * starts the path at t = 0 from z.  z, zp, zpp: [n][2][L] in/out, the current point and
 * the two accepted points before it (the first state->nhist of the three are used). */
int or_track_resume(int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
                    const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                    const double *gamma, const or_opts *o, or_state *state, double *z,
                    double *zp, double *zpp, int64_t max_stages, or_stats *st,
                    or_steplog *log, int32_t *nlog)
{
    or_path p;
    int rc = path_open(&p, L, n, mon_ptr, var_ptr, var_idx, var_exp, coef, gamma);
    if (rc) return rc;
    if (state->phase == 0) state_init(state, o);
    load_vec(L, n, z, p.z);
    load_vec(L, n, zp, p.zp);
    load_vec(L, n, zpp, p.zpp);
    int32_t nl = 0;
    run_stages(L, &p.s, p.deg, p.gam, o, state, p.z, p.zp, p.zpp, max_stages, log, &nl);
    store_vec(L, n, p.z, z);
    store_vec(L, n, p.zp, zp);
    store_vec(L, n, p.zpp, zpp);
    if (st) stats_of(state, st);
    if (nlog) *nlog = nl;
    path_close(&p);
    return 0;
}

/*
 * Replay: follow a given sequence of accepted parameter values t_1 < t_2 < ... (as a
 * tracker with any step-size controller produced them) with the predictor and the
 * corrector of or_track, and then its end game.  Every stage must converge: the oracle
 * judges each accepted step.  *fail_at gets the index of the first stage the corrector
 * rejects (status NOCONV), or -1.
 */
int or_track_replay(int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
                    const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                    const double *gamma, const double *x0, const or_opts *o, const double *tseq,
                    int nseq, double *x1, int32_t *fail_at, or_stats *st)
{
    or_path p;
    int rc = path_open(&p, L, n, mon_ptr, var_ptr, var_idx, var_exp, coef, gamma);
    if (rc) return rc;
    or_state s;
    state_init(&s, o);
    load_vec(L, n, x0, p.z);
    or_work w;
    work_alloc(&w, n);
    *fail_at = -1;
    for (int k = 0; k < nseq; k++) {
        double t1 = tseq[k];
        predict(L, n, o->predictor, s.nhist, s.t, s.tp, s.tpp, t1, p.z, p.zp, p.zpp, w.zh);
        int its, conv;
        double res, res_first;
        int nst = correct(L, &p.s, p.deg, p.gam, o, t1, o->max_it, o->eps, o->eps_x, &w, &its,
                          &conv, &res, &res_first);
        s.newton_its += its;
        s.n_corr++;
        if (!(nst == OR_OK && conv)) {
            *fail_at = k;
            s.status = OR_NOCONV;
            s.phase = 3;
            break;
        }
        accept_point(&s, n, p.z, p.zp, p.zpp, w.zh, t1);
    }
    if (s.phase == 1 && s.t >= 1.0) end_game(L, &p.s, p.deg, p.gam, o, &s, p.z, &w);
    work_free(&w);
    store_vec(L, n, p.z, x1);
    if (st) stats_of(&s, st);
    path_close(&p);
    return 0;
}
/* ------------------------------------------------------------------------------------
 * Threaded batch driver for the CPU baseline: or_eval (mode 1) over points on nthreads
 * POSIX threads, each thread a contiguous block of points.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int L, n, npoly;
    const int32_t *mon_ptr, *var_ptr, *var_idx, *var_exp;
    const double *coef, *x, *gamma;
    double t;
    double *f, *J;
    int p0, p1, rc;
} eval_job;

static void *eval_worker(void *arg)
{
    eval_job *j = (eval_job *)arg;
    size_t L2 = 2 * (size_t)j->L;
    j->rc = or_eval(j->L, 1, j->n, j->npoly, j->mon_ptr, j->var_ptr, j->var_idx, j->var_exp,
                    j->coef, j->p1 - j->p0, j->x + (size_t)j->p0 * j->n * L2, j->t, j->gamma,
                    j->f + (size_t)j->p0 * j->npoly * L2,
                    j->J ? j->J + (size_t)j->p0 * j->npoly * j->n * L2 : NULL, NULL);
    return NULL;
}

int or_eval_threads(int L, int n, int npoly, const int32_t *mon_ptr, const int32_t *var_ptr,
                    const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                    int npts, const double *x, double t, const double *gamma, double *f,
                    double *J, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > npts) nthreads = npts > 0 ? npts : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    eval_job *jobs = (eval_job *)malloc(sizeof(eval_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        eval_job *j = &jobs[k];
        j->L = L; j->n = n; j->npoly = npoly;
        j->mon_ptr = mon_ptr; j->var_ptr = var_ptr; j->var_idx = var_idx; j->var_exp = var_exp;
        j->coef = coef; j->x = x; j->gamma = gamma; j->t = t; j->f = f; j->J = J;
        j->p0 = (int)((long)npts * k / nthreads);
        j->p1 = (int)((long)npts * (k + 1) / nthreads);
        j->rc = 0;
        pthread_create(&th[k], NULL, eval_worker, j);
    }
    int rc = 0;
    for (int k = 0; k < nthreads; k++) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
    }
    free(th);
    free(jobs);
    return rc;
}

/* Threaded batch driver for the CPU baseline: or_newton_step over points on nthreads
 * POSIX threads, each thread a contiguous block of points. */
typedef struct {
    int L, n;
    const int32_t *mon_ptr, *var_ptr, *var_idx, *var_exp;
    const double *coef, *gamma;
    double t, *x, *res;
    int32_t *status, *sweeps;
    int lu_mode, max_refine, p0, p1, rc;
} newton_job;

static void *newton_worker(void *arg)
{
    newton_job *j = (newton_job *)arg;
    size_t w = (size_t)j->n * 2 * j->L;
    j->rc = or_newton_step(j->L, j->n, j->mon_ptr, j->var_ptr, j->var_idx, j->var_exp, j->coef,
                           j->p1 - j->p0, j->t, j->gamma, j->x + (size_t)j->p0 * w, j->lu_mode,
                           j->max_refine, j->res + j->p0, j->status + j->p0, j->sweeps + j->p0);
    return NULL;
}

int or_newton_threads(int L, int n, const int32_t *mon_ptr, const int32_t *var_ptr,
                      const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                      int npts, double t, const double *gamma, double *x, int lu_mode,
                      int max_refine, double *res_norm, int32_t *status, int32_t *sweeps,
                      int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > npts) nthreads = npts > 0 ? npts : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    newton_job *jobs = (newton_job *)malloc(sizeof(newton_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        newton_job *j = &jobs[k];
        j->L = L; j->n = n;
        j->mon_ptr = mon_ptr; j->var_ptr = var_ptr; j->var_idx = var_idx; j->var_exp = var_exp;
        j->coef = coef; j->gamma = gamma; j->t = t; j->x = x; j->res = res_norm;
        j->status = status; j->sweeps = sweeps; j->lu_mode = lu_mode; j->max_refine = max_refine;
        j->p0 = (int)((long)npts * k / nthreads);
        j->p1 = (int)((long)npts * (k + 1) / nthreads);
        j->rc = 0;
        pthread_create(&th[k], NULL, newton_worker, j);
    }
    int rc = 0;
    for (int k = 0; k < nthreads; k++) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
    }
    free(th);
    free(jobs);
    return rc;
}
