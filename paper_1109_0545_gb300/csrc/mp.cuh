// mp.cuh -- complex double / double-double / quad-double arithmetic for sm_103a.
//
// Extended precision from error-free transformations (Dekker 1971; Hida, Li & Bailey
// 2001), the arithmetic the paper's tracker runs in (Sec. 1, Sec. 2).  Built on the FMA:
// the exact error of a product is one fused multiply-add, so no Dekker split is needed.
//
// Every floating-point operation below goes through an explicit round-to-nearest
// intrinsic (__dadd_rn, __dmul_rn, __fma_rn): the compiler may neither contract a
// multiply and an add into one FMA nor reassociate, either of which would silently
// destroy the error terms.
//
// On GB300 the FP64 pipe is the scarce unit (about 1.6 FP64 instructions per clock per
// SM, against ~100 FP32 FMAs), so every routine is written to minimise FP64
// instructions; the comment of each states its count (negations fold into operand
// modifiers and cost nothing).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hc {

__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// s + e = a + b exactly (Knuth).  6 FP64.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = add_(a, b);
    double bb = sub_(s, a);
    e = add_(sub_(a, sub_(s, bb)), sub_(b, bb));
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker).  3 FP64.
__device__ __forceinline__ void fast_two_sum(double a, double b, double &s, double &e)
{
    s = add_(a, b);
    e = sub_(b, sub_(s, a));
}

// s + e = a + b exactly for any a, b: order the operands by exponent, then Dekker's fast
// two-sum (exact whenever the first operand's exponent is not below the second's).  The
// order comes from the high 32 bits of each operand shifted left by one (sign dropped:
// exponent and leading fraction bits) compared as unsigned integers, all on the INT pipe.
// (Clearing the sign bit with a mask instead is compiled as an FP64 absolute value, two
// more FP64 instructions.)  3 FP64.
__device__ __forceinline__ void two_sum_ord(double a, double b, double &s, double &e)
{
    const unsigned ha = (unsigned)__double2hiint(a) << 1;
    const unsigned hb = (unsigned)__double2hiint(b) << 1;
    const bool keep = ha >= hb;
    fast_two_sum(keep ? a : b, keep ? b : a, s, e);
}

// x * 2^k exactly.  Exponent arithmetic on the bit pattern (no FP64 instruction) for
// zero and for normal x whose result stays normal; a multiply otherwise.
__device__ __forceinline__ double ldexp_exact(double x, int k)
{
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (((unsigned long long)b << 1) == 0ULL) return x;
    if (ex > 0 && ex + k > 0 && ex + k < 0x7ff) return __longlong_as_double(b + ((long long)k << 52));
    return mul_(x, __longlong_as_double((long long)(1023 + k) << 52));
}

// p + e = a * b exactly (FMA).  2 FP64.
__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e)
{
    p = mul_(a, b);
    e = fma_(a, b, -p);
}

template <int L> struct R { double v[L]; };
template <int L> struct C { R<L> re, im; };

template <int L> __device__ __forceinline__ R<L> r_zero()
{
    R<L> r;
#pragma unroll
    for (int j = 0; j < L; j++) r.v[j] = 0.0;
    return r;
}
template <int L> __device__ __forceinline__ R<L> r_from(double d)
{
    R<L> r = r_zero<L>();
    r.v[0] = d;
    return r;
}
template <int L> __device__ __forceinline__ R<L> r_neg(R<L> a)
{
#pragma unroll
    for (int j = 0; j < L; j++) a.v[j] = -a.v[j];
    return a;
}

// ---------------------------------------------------------------- renormalisation (QD)
// Five components of roughly decreasing magnitude -> four limbs.  Bottom-up two-sums
// carry the value up exactly (two-sums, not fast-two-sums: after a cancellation the
// components need not be ordered); the top-down fast-two-sums then re-split it.  22 FP64.
__device__ __forceinline__ R<4> renorm5_pass(double c0, double c1, double c2, double c3, double c4)
{
    double s, t3, t2, t1, t0;
    two_sum_ord(c3, c4, s, t3);
    two_sum_ord(c2, s, s, t2);
    two_sum_ord(c1, s, s, t1);
    two_sum_ord(c0, s, c0, t0);
    R<4> r;
    double e;
    fast_two_sum(c0, t0, r.v[0], e);
    fast_two_sum(e, t1, r.v[1], e);
    fast_two_sum(e, t2, r.v[2], e);
    r.v[3] = add_(e, t3);
    return r;
}

// Biased exponent field of x (0 for zero and subnormals), on the INT pipe.
__device__ __forceinline__ int exp_field(double x)
{
    return (int)(((unsigned)__double2hiint(x) << 1) >> 21);
}

// The limbs are nonoverlapping: each nonzero limb has an exponent at least 53 below the
// one above it (so it is below a unit in the last place of that limb), and the leading
// limb is the value to within a unit in its last place.  Integer comparisons only.
__device__ __forceinline__ bool qd_separated(const R<4> &r)
{
    const int e0 = exp_field(r.v[0]), e1 = exp_field(r.v[1]), e2 = exp_field(r.v[2]), e3 = exp_field(r.v[3]);
    return !((e1 && e1 + 53 > e0) || (e2 && e2 + 53 > e1) || (e3 && e3 + 53 > e2));
}

// Renormalisation.  When the components cancel at the top (say c0 + the sum of the rest
// is zero or a few units in its last place, as in the difference of two nearly equal
// values), one pass leaves the value in the lower limbs: the leading limb is zero or
// much smaller than the next one, although the sum of the limbs is exact.  Code that
// reads only the leading limb (norms, pivots, the right-hand side of an FP64
// refinement solve) would then see the wrong value, so such a result takes a second
// pass, whose input no longer cancels.  22 FP64 (44 in the rare second pass).
__device__ __forceinline__ R<4> renorm5(double c0, double c1, double c2, double c3, double c4)
{
    R<4> r = renorm5_pass(c0, c1, c2, c3, c4);
    if (!qd_separated(r)) r = renorm5_pass(r.v[0], r.v[1], r.v[2], r.v[3], 0.0);
    return r;
}

// ---------------------------------------------------------------- addition
__device__ __forceinline__ R<1> r_add(R<1> a, R<1> b)  // 1 FP64
{
    R<1> r;
    r.v[0] = add_(a.v[0], b.v[0]);
    return r;
}
// double-double: two-sum of the leading limbs, lower limbs added into the error.  8 FP64.
// Accepts an unnormalised operand (lower limb up to a few units in the last place of
// the leading one); the result is normalised.
__device__ __forceinline__ R<2> r_add(R<2> a, R<2> b)
{
    double s, e;
    two_sum_ord(a.v[0], b.v[0], s, e);
    e = add_(e, add_(a.v[1], b.v[1]));
    R<2> r;
    fast_two_sum(s, e, r.v[0], r.v[1]);
    return r;
}
// quad-double: limb-wise two-sums, errors cascaded one order down, renormalised.  47 FP64.
__device__ __forceinline__ R<4> r_add(R<4> a, R<4> b)
{
    double s0, s1, s2, s3, t0, t1, t2, t3, u, w;
    two_sum_ord(a.v[0], b.v[0], s0, t0);
    two_sum_ord(a.v[1], b.v[1], s1, t1);
    two_sum_ord(a.v[2], b.v[2], s2, t2);
    two_sum_ord(a.v[3], b.v[3], s3, t3);
    two_sum_ord(s1, t0, s1, t0);           // order 1 -> s1, order-2 error t0
    two_sum_ord(s2, t1, s2, u);            // order 2: s2 + t1 + t0
    two_sum_ord(s2, t0, s2, w);
    double c3 = add_(add_(add_(s3, t2), add_(u, w)), t3);  // order 3
    return renorm5(s0, s1, s2, c3, 0.0);
}

template <int L> __device__ __forceinline__ R<L> r_sub(R<L> a, R<L> b) { return r_add(a, r_neg(b)); }

// Running sums (sums read back only at their end).  Double-double: the leading limbs are
// added by a two-sum, and its error and the lower limbs gather in the lower limb, which
// is not renormalised: 5 FP64 instead of 8.  The lower limb may then grow past a unit in
// the last place of the leading limb (after cancellation, past the leading limb itself);
// r_settle renormalises the pair once, at the end (3 FP64).  Every two-sum is exact, so
// the error of m terms is that of m rounded additions of lower limbs, a small multiple of
// m 2^-106 of the largest partial sum.  Double and quad double accumulate with the
// normalised addition.
template <int L> __device__ __forceinline__ R<L> r_acc(R<L> a, R<L> b) { return r_add(a, b); }
template <> __device__ __forceinline__ R<2> r_acc<2>(R<2> a, R<2> b)
{
    double s, e;
    two_sum_ord(a.v[0], b.v[0], s, e);
    R<2> r;
    r.v[0] = s;
    r.v[1] = add_(a.v[1], add_(b.v[1], e));
    return r;
}
template <int L> __device__ __forceinline__ R<L> r_settle(R<L> a) { return a; }
template <> __device__ __forceinline__ R<2> r_settle<2>(R<2> a)
{
    R<2> r;
    two_sum_ord(a.v[0], a.v[1], r.v[0], r.v[1]);
    return r;
}

// ---------------------------------------------------------------- multiplication
__device__ __forceinline__ R<1> r_mul(R<1> a, R<1> b)  // 1 FP64
{
    R<1> r;
    r.v[0] = mul_(a.v[0], b.v[0]);
    return r;
}
// double-double: exact leading product plus the two cross terms.  7 FP64.
__device__ __forceinline__ R<2> r_mul(R<2> a, R<2> b)
{
    double p, e;
    two_prod(a.v[0], b.v[0], p, e);
    e = fma_(a.v[0], b.v[1], e);
    e = fma_(a.v[1], b.v[0], e);
    R<2> r;
    fast_two_sum(p, e, r.v[0], r.v[1]);
    return r;
}
// quad-double: products of order 0..2 exact, order 3 rounded, order 4 dropped; each
// order summed with two-sums whose errors fall into the next order.  71 FP64.
__device__ __forceinline__ R<4> r_mul(R<4> a, R<4> b)
{
    double p00, e00, p01, e01, p10, e10, p02, e02, p11, e11, p20, e20;
    two_prod(a.v[0], b.v[0], p00, e00);
    two_prod(a.v[0], b.v[1], p01, e01);
    two_prod(a.v[1], b.v[0], p10, e10);
    two_prod(a.v[0], b.v[2], p02, e02);
    two_prod(a.v[1], b.v[1], p11, e11);
    two_prod(a.v[2], b.v[0], p20, e20);
    double c1, u1, u2, s;
    two_sum_ord(p01, p10, s, u1);
    two_sum_ord(s, e00, c1, u2);                       // order 1
    double c2, v1, v2, v3, v4, v5, v6;
    two_sum_ord(p02, p11, s, v1);
    two_sum_ord(s, p20, s, v2);
    two_sum_ord(s, e01, s, v3);
    two_sum_ord(s, e10, s, v4);
    two_sum_ord(s, u1, s, v5);
    two_sum_ord(s, u2, c2, v6);                        // order 2
    double c3 = fma_(a.v[0], b.v[3], fma_(a.v[1], b.v[2], fma_(a.v[2], b.v[1], mul_(a.v[3], b.v[0]))));
    c3 = add_(c3, add_(add_(e02, e11), e20));
    c3 = add_(c3, add_(add_(add_(v1, v2), add_(v3, v4)), add_(v5, v6)));  // order 3
    return renorm5(p00, c1, c2, c3, 0.0);
}

// times a double.  DD: 6 FP64.
__device__ __forceinline__ R<1> r_mul_d(R<1> a, double d) { R<1> r; r.v[0] = mul_(a.v[0], d); return r; }
__device__ __forceinline__ R<2> r_mul_d(R<2> a, double d)
{
    double p, e;
    two_prod(a.v[0], d, p, e);
    e = fma_(a.v[1], d, e);
    R<2> r;
    fast_two_sum(p, e, r.v[0], r.v[1]);
    return r;
}
__device__ __forceinline__ R<4> r_mul_d(R<4> a, double d)
{
    double p0, e0, p1, e1, p2, e2;
    two_prod(a.v[0], d, p0, e0);
    two_prod(a.v[1], d, p1, e1);
    two_prod(a.v[2], d, p2, e2);
    double c1, u;
    two_sum_ord(p1, e0, c1, u);
    double c2, w1, w2;
    two_sum_ord(p2, e1, c2, w1);
    two_sum_ord(c2, u, c2, w2);
    double c3 = fma_(a.v[3], d, add_(add_(e2, w1), w2));
    return renorm5(p0, c1, c2, c3, 0.0);
}

// ---------------------------------------------------------------- division
// Long division: quotient digits q_j = r_lead / b_lead, remainder r -= q_j b exactly
// to working precision, then the digits renormalised.
__device__ __forceinline__ R<1> r_div(R<1> a, R<1> b) { R<1> r; r.v[0] = __ddiv_rn(a.v[0], b.v[0]); return r; }
__device__ __forceinline__ R<2> r_div(R<2> a, R<2> b)
{
    double q1 = __ddiv_rn(a.v[0], b.v[0]);
    R<2> r = r_sub(a, r_mul_d(b, q1));
    double q2 = __ddiv_rn(r.v[0], b.v[0]);
    r = r_sub(r, r_mul_d(b, q2));
    double q3 = __ddiv_rn(r.v[0], b.v[0]);
    double s, e;
    fast_two_sum(q1, q2, s, e);
    e = add_(e, q3);
    R<2> out;
    fast_two_sum(s, e, out.v[0], out.v[1]);
    return out;
}
__device__ __forceinline__ R<4> r_div(R<4> a, R<4> b)
{
    double q[5];
    R<4> r = a;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        q[j] = __ddiv_rn(r.v[0], b.v[0]);
        if (j < 4) r = r_sub(r, r_mul_d(b, q[j]));
    }
    return renorm5(q[0], q[1], q[2], q[3], q[4]);
}

// ---------------------------------------------------------------- small integers
// the double of an integer 1 <= k < 2^52 built from its bits (no FP64 conversion
// instruction): exponent from the leading bit, the bits below it as the fraction
__device__ __forceinline__ double int_to_double_exact(int k)
{
    const int e = 31 - __clz(k);
    const unsigned long long frac = ((unsigned long long)k << (52 - e)) & 0xfffffffffffffULL;
    return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | frac));
}

// a * k for a small positive integer k: exact for powers of two (exponent arithmetic,
// no FP64 instruction), r_mul_d otherwise.
template <int L> __device__ __forceinline__ R<L> r_scale_int(R<L> a, int k)
{
    if (k == 1) return a;
    if ((k & (k - 1)) == 0) {
        const int e = __ffs(k) - 1;
#pragma unroll
        for (int j = 0; j < L; j++) a.v[j] = ldexp_exact(a.v[j], e);
        return a;
    }
    return r_mul_d(a, int_to_double_exact(k));
}

// ---------------------------------------------------------------- complex
template <int L> __device__ __forceinline__ C<L> c_zero() { C<L> z; z.re = r_zero<L>(); z.im = r_zero<L>(); return z; }
template <int L> __device__ __forceinline__ C<L> c_from(double re, double im)
{
    C<L> z;
    z.re = r_from<L>(re);
    z.im = r_from<L>(im);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_add(C<L> a, C<L> b)
{
    C<L> z;
    z.re = r_add(a.re, b.re);
    z.im = r_add(a.im, b.im);
    return z;
}
// running sums (r_acc): 10 FP64 in DD; c_settle renormalises at the end (6 FP64 in DD)
template <int L> __device__ __forceinline__ C<L> c_acc(C<L> a, C<L> b)
{
    C<L> z;
    z.re = r_acc<L>(a.re, b.re);
    z.im = r_acc<L>(a.im, b.im);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_settle(C<L> a)
{
    C<L> z;
    z.re = r_settle<L>(a.re);
    z.im = r_settle<L>(a.im);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_sub(C<L> a, C<L> b)
{
    C<L> z;
    z.re = r_sub(a.re, b.re);
    z.im = r_sub(a.im, b.im);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_mul_d(C<L> a, double d)
{
    C<L> z;
    z.re = r_mul_d(a.re, d);
    z.im = r_mul_d(a.im, d);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_mul_r(C<L> a, R<L> s)
{
    C<L> z;
    z.re = r_mul(a.re, s);
    z.im = r_mul(a.im, s);
    return z;
}
template <int L> __device__ __forceinline__ C<L> c_scale_int(C<L> a, int k)
{
    C<L> z;
    z.re = r_scale_int(a.re, k);
    z.im = r_scale_int(a.im, k);
    return z;
}

// generic complex product: four real products, two sums
template <int L> __device__ __forceinline__ C<L> c_mul(C<L> a, C<L> b)
{
    C<L> z;
    z.re = r_sub(r_mul(a.re, b.re), r_mul(a.im, b.im));
    z.im = r_add(r_mul(a.re, b.im), r_mul(a.im, b.re));
    return z;
}
// complex double: 4 FP64
template <> __device__ __forceinline__ C<1> c_mul<1>(C<1> a, C<1> b)
{
    C<1> z;
    z.re.v[0] = fma_(a.re.v[0], b.re.v[0], -mul_(a.im.v[0], b.im.v[0]));
    z.im.v[0] = fma_(a.re.v[0], b.im.v[0], mul_(a.im.v[0], b.re.v[0]));
    return z;
}
// complex double-double, each part as ONE fused dot product of two DD products:
// exact leading products, their sum by an ordered two-sum, all order-1 terms (product
// errors and the four cross terms) accumulated into the error by FMAs, one
// renormalising fast-two-sum.  16 FP64 per part, 32 in all (50 for 4 mul + 2 add).
// Without the final renormalisation (NORM = false) the pair (s, e) is returned as is:
// 13 per part, 26 in all.  Such an unnormalised value may only feed another product or an
// addition (both renormalise): its lower limb is a few ulps of its leading limb, or after
// cancellation a few ulps of the products' magnitude, so the normwise error stays at
// 2^-106 of the terms' magnitude.
template <bool NORM>
__device__ __forceinline__ void dd_dot2(double a0, double a1, double b0, double b1,
                                        double c0, double c1, double d0, double d1,
                                        double &hi, double &lo)
{
    // a*b + c*d
    double p, q, ep, eq, s, e;
    two_prod(a0, b0, p, ep);
    two_prod(c0, d0, q, eq);
    two_sum_ord(p, q, s, e);
    e = add_(e, add_(ep, eq));
    e = fma_(a0, b1, e);
    e = fma_(a1, b0, e);
    e = fma_(c0, d1, e);
    e = fma_(c1, d0, e);
    if (NORM) {
        fast_two_sum(s, e, hi, lo);
    } else {
        hi = s;
        lo = e;
    }
}
template <> __device__ __forceinline__ C<2> c_mul<2>(C<2> a, C<2> b)
{
    C<2> z;
    dd_dot2<true>(a.re.v[0], a.re.v[1], b.re.v[0], b.re.v[1],
                  -a.im.v[0], -a.im.v[1], b.im.v[0], b.im.v[1], z.re.v[0], z.re.v[1]);
    dd_dot2<true>(a.re.v[0], a.re.v[1], b.im.v[0], b.im.v[1],
                  a.im.v[0], a.im.v[1], b.re.v[0], b.re.v[1], z.im.v[0], z.im.v[1]);
    return z;
}

// Product whose result only feeds another product or an addition: unnormalised in DD
// (26 FP64), the plain product otherwise.
template <int L> __device__ __forceinline__ C<L> c_mul_nn(C<L> a, C<L> b) { return c_mul(a, b); }
template <> __device__ __forceinline__ C<2> c_mul_nn<2>(C<2> a, C<2> b)
{
    C<2> z;
    dd_dot2<false>(a.re.v[0], a.re.v[1], b.re.v[0], b.re.v[1],
                   -a.im.v[0], -a.im.v[1], b.im.v[0], b.im.v[1], z.re.v[0], z.re.v[1]);
    dd_dot2<false>(a.re.v[0], a.re.v[1], b.im.v[0], b.im.v[1],
                   a.im.v[0], a.im.v[1], b.re.v[0], b.re.v[1], z.im.v[0], z.im.v[1]);
    return z;
}

// acc - l * b (the elimination update of Sec. 4); generic: product then subtraction.
template <int L> __device__ __forceinline__ C<L> c_fnma(C<L> acc, C<L> l, C<L> b)
{
    return c_sub(acc, c_mul(l, b));
}
// DD: each part as one fused three-term sum a - (l.re b.re - l.im b.im) etc.  21 FP64
// per part, 42 in all (48 for a product and a subtraction).
__device__ __forceinline__ void dd_fnma_part(double a0, double a1, double x0, double x1, double y0,
                                             double y1, double u0, double u1, double v0, double v1,
                                             double &hi, double &lo)
{
    // a - x*y + u*v
    double p, q, ep, eq, s, t, e1, e2;
    two_prod(x0, y0, p, ep);
    two_prod(u0, v0, q, eq);
    two_sum_ord(a0, -p, s, e1);
    two_sum_ord(s, q, t, e2);
    double e = add_(add_(e1, e2), add_(a1, sub_(eq, ep)));
    e = fma_(-x0, y1, e);
    e = fma_(-x1, y0, e);
    e = fma_(u0, v1, e);
    e = fma_(u1, v0, e);
    fast_two_sum(t, e, hi, lo);
}
template <> __device__ __forceinline__ C<2> c_fnma<2>(C<2> acc, C<2> l, C<2> b)
{
    C<2> z;
    // re: acc.re - l.re b.re + l.im b.im ; im: acc.im - l.re b.im - l.im b.re
    dd_fnma_part(acc.re.v[0], acc.re.v[1], l.re.v[0], l.re.v[1], b.re.v[0], b.re.v[1],
                 l.im.v[0], l.im.v[1], b.im.v[0], b.im.v[1], z.re.v[0], z.re.v[1]);
    dd_fnma_part(acc.im.v[0], acc.im.v[1], l.re.v[0], l.re.v[1], b.im.v[0], b.im.v[1],
                 -l.im.v[0], -l.im.v[1], b.re.v[0], b.re.v[1], z.im.v[0], z.im.v[1]);
    return z;
}

// quad-double a*b + c*d as one sum: products of order 0..2 exact (two-products), order 3
// rounded, order 4 dropped; each order summed by ordered two-sums whose errors fall into
// the next order; one renormalisation.  141 FP64 (4 products and 2 sums: 378 for the
// complex product's two parts together, 282 this way).
__device__ __forceinline__ R<4> qd_dot2(const R<4> &a, const R<4> &b, const R<4> &c, const R<4> &d)
{
    double p0, e0, q0, f0, s0, u;
    two_prod(a.v[0], b.v[0], p0, e0);
    two_prod(c.v[0], d.v[0], q0, f0);
    two_sum_ord(p0, q0, s0, u);
    // order 1
    double p01, e01, p10, e10, q01, f01, q10, f10;
    two_prod(a.v[0], b.v[1], p01, e01);
    two_prod(a.v[1], b.v[0], p10, e10);
    two_prod(c.v[0], d.v[1], q01, f01);
    two_prod(c.v[1], d.v[0], q10, f10);
    double s1 = u, g1, g2, g3, g4, g5, g6;
    two_sum_ord(s1, e0, s1, g1);
    two_sum_ord(s1, f0, s1, g2);
    two_sum_ord(s1, p01, s1, g3);
    two_sum_ord(s1, p10, s1, g4);
    two_sum_ord(s1, q01, s1, g5);
    two_sum_ord(s1, q10, s1, g6);
    // order 2
    double p02, e02, p11, e11, p20, e20, q02, f02, q11, f11, q20, f20;
    two_prod(a.v[0], b.v[2], p02, e02);
    two_prod(a.v[1], b.v[1], p11, e11);
    two_prod(a.v[2], b.v[0], p20, e20);
    two_prod(c.v[0], d.v[2], q02, f02);
    two_prod(c.v[1], d.v[1], q11, f11);
    two_prod(c.v[2], d.v[0], q20, f20);
    const double o2[15] = {g2, g3, g4, g5, g6, e01, e10, f01, f10, p02, p11, p20, q02, q11, q20};
    double s2 = g1, h = 0.0;
#pragma unroll
    for (int i = 0; i < 15; i++) {
        double r;
        two_sum_ord(s2, o2[i], s2, r);
        h = add_(h, r);
    }
    // order 3
    double s3 = fma_(a.v[0], b.v[3], fma_(a.v[1], b.v[2], fma_(a.v[2], b.v[1], mul_(a.v[3], b.v[0]))));
    s3 = fma_(c.v[0], d.v[3], fma_(c.v[1], d.v[2], fma_(c.v[2], d.v[1], fma_(c.v[3], d.v[0], s3))));
    s3 = add_(s3, add_(add_(add_(e02, e11), add_(e20, f02)), add_(f11, f20)));
    s3 = add_(s3, h);
    return renorm5(s0, s1, s2, s3, 0.0);
}

template <> __device__ __forceinline__ C<4> c_mul<4>(C<4> a, C<4> b)
{
    C<4> z;
    z.re = qd_dot2(a.re, b.re, r_neg(a.im), b.im);
    z.im = qd_dot2(a.re, b.im, a.im, b.re);
    return z;
}

// 1 / b = conj(b) / |b|^2
template <int L> __device__ __forceinline__ C<L> c_inv(C<L> b)
{
    R<L> den = r_add(r_mul(b.re, b.re), r_mul(b.im, b.im));
    C<L> z;
    z.re = r_div(b.re, den);
    z.im = r_neg(r_div(b.im, den));
    return z;
}

// |z|^2 of the leading limbs in plain double (pivot and norm measure): 3 FP64.
template <int L> __device__ __forceinline__ double c_abs2_lead(const C<L> &z)
{
    return add_(mul_(z.re.v[0], z.re.v[0]), mul_(z.im.v[0], z.im.v[0]));
}

// z^e by binary powering, z^0 = 1
template <int L> __device__ __forceinline__ C<L> c_pow(C<L> z, int e)
{
    C<L> r = c_from<L>(1.0, 0.0);
    bool first = true;
    while (e > 0) {
        if (e & 1) {
            r = first ? z : c_mul(r, z);
            first = false;
        }
        e >>= 1;
        if (e) z = c_mul(z, z);
    }
    return r;
}

// ---------------------------------------------------------------- structure-of-arrays I/O
// A complex L-limb array stored as [2][L][...] with plane stride `plane` doubles:
// part c (0 re, 1 im), limb l lives at base[(c * L + l) * plane + off].
template <int L> __device__ __forceinline__ C<L> ld_c(const double *__restrict__ base, size_t plane, size_t off)
{
    C<L> z;
#pragma unroll
    for (int l = 0; l < L; l++) {
        z.re.v[l] = base[(size_t)l * plane + off];
        z.im.v[l] = base[(size_t)(L + l) * plane + off];
    }
    return z;
}
template <int L> __device__ __forceinline__ void st_c(double *__restrict__ base, size_t plane, size_t off, const C<L> &z)
{
#pragma unroll
    for (int l = 0; l < L; l++) {
        base[(size_t)l * plane + off] = z.re.v[l];
        base[(size_t)(L + l) * plane + off] = z.im.v[l];
    }
}
// leading limbs only
template <int L> __device__ __forceinline__ void ld_lead(const double *__restrict__ base, size_t plane, size_t off,
                                                         double &re, double &im)
{
    re = base[off];
    im = base[(size_t)L * plane + off];
}

template <int L> __device__ __forceinline__ bool c_finite_lead(const C<L> &z)
{
    return isfinite(z.re.v[0]) && isfinite(z.im.v[0]);
}

}  // namespace hc
