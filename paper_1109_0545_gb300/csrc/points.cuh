// points.cuh -- one lane per evaluation point: every lane of a warp walks the same
// monomial stream (warp-uniform control flow, broadcast table loads) and keeps its own
// point's values.  Used by hc_eval_jac and hc_newton_step.
#pragma once
#include "hc_internal.h"
#include "mp.cuh"

namespace hc {

#define HC_KLOCAL 32  // variables per monomial handled by the point kernels

// Views of the structure-of-arrays buffers of one point p (npts points in all).
template <int L> struct PointView {
    const double *X;   // X[2][L][n][npts]
    const double *PW;  // PW[e-2][2][L][n][npts], e = 2 .. max_exp-1
    size_t xplane;     // n * npts
    int npts, p;
    __device__ __forceinline__ C<L> x(int j) const { return ld_c<L>(X, xplane, (size_t)j * npts + p); }
    // x_j^e for 1 <= e <= max_exp - 1
    __device__ __forceinline__ C<L> pw(int j, int e) const
    {
        if (e == 1) return x(j);
        return ld_c<L>(PW + (size_t)(e - 2) * 2 * L * xplane, xplane, (size_t)j * npts + p);
    }
};

// gamma (1 - t) with 1 - t formed exactly (two-sum) before rounding to L limbs
template <int L> __device__ __forceinline__ C<L> gamma_one_minus_t(double gre, double gim, double t)
{
    double s, e;
    two_sum(1.0, -t, s, e);
    R<L> omt = r_zero<L>();
    omt.v[0] = s;
    if (L > 1) omt.v[1] = e;
    return c_mul_r(c_from<L>(gre, gim), omt);
}

//
// Rows r0..r1-1 of f (and of J) at point p.
//
// Per monomial c x_{i1}^{a1} ... x_{ik}^{ak} (indices and exponents warp-uniform):
//   CF'   = c * prod_{a_j >= 2} x_{ij}^{a_j - 1}        the common factor of Sec. 6 with
//                                                       the coefficient folded in
//   Pre_j = CF' * x_{i1} ... x_{i(j-1)}                 prefix products (k-1 mults)
//   D_k   = Pre_k,  D_j = Pre_j * Suf_j,  Suf_j = x_{i(j+1)} ... x_{ik}
//                                                       (backward sweep, 2k-3 mults)
//   value = Pre_k * x_{ik}
// so D_j = c x^{a - e_j} and value = c x^a: the Speelpenning products omega_j of Sec. 6
// times the common factor and the coefficient, in 3k-3 multiplications in all instead of
// the 3k-6 + k + 1 of the paper plus its k+1 coefficient products.  Then
// Coefficient_Product (Alg. 4.1) reduces to f_i += value, J_{i,ij} += a_j D_j.
// J is accumulated in place in the output buffer (this lane is its only writer).
// Products inside the chain stay unnormalised (c_mul_nn).  f_i and the J row are running
// sums (c_acc, not renormalised in double-double), renormalised once when the row is
// complete (c_settle), so every value stored at the end is normalised.
//
template <int L, bool JAC>
__device__ void eval_rows_point(const DevSys &S, const PointView<L> &V, bool live, double t,
                                const C<L> &gs, double *__restrict__ F, double *__restrict__ J,
                                int r0, int r1)
{
    const int n = S.n, npts = V.npts, p = V.p;
    const size_t fplane = (size_t)S.npoly * npts;
    const size_t jplane = (size_t)S.npoly * n * npts;
    C<L> pre[HC_KLOCAL];
    for (int i = r0; i < r1; i++) {
        C<L> fi = c_zero<L>();
        const size_t jrow = (size_t)i * n * npts + p;
        if (JAC && live)
            for (int j = 0; j < n; j++) st_c<L>(J, jplane, jrow + (size_t)j * npts, c_zero<L>());
        const int m0 = __ldg(S.mon_ptr + i), m1 = __ldg(S.mon_ptr + i + 1);
        for (int m = m0; m < m1; m++) {
            const int q0 = __ldg(S.var_ptr + m), k = __ldg(S.var_ptr + m + 1) - q0;
            C<L> c = ld_c<L>(S.coef + (size_t)m * 2 * L, 1, 0);
            if (k == 0) {
                fi = c_acc(fi, c);
                continue;
            }
            // common factor with the coefficient folded in
            C<L> cf = c;
            for (int j = 0; j < k; j++) {
                const int pk = __ldg(S.var_pack + q0 + j);
                const int e = pk >> 16;
                if (e >= 2) cf = c_mul_nn(cf, V.pw(pk & 0xffff, e - 1));
            }
            if (!JAC) {
                for (int j = 0; j < k; j++) cf = c_mul_nn(cf, V.x(__ldg(S.var_pack + q0 + j) & 0xffff));
                fi = c_acc(fi, cf);
                continue;
            }
            // prefix products
            pre[0] = cf;
            for (int j = 1; j < k; j++) pre[j] = c_mul_nn(pre[j - 1], V.x(__ldg(S.var_pack + q0 + j - 1) & 0xffff));
            const int pk_last = __ldg(S.var_pack + q0 + k - 1);
            const C<L> xl = V.x(pk_last & 0xffff);
            fi = c_acc(fi, c_mul_nn(pre[k - 1], xl));
            // backward sweep: D_j = pre_j * suf_j
            if (live) {
                const size_t o = jrow + (size_t)(pk_last & 0xffff) * npts;
                st_c<L>(J, jplane, o, c_acc(ld_c<L>(J, jplane, o), c_scale_int(pre[k - 1], pk_last >> 16)));
            }
            C<L> suf = xl;
            for (int j = k - 2; j >= 0; j--) {
                const int pk = __ldg(S.var_pack + q0 + j);
                const C<L> d = c_scale_int(c_mul_nn(pre[j], suf), pk >> 16);
                if (live) {
                    const size_t o = jrow + (size_t)(pk & 0xffff) * npts;
                    st_c<L>(J, jplane, o, c_acc(ld_c<L>(J, jplane, o), d));
                }
                if (j > 0) suf = c_mul_nn(suf, V.x(pk & 0xffff));
            }
        }
        fi = c_settle(fi);
        if (t >= 0.0) {
            // homotopy assembly: h_i = gamma (1-t) (x_i^d - 1) + t f_i,
            // dh_i/dx_j = t J_ij + [i == j] gamma (1-t) d x_i^(d-1)
            const int d = __ldg(S.deg + i);
            const C<L> xi = V.x(i);
            const C<L> xd1 = c_pow(xi, d - 1);
            C<L> g = c_mul(xd1, xi);
            g.re = r_sub(g.re, r_from<L>(1.0));
            fi = c_add(c_mul(gs, g), c_mul_d(fi, t));
            if (JAC && live) {
                for (int j = 0; j < n; j++) {
                    const size_t o = jrow + (size_t)j * npts;
                    C<L> v = c_mul_d(c_settle(ld_c<L>(J, jplane, o)), t);
                    if (j == i) v = c_add(v, c_mul(gs, c_scale_int(xd1, d)));
                    st_c<L>(J, jplane, o, v);
                }
            }
        } else if (L == 2 && JAC && live) {
            for (int j = 0; j < n; j++) {
                const size_t o = jrow + (size_t)j * npts;
                st_c<L>(J, jplane, o, c_settle(ld_c<L>(J, jplane, o)));
            }
        }
        if (live) st_c<L>(F, fplane, (size_t)i * npts + p, fi);
    }
}

}  // namespace hc
