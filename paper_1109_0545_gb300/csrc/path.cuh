// path.cuh -- one thread block per path: evaluation of h and its Jacobian at one point of
// the path's own system, and the Newton corrector of Alg. 4.1 on it, block-cooperative.
// Used by the path tracker (hc_track.cu).
#pragma once
#include "points.cuh"

namespace hc {

#define HC_TB 128          // threads per block of the whole-GPU engine's kernels; the block
                           // engine's default (its block size is the template parameter TB)
#define HC_TWMAX 32        // warps of the largest block using the block reductions (1024)

// per-slot scratch of one block (global memory sized for the largest system; the solve's
// vectors, and the FP64 factors where they fit, in shared memory)
template <int L> struct Slot {
    double *PW;    // [max_exp-2][2][L][n]
    double *V;     // [2][L][nvar+nmon] (plane = nvar+nmon): partials, then values
    double *HS;    // [2][L][3n] start-system terms of the homotopy per row: gamma (1-t)
                   // (x_i^d_i - 1), gamma (1-t) d_i x_i^(d_i - 1), gamma (x_i^d_i - 1)
    double *HT;    // [2][n] leading limbs of dh/dt = f - gamma g, or NULL (not needed)
    double *H;     // [2][L][n]
    double *JH;    // [2][L][n][n]
    double *B;     // [2][n][n] FP64 factors
    double *RV;    // [2][n] right-hand side of an FP64 solve
    double *Y;     // [2][n] solution of an FP64 solve
    double *DZ;    // [2][L][n]
    double *ZP;    // [2][L][n] the predicted point of the current stage
    int32_t *PIV;  // [n] row permutation of the factors
};

struct BlockShared {
    double rv[HC_TWMAX];
    double rv2[HC_TWMAX];
    long long rk[HC_TWMAX];
    int ri[HC_TWMAX];
    double pre[HC_TWMAX];  // the pivot candidates' values (block_argmax_piv)
    double pim[HC_TWMAX];
    double bc[4];
    int ibc[4];
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The last step of a block reduction: after the barrier that published each warp's value
// in sh (rv[w], and ri[w] for an argmax), every warp loads the TB / 32 values into its
// lanes and reduces them with log2(TB / 32) shuffles, then lane 0's result is broadcast.
// Looping over the warps instead would cost every thread one FP64 comparison (FP64 pipe)
// per warp: with 32 warps, more than the work a column of the LU reduces.
template <int TB> __device__ __forceinline__ double merge_max(const double *rv)
{
    constexpr int NW = TB / 32;
    if (NW == 1) return rv[0];
    const int lane = threadIdx.x & 31;
    double m = lane < NW ? rv[lane] : -INFINITY;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    return __shfl_sync(0xffffffffu, m, 0);
}

// Pivot searches compare squared moduli, which are nonnegative: the bit pattern of a
// nonnegative double orders like its value, so the searches compare 64-bit integer keys
// (INT pipe) instead of doubles (FP64 pipe; a block-wide argmax per column of an LU would
// otherwise issue more FP64 comparisons than the column's elimination issues FMAs).
// "No candidate" is key -1; a NaN modulus becomes the largest key.
__device__ __forceinline__ long long amax_key(double v)
{
    const long long b = __double_as_longlong(v);
    return b < 0 ? -1LL : b;
}
__device__ __forceinline__ double amax_value(long long k) { return k < 0 ? -1.0 : __longlong_as_double(k); }

// (k, i) against (k2, i2): larger key, ties to the lower index
__device__ __forceinline__ void amax_take(long long &k, int &i, long long k2, int i2)
{
    if (k2 > k || (k2 == k && i2 < i)) {
        k = k2;
        i = i2;
    }
}

__device__ __forceinline__ void warp_argmax_key(long long &k, int &i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        amax_take(k, i, k2, i2);
    }
}

// argmax of the published (rk[w], ri[w]), ties to the lowest index
template <int TB> __device__ __forceinline__ void merge_argmax_key(const long long *rk, const int *ri, long long &k, int &i)
{
    constexpr int NW = TB / 32;
    if (NW == 1) {
        k = rk[0];
        i = ri[0];
        return;
    }
    const int lane = threadIdx.x & 31;
    k = lane < NW ? rk[lane] : -1LL;
    i = lane < NW ? ri[lane] : 0x7fffffff;
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        amax_take(k, i, k2, i2);
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    i = __shfl_sync(0xffffffffu, i, 0);
}

// A pivot candidate: integer key, row, and the FP64 value itself, which travels with the
// winner, so that the elimination step takes the pivot from registers instead of reading
// the matrix entry that the same step overwrites with a multiplier
struct Piv {
    long long k;
    int i;
    double re, im;
};
__device__ __forceinline__ Piv piv_none() { return Piv{-1LL, 0x7fffffff, 0.0, 0.0}; }
__device__ __forceinline__ void piv_take(Piv &p, long long k2, int i2, double re2, double im2)
{
    if (k2 > p.k || (k2 == p.k && i2 < p.i)) p = Piv{k2, i2, re2, im2};
}
__device__ __forceinline__ void warp_argmax_piv(Piv &p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, p.k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, p.i, o);
        const double re2 = __shfl_xor_sync(0xffffffffu, p.re, o);
        const double im2 = __shfl_xor_sync(0xffffffffu, p.im, o);
        piv_take(p, k2, i2, re2, im2);
    }
}
// the warps' candidates published by warp_argmax_piv + piv_publish, merged after a barrier
__device__ __forceinline__ void piv_publish(const Piv &p, BlockShared &sh)
{
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        sh.rk[w] = p.k;
        sh.ri[w] = p.i;
        sh.pre[w] = p.re;
        sh.pim[w] = p.im;
    }
}
template <int TB> __device__ __forceinline__ Piv piv_merge(const BlockShared &sh)
{
    constexpr int NW = TB / 32;
    if (NW == 1) return Piv{sh.rk[0], sh.ri[0], sh.pre[0], sh.pim[0]};
    const int lane = threadIdx.x & 31;
    Piv p = lane < NW ? Piv{sh.rk[lane], sh.ri[lane], sh.pre[lane], sh.pim[lane]} : piv_none();
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, p.k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, p.i, o);
        const double re2 = __shfl_xor_sync(0xffffffffu, p.re, o);
        const double im2 = __shfl_xor_sync(0xffffffffu, p.im, o);
        piv_take(p, k2, i2, re2, im2);
    }
    p.k = __shfl_sync(0xffffffffu, p.k, 0);
    p.i = __shfl_sync(0xffffffffu, p.i, 0);
    p.re = __shfl_sync(0xffffffffu, p.re, 0);
    p.im = __shfl_sync(0xffffffffu, p.im, 0);
    return p;
}
template <int TB> __device__ __forceinline__ Piv block_argmax_piv(Piv p, BlockShared &sh)
{
    warp_argmax_piv(p);
    __syncthreads();
    piv_publish(p, sh);
    __syncthreads();
    return piv_merge<TB>(sh);
}

// max over the block of TB threads; every thread gets the same value
template <int TB> __device__ __forceinline__ double block_max(double v, BlockShared &sh)
{
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.rv[threadIdx.x >> 5] = v;
    __syncthreads();
    return merge_max<TB>(sh.rv);
}

// two maxima over the block with one pair of barriers
template <int TB> __device__ __forceinline__ void block_max2(double &a, double &b, BlockShared &sh)
{
    a = warp_max(a);
    b = warp_max(b);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh.rv[threadIdx.x >> 5] = a;
        sh.rv2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    a = merge_max<TB>(sh.rv);
    b = merge_max<TB>(sh.rv2);
}

__device__ __forceinline__ int block_and(int v, BlockShared &sh)
{
    return __syncthreads_and(v);
}

// argmax of the keys (k, i) over the block, ties to the lowest i; every thread gets the
// winner
template <int TB> __device__ __forceinline__ void block_argmax_key(long long &k, int &i, BlockShared &sh)
{
    warp_argmax_key(k, i);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sh.rk[threadIdx.x >> 5] = k;
        sh.ri[threadIdx.x >> 5] = i;
    }
    __syncthreads();
    merge_argmax_key<TB>(sh.rk, sh.ri, k, i);
}

// ------------------------------------------------------------------------------ evaluation
//
// h(z, t) (t >= 0) or f(z) (t < 0) and the Jacobian at one point z[2][L][n], into
// w.H[2][L][n] and w.JH[2][L][n][n].  Two phases:
//   1. monomial-parallel, over the monomials in shape order (so a warp's monomials have
//      equal length): the common factor with the coefficient folded in, prefix products
//      and the backward sweep of points.cuh give each monomial's value c x^a and its
//      scaled partials a_j c x^(a - e_j), stored in V;
//   2. entry-parallel: each thread owns entries (i, j) and adds their contributions in
//      the original monomial order (transpose table), then assembles the homotopy.
//
// Phase 1 for one monomial m: its value c x^a (slot nvar + m of V) and its scaled
// partials a_j c x^(a - e_j) (slots var_ptr[m] + j), by the common factor with the
// coefficient folded in, prefix products and a backward sweep (as in points.cuh).
template <int L>
__device__ __forceinline__ void monomial_to_V(const DevSys &S, int m, const double *__restrict__ z,
                                              const double *__restrict__ PW, double *__restrict__ V)
{
    const int n = S.n;
    const size_t vplane = (size_t)S.nvar + S.nmon;
    auto X = [&](int j) { return ld_c<L>(z, n, j); };
    auto P = [&](int j, int e) { return e == 1 ? X(j) : ld_c<L>(PW + (size_t)(e - 2) * 2 * L * n, n, j); };
    const int q0 = __ldg(S.var_ptr + m), k = __ldg(S.var_ptr + m + 1) - q0;
    const C<L> c = ld_c<L>(S.coef + (size_t)m * 2 * L, 1, 0);
    if (k == 0) {
        st_c<L>(V, vplane, (size_t)S.nvar + m, c);
        return;
    }
    C<L> pre[HC_KLOCAL];
    C<L> cf = c;
    for (int j = 0; j < k; j++) {
        const int pk = __ldg(S.var_pack + q0 + j);
        if ((pk >> 16) >= 2) cf = c_mul_nn(cf, P(pk & 0xffff, (pk >> 16) - 1));
    }
    pre[0] = cf;
    for (int j = 1; j < k; j++) pre[j] = c_mul_nn(pre[j - 1], X(__ldg(S.var_pack + q0 + j - 1) & 0xffff));
    const int pkl = __ldg(S.var_pack + q0 + k - 1);
    const C<L> xl = X(pkl & 0xffff);
    st_c<L>(V, vplane, (size_t)S.nvar + m, c_mul_nn(pre[k - 1], xl));
    st_c<L>(V, vplane, (size_t)q0 + k - 1, c_scale_int(pre[k - 1], pkl >> 16));
    C<L> suf = xl;
    for (int j = k - 2; j >= 0; j--) {
        const int pk = __ldg(S.var_pack + q0 + j);
        st_c<L>(V, vplane, (size_t)q0 + j, c_scale_int(c_mul_nn(pre[j], suf), pk >> 16));
        if (j > 0) suf = c_mul_nn(suf, X(pk & 0xffff));
    }
}

// power table of the point z: PW[e-2] = z^e, e = 2 .. max_exp-1, for variable j
template <int L>
__device__ __forceinline__ void powers_of(const DevSys &S, int j, const double *__restrict__ z, double *__restrict__ PW)
{
    const int n = S.n;
    const C<L> x = ld_c<L>(z, n, j);
    C<L> v = x;
    for (int e = 2; e < S.max_exp; e++) {
        v = c_mul(v, x);
        st_c<L>(PW + (size_t)(e - 2) * 2 * L * n, n, j, v);
    }
}

// Start-system terms of row i of the homotopy at (z, t), t >= 0: gamma (1-t) (x_i^d - 1)
// into HS[i], gamma (1-t) d x_i^(d-1) into HS[n + i] (d = deg f_i), gs = gamma (1-t); with
// tangent, also gamma (x_i^d - 1) into HS[2n + i] (for dh/dt).
template <int L>
__device__ __forceinline__ void homotopy_terms(const DevSys &S, int i, const double *__restrict__ z,
                                               const C<L> &gs, double *__restrict__ HS, bool tangent)
{
    const int n = S.n, d = __ldg(S.deg + i);
    const C<L> xi = ld_c<L>(z, n, i);
    const C<L> xd1 = c_pow(xi, d - 1);
    C<L> g = c_mul(xd1, xi);
    g.re = r_sub(g.re, r_from<L>(1.0));
    st_c<L>(HS, 3 * n, i, c_mul(gs, g));
    st_c<L>(HS, 3 * n, n + i, c_mul(gs, c_scale_int(xd1, d)));
    if (tangent) st_c<L>(HS, 3 * n, 2 * n + i, c_mul(c_from<L>(S.gre, S.gim), g));
}

// The homotopy (t >= 0) on the sum acc of entry e = i (n+1) + j, and its store: j == n is
// h_i (and, with HT, dh_i/dt), else dh_i/dx_j.
template <int L>
__device__ __forceinline__ void entry_finish(const DevSys &S, int e, double t, C<L> acc, const double *__restrict__ HS,
                                             double *__restrict__ H, double *__restrict__ JH, double *__restrict__ HT)
{
    const int n = S.n;
    const int i = e / (n + 1), j = e - i * (n + 1);
    if (t >= 0.0) {
        if (j == n) {
            if (HT) {
                // dh_i/dt = f_i - gamma g_i, leading limbs
                const C<L> dt = c_sub(acc, ld_c<L>(HS, 3 * n, 2 * n + i));
                HT[i] = dt.re.v[0];
                HT[n + i] = dt.im.v[0];
            }
            acc = c_add(ld_c<L>(HS, 3 * n, i), c_mul_d(acc, t));
        } else {
            acc = c_mul_d(acc, t);
            if (i == j) acc = c_add(acc, ld_c<L>(HS, 3 * n, n + i));
        }
    }
    if (j == n)
        st_c<L>(H, n, i, acc);
    else
        st_c<L>(JH, (size_t)n * n, (size_t)i * n + j, acc);
}

// The contributions r0 .. r1-1 of the transpose table summed in order (a running sum,
// renormalised at the end)
template <int L>
__device__ __forceinline__ C<L> sum_contributions(const DevSys &S, int r0, int r1, const double *__restrict__ V)
{
    const size_t vplane = (size_t)S.nvar + S.nmon;
    C<L> acc = c_zero<L>();
    // unrolled so that the gathers of several contributions are in flight together; the
    // additions keep their order
#pragma unroll 4
    for (int r = r0; r < r1; r++) acc = c_acc(acc, ld_c<L>(V, vplane, __ldg(S.tlist + r)));
    return c_settle(acc);
}

// Phase 2 for one entry e: the sum of its contributions in the original monomial order,
// then the homotopy
template <int L>
__device__ __forceinline__ void entry_from_V(const DevSys &S, int e, double t, const double *__restrict__ V,
                                             const double *__restrict__ HS, double *__restrict__ H,
                                             double *__restrict__ JH, double *__restrict__ HT = nullptr)
{
    const C<L> acc = sum_contributions<L>(S, __ldg(S.tptr + e), __ldg(S.tptr + e + 1), V);
    entry_finish<L>(S, e, t, acc, HS, H, JH, HT);
}

// h(z, t) (or f(z) for t < 0) and its Jacobian by the block; entries are taken in the
// order of S.eperm (longest contribution lists first)
template <int L, int TB>
__device__ void block_eval(const DevSys &S, const double *__restrict__ z, double t, const Slot<L> &w)
{
    const int n = S.n, tid = threadIdx.x;
    const C<L> gs = gamma_one_minus_t<L>(S.gre, S.gim, t < 0.0 ? 0.0 : t);
    for (int j = tid; j < n; j += TB) {
        powers_of<L>(S, j, z, w.PW);
        if (t >= 0.0 && j < S.npoly) homotopy_terms<L>(S, j, z, gs, w.HS, w.HT != nullptr);
    }
    __syncthreads();
    for (int q = tid; q < S.nmon; q += TB) monomial_to_V<L>(S, __ldg(S.perm + q), z, w.PW, w.V);
    __syncthreads();
    const int ne = S.npoly * (n + 1);
    for (int q = tid; q < ne; q += TB) entry_from_V<L>(S, __ldg(S.eperm + q), t, w.V, w.HS, w.H, w.JH, w.HT);
    __syncthreads();
}

// ------------------------------------------------------------------------------ solves
// The flat indices tid, tid + TB, tid + 2 TB, ... below cnt, as (idx / w, idx % w) pairs:
// one division per walk, then an increment with a carry (the trailing updates of the
// eliminations visit w x w entries; a division per entry is dozens of integer
// instructions).
struct DivWalk {
    int hi, lo, dhi, dlo, w;
    __device__ __forceinline__ DivWalk(int idx, int step, int w_) : w(w_)
    {
        hi = idx / w;
        lo = idx - hi * w;
        dhi = step / w;
        dlo = step - dhi * w;
    }
    __device__ __forceinline__ void next()
    {
        hi += dhi;
        lo += dlo;
        if (lo >= w) {
            lo -= w;
            hi++;
        }
    }
};
// Elimination with partial pivoting on [A b] in the working precision (Sec. 4), block
// version: the pivot is the entry of largest leading-limb |.|^2 (ties to the lowest row),
// rows are swapped, the pivot's reciprocal replaces it, multipliers replace the column
// below it, the trailing block and b are updated; back substitution leaves z = A^-1 b in b.
// *cond gets log10 of the ratio of the largest to the smallest pivot modulus.
template <int L, int TB>
__device__ int block_ge(int n, double *__restrict__ A, double *__restrict__ b, BlockShared &sh, double *cond)
{
    const int tid = threadIdx.x;
    const size_t ap = (size_t)n * n;
    double pmax = 0.0, pmin = INFINITY;
    for (int k = 0; k < n; k++) {
        long long bk = -1;
        int bi = 0x7fffffff;
        for (int i = k + tid; i < n; i += TB) {
            const long long key = amax_key(c_abs2_lead(ld_c<L>(A, ap, (size_t)i * n + k)));
            if (key > bk) {
                bk = key;
                bi = i;
            }
        }
        block_argmax_key<TB>(bk, bi, sh);
        const double bv = amax_value(bk);
        if (!(bv > 0.0)) return HC_SINGULAR;
        pmax = fmax(pmax, bv);
        pmin = fmin(pmin, bv);
        const int piv = bi;
        if (piv != k) {
            for (int j = k + tid; j < n; j += TB) {
                const C<L> t0 = ld_c<L>(A, ap, (size_t)k * n + j);
                st_c<L>(A, ap, (size_t)k * n + j, ld_c<L>(A, ap, (size_t)piv * n + j));
                st_c<L>(A, ap, (size_t)piv * n + j, t0);
            }
            if (tid == 0) {
                const C<L> t0 = ld_c<L>(b, n, k);
                st_c<L>(b, n, k, ld_c<L>(b, n, piv));
                st_c<L>(b, n, piv, t0);
            }
        }
        __syncthreads();
        if (tid == 0) st_c<L>(A, ap, (size_t)k * n + k, c_inv(ld_c<L>(A, ap, (size_t)k * n + k)));
        __syncthreads();
        const C<L> inv = ld_c<L>(A, ap, (size_t)k * n + k);
        for (int i = k + 1 + tid; i < n; i += TB)
            st_c<L>(A, ap, (size_t)i * n + k, c_mul(ld_c<L>(A, ap, (size_t)i * n + k), inv));
        __syncthreads();
        const int w = n - k;  // columns k+1..n-1 and b
        const int cnt = (n - k - 1) * w;
        DivWalk dw(tid, TB, w);
        for (int idx = tid; idx < cnt; idx += TB, dw.next()) {
            const int i = k + 1 + dw.hi, j = k + 1 + dw.lo;
            const C<L> l = ld_c<L>(A, ap, (size_t)i * n + k);
            if (j < n)
                st_c<L>(A, ap, (size_t)i * n + j, c_fnma(ld_c<L>(A, ap, (size_t)i * n + j), l, ld_c<L>(A, ap, (size_t)k * n + j)));
            else
                st_c<L>(b, n, i, c_fnma(ld_c<L>(b, n, i), l, ld_c<L>(b, n, k)));
        }
        __syncthreads();
    }
    for (int i = n - 1; i >= 0; i--) {
        if (tid == 0) st_c<L>(b, n, i, c_mul(ld_c<L>(b, n, i), ld_c<L>(A, ap, (size_t)i * n + i)));
        __syncthreads();
        const C<L> zi = ld_c<L>(b, n, i);
        for (int r = tid; r < i; r += TB)
            st_c<L>(b, n, r, c_fnma(ld_c<L>(b, n, r), ld_c<L>(A, ap, (size_t)r * n + i), zi));
        __syncthreads();
    }
    *cond = 0.5 * log10(pmax / pmin);
    return HC_OK;
}

struct cdv { double re, im; };
__device__ __forceinline__ cdv cdv_mul(cdv a, cdv b) { return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)}; }
__device__ __forceinline__ cdv cdv_fnma(cdv acc, cdv a, cdv b)
{
    return {fma(-a.re, b.re, fma(a.im, b.im, acc.re)), fma(-a.re, b.im, fma(-a.im, b.re, acc.im))};
}

// FP64 LU of the leading limbs with partial pivoting (the same pivot rule), block version.
// B[2][n][n], column-major (entry (i, j) at j n + i, so that the column walks of the
// pivot search, the multipliers, the trailing update and the triangular solves are
// contiguous), gets L (unit, below the diagonal), U, and the reciprocals of U's diagonal;
// PIV[k] is the original row that ends in row k (the row swaps composed).
template <int L, int TB>
__device__ int block_lu64(int n, const double *__restrict__ A, double *__restrict__ B, int32_t *__restrict__ PIV,
                          BlockShared &sh, double *cond)
{
    const int tid = threadIdx.x;
    const size_t ap = (size_t)n * n;
    for (int q = tid; q < n * n; q += TB) {
        const int j = q / n, i = q - j * n;
        double re, im;
        ld_lead<L>(A, ap, (size_t)i * n + j, re, im);
        B[q] = re;
        B[ap + q] = im;
    }
    for (int q = tid; q < n; q += TB) PIV[q] = q;
    __syncthreads();
    auto ld = [&](int i, int j) { return cdv{B[(size_t)j * n + i], B[ap + (size_t)j * n + i]}; };
    auto st = [&](int i, int j, cdv v) { B[(size_t)j * n + i] = v.re; B[ap + (size_t)j * n + i] = v.im; };
    auto mag = [&](cdv a) { return add_(mul_(a.re, a.re), mul_(a.im, a.im)); };
    // pivot of column 0
    Piv pv = piv_none();
    for (int i = tid; i < n; i += TB) {
        const cdv v = ld(i, 0);
        piv_take(pv, amax_key(mag(v)), i, v.re, v.im);
    }
    pv = block_argmax_piv<TB>(pv, sh);
    double pmax = 0.0, pmin = INFINITY;
    // Two barriers per column: (A) multipliers and row swap, (B) trailing update, which also
    // finds the next column's pivot (its warps' candidates meet after the barrier)
    for (int k = 0; k < n; k++) {
        const double bv = amax_value(pv.k);
        if (!(bv > 0.0)) return HC_SINGULAR;
        pmax = fmax(pmax, bv);
        pmin = fmin(pmin, bv);
        const int piv = pv.i;
        // (A) the pivot row's value moves to row k: multipliers of column k from the rows
        // before the swap (row piv takes the old row k's entry), the other columns swapped.
        // The pivot's reciprocal conj(a) / |a|^2 is formed only by the threads that use it
        // (a division is a long FP64 sequence: every thread of a large block forming it
        // would cost more than the factorisation itself), from the pivot value carried by
        // the search (entry (piv, k) is overwritten by a multiplier in this phase)
        cdv inv = {0.0, 0.0};
        if (tid == 0 || k + 1 + tid < n) {
            const double r = 1.0 / bv;
            inv = {pv.re * r, -pv.im * r};
        }
        for (int i = k + 1 + tid; i < n; i += TB) st(i, k, cdv_mul(ld(i == piv ? k : i, k), inv));
        if (piv != k) {
            if (tid == 0) {
                const int t0 = PIV[k];
                PIV[k] = PIV[piv];
                PIV[piv] = t0;
            }
            for (int j = tid; j < n; j += TB) {
                if (j == k) continue;
                const cdv t0 = ld(k, j);
                st(k, j, ld(piv, j));
                st(piv, j, t0);
            }
        }
        __syncthreads();
        // (B) the reciprocal on the diagonal, the trailing update, the next pivot
        if (tid == 0) st(k, k, inv);
        const int w = n - k - 1;
        pv = piv_none();
        DivWalk dw(tid, TB, w > 0 ? w : 1);
        for (int idx = tid; idx < w * w; idx += TB, dw.next()) {
            const int j = k + 1 + dw.hi, i = k + 1 + dw.lo;
            const cdv v = cdv_fnma(ld(i, j), ld(i, k), ld(k, j));
            st(i, j, v);
            if (j == k + 1) piv_take(pv, amax_key(mag(v)), i, v.re, v.im);
        }
        warp_argmax_piv(pv);
        piv_publish(pv, sh);
        __syncthreads();
        pv = piv_merge<TB>(sh);
    }
    *cond = 0.5 * log10(pmax / pmin);
    return HC_OK;
}

// y = A^-1 r with the (column-major) FP64 factors of block_lu64, by one warp (the calling
// warp): r[2][n] in the original row order is permuted into y, then forward and back
// substitution with warp barriers only.  y must not alias r.  The caller synchronises the
// block before other warps read y.
__device__ __forceinline__ void warp_lu64_solve(int n, const double *__restrict__ B, const int32_t *__restrict__ PIV,
                                                const double *__restrict__ r, double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const size_t ap = (size_t)n * n;
    for (int i = lane; i < n; i += 32) {
        const int p = PIV[i];
        y[i] = r[p];
        y[n + i] = r[n + p];
    }
    __syncwarp();
    for (int k = 0; k < n - 1; k++) {
        const cdv yk = {y[k], y[n + k]};
        for (int i = k + 1 + lane; i < n; i += 32) {
            const cdv v = cdv_fnma(cdv{y[i], y[n + i]}, cdv{B[(size_t)k * n + i], B[ap + (size_t)k * n + i]}, yk);
            y[i] = v.re;
            y[n + i] = v.im;
        }
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; i--) {
        const cdv zi = cdv_mul(cdv{y[i], y[n + i]}, cdv{B[(size_t)i * n + i], B[ap + (size_t)i * n + i]});
        __syncwarp();
        if (lane == 0) {
            y[i] = zi.re;
            y[n + i] = zi.im;
        }
        for (int q = lane; q < i; q += 32) {
            const cdv v = cdv_fnma(cdv{y[q], y[n + q]}, cdv{B[(size_t)i * n + q], B[ap + (size_t)i * n + q]}, zi);
            y[q] = v.re;
            y[n + q] = v.im;
        }
        __syncwarp();
    }
}

// r_i = -h_i - sum_j J_ij dz_j in L limbs, leading limbs into RV: T = 8 threads per row,
// each summing a strided part of the row, then a fixed shuffle tree adds the 8 parts;
// TB / 8 rows at a time.  The order of the sums does not depend on the block size, so
// every block size gives the same bits.
template <int L, int TB>
__device__ __forceinline__ void block_refine_residual(int n, const double *__restrict__ JH, const double *__restrict__ H,
                                                      const double *__restrict__ DZ, double *__restrict__ RV)
{
    constexpr int T = 8;
    const int g = threadIdx.x / T, q = threadIdx.x % T, rows = TB / T;
    for (int base = 0; base < n; base += rows) {
        const int i = base + g;
        C<L> acc = c_zero<L>();
        if (i < n)
            for (int j = q; j < n; j += T)
                acc = c_fnma(acc, ld_c<L>(JH, (size_t)n * n, (size_t)i * n + j), ld_c<L>(DZ, n, j));
        for (int o = T >> 1; o > 0; o >>= 1) {
            C<L> other;
#pragma unroll
            for (int l = 0; l < L; l++) {
                other.re.v[l] = __shfl_xor_sync(0xffffffffu, acc.re.v[l], o);
                other.im.v[l] = __shfl_xor_sync(0xffffffffu, acc.im.v[l], o);
            }
            acc = c_add(acc, other);
        }
        if (i < n && q == 0) {
            const C<L> r = c_sub(acc, ld_c<L>(H, n, i));
            RV[i] = r.re.v[0];
            RV[n + i] = r.im.v[0];
        }
    }
}

struct NewtonOut {
    double res, dzn, zn, cond;
    int status, sweeps;
};

//
// One Newton iteration of Alg. 4.1 at z (in place): evaluate h and J, the residual of the
// incoming z (max_i |h_i| of the leading limbs), solve J dz = -h, z += dz (all or nothing
// on non-finite values).  Same readings as hc_newton_step.
//
template <int L, int TB>
__device__ NewtonOut block_newton(const DevSys &S, double *__restrict__ z, double t, int lu_mode, int max_refine,
                                  const Slot<L> &w, BlockShared &sh)
{
    const int n = S.n, tid = threadIdx.x;
    NewtonOut o{0.0, 0.0, 0.0, 0.0, HC_OK, 0};
    block_eval<L, TB>(S, z, t, w);
    double r2 = 0.0;
    int fin = 1;
    for (int i = tid; i < n; i += TB) {
        double re, im;
        ld_lead<L>(w.H, n, i, re, im);
        const double v = add_(mul_(re, re), mul_(im, im));
        if (!isfinite(v)) fin = 0;
        r2 = fmax(r2, v);
    }
    fin = block_and(fin, sh);
    o.res = sqrt(block_max<TB>(r2, sh));
    if (!fin) {
        o.status = HC_NONFINITE;
        return o;
    }
    const double *D;  // the update, [2][L][n]
    bool subtract;
    if (lu_mode == HC_LU_NATIVE) {
        o.status = block_ge<L, TB>(n, w.JH, w.H, sh, &o.cond);
        if (o.status != HC_OK) return o;
        D = w.H;
        subtract = true;
    } else {
        o.status = block_lu64<L, TB>(n, w.JH, w.B, w.PIV, sh, &o.cond);
        if (o.status != HC_OK) return o;
        for (int i = tid; i < n; i += TB) {
            double re, im;
            ld_lead<L>(w.H, n, i, re, im);
            w.RV[i] = -re;
            w.RV[n + i] = -im;
        }
        __syncthreads();
        if (tid < 32) warp_lu64_solve(n, w.B, w.PIV, w.RV, w.Y);
        __syncthreads();
        double xn = 0.0;
        for (int i = tid; i < n; i += TB) {
            st_c<L>(w.DZ, n, i, c_from<L>(w.Y[i], w.Y[n + i]));
            double re, im;
            ld_lead<L>(z, n, i, re, im);
            xn = fmax(xn, sqrt(add_(mul_(re, re), mul_(im, im))));
        }
        xn = block_max<TB>(xn, sh);
        const double tol = ldexp(1.0, -53 * L);
        double prev = INFINITY;
        for (int it = 1; it <= max_refine; it++) {
            block_refine_residual<L, TB>(n, w.JH, w.H, w.DZ, w.RV);
            __syncthreads();
            if (tid < 32) warp_lu64_solve(n, w.B, w.PIV, w.RV, w.Y);
            __syncthreads();
            double dn = 0.0, zz = 0.0;
            for (int i = tid; i < n; i += TB) {
                const double dr = w.Y[i], di = w.Y[n + i];
                dn = fmax(dn, sqrt(add_(mul_(dr, dr), mul_(di, di))));
            }
            dn = block_max<TB>(dn, sh);
            o.sweeps = it;
            if (dn >= prev) break;  // no longer shrinking: at the rounding floor, not applied
            for (int i = tid; i < n; i += TB) {
                const C<L> v = c_add(ld_c<L>(w.DZ, n, i), c_from<L>(w.Y[i], w.Y[n + i]));
                st_c<L>(w.DZ, n, i, v);
                zz = fmax(zz, sqrt(c_abs2_lead(v)));
            }
            zz = block_max<TB>(zz, sh);
            if (dn <= tol * fmax(xn, zz)) break;
            prev = dn;
        }
        D = w.DZ;
        subtract = false;
    }
    // update, all or nothing
    int ok = 1;
    double dzn = 0.0, zn = 0.0;
    for (int i = tid; i < n; i += TB) {
        const C<L> d = ld_c<L>(D, n, i);
        const C<L> v = subtract ? c_sub(ld_c<L>(z, n, i), d) : c_add(ld_c<L>(z, n, i), d);
        if (!c_finite_lead(v)) ok = 0;
        dzn = fmax(dzn, sqrt(c_abs2_lead(d)));
        zn = fmax(zn, sqrt(c_abs2_lead(v)));
    }
    ok = block_and(ok, sh);
    block_max2<TB>(dzn, zn, sh);
    o.dzn = dzn;
    o.zn = zn;
    if (!ok) {
        o.status = HC_NONFINITE;
        return o;
    }
    for (int i = tid; i < n; i += TB) {
        const C<L> d = ld_c<L>(D, n, i);
        st_c<L>(z, n, i, subtract ? c_sub(ld_c<L>(z, n, i), d) : c_add(ld_c<L>(z, n, i), d));
    }
    __syncthreads();
    return o;
}

}  // namespace hc
