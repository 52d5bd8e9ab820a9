// hc_grid.cu -- one large path on the whole GPU (hc_track_path with HC_TRACK_GRID).
//
// A path whose system has ~10^5 monomials is too much for one thread block (one SM).
// Here one predictor-corrector stage of Alg. 3.1 is a fixed sequence of kernels,
// captured once as a CUDA graph and replayed by the host until the path ends:
//
//   begin (1 block)                      init, predictor (or end-game set-up)
//   max_it x Newton iteration (Alg. 4.1):
//     powers (n blocks of 1 thread)      x_j^e
//     monomials (grid)                   values and partials of every monomial -> V
//     (beside powers .. chunks, a branch of the graph: start-system terms, n blocks of 1)
//     entries (grid)                     sums per Jacobian entry + homotopy -> H, J
//     lu prep (1 block of 1024)          residual, leading limbs of J
//     ceil(n / 16) x [panel (1 block), update (grid)]   FP64 LU with partial pivoting
//     inverse (n warps)                  the FP64 inverse, one column per warp
//     gemv (grid), apply (1 block)       dz_0 = inverse x (-h)
//     max_refine x [residual rows (n blocks of 4 warps), gemv, apply]   refinement in L limbs
//     update (1 block)                   z += dz, convergence test
//   end (1 block)                        accept / step back, step size, stop tests
//
// The refinement applies the explicit inverse of the FP64 factors (n triangular solves
// in parallel, once per factorisation) instead of a triangular solve per sweep: each
// sweep's correction is then a matrix-vector product of a few microseconds, where one
// warp's substitution took a quarter of a millisecond.  Like the factors it stands in for,
// the inverse is an FP64 approximation of J^-1; the sweeps converge to the same solution
// in L limbs.
//
// The control flow of the method is data dependent; every kernel first reads the stage
// state and returns at once when its work is not needed (the corrector converged, the
// refinement stopped, the path ended), so a fixed graph carries it.  No kernel waits on
// another: kernel boundaries are the only synchronisation.
#include <string.h>

#include <vector>

#include "track.cuh"

#include <vector>

namespace hc {

struct GStage {
    double t1, h, res, res_first, cond, dzn, zn, xn, prev_dn;
    double pmax, pmin;        // the blocked LU's largest and smallest pivot so far
    int it, conv, nst, allowed, refine_active, sweeps, pad[2];
};

struct GArgs {
    DevSys S;
    PathState *st;
    GStage *g;
    const double *x0;
    double *z, *zp, *zpp, *zh, *ZP, *PW, *V, *HS, *H, *JH, *B, *RV, *DZ;
    double *INV;              // [2][n][n] the inverse of the FP64 factors, column-major
    double *D;                // [2][n] the FP64 correction of a solve or sweep
    double *DNB;              // [ceil(n / HC_GEMV_ROWS)] its largest moduli, per block
    int32_t *PIV;
    int32_t *PSTEP;           // [n] the blocked LU's pivot row of each step
    // the entries' contribution lists cut into chunks of at most `chunk`, summed in
    // parallel (k_g_chunks), then per entry in chunk order (k_g_entries)
    const int32_t *cbeg;      // [nchunks+1] chunk c covers tlist[cbeg[c] .. cend[c])
    const int32_t *cend;
    const int32_t *eptr;      // [ne+1] the chunks of entry e: eptr[e] .. eptr[e+1]-1
    const int32_t *eord;      // [ne] the entries with HC_GLONG chunks or more, then the rest
    int nlong;                //      (longest first): the order of k_g_entries
    double *P;                // [2][L][nchunks] chunk sums
    int nchunks;
    hc_track_opts o;
    hc_step_record *log;
    int log_cap;
    long long log0;           // corrector stages before this call (the log's offset)
};

__device__ __forceinline__ bool g_active(const GStage &g)
{
    return g.it < g.allowed && !g.conv && g.nst == HC_OK;
}

template <int L> __global__ void __launch_bounds__(HC_TB) k_g_begin(GArgs a)
{
    PathState st = *a.st;
    GStage &g = *a.g;
    const int n = a.S.n, tid = threadIdx.x;
    if (st.phase == 0) {
        for (int q = tid; q < 2 * L * n; q += HC_TB) a.z[q] = a.x0[q];
        path_init(st, a.o, 0);
        __syncthreads();
        if (tid == 0) *a.st = st;
    }
    __syncthreads();
    if (st.phase == 1) {
        double t1, h;
        stage_predict<L, HC_TB>(a.o, st, n, a.z, a.zp, a.zpp, nullptr, a.zh, a.ZP, t1, h);
        if (tid == 0) {
            g.t1 = t1;
            g.h = h;
            g.allowed = a.o.max_it;
        }
    } else if (st.phase == 2) {
        for (int q = tid; q < 2 * L * n; q += HC_TB) a.zh[q] = a.z[q];
        if (tid == 0) {
            g.t1 = 1.0;
            g.h = 0.0;
            g.allowed = min(a.o.max_it, a.o.end_it - st.end_its);
        }
    } else if (tid == 0) {
        g.allowed = 0;
    }
    if (tid == 0) {
        g.it = 0;
        g.conv = 0;
        g.nst = HC_OK;
        g.res = 1.0;
        g.res_first = -1.0;
        g.cond = 0.0;
        g.refine_active = 0;
    }
}

// The power table (k_g_powers, one variable per block) and the start-system terms of the
// homotopy (k_g_terms, one row per block): one dependent chain of complex products per
// index, each in a block of its own so that the chains spread over the SMs.  Both are
// bound by the latency of their chains (a row's x_i^(d-1) by binary powering is about a
// dozen quad-double products in a row: 0.14 ms at n = 96), so the terms, which only the
// entry sums need, run in a branch of the stage graph beside the power table, the
// monomials and the chunk sums.
template <int L> __global__ void __launch_bounds__(1) k_g_powers(GArgs a)
{
    if (!g_active(*a.g)) return;
    powers_of<L>(a.S, blockIdx.x, a.zh, a.PW);
}
template <int L> __global__ void __launch_bounds__(1) k_g_terms(GArgs a)
{
    const GStage &g = *a.g;
    if (!g_active(g)) return;
    const C<L> gs = gamma_one_minus_t<L>(a.S.gre, a.S.gim, g.t1);
    homotopy_terms<L>(a.S, blockIdx.x, a.zh, gs, a.HS, false);
}

// one thread per monomial in one-warp blocks: all blocks are resident at once (20 or 21
// per SM for 98,304 monomials), so every SM gets nearly the same number of monomials;
// with 128-thread blocks 8 SMs took a sixth block while 144 had five, and the SMs that
// finished first idled for a sixth of the kernel
#define HC_GMONO 32
template <int L> __global__ void __launch_bounds__(HC_GMONO) k_g_monomials(GArgs a)
{
    if (!g_active(*a.g)) return;
    const int q = blockIdx.x * HC_GMONO + threadIdx.x;
    if (q < a.S.nmon) monomial_to_V<L>(a.S, __ldg(a.S.perm + q), a.zh, a.PW, a.V);
}

// one chunk per thread, in one-warp blocks: the chunks' sums are chains of additions
// bound by their latency, so every SM should hold the same number of warps (in
// 128-thread blocks, 347 blocks on 152 SMs left the FP64 pipes 62 % busy over the kernel
// against 83 % while active)
#define HC_GCHUNK 32
template <int L> __global__ void __launch_bounds__(HC_GCHUNK) k_g_chunks(GArgs a)
{
    const GStage &g = *a.g;
    if (!g_active(g)) return;
    const int c = blockIdx.x * HC_GCHUNK + threadIdx.x;
    if (c >= a.nchunks) return;
    st_c<L>(a.P, a.nchunks, c, sum_contributions<L>(a.S, __ldg(a.cbeg + c), __ldg(a.cend + c), a.V));
}

// the chunk sums of each entry added in a fixed order, then the homotopy, in one-warp
// blocks.  An entry of fewer than HC_GLONG chunks is one thread's, its chunks added in
// order (an entry of one chunk takes its sum as is: the same value as one sequential sum,
// as in the block engine).  A longer entry (the value entries of long rows: 32 chunks for
// 1,024 terms) is one warp's: lane l adds the chunks c0 + l, c0 + l + 32, ... in order,
// then a fixed shuffle tree adds the lanes.  In one thread each, the value entries were
// chains of 31 quad-double additions, taken longest first by one block on one SM.
#define HC_GLONG 8
template <int L> __global__ void __launch_bounds__(32) k_g_entries(GArgs a)
{
    const GStage &g = *a.g;
    if (!g_active(g)) return;
    const int lane = threadIdx.x, ne = a.S.npoly * (a.S.n + 1);
    if ((int)blockIdx.x < a.nlong) {
        const int e = __ldg(a.eord + blockIdx.x);
        const int c0 = __ldg(a.eptr + e), c1 = __ldg(a.eptr + e + 1);
        C<L> acc = c_zero<L>();
        for (int c = c0 + lane; c < c1; c += 32) acc = c_add(acc, ld_c<L>(a.P, a.nchunks, c));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            C<L> other;
#pragma unroll
            for (int l = 0; l < L; l++) {
                other.re.v[l] = __shfl_down_sync(0xffffffffu, acc.re.v[l], o);
                other.im.v[l] = __shfl_down_sync(0xffffffffu, acc.im.v[l], o);
            }
            acc = c_add(acc, other);
        }
        if (lane == 0) entry_finish<L>(a.S, e, g.t1, acc, a.HS, a.H, a.JH, nullptr);
        return;
    }
    const int q = a.nlong + ((int)blockIdx.x - a.nlong) * 32 + lane;
    if (q >= ne) return;
    const int e = __ldg(a.eord + q);
    const int c0 = __ldg(a.eptr + e), c1 = __ldg(a.eptr + e + 1);
    C<L> acc = ld_c<L>(a.P, a.nchunks, c0);
    for (int c = c0 + 1; c < c1; c++) acc = c_add(acc, ld_c<L>(a.P, a.nchunks, c));
    entry_finish<L>(a.S, e, g.t1, acc, a.HS, a.H, a.JH, nullptr);
}

#define HC_GLU 1024  // threads of the LU preparation block

// The residual ||h|| and ||x|| of the incoming point (leading limbs), every thread
// getting them; returns 0 if h is not finite
template <int L> __device__ __forceinline__ int g_residual(const GArgs &a, BlockShared &sh, double &res, double &xn)
{
    const int n = a.S.n;
    double r2 = 0.0;
    xn = 0.0;
    int fin = 1;
    for (int i = threadIdx.x; i < n; i += HC_GLU) {
        double re, im;
        ld_lead<L>(a.H, n, i, re, im);
        const double v = add_(mul_(re, re), mul_(im, im));
        if (!isfinite(v)) fin = 0;
        r2 = fmax(r2, v);
        ld_lead<L>(a.zh, n, i, re, im);
        xn = fmax(xn, sqrt(add_(mul_(re, re), mul_(im, im))));
    }
    fin = block_and(fin, sh);
    block_max2<HC_GLU>(r2, xn, sh);
    res = sqrt(r2);
    return fin;
}

// ---- The blocked FP64 LU: the same factors, pivots and condition estimate as
// block_lu64, bit for bit, in panels of HC_GLU_NB columns spread over the GPU.  A single
// block's LU is bound by one SM's FP64 pipe (two lanes a clock: 0.57 ms at n = 96), while
// its trailing updates are independent per column.  Per panel:
//   k_g_panel (1 block)     the panel's columns factored in shared memory: pivot search,
//                           row swap (within the panel), multipliers, rank-1 updates
//   k_g_lu_update (grid)    every other column: the panel's row swaps, then the panel's
//                           eliminations in step order (forward substitution with the unit
//                           lower triangle and the update of the rows below, one sweep)
// Every entry receives the same operations in the same order as in block_lu64 (the
// updates a_ij -= l_ik a_kj by increasing k, the swaps by increasing step), so the results
// are identical.
#define HC_GLU_NB 16
#define HC_GPANEL 256
#define HC_GUPD 4   // columns (warps) per block of k_g_lu_update

// residual, norms, the leading limbs of J into B (column-major), the identity permutation
template <int L> __global__ void __launch_bounds__(HC_GLU, 1) k_g_lu_prep(GArgs a)
{
    __shared__ BlockShared sh;
    GStage &g = *a.g;
    if (!g_active(g)) return;
    const int n = a.S.n, tid = threadIdx.x;
    double res, xn;
    const int fin = g_residual<L>(a, sh, res, xn);
    const size_t ap = (size_t)n * n;
    if (fin) {
        for (int q = tid; q < n * n; q += HC_GLU) {
            const int j = q / n, i = q - j * n;
            double re, im;
            ld_lead<L>(a.JH, ap, (size_t)i * n + j, re, im);
            a.B[q] = re;
            a.B[ap + q] = im;
        }
        for (int q = tid; q < n; q += HC_GLU) a.PIV[q] = q;
    }
    if (tid == 0) {
        g.res = res;
        if (g.res_first < 0) g.res_first = res;
        g.cond = 0.0;
        g.xn = xn;
        g.pmax = 0.0;
        g.pmin = INFINITY;
        g.refine_active = 0;
        g.prev_dn = INFINITY;
        g.sweeps = 0;
        if (!fin) {
            g.it++;
            g.nst = HC_NONFINITE;
        }
    }
}

// columns kb .. kb+nb-1, rows kb .. n-1 (m rows), factored in shared memory with the
// steps of block_lu64 restricted to the panel: two barriers per column, (A) multipliers
// and the row swap within the panel, (B) the rank-1 update of the panel's later columns,
// which also finds the next column's pivot
template <int L> __global__ void __launch_bounds__(HC_GPANEL) k_g_panel(GArgs a, int kb)
{
    __shared__ BlockShared sh;
    extern __shared__ double psh[];  // [2][nb][m], column-major
    GStage &g = *a.g;
    if (!g_active(g)) return;
    const int n = a.S.n, tid = threadIdx.x, m = n - kb, nb = min(HC_GLU_NB, m);
    const size_t ap = (size_t)n * n, pp = (size_t)nb * m;
    for (int q = tid; q < nb * m; q += HC_GPANEL) {
        const int c = q / m, r = q - c * m;
        const size_t o = (size_t)(kb + c) * n + kb + r;
        psh[q] = a.B[o];
        psh[pp + q] = a.B[ap + o];
    }
    __syncthreads();
    auto ld = [&](int i, int c) { return cdv{psh[(size_t)c * m + i], psh[pp + (size_t)c * m + i]}; };
    auto st = [&](int i, int c, cdv v) { psh[(size_t)c * m + i] = v.re; psh[pp + (size_t)c * m + i] = v.im; };
    auto mag = [&](cdv v) { return add_(mul_(v.re, v.re), mul_(v.im, v.im)); };
    double pmax = g.pmax, pmin = g.pmin;
    // pivot of the panel's first column: the largest squared modulus, ties to the lowest row
    Piv pv = piv_none();
    for (int i = tid; i < m; i += HC_GPANEL) {
        const cdv v = ld(i, 0);
        piv_take(pv, amax_key(mag(v)), i, v.re, v.im);
    }
    pv = block_argmax_piv<HC_GPANEL>(pv, sh);
    for (int c = 0; c < nb; c++) {
        const double bv = amax_value(pv.k);
        if (!(bv > 0.0)) {
            if (tid == 0) {
                g.it++;
                g.nst = HC_SINGULAR;
            }
            return;
        }
        pmax = fmax(pmax, bv);
        pmin = fmin(pmin, bv);
        const int piv = pv.i;
        // (A) multipliers of column c from the rows before the swap (row piv takes the old
        // row c's entry), the panel's other columns swapped; the pivot's reciprocal from
        // the value carried by the search
        cdv inv = {0.0, 0.0};
        if (tid == 0 || c + 1 + tid < m) {
            const double r = 1.0 / bv;
            inv = {pv.re * r, -pv.im * r};
        }
        for (int i = c + 1 + tid; i < m; i += HC_GPANEL) st(i, c, cdv_mul(ld(i == piv ? c : i, c), inv));
        if (piv != c)
            for (int cc = tid; cc < nb; cc += HC_GPANEL) {
                if (cc == c) continue;
                const cdv t0 = ld(c, cc);
                st(c, cc, ld(piv, cc));
                st(piv, cc, t0);
            }
        if (tid == 0) {
            a.PSTEP[kb + c] = kb + piv;
            if (piv != c) {
                const int t0 = a.PIV[kb + c];
                a.PIV[kb + c] = a.PIV[kb + piv];
                a.PIV[kb + piv] = t0;
            }
        }
        __syncthreads();
        // (B) the reciprocal on the diagonal, the rank-1 update of columns c+1 .. nb-1,
        // the next column's pivot
        if (tid == 0) st(c, c, inv);
        const int w = m - c - 1, wc = nb - c - 1;
        pv = piv_none();
        DivWalk dw(tid, HC_GPANEL, w > 0 ? w : 1);
        for (int idx = tid; idx < w * wc; idx += HC_GPANEL, dw.next()) {
            const int cj = c + 1 + dw.hi, i = c + 1 + dw.lo;
            const cdv v = cdv_fnma(ld(i, cj), ld(i, c), ld(c, cj));
            st(i, cj, v);
            if (cj == c + 1) piv_take(pv, amax_key(mag(v)), i, v.re, v.im);
        }
        warp_argmax_piv(pv);
        piv_publish(pv, sh);
        __syncthreads();
        pv = piv_merge<HC_GPANEL>(sh);
    }
    for (int q = tid; q < nb * m; q += HC_GPANEL) {
        const int c = q / m, r = q - c * m;
        const size_t o = (size_t)(kb + c) * n + kb + r;
        a.B[o] = psh[q];
        a.B[ap + o] = psh[pp + q];
    }
    if (tid == 0) {
        g.pmax = pmax;
        g.pmin = pmin;
        if (kb + nb == n) g.cond = 0.5 * log10(pmax / pmin);
    }
}

// every column outside the panel kb .. kb+nb-1, one warp each: rows kb .. n-1 of the
// column in shared memory, the panel's swaps, and (columns right of the panel) the
// panel's eliminations, with the panel's multipliers from a shared-memory copy
template <int L> __global__ void __launch_bounds__(32 * HC_GUPD) k_g_lu_update(GArgs a, int kb)
{
    extern __shared__ double ush[];  // multipliers [2][nb][m], then per warp a column [2][m]
    const GStage &g = *a.g;
    if (!g_active(g)) return;
    const int n = a.S.n, m = n - kb, nb = min(HC_GLU_NB, m), lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t ap = (size_t)n * n, pp = (size_t)nb * m;
    int j = blockIdx.x * HC_GUPD + wid;
    if (j >= kb) j += nb;
    double *lm = ush, *col = ush + 2 * pp + (size_t)wid * 2 * m;
    for (int q = threadIdx.x; q < nb * m; q += 32 * HC_GUPD) {
        const int c = q / m, r = q - c * m;
        const size_t o = (size_t)(kb + c) * n + kb + r;
        lm[q] = a.B[o];
        lm[pp + q] = a.B[ap + o];
    }
    __syncthreads();
    if (j >= n) return;
    const size_t co = (size_t)j * n + kb;
    for (int i = lane; i < m; i += 32) {
        col[i] = a.B[co + i];
        col[m + i] = a.B[ap + co + i];
    }
    __syncwarp();
    if (lane == 0)
        for (int c = 0; c < nb; c++) {
            const int p = a.PSTEP[kb + c] - kb;
            if (p != c) {
                const double tr = col[c], ti = col[m + c];
                col[c] = col[p];
                col[m + c] = col[m + p];
                col[p] = tr;
                col[m + p] = ti;
            }
        }
    __syncwarp();
    if (j > kb)
        for (int c = 0; c < nb; c++) {
            const cdv u = {col[c], col[m + c]};
            for (int i = c + 1 + lane; i < m; i += 32) {
                const cdv v = cdv_fnma(cdv{col[i], col[m + i]}, cdv{lm[(size_t)c * m + i], lm[pp + (size_t)c * m + i]}, u);
                col[i] = v.re;
                col[m + i] = v.im;
            }
            __syncwarp();
        }
    for (int i = lane; i < m; i += 32) {
        a.B[co + i] = col[i];
        a.B[ap + co + i] = col[m + i];
    }
}

// column j = blockIdx.x of the inverse of the FP64 factors: the solve of e_j by one warp
// (warp_lu64_solve), from a shared-memory copy of the factors when they fit.  The block's
// other warps only help with that copy (2 n^2 doubles from L2: 576 loads per lane for
// one warp alone at n = 96).
#define HC_GINV 256
template <int L> __global__ void __launch_bounds__(HC_GINV) k_g_inverse(GArgs a, int b_smem)
{
    extern __shared__ double ish[];  // e_j [2][n], y [2][n], then (b_smem) the factors
    const GStage &g = *a.g;
    if (!g_active(g)) return;
    const int n = a.S.n, j = blockIdx.x, lane = threadIdx.x;
    double *ej = ish, *y = ish + 2 * n;
    const double *Bf = a.B;
    if (b_smem) {
        double *Bs = ish + 4 * n;
        for (int q = threadIdx.x; q < 2 * n * n; q += HC_GINV) Bs[q] = a.B[q];
        Bf = Bs;
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    for (int q = lane; q < 2 * n; q += 32) ej[q] = q == j ? 1.0 : 0.0;
    __syncwarp();
    warp_lu64_solve(n, Bf, a.PIV, ej, y);
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        a.INV[(size_t)j * n + i] = y[i];
        a.INV[(size_t)n * n + (size_t)j * n + i] = y[n + i];
    }
}

// d = INV r in FP64, HC_GEMV_ROWS rows per block (spread over the GPU: in one block the
// product was bound by one SM's FP64 pipe): 8 lanes per row, each summing the columns
// j = lane (mod 8) in order, then a fixed shuffle tree.  first: r = -h (the first solve);
// else r = the residual of k_g_refine_rows.  d goes to D, each block's largest |d_i| to
// DNB[block].
#define HC_GEMV_ROWS 8
template <int L> __global__ void __launch_bounds__(8 * HC_GEMV_ROWS) k_g_gemv(GArgs a, int first)
{
    __shared__ double rsh[2 * 256];
    __shared__ double msh[HC_GEMV_ROWS];
    const GStage &g = *a.g;
    if (!g_active(g) || (!first && !g.refine_active)) return;
    const int n = a.S.n, tid = threadIdx.x;
    for (int i = tid; i < n; i += 8 * HC_GEMV_ROWS) {
        if (first) {
            double re, im;
            ld_lead<L>(a.H, n, i, re, im);
            rsh[i] = -re;
            rsh[n + i] = -im;
        } else {
            rsh[i] = a.RV[i];
            rsh[n + i] = a.RV[n + i];
        }
    }
    __syncthreads();
    const size_t ip = (size_t)n * n;
    const int q = tid & 7, r = tid >> 3, i = blockIdx.x * HC_GEMV_ROWS + r;
    cdv d = {0.0, 0.0};
    if (i < n)
        for (int j = q; j < n; j += 8)
            d = cdv_fnma(d, cdv{-a.INV[(size_t)j * n + i], -a.INV[ip + (size_t)j * n + i]}, cdv{rsh[j], rsh[n + j]});
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        d.re = add_(d.re, __shfl_xor_sync(0xffffffffu, d.re, o));
        d.im = add_(d.im, __shfl_xor_sync(0xffffffffu, d.im, o));
    }
    if (q == 0) {
        double m = 0.0;
        if (i < n) {
            a.D[i] = d.re;
            a.D[n + i] = d.im;
            m = sqrt(add_(mul_(d.re, d.re), mul_(d.im, d.im)));
        }
        msh[r] = m;
    }
    __syncthreads();
    if (tid == 0) {
        double m = msh[0];
        for (int k = 1; k < HC_GEMV_ROWS; k++) m = fmax(m, msh[k]);
        a.DNB[blockIdx.x] = m;
    }
}

// The correction of k_g_gemv applied.  first: dz = d; else dz += d, and the refinement's
// stop test: ||d|| <= 2^(-53 L) max(||x||, ||dz||) or max_refine sweeps; a d no smaller
// than the previous one ends it without being added
#define HC_GAPPLY 256
template <int L> __global__ void __launch_bounds__(HC_GAPPLY) k_g_apply(GArgs a, int first)
{
    __shared__ BlockShared sh;
    GStage &g = *a.g;
    if (!g_active(g) || (!first && !g.refine_active)) return;
    const int n = a.S.n, tid = threadIdx.x, nb = (n + HC_GEMV_ROWS - 1) / HC_GEMV_ROWS;
    double dn = 0.0, zz = 0.0;
    for (int k = tid; k < nb; k += HC_GAPPLY) dn = fmax(dn, a.DNB[k]);
    dn = block_max<HC_GAPPLY>(dn, sh);
    // a refinement correction no smaller than the previous one (the residual is at its
    // rounding floor) ends the refinement without being added
    const bool apply = first || dn < g.prev_dn;
    if (apply) {
        for (int i = tid; i < n; i += HC_GAPPLY) {
            const C<L> d = c_from<L>(a.D[i], a.D[n + i]);
            const C<L> v = first ? d : c_add(ld_c<L>(a.DZ, n, i), d);
            st_c<L>(a.DZ, n, i, v);
            zz = fmax(zz, sqrt(c_abs2_lead(v)));
        }
    }
    zz = block_max<HC_GAPPLY>(zz, sh);
    if (tid == 0) {
        if (first) {
            g.refine_active = a.o.max_refine > 0;
        } else {
            g.sweeps++;
            const double tol = ldexp(1.0, -53 * L);
            if (!apply || dn <= tol * fmax(g.xn, zz) || g.sweeps >= a.o.max_refine) g.refine_active = 0;
            g.prev_dn = dn;
        }
    }
}

// r_i = -h_i - sum_j J_ij dz_j in L limbs, one block of HC_GREF threads per row: each
// thread takes the columns j = tid (mod HC_GREF), a fixed shuffle tree adds a warp's
// parts, and thread 0 adds the warps' sums in warp order.  The row's quad-double chain is
// what bounds this kernel (one warp per row: three products and five additions in a row,
// 75 us a sweep at n = 96); spreading the columns over four warps shortens it.
#define HC_GREF 128
template <int L> __global__ void __launch_bounds__(HC_GREF) k_g_refine_rows(GArgs a)
{
    __shared__ double part[HC_GREF / 32][2 * L];
    const GStage &g = *a.g;
    if (!g_active(g) || !g.refine_active) return;
    const int n = a.S.n, i = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    C<L> acc = c_zero<L>();
    for (int j = threadIdx.x; j < n; j += HC_GREF)
        acc = c_fnma(acc, ld_c<L>(a.JH, (size_t)n * n, (size_t)i * n + j), ld_c<L>(a.DZ, n, j));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        C<L> other;
#pragma unroll
        for (int l = 0; l < L; l++) {
            other.re.v[l] = __shfl_down_sync(0xffffffffu, acc.re.v[l], o);
            other.im.v[l] = __shfl_down_sync(0xffffffffu, acc.im.v[l], o);
        }
        acc = c_add(acc, other);
    }
    if (lane == 0)
#pragma unroll
        for (int l = 0; l < L; l++) {
            part[w][l] = acc.re.v[l];
            part[w][L + l] = acc.im.v[l];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < HC_GREF / 32; q++) {
            C<L> other;
#pragma unroll
            for (int l = 0; l < L; l++) {
                other.re.v[l] = part[q][l];
                other.im.v[l] = part[q][L + l];
            }
            acc = c_add(acc, other);
        }
        // acc = -sum_j J_ij dz_j, so r = acc - h_i
        const C<L> r = c_sub(acc, ld_c<L>(a.H, n, i));
        a.RV[i] = r.re.v[0];
        a.RV[n + i] = r.im.v[0];
    }
}

// z += dz (all or nothing), the convergence test of the corrector or of the end game
template <int L> __global__ void __launch_bounds__(HC_TB) k_g_update(GArgs a)
{
    __shared__ BlockShared sh;
    GStage &g = *a.g;
    if (!g_active(g)) return;
    const int n = a.S.n, tid = threadIdx.x;
    int ok = 1;
    double dzn = 0.0, zn = 0.0;
    for (int i = tid; i < n; i += HC_TB) {
        const C<L> d = ld_c<L>(a.DZ, n, i);
        const C<L> v = c_add(ld_c<L>(a.zh, n, i), d);
        if (!c_finite_lead(v)) ok = 0;
        dzn = fmax(dzn, sqrt(c_abs2_lead(d)));
        zn = fmax(zn, sqrt(c_abs2_lead(v)));
    }
    ok = block_and(ok, sh);
    dzn = block_max<HC_TB>(dzn, sh);
    zn = block_max<HC_TB>(zn, sh);
    if (ok)
        for (int i = tid; i < n; i += HC_TB) st_c<L>(a.zh, n, i, c_add(ld_c<L>(a.zh, n, i), ld_c<L>(a.DZ, n, i)));
    __syncthreads();
    if (tid == 0) {
        g.it++;
        g.dzn = dzn;
        g.zn = zn;
        if (!ok) {
            g.nst = HC_NONFINITE;
        } else {
            const bool end = a.st->phase == 2;
            const double eps = end ? a.o.eps_end : a.o.eps, epsx = end ? a.o.eps_end_x : a.o.eps_x;
            g.conv = (g.res <= eps) || (dzn <= epsx * (zn > 1.0 ? zn : 1.0));
        }
    }
}

template <int L> __global__ void __launch_bounds__(HC_TB) k_g_end(GArgs a)
{
    __shared__ BlockShared sh;
    PathState st = *a.st;
    const GStage g = *a.g;
    const int n = a.S.n, tid = threadIdx.x;
    if (st.phase == 1) {
        stage_finish<L, HC_TB>(a.o, st, sh, n, a.z, a.zp, a.zpp, a.zh, a.ZP, g.t1, g.h, g.it, g.nst, g.conv, g.res,
                        g.res_first, g.cond, a.log, a.log_cap, a.log0);
    } else if (st.phase == 2) {
        for (int q = tid; q < 2 * L * n; q += HC_TB) a.z[q] = a.zh[q];
        st.end_its += g.it;
        if (g.nst != HC_OK) {
            st.status = g.nst;
            st.res_end = g.res;
            st.phase = 3;
        } else if (g.conv || st.end_its >= a.o.end_it) {
            st.res_end = g.res;
            if (!g.conv && st.status == HC_OK) st.status = HC_NOCONV;
            st.phase = 3;
        }
    }
    __syncthreads();
    if (tid == 0) *a.st = st;
}

template <int L>
static int grid_capture(const GArgs &a, int max_it, int max_refine, cudaStream_t cs, cudaGraphExec_t *exec)
{
    const int mblocks = (a.S.nmon + HC_GMONO - 1) / HC_GMONO;
    const int eblocks = a.nlong + (a.S.npoly * (a.S.n + 1) - a.nlong + 31) / 32;
    // each column solve of the inverse from a shared-memory copy of the factors when they
    // fit (n <= 110)
    const size_t bsm = sizeof(double) * 2 * (size_t)a.S.n * a.S.n;
    const size_t vec4 = sizeof(double) * 4 * (size_t)a.S.n;
    const int b_smem = vec4 + bsm <= 200 * 1024;
    const size_t inv_bytes = vec4 + (b_smem ? bsm : 0);
    // the blocked LU's panel and the update kernel's copies in shared memory (at most
    // 82 KB for the tracker's n <= 256)
    const int n = a.S.n, nb0 = n < HC_GLU_NB ? n : HC_GLU_NB;
    auto panel_bytes = [&](int m, int nb) { return sizeof(double) * 2 * (size_t)nb * m; };
    auto upd_bytes = [&](int m, int nb) { return sizeof(double) * 2 * (size_t)m * (nb + HC_GUPD); };
    cudaError_t ea = cudaFuncSetAttribute(k_g_inverse<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_bytes);
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(k_g_panel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_bytes(n, nb0));
    if (ea == cudaSuccess)
        ea = cudaFuncSetAttribute(k_g_lu_update<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_bytes(n, nb0));
    if (ea != cudaSuccess) return hc_cuda_fail(ea, "whole-GPU engine shared memory");
    // the branch of the start-system terms: a second stream forked from and joined back
    // into the capturing stream
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    auto release = [&]() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
    };
    if (e != cudaSuccess) {
        release();
        return hc_cuda_fail(e, "whole-GPU engine: graph branch stream");
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        release();
        return hc_cuda_fail(e, "cudaStreamBeginCapture");
    }
    k_g_begin<L><<<1, HC_TB, 0, cs>>>(a);
    for (int it = 0; it < max_it; it++) {
        cudaEventRecord(fork, cs);
        cudaStreamWaitEvent(side, fork, 0);
        k_g_terms<L><<<a.S.n, 1, 0, side>>>(a);
        cudaEventRecord(join, side);
        k_g_powers<L><<<a.S.n, 1, 0, cs>>>(a);
        k_g_monomials<L><<<mblocks > 0 ? mblocks : 1, HC_GMONO, 0, cs>>>(a);
        k_g_chunks<L><<<(a.nchunks + HC_GCHUNK - 1) / HC_GCHUNK, HC_GCHUNK, 0, cs>>>(a);
        cudaStreamWaitEvent(cs, join, 0);
        k_g_entries<L><<<eblocks, 32, 0, cs>>>(a);
        k_g_lu_prep<L><<<1, HC_GLU, 0, cs>>>(a);
        for (int kb = 0; kb < n; kb += HC_GLU_NB) {
            const int m = n - kb, nb = m < HC_GLU_NB ? m : HC_GLU_NB, others = n - nb;
            k_g_panel<L><<<1, HC_GPANEL, panel_bytes(m, nb), cs>>>(a, kb);
            if (others > 0)
                k_g_lu_update<L><<<(others + HC_GUPD - 1) / HC_GUPD, 32 * HC_GUPD, upd_bytes(m, nb), cs>>>(a, kb);
        }
        k_g_inverse<L><<<a.S.n, HC_GINV, inv_bytes, cs>>>(a, b_smem);
        const int gblocks = (a.S.n + HC_GEMV_ROWS - 1) / HC_GEMV_ROWS;
        k_g_gemv<L><<<gblocks, 8 * HC_GEMV_ROWS, 0, cs>>>(a, 1);
        k_g_apply<L><<<1, HC_GAPPLY, 0, cs>>>(a, 1);
        for (int r = 0; r < max_refine; r++) {
            k_g_refine_rows<L><<<a.S.n, HC_GREF, 0, cs>>>(a);
            k_g_gemv<L><<<gblocks, 8 * HC_GEMV_ROWS, 0, cs>>>(a, 0);
            k_g_apply<L><<<1, HC_GAPPLY, 0, cs>>>(a, 0);
        }
        k_g_update<L><<<1, HC_TB, 0, cs>>>(a);
    }
    k_g_end<L><<<1, HC_TB, 0, cs>>>(a);
    e = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    release();
    if (e != cudaSuccess) return hc_cuda_fail(e, "capturing the stage graph");
    return HC_SUCCESS;
}

}  // namespace hc

using namespace hc;

void hc_stats_of(const PathState &q, hc_path_stats &r);

// One path per call to this function: workspace, graph, replays, statistics.  With a
// state (hc_track_resume) the path starts from it, the previous points are the caller's
// hist (x0 == x1 is the current point), and at most max_stages stages run.  An entry's
// contribution list is summed in chunks of `chunk` (the tracker tiles' grid_chunk).
int hc_track_grid_path(const hc_system *s, const double *x0, double *x1, double *hist,
                       hc_path_state *state, int max_stages, const hc_track_opts *o,
                       hc_path_stats *stats, hc_step_record *log, int log_cap, int chunk, cudaStream_t st)
{
    const int n = s->n, L = s->prec;
    const size_t vec = sizeof(double) * 2 * L * (size_t)n;
    const size_t vplane = (size_t)s->nvar + s->nmon;
    size_t off = 0;
    auto put = [&](size_t b) { size_t at = off; off = hc_align256(off + b); return at; };
    const size_t o_st = put(sizeof(PathState)), o_g = put(sizeof(GStage));
    const size_t o_zp = put(vec), o_zpp = put(vec), o_zh = put(vec), o_ZP = put(vec);
    const size_t o_pw = put(vec * (s->max_exp > 2 ? s->max_exp - 2 : 1));
    const size_t o_v = put(sizeof(double) * 2 * L * (vplane > 0 ? vplane : 1));
    const size_t o_hs = put(3 * vec), o_h = put(vec), o_jh = put(vec * n), o_b = put(sizeof(double) * 2 * (size_t)n * n),
                 o_inv = put(sizeof(double) * 2 * (size_t)n * n), o_d = put(sizeof(double) * 2 * (size_t)n),
                 o_dnb = put(sizeof(double) * ((size_t)n + HC_GEMV_ROWS - 1) / HC_GEMV_ROWS);
    const size_t o_rv = put(sizeof(double) * 2 * (size_t)n), o_dz = put(vec), o_piv = put(sizeof(int32_t) * n),
                 o_pstep = put(sizeof(int32_t) * n);
    // chunks of the entries' contribution lists (from the transpose table's offsets)
    const int ne = s->npoly * (n + 1);
    std::vector<int32_t> tptr((size_t)ne + 1), cbeg, cend, eptr((size_t)ne + 1, 0);
    HC_CUDA_TRY(cudaMemcpy(tptr.data(), s->dev.tptr, sizeof(int32_t) * (ne + 1), cudaMemcpyDeviceToHost));
    for (int e = 0; e < ne; e++) {
        int r = tptr[e];
        do {
            const int r1 = r + chunk < tptr[e + 1] ? r + chunk : tptr[e + 1];
            cbeg.push_back(r);
            cend.push_back(r1);
            r = r1;
        } while (r < tptr[e + 1]);
        eptr[e + 1] = (int32_t)cbeg.size();
    }
    const int nchunks = (int)cbeg.size();
    // the order of k_g_entries: the long entries (one warp each), then the others in the
    // system's longest-first order (one thread each)
    std::vector<int32_t> eperm((size_t)ne), eord;
    HC_CUDA_TRY(cudaMemcpy(eperm.data(), s->dev.eperm, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost));
    for (int e = 0; e < ne; e++)
        if (eptr[e + 1] - eptr[e] >= HC_GLONG) eord.push_back(e);
    const int nlong = (int)eord.size();
    for (int q = 0; q < ne; q++)
        if (eptr[eperm[q] + 1] - eptr[eperm[q]] < HC_GLONG) eord.push_back(eperm[q]);
    const size_t o_cb = put(sizeof(int32_t) * nchunks), o_ce = put(sizeof(int32_t) * nchunks),
                 o_ep = put(sizeof(int32_t) * (ne + 1)), o_eo = put(sizeof(int32_t) * ne),
                 o_p = put(sizeof(double) * 2 * L * (size_t)nchunks);
    void *ws = nullptr;
    HC_CUDA_TRY(cudaMalloc(&ws, off));
    char *b = (char *)ws;
    GArgs a;
    a.S = s->dev;
    a.st = (PathState *)(b + o_st);
    a.g = (GStage *)(b + o_g);
    a.x0 = x0;
    a.z = x1;
    a.zp = hist ? hist : (double *)(b + o_zp);
    a.zpp = hist ? hist + 2 * L * (size_t)n : (double *)(b + o_zpp);
    a.zh = (double *)(b + o_zh);
    a.ZP = (double *)(b + o_ZP);
    a.PW = (double *)(b + o_pw);
    a.V = (double *)(b + o_v);
    a.HS = (double *)(b + o_hs);
    a.H = (double *)(b + o_h);
    a.JH = (double *)(b + o_jh);
    a.B = (double *)(b + o_b);
    a.INV = (double *)(b + o_inv);
    a.D = (double *)(b + o_d);
    a.DNB = (double *)(b + o_dnb);
    a.RV = (double *)(b + o_rv);
    a.DZ = (double *)(b + o_dz);
    a.PIV = (int32_t *)(b + o_piv);
    a.PSTEP = (int32_t *)(b + o_pstep);
    a.cbeg = (const int32_t *)(b + o_cb);
    a.cend = (const int32_t *)(b + o_ce);
    a.eptr = (const int32_t *)(b + o_ep);
    a.eord = (const int32_t *)(b + o_eo);
    a.nlong = nlong;
    a.P = (double *)(b + o_p);
    a.nchunks = nchunks;
    a.o = *o;
    a.log = log;
    a.log_cap = log_cap;
    const long long n0 = state && state->phase != 0 ? state->n_corr : 0;
    a.log0 = n0;
    cudaStream_t cs = nullptr;
    cudaEvent_t ready = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = HC_SUCCESS;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, off, st);
    if (e == cudaSuccess && state) e = cudaMemcpyAsync(a.st, state, sizeof(PathState), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_cb, cbeg.data(), sizeof(int32_t) * nchunks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_ce, cend.data(), sizeof(int32_t) * nchunks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_ep, eptr.data(), sizeof(int32_t) * (ne + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_eo, eord.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(ready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
    if (e != cudaSuccess) rc = hc_cuda_fail(e, "grid tracker set-up");
    if (!rc) {
        if (L == 1) rc = grid_capture<1>(a, o->max_it, o->max_refine, cs, &exec);
        else if (L == 2) rc = grid_capture<2>(a, o->max_it, o->max_refine, cs, &exec);
        else rc = grid_capture<4>(a, o->max_it, o->max_refine, cs, &exec);
    }
    PathState hs;
    memset(&hs, 0, sizeof hs);
    if (state) hs = *state;
    // every replay is one corrector stage, or end-game iterations; the path ends (or spends
    // this call's stages) within min(max_steps, max_stages) stages and end_it / max_it + 1
    // end-game replays
    const long long cap = o->max_steps < max_stages ? o->max_steps : max_stages;
    const long long limit = cap + o->end_it + 2;
    bool spent = hs.phase == 3;
    for (long long r = 0; !rc && !spent && r < limit; r++) {
        e = cudaGraphLaunch(exec, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, a.st, sizeof hs, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) rc = hc_cuda_fail(e, "stage graph replay");
        spent = hs.phase == 3 || (hs.phase == 1 && hs.n_corr - n0 >= max_stages);
    }
    if (!rc && !spent) rc = hc_fail(HC_ETIMEOUT, "large path unfinished after the replay limit");
    if (exec) cudaGraphExecDestroy(exec);
    if (ready) {
        cudaEventRecord(ready, cs);
        cudaStreamWaitEvent(st, ready, 0);
        cudaEventDestroy(ready);
    }
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    cudaFree(ws);
    if (rc) return rc;
    hc_stats_of(hs, *stats);
    if (state) *state = hs;
    return HC_SUCCESS;
}
