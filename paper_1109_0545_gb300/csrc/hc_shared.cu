// hc_shared.cu -- evaluation with shared monomials, one lane per point: for systems whose
// polynomials repeat one another's monomials (a common support, as in the experiment of
// Sec. 4 that reports the cost split of Table 1), each distinct monomial and its partial
// derivatives are evaluated once per point (the scheme of Sec. 6 with coefficient 1), then
// every term that uses it adds its coefficient times these values to its polynomial and
// Jacobian row (Coefficient_Product of Alg. 4.1, done per term).
#include "hc_eval.cuh"

namespace hc {

// Rows r0..r1-1 of f (and J) at point p, from the distinct monomials u0..u1-1: each is
// evaluated, and the terms of rows r0..r1-1 that use it are applied (the uses of a
// monomial are sorted by row, so they form one range, found by bisection).  With
// `consts`, the rows' constant terms are added too.  f and J are running sums in the
// output buffers (c_acc), started at zero here; the caller renormalises them
// (shared_rows_finish).
template <int L, bool JAC>
__device__ void eval_shared_point(const DevSys &S, const PointView<L> &V, bool live, double *__restrict__ F,
                                  double *__restrict__ J, int r0, int r1, int u0, int u1, bool consts)
{
    const int n = S.n, npts = V.npts, p = V.p;
    const size_t fplane = (size_t)S.npoly * npts;
    const size_t jplane = (size_t)S.npoly * n * npts;
    // constant terms, zero Jacobian rows
    if (live)
        for (int i = r0; i < r1; i++) {
            C<L> fi = c_zero<L>();
            if (consts)
                for (int q = __ldg(S.cptr + i); q < __ldg(S.cptr + i + 1); q++)
                    fi = c_acc(fi, ld_c<L>(S.coef + (size_t)__ldg(S.cterm + q) * 2 * L, 1, 0));
            st_c<L>(F, fplane, (size_t)i * npts + p, fi);
            if (JAC)
                for (int j = 0; j < n; j++) st_c<L>(J, jplane, ((size_t)i * n + j) * npts + p, c_zero<L>());
        }
    C<L> d[HC_KLOCAL];
    for (int u = u0; u < u1; u++) {
        const int q0 = __ldg(S.uvar_ptr + u), k = __ldg(S.uvar_ptr + u + 1) - q0;
        // common factor prod x_j^(a_j - 1) over a_j >= 2; `one` while it is exactly 1
        C<L> cf = c_from<L>(1.0, 0.0);
        bool one = true;
        for (int j = 0; j < k; j++) {
            const int pk = __ldg(S.uvar_pack + q0 + j), e = pk >> 16;
            if (e >= 2) {
                cf = one ? V.pw(pk & 0xffff, e - 1) : c_mul_nn(cf, V.pw(pk & 0xffff, e - 1));
                one = false;
            }
        }
        // prefix products d_j = cf x_{i1} ... x_{i(j-1)}, the value, the backward sweep
        d[0] = cf;
        for (int j = 1; j < k; j++) {
            const C<L> xj = V.x(__ldg(S.uvar_pack + q0 + j - 1) & 0xffff);
            d[j] = (j == 1 && one) ? xj : c_mul_nn(d[j - 1], xj);
        }
        const int pkl = __ldg(S.uvar_pack + q0 + k - 1);
        const C<L> xl = V.x(pkl & 0xffff);
        const C<L> value = (k == 1 && one) ? xl : c_mul_nn(d[k - 1], xl);
        if (JAC) {
            d[k - 1] = c_scale_int(d[k - 1], pkl >> 16);
            C<L> suf = xl;
            for (int j = k - 2; j >= 0; j--) {
                const int pk = __ldg(S.uvar_pack + q0 + j);
                d[j] = c_scale_int((j == 0 && one) ? suf : c_mul_nn(d[j], suf), pk >> 16);
                if (j > 0) suf = c_mul_nn(suf, V.x(pk & 0xffff));
            }
        }
        // the uses in rows r0..r1-1: f_i += c value, J_{i,ij} += c a_j x^(a - e_j)
        int lo = __ldg(S.uuse_ptr + u), hi = __ldg(S.uuse_ptr + u + 1);
        for (int a = lo, b = hi; a < b;) {
            const int mid = (a + b) >> 1;
            if (__ldg(S.term_row + __ldg(S.uuse + mid)) < r0) a = lo = mid + 1;
            else b = mid;
        }
        for (int r = lo; r < hi; r++) {
            const int m = __ldg(S.uuse + r), i = __ldg(S.term_row + m);
            if (i >= r1) break;
            const C<L> c = ld_c<L>(S.coef + (size_t)m * 2 * L, 1, 0);
            if (!live) continue;
            const size_t fo = (size_t)i * npts + p;
            st_c<L>(F, fplane, fo, c_acc(ld_c<L>(F, fplane, fo), c_mul_nn(c, value)));
            if (JAC) {
                // four entries at a time: their loads are issued together (the entries of
                // one term are distinct, but the compiler cannot know it)
                const size_t rowo = (size_t)i * n;
                for (int j0 = 0; j0 < k; j0 += 4) {
                    C<L> acc[4];
                    size_t o[4];
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (j0 + q < k) {
                            o[q] = (rowo + (__ldg(S.uvar_pack + q0 + j0 + q) & 0xffff)) * npts + p;
                            acc[q] = ld_c<L>(J, jplane, o[q]);
                        }
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (j0 + q < k) st_c<L>(J, jplane, o[q], c_acc(acc[q], c_mul_nn(c, d[j0 + q])));
                }
            }
        }
    }
}

// Rows r0..r1-1 of f (and J) at point p after their sums: the homotopy (t >= 0, as in
// eval_rows_point), or for f alone (t < 0) the running sums renormalised
template <int L, bool JAC>
__device__ void shared_rows_finish(const DevSys &S, const PointView<L> &V, bool live, double t, const C<L> &gs,
                                   double *__restrict__ F, double *__restrict__ J, int r0, int r1)
{
    const int n = S.n, npts = V.npts, p = V.p;
    const size_t fplane = (size_t)S.npoly * npts;
    const size_t jplane = (size_t)S.npoly * n * npts;
    if (t >= 0.0 && live) {
        // homotopy assembly, as in eval_rows_point
        for (int i = r0; i < r1; i++) {
            const int dg = __ldg(S.deg + i);
            const C<L> xi = V.x(i);
            const C<L> xd1 = c_pow(xi, dg - 1);
            C<L> g = c_mul(xd1, xi);
            g.re = r_sub(g.re, r_from<L>(1.0));
            const size_t fo = (size_t)i * npts + p;
            st_c<L>(F, fplane, fo, c_add(c_mul(gs, g), c_mul_d(c_settle(ld_c<L>(F, fplane, fo)), t)));
            if (JAC)
                for (int j = 0; j < n; j++) {
                    const size_t o = ((size_t)i * n + j) * npts + p;
                    C<L> v = c_mul_d(c_settle(ld_c<L>(J, jplane, o)), t);
                    if (j == i) v = c_add(v, c_mul(gs, c_scale_int(xd1, dg)));
                    st_c<L>(J, jplane, o, v);
                }
        }
    } else if (L == 2 && live) {
        // f (t < 0): the running sums renormalised
        for (int i = r0; i < r1; i++) {
            const size_t fo = (size_t)i * npts + p;
            st_c<L>(F, fplane, fo, c_settle(ld_c<L>(F, fplane, fo)));
            if (JAC)
                for (int j = 0; j < n; j++) {
                    const size_t o = ((size_t)i * n + j) * npts + p;
                    st_c<L>(J, jplane, o, c_settle(ld_c<L>(J, jplane, o)));
                }
        }
    }
}

// Two task decompositions (a task is one warp, one warp per block, so that the block
// scheduler deals the warps out to the SMs one at a time: with four-warp blocks, 320
// blocks on 152 SMs put three blocks on some SMs and two on the rest, and the FP64 pipes
// of the latter idled for a third of the time):
//   - enough 32-point tiles: a task is a tile and a group of rows, every distinct monomial;
//   - few tiles (the SMs want about 1,216 warps): a task is a tile and a group of distinct
//     monomials (cut by their FP64 cost), every row, into partial sums of its own; a
//     second kernel adds the groups' partial sums in group order and forms the homotopy.
//     Cutting the rows instead would evaluate every monomial once per row group (five
//     groups at 8,192 points: a quarter of the work again).
#define HC_SHARED_TB 32
#define HC_SHARED_WANT_WARPS_PER_SM 8
#define HC_SHARED_MAX_GROUPS 64

template <int L, bool JAC>
__global__ void __launch_bounds__(HC_SHARED_TB) k_eval_shared(DevSys S, int npts, double t, const double *__restrict__ X,
                                                     const double *__restrict__ PW, double *__restrict__ F,
                                                     double *__restrict__ J, int rows_per_task)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ntiles = (npts + 31) >> 5;
    const int ngroups = (S.npoly + rows_per_task - 1) / rows_per_task;
    const C<L> gs = gamma_one_minus_t<L>(S.gre, S.gim, t < 0.0 ? 0.0 : t);
    for (int task = warp; task < ntiles * ngroups; task += nwarps) {
        const int tile = task / ngroups, grp = task - tile * ngroups;
        const int p = tile * 32 + lane;
        const bool live = p < npts;
        PointView<L> V{X, PW, (size_t)S.n * npts, npts, live ? p : npts - 1};
        const int r0 = grp * rows_per_task, r1 = min(r0 + rows_per_task, S.npoly);
        eval_shared_point<L, JAC>(S, V, live, F, J, r0, r1, 0, S.nuniq, true);
        shared_rows_finish<L, JAC>(S, V, live, t, gs, F, J, r0, r1);
    }
}

// the first distinct monomial of group g of G: the first whose cost prefix reaches g/G of
// the total
__device__ __forceinline__ int shared_group_start(const DevSys &S, int g, int G)
{
    if (g <= 0) return 0;
    if (g >= G) return S.nuniq;
    const double cut = __ldg(S.ucost + S.nuniq) * g / G;
    int lo = 0, hi = S.nuniq;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(S.ucost + mid + 1) < cut) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// tasks (tile, monomial group g): partial sums PF[g] (, PJ[g]) over every row, each laid
// out as F (, J); group 0 takes the constant terms
template <int L, bool JAC>
__global__ void __launch_bounds__(HC_SHARED_TB) k_eval_shared_part(DevSys S, int npts, const double *__restrict__ X,
                                                          const double *__restrict__ PW, double *__restrict__ PF,
                                                          double *__restrict__ PJ, int G)
{
    const int lane = threadIdx.x & 31;
    const int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int ntiles = (npts + 31) >> 5;
    if (task >= ntiles * G) return;
    const int tile = task / G, g = task - tile * G;
    const int p = tile * 32 + lane;
    const bool live = p < npts;
    PointView<L> V{X, PW, (size_t)S.n * npts, npts, live ? p : npts - 1};
    const size_t fs = (size_t)2 * L * S.npoly * npts, js = (size_t)2 * L * S.npoly * S.n * npts;
    double *F = PF + g * fs, *J = JAC ? PJ + g * js : nullptr;
    eval_shared_point<L, JAC>(S, V, live, F, J, 0, S.npoly, shared_group_start(S, g, G),
                              shared_group_start(S, g + 1, G), g == 0);
    shared_rows_finish<L, JAC>(S, V, live, -1.0, c_zero<L>(), F, J, 0, S.npoly);  // renormalised
}

// one thread per (point, row): the groups' partial sums added in group order, then the
// homotopy (or, for f alone, the sums as they are)
template <int L, bool JAC>
__global__ void __launch_bounds__(128) k_eval_shared_sum(DevSys S, int npts, double t, const double *__restrict__ X,
                                                        const double *__restrict__ PW, const double *__restrict__ PF,
                                                        const double *__restrict__ PJ, int G, double *__restrict__ F,
                                                        double *__restrict__ J)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)npts * S.npoly) return;
    const int i = (int)(q / npts), p = (int)(q - (long long)i * npts);
    const int n = S.n;
    const size_t fplane = (size_t)S.npoly * npts, jplane = (size_t)S.npoly * n * npts;
    const size_t fs = 2 * L * fplane, js = 2 * L * jplane;
    const size_t fo = (size_t)i * npts + p;
    C<L> fi = ld_c<L>(PF, fplane, fo);
    for (int g = 1; g < G; g++) fi = c_add(fi, ld_c<L>(PF + g * fs, fplane, fo));
    st_c<L>(F, fplane, fo, fi);
    if (JAC)
        for (int j = 0; j < n; j++) {
            const size_t o = ((size_t)i * n + j) * npts + p;
            C<L> v = ld_c<L>(PJ, jplane, o);
            for (int g = 1; g < G; g++) v = c_add(v, ld_c<L>(PJ + g * js, jplane, o));
            st_c<L>(J, jplane, o, v);
        }
    if (t >= 0.0) {
        PointView<L> V{X, PW, (size_t)n * npts, npts, p};
        const C<L> gs = gamma_one_minus_t<L>(S.gre, S.gim, t);
        shared_rows_finish<L, JAC>(S, V, true, t, gs, F, J, i, i + 1);
    }
}

}  // namespace hc

using namespace hc;

// Monomial groups of the shared scheme for npts points: 1 (row groups, no partial sums)
// when the tiles alone give the SMs enough warps
static int shared_monomial_groups(const hc_system *s, int npts)
{
    const long long want = (long long)hc_num_sms() * HC_SHARED_WANT_WARPS_PER_SM;
    const long long ntiles = (npts + 31) / 32;
    if (ntiles <= 0 || ntiles >= want || s->dev.nuniq < 2) return 1;
    long long G = (want + ntiles - 1) / ntiles;
    if (G > s->dev.nuniq) G = s->dev.nuniq;
    if (G > HC_SHARED_MAX_GROUPS) G = HC_SHARED_MAX_GROUPS;
    return (int)G;
}

size_t hc_shared_part_bytes(const hc_system *s, int npts, bool jac)
{
    if (!s->eval_shared) return 0;
    const int G = shared_monomial_groups(s, npts);
    if (G <= 1) return 0;
    const size_t rows = (size_t)s->npoly * (jac ? 1 + s->n : 1);
    return hc_align256(sizeof(double) * G * 2 * s->prec * rows * npts);
}

namespace hc {

template <int L>
int launch_eval_shared(const hc_system *s, int npts, double t, const double *X, double *PW, double *F, double *J,
                       double *part, cudaStream_t st)
{
    const DevSys &S = s->dev;
    const int sms = hc_num_sms();
    if (S.max_exp > 2) {
        const size_t work = (size_t)S.n * npts;
        size_t g = (work + 255) / 256;
        if (g > (size_t)sms * 8) g = (size_t)sms * 8;
        launch_powers<L>((int)g, S.n, npts, S.max_exp, X, PW, st);
    }
    const int ntiles = (npts + 31) / 32;
    const int G = part ? shared_monomial_groups(s, npts) : 1;
    hc_prof_mark(st, true);
    if (G > 1) {
        // tiles x monomial groups, then the sums over the groups
        const size_t fs = (size_t)2 * L * S.npoly * npts;
        double *PF = part, *PJ = J ? part + G * fs : nullptr;
        const long long tasks = (long long)ntiles * G;
        const int grid = (int)tasks;
        if (J) {
            k_eval_shared_part<L, true><<<grid, HC_SHARED_TB, 0, st>>>(S, npts, X, PW, PF, PJ, G);
        } else {
            k_eval_shared_part<L, false><<<grid, HC_SHARED_TB, 0, st>>>(S, npts, X, PW, PF, PJ, G);
        }
        const long long cells = (long long)npts * S.npoly;
        const int sgrid = (int)((cells + 127) / 128);
        if (J)
            k_eval_shared_sum<L, true><<<sgrid, 128, 0, st>>>(S, npts, t, X, PW, PF, PJ, G, F, J);
        else
            k_eval_shared_sum<L, false><<<sgrid, 128, 0, st>>>(S, npts, t, X, PW, PF, PJ, G, F, J);
    } else {
        int occ = 1;
        if (J)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval_shared<L, true>, HC_SHARED_TB, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval_shared<L, false>, HC_SHARED_TB, 0);
        if (occ < 1) occ = 1;
        // row groups: the fewest that give two warps' tasks on every SM sub-partition (each group
        // evaluates every distinct monomial again; at 8,192 points 10 groups ran 2,560 tasks on
        // 2,432 resident warps, a second round for 128 of them)
        const long long want = (long long)sms * HC_SHARED_WANT_WARPS_PER_SM;
        long long groups = (want + ntiles - 1) / ntiles;
        if (groups < 1) groups = 1;
        if (groups > S.npoly) groups = S.npoly;
        const int rpt = (int)((S.npoly + groups - 1) / groups);
        const long long tasks = (long long)ntiles * ((S.npoly + rpt - 1) / rpt);
        long long grid = (long long)sms * occ;
        if (grid > tasks) grid = tasks;
        if (grid < 1) grid = 1;
        if (J)
            k_eval_shared<L, true><<<(int)grid, HC_SHARED_TB, 0, st>>>(S, npts, t, X, PW, F, J, rpt);
        else
            k_eval_shared<L, false><<<(int)grid, HC_SHARED_TB, 0, st>>>(S, npts, t, X, PW, F, J, rpt);
    }
    hc_prof_mark(st, false);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_eval_shared launch");
    return HC_SUCCESS;
}

template int launch_eval_shared<1>(const hc_system *, int, double, const double *, double *, double *, double *,
                                   double *, cudaStream_t);
template int launch_eval_shared<2>(const hc_system *, int, double, const double *, double *, double *, double *,
                                   double *, cudaStream_t);
template int launch_eval_shared<4>(const hc_system *, int, double, const double *, double *, double *, double *,
                                   double *, cudaStream_t);

}  // namespace hc
