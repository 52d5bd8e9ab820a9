// hc_eval.cu -- hc_eval_jac: values and full Jacobians of the system (or the homotopy)
// at many points, one lane per point (Alg. 4.1 Monomial_Evaluation + Coefficient_Product
// with the scheme of Sec. 6).
#include "hc_eval.cuh"

namespace hc {

// x_j^e, e = 2 .. max_exp-1, by repeated multiplication: one thread per (j, p).
template <int L>
__global__ void __launch_bounds__(256) k_powers(int n, int npts, int max_exp,
                                                const double *__restrict__ X, double *__restrict__ PW)
{
    const size_t xplane = (size_t)n * npts;
    for (size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x; tid < xplane;
         tid += (size_t)gridDim.x * blockDim.x) {
        const C<L> x = ld_c<L>(X, xplane, tid);
        C<L> v = x;
        for (int e = 2; e < max_exp; e++) {
            v = c_mul(v, x);
            st_c<L>(PW + (size_t)(e - 2) * 2 * L * xplane, xplane, tid, v);
        }
    }
}

template <int L>
void launch_powers(int grid, int n, int npts, int max_exp, const double *X, double *PW, cudaStream_t st)
{
    k_powers<L><<<grid, 256, 0, st>>>(n, npts, max_exp, X, PW);
}
template void launch_powers<1>(int, int, int, int, const double *, double *, cudaStream_t);
template void launch_powers<2>(int, int, int, int, const double *, double *, cudaStream_t);
template void launch_powers<4>(int, int, int, int, const double *, double *, cudaStream_t);

// Persistent warps over tasks (32-point tile, group of rows); the row groups of one tile
// are consecutive tasks, so the warps of a block share their points' data in L1.  In
// quad double the register budget is that of four 128-thread blocks per SM (128
// registers; 40 bytes of spills): the warps' FP64 chains need the fourth block's warps
// to hide their latency.
template <int L, bool JAC>
__global__ void __launch_bounds__(128, L == 4 ? 4 : 1) k_eval_pts(DevSys S, int npts, double t,
                                                  const double *__restrict__ X,
                                                  const double *__restrict__ PW,
                                                  double *__restrict__ F, double *__restrict__ J,
                                                  int rows_per_task)
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
        const int r0 = grp * rows_per_task;
        const int r1 = min(r0 + rows_per_task, S.npoly);
        eval_rows_point<L, JAC>(S, V, live, t, gs, F, J, r0, r1);
    }
}

template <int L>
int launch_eval(const DevSys &S, int npts, double t, const double *X, double *PW, double *F,
                double *J, const EvalTiles &tiles, cudaStream_t st)
{
    const int sms = hc_num_sms();
    if (S.max_exp > 2) {
        const size_t work = (size_t)S.n * npts;
        size_t g = (work + 255) / 256;
        if (g > (size_t)sms * 8) g = (size_t)sms * 8;
        const int grid = (int)g;
        k_powers<L><<<grid, 256, 0, st>>>(S.n, npts, S.max_exp, X, PW);
    }
    const int ntiles = (npts + 31) / 32;
    int rpt = tiles.rows_per_task;
    if (rpt <= 0) {
        // about 16 tasks per SM sub-partition, so the static task split is balanced
        const long long want = (long long)sms * 4 * 16;
        long long groups = (want + ntiles - 1) / ntiles;
        if (groups < 1) groups = 1;
        if (groups > S.npoly) groups = S.npoly;
        rpt = (int)((S.npoly + groups - 1) / groups);
    }
    const int ngroups = (S.npoly + rpt - 1) / rpt;
    const long long tasks = (long long)ntiles * ngroups;
    const int wpb = 4;
    int occ = 1;
    if (J)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval_pts<L, true>, 32 * wpb, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_eval_pts<L, false>, 32 * wpb, 0);
    if (occ < 1) occ = 1;
    // blocks beyond residency would start late and unbalance the static task split
    int bps = tiles.blocks_per_sm > 0 ? tiles.blocks_per_sm : 4;
    if (bps > occ) bps = occ;
    long long grid = (long long)sms * bps;
    const long long need = (tasks + wpb - 1) / wpb;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    hc_prof_mark(st, true);
    if (J)
        k_eval_pts<L, true><<<(int)grid, 32 * wpb, 0, st>>>(S, npts, t, X, PW, F, J, rpt);
    else
        k_eval_pts<L, false><<<(int)grid, 32 * wpb, 0, st>>>(S, npts, t, X, PW, F, J, rpt);
    hc_prof_mark(st, false);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_eval_pts launch");
    return HC_SUCCESS;
}

template int launch_eval<1>(const DevSys &, int, double, const double *, double *, double *, double *, const EvalTiles &, cudaStream_t);
template int launch_eval<2>(const DevSys &, int, double, const double *, double *, double *, double *, const EvalTiles &, cudaStream_t);
template int launch_eval<4>(const DevSys &, int, double, const double *, double *, double *, double *, const EvalTiles &, cudaStream_t);

}  // namespace hc

using namespace hc;

size_t hc_pw_bytes(const hc_system *s, int npts)
{
    if (s->max_exp <= 2) return 0;
    return hc_align256(sizeof(double) * (size_t)(s->max_exp - 2) * 2 * s->prec * s->n * (size_t)npts);
}

int hc_check_eval_args(const hc_system *s, int npts, double t)
{
    if (!s) return hc_fail(HC_EINVAL, "sys is NULL");
    if (npts < 0) return hc_fail(HC_EINVAL, "npts = %d < 0", npts);
    if ((long long)npts * s->n > (1LL << 40)) return hc_fail(HC_EINVAL, "npts too large");
    if (!(t == t)) return hc_fail(HC_EINVAL, "t is NaN");
    if (t > 1e300) return hc_fail(HC_EINVAL, "t not finite");
    if (t >= 0.0 && s->npoly != s->n) return hc_fail(HC_EINVAL, "homotopy needs npoly == n");
    if (t >= 0.0 && s->min_deg < 1) return hc_fail(HC_EINVAL, "homotopy needs every degree >= 1");
    for (int i = 0; i < s->npoly; i++)
        for (int m = s->h_mon_ptr[i]; m < s->h_mon_ptr[i + 1]; m++)
            if (s->h_var_ptr[m + 1] - s->h_var_ptr[m] > HC_KLOCAL)
                return hc_fail(HC_EINVAL, "monomial with more than %d variables", HC_KLOCAL);
    return HC_SUCCESS;
}

int hc_eval_dispatch(hc_system *s, int npts, double t, const double *x, double *pw, double *f,
                     double *J, double *part, const EvalTiles &tiles, cudaStream_t st)
{
    if (s->eval_shared) {
        switch (s->prec) {
        case 1: return launch_eval_shared<1>(s, npts, t, x, pw, f, J, part, st);
        case 2: return launch_eval_shared<2>(s, npts, t, x, pw, f, J, part, st);
        case 4: return launch_eval_shared<4>(s, npts, t, x, pw, f, J, part, st);
        }
    }
    switch (s->prec) {
    case 1: return launch_eval<1>(s->dev, npts, t, x, pw, f, J, tiles, st);
    case 2: return launch_eval<2>(s->dev, npts, t, x, pw, f, J, tiles, st);
    case 4: return launch_eval<4>(s->dev, npts, t, x, pw, f, J, tiles, st);
    }
    return hc_fail(HC_EINVAL, "bad precision");
}

static EvalTiles g_eval_tiles;  // set by hc_set_tiles; zero = automatic
EvalTiles &hc_eval_tiles() { return g_eval_tiles; }

extern "C" int hc_eval_jac(hc_system *s, int npts, double t, const double *x, double *f, double *J,
                           void *stream)
{
    int rc = hc_check_eval_args(s, npts, t);
    if (rc) return rc;
    if (npts == 0) return HC_SUCCESS;
    if (!x || !f) return hc_fail(HC_EINVAL, "x or f is NULL");
    void *ws = NULL;
    const size_t pwb = hc_pw_bytes(s, npts), partb = hc_shared_part_bytes(s, npts, J != NULL);
    rc = hc_workspace(s, pwb + partb, &ws);
    if (rc) return rc;
    double *part = partb ? (double *)((char *)ws + pwb) : NULL;
    return hc_eval_dispatch(s, npts, t, x, (double *)ws, f, J, part, g_eval_tiles, (cudaStream_t)stream);
}

extern "C" int hc_set_tiles(int rows_per_task, int blocks_per_sm)
{
    if (rows_per_task < 0 || blocks_per_sm < 0 || blocks_per_sm > 32)
        return hc_fail(HC_EINVAL, "bad tile parameters");
    g_eval_tiles.rows_per_task = rows_per_task;
    g_eval_tiles.blocks_per_sm = blocks_per_sm;
    return HC_SUCCESS;
}
