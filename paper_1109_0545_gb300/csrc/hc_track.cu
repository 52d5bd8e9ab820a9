// hc_track.cu -- hc_track_path: the path tracker of Alg. 3.1 (predictor, Newton corrector
// of Alg. 4.1, step-size control, step back, stop criterion) for many paths of uneven
// dimension, each on its own system, one thread block per path.
//
// Two ways to run it:
//   HC_TRACK_PERSISTENT  one persistent kernel; each block takes paths from an atomic
//                        queue and tracks each to its end;
//   HC_TRACK_GRAPH       every launch advances each unfinished path by one
//                        predictor-corrector stage; the host replays a CUDA graph of
//                        several such launches until no path is left.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "track.cuh"

namespace hc {

struct SlotLayout {
    size_t pw, v, hs, ht, h, jh, b, dz, zp, stride;
};

struct TrackArgs {
    const DevSys *sys;        // [npaths]
    const long long *xoff;    // [npaths] offset (doubles) of path p in x0/x1
    const double *x0;
    double *x1;
    double *hist;             // per path at 3 xoff[p]: previous accepted point, second
                              // previous, tangent (each 2 L n doubles)
    double *zh;               // per path at xoff[p]: the predicted, then corrected point
    PathState *st;
    const long long *n0;      // [npaths] corrector stages done before this call (log
                              // offset and stage budget of the call)
    hc_track_opts o;
    char *slots;
    SlotLayout lay;
    int *queue;
    int *active;              // paths that may still advance in this call
    const int *order;         // [npaths] paths in the order they are taken: largest
                              // evaluation cost first, so the last ones to start are short
    hc_step_record *log;
    int log_cap;
    int npaths;
    int nmax;                 // largest n of the batch
    int b_smem;               // the FP64 factors in shared memory (else in the slot)
    int max_stages;           // corrector stages per path in this call
};

// Dynamic shared memory of a tracking block, in doubles: Y, RV [2][nmax] each, PIV
// [nmax] ints, then (b_smem) the FP64 factors B [2][nmax][nmax].
__host__ __device__ __forceinline__ size_t track_smem_doubles(int nmax, int b_smem)
{
    return 4 * (size_t)nmax + (size_t)(nmax + 1) / 2 + (b_smem ? 2 * (size_t)nmax * nmax : 0);
}

template <int L> __device__ __forceinline__ Slot<L> slot_of(const TrackArgs &a, int b, double *dsm)
{
    char *base = a.slots + (size_t)b * a.lay.stride;
    Slot<L> w;
    w.PW = (double *)(base + a.lay.pw);
    w.V = (double *)(base + a.lay.v);
    w.HS = (double *)(base + a.lay.hs);
    w.HT = a.o.predictor == HC_PRED_TANGENT ? (double *)(base + a.lay.ht) : nullptr;
    w.H = (double *)(base + a.lay.h);
    w.JH = (double *)(base + a.lay.jh);
    w.DZ = (double *)(base + a.lay.dz);
    w.ZP = (double *)(base + a.lay.zp);
    w.Y = dsm;
    w.RV = dsm + 2 * a.nmax;
    w.PIV = (int32_t *)(dsm + 4 * a.nmax);
    w.B = a.b_smem ? dsm + 4 * (size_t)a.nmax + (a.nmax + 1) / 2 : (double *)(base + a.lay.b);
    return w;
}


//
// Advance path p by at most max_stages corrector stages (then its end game, once t = 1),
// within the call's budget of a.max_stages stages per path.
// Every thread keeps the same copy of the path's scalars: each decision is taken from
// values that block reductions broadcast, so all threads follow the same branch.
//
template <int L>
__device__ void path_run(const TrackArgs &a, int p, const Slot<L> &w, BlockShared &sh, int max_stages)
{
    const DevSys S = a.sys[p];
    const hc_track_opts &o = a.o;
    const int n = S.n, tid = threadIdx.x;
    double *z = a.x1 + a.xoff[p];
    double *zp = a.hist + 3 * a.xoff[p];
    double *zpp = zp + 2 * L * n;
    double *tv = zpp + 2 * L * n;  // [2][n] dx/dt at the last accepted point (tangent predictor)
    double *zh = a.zh + a.xoff[p];
    const bool tangent = o.predictor == HC_PRED_TANGENT;
    PathState st = a.st[p];
    const long long n0 = a.n0[p];
    // done, or this call's stages spent (the path was counted out of `active` then)
    if (st.phase == 3 || (st.phase == 1 && st.n_corr - n0 >= a.max_stages)) return;
    if (st.phase == 0) {
        for (int q = tid; q < 2 * L * n; q += HC_TB) z[q] = a.x0[a.xoff[p] + q];
        path_init(st, o, p);
        __syncthreads();
    }
    hc_step_record *log = a.log ? a.log + (size_t)p * a.log_cap : nullptr;
    int stages = 0;
    while (st.phase == 1 && stages < max_stages && st.n_corr - n0 < a.max_stages) {
        double t1, h;
        stage_predict<L>(o, st, n, z, zp, zpp, tv, zh, w.ZP, t1, h);
        // corrector: Alg. 4.1
        double res = 1.0, res_first = -1.0, cond = 0.0;
        int it = 0, nst = HC_OK, conv = 0;
        while (!conv && it < o.max_it) {
            const NewtonOut no = block_newton<L>(S, zh, t1, o.lu_mode, o.max_refine, w, sh);
            res = no.res;
            if (res_first < 0) res_first = res;
            it++;
            nst = no.status;
            cond = no.cond;
            if (nst != HC_OK) break;
            conv = (res <= o.eps) || (no.dzn <= o.eps_x * (no.zn > 1.0 ? no.zn : 1.0));
        }
        // tangent at the corrected point: dx/dt = -J^-1 dh/dt from the last iteration's
        // evaluation and FP64 factors, kept if the stage is accepted
        if (tangent && conv && nst == HC_OK) {
            if (tid < 32) warp_lu64_solve(n, w.B, w.PIV, w.HT, w.Y);
            __syncthreads();
        }
        const long long succ0 = st.n_succ;
        stage_finish<L>(o, st, sh, n, z, zp, zpp, zh, w.ZP, t1, h, it, nst, conv, res, res_first, cond,
                        log, a.log_cap, n0);
        if (tangent && st.n_succ > succ0) {
            for (int q = tid; q < 2 * n; q += HC_TB) tv[q] = -w.Y[q];
            __syncthreads();
        }
        stages++;
    }
    if (st.phase == 2) {
        // end game at t = 1: Newton on f until converged with the end tolerances
        double res = 1.0;
        int conv = 0;
        while (!conv && st.end_its < o.end_it) {
            const NewtonOut no = block_newton<L>(S, z, 1.0, o.lu_mode, o.max_refine, w, sh);
            st.end_its++;
            res = no.res;
            if (no.status != HC_OK) {
                st.status = no.status;
                break;
            }
            conv = (res <= o.eps_end) || (no.dzn <= o.eps_end_x * (no.zn > 1.0 ? no.zn : 1.0));
        }
        st.res_end = res;
        if (st.status == HC_OK && !conv) st.status = HC_NOCONV;
        st.phase = 3;
    }
    __syncthreads();
    if (tid == 0) {
        a.st[p] = st;
        if (st.phase == 3 || st.n_corr - n0 >= a.max_stages) atomicSub(a.active, 1);
    }
    __syncthreads();
}

template <int L>
__global__ void __launch_bounds__(HC_TB, L == 4 ? 3 : 4) k_track(TrackArgs a, int persistent)
{
    __shared__ BlockShared sh;
    __shared__ int s_p;
    extern __shared__ double dsm[];
    const Slot<L> w = slot_of<L>(a, blockIdx.x, dsm);
    if (persistent) {
        for (;;) {
            if (threadIdx.x == 0) s_p = atomicAdd(a.queue, 1);
            __syncthreads();
            const int q = s_p;
            __syncthreads();
            if (q >= a.npaths) break;
            path_run<L>(a, a.order[q], w, sh, 0x7fffffff);
        }
    } else {
        for (int q = blockIdx.x; q < a.npaths; q += gridDim.x) path_run<L>(a, a.order[q], w, sh, 1);
    }
}

}  // namespace hc

using namespace hc;

int hc_track_grid_path(const hc_system *s, const double *x0, double *x1, double *hist,
                       hc_path_state *state, int max_stages, const hc_track_opts *o,
                       hc_path_stats *stats, hc_step_record *log, int log_cap, cudaStream_t st);

extern "C" void hc_track_opts_default(hc_track_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->lambda0 = 0.01;
    o->lambda_min = 1e-12;
    o->lambda_max = 0.08;
    o->grow = 2.0;
    o->shrink = 0.5;
    o->eps = 1e-26;
    o->eps_x = 1e-8;
    o->eps_end = 1e-26;
    o->eps_end_x = 1e-26;
    o->div_bound = 1e6;
    o->max_it = 3;
    o->end_it = 8;
    o->grow_after = 3;
    o->max_steps = 100000;
    o->predictor = HC_PRED_SECANT;
    o->lu_mode = HC_LU_NATIVE;
    o->max_refine = 4;
    o->mode = HC_TRACK_PERSISTENT;
    o->graph_steps = 16;
    o->proposer = NULL;
    o->proposer_margin = 0.5;
    o->explore = 0.0;
    o->explore_seed = 0;
}

static int check_opts(const hc_track_opts *o)
{
    if (!o) return hc_fail(HC_EINVAL, "opts is NULL");
    if (!(o->lambda0 > 0) || !(o->lambda_min > 0) || !(o->lambda_max >= o->lambda0))
        return hc_fail(HC_EINVAL, "step sizes must satisfy 0 < lambda_min, 0 < lambda0 <= lambda_max");
    if (!(o->grow >= 1.0) || !(o->shrink > 0.0 && o->shrink < 1.0))
        return hc_fail(HC_EINVAL, "need grow >= 1 and 0 < shrink < 1");
    if (o->max_it < 1 || o->end_it < 0 || o->grow_after < 1 || o->max_steps < 1)
        return hc_fail(HC_EINVAL, "need max_it >= 1, end_it >= 0, grow_after >= 1, max_steps >= 1");
    if (o->predictor != HC_PRED_SECANT && o->predictor != HC_PRED_QUADRATIC && o->predictor != HC_PRED_TANGENT)
        return hc_fail(HC_EINVAL, "unknown predictor %d", o->predictor);
    if (o->predictor == HC_PRED_TANGENT && (o->lu_mode != HC_LU_FP64_REFINE || o->mode == HC_TRACK_GRID))
        return hc_fail(HC_EINVAL, "the tangent predictor needs HC_LU_FP64_REFINE and a block mode");
    if (o->lu_mode != HC_LU_NATIVE && o->lu_mode != HC_LU_FP64_REFINE)
        return hc_fail(HC_EINVAL, "unknown lu_mode %d", o->lu_mode);
    if (o->lu_mode == HC_LU_FP64_REFINE && (o->max_refine < 1 || o->max_refine > 64))
        return hc_fail(HC_EINVAL, "max_refine out of [1, 64]");
    if (o->mode != HC_TRACK_PERSISTENT && o->mode != HC_TRACK_GRAPH && o->mode != HC_TRACK_GRID)
        return hc_fail(HC_EINVAL, "unknown mode %d", o->mode);
    if (o->mode == HC_TRACK_GRID && o->lu_mode != HC_LU_FP64_REFINE)
        return hc_fail(HC_EINVAL, "HC_TRACK_GRID runs the FP64 LU with refinement (HC_LU_FP64_REFINE)");
    if (o->mode == HC_TRACK_GRAPH && (o->graph_steps < 1 || o->graph_steps > 1024))
        return hc_fail(HC_EINVAL, "graph_steps out of [1, 1024]");
    if (o->proposer && !(o->proposer_margin >= 0.0 && o->proposer_margin < 64.0))
        return hc_fail(HC_EINVAL, "proposer_margin out of [0, 64)");
    if (!(o->explore >= 0.0 && o->explore <= 8.0)) return hc_fail(HC_EINVAL, "explore out of [0, 8]");
    return HC_SUCCESS;
}

template <int L>
static int launch_track(TrackArgs &a, int grid, int persistent, size_t smem, cudaStream_t st)
{
    k_track<L><<<grid, HC_TB, smem, st>>>(a, persistent);
    return HC_SUCCESS;
}

// blocks per SM at this dynamic shared memory size (which is opted into first)
template <int L> static int occupancy_track(size_t smem)
{
    cudaFuncSetAttribute(k_track<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_track<L>, HC_TB, smem);
    return occ < 1 ? 1 : occ;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

// hc_path_stats of a path state (the statistics of Tables 2-3)
void hc_stats_of(const PathState &q, hc_path_stats &r)
{
    r.n_succ = q.n_succ;
    r.n_corr = q.n_corr;
    r.newton_its = q.nits;
    r.min_step = q.n_succ ? q.minstep : 0.0;
    r.avg_step = q.n_succ ? q.sumstep / (double)q.n_succ : 0.0;
    r.t_end = q.t;
    r.res_end = q.res_end;
    r.status = q.status;
    r.end_its = q.end_its;
}

// A state handed to hc_track_resume: a known phase, a history that fits, a step.
int hc_check_state(const hc_path_state &q, int p)
{
    if (q.phase < 0 || q.phase > 3) return hc_fail(HC_EINVAL, "state %d: unknown phase %d", p, q.phase);
    if (q.phase == 0 || q.phase == 3) return HC_SUCCESS;
    if (q.nhist < 1 || q.nhist > 3) return hc_fail(HC_EINVAL, "state %d: nhist %d out of [1, 3]", p, q.nhist);
    if (!(q.lambda > 0.0) || !(q.t >= 0.0 && q.t <= 1.0) || q.n_corr < 0)
        return hc_fail(HC_EINVAL, "state %d: bad t, lambda or stage count", p);
    if (q.phase == 2 && q.t < 1.0) return hc_fail(HC_EINVAL, "state %d: end game before t = 1", p);
    if (q.phase == 1 && q.t >= 1.0) return hc_fail(HC_EINVAL, "state %d: tracking at t = 1", p);
    return HC_SUCCESS;
}

// hc_track_path (state == NULL: every path from t = 0, no stage budget) and
// hc_track_resume (state != NULL: the caller's states, x in place, the caller's hist).
static int track_impl(hc_system *const *sys, int npaths, const double *x0, double *x1, double *hist_io,
                      hc_path_state *state_io, int max_stages, const hc_track_opts *opts,
                      hc_path_stats *stats, hc_step_record *log, int log_cap, void *stream)
{
    if (log_cap < 0 || (log_cap > 0 && !log)) return hc_fail(HC_EINVAL, "bad log buffer");
    int rc = check_opts(opts);
    if (rc) return rc;
    int L = 0, nmax = 0, emax = 1;
    long long vmax = 0, total = 0;
    std::vector<DevSys> hs((size_t)npaths);
    std::vector<long long> off((size_t)npaths);
    for (int p = 0; p < npaths; p++) {
        const hc_system *s = sys[p];
        if (!s) return hc_fail(HC_EINVAL, "system %d is NULL", p);
        if (p == 0) L = s->prec;
        if (s->prec != L) return hc_fail(HC_EINVAL, "systems of different precision");
        if (s->npoly != s->n) return hc_fail(HC_EINVAL, "system %d: tracking needs npoly == n", p);
        if (s->min_deg < 1) return hc_fail(HC_EINVAL, "system %d: a polynomial of degree 0", p);
        if (s->n > 256) return hc_fail(HC_EINVAL, "system %d: n = %d above the tracker's 256", p, s->n);
        if (state_io && (rc = hc_check_state(state_io[p], p))) return rc;
        hs[p] = s->dev;
        off[p] = total;
        total += 2LL * L * s->n;
        nmax = s->n > nmax ? s->n : nmax;
        emax = s->max_exp > emax ? s->max_exp : emax;
        const long long v = (long long)s->nvar + s->nmon;
        vmax = v > vmax ? v : vmax;
    }
    if (opts->mode == HC_TRACK_GRID) {
        // one path at a time, each on the whole GPU
        for (int p = 0; p < npaths; p++) {
            hc_path_stats tmp;
            rc = hc_track_grid_path(sys[p], x0 + off[p], x1 + off[p], hist_io ? hist_io + 3 * off[p] : nullptr,
                                    state_io ? &state_io[p] : nullptr, max_stages, opts, stats ? &stats[p] : &tmp,
                                    log_cap > 0 ? log + (size_t)p * log_cap : nullptr, log_cap,
                                    (cudaStream_t)stream);
            if (rc) return rc;
        }
        return HC_SUCCESS;
    }
    const int sms = hc_num_sms();
    // the FP64 factors go to shared memory when a block's share stays within what the
    // register limit's blocks per SM leave of the SM's 228 KiB: four blocks (128 registers)
    // for double and DD, 54 KiB each; three for QD (168 registers), 72 KiB each.  With four
    // blocks and the factors in global memory the tracker still runs 8 % more stages per
    // second than with three and the factors in shared memory (uneven family, n <= 64).
    const size_t smem_cap = L == 4 ? 72 * 1024 : 54 * 1024;
    const int b_smem = sizeof(double) * track_smem_doubles(nmax, 1) <= smem_cap;
    const size_t smem = sizeof(double) * track_smem_doubles(nmax, b_smem);
    int occ = L == 1 ? occupancy_track<1>(smem) : L == 2 ? occupancy_track<2>(smem) : occupancy_track<4>(smem);
    const int grid = (int)(npaths < (long long)sms * occ ? npaths : (long long)sms * occ);

    SlotLayout lay;
    size_t o = 0;
    auto put = [&](size_t bytes) { size_t at = o; o = hc_align256(o + bytes); return at; };
    lay.pw = put(sizeof(double) * 2 * L * (size_t)nmax * (emax > 2 ? emax - 2 : 1));
    lay.v = put(sizeof(double) * 2 * L * (size_t)(vmax > 0 ? vmax : 1));
    lay.hs = put(sizeof(double) * 2 * L * 3 * (size_t)nmax);
    lay.ht = put(sizeof(double) * 2 * (size_t)nmax);
    lay.h = put(sizeof(double) * 2 * L * (size_t)nmax);
    lay.jh = put(sizeof(double) * 2 * L * (size_t)nmax * nmax);
    lay.b = put(b_smem ? 0 : sizeof(double) * 2 * (size_t)nmax * nmax);
    lay.dz = put(sizeof(double) * 2 * L * (size_t)nmax);
    lay.zp = put(sizeof(double) * 2 * L * (size_t)nmax);
    lay.stride = o;

    size_t b_sys = hc_align256(sizeof(DevSys) * npaths);
    size_t b_off = hc_align256(sizeof(long long) * npaths);
    size_t b_n0 = hc_align256(sizeof(long long) * npaths);
    size_t b_hist = hist_io ? 0 : hc_align256(sizeof(double) * 3 * (size_t)total);
    size_t b_zh = hc_align256(sizeof(double) * (size_t)total);
    size_t b_st = hc_align256(sizeof(PathState) * npaths);
    size_t b_ord = hc_align256(sizeof(int) * npaths);
    size_t b_ctr = 256;
    size_t bytes = b_sys + b_off + b_n0 + b_hist + b_zh + b_st + b_ord + b_ctr + lay.stride * (size_t)grid;
    DevBuf ws;
    HC_CUDA_TRY(cudaMalloc(&ws.p, bytes));
    char *b = (char *)ws.p;
    auto take = [&](size_t nb) { char *at = b; b += nb; return at; };
    cudaStream_t st = (cudaStream_t)stream;
    TrackArgs a;
    a.sys = (const DevSys *)take(b_sys);
    a.xoff = (const long long *)take(b_off);
    long long *n0 = (long long *)take(b_n0);
    a.n0 = n0;
    a.hist = hist_io ? hist_io : (double *)take(b_hist);
    a.zh = (double *)take(b_zh);
    a.st = (PathState *)take(b_st);
    int *ord = (int *)take(b_ord);
    int *ctr = (int *)take(b_ctr);
    a.queue = ctr;
    a.active = ctr + 1;
    a.order = ord;
    a.slots = b;
    a.lay = lay;
    a.x0 = x0;
    a.x1 = x1;
    a.o = *opts;
    a.log = log_cap > 0 ? log : nullptr;
    a.log_cap = log_cap;
    a.npaths = npaths;
    a.nmax = nmax;
    a.b_smem = b_smem;
    a.max_stages = max_stages;
    HC_CUDA_TRY(cudaMemcpyAsync((void *)a.sys, hs.data(), sizeof(DevSys) * npaths, cudaMemcpyHostToDevice, st));
    HC_CUDA_TRY(cudaMemcpyAsync((void *)a.xoff, off.data(), sizeof(long long) * npaths, cudaMemcpyHostToDevice, st));
    std::vector<long long> hn0((size_t)npaths, 0);
    int h_active = npaths;
    if (state_io) {
        h_active = 0;
        for (int p = 0; p < npaths; p++) {
            hn0[p] = state_io[p].phase == 0 ? 0 : state_io[p].n_corr;
            h_active += state_io[p].phase != 3;
        }
        HC_CUDA_TRY(cudaMemcpyAsync(a.st, state_io, sizeof(PathState) * npaths, cudaMemcpyHostToDevice, st));
    } else {
        HC_CUDA_TRY(cudaMemsetAsync(a.st, 0, sizeof(PathState) * npaths, st));
    }
    HC_CUDA_TRY(cudaMemcpyAsync(n0, hn0.data(), sizeof(long long) * npaths, cudaMemcpyHostToDevice, st));
    // largest first by the cost of a stage (FP64 instructions of one evaluation plus the LU;
    // the number of stages is not known in advance), so the last paths to start are short.
    // The first wave (one path per resident block) is then shuffled: the block scheduler
    // places consecutive blocks on the same SM, and the largest paths in consecutive
    // blocks would share SMs (measured: 21 % fewer stages per second for 608 paths).
    std::vector<int> horder((size_t)npaths);
    std::vector<double> cost((size_t)npaths);
    for (int p = 0; p < npaths; p++) {
        horder[p] = p;
        cost[p] = sys[p]->ops_term + 4.0 / 3.0 * (double)sys[p]->n * sys[p]->n * sys[p]->n;
    }
    std::stable_sort(horder.begin(), horder.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    {
        // Fisher-Yates over the first wave with a fixed SplitMix64 stream (deterministic)
        unsigned long long x = 0x5eedULL;
        const int wave = npaths < grid ? npaths : grid;
        for (int q = wave - 1; q > 0; q--) {
            unsigned long long z = (x += 0x9e3779b97f4a7c15ULL);
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
            z ^= z >> 31;
            const int r = (int)(z % (unsigned long long)(q + 1));
            const int t0 = horder[q];
            horder[q] = horder[r];
            horder[r] = t0;
        }
    }
    HC_CUDA_TRY(cudaMemcpyAsync(ord, horder.data(), sizeof(int) * npaths, cudaMemcpyHostToDevice, st));
    int hctr[2] = {0, h_active};
    HC_CUDA_TRY(cudaMemcpyAsync(ctr, hctr, sizeof hctr, cudaMemcpyHostToDevice, st));

    if (opts->mode == HC_TRACK_PERSISTENT) {
        if (L == 1) launch_track<1>(a, grid, 1, smem, st);
        else if (L == 2) launch_track<2>(a, grid, 1, smem, st);
        else launch_track<4>(a, grid, 1, smem, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return hc_cuda_fail(e, "k_track launch");
    } else if (h_active > 0) {
        // one predictor-corrector stage per launch, graph_steps launches per graph
        cudaStream_t cs;
        HC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaEvent_t ready;
        cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        cudaEventRecord(ready, st);
        cudaStreamWaitEvent(cs, ready, 0);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int g = 0; g < opts->graph_steps; g++) {
                if (L == 1) launch_track<1>(a, grid, 0, smem, cs);
                else if (L == 2) launch_track<2>(a, grid, 0, smem, cs);
                else launch_track<4>(a, grid, 0, smem, cs);
            }
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        // every stage either accepts, halves the step or ends the path, so a path ends (or
        // spends this call's stages) within min(max_steps, max_stages) stages, plus its
        // end game, taken in the same launch
        const long long cap = opts->max_steps < max_stages ? opts->max_steps : max_stages;
        const long long max_replays = cap / opts->graph_steps + 2;
        for (long long r = 0; e == cudaSuccess && r < max_replays && h_active > 0; r++) {
            e = cudaGraphLaunch(exec, cs);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, a.active, sizeof(int), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaEventRecord(ready, cs);
        cudaStreamWaitEvent(st, ready, 0);
        cudaEventDestroy(ready);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return hc_cuda_fail(e, "graph-stepped tracking");
        if (h_active > 0) return hc_fail(HC_ETIMEOUT, "%d paths unfinished after the replay limit", h_active);
    }
    std::vector<PathState> hst((size_t)npaths);
    HC_CUDA_TRY(cudaMemcpyAsync(hst.data(), a.st, sizeof(PathState) * npaths, cudaMemcpyDeviceToHost, st));
    HC_CUDA_TRY(cudaStreamSynchronize(st));
    for (int p = 0; p < npaths; p++) {
        if (stats) hc_stats_of(hst[p], stats[p]);
        if (state_io) state_io[p] = hst[p];
    }
    return HC_SUCCESS;
}

extern "C" int hc_track_path(hc_system *const *sys, int npaths, const double *x0, double *x1,
                             const hc_track_opts *opts, hc_path_stats *stats, hc_step_record *log,
                             int log_cap, void *stream)
{
    if (!sys || npaths < 1) return hc_fail(HC_EINVAL, "need npaths >= 1 systems");
    if (!x0 || !x1 || !stats) return hc_fail(HC_EINVAL, "x0, x1 or stats is NULL");
    return track_impl(sys, npaths, x0, x1, nullptr, nullptr, 0x7fffffff, opts, stats, log, log_cap, stream);
}

extern "C" int hc_track_resume(hc_system *const *sys, int npaths, double *x, double *hist,
                               hc_path_state *state, int max_stages, const hc_track_opts *opts,
                               hc_path_stats *stats, hc_step_record *log, int log_cap, void *stream)
{
    if (!sys || npaths < 1) return hc_fail(HC_EINVAL, "need npaths >= 1 systems");
    if (!x || !hist || !state) return hc_fail(HC_EINVAL, "x, hist or state is NULL");
    if (max_stages < 1) return hc_fail(HC_EINVAL, "max_stages = %d < 1", max_stages);
    return track_impl(sys, npaths, x, x, hist, state, max_stages, opts, stats, log, log_cap, stream);
}
