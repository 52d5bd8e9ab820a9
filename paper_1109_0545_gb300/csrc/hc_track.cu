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

#include "track_kernel.cuh"

namespace hc {
HC_TRACK_INSTANTIATE(128)
}  // namespace hc


using namespace hc;

int hc_track_grid_path(const hc_system *s, const double *x0, double *x1, double *hist,
                       hc_path_state *state, int max_stages, const hc_track_opts *o,
                       hc_path_stats *stats, hc_step_record *log, int log_cap, int chunk, cudaStream_t st);

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

// Tiles of the tracker (hc_set_track_tiles), process-wide; 0 = automatic.
static int g_track_tb = 0;       // threads per path block: 64, 128, 256 or 512
static int g_track_bps = 0;      // path blocks per SM (capped by occupancy)
static int g_track_factors = 0;  // 0/1: FP64 factors in shared memory when they fit; 2: global
static int g_grid_chunk = 0;     // contributions per chunk of the whole-GPU engine's entry sums

// 512-thread blocks exist for double and double-double only (a quad-double block of 512
// threads would have to live in 128 registers a thread and spill); quad double runs 256
template <int L> static int launch_track(int tb, TrackArgs &a, int grid, int persistent, size_t smem, cudaStream_t st)
{
    if constexpr (L <= 2)
        if (tb == 512) return track_launch<L, 512>(a, grid, persistent, smem, st);
    return tb == 64 ? track_launch<L, 64>(a, grid, persistent, smem, st)
         : tb >= 256 ? track_launch<L, 256>(a, grid, persistent, smem, st)
                     : track_launch<L, 128>(a, grid, persistent, smem, st);
}

template <int L> static int occupancy_track(int tb, size_t smem)
{
    if constexpr (L <= 2)
        if (tb == 512) return track_occupancy<L, 512>(smem);
    return tb == 64 ? track_occupancy<L, 64>(smem) : tb >= 256 ? track_occupancy<L, 256>(smem)
                                                   : track_occupancy<L, 128>(smem);
}

static int launch_track_any(int L, int tb, TrackArgs &a, int grid, int persistent, size_t smem, cudaStream_t st)
{
    return L == 1 ? launch_track<1>(tb, a, grid, persistent, smem, st)
         : L == 2 ? launch_track<2>(tb, a, grid, persistent, smem, st)
                  : launch_track<4>(tb, a, grid, persistent, smem, st);
}

extern "C" int hc_set_track_tiles(int threads_per_block, int blocks_per_sm, int factors, int grid_chunk)
{
    if (threads_per_block != 0 && threads_per_block != 64 && threads_per_block != 128 && threads_per_block != 256 &&
        threads_per_block != 512)
        return hc_fail(HC_EINVAL, "threads_per_block must be 0, 64, 128, 256 or 512");
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return hc_fail(HC_EINVAL, "blocks_per_sm out of [0, 32]");
    if (factors < 0 || factors > 2) return hc_fail(HC_EINVAL, "factors must be 0, 1 or 2");
    if (grid_chunk < 0 || grid_chunk > 4096) return hc_fail(HC_EINVAL, "grid_chunk out of [0, 4096]");
    g_track_tb = threads_per_block;
    g_track_bps = blocks_per_sm;
    g_track_factors = factors;
    g_grid_chunk = grid_chunk;
    return HC_SUCCESS;
}

extern "C" int hc_get_track_tiles(int *threads_per_block, int *blocks_per_sm, int *factors, int *grid_chunk)
{
    if (threads_per_block) *threads_per_block = g_track_tb;
    if (blocks_per_sm) *blocks_per_sm = g_track_bps;
    if (factors) *factors = g_track_factors;
    if (grid_chunk) *grid_chunk = g_grid_chunk;
    return HC_SUCCESS;
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
                                    g_grid_chunk ? g_grid_chunk : 32, (cudaStream_t)stream);
            if (rc) return rc;
        }
        return HC_SUCCESS;
    }
    const int sms = hc_num_sms();
    const int tb = g_track_tb ? g_track_tb : 128;
    // The FP64 factors go to shared memory when a block's share stays within what the
    // blocks the register budget allows per SM leave of the SM's 228 KiB: 512 (double, DD)
    // or 384 (QD) threads per SM, e.g. four 128-thread blocks of 54 KiB or three QD blocks
    // of 72 KiB.  (With four 128-thread blocks and the factors in global memory the tracker
    // still runs 8 % more stages per second than with three and the factors in shared
    // memory: uneven family, n <= 64.)  hc_set_track_tiles can keep them in global memory.
    const int reg_blocks = ((L == 4 ? 384 : 512) / tb) > 0 ? (L == 4 ? 384 : 512) / tb : 1;
    const size_t smem_cap = 228 * 1024 / reg_blocks - 3 * 1024;
    const int b_smem = g_track_factors != 2 && sizeof(double) * track_smem_doubles(nmax, 1) <= smem_cap;
    const size_t smem = sizeof(double) * track_smem_doubles(nmax, b_smem);
    int occ = L == 1 ? occupancy_track<1>(tb, smem) : L == 2 ? occupancy_track<2>(tb, smem) : occupancy_track<4>(tb, smem);
    if (g_track_bps > 0 && g_track_bps < occ) occ = g_track_bps;
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
        launch_track_any(L, tb, a, grid, 1, smem, st);
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
                launch_track_any(L, tb, a, grid, 0, smem, cs);
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
