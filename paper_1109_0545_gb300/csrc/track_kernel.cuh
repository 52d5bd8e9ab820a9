// track_kernel.cuh -- the device side of hc_track_path / hc_track_resume's block engine
// (Alg. 3.1 with the corrector of Alg. 4.1, one thread block per path), templated on the
// precision L and the block size TB; instantiated for TB = 64, 128, 256 in three
// translation units (hc_track.cu and hc_track_tb*.cu) that compile in parallel.
#pragma once
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
template <int L, int TB>
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
        for (int q = tid; q < 2 * L * n; q += TB) z[q] = a.x0[a.xoff[p] + q];
        path_init(st, o, p);
        __syncthreads();
    }
    hc_step_record *log = a.log ? a.log + (size_t)p * a.log_cap : nullptr;
    int stages = 0;
    while (st.phase == 1 && stages < max_stages && st.n_corr - n0 < a.max_stages) {
        double t1, h;
        stage_predict<L, TB>(o, st, n, z, zp, zpp, tv, zh, w.ZP, t1, h);
        // corrector: Alg. 4.1
        double res = 1.0, res_first = -1.0, cond = 0.0;
        int it = 0, nst = HC_OK, conv = 0;
        while (!conv && it < o.max_it) {
            const NewtonOut no = block_newton<L, TB>(S, zh, t1, o.lu_mode, o.max_refine, w, sh);
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
        stage_finish<L, TB>(o, st, sh, n, z, zp, zpp, zh, w.ZP, t1, h, it, nst, conv, res, res_first, cond,
                        log, a.log_cap, n0);
        if (tangent && st.n_succ > succ0) {
            for (int q = tid; q < 2 * n; q += TB) tv[q] = -w.Y[q];
            __syncthreads();
        }
        stages++;
    }
    if (st.phase == 2) {
        // end game at t = 1: Newton on f until converged with the end tolerances
        double res = 1.0;
        int conv = 0;
        while (!conv && st.end_its < o.end_it) {
            const NewtonOut no = block_newton<L, TB>(S, z, 1.0, o.lu_mode, o.max_refine, w, sh);
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

// Blocks of TB threads; the register budget per thread is that of 128-thread blocks at
// four (double, DD) or three (QD) blocks per SM, whatever TB: 128 and 168 registers.
template <int L, int TB>
__global__ void __launch_bounds__(TB, (L == 4 ? 384 : 512) / TB > 0 ? (L == 4 ? 384 : 512) / TB : 1)
    k_track(TrackArgs a, int persistent)
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
            path_run<L, TB>(a, a.order[q], w, sh, 0x7fffffff);
        }
    } else {
        for (int q = blockIdx.x; q < a.npaths; q += gridDim.x) path_run<L, TB>(a, a.order[q], w, sh, 1);
    }
}


// launch and occupancy of k_track<L, TB> (instantiated in hc_track*.cu)
template <int L, int TB> int track_launch(TrackArgs &a, int grid, int persistent, size_t smem, cudaStream_t st);
template <int L, int TB> int track_occupancy(size_t smem);

#define HC_TRACK_INSTANTIATE(TB)                                                                         \
    template <> int track_launch<1, TB>(TrackArgs & a, int grid, int persistent, size_t smem, cudaStream_t st) \
    {                                                                                                     \
        k_track<1, TB><<<grid, TB, smem, st>>>(a, persistent);                                          \
        return HC_SUCCESS;                                                                                \
    }                                                                                                     \
    template <> int track_launch<2, TB>(TrackArgs & a, int grid, int persistent, size_t smem, cudaStream_t st) \
    {                                                                                                     \
        k_track<2, TB><<<grid, TB, smem, st>>>(a, persistent);                                          \
        return HC_SUCCESS;                                                                                \
    }                                                                                                     \
    template <> int track_launch<4, TB>(TrackArgs & a, int grid, int persistent, size_t smem, cudaStream_t st) \
    {                                                                                                     \
        k_track<4, TB><<<grid, TB, smem, st>>>(a, persistent);                                          \
        return HC_SUCCESS;                                                                                \
    }                                                                                                     \
    template <> int track_occupancy<1, TB>(size_t smem) { return track_occ_of(k_track<1, TB>, TB, smem); } \
    template <> int track_occupancy<2, TB>(size_t smem) { return track_occ_of(k_track<2, TB>, TB, smem); } \
    template <> int track_occupancy<4, TB>(size_t smem) { return track_occ_of(k_track<4, TB>, TB, smem); }

// double and double-double only (512-thread blocks)
#define HC_TRACK_INSTANTIATE_D_DD(TB)                                                                    \
    template <> int track_launch<1, TB>(TrackArgs & a, int grid, int persistent, size_t smem, cudaStream_t st) \
    {                                                                                                     \
        k_track<1, TB><<<grid, TB, smem, st>>>(a, persistent);                                          \
        return HC_SUCCESS;                                                                                \
    }                                                                                                     \
    template <> int track_launch<2, TB>(TrackArgs & a, int grid, int persistent, size_t smem, cudaStream_t st) \
    {                                                                                                     \
        k_track<2, TB><<<grid, TB, smem, st>>>(a, persistent);                                          \
        return HC_SUCCESS;                                                                                \
    }                                                                                                     \
    template <> int track_occupancy<1, TB>(size_t smem) { return track_occ_of(k_track<1, TB>, TB, smem); } \
    template <> int track_occupancy<2, TB>(size_t smem) { return track_occ_of(k_track<2, TB>, TB, smem); }

// blocks per SM of kernel k at this dynamic shared memory size (which is opted into first)
template <typename K> inline int track_occ_of(K k, int tb, size_t smem)
{
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tb, smem);
    return occ < 1 ? 1 : occ;
}

}  // namespace hc
