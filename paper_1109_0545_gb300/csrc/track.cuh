// track.cuh -- the stage logic of the path tracker (Alg. 3.1), shared by the
// block-per-path engine (hc_track.cu) and the whole-GPU engine for one large path
// (hc_grid.cu): the path's scalars, the predictor, and the bookkeeping of a finished
// corrector stage (accept or step back, step-size control, stop criterion).
#pragma once
#include "mlp.cuh"
#include "path.cuh"

namespace hc {

// The path's scalars between corrector stages: the public hc_path_state (include/hc.h),
// which hc_track_resume saves and restarts from.
typedef hc_path_state PathState;

// SplitMix64 (Steele, Lea & Flood 2014): one output of the generator at counter x
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

// Features of the step proposer before the next stage, each scaled to order one:
//   0      t
//   1..3   log2(lambda / lambda0) / 8 of the last three attempted steps
//   4..6   their Newton iteration counts / 4
//   7..9   log10 of their last residuals, clipped to [-40, 5], / 10
//   10     log10 of the last predictor-corrector distance, clipped, / 10 (-4 after a
//          rejection)
//   11     log10 of the last condition estimate / 4
// Missing history reads as steps of lambda0, 0 iterations, residual -40 (i.e. -4),
// condition 0.
__device__ __forceinline__ void proposer_features(const PathState &st, double lambda0, float *f)
{
    f[0] = (float)st.t;
    for (int j = 0; j < 3; j++) {
        f[1 + j] = (float)(log2(st.hl[j] / lambda0) / 8.0);
        f[4 + j] = (float)(st.hi[j] / 4.0);
        f[7 + j] = st.hr[j] > 0.0 ? (float)(fmin(fmax(log10(st.hr[j]), -40.0), 5.0) / 10.0) : -4.0f;
    }
    f[10] = st.pcd > 0.0 ? (float)(fmin(fmax(log10(st.pcd), -40.0), 5.0) / 10.0) : -4.0f;
    f[11] = (float)(st.cond / 4.0);
}


// ||v||_inf from the leading limbs, the same value on every thread of a TB-thread block
template <int L, int TB> __device__ __forceinline__ double vec_norm(int n, const double *v, BlockShared &sh)
{
    double m = 0.0;
    for (int j = threadIdx.x; j < n; j += TB) m = fmax(m, sqrt(c_abs2_lead(ld_c<L>(v, n, j))));
    return block_max<TB>(m, sh);
}

__device__ __forceinline__ void path_init(PathState &st, const hc_track_opts &o, long long pid)
{
    st.pid = pid;
    st.t = st.tp = st.tpp = 0.0;
    st.lambda = o.lambda0;
    st.minstep = INFINITY;
    st.sumstep = 0.0;
    st.res_end = -1.0;
    st.n_succ = st.n_corr = st.nits = 0;
    st.nhist = 1;
    st.consec = 0;
    st.status = HC_OK;
    st.phase = 1;
    st.end_its = 0;
    for (int j = 0; j < 3; j++) {
        st.hl[j] = o.lambda0;
        st.hr[j] = 0.0;
        st.hi[j] = 0;
    }
    st.pcd = -1.0;
    st.cond = 0.0;
    st.lam_plain = o.lambda0;
}

// Predictor (Alg. 3.1 "predict"; Sec. 5 for the quadratic one) at t1 = min(t + lambda, 1):
// writes the predicted point into zh and its copy ZP; block-level, ends synchronised.
template <int L, int TB>
__device__ void stage_predict(const hc_track_opts &o, const PathState &st, int n, const double *z,
                              const double *zp, const double *zpp, const double *tv, double *zh, double *ZP,
                              double &t1_out, double &h_out)
{
    const int tid = threadIdx.x;
    double t1 = add_(st.t, st.lambda);
    if (t1 > 1.0) t1 = 1.0;
    const double h = sub_(t1, st.t);
    t1_out = t1;
    h_out = h;
    double *const wzp = ZP;
        // predictor (Alg. 3.1 "predict"; Sec. 5 for the quadratic one)
        if (o.predictor == HC_PRED_TANGENT && tv && st.nhist >= 2) {
            // tv[2][n] = dx/dt at the last accepted point (FP64)
            for (int j = tid; j < n; j += TB) {
                const C<L> v = c_add(ld_c<L>(z, n, j), c_from<L>(mul_(h, tv[j]), mul_(h, tv[n + j])));
                st_c<L>(zh, n, j, v);
                st_c<L>(wzp, n, j, v);
            }
        } else if (o.predictor == HC_PRED_QUADRATIC && st.nhist >= 3) {
            const double w0 = __ddiv_rn(mul_(sub_(t1, st.tp), sub_(t1, st.t)), mul_(sub_(st.tpp, st.tp), sub_(st.tpp, st.t)));
            const double w1 = __ddiv_rn(mul_(sub_(t1, st.tpp), sub_(t1, st.t)), mul_(sub_(st.tp, st.tpp), sub_(st.tp, st.t)));
            const double w2 = __ddiv_rn(mul_(sub_(t1, st.tpp), sub_(t1, st.tp)), mul_(sub_(st.t, st.tpp), sub_(st.t, st.tp)));
            for (int j = tid; j < n; j += TB) {
                const C<L> v = c_add(c_add(c_mul_d(ld_c<L>(zpp, n, j), w0), c_mul_d(ld_c<L>(zp, n, j), w1)),
                                     c_mul_d(ld_c<L>(z, n, j), w2));
                st_c<L>(zh, n, j, v);
                st_c<L>(wzp, n, j, v);
            }
        } else if (st.nhist >= 2) {
            const double r = __ddiv_rn(h, sub_(st.t, st.tp));
            for (int j = tid; j < n; j += TB) {
                const C<L> zj = ld_c<L>(z, n, j);
                const C<L> v = c_add(zj, c_mul_d(c_sub(zj, ld_c<L>(zp, n, j)), r));
                st_c<L>(zh, n, j, v);
                st_c<L>(wzp, n, j, v);
            }
        } else {
            for (int j = tid; j < n; j += TB) {
                const C<L> v = ld_c<L>(z, n, j);
                st_c<L>(zh, n, j, v);
                st_c<L>(wzp, n, j, v);
            }
        }
        __syncthreads();
}

// Bookkeeping of a finished corrector stage (it Newton iterations, status nst,
// converged conv, last residual res): the divergence test, the log record, accept (shift
// the history, grow lambda) or step back (shrink lambda), the proposer, the stop tests.
// Block-level; st is updated identically on every thread.
template <int L, int TB>
__device__ void stage_finish(const hc_track_opts &o, PathState &st, BlockShared &sh, int n, double *z,
                             double *zp, double *zpp, const double *zh, const double *ZP, double t1, double h,
                             int it, int nst, int conv, double res, double res_first, double cond,
                             hc_step_record *log, int log_cap, long long log0)
{
    const int tid = threadIdx.x;
        st.nits += it;
        st.n_corr++;
        int ok = (nst == HC_OK) && conv;
        const double znorm = vec_norm<L, TB>(n, zh, sh);
        int stop = 0;
        if (ok && !(znorm <= o.div_bound)) {
            ok = 0;
            st.status = isfinite(znorm) ? HC_DIVERGED : HC_NONFINITE;
            stop = 1;
        }
        double pcd = -1.0;
        if (ok) {
            double m = 0.0;
            for (int j = tid; j < n; j += TB)
                m = fmax(m, sqrt(c_abs2_lead(c_sub(ld_c<L>(zh, n, j), ld_c<L>(ZP, n, j)))));
            pcd = block_max<TB>(m, sh);
        }
        // the log holds the stages of this call: stage n_corr is record n_corr - 1 - log0
        if (log && tid == 0 && st.n_corr - log0 <= log_cap) {
            hc_step_record &r = log[st.n_corr - 1 - log0];
            r.t = st.t;
            r.lambda = h;
            r.res_first = res_first;
            r.res_last = res;
            r.pc_dist = pcd;
            r.cond_log10 = cond;
            r.iters = it;
            r.accepted = ok;
        }
        if (ok) {
            for (int j = tid; j < n; j += TB) {
                st_c<L>(zpp, n, j, ld_c<L>(zp, n, j));
                st_c<L>(zp, n, j, ld_c<L>(z, n, j));
                st_c<L>(z, n, j, ld_c<L>(zh, n, j));
            }
            st.tpp = st.tp;
            st.tp = st.t;
            st.t = t1;
            if (st.nhist < 3) st.nhist++;
            st.n_succ++;
            st.sumstep = add_(st.sumstep, h);
            if (h < st.minstep) st.minstep = h;
            st.consec++;
            if (st.consec >= o.grow_after) {
                st.lam_plain = mul_(st.lam_plain, o.grow);
                if (st.lam_plain > o.lambda_max) st.lam_plain = o.lambda_max;
                st.consec = 0;
            }
            st.lambda = st.lam_plain;
        } else if (!stop) {
            st.consec = 0;
            st.lam_plain = mul_(st.lam_plain, o.shrink);
            st.lambda = st.lam_plain;
            if (!o.proposer && st.lambda < o.lambda_min) {
                stop = 1;
                st.status = HC_MIN_STEP;
            }
        }
        // history of the last three stages; with a proposer its estimate of the largest
        // acceptable step sets the next one (the plain halving stays the fallback after a
        // failure; the corrector still judges every step)
        for (int j = 2; j > 0; j--) {
            st.hl[j] = st.hl[j - 1];
            st.hr[j] = st.hr[j - 1];
            st.hi[j] = st.hi[j - 1];
        }
        st.hl[0] = h;
        st.hr[0] = res;
        st.hi[0] = it;
        st.pcd = pcd;
        st.cond = cond;
        if (o.proposer && !stop) {
            if (tid == 0) {
                float f[MLP_IN];
                proposer_features(st, o.lambda0, f);
                sh.bc[0] = (double)mlp_forward_thread(o.proposer, f);
            }
            __syncthreads();
            const double lam_p = h * exp2(sh.bc[0] - o.proposer_margin);
            __syncthreads();
            // after a failure the step is at most shrink times the step that failed (the
            // plain rule applied to the actual step); after a success the proposal may
            // shrink the step ahead of a failure, but not below a quarter of the plain
            // controller's step (lam_plain, run alongside on the same outcomes), so a path
            // cannot crawl on tiny accepted steps
            if (ok) {
                st.lambda = fmin(fmax(lam_p, fmax(o.lambda_min, 0.25 * st.lam_plain)), o.lambda_max);
            } else {
                // the stop criterion follows the actual step
                st.lambda = fmin(mul_(h, o.shrink), lam_p);
                if (st.lambda < o.lambda_min) {
                    stop = 1;
                    st.status = HC_MIN_STEP;
                }
            }
        }
        // exploration for training data: the next step times 2^u, u uniform in
        // [-explore, explore] (same value on every thread)
        if (o.explore > 0.0 && !o.proposer && !stop) {
            const unsigned long long r = splitmix64(o.explore_seed ^ ((unsigned long long)st.pid << 32) ^
                                                    (unsigned long long)st.n_corr);
            const double u = (double)(r >> 11) * 0x1.0p-53;
            st.lambda = fmin(fmax(st.lambda * exp2(o.explore * (2.0 * u - 1.0)), o.lambda_min), o.lambda_max);
        }
        if (!stop && st.t < 1.0 && st.n_corr >= o.max_steps) {
            stop = 1;
            st.status = HC_MAX_STEPS;
        }
        __syncthreads();
        if (stop)
            st.phase = 3;
        else if (st.t >= 1.0)
            st.phase = 2;
}

}  // namespace hc
