// hc_newton.cu -- hc_newton_step: one pass of the loop body of Alg. 4.1 at many points.
// Evaluation (hc_eval.cu) writes h and its Jacobian into the workspace; one thread per
// point then takes the residual and solves J dz = -h by Gaussian elimination with
// partial pivoting on [J h] (Sec. 4), either in the working precision or as an FP64 LU
// whose solution is refined with residuals in the working precision.
#include "hc_eval.cuh"

size_t hc_newton_core_bytes(const hc_system *s, int npts, int lu_mode);  // below

namespace hc {

// max_i |h_i| from the leading limbs (re^2 + im^2 in double, as the pivot measure);
// returns false if some h_i is not finite.
template <int L>
__device__ __forceinline__ bool residual_norm(int n, int npts, int p, const double *__restrict__ H,
                                              double &res)
{
    const size_t plane = (size_t)n * npts;
    double r2 = 0.0;
    bool finite = true;
    for (int i = 0; i < n; i++) {
        double re, im;
        ld_lead<L>(H, plane, (size_t)i * npts + p, re, im);
        const double v = add_(mul_(re, re), mul_(im, im));
        if (!isfinite(v)) finite = false;
        if (v > r2) r2 = v;
    }
    res = sqrt(r2);
    return finite;
}

// x -= z (the solution of J z = h, so dz = -z), all or nothing on non-finite values
template <int L>
__device__ __forceinline__ int apply_update(int n, int npts, int p, double *__restrict__ X,
                                            const double *__restrict__ Z, bool subtract)
{
    const size_t plane = (size_t)n * npts;
    bool ok = true;
    for (int i = 0; i < n; i++) {
        const size_t o = (size_t)i * npts + p;
        C<L> z = ld_c<L>(Z, plane, o);
        C<L> v = subtract ? c_sub(ld_c<L>(X, plane, o), z) : c_add(ld_c<L>(X, plane, o), z);
        if (!c_finite_lead(v)) ok = false;
    }
    if (!ok) return HC_NONFINITE;
    for (int i = 0; i < n; i++) {
        const size_t o = (size_t)i * npts + p;
        C<L> z = ld_c<L>(Z, plane, o);
        C<L> v = subtract ? c_sub(ld_c<L>(X, plane, o), z) : c_add(ld_c<L>(X, plane, o), z);
        st_c<L>(X, plane, o, v);
    }
    return HC_OK;
}

// Native: elimination with partial pivoting on [A h] in the working precision, in place.
// The pivot is the entry of largest |.|^2 of the leading limbs, ties to the lowest row.
// The pivot's reciprocal replaces it; back substitution overwrites h with z = A^{-1} h.
template <int L>
__global__ void __launch_bounds__(64) k_newton_native(int n, int npts, double *__restrict__ X,
                                                      double *__restrict__ H, double *__restrict__ A,
                                                      double *__restrict__ res_norm,
                                                      int32_t *__restrict__ status,
                                                      int32_t *__restrict__ sweeps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const size_t hplane = (size_t)n * npts, aplane = (size_t)n * n * npts;
#define AO(i, j) (((size_t)(i) * n + (j)) * npts + p)
#define HO(i) ((size_t)(i) * npts + p)
    double res;
    const bool finite = residual_norm<L>(n, npts, p, H, res);
    if (res_norm) res_norm[p] = res;
    if (sweeps) sweeps[p] = 0;
    if (!finite) {
        status[p] = HC_NONFINITE;
        return;
    }
    for (int k = 0; k < n; k++) {
        double re, im;
        ld_lead<L>(A, aplane, AO(k, k), re, im);
        double best = add_(mul_(re, re), mul_(im, im));
        int piv = k;
        for (int i = k + 1; i < n; i++) {
            ld_lead<L>(A, aplane, AO(i, k), re, im);
            const double v = add_(mul_(re, re), mul_(im, im));
            if (v > best) {
                best = v;
                piv = i;
            }
        }
        if (!(best > 0.0)) {
            status[p] = HC_SINGULAR;
            return;
        }
        if (piv != k) {
            for (int j = k; j < n; j++) {
                const C<L> a = ld_c<L>(A, aplane, AO(k, j));
                st_c<L>(A, aplane, AO(k, j), ld_c<L>(A, aplane, AO(piv, j)));
                st_c<L>(A, aplane, AO(piv, j), a);
            }
            const C<L> h = ld_c<L>(H, hplane, HO(k));
            st_c<L>(H, hplane, HO(k), ld_c<L>(H, hplane, HO(piv)));
            st_c<L>(H, hplane, HO(piv), h);
        }
        const C<L> inv = c_inv(ld_c<L>(A, aplane, AO(k, k)));
        st_c<L>(A, aplane, AO(k, k), inv);
        const C<L> hk = ld_c<L>(H, hplane, HO(k));
        for (int i = k + 1; i < n; i++) {
            const C<L> l = c_mul(ld_c<L>(A, aplane, AO(i, k)), inv);
            for (int j = k + 1; j < n; j++)
                st_c<L>(A, aplane, AO(i, j), c_fnma(ld_c<L>(A, aplane, AO(i, j)), l, ld_c<L>(A, aplane, AO(k, j))));
            st_c<L>(H, hplane, HO(i), c_fnma(ld_c<L>(H, hplane, HO(i)), l, hk));
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        C<L> s = ld_c<L>(H, hplane, HO(i));
        for (int j = i + 1; j < n; j++) s = c_fnma(s, ld_c<L>(A, aplane, AO(i, j)), ld_c<L>(H, hplane, HO(j)));
        st_c<L>(H, hplane, HO(i), c_mul(s, ld_c<L>(A, aplane, AO(i, i))));
    }
    status[p] = apply_update<L>(n, npts, p, X, H, true);
#undef AO
#undef HO
}

// complex double helpers for the FP64 factorisation
struct cd { double re, im; };
__device__ __forceinline__ cd cd_mul(cd a, cd b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cd cd_fnma(cd acc, cd a, cd b)  // acc - a*b
{
    return {fma(-a.re, b.re, fma(a.im, b.im, acc.re)), fma(-a.re, b.im, fma(-a.im, b.re, acc.im))};
}

// Mixed: LU of the leading limbs in double (row swaps recorded), then
//   dz_0 = LU^{-1} lead(-h);  repeat  r = -h - J dz (working precision),
//   d = LU^{-1} lead(r), dz += d
// until ||d|| <= 2^(-53 L) max(||x||, ||dz||) (the update x + dz is then exact to the
// working precision), or max_refine sweeps; a d no smaller than the previous one (the
// residual is at its rounding floor, or the FP64 factors cannot reduce it) ends the
// refinement without being added.
template <int L>
__global__ void __launch_bounds__(64) k_newton_mixed(int n, int npts, double *__restrict__ X,
                                                     const double *__restrict__ H,
                                                     const double *__restrict__ A,
                                                     double *__restrict__ B /* [2][n][n][npts] */,
                                                     double *__restrict__ RV /* [2][n][npts] */,
                                                     double *__restrict__ DZ /* [2][L][n][npts] */,
                                                     int32_t *__restrict__ PIV /* [n][npts] */,
                                                     int max_refine, double *__restrict__ res_norm,
                                                     int32_t *__restrict__ status,
                                                     int32_t *__restrict__ sweeps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    const size_t hplane = (size_t)n * npts, aplane = (size_t)n * n * npts;
#define AO(i, j) (((size_t)(i) * n + (j)) * npts + p)
#define HO(i) ((size_t)(i) * npts + p)
    double res;
    const bool finite = residual_norm<L>(n, npts, p, H, res);
    if (res_norm) res_norm[p] = res;
    if (sweeps) sweeps[p] = 0;
    if (!finite) {
        status[p] = HC_NONFINITE;
        return;
    }
    // double copy and factorisation
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double re, im;
            ld_lead<L>(A, aplane, AO(i, j), re, im);
            B[AO(i, j)] = re;
            B[aplane + AO(i, j)] = im;
        }
    auto ldB = [&](int i, int j) { return cd{B[AO(i, j)], B[aplane + AO(i, j)]}; };
    auto stB = [&](int i, int j, cd v) { B[AO(i, j)] = v.re; B[aplane + AO(i, j)] = v.im; };
    for (int k = 0; k < n; k++) {
        cd a = ldB(k, k);
        double best = add_(mul_(a.re, a.re), mul_(a.im, a.im));
        int piv = k;
        for (int i = k + 1; i < n; i++) {
            const cd v = ldB(i, k);
            const double m = add_(mul_(v.re, v.re), mul_(v.im, v.im));
            if (m > best) {
                best = m;
                piv = i;
            }
        }
        if (!(best > 0.0)) {
            status[p] = HC_SINGULAR;
            return;
        }
        PIV[HO(k)] = piv;
        if (piv != k)
            for (int j = 0; j < n; j++) {
                const cd t = ldB(k, j);
                stB(k, j, ldB(piv, j));
                stB(piv, j, t);
            }
        a = ldB(k, k);
        const cd inv = {a.re / best, -a.im / best};
        stB(k, k, inv);
        for (int i = k + 1; i < n; i++) {
            const cd l = cd_mul(ldB(i, k), inv);
            stB(i, k, l);
            for (int j = k + 1; j < n; j++) stB(i, j, cd_fnma(ldB(i, j), l, ldB(k, j)));
        }
    }
    // solve LU v = RV in place (RV holds the right-hand side in double)
    auto lu_solve = [&]() {
        for (int k = 0; k < n; k++) {
            const int piv = PIV[HO(k)];
            if (piv != k) {
                const double r = RV[HO(k)], i = RV[hplane + HO(k)];
                RV[HO(k)] = RV[HO(piv)];
                RV[hplane + HO(k)] = RV[hplane + HO(piv)];
                RV[HO(piv)] = r;
                RV[hplane + HO(piv)] = i;
            }
        }
        for (int i = 1; i < n; i++) {
            cd s = {RV[HO(i)], RV[hplane + HO(i)]};
            for (int j = 0; j < i; j++) s = cd_fnma(s, ldB(i, j), cd{RV[HO(j)], RV[hplane + HO(j)]});
            RV[HO(i)] = s.re;
            RV[hplane + HO(i)] = s.im;
        }
        for (int i = n - 1; i >= 0; i--) {
            cd s = {RV[HO(i)], RV[hplane + HO(i)]};
            for (int j = i + 1; j < n; j++) s = cd_fnma(s, ldB(i, j), cd{RV[HO(j)], RV[hplane + HO(j)]});
            s = cd_mul(s, ldB(i, i));
            RV[HO(i)] = s.re;
            RV[hplane + HO(i)] = s.im;
        }
    };
    for (int i = 0; i < n; i++) {
        double re, im;
        ld_lead<L>(H, hplane, HO(i), re, im);
        RV[HO(i)] = -re;
        RV[hplane + HO(i)] = -im;
    }
    lu_solve();
    for (int i = 0; i < n; i++) st_c<L>(DZ, hplane, HO(i), c_from<L>(RV[HO(i)], RV[hplane + HO(i)]));
    double xn = 0.0;
    for (int i = 0; i < n; i++) {
        double re, im;
        ld_lead<L>(X, hplane, HO(i), re, im);
        const double v = sqrt(add_(mul_(re, re), mul_(im, im)));
        if (v > xn) xn = v;
    }
    const double tol = ldexp(1.0, -53 * L);
    double prev = INFINITY;
    int sw = 0;
    for (int it = 1; it <= max_refine; it++) {
        for (int i = 0; i < n; i++) {
            C<L> acc = ld_c<L>(H, hplane, HO(i));
            acc.re = r_neg(acc.re);
            acc.im = r_neg(acc.im);
            for (int j = 0; j < n; j++) acc = c_fnma(acc, ld_c<L>(A, aplane, AO(i, j)), ld_c<L>(DZ, hplane, HO(j)));
            RV[HO(i)] = acc.re.v[0];
            RV[hplane + HO(i)] = acc.im.v[0];
        }
        lu_solve();
        double dn = 0.0, zn = 0.0;
        for (int i = 0; i < n; i++) {
            const double dr = RV[HO(i)], di = RV[hplane + HO(i)];
            const double dv = sqrt(add_(mul_(dr, dr), mul_(di, di)));
            if (dv > dn) dn = dv;
        }
        sw = it;
        if (dn >= prev) break;  // no longer shrinking: at the rounding floor, not applied
        for (int i = 0; i < n; i++) {
            const C<L> z = c_add(ld_c<L>(DZ, hplane, HO(i)), c_from<L>(RV[HO(i)], RV[hplane + HO(i)]));
            st_c<L>(DZ, hplane, HO(i), z);
            const double zv = sqrt(c_abs2_lead(z));
            if (zv > zn) zn = zv;
        }
        if (dn <= tol * fmax(xn, zn)) break;
        prev = dn;
    }
    if (sweeps) sweeps[p] = sw;
    status[p] = apply_update<L>(n, npts, p, X, DZ, false);
#undef AO
#undef HO
}

template <int L>
int launch_newton(hc_system *s, int npts, double t, double *X, int lu_mode, int max_refine,
                  double *res_norm, int32_t *status, int32_t *sweeps, char *ws, const EvalTiles &tiles,
                  cudaStream_t st)
{
    const int n = s->n;
    const size_t pw = hc_pw_bytes(s, npts);
    const size_t hb = hc_align256(sizeof(double) * 2 * L * (size_t)n * npts);
    const size_t ab = hc_align256(sizeof(double) * 2 * L * (size_t)n * n * npts);
    double *PW = (double *)ws;
    double *H = (double *)(ws + pw);
    double *A = (double *)(ws + pw + hb);
    // the shared scheme's partial sums after everything else
    double *part = hc_shared_part_bytes(s, npts, true) ? (double *)(ws + hc_newton_core_bytes(s, npts, lu_mode)) : nullptr;
    int rc = s->eval_shared ? launch_eval_shared<L>(s, npts, t, X, PW, H, A, part, st)
                            : launch_eval<L>(s->dev, npts, t, X, PW, H, A, tiles, st);
    if (rc) return rc;
    const int block = 64, grid = (npts + block - 1) / block;
    if (lu_mode == HC_LU_NATIVE) {
        k_newton_native<L><<<grid, block, 0, st>>>(n, npts, X, H, A, res_norm, status, sweeps);
    } else {
        char *b = ws + pw + hb + ab;
        double *B = (double *)b;
        b += hc_align256(sizeof(double) * 2 * (size_t)n * n * npts);
        double *RV = (double *)b;
        b += hc_align256(sizeof(double) * 2 * (size_t)n * npts);
        double *DZ = (double *)b;
        b += hb;
        int32_t *PIV = (int32_t *)b;
        k_newton_mixed<L><<<grid, block, 0, st>>>(n, npts, X, H, A, B, RV, DZ, PIV, max_refine, res_norm,
                                                  status, sweeps);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_newton launch");
    return HC_SUCCESS;
}

}  // namespace hc

using namespace hc;

size_t hc_newton_core_bytes(const hc_system *s, int npts, int lu_mode)
{
    const size_t n = s->n, L = s->prec;
    size_t b = hc_pw_bytes(s, npts);
    b += hc_align256(sizeof(double) * 2 * L * n * npts);          // H
    b += hc_align256(sizeof(double) * 2 * L * n * n * npts);      // J
    if (lu_mode == HC_LU_FP64_REFINE) {
        b += hc_align256(sizeof(double) * 2 * n * n * npts);      // FP64 factors
        b += hc_align256(sizeof(double) * 2 * n * npts);          // FP64 right-hand side
        b += hc_align256(sizeof(double) * 2 * L * n * npts);      // dz
        b += hc_align256(sizeof(int32_t) * n * npts);             // pivots
    }
    return b;
}

size_t hc_newton_ws_bytes(const hc_system *s, int npts, int lu_mode)
{
    return hc_newton_core_bytes(s, npts, lu_mode) + hc_shared_part_bytes(s, npts, true);
}

int hc_check_newton_args(const hc_system *s, int npts, double t, const double *x, int lu_mode,
                         int max_refine, const int32_t *status)
{
    int rc = hc_check_eval_args(s, npts, t);
    if (rc) return rc;
    if (s->npoly != s->n) return hc_fail(HC_EINVAL, "Newton needs npoly == n");
    if (lu_mode != HC_LU_NATIVE && lu_mode != HC_LU_FP64_REFINE) return hc_fail(HC_EINVAL, "bad lu_mode %d", lu_mode);
    if (lu_mode == HC_LU_FP64_REFINE && (max_refine < 1 || max_refine > 64))
        return hc_fail(HC_EINVAL, "max_refine = %d out of [1, 64]", max_refine);
    if (npts > 0 && (!x || !status)) return hc_fail(HC_EINVAL, "x or status is NULL");
    return HC_SUCCESS;
}

int hc_newton_dispatch(hc_system *s, int npts, double t, double *x, int lu_mode, int max_refine,
                       double *res_norm, int32_t *status, int32_t *sweeps, char *ws, cudaStream_t st)
{
    const EvalTiles &tiles = hc_eval_tiles();
    switch (s->prec) {
    case 1: return launch_newton<1>(s, npts, t, x, lu_mode, max_refine, res_norm, status, sweeps, ws, tiles, st);
    case 2: return launch_newton<2>(s, npts, t, x, lu_mode, max_refine, res_norm, status, sweeps, ws, tiles, st);
    case 4: return launch_newton<4>(s, npts, t, x, lu_mode, max_refine, res_norm, status, sweeps, ws, tiles, st);
    }
    return hc_fail(HC_EINVAL, "bad precision");
}

extern "C" int hc_newton_step(hc_system *s, int npts, double t, double *x, int lu_mode, int max_refine,
                              double *res_norm, int32_t *status, int32_t *sweeps, void *stream)
{
    int rc = hc_check_newton_args(s, npts, t, x, lu_mode, max_refine, status);
    if (rc) return rc;
    if (npts == 0) return HC_SUCCESS;
    void *ws = NULL;
    rc = hc_workspace(s, hc_newton_ws_bytes(s, npts, lu_mode), &ws);
    if (rc) return rc;
    return hc_newton_dispatch(s, npts, t, x, lu_mode, max_refine, res_norm, status, sweeps, (char *)ws,
                              (cudaStream_t)stream);
}
