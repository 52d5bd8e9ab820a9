// hc_system.cu -- loading a sparse system (the normalised monomial form of Sec. 6),
// error reporting, workspace, and the FP64 peak probe.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>

#include "hc_internal.h"

static thread_local char g_err[512];

extern "C" const char *hc_last_error(void) { return g_err; }

int hc_fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int hc_cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_err, sizeof g_err, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HC_ENOMEM : HC_ECUDA;
}

int hc_num_sms(void)
{
    static int cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------------
// Event timing of the evaluation kernel: each launch is bracketed by two events on the
// stream it runs on; hc_prof_read waits for them and sums the intervals.
// ---------------------------------------------------------------------------------
#include <vector>
static bool g_prof = false;
static std::vector<cudaEvent_t> g_prof_ev;  // begin, end, begin, end, ...

bool hc_prof_on(void) { return g_prof; }

void hc_prof_mark(cudaStream_t st, bool begin)
{
    if (!g_prof) return;
    if (begin != (g_prof_ev.size() % 2 == 0)) return;  // keep begin/end paired
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    g_prof_ev.push_back(e);
}

extern "C" int hc_prof_enable(int on)
{
    g_prof = on != 0;
    return HC_SUCCESS;
}

extern "C" int hc_prof_read(double *ms, int *launches)
{
    double total = 0.0;
    int n = 0;
    cudaError_t err = cudaSuccess;
    for (size_t i = 0; i + 1 < g_prof_ev.size(); i += 2) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(g_prof_ev[i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, g_prof_ev[i], g_prof_ev[i + 1]);
        if (e != cudaSuccess) err = e;
        total += t;
        n++;
    }
    for (cudaEvent_t e : g_prof_ev) cudaEventDestroy(e);
    g_prof_ev.clear();
    if (ms) *ms = total;
    if (launches) *launches = n;
    if (err != cudaSuccess) return hc_cuda_fail(err, "hc_prof_read");
    return HC_SUCCESS;
}

int hc_workspace(hc_system *s, size_t bytes, void **out)
{
    if (bytes == 0) bytes = 256;
    if (s->ws_bytes < bytes) {
        if (s->ws) {
            // the old workspace may still be in use by queued work
            HC_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(s->ws);
            s->ws = NULL;
            s->ws_bytes = 0;
        }
        void *p = NULL;
        HC_CUDA_TRY(cudaMalloc(&p, bytes));
        s->ws = p;
        s->ws_bytes = bytes;
    }
    *out = s->ws;
    return HC_SUCCESS;
}

// Validation of the normalised form: every failure is HC_EINVAL with a message.
static int validate(int n, int npoly, const int32_t *mon_ptr, const int32_t *var_ptr,
                    const int32_t *var_idx, const int32_t *var_exp, const double *coef,
                    int prec, const double *gamma)
{
    if (n < 1 || n > HC_NMAX) return hc_fail(HC_EINVAL, "n = %d out of [1, %d]", n, HC_NMAX);
    if (npoly < 1 || npoly > HC_NMAX) return hc_fail(HC_EINVAL, "npoly = %d out of range", npoly);
    if (prec != 1 && prec != 2 && prec != 4) return hc_fail(HC_EINVAL, "prec = %d not 1, 2 or 4", prec);
    if (!mon_ptr || !var_ptr || !coef || !gamma) return hc_fail(HC_EINVAL, "NULL array");
    if (mon_ptr[0] != 0) return hc_fail(HC_EINVAL, "mon_ptr[0] != 0");
    for (int i = 0; i < npoly; i++)
        if (mon_ptr[i + 1] < mon_ptr[i]) return hc_fail(HC_EINVAL, "mon_ptr decreases at %d", i);
    long long nmon = mon_ptr[npoly];
    if (nmon > (1LL << 30)) return hc_fail(HC_EINVAL, "too many monomials");
    if (var_ptr[0] != 0) return hc_fail(HC_EINVAL, "var_ptr[0] != 0");
    for (long long m = 0; m < nmon; m++) {
        int q0 = var_ptr[m], q1 = var_ptr[m + 1];
        if (q1 < q0) return hc_fail(HC_EINVAL, "var_ptr decreases at monomial %lld", m);
        if (q1 - q0 > HC_KMAX) return hc_fail(HC_EINVAL, "monomial %lld has %d > %d variables", m, q1 - q0, HC_KMAX);
        for (int q = q0; q < q1; q++) {
            if (!var_idx || !var_exp) return hc_fail(HC_EINVAL, "NULL var arrays");
            if (var_idx[q] < 0 || var_idx[q] >= n)
                return hc_fail(HC_EINVAL, "monomial %lld: index %d out of [0,%d)", m, var_idx[q], n);
            if (var_exp[q] < 1 || var_exp[q] > HC_EXPMAX)
                return hc_fail(HC_EINVAL, "monomial %lld: exponent %d out of [1,%d]", m, var_exp[q], HC_EXPMAX);
            if (q > q0 && var_idx[q] <= var_idx[q - 1])
                return hc_fail(HC_EINVAL, "monomial %lld: indices not strictly increasing", m);
        }
        for (int c = 0; c < 2 * prec; c++)
            if (!std::isfinite(coef[m * 2 * prec + c]))
                return hc_fail(HC_EINVAL, "monomial %lld: coefficient not finite", m);
    }
    if (!std::isfinite(gamma[0]) || !std::isfinite(gamma[1])) return hc_fail(HC_EINVAL, "gamma not finite");
    return HC_SUCCESS;
}

static int build_shared_tables(hc_system *s);

extern "C" int hc_system_load(hc_system **out, int n, int npoly, const int32_t *mon_ptr,
                              const int32_t *var_ptr, const int32_t *var_idx,
                              const int32_t *var_exp, const double *coef, int prec,
                              const double gamma[2])
{
    if (!out) return hc_fail(HC_EINVAL, "out is NULL");
    *out = NULL;
    int rc = validate(n, npoly, mon_ptr, var_ptr, var_idx, var_exp, coef, prec, gamma);
    if (rc) return rc;
    int nmon = mon_ptr[npoly];
    int nvar = var_ptr[nmon];

    hc_system *s = (hc_system *)calloc(1, sizeof(hc_system));
    if (!s) return hc_fail(HC_ENOMEM, "host allocation failed");
    s->n = n;
    s->npoly = npoly;
    s->nmon = nmon;
    s->nvar = nvar;
    s->prec = prec;
    s->gamma[0] = gamma[0];
    s->gamma[1] = gamma[1];
    cudaGetDevice(&s->device);

    // host tables: packed (index, exponent), degrees
    s->h_mon_ptr = (int32_t *)malloc(sizeof(int32_t) * (npoly + 1));
    s->h_var_ptr = (int32_t *)malloc(sizeof(int32_t) * (nmon + 1));
    s->h_var_pack = (int32_t *)malloc(sizeof(int32_t) * (nvar > 0 ? nvar : 1));
    s->h_deg = (int32_t *)malloc(sizeof(int32_t) * npoly);
    if (!s->h_mon_ptr || !s->h_var_ptr || !s->h_var_pack || !s->h_deg) {
        hc_system_free(s);
        return hc_fail(HC_ENOMEM, "host allocation failed");
    }
    memcpy(s->h_mon_ptr, mon_ptr, sizeof(int32_t) * (npoly + 1));
    memcpy(s->h_var_ptr, var_ptr, sizeof(int32_t) * (nmon + 1));
    int max_exp = 1;
    for (int q = 0; q < nvar; q++) {
        s->h_var_pack[q] = var_idx[q] | (var_exp[q] << 16);
        if (var_exp[q] > max_exp) max_exp = var_exp[q];
    }
    int max_deg = 0, min_deg = 1 << 30;
    for (int i = 0; i < npoly; i++) {
        int d = 0;
        for (int m = mon_ptr[i]; m < mon_ptr[i + 1]; m++) {
            int tot = 0;
            for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++) tot += var_exp[q];
            if (tot > d) d = tot;
        }
        s->h_deg[i] = d;
        if (d > max_deg) max_deg = d;
        if (d < min_deg) min_deg = d;
    }
    s->max_exp = max_exp;
    s->max_deg = max_deg;
    s->min_deg = min_deg;

    // tables of the block-per-path engine: monomials ordered by shape so the warps of a
    // block walk monomials of equal length, and the transpose (entry -> contributions)
    const int ne = npoly * (n + 1);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (nmon > 0 ? nmon : 1));
    int32_t *tptr = (int32_t *)calloc((size_t)ne + 1, sizeof(int32_t));
    int32_t *tlist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nvar + nmon > 0 ? nvar + nmon : 1));
    std::vector<int32_t> eperm((size_t)(ne > 0 ? ne : 1));
    if (!perm || !tptr || !tlist) {
        free(perm); free(tptr); free(tlist);
        hc_system_free(s);
        return hc_fail(HC_ENOMEM, "host allocation failed");
    }
    {
        // counting sort by key = k * 64 + (exponents >= 2), stable
        const int nkey = (HC_KMAX + 1) * 64;
        int32_t *cnt = (int32_t *)calloc((size_t)nkey + 1, sizeof(int32_t));
        if (!cnt) { free(perm); free(tptr); free(tlist); hc_system_free(s); return hc_fail(HC_ENOMEM, "host allocation failed"); }
        auto key = [&](int m) {
            int k = var_ptr[m + 1] - var_ptr[m], n2 = 0;
            for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++) n2 += var_exp[q] >= 2;
            return k * 64 + n2;
        };
        for (int m = 0; m < nmon; m++) cnt[key(m) + 1]++;
        for (int k = 0; k < nkey; k++) cnt[k + 1] += cnt[k];
        for (int m = 0; m < nmon; m++) perm[cnt[key(m)]++] = m;
        free(cnt);
        // transpose: count, prefix, fill in monomial order
        for (int i = 0; i < npoly; i++)
            for (int m = mon_ptr[i]; m < mon_ptr[i + 1]; m++) {
                tptr[i * (n + 1) + n + 1]++;
                for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++) tptr[i * (n + 1) + var_idx[q] + 1]++;
            }
        for (int e = 0; e < ne; e++) tptr[e + 1] += tptr[e];
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
        if (!fill) { free(perm); free(tptr); free(tlist); hc_system_free(s); return hc_fail(HC_ENOMEM, "host allocation failed"); }
        memcpy(fill, tptr, sizeof(int32_t) * (size_t)ne);
        for (int i = 0; i < npoly; i++)
            for (int m = mon_ptr[i]; m < mon_ptr[i + 1]; m++) {
                tlist[fill[i * (n + 1) + n]++] = nvar + m;
                for (int q = var_ptr[m]; q < var_ptr[m + 1]; q++)
                    tlist[fill[i * (n + 1) + var_idx[q]]++] = q;
            }
        free(fill);
        // entries by contribution count, longest first; the sort is stable
        for (int q = 0; q < ne; q++) eperm[q] = q;
        std::stable_sort(eperm.begin(), eperm.begin() + ne, [&](int32_t a, int32_t b) {
            return tptr[a + 1] - tptr[a] > tptr[b + 1] - tptr[b];
        });
    }

    // one device block: mon_ptr | var_ptr | var_pack | deg | perm | tptr | tlist | eperm | coef
    size_t o_mon = 0;
    size_t o_var = hc_align256(o_mon + sizeof(int32_t) * (npoly + 1));
    size_t o_pack = hc_align256(o_var + sizeof(int32_t) * (nmon + 1));
    size_t o_deg = hc_align256(o_pack + sizeof(int32_t) * (nvar > 0 ? nvar : 1));
    size_t o_perm = hc_align256(o_deg + sizeof(int32_t) * npoly);
    size_t o_tptr = hc_align256(o_perm + sizeof(int32_t) * (nmon > 0 ? nmon : 1));
    size_t o_tlist = hc_align256(o_tptr + sizeof(int32_t) * ((size_t)ne + 1));
    size_t o_eperm = hc_align256(o_tlist + sizeof(int32_t) * (size_t)(nvar + nmon > 0 ? nvar + nmon : 1));
    size_t o_coef = hc_align256(o_eperm + sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
    size_t total = hc_align256(o_coef + sizeof(double) * 2 * prec * (size_t)(nmon > 0 ? nmon : 1));
    cudaError_t e = cudaMalloc(&s->dev_block, total);
    if (e != cudaSuccess) {
        free(perm); free(tptr); free(tlist);
        hc_system_free(s);
        return hc_cuda_fail(e, "cudaMalloc(system tables)");
    }
    char *b = (char *)s->dev_block;
    e = cudaMemcpy(b + o_mon, s->h_mon_ptr, sizeof(int32_t) * (npoly + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_var, s->h_var_ptr, sizeof(int32_t) * (nmon + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nvar > 0) e = cudaMemcpy(b + o_pack, s->h_var_pack, sizeof(int32_t) * nvar, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_deg, s->h_deg, sizeof(int32_t) * npoly, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nmon > 0) e = cudaMemcpy(b + o_perm, perm, sizeof(int32_t) * nmon, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_tptr, tptr, sizeof(int32_t) * ((size_t)ne + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nvar + nmon > 0)
        e = cudaMemcpy(b + o_tlist, tlist, sizeof(int32_t) * (size_t)(nvar + nmon), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && ne > 0)
        e = cudaMemcpy(b + o_eperm, eperm.data(), sizeof(int32_t) * (size_t)ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nmon > 0)
        e = cudaMemcpy(b + o_coef, coef, sizeof(double) * 2 * prec * (size_t)nmon, cudaMemcpyHostToDevice);
    free(perm);
    free(tptr);
    free(tlist);
    if (e != cudaSuccess) {
        hc_system_free(s);
        return hc_cuda_fail(e, "cudaMemcpy(system tables)");
    }
    DevSys &d = s->dev;
    d.n = n;
    d.npoly = npoly;
    d.nmon = nmon;
    d.nvar = nvar;
    d.max_exp = max_exp;
    d.mon_ptr = (const int32_t *)(b + o_mon);
    d.var_ptr = (const int32_t *)(b + o_var);
    d.var_pack = (const int32_t *)(b + o_pack);
    d.deg = (const int32_t *)(b + o_deg);
    d.perm = (const int32_t *)(b + o_perm);
    d.tptr = (const int32_t *)(b + o_tptr);
    d.tlist = (const int32_t *)(b + o_tlist);
    d.eperm = (const int32_t *)(b + o_eperm);
    d.coef = (const double *)(b + o_coef);
    d.gre = gamma[0];
    d.gim = gamma[1];
    const int rc_shared = build_shared_tables(s);
    if (rc_shared) {
        hc_system_free(s);
        return rc_shared;
    }
    *out = s;
    return HC_SUCCESS;
}

// FP64 instructions (complex DD weights) of one monomial's evaluation with its partials:
// the common factor, prefix products, value and backward sweep (with_coef: the
// coefficient folded into the common factor), and the integer scalings of the partials
static double monomial_ops(const int32_t *pack, int k, bool with_coef)
{
    if (k == 0) return 0.0;
    int n2 = 0;
    double scale = 0.0;
    for (int q = 0; q < k; q++) {
        const int e = pack[q] >> 16;
        n2 += e >= 2;
        if (e != 1 && (e & (e - 1)) != 0) scale += 12.0;
    }
    int mults = n2 + (k >= 2 ? 3 * k - 3 : 1);
    if (!with_coef && n2 == 0) mults -= 1;  // the common factor is exactly 1
    return 26.0 * mults + scale;
}

// The shared-monomial tables: distinct non-constant monomials in order of first use, the
// terms using each, the polynomial of each term, each polynomial's constant terms; and the
// FP64 counts of the per-term and shared evaluation schemes.
static int build_shared_tables(hc_system *s)
{
    const int nmon = s->nmon, npoly = s->npoly;
    const int32_t *vp = s->h_var_ptr, *pack = s->h_var_pack;
    std::map<std::vector<int32_t>, int> ids;
    std::vector<int32_t> uid((size_t)nmon, -1), first, term_row((size_t)nmon), cptr((size_t)npoly + 1, 0), cterm;
    double ops_term = 0.0, ops_shared = 0.0;
    for (int i = 0; i < npoly; i++) {
        for (int m = s->h_mon_ptr[i]; m < s->h_mon_ptr[i + 1]; m++) {
            term_row[m] = i;
            const int k = vp[m + 1] - vp[m];
            if (k == 0) {
                cterm.push_back(m);
                ops_term += 10.0;
                ops_shared += 10.0;
                continue;
            }
            std::vector<int32_t> key(pack + vp[m], pack + vp[m + 1]);
            auto it = ids.find(key);
            if (it == ids.end()) {
                it = ids.emplace(std::move(key), (int)first.size()).first;
                first.push_back(m);
                ops_shared += monomial_ops(pack + vp[m], k, false);
            }
            uid[m] = it->second;
            ops_term += monomial_ops(pack + vp[m], k, true) + 10.0 * (k + 1);
            ops_shared += 36.0 * (k + 1);
        }
        cptr[i + 1] = (int32_t)cterm.size();
    }
    // f_i and the Jacobian row are running sums (10 FP64 a term), renormalised once (6)
    ops_term += 6.0 * npoly * (s->n + 1);
    ops_shared += 6.0 * npoly * (s->n + 1);
    const int nuniq = (int)first.size();
    std::vector<int32_t> uvar_ptr((size_t)nuniq + 1, 0), uvar_pack, uuse_ptr((size_t)nuniq + 1, 0), uuse;
    // FP64 cost of each distinct monomial (evaluation, then 36 a partial or value per use)
    std::vector<double> ucost((size_t)nuniq + 1, 0.0);
    for (int m = 0; m < nmon; m++)
        if (uid[m] >= 0) ucost[uid[m] + 1] += 36.0 * (vp[m + 1] - vp[m] + 1);
    for (int u = 0; u < nuniq; u++)
        ucost[u + 1] += ucost[u] + monomial_ops(pack + vp[first[u]], vp[first[u] + 1] - vp[first[u]], false);
    for (int u = 0; u < nuniq; u++) {
        const int m = first[u];
        uvar_pack.insert(uvar_pack.end(), pack + vp[m], pack + vp[m + 1]);
        uvar_ptr[u + 1] = (int32_t)uvar_pack.size();
    }
    for (int m = 0; m < nmon; m++)
        if (uid[m] >= 0) uuse_ptr[uid[m] + 1]++;
    for (int u = 0; u < nuniq; u++) uuse_ptr[u + 1] += uuse_ptr[u];
    uuse.resize((size_t)uuse_ptr[nuniq]);
    {
        std::vector<int32_t> fill(uuse_ptr.begin(), uuse_ptr.end() - 1);
        for (int m = 0; m < nmon; m++)
            if (uid[m] >= 0) uuse[fill[uid[m]]++] = m;
    }
    // one device block: uvar_ptr | uvar_pack | uuse_ptr | uuse | term_row | cptr | cterm | ucost
    auto sz = [](size_t n) { return hc_align256(sizeof(int32_t) * (n > 0 ? n : 1)); };
    const size_t o1 = 0, o2 = o1 + sz(uvar_ptr.size()), o3 = o2 + sz(uvar_pack.size()),
                 o4 = o3 + sz(uuse_ptr.size()), o5 = o4 + sz(uuse.size()), o6 = o5 + sz(term_row.size()),
                 o7 = o6 + sz(cptr.size()), o8 = o7 + sz(cterm.size()),
                 total = o8 + hc_align256(sizeof(double) * ucost.size());
    cudaError_t e = cudaMalloc(&s->dev_shared, total);
    if (e != cudaSuccess) return hc_cuda_fail(e, "cudaMalloc(shared tables)");
    char *b = (char *)s->dev_shared;
    auto put = [&](size_t off, const std::vector<int32_t> &v) {
        if (e == cudaSuccess && !v.empty())
            e = cudaMemcpy(b + off, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
    };
    put(o1, uvar_ptr);
    put(o2, uvar_pack);
    put(o3, uuse_ptr);
    put(o4, uuse);
    put(o5, term_row);
    put(o6, cptr);
    put(o7, cterm);
    if (e == cudaSuccess)
        e = cudaMemcpy(b + o8, ucost.data(), sizeof(double) * ucost.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return hc_cuda_fail(e, "cudaMemcpy(shared tables)");
    DevSys &d = s->dev;
    d.nuniq = nuniq;
    d.uvar_ptr = (const int32_t *)(b + o1);
    d.uvar_pack = (const int32_t *)(b + o2);
    d.uuse_ptr = (const int32_t *)(b + o3);
    d.uuse = (const int32_t *)(b + o4);
    d.term_row = (const int32_t *)(b + o5);
    d.cptr = (const int32_t *)(b + o6);
    d.cterm = (const int32_t *)(b + o7);
    d.ucost = (const double *)(b + o8);
    s->ops_term = ops_term;
    s->ops_shared = ops_shared;
    // the shared scheme when it saves at least a tenth of the FP64 instructions
    s->eval_shared = ops_shared < 0.9 * ops_term;
    return HC_SUCCESS;
}

extern "C" int hc_system_set_eval_mode(hc_system *s, int mode)
{
    if (!s) return hc_fail(HC_EINVAL, "sys is NULL");
    if (mode == HC_EVAL_AUTO) s->eval_shared = s->ops_shared < 0.9 * s->ops_term;
    else if (mode == HC_EVAL_PER_TERM) s->eval_shared = 0;
    else if (mode == HC_EVAL_SHARED) s->eval_shared = 1;
    else return hc_fail(HC_EINVAL, "unknown evaluation mode %d", mode);
    return HC_SUCCESS;
}

extern "C" int hc_system_eval_mode(const hc_system *s, double *ops_per_term, double *ops_shared)
{
    if (!s) return hc_fail(HC_EINVAL, "sys is NULL");
    if (ops_per_term) *ops_per_term = s->ops_term;
    if (ops_shared) *ops_shared = s->ops_shared;
    return s->eval_shared ? HC_EVAL_SHARED : HC_EVAL_PER_TERM;
}

extern "C" void hc_system_free(hc_system *s)
{
    if (!s) return;
    if (s->dev_block || s->ws || s->dev_shared) cudaDeviceSynchronize();
    if (s->dev_block) cudaFree(s->dev_block);
    if (s->dev_shared) cudaFree(s->dev_shared);
    if (s->ws) cudaFree(s->ws);
    free(s->h_mon_ptr);
    free(s->h_var_ptr);
    free(s->h_var_pack);
    free(s->h_deg);
    free(s);
}

extern "C" int hc_system_info(const hc_system *s, int *n, int *npoly, int *nmon, int *nvar,
                              int *prec, int *max_exp, int *max_deg)
{
    if (!s) return hc_fail(HC_EINVAL, "sys is NULL");
    if (n) *n = s->n;
    if (npoly) *npoly = s->npoly;
    if (nmon) *nmon = s->nmon;
    if (nvar) *nvar = s->nvar;
    if (prec) *prec = s->prec;
    if (max_exp) *max_exp = s->max_exp;
    if (max_deg) *max_deg = s->max_deg;
    return HC_SUCCESS;
}

// ---------------------------------------------------------------------------------
// FP64 peak probe: CHAINS independent FMA chains per thread, every SM busy.
// ---------------------------------------------------------------------------------
#define PROBE_CHAINS 8
#define PROBE_ITERS 4096

__global__ void k_probe_dfma(double *out, double a, double b)
{
    double v[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) v[c] = threadIdx.x * 1e-3 + c;
#pragma unroll 4
    for (int i = 0; i < PROBE_ITERS; i++) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; c++) v[c] = __fma_rn(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" int hc_probe_fp64_peak(double *gops)
{
    if (!gops) return hc_fail(HC_EINVAL, "gops is NULL");
    const int sms = hc_num_sms(), block = 256, grid = sms * 4;
    double *out = NULL;
    HC_CUDA_TRY(cudaMalloc(&out, sizeof(double) * (size_t)grid * block));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0, 0);
        k_probe_dfma<<<grid, block>>>(out, 0.999999, 1e-7);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return hc_cuda_fail(err, "k_probe_dfma");
    double ops = (double)grid * block * PROBE_ITERS * PROBE_CHAINS;
    *gops = ops / (best * 1e-3) * 1e-9;
    return HC_SUCCESS;
}
