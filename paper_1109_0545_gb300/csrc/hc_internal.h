// hc_internal.h -- library-private state shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/hc.h"

#define HC_KMAX 32     // variables per monomial
#define HC_EXPMAX 64   // exponent bound
#define HC_NMAX 1024   // unknowns

// Device view of a loaded system, passed to kernels by value.
struct DevSys {
    int n, npoly, nmon, nvar;
    int max_exp;        // largest exponent
    const int32_t *mon_ptr;   // [npoly+1]
    const int32_t *var_ptr;   // [nmon+1]
    const int32_t *var_pack;  // [nvar]: index | exponent << 16
    const double *coef;       // [nmon][2][L]
    const int32_t *deg;       // [npoly]
    double gre, gim;          // gamma
    // tables of the block-per-path engine (hc_track_path)
    const int32_t *perm;      // [nmon] monomials ordered by (k, number of exponents >= 2)
    const int32_t *tptr;      // [npoly*(n+1)+1] contributions of entry (i, j), j == n is f_i
    const int32_t *tlist;     // [nvar+nmon] slot in V of each contribution: var_ptr[m]+q for
                              // the partial of monomial m in its q-th variable, nvar+m for
                              // its value; original monomial order within an entry
    const int32_t *eperm;     // [npoly*(n+1)] entries by contribution count, descending (ties
                              // by entry), so the lanes of a warp sum lists of equal length
    // shared-monomial evaluation (polynomials that repeat one another's monomials, e.g. a
    // common support): the distinct non-constant monomials and the terms that use each
    int nuniq;                // distinct non-constant monomials (0: tables not built)
    const int32_t *uvar_ptr;  // [nuniq+1] into uvar_pack
    const int32_t *uvar_pack; // index | exponent << 16, as var_pack
    const int32_t *uuse_ptr;  // [nuniq+1] into uuse
    const int32_t *uuse;      // term index m of each use, increasing within a monomial
    const int32_t *term_row;  // [nmon] the polynomial of term m
    const int32_t *cptr;      // [npoly+1] into cterm
    const int32_t *cterm;     // constant terms (k = 0) of each polynomial, increasing
    const double *ucost;      // [nuniq+1] prefix sums of the distinct monomials' FP64 cost
                              // (evaluation and uses), to cut them into balanced groups
};

struct hc_system {
    int n, npoly, nmon, nvar, prec, max_exp, max_deg;
    int min_deg;
    double gamma[2];
    int device;
    DevSys dev;
    void *dev_block;       // one allocation holding every table
    // workspace, grown on demand
    void *ws;
    size_t ws_bytes;
    // host copies (used to build per-kernel layouts)
    int32_t *h_mon_ptr, *h_var_ptr, *h_var_pack, *h_deg;
    // evaluation scheme of the point kernels: 0 per term (each term's monomial evaluated
    // with its coefficient folded in), 1 shared (each distinct monomial once, then the
    // coefficient products); chosen at load by the FP64 instruction counts of the two,
    // changeable with hc_system_set_eval_mode
    int eval_shared;
    double ops_term, ops_shared;  // FP64 instructions per point of each scheme (DD weights)
    void *dev_shared;             // device block of the shared tables
};

// error reporting (thread-local message)
int hc_fail(int code, const char *fmt, ...);
int hc_cuda_fail(cudaError_t e, const char *what);
#define HC_CUDA_TRY(call)                                         \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return hc_cuda_fail(_e, #call);   \
    } while (0)

// workspace of at least `bytes`, 256-byte aligned; grows (synchronising) if needed
int hc_workspace(hc_system *s, size_t bytes, void **out);

// event timing of the evaluation kernel (hc_prof_enable / hc_prof_read)
bool hc_prof_on(void);
void hc_prof_mark(cudaStream_t st, bool begin);

// number of SMs of the current device (cached)
int hc_num_sms(void);

static inline size_t hc_align256(size_t b) { return (b + 255) & ~(size_t)255; }
