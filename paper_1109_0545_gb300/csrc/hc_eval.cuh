// hc_eval.cuh -- evaluation entry points shared between translation units.
#pragma once
#include "points.cuh"

struct EvalTiles {
    int rows_per_task = 0;  // polynomials per warp task (0 = automatic)
    int blocks_per_sm = 0;  // resident 4-warp blocks per SM (0 = automatic)
};

namespace hc {
template <int L>
int launch_eval(const DevSys &S, int npts, double t, const double *X, double *PW, double *F,
                double *J, const EvalTiles &tiles, cudaStream_t st);
// the shared-monomial scheme (hc_shared.cu); part: hc_shared_part_bytes of workspace for
// the monomial groups' partial sums, or NULL (row groups only)
template <int L>
int launch_eval_shared(const hc_system *s, int npts, double t, const double *X, double *PW, double *F, double *J,
                       double *part, cudaStream_t st);
// the power table PW of the points X (k_powers)
template <int L>
void launch_powers(int grid, int n, int npts, int max_exp, const double *X, double *PW, cudaStream_t st);
}

EvalTiles &hc_eval_tiles();  // process-wide tile choice (hc_set_tiles)
size_t hc_pw_bytes(const hc_system *s, int npts);
size_t hc_shared_part_bytes(const hc_system *s, int npts, bool jac);
int hc_check_eval_args(const hc_system *s, int npts, double t);
int hc_eval_dispatch(hc_system *s, int npts, double t, const double *x, double *pw, double *f,
                     double *J, double *part, const EvalTiles &tiles, cudaStream_t st);
