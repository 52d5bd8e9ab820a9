// hc_noalloc.cu -- hc_eval_jac_noalloc: the evaluation entry point for callers that
// cannot allocate device memory.
//
// hc_eval_jac keeps its workspace (the power table x_j^e) in memory it allocates on first
// use.  Some callers cannot allow that: a process that hands all device memory to its own
// pool allocator (a framework's caching allocator, a server with a memory budget reserved
// at start-up) would see a library cudaMalloc fail or fragment its pool, and cudaMalloc /
// cudaFree may synchronise the device in the middle of a latency-critical loop.  This
// variant allocates nothing: its workspace is the fixed device array below, compiled into
// the library.
#include <mutex>

#include "hc_eval.cuh"

// Size of the fixed workspace.  A device keeps it from the first call of this entry point
// on that device (or from module load, without lazy module loading) until process exit.
#define HC_NOALLOC_SCRATCH_BYTES (32u << 20)
#define HC_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[HC_NOALLOC_SCRATCH_BYTES / sizeof(double)];

// The array's device address per device.  In host code the symbol names a host-side
// stand-in, never the device memory, so the address must come from cudaGetSymbolAddress,
// called with the device current.
static double *g_noalloc_addr[HC_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_lock;

static int noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hc_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= HC_NOALLOC_MAX_DEVICES)
        return hc_fail(HC_EINVAL, "device %d beyond the %d devices supported", dev, HC_NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> guard(g_noalloc_lock);
    if (!g_noalloc_addr[dev]) {
        void *p = NULL;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return hc_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = (double *)p;
    }
    *out = g_noalloc_addr[dev];
    return HC_SUCCESS;
}

extern "C" int hc_eval_jac_noalloc(hc_system *s, int npts, double t, const double *x, double *f,
                                   double *J, void *stream)
{
    int rc = hc_check_eval_args(s, npts, t);
    if (rc) return rc;
    if (npts == 0) return HC_SUCCESS;
    if (!x || !f) return hc_fail(HC_EINVAL, "x or f is NULL");
    const size_t need = hc_pw_bytes(s, npts);
    if (need > HC_NOALLOC_SCRATCH_BYTES)
        return hc_fail(HC_EINVAL,
                       "hc_eval_jac_noalloc: %d points need %zu bytes of workspace, more than its "
                       "fixed %u bytes; evaluate at most %zu points per call",
                       npts, need, HC_NOALLOC_SCRATCH_BYTES,
                       (size_t)npts * HC_NOALLOC_SCRATCH_BYTES / need);
    double *pw = NULL;
    rc = noalloc_scratch(&pw);
    if (rc) return rc;
    // The power table is written in full by this call before it is read, so the previous
    // call's contents need no clearing.
    // (the shared scheme runs its row groups here: no room for partial sums)
    return hc_eval_dispatch(s, npts, t, x, pw, f, J, NULL, hc_eval_tiles(), (cudaStream_t)stream);
}
