// hc_mlp.cu -- training and inference kernels of the learned step-size proposer.
//
// Training: k_mlp_grad runs the forward and backward pass of a tile of logged corrector
// stages per block (bfloat16 operands, float32 accumulation, every sum in a fixed order)
// and writes the block's partial gradient; k_mlp_reduce sums the partials over blocks in
// block order (so the gradient is bit-reproducible); k_mlp_adamw applies AdamW to the
// float32 master weights.
//
// Loss of a stage with attempted log2 step ratio r and outcome a (1 accepted):
//   z = m - r,  l = softplus(-kappa z) if a else softplus(kappa z),  dl/dm = kappa (sigma(kappa z) - a)
// averaged over the records.
#include "hc_internal.h"
#include "mlp.cuh"

namespace hc {

#define MLP_TILE 64
#define MLP_THREADS 256

__device__ __forceinline__ float softplus_f(float v) { return v > 20.0f ? v : log1pf(expf(v)); }

__global__ void __launch_bounds__(MLP_THREADS) k_mlp_grad(const float *__restrict__ p, int nrec,
                                                          const float *__restrict__ feat,
                                                          const float *__restrict__ target,
                                                          const int32_t *__restrict__ accepted,
                                                          float kappa, float inv_n,
                                                          float *__restrict__ partial)
{
    extern __shared__ float sm[];
    float *W1 = sm;                          // 768
    float *W2 = W1 + MLP_H * MLP_IN;         // 4096
    float *W3 = W2 + MLP_H * MLP_H;          // 64
    float *B1 = W3 + MLP_H;                  // 64
    float *B2 = B1 + MLP_H;                  // 64
    float *X = B2 + MLP_H;                   // TILE x 12
    float *U1 = X + MLP_TILE * MLP_IN;       // TILE x 64 (then dU1)
    float *A1 = U1 + MLP_TILE * MLP_H;       // TILE x 64
    float *U2 = A1 + MLP_TILE * MLP_H;       // TILE x 64 (then dU2)
    float *A2 = U2 + MLP_TILE * MLP_H;       // TILE x 64
    float *DM = A2 + MLP_TILE * MLP_H;       // TILE
    float *LS = DM + MLP_TILE;               // TILE
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * MLP_TILE;
    for (int q = tid; q < MLP_H * MLP_IN; q += MLP_THREADS) W1[q] = bf16r(p[MLP_W1 + q]);
    for (int q = tid; q < MLP_H * MLP_H; q += MLP_THREADS) W2[q] = bf16r(p[MLP_W2 + q]);
    for (int q = tid; q < MLP_H; q += MLP_THREADS) {
        W3[q] = bf16r(p[MLP_W3 + q]);
        B1[q] = p[MLP_B1 + q];
        B2[q] = p[MLP_B2 + q];
    }
    for (int q = tid; q < MLP_TILE * MLP_IN; q += MLP_THREADS) {
        const int s = s0 + q / MLP_IN;
        X[q] = s < nrec ? bf16r(feat[(size_t)s * MLP_IN + q % MLP_IN]) : 0.0f;
    }
    __syncthreads();
    for (int q = tid; q < MLP_TILE * MLP_H; q += MLP_THREADS) {
        const int t = q / MLP_H, o = q % MLP_H;
        float u = B1[o];
        for (int i = 0; i < MLP_IN; i++) u = fmaf(W1[o * MLP_IN + i], X[t * MLP_IN + i], u);
        U1[q] = u;
        A1[q] = bf16r(gelu_f(u));
    }
    __syncthreads();
    for (int q = tid; q < MLP_TILE * MLP_H; q += MLP_THREADS) {
        const int t = q / MLP_H, o = q % MLP_H;
        float u = B2[o];
        for (int i = 0; i < MLP_H; i++) u = fmaf(W2[o * MLP_H + i], A1[t * MLP_H + i], u);
        U2[q] = u;
        A2[q] = bf16r(gelu_f(u));
    }
    __syncthreads();
    if (tid < MLP_TILE) {
        const int s = s0 + tid;
        float dm = 0.0f, ls = 0.0f;
        if (s < nrec) {
            float m = p[MLP_B3];
            for (int i = 0; i < MLP_H; i++) m = fmaf(W3[i], A2[tid * MLP_H + i], m);
            const float z = m - target[s];
            const float a = accepted[s] ? 1.0f : 0.0f;
            const float sig = 1.0f / (1.0f + expf(-kappa * z));
            dm = kappa * (sig - a) * inv_n;
            ls = a > 0.0f ? softplus_f(-kappa * z) : softplus_f(kappa * z);
        }
        DM[tid] = dm;
        LS[tid] = ls;
    }
    __syncthreads();
    // dU2 = dm W3 gelu'(U2), in place
    for (int q = tid; q < MLP_TILE * MLP_H; q += MLP_THREADS) {
        const int t = q / MLP_H, o = q % MLP_H;
        U2[q] = DM[t] * W3[o] * gelu_df(U2[q]);
    }
    __syncthreads();
    // dU1 = (dU2 W2) gelu'(U1), in place
    for (int q = tid; q < MLP_TILE * MLP_H; q += MLP_THREADS) {
        const int t = q / MLP_H, i = q % MLP_H;
        float d = 0.0f;
        for (int o = 0; o < MLP_H; o++) d = fmaf(U2[t * MLP_H + o], W2[o * MLP_H + i], d);
        U1[q] = d * gelu_df(U1[q]);
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * (MLP_NP + 1);
    for (int q = tid; q < MLP_H * MLP_H; q += MLP_THREADS) {    // dW2[o][i]
        const int o = q / MLP_H, i = q % MLP_H;
        float g = 0.0f;
        for (int t = 0; t < MLP_TILE; t++) g = fmaf(U2[t * MLP_H + o], A1[t * MLP_H + i], g);
        out[MLP_W2 + q] = g;
    }
    for (int q = tid; q < MLP_H * MLP_IN; q += MLP_THREADS) {   // dW1[o][i]
        const int o = q / MLP_IN, i = q % MLP_IN;
        float g = 0.0f;
        for (int t = 0; t < MLP_TILE; t++) g = fmaf(U1[t * MLP_H + o], X[t * MLP_IN + i], g);
        out[MLP_W1 + q] = g;
    }
    if (tid < MLP_H) {
        float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
        for (int t = 0; t < MLP_TILE; t++) {
            g1 += U1[t * MLP_H + tid];
            g2 += U2[t * MLP_H + tid];
            g3 = fmaf(DM[t], A2[t * MLP_H + tid], g3);
        }
        out[MLP_B1 + tid] = g1;
        out[MLP_B2 + tid] = g2;
        out[MLP_W3 + tid] = g3;
    }
    if (tid == 0) {
        float g = 0.0f, l = 0.0f;
        for (int t = 0; t < MLP_TILE; t++) {
            g += DM[t];
            l += LS[t];
        }
        out[MLP_B3] = g;
        out[MLP_NP] = l;
    }
}

// grad[q] = sum over blocks of partial[b][q] in block order; loss = sum / nrec
__global__ void k_mlp_reduce(const float *__restrict__ partial, int nblk, float inv_n,
                             float *__restrict__ grad, float *__restrict__ loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > MLP_NP) return;
    float s = 0.0f;
    for (int b = 0; b < nblk; b++) s += partial[(size_t)b * (MLP_NP + 1) + q];
    if (q < MLP_NP)
        grad[q] = s;
    else if (loss)
        *loss = s * inv_n;
}

// AdamW (decoupled weight decay) on the float32 master weights
__global__ void k_mlp_adamw(float *__restrict__ p, float *__restrict__ m1, float *__restrict__ m2,
                            const float *__restrict__ g, float lr, float beta1, float beta2, float eps,
                            float wd, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MLP_NP) return;
    const float gq = g[q];
    const float a = beta1 * m1[q] + (1.0f - beta1) * gq;
    const float b = beta2 * m2[q] + (1.0f - beta2) * gq * gq;
    m1[q] = a;
    m2[q] = b;
    const float mh = a / c1, vh = b / c2;
    p[q] = p[q] - lr * (mh / (sqrtf(vh) + eps) + wd * p[q]);
}

__global__ void k_mlp_forward(const float *__restrict__ p, int nrec, const float *__restrict__ feat,
                              float *__restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nrec) return;
    out[s] = mlp_forward_thread(p, feat + (size_t)s * MLP_IN);
}

static size_t grad_smem()
{
    return sizeof(float) * (MLP_H * MLP_IN + MLP_H * MLP_H + 3 * MLP_H + MLP_TILE * MLP_IN +
                            4 * MLP_TILE * MLP_H + 2 * MLP_TILE);
}

}  // namespace hc

using namespace hc;

// per-device workspace of the partial gradients (grown on demand) and the kernel's
// shared-memory attribute, each keyed by the device that is current at the call
#define HC_MLP_MAX_DEVICES 64
static float *g_mlp_partial[HC_MLP_MAX_DEVICES];
static size_t g_mlp_partial_bytes[HC_MLP_MAX_DEVICES];

extern "C" int hc_mlp_grad(const float *params, int nrec, const float *feat, const float *target,
                           const int32_t *accepted, float kappa, float *grad, float *loss, void *stream)
{
    if (!params || !feat || !target || !accepted || !grad) return hc_fail(HC_EINVAL, "NULL argument");
    if (nrec < 1) return hc_fail(HC_EINVAL, "nrec = %d < 1", nrec);
    if (!(kappa > 0.0f)) return hc_fail(HC_EINVAL, "kappa must be positive");
    int dev = 0;
    HC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= HC_MLP_MAX_DEVICES)
        return hc_fail(HC_EINVAL, "device %d beyond the %d supported", dev, HC_MLP_MAX_DEVICES);
    const int nblk = (nrec + MLP_TILE - 1) / MLP_TILE;
    const size_t need = sizeof(float) * (size_t)nblk * (MLP_NP + 1);
    if (need > g_mlp_partial_bytes[dev]) {
        if (g_mlp_partial[dev]) {
            HC_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(g_mlp_partial[dev]);
            g_mlp_partial[dev] = nullptr;
            g_mlp_partial_bytes[dev] = 0;
        }
        HC_CUDA_TRY(cudaMalloc(&g_mlp_partial[dev], need));
        g_mlp_partial_bytes[dev] = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the dynamic shared-memory limit is a per-device attribute of the kernel
    static bool attr[HC_MLP_MAX_DEVICES];
    if (!attr[dev]) {
        HC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
        attr[dev] = true;
    }
    const float inv_n = 1.0f / (float)nrec;
    k_mlp_grad<<<nblk, MLP_THREADS, grad_smem(), st>>>(params, nrec, feat, target, accepted, kappa, inv_n,
                                                       g_mlp_partial[dev]);
    k_mlp_reduce<<<(MLP_NP + 1 + 255) / 256, 256, 0, st>>>(g_mlp_partial[dev], nblk, inv_n, grad, loss);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_mlp_grad launch");
    return HC_SUCCESS;
}

extern "C" int hc_mlp_adamw(float *params, float *m1, float *m2, const float *grad, int step, float lr,
                            float beta1, float beta2, float eps, float wd, void *stream)
{
    if (!params || !m1 || !m2 || !grad) return hc_fail(HC_EINVAL, "NULL argument");
    if (step < 1) return hc_fail(HC_EINVAL, "step counts from 1");
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_mlp_adamw<<<(MLP_NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m1, m2, grad, lr, beta1, beta2,
                                                                      eps, wd, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_mlp_adamw launch");
    return HC_SUCCESS;
}

extern "C" int hc_mlp_forward(const float *params, int nrec, const float *feat, float *out, void *stream)
{
    if (!params || !feat || !out) return hc_fail(HC_EINVAL, "NULL argument");
    if (nrec < 0) return hc_fail(HC_EINVAL, "nrec < 0");
    if (nrec == 0) return HC_SUCCESS;
    k_mlp_forward<<<(nrec + 127) / 128, 128, 0, (cudaStream_t)stream>>>(params, nrec, feat, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hc_cuda_fail(e, "k_mlp_forward launch");
    return HC_SUCCESS;
}
