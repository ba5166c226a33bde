// mlp.cu -- the BF16 surrogate MLP 3 -> 64 -> 64 -> 2 (ReLU) that maps
// (beta, J, h) to (<E>/N, <M>/N).  Not part of the paper; it warm-starts the
// parameter fit.  Weights are held as an FP32 master copy; the kernels round
// weights, the normalised input and both hidden activations to BF16 and
// accumulate in FP32.
//
// Parameter layout (floats): W1[64][3] | b1[64] | W2[64][64] | b2[64] |
// W3[2][64] | b3[2]  (4546 values).
//
// The network is tiny (4.5k parameters, batches of at most ~10^4 samples):
// one training step is ~0.1 GFLOP, far below a microsecond of tensor-core
// time, so the kernels are latency-bound and use plain FP32 FMA with weights
// broadcast from shared memory.  The backward pass reduces gradients in two
// deterministic levels (per-block partials, then a fixed-order sum).
#include <cuda_bf16.h>

#include "internal.h"

namespace spinmc {

namespace {

constexpr int D0 = 3, D1 = 64, D2 = 64, D3 = 2;
constexpr int OW1 = 0, OB1 = OW1 + D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + D2 * D1, OW3 = OB2 + D2,
              OB3 = OW3 + D3 * D2, NPARAM = OB3 + D3;
constexpr int TB = 128;  // samples per block
constexpr int PD = 65;   // padded row stride of the per-sample activations (bank-conflict free)

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void load_weights(const float *params, float *w) {
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) w[k] = bf(params[k]);
    __syncthreads();
}

// Forward of one sample; h1 and a2 (BF16-rounded activations) optionally kept.
__device__ __forceinline__ void forward_one(const float *w, const float *x, float *xn,
                                            const float *mu, const float *inv, float *h1,
                                            float *a2, float &y0, float &y1) {
#pragma unroll
    for (int j = 0; j < D0; ++j) xn[j] = bf((x[j] - mu[j]) * inv[j]);
#pragma unroll 8
    for (int k = 0; k < D1; ++k) {
        float z = w[OB1 + k];
#pragma unroll
        for (int j = 0; j < D0; ++j) z = fmaf(w[OW1 + k * D0 + j], xn[j], z);
        h1[k] = bf(fmaxf(z, 0.0f));
    }
    y0 = w[OB3];
    y1 = w[OB3 + 1];
    for (int o = 0; o < D2; ++o) {
        float z = w[OB2 + o];
#pragma unroll 16
        for (int k = 0; k < D1; ++k) z = fmaf(w[OW2 + o * D1 + k], h1[k], z);
        const float a = bf(fmaxf(z, 0.0f));
        if (a2) a2[o] = a;
        y0 = fmaf(w[OW3 + o], a, y0);
        y1 = fmaf(w[OW3 + D2 + o], a, y1);
    }
}

__global__ void __launch_bounds__(TB) mlp_forward_kernel(const float *params, const float *mu,
                                                         const float *inv, const float *X, int n,
                                                         float *Y) {
    __shared__ float w[NPARAM];
    load_weights(params, w);
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i >= n) return;
    float x[D0], xn[D0], h1[D1], y0, y1;
    const float m[D0] = {mu[0], mu[1], mu[2]}, iv[D0] = {inv[0], inv[1], inv[2]};
#pragma unroll
    for (int j = 0; j < D0; ++j) x[j] = X[(size_t)i * D0 + j];
    forward_one(w, x, xn, m, iv, h1, nullptr, y0, y1);
    Y[2 * (size_t)i] = y0;
    Y[2 * (size_t)i + 1] = y1;
}

// Backward of a block of TB samples: partial gradients of the block into
// part[blockIdx.x][NPARAM + 1] (last slot: partial loss).
__global__ void __launch_bounds__(TB) mlp_backward_kernel(const float *params, const float *mu,
                                                          const float *inv, const float *X,
                                                          const float *T, int n, float *part,
                                                          float *dX) {
    extern __shared__ float sm[];
    float *w = sm;                   // NPARAM
    float *sh1 = w + NPARAM;         // [TB][PD]  activations layer 1
    float *sdz2 = sh1 + TB * PD;     // [TB][PD]  dL/dz2
    float *sa2 = sdz2 + TB * PD;     // [TB][PD]  activations layer 2
    float *sdz1 = sa2 + TB * PD;     // [TB][PD]  dL/dz1
    float *sxn = sdz1 + TB * PD;     // [TB][D0]
    float *sdy = sxn + TB * D0;      // [TB][D3]
    float *sloss = sdy + TB * D3;    // [TB]
    load_weights(params, w);
    const int s = threadIdx.x;
    const int i = blockIdx.x * TB + s;
    const float invn = 1.0f / (float)n;
    if (i < n) {
        float x[D0], xn[D0], y0, y1;
        const float m[D0] = {mu[0], mu[1], mu[2]}, iv[D0] = {inv[0], inv[1], inv[2]};
#pragma unroll
        for (int j = 0; j < D0; ++j) x[j] = X[(size_t)i * D0 + j];
        forward_one(w, x, xn, m, iv, sh1 + s * PD, sa2 + s * PD, y0, y1);
#pragma unroll
        for (int j = 0; j < D0; ++j) sxn[s * D0 + j] = xn[j];
        const float e0 = y0 - T[2 * (size_t)i], e1 = y1 - T[2 * (size_t)i + 1];
        sdy[s * D3] = e0 * invn;
        sdy[s * D3 + 1] = e1 * invn;
        sloss[s] = 0.5f * (e0 * e0 + e1 * e1) * invn;
        // dz2 = (W3^T dy) * [a2 > 0]
        for (int o = 0; o < D2; ++o) {
            const float da = w[OW3 + o] * sdy[s * D3] + w[OW3 + D2 + o] * sdy[s * D3 + 1];
            sdz2[s * PD + o] = sa2[s * PD + o] > 0.0f ? da : 0.0f;
        }
        // dz1 = (W2^T dz2) * [h1 > 0]
        for (int k = 0; k < D1; ++k) {
            float acc = 0.0f;
            for (int o = 0; o < D2; ++o) acc = fmaf(w[OW2 + o * D1 + k], sdz2[s * PD + o], acc);
            sdz1[s * PD + k] = sh1[s * PD + k] > 0.0f ? acc : 0.0f;
        }
        if (dX) {
#pragma unroll
            for (int j = 0; j < D0; ++j) {
                float acc = 0.0f;
                for (int k = 0; k < D1; ++k) acc = fmaf(w[OW1 + k * D0 + j], sdz1[s * PD + k], acc);
                dX[(size_t)i * D0 + j] = acc * iv[j];
            }
        }
    } else {
        for (int k = 0; k < D1; ++k) sh1[s * PD + k] = 0.0f, sdz1[s * PD + k] = 0.0f;
        for (int o = 0; o < D2; ++o) sdz2[s * PD + o] = 0.0f, sa2[s * PD + o] = 0.0f;
        for (int j = 0; j < D0; ++j) sxn[s * D0 + j] = 0.0f;
        sdy[s * D3] = sdy[s * D3 + 1] = 0.0f;
        sloss[s] = 0.0f;
    }
    __syncthreads();
    float *out = part + (size_t)blockIdx.x * (NPARAM + 1);
    // parameter gradients: each thread owns a strided set of parameters and
    // sums over the block's samples in a fixed order.
    for (int p = threadIdx.x; p < NPARAM + 1; p += TB) {
        float acc = 0.0f;
        if (p < OB1) {                       // W1[k][j]
            const int k = p / D0, j = p - k * D0;
            for (int q = 0; q < TB; ++q) acc = fmaf(sdz1[q * PD + k], sxn[q * D0 + j], acc);
        } else if (p < OW2) {                // b1[k]
            const int k = p - OB1;
            for (int q = 0; q < TB; ++q) acc += sdz1[q * PD + k];
        } else if (p < OB2) {                // W2[o][k]
            const int o = (p - OW2) / D1, k = (p - OW2) - o * D1;
            for (int q = 0; q < TB; ++q) acc = fmaf(sdz2[q * PD + o], sh1[q * PD + k], acc);
        } else if (p < OW3) {                // b2[o]
            const int o = p - OB2;
            for (int q = 0; q < TB; ++q) acc += sdz2[q * PD + o];
        } else if (p < OB3) {                // W3[j][o]
            const int j = (p - OW3) / D2, o = (p - OW3) - j * D2;
            for (int q = 0; q < TB; ++q) acc = fmaf(sdy[q * D3 + j], sa2[q * PD + o], acc);
        } else if (p < NPARAM) {             // b3[j]
            const int j = p - OB3;
            for (int q = 0; q < TB; ++q) acc += sdy[q * D3 + j];
        } else {                             // loss
            for (int q = 0; q < TB; ++q) acc += sloss[q];
        }
        out[p] = acc;
    }
}

__global__ void mlp_reduce_kernel(const float *part, int nblk, float *grad, float *loss) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPARAM + 1; p += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * (NPARAM + 1) + p];
        if (p < NPARAM)
            grad[p] = acc;
        else if (loss)
            *loss = acc;
    }
}

__global__ void mlp_adam_kernel(float *params, const float *grad, float *m, float *v, int n, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        float pp = params[p], mm = m[p], vv = v[p];
        adam_element(pp, mm, vv, grad[p], lr, b1, b2, eps, c1, c2);
        m[p] = mm;
        v[p] = vv;
        params[p] = pp;
    }
}

size_t backward_smem() {
    return sizeof(float) * (size_t)(NPARAM + TB * (4 * PD + D0 + D3 + 1));
}

}  // namespace

int mlp_param_count() { return NPARAM; }

cudaError_t launch_mlp_forward(const float *params, const float *mu, const float *inv_sigma,
                               const float *X, int n, float *Y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(n + TB - 1) / TB, TB, 0, s>>>(params, mu, inv_sigma, X, n, Y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *params, const float *mu, const float *inv_sigma,
                                const float *X, const float *T, int n, float *grad, float *loss,
                                float *dX, cudaStream_t s) {
    if (n <= 0) return cudaErrorInvalidValue;
    const int nblk = (n + TB - 1) / TB;
    const size_t smem = backward_smem();
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    float *part = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&part), sizeof(float) * (size_t)nblk * (NPARAM + 1), s);
    if (e) return e;
    mlp_backward_kernel<<<nblk, TB, smem, s>>>(params, mu, inv_sigma, X, T, n, part, dX);
    mlp_reduce_kernel<<<(NPARAM + 256) / 256, 256, 0, s>>>(part, nblk, grad, loss);
    e = cudaGetLastError();
    cudaError_t f = cudaFreeAsync(part, s);
    return e ? e : f;
}

cudaError_t launch_adam(float *params, const float *grad, float *m, float *v, int n, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    float c1, c2;
    adam_bias(step, b1, b2, c1, c2);
    int blocks = (n + 255) / 256;
    blocks = blocks > 1024 ? 1024 : blocks;
    mlp_adam_kernel<<<blocks, 256, 0, s>>>(params, grad, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *params, const float *grad, float *m, float *v, int step,
                            float lr, float b1, float b2, float eps, cudaStream_t s) {
    return launch_adam(params, grad, m, v, NPARAM, step, lr, b1, b2, eps, s);
}

}  // namespace spinmc
