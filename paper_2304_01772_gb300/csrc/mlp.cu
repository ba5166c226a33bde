// mlp.cu -- the BF16 surrogate MLP 3 -> 64 -> 64 -> 2 (ReLU) that maps
// (beta, J, h) to (<E>/N, <M>/N).  Not part of the paper; it warm-starts the
// parameter fit.  Weights are held as an FP32 master copy; the kernels round
// weights, the normalised input and both hidden activations to BF16 and
// accumulate in FP32.
//
// Parameter layout (floats): W1[64][3] | b1[64] | W2[64][64] | b2[64] |
// W3[2][64] | b3[2]  (4546 values).
//
// A block takes 64 samples (two warps of 32).  The three 64-wide
// contractions run on the tensor cores as BF16 mma.sync m16n8k16 with FP32
// accumulation, from BF16 tiles in shared memory (ldmatrix): the forward
// z2 = h1 W2^T, and in the backward pass da1 = dz2 W2 and the block's share of
// dL/dW2 = dz2^T h1 (dz2 rounded to BF16 once, and used so in these products
// and in dL/db2).  The thin layers (3 -> 64, 64 -> 2) and the per-sample
// gradient pieces stay on FP32 FMA.  Parameter gradients are reduced in two
// deterministic levels (per-block partials in a fixed order, then a fixed-order
// sum over blocks).
#include <cuda_bf16.h>

#include "internal.h"

namespace spinmc {

namespace {

constexpr int D0 = 3, D1 = 64, D2 = 64, D3 = 2;
constexpr int OW1 = 0, OB1 = OW1 + D1 * D0, OW2 = OB1 + D1, OB2 = OW2 + D2 * D1, OW3 = OB2 + D2,
              OB3 = OW3 + D3 * D2, NPARAM = OB3 + D3;
constexpr int TB = 64;   // samples per block, one thread each
constexpr int NWARPS = TB / 32;
constexpr int OMT = 64 / (16 * NWARPS);   // m-tiles of dL/dW2 rows per warp
constexpr int BS = 72;   // row stride (bf16) of the [rows][64] tiles: 144-byte rows, conflict-free ldmatrix
constexpr int FS = 65;   // row stride (float) of dz1

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Shared-memory layout of a block (byte offsets; all 16-byte aligned).
constexpr size_t SM_W = 0;                                        // float w[NPARAM] (BF16 values)
constexpr size_t SM_W2B = ((NPARAM * 4 + 15) / 16) * 16;          // bf16 W2[64][BS]
constexpr size_t SM_H1 = SM_W2B + 64 * BS * 2;                    // bf16 h1[TB][BS]
constexpr size_t SM_A2 = SM_H1 + TB * BS * 2;                     // bf16 a2[TB][BS]
constexpr size_t SM_XN = SM_A2 + TB * BS * 2;                     // float xn[TB][3]
constexpr size_t SM_FWD = SM_XN + TB * D0 * 4;                    // end of the forward pass's share
constexpr size_t SM_DZ2 = ((SM_FWD + 15) / 16) * 16;              // bf16 dz2[TB][BS]
constexpr size_t SM_DZ1 = SM_DZ2 + TB * BS * 2;                   // float dz1[TB][FS]
constexpr size_t SM_DY = SM_DZ1 + ((TB * FS * 4 + 15) / 16) * 16; // float dy[TB][2]
constexpr size_t SM_LOSS = SM_DY + TB * D3 * 4;                   // float loss[TB]
constexpr size_t SM_BWD = SM_LOSS + TB * 4;

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// D += A B: A 16x16 (row-major fragments), B 16x8 (column-major fragments), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
                 "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Address of the row this lane feeds to ldmatrix.x4 for a 16 x 16 tile at
// (r0, c0) of a [rows][BS] bf16 array: matrix m = lane / 8 covers rows
// r0 + 8 (m & 1) and columns c0 + 8 (m >> 1) (A-fragment order), or with
// swap the other way round (rows r0 + 8 (m >> 1), columns c0 + 8 (m & 1)).
__device__ __forceinline__ uint32_t tile_addr(uint32_t base, int r0, int c0, int lane, bool swap) {
    const int m = lane >> 3, r = lane & 7;
    const int row = r0 + r + 8 * (swap ? (m >> 1) : (m & 1));
    const int col = c0 + 8 * (swap ? (m & 1) : (m >> 1));
    return base + (uint32_t)(row * BS + col) * 2u;
}

// Weights into shared memory (BF16-rounded floats; W2 also as a BF16 tile).
__device__ __forceinline__ void load_weights(const float *params, unsigned char *sm) {
    float *w = reinterpret_cast<float *>(sm + SM_W);
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(sm + SM_W2B);
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) w[k] = bf(params[k]);
    for (int k = threadIdx.x; k < D2 * D1; k += blockDim.x)
        w2[(k / D1) * BS + (k % D1)] = __float2bfloat16_rn(params[OW2 + k]);
    __syncthreads();
}

// Forward pass of the block's samples: xn, h1 and a2 into shared memory
// (zero rows for samples past n); returns this thread's sample output.
__device__ void forward_block(const float *params, const float *mu, const float *inv, const float *X, int n,
                              unsigned char *sm, float &y0, float &y1) {
    load_weights(params, sm);
    const float *w = reinterpret_cast<const float *>(sm + SM_W);
    __nv_bfloat16 *h1 = reinterpret_cast<__nv_bfloat16 *>(sm + SM_H1);
    __nv_bfloat16 *a2 = reinterpret_cast<__nv_bfloat16 *>(sm + SM_A2);
    float *sxn = reinterpret_cast<float *>(sm + SM_XN);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i = blockIdx.x * TB + t;
    const bool live = i < n;
    // layer 1 (3 -> 64) on FMA, one sample per thread
    float xn[D0];
#pragma unroll
    for (int j = 0; j < D0; ++j) {
        xn[j] = live ? bf((X[(size_t)i * D0 + j] - mu[j]) * inv[j]) : 0.0f;
        sxn[t * D0 + j] = xn[j];
    }
    uint32_t *h1w = reinterpret_cast<uint32_t *>(h1 + t * BS);
#pragma unroll 4
    for (int k = 0; k < D1; k += 2) {
        float z0 = w[OB1 + k], z1 = w[OB1 + k + 1];
#pragma unroll
        for (int j = 0; j < D0; ++j) {
            z0 = fmaf(w[OW1 + k * D0 + j], xn[j], z0);
            z1 = fmaf(w[OW1 + (k + 1) * D0 + j], xn[j], z1);
        }
        h1w[k >> 1] = live ? pack_bf2(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f)) : 0u;
    }
    __syncthreads();
    // layer 2 (64 -> 64) on the tensor cores: warp w computes samples 32w .. 32w + 31
    const uint32_t bh1 = (uint32_t)__cvta_generic_to_shared(h1);
    const uint32_t bw2 = (uint32_t)__cvta_generic_to_shared(sm + SM_W2B);
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) ldsm_x4(a[mt], tile_addr(bh1, 32 * warp + 16 * mt, 16 * kk, lane, false));
#pragma unroll
        for (int nt = 0; nt < 8; nt += 2) {
            // W2 rows are the B operand's columns: [b0, b1] of n-tiles nt and nt + 1
            uint32_t b[4];
            ldsm_x4(b, tile_addr(bw2, 8 * nt, 16 * kk, lane, true));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma16816(acc[mt][nt], a[mt], b[0], b[1]);
                mma16816(acc[mt][nt + 1], a[mt], b[2], b[3]);
            }
        }
    }
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int r = 32 * warp + 16 * mt + g, col = 8 * nt + 2 * c;
            const float bb0 = w[OB2 + col], bb1 = w[OB2 + col + 1];
            const bool l0 = blockIdx.x * TB + r < n, l1 = blockIdx.x * TB + r + 8 < n;
            reinterpret_cast<uint32_t *>(a2 + r * BS)[col >> 1] =
                l0 ? pack_bf2(fmaxf(acc[mt][nt][0] + bb0, 0.0f), fmaxf(acc[mt][nt][1] + bb1, 0.0f)) : 0u;
            reinterpret_cast<uint32_t *>(a2 + (r + 8) * BS)[col >> 1] =
                l1 ? pack_bf2(fmaxf(acc[mt][nt][2] + bb0, 0.0f), fmaxf(acc[mt][nt][3] + bb1, 0.0f)) : 0u;
        }
    __syncthreads();
    // layer 3 (64 -> 2) on FMA, one sample per thread
    y0 = w[OB3];
    y1 = w[OB3 + 1];
    const __nv_bfloat162 *a2r = reinterpret_cast<const __nv_bfloat162 *>(a2 + t * BS);
#pragma unroll 8
    for (int o = 0; o < D2; o += 2) {
        const float2 av = __bfloat1622float2(a2r[o >> 1]);
        y0 = fmaf(w[OW3 + o], av.x, y0);
        y1 = fmaf(w[OW3 + D2 + o], av.x, y1);
        y0 = fmaf(w[OW3 + o + 1], av.y, y0);
        y1 = fmaf(w[OW3 + D2 + o + 1], av.y, y1);
    }
}

__global__ void __launch_bounds__(TB) mlp_forward_kernel(const float *params, const float *mu,
                                                         const float *inv, const float *X, int n,
                                                         float *Y) {
    extern __shared__ __align__(16) unsigned char sm[];
    float y0, y1;
    forward_block(params, mu, inv, X, n, sm, y0, y1);
    const int i = blockIdx.x * TB + threadIdx.x;
    if (i < n) {
        Y[2 * (size_t)i] = y0;
        Y[2 * (size_t)i + 1] = y1;
    }
}

// Backward of a block of TB samples: partial gradients of the block into
// part[blockIdx.x][NPARAM + 1] (last slot: partial loss).
__global__ void __launch_bounds__(TB) mlp_backward_kernel(const float *params, const float *mu,
                                                          const float *inv, const float *X,
                                                          const float *T, int n, float *part,
                                                          float *dX) {
    extern __shared__ __align__(16) unsigned char sm[];
    float y0, y1;
    forward_block(params, mu, inv, X, n, sm, y0, y1);
    const float *w = reinterpret_cast<const float *>(sm + SM_W);
    const __nv_bfloat16 *h1 = reinterpret_cast<const __nv_bfloat16 *>(sm + SM_H1);
    const __nv_bfloat16 *a2 = reinterpret_cast<const __nv_bfloat16 *>(sm + SM_A2);
    const float *sxn = reinterpret_cast<const float *>(sm + SM_XN);
    __nv_bfloat16 *dz2 = reinterpret_cast<__nv_bfloat16 *>(sm + SM_DZ2);
    float *dz1 = reinterpret_cast<float *>(sm + SM_DZ1);
    float *sdy = reinterpret_cast<float *>(sm + SM_DY);
    float *sloss = reinterpret_cast<float *>(sm + SM_LOSS);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int i = blockIdx.x * TB + t;
    const bool live = i < n;
    const float invn = 1.0f / (float)n;
    // output error, loss, and dz2 = (W3^T dy) [a2 > 0], rounded to BF16 once
    const float e0 = live ? y0 - T[2 * (size_t)i] : 0.0f, e1 = live ? y1 - T[2 * (size_t)i + 1] : 0.0f;
    const float dy0 = e0 * invn, dy1 = e1 * invn;
    sdy[t * D3] = dy0;
    sdy[t * D3 + 1] = dy1;
    sloss[t] = 0.5f * (e0 * e0 + e1 * e1) * invn;
    {
        const __nv_bfloat162 *a2r = reinterpret_cast<const __nv_bfloat162 *>(a2 + t * BS);
        uint32_t *dzr = reinterpret_cast<uint32_t *>(dz2 + t * BS);
#pragma unroll 8
        for (int o = 0; o < D2; o += 2) {
            const float2 av = __bfloat1622float2(a2r[o >> 1]);
            const float d0 = w[OW3 + o] * dy0 + w[OW3 + D2 + o] * dy1;
            const float d1 = w[OW3 + o + 1] * dy0 + w[OW3 + D2 + o + 1] * dy1;
            dzr[o >> 1] = pack_bf2(av.x > 0.0f ? d0 : 0.0f, av.y > 0.0f ? d1 : 0.0f);
        }
    }
    __syncthreads();
    const int g = lane >> 2, c = lane & 3;
    const uint32_t bdz2 = (uint32_t)__cvta_generic_to_shared(dz2);
    const uint32_t bh1 = (uint32_t)__cvta_generic_to_shared(sm + SM_H1);
    const uint32_t bw2 = (uint32_t)__cvta_generic_to_shared(sm + SM_W2B);
    // da1 = dz2 W2 (tensor cores; warp w: samples 32w .. 32w + 31), dz1 = da1 [h1 > 0]
    {
        float acc[2][8][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) ldsm_x4(a[mt], tile_addr(bdz2, 32 * warp + 16 * mt, 16 * kk, lane, false));
#pragma unroll
            for (int nt = 0; nt < 8; nt += 2) {
                // B[k = o][n = j] = W2[o][j]: W2's rows transposed into the fragments
                uint32_t b[4];
                ldsm_x4_t(b, tile_addr(bw2, 16 * kk, 8 * nt, lane, false));
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma16816(acc[mt][nt], a[mt], b[0], b[1]);
                    mma16816(acc[mt][nt + 1], a[mt], b[2], b[3]);
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int r = 32 * warp + 16 * mt + g, col = 8 * nt + 2 * c;
                const float2 h0 = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(h1 + r * BS)[col >> 1]);
                const float2 h8 = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(h1 + (r + 8) * BS)[col >> 1]);
                dz1[r * FS + col] = h0.x > 0.0f ? acc[mt][nt][0] : 0.0f;
                dz1[r * FS + col + 1] = h0.y > 0.0f ? acc[mt][nt][1] : 0.0f;
                dz1[(r + 8) * FS + col] = h8.x > 0.0f ? acc[mt][nt][2] : 0.0f;
                dz1[(r + 8) * FS + col + 1] = h8.y > 0.0f ? acc[mt][nt][3] : 0.0f;
            }
    }
    float *out = part + (size_t)blockIdx.x * (NPARAM + 1);
    // the block's dL/dW2 = dz2^T h1 over its samples (tensor cores; warp w:
    // rows o = 16 OMT w .. 16 OMT (w + 1) - 1)
    {
        float acc[OMT][8][4];
#pragma unroll
        for (int mt = 0; mt < OMT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < TB / 16; ++kk) {
            // A[m = o][k = s] = dz2[s][o]: dz2's 16 x 16 tiles transposed
            uint32_t a[OMT][4];
#pragma unroll
            for (int mt = 0; mt < OMT; ++mt)
                ldsm_x4_t(a[mt], tile_addr(bdz2, 16 * kk, 16 * (OMT * warp + mt), lane, true));
#pragma unroll
            for (int nt = 0; nt < 8; nt += 2) {
                // B[k = s][n = j] = h1[s][j]
                uint32_t b[4];
                ldsm_x4_t(b, tile_addr(bh1, 16 * kk, 8 * nt, lane, false));
#pragma unroll
                for (int mt = 0; mt < OMT; ++mt) {
                    mma16816(acc[mt][nt], a[mt], b[0], b[1]);
                    mma16816(acc[mt][nt + 1], a[mt], b[2], b[3]);
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < OMT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int o = 16 * (OMT * warp + mt) + g, j = 8 * nt + 2 * c;
                out[OW2 + o * D1 + j] = acc[mt][nt][0];
                out[OW2 + o * D1 + j + 1] = acc[mt][nt][1];
                out[OW2 + (o + 8) * D1 + j] = acc[mt][nt][2];
                out[OW2 + (o + 8) * D1 + j + 1] = acc[mt][nt][3];
            }
    }
    __syncthreads();
    // dX = (W1^T dz1) inv, one sample per thread
    if (dX && live) {
#pragma unroll
        for (int j = 0; j < D0; ++j) {
            float accx = 0.0f;
            for (int k = 0; k < D1; ++k) accx = fmaf(w[OW1 + k * D0 + j], dz1[t * FS + k], accx);
            dX[(size_t)i * D0 + j] = accx * inv[j];
        }
    }
    // the other parameter gradients: each thread owns a strided set of
    // parameters and sums over the block's samples in a fixed order
    for (int p = threadIdx.x; p < NPARAM + 1; p += TB) {
        if (p >= OW2 && p < OB2) continue;   // dL/dW2: the tensor-core pass above
        float accp = 0.0f;
        if (p < OB1) {                       // W1[k][j]
            const int k = p / D0, j = p - k * D0;
            for (int q = 0; q < TB; ++q) accp = fmaf(dz1[q * FS + k], sxn[q * D0 + j], accp);
        } else if (p < OW2) {                // b1[k]
            const int k = p - OB1;
            for (int q = 0; q < TB; ++q) accp += dz1[q * FS + k];
        } else if (p < OW3) {                // b2[o]
            const int o = p - OB2;
            for (int q = 0; q < TB; ++q) accp += __bfloat162float(dz2[q * BS + o]);
        } else if (p < OB3) {                // W3[j][o]
            const int j = (p - OW3) / D2, o = (p - OW3) - j * D2;
            for (int q = 0; q < TB; ++q) accp = fmaf(sdy[q * D3 + j], __bfloat162float(a2[q * BS + o]), accp);
        } else if (p < NPARAM) {             // b3[j]
            const int j = p - OB3;
            for (int q = 0; q < TB; ++q) accp += sdy[q * D3 + j];
        } else {                             // loss
            for (int q = 0; q < TB; ++q) accp += sloss[q];
        }
        out[p] = accp;
    }
}

// Sum of the blocks' partials per parameter in a fixed order, so every call
// gives the same bits: a block takes 32 parameters; its eight warps each sum
// every eighth partial of all 32 (lanes over parameters: coalesced), and
// warp 0 adds the eight sums in order.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(32 * kRedWarps) mlp_reduce_kernel(const float *part, int nblk, float *grad,
                                                                    float *loss) {
    __shared__ float sums[kRedWarps][32];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (p < NPARAM + 1)
        for (int b = wq; b < nblk; b += kRedWarps) acc += part[(size_t)b * (NPARAM + 1) + p];
    sums[wq][lane] = acc;
    __syncthreads();
    if (wq == 0 && p < NPARAM + 1) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < kRedWarps; ++k) t += sums[k][lane];
        if (p < NPARAM)
            grad[p] = t;
        else if (loss)
            *loss = t;
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

}  // namespace

int mlp_param_count() { return NPARAM; }

cudaError_t launch_mlp_forward(const float *params, const float *mu, const float *inv_sigma,
                               const float *X, int n, float *Y, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SM_FWD);
    if (e) return e;
    mlp_forward_kernel<<<(n + TB - 1) / TB, TB, SM_FWD, s>>>(params, mu, inv_sigma, X, n, Y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_backward(const float *params, const float *mu, const float *inv_sigma,
                                const float *X, const float *T, int n, float *grad, float *loss,
                                float *dX, cudaStream_t s) {
    if (n <= 0) return cudaErrorInvalidValue;
    const int nblk = (n + TB - 1) / TB;
    const size_t smem = SM_BWD;
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    float *part = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&part), sizeof(float) * (size_t)nblk * (NPARAM + 1), s);
    if (e) return e;
    mlp_backward_kernel<<<nblk, TB, smem, s>>>(params, mu, inv_sigma, X, T, n, part, dX);
    mlp_reduce_kernel<<<(NPARAM + 1 + 31) / 32, 32 * kRedWarps, 0, s>>>(part, nblk, grad, loss);
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
