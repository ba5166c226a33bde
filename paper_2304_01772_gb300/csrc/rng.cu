// rng.cu -- the Philox4x32-10 stream of the sweeps on its own.
//
// Every Ising update consumes one 32-bit word of Philox4x32-10 (Salmon et al.,
// SC'11) keyed by the seed, counter (g, lattice, sweep, colour); Potts and CPM
// updates consume two.  This kernel draws the blocks of a range of g with the
// same code path as the sweeps (the two g-independent products of rounds 1 and
// 2 hoisted, round keys from the kernel parameters) and reduces them to one
// XOR digest.  Compared with an independent implementation it checks the
// stream; timed, it is the rate at which this GPU can produce the draws alone,
// an upper bound on the update rate of any sweep that uses this stream.
#include "internal.h"
#include "strip.cuh"

namespace spinmc {

namespace {

constexpr int kRngThreads = 256;

__global__ void __launch_bounds__(kRngThreads) philox_xor_kernel(uint32_t g0, uint32_t n, uint32_t lat,
                                                                 uint32_t t, uint32_t c, PhiloxKeys rk,
                                                                 uint32_t *out) {
    const PhiloxPrefix P = philox_prefix(lat, t, c, rk);
    uint32_t acc = 0;
    const uint32_t stride = gridDim.x * kRngThreads;
    for (uint32_t i = blockIdx.x * kRngThreads + threadIdx.x; i < n; i += stride) {
        const uint4 r = philox_from_prefix(g0 + i, P, rk);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicXor(out, acc);
}

}  // namespace

cudaError_t launch_philox_xor(uint32_t g0, uint32_t n, uint32_t lat, uint32_t t, uint32_t c,
                              uint32_t k0, uint32_t k1, uint32_t *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    if (e || n == 0) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    // eight resident blocks per SM, each thread drawing many blocks in turn
    const uint32_t want = (n + kRngThreads - 1) / kRngThreads;
    const uint32_t grid = want < (uint32_t)(8 * sms) ? want : (uint32_t)(8 * sms);
    philox_xor_kernel<<<grid, kRngThreads, 0, s>>>(g0, n, lat, t, c, philox_keys(k0, k1), out);
    return cudaGetLastError();
}

}  // namespace spinmc
