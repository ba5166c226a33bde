// sweep_potts.cu -- checkerboard Metropolis sweeps of batched q-state Potts
// lattices (Sec. "Potts model" of Farias et al., arXiv 2304.01772: a site
// proposes one of the q - 1 other states; H = -J sum delta(s_i, s_j)).
//
// Spins are uint8 in [0, q).  Per active site the proposal is
// s' = (s + 1 + mulhi(u1, q - 1)) mod q and the table key is
// d = n_same(s) - n_same(s') + 4 in [0, 8] (dE = J d).  The kernel forms the
// equality counts directly instead of the paper's four one-hot convolutions.
//
// Statistics per lattice: (B_eq, n_0, .., n_{q-1}).  B_eq changes by -d on
// acceptance (table delta); the state counts change by -1 / +1.  For q <= 8
// each thread keeps the count changes in two 64-bit words of four signed
// 16-bit fields; larger q use a shared-memory histogram.
#include "internal.h"

namespace spinmc {

namespace {

struct PottsAcc {
    int b;                    // sum of dB_eq
    unsigned long long lo;    // states 0..3, 16-bit signed fields
    unsigned long long hi;    // states 4..7
};

__device__ __forceinline__ void potts_count(PottsAcc &a, uint32_t s, long long sign,
                                            int *shist, bool small_q) {
    if (small_q) {
        const unsigned long long v = (unsigned long long)(sign) << (16u * (s & 3u));
        if (s & 4u)
            a.hi += v;
        else
            a.lo += v;
    } else {
        atomicAdd(shist + (s & 0xFFu), (int)sign);
    }
}

// Update the colour-`c` sites of one 16-byte row chunk; Philox group of word
// i is gbase + i, active bytes p and p + 2 use lanes (0, 1) and (2, 3).
__device__ __forceinline__ uint4 potts_chunk(uint4 C, uint4 U, uint4 D, uint32_t lw, uint32_t rw,
                                             uint32_t gbase, int p, uint32_t lat, uint32_t t,
                                             uint32_t c, uint32_t k0, uint32_t k1, uint32_t q,
                                             const TabEntry *stab, bool count, PottsAcc &acc,
                                             int *shist, bool small_q) {
    const uint32_t w[6] = {lw, C.x, C.y, C.z, C.w, rw};
    const uint32_t up[4] = {U.x, U.y, U.z, U.w};
    const uint32_t dn[4] = {D.x, D.y, D.z, D.w};
    uint32_t out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 r = philox4x32_10(make_uint4(gbase + (uint32_t)i, lat, t, c), k0, k1);
        const uint32_t W = w[i + 1];
        const uint32_t lf = __funnelshift_l(w[i], W, 8);
        const uint32_t rt = __funnelshift_r(W, w[i + 2], 8);
        uint32_t nw = W;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const uint32_t sh = 8u * (uint32_t)(p + 2 * bb);
            const uint32_t s = (W >> sh) & 0xFFu;
            const uint32_t nu = (up[i] >> sh) & 0xFFu, nd = (dn[i] >> sh) & 0xFFu;
            const uint32_t nl = (lf >> sh) & 0xFFu, nr = (rt >> sh) & 0xFFu;
            const uint32_t u0 = bb ? r.z : r.x;
            const uint32_t u1 = bb ? r.w : r.y;
            uint32_t sp = s + 1u + __umulhi(u1, q - 1u);
            sp = sp >= q ? sp - q : sp;
            const int n_old = (nu == s) + (nd == s) + (nl == s) + (nr == s);
            const int n_new = (nu == sp) + (nd == sp) + (nl == sp) + (nr == sp);
            const TabEntry e = stab[n_old - n_new + 4];
            if (u0 <= e.thr) {
                nw = (nw & ~(0xFFu << sh)) | ((sp & 0xFFu) << sh);
                if (count && s < q) {
                    acc.b += e.delta;
                    potts_count(acc, s, -1, shist, small_q);
                    potts_count(acc, sp, 1, shist, small_q);
                }
            }
        }
        out[i] = nw;
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}

// Per-thread sums -> one atomic per statistic per block.
template <int THREADS>
__device__ void flush_potts_acc(const PottsAcc &acc, int q, int64_t *delta_lat, int *red,
                                int *shist, bool small_q) {
    int f[9];
    f[0] = acc.b;
    unsigned long long v = acc.lo;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = (int)(int16_t)(v & 0xFFFFull);
        f[1 + k] = x;
        v = (v - (unsigned long long)(long long)x) >> 16;
    }
    v = acc.hi;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = (int)(int16_t)(v & 0xFFFFull);
        f[5 + k] = x;
        v = (v - (unsigned long long)(long long)x) >> 16;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f[k] += __shfl_xor_sync(0xFFFFFFFFu, f[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 9; ++k) red[9 * warp + k] = f[k];
    __syncthreads();
    const int nk = small_q ? q + 1 : 1;
    if (threadIdx.x < nk) {
        long long s = 0;
        for (int w = 0; w < THREADS / 32; ++w) s += red[9 * w + threadIdx.x];
        if (s) atomicAdd(reinterpret_cast<unsigned long long *>(delta_lat + threadIdx.x), (unsigned long long)s);
    }
    if (!small_q) {
        for (int k = threadIdx.x; k < q; k += THREADS) {
            const int s = shist[k];
            if (s) atomicAdd(reinterpret_cast<unsigned long long *>(delta_lat + 1 + k), (unsigned long long)(long long)s);
            shist[k] = 0;
        }
    }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) potts_fused_kernel(PottsSweepArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ TabEntry stab[kTabStride];
    __shared__ int red[9 * (THREADS / 32)];
    __shared__ int shist[256];
    uint4 *sm4 = reinterpret_cast<uint4 *>(sm);
    const uint32_t *sm32 = reinterpret_cast<const uint32_t *>(sm);
    for (int k = threadIdx.x; k < 256; k += THREADS) shist[k] = 0;
    const uint32_t t = a.state->t;
    for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
        const Item w = a.items[it];
        const LatDev ld = a.lats[w.lat];
        const int L = ld.L, Lv = L >> 4;
        const uint32_t q = (uint32_t)ld.q;
        const bool small_q = q <= 8;
        const int halo = w.whole ? 0 : 2;
        const int nload = w.nrows + 2 * halo;
        const uint4 *S = reinterpret_cast<const uint4 *>(a.src + ld.offset);
        uint4 *Dg = reinterpret_cast<uint4 *>(a.dst + ld.offset);
        for (int v = threadIdx.x; v < nload * Lv; v += THREADS) {
            const int i = v / Lv, j = v - i * Lv;
            int gy = w.r0 - halo + i;
            gy = gy < 0 ? gy + L : (gy >= L ? gy - L : gy);
            sm4[v] = __ldg(S + (size_t)gy * Lv + j);
        }
        if (threadIdx.x < kTabStride) stab[threadIdx.x] = a.tabs[w.lat * kTabStride + threadIdx.x];
        __syncthreads();
        PottsAcc acc = {0, 0ull, 0ull};
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            const int lo = w.whole ? 0 : (c == 0 ? 1 : 2);
            const int hi = w.whole ? w.nrows : (c == 0 ? w.nrows + 3 : w.nrows + 2);
            const int n_units = (hi - lo) * Lv;
            for (int v = threadIdx.x; v < n_units; v += THREADS) {
                const int i = lo + v / Lv, j = v % Lv;
                const int iu = (i == 0) ? nload - 1 : i - 1;
                const int id = (i == nload - 1) ? 0 : i + 1;
                int gy = w.r0 - halo + i;
                gy = gy < 0 ? gy + L : (gy >= L ? gy - L : gy);
                const uint4 Cc = sm4[i * Lv + j];
                const uint4 Uc = sm4[iu * Lv + j];
                const uint4 Dc = sm4[id * Lv + j];
                const uint32_t lw = sm32[(i * Lv + (j == 0 ? Lv - 1 : j - 1)) * 4 + 3];
                const uint32_t rw = sm32[(i * Lv + (j == Lv - 1 ? 0 : j + 1)) * 4];
                const bool count = (i >= halo) && (i < halo + w.nrows);
                const uint32_t gbase = (uint32_t)gy * (uint32_t)(L >> 2) + 4u * (uint32_t)j;
                sm4[i * Lv + j] =
                    potts_chunk(Cc, Uc, Dc, lw, rw, gbase, (c ^ gy) & 1, (uint32_t)w.lat, t,
                                (uint32_t)c, a.k0, a.k1, q, stab, count, acc, shist, small_q);
            }
            __syncthreads();
        }
        for (int v = threadIdx.x; v < w.nrows * Lv; v += THREADS) {
            const int i = v / Lv, j = v - i * Lv;
            Dg[(size_t)(w.r0 + i) * Lv + j] = sm4[(halo + i) * Lv + j];
        }
        flush_potts_acc<THREADS>(acc, (int)q, a.delta + (size_t)a.width * w.lat, red, shist, small_q);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) potts_plain_kernel(uint8_t *spins, int L, uint32_t lat,
                                                          uint32_t q, const TabEntry *tab,
                                                          uint32_t k0, uint32_t k1,
                                                          const DevState *state, int64_t *delta,
                                                          int c) {
    __shared__ TabEntry stab[kTabStride];
    __shared__ int red[9 * 8];
    __shared__ int shist[256];
    const bool small_q = q <= 8;
    for (int k = threadIdx.x; k < 256; k += 256) shist[k] = 0;
    if (threadIdx.x < kTabStride) stab[threadIdx.x] = tab[threadIdx.x];
    __syncthreads();
    const uint32_t t = state->t;
    const int Lv = L >> 4;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    PottsAcc acc = {0, 0ull, 0ull};
    if (v < L * Lv) {
        uint4 *S = reinterpret_cast<uint4 *>(spins);
        const uint32_t *S32 = reinterpret_cast<const uint32_t *>(spins);
        const int i = v / Lv, j = v - i * Lv;
        const int iu = i == 0 ? L - 1 : i - 1, id = i == L - 1 ? 0 : i + 1;
        const uint4 Cc = S[(size_t)i * Lv + j];
        const uint4 Uc = S[(size_t)iu * Lv + j];
        const uint4 Dc = S[(size_t)id * Lv + j];
        const uint32_t lw = S32[((size_t)i * Lv + (j == 0 ? Lv - 1 : j - 1)) * 4 + 3];
        const uint32_t rw = S32[((size_t)i * Lv + (j == Lv - 1 ? 0 : j + 1)) * 4];
        const uint32_t gbase = (uint32_t)i * (uint32_t)(L >> 2) + 4u * (uint32_t)j;
        S[(size_t)i * Lv + j] = potts_chunk(Cc, Uc, Dc, lw, rw, gbase, (c ^ i) & 1, lat, t,
                                            (uint32_t)c, k0, k1, q, stab, true, acc, shist, small_q);
    }
    __syncthreads();
    flush_potts_acc<256>(acc, (int)q, delta, red, shist, small_q);
}

// Any even L: one thread per site (two passes as for Ising).
__global__ void potts_generic_kernel(const uint8_t *src, uint8_t *dst, const int32_t *lat_ids,
                                     const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                     uint32_t k1, const DevState *state, int64_t *delta, int width,
                                     int c) {
    const int lat = lat_ids[blockIdx.y];
    const LatDev ld = lats[lat];
    const int L = ld.L;
    const uint32_t q = (uint32_t)ld.q;
    const uint8_t *S = (c == 0 ? src : dst) + ld.offset;
    uint8_t *D = dst + ld.offset;
    const uint32_t t = state->t;
    int64_t *dl = delta + (size_t)width * lat;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L, x = i - y * L;
        const uint32_t s = S[i];
        if (((x + y) & 1) != c) {
            if (c == 0) D[i] = (uint8_t)s;
            continue;
        }
        const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
        const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
        const uint32_t nb[4] = {S[yu * L + x], S[yd * L + x], S[y * L + xl], S[y * L + xr]};
        const uint32_t k = (uint32_t)i >> 1;
        const uint4 r = philox4x32_10(make_uint4(k >> 1, (uint32_t)lat, t, (uint32_t)c), k0, k1);
        const uint32_t u0 = (k & 1u) ? r.z : r.x;
        const uint32_t u1 = (k & 1u) ? r.w : r.y;
        uint32_t sp = s + 1u + __umulhi(u1, q - 1u);
        sp = sp >= q ? sp - q : sp;
        int n_old = 0, n_new = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            n_old += nb[m] == s;
            n_new += nb[m] == sp;
        }
        const TabEntry e = tabs[lat * kTabStride + n_old - n_new + 4];
        if (u0 <= e.thr && s < q) {
            D[i] = (uint8_t)sp;
            atomicAdd(reinterpret_cast<unsigned long long *>(dl), (unsigned long long)(long long)e.delta);
            atomicAdd(reinterpret_cast<unsigned long long *>(dl + 1 + s), (unsigned long long)(-1ll));
            atomicAdd(reinterpret_cast<unsigned long long *>(dl + 1 + sp), 1ull);
        } else if (c == 0) {
            D[i] = (uint8_t)s;
        }
    }
}
// (states >= q can only come from a caller-supplied lattice; they are left
// unchanged by the generic kernel and never index the statistics)

}  // namespace

cudaError_t launch_potts_fused(const PottsSweepArgs &a, int grid, int threads, size_t smem,
                               cudaStream_t s) {
    switch (threads) {
        case 128:
            potts_fused_kernel<128><<<grid, 128, smem, s>>>(a);
            break;
        case 256:
            potts_fused_kernel<256><<<grid, 256, smem, s>>>(a);
            break;
        case 512:
            potts_fused_kernel<512><<<grid, 512, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The dynamic shared-memory limit of a kernel is process-wide state: it is
// only ever raised (per device), so one caller can never lower it below what
// another caller's launches need.  48 KB needs no opt-in.
cudaError_t set_potts_fused_smem(size_t smem) {
    static size_t raised[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (smem <= 48 * 1024 || dev < 0 || dev >= 64 || smem <= raised[dev]) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    raised[dev] = smem;
    return cudaSuccess;
}

cudaError_t launch_potts_plain(uint8_t *spins, const LatDev *, int lat, int L, int q,
                               const TabEntry *tabs, uint32_t k0, uint32_t k1,
                               const DevState *state, int64_t *delta, int width, int colour,
                               cudaStream_t s) {
    const int units = L * (L >> 4);
    potts_plain_kernel<<<(units + 255) / 256, 256, 0, s>>>(
        spins, L, (uint32_t)lat, (uint32_t)q, tabs + lat * kTabStride, k0, k1, state,
        delta + (size_t)width * lat, colour);
    return cudaGetLastError();
}

cudaError_t launch_potts_generic(const uint8_t *src, uint8_t *dst, const int32_t *lat_ids, int n,
                                 int maxL, const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                 uint32_t k1, const DevState *state, int64_t *delta, int width,
                                 int colour, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (maxL * maxL + 255) / 256;
    dim3 grid(blocks < 64 ? blocks : 64, n);
    potts_generic_kernel<<<grid, 256, 0, s>>>(src, dst, lat_ids, lats, tabs, k0, k1, state, delta,
                                              width, colour);
    return cudaGetLastError();
}

}  // namespace spinmc
