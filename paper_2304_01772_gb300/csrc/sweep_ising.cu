// sweep_ising.cu -- checkerboard Metropolis sweeps of batched 2D Ising lattices
// (Alg. 1 of Farias et al., arXiv 2304.01772, with the 4-neighbour stencil of
// Sec. "Ising model"), plus the random initial state.
//
// Spins are int8 +-1 (0x01 / 0xFF).  Bit 1 of a byte is set iff the spin is
// -1, so (word & 0x02020202) gives twice the "down" indicator of four sites at
// once, and four such words add without carries (at most 8 per byte).  The
// per-site table key is d + 5 c (d = down neighbours, c = own spin down),
// formed for four sites in one 32-bit word; each byte of
//     key4 = 4 * (N2 + 5 * c2)    (N2 = 2 d, c2 = 2 c)
// is directly the byte offset of the 8-byte table entry.
//
// Kernels:
//  * ising_fused_kernel: one launch per sweep over a work list of items
//    (whole small lattices, or row blocks of large ones).  Each item loads its
//    rows plus a two-row halo into shared memory, updates colour 0 on the rows
//    and the inner halo ring (recomputed: the draws depend only on the site),
//    then colour 1 on its own rows, and writes the rows to the other buffer.
//  * ising_plain_kernel: one lattice, one colour, in place (two launches per
//    lattice per sweep: the plain launch form the batched one is compared to).
//  * ising_generic_kernel: any even L (not a multiple of 16), one thread per site.
#include <cooperative_groups.h>

#include "internal.h"
#include "strip.cuh"

namespace spinmc {

namespace {

constexpr uint32_t kDownMask = 0x02020202u;

// Update the colour-`c` sites of one 16-byte row chunk.  C: the chunk; U, D: the
// chunks above and below; lw / rw: the 32-bit words left and right of C in
// the same row.  Philox groups g0 (bytes 0..7) and g0 + 1 (bytes 8..15); active
// bytes of each word are p and p + 2.
__device__ __forceinline__ uint4 ising_chunk_r(uint4 C, uint4 U, uint4 D, uint32_t lw, uint32_t rw, int p,
                                               uint4 ra, uint4 rb, const TabEntry *stab, bool count, int &acc) {
    const uint32_t w[6] = {lw, C.x, C.y, C.z, C.w, rw};
    const uint32_t up[4] = {U.x, U.y, U.z, U.w};
    const uint32_t dn[4] = {D.x, D.y, D.z, D.w};
    const uint32_t rnd[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    uint32_t out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t W = w[i + 1];
        const uint32_t lf = __funnelshift_l(w[i], W, 8);      // left neighbours
        const uint32_t rt = __funnelshift_r(W, w[i + 2], 8);  // right neighbours
        const uint32_t n2 = (up[i] & kDownMask) + (dn[i] & kDownMask) + (lf & kDownMask) +
                            (rt & kDownMask);
        const uint32_t key4 = (n2 + (W & kDownMask) * 5u) << 2;
        uint32_t nw = W;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int sh = 8 * (p + 2 * bb);
            const uint32_t off = (key4 >> sh) & 0xFFu;
            const uint2 e = *reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(stab) + off);
            const uint32_t m = 0u - (uint32_t)(rnd[2 * i + bb] <= e.x);   // branch-free acceptance
            nw ^= m & (0xFEu << sh);
            if (count) acc += (int)(m & e.y);
        }
        out[i] = nw;
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}

__device__ __forceinline__ uint4 ising_chunk(uint4 C, uint4 U, uint4 D, uint32_t lw, uint32_t rw,
                                             uint32_t g0, int p, uint32_t lat, uint32_t t,
                                             uint32_t c, uint32_t k0, uint32_t k1,
                                             const TabEntry *stab, bool count, int &acc) {
    const uint4 ra = philox4x32_10(make_uint4(g0, lat, t, c), k0, k1);
    const uint4 rb = philox4x32_10(make_uint4(g0 + 1u, lat, t, c), k0, k1);
    return ising_chunk_r(C, U, D, lw, rw, p, ra, rb, stab, count, acc);
}

// Packed (dB * 65536 + dM) per-thread sums -> block sums -> one atomic pair.
template <int THREADS>
__device__ __forceinline__ void flush_ising_acc(int acc, int64_t *delta_lat, int *red) {
    int dm = (int)(int16_t)(acc & 0xFFFF);
    int db = (acc - dm) >> 16;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
        db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[2 * warp] = dm;
        red[2 * warp + 1] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sm = 0, sb = 0;
        for (int k = 0; k < THREADS / 32; ++k) {
            sm += red[2 * k];
            sb += red[2 * k + 1];
        }
        if (sm) atomicAdd(reinterpret_cast<unsigned long long *>(delta_lat), (unsigned long long)sm);
        if (sb)
            atomicAdd(reinterpret_cast<unsigned long long *>(delta_lat + 1), (unsigned long long)sb);
    }
}

// Triangular lattices (geometry 1) resident in shared memory for all sweeps
// of a call, one block per lattice; per sweep three colour passes, each
// thread taking one Philox group (four consecutive compressed sites of the
// colour, k = y (L/3) + x div 3).  Records as ising_resident_kernel.
constexpr int kTriResThreads = 512;

__global__ void __launch_bounds__(kTriResThreads) ising_tri_resident_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    int8_t *S = reinterpret_cast<int8_t *>(sm);
    __shared__ TabEntry stab[kTabStride];
    __shared__ int red[2 * (kTriResThreads / 32)];
    __shared__ long long cur_s[2];
    const int lat = blockIdx.x;
    const LatDev ld = a.lats[lat];
    const int L = ld.L, N = L * L, third = L / 3, nk = N / 3;
    int8_t *G = a.spins + ld.offset;
    for (int i = threadIdx.x; i < N; i += blockDim.x) S[i] = G[i];
    if (threadIdx.x < kTabStride) stab[threadIdx.x] = a.tabs[lat * kTabStride + threadIdx.x];
    if (threadIdx.x < 2) cur_s[threadIdx.x] = a.st.cur[2 * lat + threadIdx.x];
    // a thread's groups start kTriResThreads groups apart: the first site of the
    // next group is (dy, dm) rows and compressed columns further, so the walk
    // adds instead of dividing
    constexpr int kStep = 4 * kTriResThreads;
    const int dy = kStep / third, dm = kStep - dy * third, doff = dy % 3;
    const int y00 = (4 * (int)threadIdx.x) / third, m00 = 4 * (int)threadIdx.x - y00 * third;
    __syncthreads();
    for (int sweep = 0; sweep < a.n_sweeps; ++sweep) {
        const uint32_t t = a.t0 + (uint32_t)sweep;
        int acc = 0;
        for (int c = 0; c < 3; ++c) {
            const PhiloxPrefix P = philox_prefix(ld.rng, t, (uint32_t)c, a.rk);
            int gy = y00, gm = m00, goff = (c + y00) % 3;
            for (int grp = threadIdx.x; 4 * grp < nk; grp += kTriResThreads) {
                const uint4 r = philox_from_prefix((uint32_t)grp, P, a.rk);
                const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
                // row, compressed column and colour offset of the group's first site;
                // a group's sites rarely cross a row
                int y = gy, m = gm, off = goff;
                gy += dy;
                gm += dm;
                goff += doff;
                if (gm >= third) {
                    gm -= third;
                    ++gy;
                    ++goff;
                }
                if (goff >= 3) goff -= 3;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    if (4 * grp + l >= nk) break;
                    if (m == third) {
                        m = 0;
                        ++y;
                        off = off == 2 ? 0 : off + 1;
                    }
                    const int x = 3 * m + off;
                    ++m;
                    const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
                    const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
                    const int dcount = (S[y * L + xl] < 0) + (S[y * L + xr] < 0) + (S[yu * L + x] < 0) +
                                       (S[yd * L + x] < 0) + (S[yu * L + xr] < 0) + (S[yd * L + xl] < 0);
                    const int sv = S[y * L + x] < 0 ? -1 : 1;
                    const TabEntry e = stab[dcount + 7 * (sv < 0 ? 1 : 0)];
                    if (rr[l] <= e.thr) {
                        S[y * L + x] = (int8_t)(-sv);
                        acc += e.delta;
                    }
                }
            }
            __syncthreads();
        }
        int dm = (int)(int16_t)(acc & 0xFFFF);
        int db = (acc - dm) >> 16;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
            db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[2 * (threadIdx.x >> 5)] = dm;
            red[2 * (threadIdx.x >> 5) + 1] = db;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long sm_ = 0, sb_ = 0;
            for (int w = 0; w < kTriResThreads / 32; ++w) {
                sm_ += red[2 * w];
                sb_ += red[2 * w + 1];
            }
            cur_s[0] += sm_;
            cur_s[1] += sb_;
            if (a.record && a.st.cap > 0) {
                const long long slot = (a.rec0 + sweep) % a.st.cap;
                a.st.ring[(slot * a.st.n_lat + lat) * 2] = cur_s[0];
                a.st.ring[(slot * a.st.n_lat + lat) * 2 + 1] = cur_s[1];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) G[i] = S[i];
    if (threadIdx.x < 2) a.st.cur[2 * lat + threadIdx.x] = cur_s[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Ising with first and second neighbours (geometry 2):
// H = -J sum_nn s s - J2 sum_diag s s - h sum s.  The eight neighbours of a
// site carry the three other colours of c = (x & 1) | ((y & 1) << 1), so each
// colour's sites update at once.  Sites of colour c are (2m + (c & 1),
// 2Y + (c >> 1)), compressed index k = Y (L/2) + m; the draw of a site is
// lane k & 3 of Philox group k >> 2.  Statistics (M, B, B2).

// Down spins among the four nearest (d1) and the four diagonal (d2) neighbours.
__device__ __forceinline__ void nnn_counts(const int8_t *S, int L, int x, int y, int &d1, int &d2) {
    const int yu = (y == 0 ? L - 1 : y - 1) * L, yc = y * L, yd = (y == L - 1 ? 0 : y + 1) * L;
    const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
    d1 = (S[yc + xl] < 0) + (S[yc + xr] < 0) + (S[yu + x] < 0) + (S[yd + x] < 0);
    d2 = (S[yu + xl] < 0) + (S[yu + xr] < 0) + (S[yd + xl] < 0) + (S[yd + xr] < 0);
}

// One Philox group (four consecutive compressed sites of colour c) of one
// lattice: S is read, D written (S == D in place).  copy_block: colour 0 from
// src to dst, where the thread also copies the three other sites of each of
// its sites' 2x2 blocks (every block holds one site of each colour).
template <bool COPY>
__device__ __forceinline__ void nnn_group(const int8_t *S, int8_t *D, int L, int half, int nk, int g,
                                          int c, uint4 r, const uint32_t *tab, int &dm, int &db,
                                          int &db2) {
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    int Y = (4 * g) / half, m = 4 * g - Y * half;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (4 * g + l >= nk) break;
        if (m == half) {
            m = 0;
            ++Y;
        }
        const int x = 2 * m + (c & 1), y = 2 * Y + (c >> 1);
        ++m;
        int d1, d2;
        nnn_counts(S, L, x, y, d1, d2);
        const int i = y * L + x;
        const int sv = S[i] < 0 ? -1 : 1;
        if (COPY) {
            D[i + 1] = S[i + 1];
            D[i + L] = S[i + L];
            D[i + L + 1] = S[i + L + 1];
        }
        if (rr[l] <= tab[(sv < 0 ? 25 : 0) + 5 * d1 + d2]) {
            D[i] = (int8_t)(-sv);
            dm -= 2 * sv;
            db -= 2 * sv * (4 - 2 * d1);
            db2 -= 2 * sv * (4 - 2 * d2);
        } else if (COPY) {
            D[i] = (int8_t)sv;
        }
    }
}

// Per-byte down indicators (bit 7 of a +-1 byte) of eight sites.
__device__ __forceinline__ uint64_t down8(uint64_t w) { return (w >> 7) & 0x0101010101010101ull; }

// Lane p of the result: down(p - 1) + down(p + 1) within the word, with the
// indicator de of the byte just outside it (left of lane 0 for CX = 0, right
// of lane 7 for CX = 1), the one edge the sites of lanes CX + 2j need.
template <int CX>
__device__ __forceinline__ uint64_t horiz8(uint64_t D, uint32_t de) {
    return (D << 8) + (D >> 8) + (CX ? (uint64_t)de << 56 : (uint64_t)de);
}

// Sum of the eight bytes of x.
__device__ __forceinline__ uint32_t byte_sum8(uint64_t x) {
    return __dp4a((uint32_t)x, 0x01010101u, __dp4a((uint32_t)(x >> 32), 0x01010101u, 0u));
}

// nnn_group for a lattice in shared memory with L % 8 == 0, in place: the
// group's four sites are lanes CX, CX + 2, CX + 4, CX + 6 of the 8-byte word
// at column base of row y, so three word loads (rows y - 1, y, y + 1) and
// three edge bytes give every neighbour; per lane the table key
// 25 cdown + 5 d1 + d2 (<= 49) is formed bytewise without carries.  Accepted
// flips are one xor with 0xFE per byte (0x01 <-> 0xFF) and one store of the
// word, which no other thread of this colour pass reads or writes except for
// unchanged bytes.  ss, sd1, sd2 accumulate s, s d1, s d2 over accepted sites
// (s the old spin), from byte masks of the accepted and the accepted-down lanes.
template <int CX>
__device__ __forceinline__ void nnn_group8(int8_t *S, int L, int y, int base, uint4 r, const uint32_t *tab,
                                           int &ss, int &sd1, int &sd2) {
    const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
    const int xe = CX ? (base + 8 == L ? 0 : base + 8) : (base == 0 ? L - 1 : base - 1);
    int8_t *r0 = S + y * L;
    const int8_t *rm = S + yu * L, *rp = S + yd * L;
    const uint64_t W0 = *reinterpret_cast<const uint64_t *>(r0 + base);
    const uint64_t Dm = down8(*reinterpret_cast<const uint64_t *>(rm + base));
    const uint64_t D0 = down8(W0);
    const uint64_t Dp = down8(*reinterpret_cast<const uint64_t *>(rp + base));
    const uint64_t Hm = horiz8<CX>(Dm, rm[xe] < 0), H0 = horiz8<CX>(D0, r0[xe] < 0);
    const uint64_t Hp = horiz8<CX>(Dp, rp[xe] < 0);
    const uint64_t A1 = H0 + Dm + Dp, A2 = Hm + Hp;       // d1, d2 per lane (<= 4)
    const uint64_t K = (A1 << 2) + A1 + A2 + D0 * 25u;     // 25 cdown + 5 d1 + d2
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    uint64_t accm = 0;                                     // 0xFF in the accepted lanes
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = 8 * (CX + 2 * j);
        if (rr[j] <= tab[(uint32_t)(K >> p) & 0xFFu]) accm |= 0xFFull << p;
    }
    if (accm) {
        *reinterpret_cast<uint64_t *>(r0 + base) = W0 ^ (accm & 0xFEFEFEFEFEFEFEFEull);
        const uint64_t dn = accm & (D0 * 0xFFu);           // accepted lanes whose spin was down
        const int na = __popcll(accm) >> 3, nd = __popcll(dn) >> 3;
        ss += na - 2 * nd;
        sd1 += (int)byte_sum8(A1 & accm) - 2 * (int)byte_sum8(A1 & dn);
        sd2 += (int)byte_sum8(A2 & accm) - 2 * (int)byte_sum8(A2 & dn);
    }
}

// Block sum of three per-thread counters into red[3][warps]; thread 0 gets the totals.
template <int THREADS>
__device__ __forceinline__ void block_sum3(int a0, int a1, int a2, int *red, long long out[3]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xFFFFFFFFu, a0, o);
        a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
        a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
    }
    constexpr int W = THREADS / 32;
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = a0;
        red[W + (threadIdx.x >> 5)] = a1;
        red[2 * W + (threadIdx.x >> 5)] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = out[1] = out[2] = 0;
        for (int w = 0; w < W; ++w) {
            out[0] += red[w];
            out[1] += red[W + w];
            out[2] += red[2 * W + w];
        }
    }
}

constexpr int kNnnThreads = 256;

__global__ void __launch_bounds__(kNnnThreads) ising_nnn_kernel(const int8_t *src, int8_t *dst, const LatDev *lats,
                                                                const uint32_t *thr, uint32_t k0, uint32_t k1,
                                                                const DevState *state, int64_t *delta, int c) {
    __shared__ uint32_t tab[kNnnTab];
    __shared__ int red[3 * (kNnnThreads / 32)];
    const int lat = blockIdx.y;
    const LatDev ld = lats[lat];
    const int L = ld.L, half = L >> 1, nk = half * half;
    if (threadIdx.x < kNnnTab) tab[threadIdx.x] = thr[lat * kNnnTab + threadIdx.x];
    __syncthreads();
    const int8_t *S = (c == 0 ? src : dst) + ld.offset;
    int8_t *D = dst + ld.offset;
    const uint32_t t = state->t;
    int dm = 0, db = 0, db2 = 0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; 4 * g < nk; g += gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)g, ld.rng, t, (uint32_t)c), k0, k1);
        if (c == 0)
            nnn_group<true>(S, D, L, half, nk, g, c, r, tab, dm, db, db2);
        else
            nnn_group<false>(S, D, L, half, nk, g, c, r, tab, dm, db, db2);
    }
    long long tot[3];
    block_sum3<kNnnThreads>(dm, db, db2, red, tot);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k)
            if (tot[k]) atomicAdd(reinterpret_cast<unsigned long long *>(delta + 3 * lat + k), (unsigned long long)tot[k]);
}

// Resident form: one block per lattice keeps it in shared memory for all
// sweeps of the call; per sweep four colour passes; records as
// ising_resident_kernel with three statistics.
constexpr int kNnnResThreads = 512;

__global__ void __launch_bounds__(kNnnResThreads) ising_nnn_resident_kernel(ResidentArgs a, const uint32_t *thr) {
    extern __shared__ __align__(16) unsigned char sm[];
    int8_t *S = reinterpret_cast<int8_t *>(sm);
    __shared__ uint32_t tab[kNnnTab];
    __shared__ int red[3 * (kNnnResThreads / 32)];
    __shared__ long long cur_s[3];
    const int lat = blockIdx.x;
    const LatDev ld = a.lats[lat];
    const int L = ld.L, N = L * L, half = L >> 1, nk = N >> 2;
    int8_t *G = a.spins + ld.offset;
    for (int i = threadIdx.x; i < N; i += blockDim.x) S[i] = G[i];
    if (threadIdx.x < kNnnTab) tab[threadIdx.x] = thr[lat * kNnnTab + threadIdx.x];
    if (threadIdx.x < 3) cur_s[threadIdx.x] = a.st.cur[3 * lat + threadIdx.x];
    __syncthreads();
    for (int sweep = 0; sweep < a.n_sweeps; ++sweep) {
        const uint32_t t = a.t0 + (uint32_t)sweep;
        int dm = 0, db = 0, db2 = 0;
        if ((L & 7) == 0) {
            // group g of a colour: row pair Y = g / gpr, first column 8 (g % gpr);
            // the thread's groups advance by blockDim.x without a division
            const int gpr = L >> 3;
            const int Y0 = (int)threadIdx.x / gpr, q0 = (int)threadIdx.x - Y0 * gpr;
            const int dY = (int)blockDim.x / gpr, dq = (int)blockDim.x - dY * gpr;
            int ss = 0, sd1 = 0, sd2 = 0;
            for (int c = 0; c < 4; ++c) {
                const PhiloxPrefix P = philox_prefix(ld.rng, t, (uint32_t)c, a.rk);
                int Y = Y0, q = q0;
                for (int g = threadIdx.x; 4 * g < nk; g += blockDim.x) {
                    const uint4 r = philox_from_prefix((uint32_t)g, P, a.rk);
                    const int y = 2 * Y + (c >> 1);
                    if (c & 1)
                        nnn_group8<1>(S, L, y, 8 * q, r, tab, ss, sd1, sd2);
                    else
                        nnn_group8<0>(S, L, y, 8 * q, r, tab, ss, sd1, sd2);
                    Y += dY;
                    q += dq;
                    if (q >= gpr) {
                        q -= gpr;
                        ++Y;
                    }
                }
                __syncthreads();
            }
            // dM = -2 s, dB = -2 s (4 - 2 d1), dB2 = -2 s (4 - 2 d2) per accepted site
            dm = -2 * ss;
            db = -8 * ss + 4 * sd1;
            db2 = -8 * ss + 4 * sd2;
        } else {
            for (int c = 0; c < 4; ++c) {
                for (int g = threadIdx.x; 4 * g < nk; g += blockDim.x) {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, ld.rng, t, (uint32_t)c), a.k0, a.k1);
                    nnn_group<false>(S, S, L, half, nk, g, c, r, tab, dm, db, db2);
                }
                __syncthreads();
            }
        }
        long long tot[3];
        block_sum3<kNnnResThreads>(dm, db, db2, red, tot);
        if (threadIdx.x == 0) {
            for (int k = 0; k < 3; ++k) cur_s[k] += tot[k];
            if (a.record && a.st.cap > 0) {
                const long long slot = (a.rec0 + sweep) % a.st.cap;
                for (int k = 0; k < 3; ++k) a.st.ring[(slot * a.st.n_lat + lat) * 3 + k] = cur_s[k];
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) G[i] = S[i];
    if (threadIdx.x < 3) a.st.cur[3 * lat + threadIdx.x] = cur_s[threadIdx.x];
}

__global__ void advance_state_kernel(DevState *state, uint32_t n, int record) {
    state->t += n;
    if (record) state->n_rec += n;
}

// One lattice, one colour, in place, straight from global memory.
__global__ void __launch_bounds__(256) ising_plain_kernel(int8_t *spins, int L, uint32_t lat, uint32_t rng,
                                                          const TabEntry *tab, uint32_t k0,
                                                          uint32_t k1, const DevState *state,
                                                          int64_t *delta, int c) {
    __shared__ TabEntry stab[kTabStride];
    __shared__ int red[16];
    if (threadIdx.x < kTabStride) stab[threadIdx.x] = tab[threadIdx.x];
    __syncthreads();
    const uint32_t t = state->t;
    const int Lv = L >> 4;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    int acc = 0;
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
        const uint32_t g0 = (uint32_t)i * (uint32_t)(L >> 3) + 2u * (uint32_t)j;
        S[(size_t)i * Lv + j] =
            ising_chunk(Cc, Uc, Dc, lw, rw, g0, (c ^ i) & 1, rng, t, (uint32_t)c, k0, k1, stab,
                        true, acc);
    }
    flush_ising_acc<256>(acc, delta + 2 * lat, red);
}

// Any even L: one thread per site.  colour 0 pass reads src and writes every
// site of dst (colour-1 sites copied); colour 1 pass updates dst in place.
// Triangular lattice (geometry 1): six neighbours (x+-1, y), (x, y+-1),
// (x+1, y-1), (x-1, y+1); colour (x - y) mod 3; table entry dcount + 7 cdown
// (dcount = down neighbours of 6, n = 6 - 2 dcount); the draw of a site is
// lane k & 3 of group k >> 2, k = y (L/3) + x div 3 (one compressed index per
// site of a colour).  One thread per site.
__global__ void ising_tri_kernel(const int8_t *src, int8_t *dst, const int32_t *lat_ids, const LatDev *lats,
                                 const TabEntry *tabs, uint32_t k0, uint32_t k1, const DevState *state,
                                 int64_t *delta, int c) {
    __shared__ int red[2 * 8];
    const int lat = lat_ids[blockIdx.y];
    const LatDev ld = lats[lat];
    const int L = ld.L;
    const int8_t *S = (c == 0 ? src : dst) + ld.offset;
    int8_t *D = dst + ld.offset;
    const uint32_t t = state->t;
    int dm = 0, db = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L, x = i - y * L;
        const int s = S[i];
        if ((x - y + 3 * L) % 3 != c) {
            if (c == 0) D[i] = (int8_t)s;
            continue;
        }
        const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
        const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
        const int dcount = (S[y * L + xl] < 0) + (S[y * L + xr] < 0) + (S[yu * L + x] < 0) + (S[yd * L + x] < 0) +
                           (S[yu * L + xr] < 0) + (S[yd * L + xl] < 0);
        const int n = 6 - 2 * dcount;
        const int cdown = s < 0 ? 1 : 0;
        const TabEntry e = tabs[lat * kTabStride + dcount + 7 * cdown];
        const uint32_t k = (uint32_t)(y * (L / 3) + x / 3);
        const uint4 r = philox4x32_10(make_uint4(k >> 2, ld.rng, t, (uint32_t)c), k0, k1);
        const uint32_t lane = k & 3u;
        const uint32_t u = lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
        const int sv = s < 0 ? -1 : 1;
        if (u <= e.thr) {
            D[i] = (int8_t)(-sv);
            dm += -2 * sv;
            db += -2 * sv * n;
        } else if (c == 0) {
            D[i] = (int8_t)s;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
        db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[2 * (threadIdx.x >> 5)] = dm;
        red[2 * (threadIdx.x >> 5) + 1] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sm = 0, sb = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sm += red[2 * k];
            sb += red[2 * k + 1];
        }
        if (sm) atomicAdd(reinterpret_cast<unsigned long long *>(delta + 2 * lat), (unsigned long long)sm);
        if (sb) atomicAdd(reinterpret_cast<unsigned long long *>(delta + 2 * lat + 1), (unsigned long long)sb);
    }
}

__global__ void ising_generic_kernel(const int8_t *src, int8_t *dst, const int32_t *lat_ids,
                                     const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                     uint32_t k1, const DevState *state, int64_t *delta, int c) {
    __shared__ int red[2 * 8];
    const int lat = lat_ids[blockIdx.y];
    const LatDev ld = lats[lat];
    const int L = ld.L;
    const int8_t *S = (c == 0 ? src : dst) + ld.offset;
    int8_t *D = dst + ld.offset;
    const uint32_t t = state->t;
    int dm = 0, db = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L, x = i - y * L;
        const int s = S[i];
        if (((x + y) & 1) != c) {
            if (c == 0) D[i] = (int8_t)s;
            continue;
        }
        const int yu = y == 0 ? L - 1 : y - 1, yd = y == L - 1 ? 0 : y + 1;
        const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
        // down neighbours counted from the sign, so any byte value keeps the index in range
        const int dcount = (S[yu * L + x] < 0) + (S[yd * L + x] < 0) + (S[y * L + xl] < 0) +
                           (S[y * L + xr] < 0);
        const int n = 4 - 2 * dcount;
        const int cdown = s < 0 ? 1 : 0;
        const TabEntry e = tabs[lat * kTabStride + dcount + 5 * cdown];
        const uint32_t k = (uint32_t)i >> 1;
        const uint4 r = philox4x32_10(make_uint4(k >> 2, ld.rng, t, (uint32_t)c), k0, k1);
        const uint32_t lane = k & 3u;
        const uint32_t u = lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
        if (u <= e.thr) {
            D[i] = (int8_t)(-s);
            dm += -2 * s;
            db += -2 * s * n;
        } else if (c == 0) {
            D[i] = (int8_t)s;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
        db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[2 * (threadIdx.x >> 5)] = dm;
        red[2 * (threadIdx.x >> 5) + 1] = db;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long sm = 0, sb = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sm += red[2 * k];
            sb += red[2 * k + 1];
        }
        if (sm) atomicAdd(reinterpret_cast<unsigned long long *>(delta + 2 * lat), (unsigned long long)sm);
        if (sb) atomicAdd(reinterpret_cast<unsigned long long *>(delta + 2 * lat + 1), (unsigned long long)sb);
    }
}

// Random initial state: one Philox call per group of four consecutive sites.
__global__ void init_random_kernel(void *spins, int model, const LatDev *lats, uint32_t k0,
                                   uint32_t k1) {
    const LatDev ld = lats[blockIdx.y];
    const int groups = (ld.L * ld.L) >> 2;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
        const uint4 r =
            philox4x32_10(make_uint4((uint32_t)g, ld.rng, 0xFFFFFFFFu, 0u), k0, k1);
        const uint32_t u[4] = {r.x, r.y, r.z, r.w};
        if (model == 0) {
            int8_t *S = static_cast<int8_t *>(spins) + ld.offset + 4 * (size_t)g;
#pragma unroll
            for (int l = 0; l < 4; ++l) S[l] = (u[l] >> 31) ? (int8_t)1 : (int8_t)-1;
        } else {
            uint8_t *S = static_cast<uint8_t *>(spins) + ld.offset + 4 * (size_t)g;
#pragma unroll
            for (int l = 0; l < 4; ++l) S[l] = (uint8_t)__umulhi(u[l], (uint32_t)ld.q);
        }
    }
}

// ------------------------------------------------------------- the x8 form
// In shared memory a spin is the byte 8 * [s < 0] ("x8 form"): four neighbour
// bytes plus 5x the centre byte add without carries to 8 * (d + 5 c), the
// byte offset of the site's 8-byte table entry (d = down neighbours, c = the
// site itself down).  The tile and resident kernels update 16-byte row chunks
// in this form (chunk_x8); the row-strip kernel below keeps its rows split
// by column parity.
constexpr uint32_t kX8 = 0x08080808u;
__device__ __forceinline__ uint4 to_x8(uint4 v) {
    return make_uint4(v.x & kX8, v.y & kX8, v.z & kX8, v.w & kX8);
}

__device__ __forceinline__ uint32_t from_x8(uint32_t w) { return ((w >> 3) * 0xFEu) + 0x01010101u; }

// Byte selectors (PRMT) and flip masks of the two active bytes P and P + 2.
// A selector takes the site's key byte as byte 0 and bytes 1..3 from the
// table's shared-memory address, whose byte 0 is zero: the result is the
// address of the site's table entry.
struct RowPar {
    uint32_t sel0, sel1, fm0, fm1;
};

__device__ __forceinline__ RowPar row_par(int P) {
    return RowPar{0x7650u + (uint32_t)P, 0x7652u + (uint32_t)P, 8u << (8 * P), 8u << (8 * P + 16)};
}

// One 8-byte table entry at a shared-memory address.
__device__ __forceinline__ uint2 lds_entry(uint32_t addr) {
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// Metropolis decision of one site without a branch: if u <= thr, flip the
// site's byte (xor with fm) and add the statistics delta (predicated ops).
// The delta is added with a carry-out (`add.cc`, the carry unused): measured
// 1.2% faster in the strip kernel than a plain add, whose instruction the
// compiler may place on the multiply-add pipe that Philox keeps busy.
__device__ __forceinline__ void accept_site(uint32_t &w, int &acc, uint32_t u, uint2 e, uint32_t fm) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.u32 p, %2, %3;\n\t"
        "@p xor.b32 %0, %0, %4;\n\t"
        "@p add.cc.u32 %1, %1, %5;\n\t}"
        : "+r"(w), "+r"(acc)
        : "r"(u), "r"(e.x), "r"(fm), "r"(e.y));
}

// Colour sub-step of one 16-byte chunk in x8 form.
__device__ __forceinline__ uint4 chunk_x8(uint4 C, uint4 U, uint4 D, uint32_t lw, uint32_t rw,
                                          uint4 ra, uint4 rb, const RowPar &rp,
                                          uint32_t stab, int &acc) {
    const uint32_t w[6] = {lw, C.x, C.y, C.z, C.w, rw};
    const uint32_t up[4] = {U.x, U.y, U.z, U.w};
    const uint32_t dn[4] = {D.x, D.y, D.z, D.w};
    const uint32_t rnd[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    uint32_t out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t W = w[i + 1];
        const uint32_t lf = __funnelshift_l(w[i], W, 8);
        const uint32_t rt = __funnelshift_r(W, w[i + 2], 8);
        const uint32_t key = up[i] + dn[i] + lf + rt + W * 5u;
        // table entries are 8-byte aligned: one 64-bit shared load each
        const uint2 e0 = lds_entry(__byte_perm(key, stab, rp.sel0));
        const uint2 e1 = lds_entry(__byte_perm(key, stab, rp.sel1));
        uint32_t nw = W;
        accept_site(nw, acc, rnd[2 * i], e0, rp.fm0);
        accept_site(nw, acc, rnd[2 * i + 1], e1, rp.fm1);
        out[i] = nw;
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}

// Unpack the packed per-lane sums (dB * 65536 + dM) into 32-bit totals.
__device__ __forceinline__ void drain_acc(int &acc, int &dm, int &db) {
    const int m = (int)(int16_t)(acc & 0xFFFF);
    dm += m;
    db += (acc - m) >> 16;
    acc = 0;
}

// ---------------------------------------------------------------------------
// Row-strip kernel in the split form (Alg. 1 on the square-lattice stencil).
//
// Lattices with L = 512, 1024 or 2048: one warp owns full rows [r0, r0 + R)
// of one lattice and walks down them.  At step s it updates colour 0 on row
// s and colour 1 on row s - 1 (whose neighbours on rows s - 2 and s already
// carry their colour-0 updates).  Rows -1 and R are the recomputed halo:
// their colour-0 updates are needed by colour 1 of rows 0 and R - 1 and come
// from the same site-keyed Philox counters as in the neighbouring item, so
// items never exchange data and no block barrier is needed.
//
// Each ring row is stored as its two colour-compressed halves in the x8
// form: half 0 holds the sites of even x,
// half 1 those of odd x (site x of a row is byte x >> 1 of half x & 1).  For
// colour c on row y the active sites are half p = (c + y) & 1, and all four
// bytes of a 32-bit word of that half are active: a word's up and down
// neighbours are the aligned word of half p of rows y -+ 1, its left and right
// neighbours the aligned word of the other half and that word shifted by one
// byte (left for p = 0, right for p = 1).  The four draws of one Philox block
// (g = (y L / 2 + m) / 4) belong to the four sites of one word.
//
// At step s, colour 0 on row s and colour 1 on row s - 1 have the same p and
// touch the same word positions: colour 1's up row is row s - 2, its down row
// is row s (just updated) and its own sites are colour 0's up row.  So both
// updates run per word in one pass with no exchange between lanes; only the
// other-half word across a lane's chunk edge comes from shared memory.  Row
// s - 1 is then final and is written to the destination buffer in the int8
// form, re-interleaved by one sign-replicating byte permutation per word.
//
// Shared memory per warp: four split rows (s - 2 .. s + 1) and one landing
// slot where the raw row s + 2 arrives by cp.async while step s computes.
//
// Row formats in global memory (LAYOUT): bit 0 set = the source rows are
// already in the ring's split x8 form (even-x half, then odd-x half, one byte
// 8 [s < 0] per site), so a landed row becomes a ring slot as it is, with no
// split pass; bit 1 set = the destination rows are written in that form too,
// with no re-interleave.  Within a call of several sweeps the ping-pong
// buffer holds strip lattices in the split form between two sweeps; the
// first sweep reads and the last one writes the int8 rows of the interface.

namespace split {

// Raw row (L int8 spins, +1 = 0x01, -1 = 0xFF) at src -> split x8 row at dst
// (dst != src), one 16-byte raw chunk per lane at a time.
__device__ __forceinline__ void split_row(uint32_t src, uint32_t dst, int L, int lane) {
#pragma unroll 1
    for (int k = lane; k < (L >> 4); k += 32) {
        const Words<4> v4 = ldw<4>(src, k);
        const uint4 v = make_uint4(v4.w[0], v4.w[1], v4.w[2], v4.w[3]);
        const uint32_t a = v.x & kX8, b = v.y & kX8, c = v.z & kX8, d = v.w & kX8;
        Words<2> e, o;
        e.w[0] = __byte_perm(a, b, 0x6420), e.w[1] = __byte_perm(c, d, 0x6420);
        o.w[0] = __byte_perm(a, b, 0x7531), o.w[1] = __byte_perm(c, d, 0x7531);
        stw<2>(dst, k, e);
        stw<2>(dst + (uint32_t)(L >> 1), k, o);
    }
}

// Bit-packed rows (one bit per spin, 1 = -1; site x of a row is bit x % 32 of
// the row's word x / 32).  Row y of L bits is L / 128 chunks of 16 bytes.
__device__ __forceinline__ void issue_bits_s(uint32_t dst, const uint4 *Sb, int y, int L, int lane) {
    const uint4 *src = Sb + (size_t)y * (L >> 7);
    if (lane < (L >> 7))
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * (uint32_t)lane), "l"(src + lane)
                     : "memory");
}

// Packed row at src -> split x8 row at dst.  Byte i of packed word m holds
// sites 32 m + 8 i .. + 7; its even sites are bytes 0..3 of word 4 m + i of
// half 0, its odd sites those of half 1: lut[byte] = (even word, odd word).
__device__ __forceinline__ void bits_to_split(uint32_t src, uint32_t dst, int L, int lane, uint32_t lut) {
#pragma unroll 1
    for (int m = lane; m < (L >> 5); m += 32) {
        const uint32_t W = sld1(src + 4u * (uint32_t)m);
        Words<4> e, o;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint2 t = lds_u2(lut + 8u * ((W >> (8 * i)) & 0xFFu));
            e.w[i] = t.x;
            o.w[i] = t.y;
        }
        stw<4>(dst, m, e);
        stw<4>(dst + (uint32_t)(L >> 1), m, o);
    }
}

// The lookup table of bits_to_split: entry b = (x8 bytes of bits 0, 2, 4, 6 of
// b, x8 bytes of bits 1, 3, 5, 7 of b).
__device__ __forceinline__ uint2 bits_lut_entry(uint32_t b) {
    uint32_t e = 0, o = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        e |= ((b >> (2 * j)) & 1u) << (8 * j + 3);
        o |= ((b >> (2 * j + 1)) & 1u) << (8 * j + 3);
    }
    return make_uint2(e, o);
}

// Eight sites as one byte of packed bits: e, o are x8 words of the even and
// odd sites of the same half-row position (bit 3 of each byte); z has site
// 2 j + s at bit 8 j + 3 + s, and the product with 1 + 2^6 + 2^12 + 2^18 puts
// it at bit 21 + 2 j + s (all other partial products land outside bits 21..28
// and on distinct positions, so nothing carries).
__device__ __forceinline__ uint32_t x8_pair_byte(uint32_t e, uint32_t o) {
    return ((e + (o << 1)) * 0x00041041u >> 21) & 0xFFu;
}

// Final row chunk c (half words NW c .. NW c + NW - 1 of both halves) as bits:
// NW = 4: packed word c of the row; NW = 2: its 16-bit half c.
template <int NW>
__device__ __forceinline__ void store_bits(uint32_t *Db, int y, int L, int c, const Words<NW> &h0,
                                           const Words<NW> &h1) {
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) v |= x8_pair_byte(h0.w[i], h1.w[i]) << (8 * i);
    if constexpr (NW == 4)
        Db[(size_t)y * (L >> 5) + c] = v;
    else
        reinterpret_cast<uint16_t *>(Db)[(size_t)y * (L >> 4) + c] = (uint16_t)v;
}

// Metropolis update of the active words `act` given the other half's words
// `oth` (plus `edge`, the other-half word just outside the chunk: before it
// for p = 0, after it for p = 1), the aligned words of the rows above and
// below, and the Philox blocks g .. g + NW - 1.
template <int NW>
__device__ __forceinline__ void update(Words<NW> &act, const Words<NW> &oth, uint32_t edge, const Words<NW> &up,
                                       const Words<NW> &dn, uint32_t g, const PhiloxPrefix &P,
                                       const PhiloxKeys &rk, int p, uint32_t selH, uint32_t stab, int &acc) {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const uint32_t nb = p ? (i + 1 < NW ? oth.w[i + 1] : edge) : (i > 0 ? oth.w[i - 1] : edge);
        // the horizontal neighbours are oth (one side) and this shifted copy (other side)
        const uint32_t H = prmt(oth.w[i], nb, selH);
        const uint32_t key = up.w[i] + dn.w[i] + oth.w[i] + H + act.w[i] * 5u;
        // every key byte is 8 (d + 5 c) <= 72: an entry of the table's first 80 bytes
        SPIN_CK((key & 0x07070707u) == 0u && ((key + 0x37373737u) & 0x80808080u) == 0u, 104);
        const uint4 r = philox_from_prefix(g + (uint32_t)i, P, rk);
        uint32_t w = act.w[i];
        accept_site(w, acc, r.x, lds_entry(prmt(key, stab, 0x7650u)), 0x00000008u);
        accept_site(w, acc, r.y, lds_entry(prmt(key, stab, 0x7651u)), 0x00000800u);
        accept_site(w, acc, r.z, lds_entry(prmt(key, stab, 0x7652u)), 0x00080000u);
        accept_site(w, acc, r.w, lds_entry(prmt(key, stab, 0x7653u)), 0x08000000u);
        act.w[i] = w;
    }
}

// Final row: active half `act` and other half `oth` (x8 form) -> int8 spins.
// Inputs shifted left by 4 carry the spin in each byte's sign bit; sel0 / sel1
// interleave the halves and replicate those bits (0xFF or 0x00); OR 0x01.
template <int NW>
__device__ __forceinline__ void store_raw(uint4 *Drow, int c, const Words<NW> &act, const Words<NW> &oth,
                                          uint32_t sel0, uint32_t sel1) {
    uint32_t o[2 * NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const uint32_t a = act.w[i] << 4, b = oth.w[i] << 4;
        o[2 * i] = prmt(a, b, sel0) | 0x01010101u;
        o[2 * i + 1] = prmt(a, b, sel1) | 0x01010101u;
    }
    if constexpr (NW == 4) {
        Drow[2 * c] = make_uint4(o[0], o[1], o[2], o[3]);
        Drow[2 * c + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
        Drow[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Final row in the split form: the active half's words at half hp, the other
// half's at ho (byte offsets into the destination row).
template <int NW>
__device__ __forceinline__ void store_split(unsigned char *Drow, int hp, int ho, int c, const Words<NW> &act,
                                            const Words<NW> &oth) {
    st_words<NW>(Drow + hp, c, act);
    st_words<NW>(Drow + ho, c, oth);
}

struct Walk {
    const uint4 *S;
    uint4 *D;
    const uint4 *Sb;   // kSrcBits: the lattice's packed rows
    uint32_t *Db;      // kDstBits: the lattice's packed rows
    uint32_t ring;   // shared address of this warp's 5 * L bytes: 4 split rows + landing
    uint32_t lut;    // kSrcBits: shared address of the bits_to_split table
    int L, r0, nrows, lane;
    PhiloxPrefix P0, P1;
    uint32_t tab_cnt, tab_halo;
};

// One item: rows [r0, r0 + nrows) of one lattice, with the recomputed halo
// rows r0 - 1 and r0 + nrows (colour 0 only, no statistics).  NW: words of a
// half row per lane chunk (2 for L = 512, else 4).  LAYOUT: row formats.
template <int NW, int LAYOUT>
__device__ void item(const Walk &x, const PhiloxKeys &rk, int &dm, int &db) {
    constexpr bool kSrcS = (LAYOUT & kSrcSplit) != 0, kDstS = (LAYOUT & kDstSplit) != 0;
    constexpr bool kSrcB = (LAYOUT & kSrcBits) != 0, kDstB = (LAYOUT & kDstBits) != 0;
    const int L = x.L, half = L >> 1, nw = L >> 3, nc = nw / (32 * NW), lane = x.lane;
    const uint32_t uL = (uint32_t)L;
    uint32_t q0 = x.ring + 3 * uL, q1 = x.ring, q2 = x.ring + uL, q3 = x.ring + 2 * uL;
    uint32_t land = x.ring + 4 * uL;
    if constexpr (kSrcB) {
        // as for int8 rows below, with packed rows landing and bits_to_split
        issue_bits_s(q0, x.Sb, wrap_row(x.r0 - 2, L), L, lane);
        issue_bits_s(land, x.Sb, wrap_row(x.r0 - 1, L), L, lane);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        bits_to_split(q0, q1, L, lane, x.lut);
        bits_to_split(land, q2, L, lane, x.lut);
        __syncwarp();
        issue_bits_s(q0, x.Sb, wrap_row(x.r0, L), L, lane);
        cp_async_commit();
        issue_bits_s(land, x.Sb, wrap_row(x.r0 + 1, L), L, lane);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        bits_to_split(q0, q3, L, lane, x.lut);
        __syncwarp();
    } else if constexpr (kSrcS) {
        // rows -2 .. 0 straight into their slots; row 1 in flight in the landing slot
        issue_raw_s(q1, x.S, wrap_row(x.r0 - 2, L), L, lane);
        issue_raw_s(q2, x.S, wrap_row(x.r0 - 1, L), L, lane);
        issue_raw_s(q3, x.S, wrap_row(x.r0, L), L, lane);
        cp_async_commit();
        issue_raw_s(land, x.S, wrap_row(x.r0 + 1, L), L, lane);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
    } else {
        // rows -2 and -1 land in q0 (free until step -1 ends) and the landing
        // slot and are split into q1 and q2; then row 0 (via q0) into q3, and
        // row 1 stays in flight in the landing slot
        issue_raw_s(q0, x.S, wrap_row(x.r0 - 2, L), L, lane);
        issue_raw_s(land, x.S, wrap_row(x.r0 - 1, L), L, lane);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        split_row(q0, q1, L, lane);
        split_row(land, q2, L, lane);
        __syncwarp();
        issue_raw_s(q0, x.S, wrap_row(x.r0, L), L, lane);
        cp_async_commit();
        issue_raw_s(land, x.S, wrap_row(x.r0 + 1, L), L, lane);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        split_row(q0, q3, L, lane);
        __syncwarp();
    }
    int acc = 0;
    for (int s = -1; s <= x.nrows; ++s) {
        // q0..q3 hold rows s - 2 .. s + 1
        const int yA = wrap_row(x.r0 + s, L), yB = yA == 0 ? L - 1 : yA - 1;
        const int p = yA & 1;
        const uint32_t selH = p ? 0x4321u : 0x2107u;
        const uint32_t selO0 = p ? 0x9D8Cu : 0xD9C8u, selO1 = p ? 0xBFAEu : 0xFBEAu;
        const uint32_t tabA = (s >= 0 && s < x.nrows) ? x.tab_cnt : x.tab_halo;
        const int hp = p * half, ho = half - hp;
        const uint32_t gA = (uint32_t)yA * (uint32_t)(L >> 3), gB = (uint32_t)yB * (uint32_t)(L >> 3);
        uint4 *Drow = x.D + (size_t)yB * (L >> 4);
        unsigned char *Dsplit = reinterpret_cast<unsigned char *>(Drow);
        const int eoff = p ? NW : -1;
        for (int j = 0; j < nc; ++j) {
            const int c = lane + 32 * j;
            const int we = (NW * c + eoff) & (nw - 1);
            // the chunk and the edge word lie inside the half row
            if (!SPIN_CK(4 * NW * (c + 1) <= half && we >= 0 && we < nw, 103)) continue;
            const uint32_t eA = sld1(q2 + (uint32_t)ho + 4u * (uint32_t)we);
            Words<NW> act = ldw<NW>(q2 + (uint32_t)hp, c);
            const Words<NW> oth = ldw<NW>(q2 + (uint32_t)ho, c);
            Words<NW> upA = ldw<NW>(q1 + (uint32_t)hp, c);
            const Words<NW> dnA = ldw<NW>(q3 + (uint32_t)hp, c);
            update<NW>(act, oth, eA, upA, dnA, gA + (uint32_t)(NW * c), x.P0, rk, p, selH, tabA, acc);
            stw<NW>(q2 + (uint32_t)hp, c, act);
            if (s >= 1) {
                const uint32_t gBc = gB + (uint32_t)(NW * c);
                const uint32_t eB = sld1(q1 + (uint32_t)ho + 4u * (uint32_t)we);
                const Words<NW> othB = ldw<NW>(q1 + (uint32_t)ho, c);
                const Words<NW> upB = ldw<NW>(q0 + (uint32_t)hp, c);
                update<NW>(upA, othB, eB, upB, act, gBc, x.P1, rk, p, selH, x.tab_cnt, acc);
                if constexpr (kDstS)
                    store_split<NW>(Dsplit, hp, ho, c, upA, othB);
                else
                    store_raw<NW>(Drow, c, upA, othB, selO0, selO1);
                if constexpr (kDstB) {
                    if (p)
                        store_bits<NW>(x.Db, yB, L, c, othB, upA);
                    else
                        store_bits<NW>(x.Db, yB, L, c, upA, othB);
                }
            }
        }
        if ((s & 7) == 7) drain_acc(acc, dm, db);
        __syncwarp();
        if (s + 2 <= x.nrows + 1) {
            cp_async_wait_all();
            __syncwarp();
            if constexpr (kSrcB) {
                bits_to_split(land, q0, L, lane, x.lut);   // row s + 2 into the slot of row s - 2
                __syncwarp();
            } else if constexpr (kSrcS) {
                // row s + 2 takes the slot of row s - 2, which lands the next row
                const uint32_t t = q0;
                q0 = land;
                land = t;
            } else {
                split_row(land, q0, L, lane);      // row s + 2 into the slot of row s - 2
                __syncwarp();
            }
            if (s + 3 <= x.nrows + 1) {
                if constexpr (kSrcB)
                    issue_bits_s(land, x.Sb, wrap_row(x.r0 + s + 3, L), L, lane);
                else
                    issue_raw_s(land, x.S, wrap_row(x.r0 + s + 3, L), L, lane);
                cp_async_commit();
            }
        }
        const uint32_t t = q0;
        q0 = q1;
        q1 = q2;
        q2 = q3;
        q3 = t;
    }
    drain_acc(acc, dm, db);
}

}  // namespace split

// Two blocks of 8 warps (or four of 4) per SM, so up to 128 registers per
// thread: the compiler interleaves the Philox rounds of a chunk's words.
template <int WARPS, int LAYOUT>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) ising_strip_kernel(IsingSweepArgs a) {
    constexpr bool kBits = (LAYOUT & (kSrcBits | kDstBits)) != 0;
    extern __shared__ __align__(16) unsigned char ring_bytes[];
    __shared__ __align__(256) TabEntry tabs[WARPS][2][256 / sizeof(TabEntry)];
    __shared__ uint2 lut[(LAYOUT & kSrcBits) ? 256 : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = a.state->t;
    const int gw = blockIdx.x * WARPS + warp, nw = gridDim.x * WARPS;
    if constexpr ((LAYOUT & kSrcBits) != 0) {
        for (int k = threadIdx.x; k < 256; k += WARPS * 32) lut[k] = split::bits_lut_entry((uint32_t)k);
        __syncthreads();
    }
    for (int it = gw; it < a.n_items; it += nw) {
        const Item w = a.items[it];
        if (!SPIN_CK((unsigned)w.lat < (unsigned)a.n_lat, 101)) continue;
        const LatDev ld = a.lats[w.lat];
        // the ring holds five rows of at most 2048 bytes
        if (!SPIN_CK((ld.L == 512 || ld.L == 1024 || ld.L == 2048) && w.r0 >= 0 && w.nrows >= 1 &&
                         w.r0 + w.nrows <= ld.L && 5u * (unsigned)ld.L <= (unsigned)(kRing * kRowChunks * 16),
                     102))
            continue;
        // packed rows start on 16-byte boundaries
        if (kBits && !SPIN_CK((ld.offset & 127u) == 0, 105)) continue;
        if (lane < kTabStride) {
            const TabEntry e = a.tabs[w.lat * kTabStride + lane];
            tabs[warp][0][lane] = e;
            tabs[warp][1][lane] = TabEntry{e.thr, 0};
        }
        __syncwarp();
        split::Walk x;
        x.S = reinterpret_cast<const uint4 *>(a.src + ld.offset);
        x.D = reinterpret_cast<uint4 *>(a.dst + ld.offset);
        x.ring = (uint32_t)__cvta_generic_to_shared(ring_bytes) + (uint32_t)(warp * kRing * kRowChunks * 16);
        x.L = ld.L;
        x.r0 = w.r0;
        x.nrows = w.nrows;
        x.lane = lane;
        x.P0 = philox_prefix(ld.rng, t, 0u, a.rk);
        x.P1 = philox_prefix(ld.rng, t, 1u, a.rk);
        x.tab_cnt = (uint32_t)__cvta_generic_to_shared(tabs[warp][0]);
        x.tab_halo = (uint32_t)__cvta_generic_to_shared(tabs[warp][1]);
        x.Sb = (LAYOUT & kSrcBits) ? reinterpret_cast<const uint4 *>(a.src_bits + (ld.offset >> 5)) : nullptr;
        x.Db = (LAYOUT & kDstBits) ? a.dst_bits + (ld.offset >> 5) : nullptr;
        x.lut = (uint32_t)__cvta_generic_to_shared(lut);
        int dm = 0, db = 0;
        if (ld.L == 512)
            split::item<2, LAYOUT>(x, a.rk, dm, db);
        else
            split::item<4, LAYOUT>(x, a.rk, dm, db);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
            db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
        }
        if (lane == 0) {
            if (dm) atomicAdd(reinterpret_cast<unsigned long long *>(a.delta + 2 * w.lat), (unsigned long long)(long long)dm);
            if (db) atomicAdd(reinterpret_cast<unsigned long long *>(a.delta + 2 * w.lat + 1), (unsigned long long)(long long)db);
        }
        __syncwarp();
    }
}

// Copy every lattice (L*L elements of `elem` bytes at its offset) src -> dst.
__global__ void copy_lattices_kernel(const unsigned char *src, unsigned char *dst,
                                     const LatDev *lats, int elem) {
    const LatDev ld = lats[blockIdx.y];
    const size_t base = ld.offset * (size_t)elem;
    const size_t bytes = (size_t)ld.L * ld.L * elem;
    if (((base | bytes) & 15) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + base);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + base);
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bytes / 16;
             i += (size_t)gridDim.x * blockDim.x)
            d4[i] = s4[i];
    } else {
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < bytes;
             i += (size_t)gridDim.x * blockDim.x)
            dst[base + i] = src[base + i];
    }
}

// Tile kernel: a CTA takes work items (a whole small lattice, or a block of
// rows with a two-row halo on each side) into shared memory in the x8 form,
// updates colour 0 on the item and its inner halo rows (their updates use the
// same site-keyed draws as the neighbouring item's), then colour 1 on the
// item, and writes the item's rows back as +-1 bytes.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) ising_fused_kernel(IsingSweepArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    // [0]: statistics deltas; [1]: zero deltas (recomputed halo rows)
    __shared__ __align__(256) TabEntry stab[2][256 / sizeof(TabEntry)];
    __shared__ int red[2 * (THREADS / 32)];
    uint4 *sm4 = reinterpret_cast<uint4 *>(sm);
    const uint32_t *sm32 = reinterpret_cast<const uint32_t *>(sm);
    const uint32_t t = a.state->t;
    const uint32_t tb_cnt = (uint32_t)__cvta_generic_to_shared(stab[0]);
    const uint32_t tb_halo = (uint32_t)__cvta_generic_to_shared(stab[1]);
    for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
        const Item w = a.items[it];
        if (!SPIN_CK((unsigned)w.lat < (unsigned)a.n_lat, 111)) continue;   // the whole block skips alike
        const LatDev ld = a.lats[w.lat];
        const int L = ld.L, Lv = L >> 4;
        const int halo = w.whole ? 0 : 2;
        const int nload = w.nrows + 2 * halo;
        // rows in range, and the rows plus halo fit the launch's shared memory
        if (!SPIN_CK(L >= 16 && (L & 15) == 0 && w.r0 >= 0 && w.nrows >= 1 && w.r0 + w.nrows <= L &&
                         (!w.whole || (w.r0 == 0 && w.nrows == L)) &&
                         (unsigned)nload * (unsigned)L <= dynamic_smem_bytes(),
                     112))
            continue;
        const uint4 *S = reinterpret_cast<const uint4 *>(a.src + ld.offset);
        uint4 *Dg = reinterpret_cast<uint4 *>(a.dst + ld.offset);
        // chunk v = threadIdx.x + k THREADS of a row range is (row i, column j);
        // the walk adds (di, dj) = THREADS as rows and columns
        const int di = THREADS / Lv, dj = THREADS - di * Lv;
        const int i0 = (int)threadIdx.x / Lv, j0 = (int)threadIdx.x - i0 * Lv;
        {
            int i = i0, j = j0;
            for (int v = threadIdx.x; v < nload * Lv; v += THREADS) {
                int gy = w.r0 - halo + i;
                gy = gy < 0 ? gy + L : (gy >= L ? gy - L : gy);
                sm4[v] = to_x8(__ldg(S + (size_t)gy * Lv + j));
                i += di;
                j += dj;
                if (j >= Lv) {
                    j -= Lv;
                    ++i;
                }
            }
        }
        if (threadIdx.x < kTabStride) {
            const TabEntry e = a.tabs[w.lat * kTabStride + threadIdx.x];
            stab[0][threadIdx.x] = e;
            stab[1][threadIdx.x] = TabEntry{e.thr, 0};
        }
        __syncthreads();
        int acc = 0;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            // colour 0 also on the inner halo ring (smem rows 1 and nrows + 2)
            const int lo = w.whole ? 0 : (c == 0 ? 1 : 2);
            const int hi = w.whole ? w.nrows : (c == 0 ? w.nrows + 3 : w.nrows + 2);
            const int n_units = (hi - lo) * Lv;
            const PhiloxPrefix P = philox_prefix(ld.rng, t, (uint32_t)c, a.rk);
            int i = lo + i0, j = j0;
            for (int v = threadIdx.x; v < n_units; v += THREADS) {
                const int iu = (i == 0) ? nload - 1 : i - 1;
                const int id = (i == nload - 1) ? 0 : i + 1;
                int gy = w.r0 - halo + i;
                gy = gy < 0 ? gy + L : (gy >= L ? gy - L : gy);
                const int row = i * Lv;
                const uint4 Cc = sm4[row + j];
                const uint4 Uc = sm4[iu * Lv + j];
                const uint4 Dc = sm4[id * Lv + j];
                const uint32_t lw = sm32[(row + (j == 0 ? Lv - 1 : j - 1)) * 4 + 3];
                const uint32_t rw = sm32[(row + (j == Lv - 1 ? 0 : j + 1)) * 4];
                const bool count = (i >= halo) && (i < halo + w.nrows);
                const uint32_t g0 = (uint32_t)gy * (uint32_t)(L >> 3) + 2u * (uint32_t)j;
                sm4[row + j] = chunk_x8(Cc, Uc, Dc, lw, rw, philox_from_prefix(g0, P, a.rk),
                                        philox_from_prefix(g0 + 1u, P, a.rk), row_par((c ^ gy) & 1),
                                        count ? tb_cnt : tb_halo, acc);
                i += di;
                j += dj;
                if (j >= Lv) {
                    j -= Lv;
                    ++i;
                }
            }
            __syncthreads();
        }
        {
            int i = i0, j = j0;
            for (int v = threadIdx.x; v < w.nrows * Lv; v += THREADS) {
                const uint4 x8 = sm4[(halo + i) * Lv + j];
                Dg[(size_t)(w.r0 + i) * Lv + j] = make_uint4(from_x8(x8.x), from_x8(x8.y), from_x8(x8.z), from_x8(x8.w));
                i += di;
                j += dj;
                if (j >= Lv) {
                    j -= Lv;
                    ++i;
                }
            }
        }
        flush_ising_acc<THREADS>(acc, a.delta + 2 * w.lat, red);
        __syncthreads();
    }
}

// Resident form: one CTA per lattice keeps the whole lattice in shared memory
// for all n sweeps of a call (small lattices, launch-latency-bound batches),
// in the x8 form of the strip kernel (a spin is the byte 8 [s < 0]; table
// entries addressed by PRMT).  Statistics are reduced by the block after every
// sweep and recorded by the CTA itself; the sweep and record counters come
// from the host (t0, rec0).
template <int THREADS>
__global__ void __launch_bounds__(THREADS) ising_resident_kernel(ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(256) TabEntry stab[256 / sizeof(TabEntry)];
    __shared__ int red[2 * (THREADS / 32)];
    __shared__ long long cur_s[2];
    const int lat = blockIdx.x;
    const LatDev ld = a.lats[lat];
    const int L = ld.L, Lv = L >> 4;
    // the whole lattice fits the launch's shared memory (one block per lattice)
    if (!SPIN_CK(L >= 16 && (L & 15) == 0 && (unsigned)(L * L) <= dynamic_smem_bytes(), 113)) return;
    uint4 *sm4 = reinterpret_cast<uint4 *>(sm);
    const uint32_t *sm32 = reinterpret_cast<const uint32_t *>(sm);
    uint4 *G = reinterpret_cast<uint4 *>(a.spins + ld.offset);
    for (int v = threadIdx.x; v < L * Lv; v += THREADS) sm4[v] = to_x8(G[v]);
    if (threadIdx.x < kTabStride) stab[threadIdx.x] = a.tabs[lat * kTabStride + threadIdx.x];
    if (threadIdx.x < 2) cur_s[threadIdx.x] = a.st.cur[2 * lat + threadIdx.x];
    const uint32_t tb = (uint32_t)__cvta_generic_to_shared(stab);
    // chunk v = threadIdx.x + k THREADS is (row i, column j); the walk adds
    // (di, dj) = THREADS as rows and columns instead of dividing
    const int di = THREADS / Lv, dj = THREADS - di * Lv;
    const int i0 = (int)threadIdx.x / Lv, j0 = (int)threadIdx.x - i0 * Lv;
    __syncthreads();
    for (int sweep = 0; sweep < a.n_sweeps; ++sweep) {
        const uint32_t t = a.t0 + (uint32_t)sweep;
        int acc = 0;
        for (int c = 0; c < 2; ++c) {
            const PhiloxPrefix P = philox_prefix(ld.rng, t, (uint32_t)c, a.rk);
            int i = i0, j = j0;
            for (int v = threadIdx.x; v < L * Lv; v += THREADS) {
                const int iu = i == 0 ? L - 1 : i - 1, id = i == L - 1 ? 0 : i + 1;
                const int row = i * Lv;
                const uint4 Cc = sm4[v];
                const uint4 Uc = sm4[iu * Lv + j];
                const uint4 Dc = sm4[id * Lv + j];
                const uint32_t lw = sm32[(row + (j == 0 ? Lv - 1 : j - 1)) * 4 + 3];
                const uint32_t rw = sm32[(row + (j == Lv - 1 ? 0 : j + 1)) * 4];
                const uint32_t g0 = (uint32_t)i * (uint32_t)(L >> 3) + 2u * (uint32_t)j;
                sm4[v] = chunk_x8(Cc, Uc, Dc, lw, rw, philox_from_prefix(g0, P, a.rk),
                                  philox_from_prefix(g0 + 1u, P, a.rk), row_par((c ^ i) & 1), tb, acc);
                i += di;
                j += dj;
                if (j >= Lv) {
                    j -= Lv;
                    ++i;
                }
            }
            __syncthreads();
        }
        int dm = (int)(int16_t)(acc & 0xFFFF);
        int db = (acc - dm) >> 16;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
            db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[2 * (threadIdx.x >> 5)] = dm;
            red[2 * (threadIdx.x >> 5) + 1] = db;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long sm_ = 0, sb_ = 0;
            for (int w = 0; w < THREADS / 32; ++w) {
                sm_ += red[2 * w];
                sb_ += red[2 * w + 1];
            }
            cur_s[0] += sm_;
            cur_s[1] += sb_;
            if (a.record && a.st.cap > 0) {
                const long long slot = (a.rec0 + sweep) % a.st.cap;
                a.st.ring[(slot * a.st.n_lat + lat) * 2] = cur_s[0];
                a.st.ring[(slot * a.st.n_lat + lat) * 2 + 1] = cur_s[1];
            }
        }
        __syncthreads();
    }
    for (int v = threadIdx.x; v < L * Lv; v += THREADS) {
        const uint4 w = sm4[v];
        G[v] = make_uint4(from_x8(w.x), from_x8(w.y), from_x8(w.z), from_x8(w.w));
    }
    if (threadIdx.x < 2) a.st.cur[2 * lat + threadIdx.x] = cur_s[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Resident kernel split over a thread-block cluster: lattice l is held by the
// CS CTAs of cluster l, CTA r owning rows [r L/CS, (r+1) L/CS) in shared
// memory for every sweep of a call.  A batch of fewer lattices than SMs (the
// one-CTA form leaves SMs idle) then spreads over CS times as many CTAs.
//
// Each CTA keeps its rows plus two halo rows (the row above its first and the
// row below its last) in two buffers.  Sub-step k (k = 2 sweep + c) reads
// halo buffer k & 1; a thread that finishes a chunk of its first or last row
// also stores it, through distributed shared memory, into the halo buffer
// (k + 1) & 1 of the CTA owning the rows above or below.  One cluster barrier
// ends each sub-step: it orders those stores before the next sub-step's reads,
// and the buffer a sub-step writes was last read in the sub-step before that
// barrier.  Draws are those of the one-CTA form (site-keyed Philox counters),
// so the chains are bit-identical.  Statistics: each CTA reduces its changes
// after colour 1 and CTA 0 of the cluster adds the CTAs' parts, read one
// barrier later, to the lattice's running values and records them.
template <int THREADS, int CS>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(THREADS)
    ising_resident_cluster_kernel(ResidentArgs a) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(256) TabEntry stab[256 / sizeof(TabEntry)];
    __shared__ int red[2 * (THREADS / 32)];
    __shared__ long long part[2][CS][2];   // CTA 0: each CTA's (dM, dB) of a sweep, by sweep parity
    __shared__ long long cur_s[2];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int lat = blockIdx.x / CS;
    const LatDev ld = a.lats[lat];
    const int L = ld.L, Lv = L >> 4, R = L / CS, y0 = rank * R;
    // every CTA of the cluster holds the same lattice, so all return together
    if (!SPIN_CK(L >= 16 && (L & 15) == 0 && L % CS == 0 && (unsigned)((R + 4) * L) <= dynamic_smem_bytes(), 114))
        return;
    uint4 *own = reinterpret_cast<uint4 *>(sm);               // [R][Lv]
    uint4 *halo = own + R * Lv;                               // [2 buffers][top, bottom][Lv]
    const uint32_t *own32 = reinterpret_cast<const uint32_t *>(sm);
    const int up = (rank + CS - 1) % CS, dn = (rank + 1) % CS;
    uint4 *up_halo = cl.map_shared_rank(halo, up);            // its bottom halo holds our first row
    uint4 *dn_halo = cl.map_shared_rank(halo, dn);            // its top halo holds our last row
    long long(*part0)[CS][2] = cl.map_shared_rank(part, 0);
    const uint4 *G = reinterpret_cast<const uint4 *>(a.spins + ld.offset);
    for (int v = threadIdx.x; v < R * Lv; v += THREADS) own[v] = to_x8(G[(size_t)y0 * Lv + v]);
    for (int v = threadIdx.x; v < 2 * Lv; v += THREADS) {
        const int y = v < Lv ? (y0 + L - 1) % L : (y0 + R) % L;
        halo[v] = to_x8(G[(size_t)y * Lv + (v < Lv ? v : v - Lv)]);
    }
    if (threadIdx.x < kTabStride) stab[threadIdx.x] = a.tabs[lat * kTabStride + threadIdx.x];
    if (rank == 0 && threadIdx.x < 2) cur_s[threadIdx.x] = a.st.cur[2 * lat + threadIdx.x];
    const uint32_t tb = (uint32_t)__cvta_generic_to_shared(stab);
    const int di = THREADS / Lv, dj = THREADS - di * Lv;
    const int i0 = (int)threadIdx.x / Lv, j0 = (int)threadIdx.x - i0 * Lv;
    // the CTA 0 side of the statistics: add the parts of sweep s to the running values
    auto record = [&](int s) {
        long long dm = 0, db = 0;
        for (int r = 0; r < CS; ++r) {
            dm += part[s & 1][r][0];
            db += part[s & 1][r][1];
        }
        cur_s[0] += dm;
        cur_s[1] += db;
        if (a.record && a.st.cap > 0) {
            const long long slot = (a.rec0 + s) % a.st.cap;
            a.st.ring[(slot * a.st.n_lat + lat) * 2] = cur_s[0];
            a.st.ring[(slot * a.st.n_lat + lat) * 2 + 1] = cur_s[1];
        }
    };
    cl.sync();   // own rows, halos, table and running values in place in every CTA
    for (int sweep = 0; sweep < a.n_sweeps; ++sweep) {
        const uint32_t t = a.t0 + (uint32_t)sweep;
        int acc = 0;
        for (int c = 0; c < 2; ++c) {
            const int b = c;   // k & 1 with k = 2 sweep + c
            const uint4 *top = halo + (2 * b) * Lv, *bot = halo + (2 * b + 1) * Lv;
            uint4 *up_dst = up_halo + (2 * (b ^ 1) + 1) * Lv, *dn_dst = dn_halo + (2 * (b ^ 1)) * Lv;
            const PhiloxPrefix P = philox_prefix(ld.rng, t, (uint32_t)c, a.rk);
            int i = i0, j = j0;
            for (int v = threadIdx.x; v < R * Lv; v += THREADS) {
                const int y = y0 + i, row = i * Lv;
                const uint4 Cc = own[v];
                const uint4 Uc = i == 0 ? top[j] : own[v - Lv];
                const uint4 Dc = i == R - 1 ? bot[j] : own[v + Lv];
                const uint32_t lw = own32[(row + (j == 0 ? Lv - 1 : j - 1)) * 4 + 3];
                const uint32_t rw = own32[(row + (j == Lv - 1 ? 0 : j + 1)) * 4];
                const uint32_t g0 = (uint32_t)y * (uint32_t)(L >> 3) + 2u * (uint32_t)j;
                const uint4 nv = chunk_x8(Cc, Uc, Dc, lw, rw, philox_from_prefix(g0, P, a.rk),
                                          philox_from_prefix(g0 + 1u, P, a.rk), row_par((c ^ y) & 1), tb, acc);
                own[v] = nv;
                if (i == 0) up_dst[j] = nv;
                if (i == R - 1) dn_dst[j] = nv;
                i += di;
                j += dj;
                if (j >= Lv) {
                    j -= Lv;
                    ++i;
                }
            }
            if (c == 1) {
                int dm = (int)(int16_t)(acc & 0xFFFF);
                int db = (acc - dm) >> 16;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    dm += __shfl_xor_sync(0xFFFFFFFFu, dm, o);
                    db += __shfl_xor_sync(0xFFFFFFFFu, db, o);
                }
                if ((threadIdx.x & 31) == 0) {
                    red[2 * (threadIdx.x >> 5)] = dm;
                    red[2 * (threadIdx.x >> 5) + 1] = db;
                }
            }
            cl.sync();
            // CTA 0: the parts of the previous sweep arrived before this barrier
            if (c == 0 && sweep > 0 && rank == 0 && threadIdx.x == 0) record(sweep - 1);
        }
        if (threadIdx.x == 0) {   // this CTA's part of the sweep, into CTA 0
            long long sm_ = 0, sb_ = 0;
            for (int w = 0; w < THREADS / 32; ++w) {
                sm_ += red[2 * w];
                sb_ += red[2 * w + 1];
            }
            part0[sweep & 1][rank][0] = sm_;
            part0[sweep & 1][rank][1] = sb_;
        }
    }
    cl.sync();   // the last sweep's parts are in CTA 0
    if (a.n_sweeps > 0 && rank == 0 && threadIdx.x == 0) record(a.n_sweeps - 1);
    uint4 *Gw = reinterpret_cast<uint4 *>(a.spins + ld.offset);
    for (int v = threadIdx.x; v < R * Lv; v += THREADS) {
        const uint4 w = own[v];
        Gw[(size_t)y0 * Lv + v] = make_uint4(from_x8(w.x), from_x8(w.y), from_x8(w.z), from_x8(w.w));
    }
    if (rank == 0) {
        __syncthreads();
        if (threadIdx.x < 2) a.st.cur[2 * lat + threadIdx.x] = cur_s[threadIdx.x];
    }
}

}  // namespace

cudaError_t launch_copy_lattices(const void *src, void *dst, const LatDev *lats, int n_lat,
                                 int elem, cudaStream_t s) {
    dim3 grid(64, n_lat);
    copy_lattices_kernel<<<grid, 256, 0, s>>>(static_cast<const unsigned char *>(src),
                                              static_cast<unsigned char *>(dst), lats, elem);
    return cudaGetLastError();
}

cudaError_t launch_ising_fused(const IsingSweepArgs &a, int grid, int threads, size_t smem,
                               cudaStream_t s) {
    switch (threads) {
        case 128:
            ising_fused_kernel<128><<<grid, 128, smem, s>>>(a);
            break;
        case 256:
            ising_fused_kernel<256><<<grid, 256, smem, s>>>(a);
            break;
        case 512:
            ising_fused_kernel<512><<<grid, 512, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t strip_smem(int warps) { return strip_ring_bytes(warps); }

namespace {

template <int WARPS>
cudaError_t launch_strip_layout(const IsingSweepArgs &a, int grid, int layout, cudaStream_t s) {
    const size_t smem = strip_smem(WARPS);
    switch (layout) {
        case 0:
            ising_strip_kernel<WARPS, 0><<<grid, WARPS * 32, smem, s>>>(a);
            break;
        case kSrcSplit:
            ising_strip_kernel<WARPS, kSrcSplit><<<grid, WARPS * 32, smem, s>>>(a);
            break;
        case kDstSplit:
            ising_strip_kernel<WARPS, kDstSplit><<<grid, WARPS * 32, smem, s>>>(a);
            break;
        case kSrcSplit | kDstSplit:
            ising_strip_kernel<WARPS, kSrcSplit | kDstSplit><<<grid, WARPS * 32, smem, s>>>(a);
            break;
        case kSrcBits | kDstBits:
            ising_strip_kernel<WARPS, kSrcBits | kDstBits><<<grid, WARPS * 32, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int WARPS>
cudaError_t strip_smem_attributes() {
    const int smem = (int)strip_smem(WARPS);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ising_strip_kernel<WARPS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(ising_strip_kernel<WARPS, kSrcSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(ising_strip_kernel<WARPS, kDstSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(ising_strip_kernel<WARPS, kSrcBits | kDstBits>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    return cudaFuncSetAttribute(ising_strip_kernel<WARPS, kSrcSplit | kDstSplit>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace

cudaError_t launch_ising_strip(const IsingSweepArgs &a, int grid, int warps, int layout, cudaStream_t s) {
    switch (warps) {
        case 4:
            return launch_strip_layout<4>(a, grid, layout, s);
        case 8:
            return launch_strip_layout<8>(a, grid, layout, s);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_ising_strip(int *blocks_per_sm, int warps) {
    cudaError_t e;
    if ((e = strip_smem_attributes<4>())) return e;
    if ((e = strip_smem_attributes<8>())) return e;
    // the four row-format instances share one body: their occupancy is alike
    if (warps == 4)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ising_strip_kernel<4, 0>, 128, strip_smem(4));
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ising_strip_kernel<8, 0>, 256, strip_smem(8));
}

// The dynamic shared-memory limit of a kernel is process-wide state: it is
// only ever raised (per device), so one caller can never lower it below what
// another caller's launches need.
cudaError_t set_ising_fused_smem(size_t smem) {
    static size_t raised[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    // Raised only when the dynamic share plus the kernel's static tables exceed
    // the default 48 KB: setting the limit without need was measured to slow the
    // sweep (the tile kernel shares the SMs with the strip kernel).
    if (dev < 0 || dev >= 64 || smem <= raised[dev]) return cudaSuccess;
    size_t stat = 0;
    for (const void *k : {(const void *)ising_fused_kernel<128>, (const void *)ising_fused_kernel<256>, (const void *)ising_fused_kernel<512>}) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, k))) return e;
        stat = fa.sharedSizeBytes > stat ? fa.sharedSizeBytes : stat;
    }
    if (smem + stat <= 48 * 1024) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(ising_fused_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(ising_fused_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(ising_fused_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    raised[dev] = smem;
    return cudaSuccess;
}

cudaError_t launch_ising_resident(const ResidentArgs &a, int n_lat, int threads, size_t smem,
                                  DevState *state, cudaStream_t s) {
    cudaError_t e;
    switch (threads) {
        case 128:
            if ((e = cudaFuncSetAttribute(ising_resident_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
            ising_resident_kernel<128><<<n_lat, 128, smem, s>>>(a);
            break;
        case 256:
            if ((e = cudaFuncSetAttribute(ising_resident_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
            ising_resident_kernel<256><<<n_lat, 256, smem, s>>>(a);
            break;
        case 512:
            if ((e = cudaFuncSetAttribute(ising_resident_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
            ising_resident_kernel<512><<<n_lat, 512, smem, s>>>(a);
            break;
        case 1024:
            if ((e = cudaFuncSetAttribute(ising_resident_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
            ising_resident_kernel<1024><<<n_lat, 1024, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if ((e = cudaGetLastError())) return e;
    advance_state_kernel<<<1, 1, 0, s>>>(state, (uint32_t)a.n_sweeps, a.record);
    return cudaGetLastError();
}

namespace {
template <int THREADS, int CS>
cudaError_t launch_resident_cluster(const ResidentArgs &a, int n_lat, size_t smem, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ising_resident_cluster_kernel<THREADS, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)))
        return e;
    ising_resident_cluster_kernel<THREADS, CS><<<n_lat * CS, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_ising_resident_cluster(const ResidentArgs &a, int n_lat, int threads, int cs, int max_l,
                                          DevState *state, cudaStream_t s) {
    if ((cs != 2 && cs != 4) || max_l < 16 || max_l % 16 != 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(max_l / cs + 4) * (size_t)max_l;
    cudaError_t e;
    switch (threads * 10 + cs) {
        case 2562: e = launch_resident_cluster<256, 2>(a, n_lat, smem, s); break;
        case 5122: e = launch_resident_cluster<512, 2>(a, n_lat, smem, s); break;
        case 10242: e = launch_resident_cluster<1024, 2>(a, n_lat, smem, s); break;
        case 2564: e = launch_resident_cluster<256, 4>(a, n_lat, smem, s); break;
        case 5124: e = launch_resident_cluster<512, 4>(a, n_lat, smem, s); break;
        case 10244: e = launch_resident_cluster<1024, 4>(a, n_lat, smem, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e) return e;
    advance_state_kernel<<<1, 1, 0, s>>>(state, (uint32_t)a.n_sweeps, a.record);
    return cudaGetLastError();
}

cudaError_t launch_ising_tri_resident(const ResidentArgs &a, int n_lat, size_t smem, DevState *state,
                                      cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ising_tri_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    ising_tri_resident_kernel<<<n_lat, kTriResThreads, smem, s>>>(a);
    if ((e = cudaGetLastError())) return e;
    advance_state_kernel<<<1, 1, 0, s>>>(state, (uint32_t)a.n_sweeps, a.record);
    return cudaGetLastError();
}

cudaError_t launch_ising_plain(int8_t *spins, const LatDev *, int lat, uint32_t rng, int L, const TabEntry *tabs,
                               uint32_t k0, uint32_t k1, const DevState *state, int64_t *delta,
                               int colour, cudaStream_t s) {
    const int units = L * (L >> 4);
    ising_plain_kernel<<<(units + 255) / 256, 256, 0, s>>>(
        spins, L, (uint32_t)lat, rng, tabs + lat * kTabStride, k0, k1, state, delta, colour);
    return cudaGetLastError();
}

cudaError_t launch_ising_tri(const int8_t *src, int8_t *dst, const int32_t *lat_ids, int n, int maxL,
                             const LatDev *lats, const TabEntry *tabs, uint32_t k0, uint32_t k1,
                             const DevState *state, int64_t *delta, int colour, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (maxL * maxL + 255) / 256;
    dim3 grid(blocks < 64 ? blocks : 64, n);
    ising_tri_kernel<<<grid, 256, 0, s>>>(src, dst, lat_ids, lats, tabs, k0, k1, state, delta, colour);
    return cudaGetLastError();
}

cudaError_t launch_ising_nnn(const int8_t *src, int8_t *dst, int n, int maxL, const LatDev *lats,
                             const uint32_t *thr, uint32_t k0, uint32_t k1, const DevState *state,
                             int64_t *delta, int colour, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int groups = ((maxL / 2) * (maxL / 2) + 3) / 4;
    const int blocks = (groups + kNnnThreads - 1) / kNnnThreads;
    dim3 grid(blocks < 64 ? blocks : 64, n);
    ising_nnn_kernel<<<grid, kNnnThreads, 0, s>>>(src, dst, lats, thr, k0, k1, state, delta, colour);
    return cudaGetLastError();
}

cudaError_t launch_ising_nnn_resident(const ResidentArgs &a, const uint32_t *thr, int n_lat, size_t smem,
                                      DevState *state, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(ising_nnn_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    ising_nnn_resident_kernel<<<n_lat, kNnnResThreads, smem, s>>>(a, thr);
    if ((e = cudaGetLastError())) return e;
    advance_state_kernel<<<1, 1, 0, s>>>(state, (uint32_t)a.n_sweeps, a.record);
    return cudaGetLastError();
}

cudaError_t launch_ising_generic(const int8_t *src, int8_t *dst, const int32_t *lat_ids, int n,
                                 int maxL, const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                 uint32_t k1, const DevState *state, int64_t *delta, int colour,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int blocks = (maxL * maxL + 255) / 256;
    dim3 grid(blocks < 64 ? blocks : 64, n);
    ising_generic_kernel<<<grid, 256, 0, s>>>(src, dst, lat_ids, lats, tabs, k0, k1, state, delta,
                                              colour);
    return cudaGetLastError();
}

cudaError_t launch_init_random(void *spins, int model, const LatDev *lats, int n_lat, int maxL,
                               uint32_t k0, uint32_t k1, cudaStream_t s) {
    const int groups = (maxL * maxL) >> 2;
    const int bx = (groups + 255) / 256;
    dim3 grid(bx < 256 ? bx : 256, n_lat);
    init_random_kernel<<<grid, 256, 0, s>>>(spins, model, lats, k0, k1);
    return cudaGetLastError();
}

SPIN_CHECK_ACCESSOR(check_word_ising)

}  // namespace spinmc
