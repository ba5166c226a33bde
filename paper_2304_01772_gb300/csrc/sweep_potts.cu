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
#include "strip.cuh"

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
        if (!SPIN_CK((unsigned)w.lat < (unsigned)a.n_lat, 123)) continue;   // the whole block skips alike
        const LatDev ld = a.lats[w.lat];
        const int L = ld.L, Lv = L >> 4;
        const uint32_t q = (uint32_t)ld.q;
        const bool small_q = q <= 8;
        const int halo = w.whole ? 0 : 2;
        const int nload = w.nrows + 2 * halo;
        if (!SPIN_CK(L >= 16 && (L & 15) == 0 && w.r0 >= 0 && w.nrows >= 1 && w.r0 + w.nrows <= L &&
                         (unsigned)nload * (unsigned)L <= dynamic_smem_bytes(),
                     124))
            continue;
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
                    potts_chunk(Cc, Uc, Dc, lw, rw, gbase, (c ^ gy) & 1, ld.rng, t,
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

// ------------------------------------------------------------ strip kernel
// Lattices with q <= 8 and L = 512, 1024 or 2048, in the split form of the
// Ising strip kernel: one warp walks full rows [r0, r0 + R) of one lattice;
// step s updates colour 0 on row s, then colour 1 on row s - 1, both on the
// words of half p = y_s & 1 of the rows (rows are held as colour-compressed
// halves: sites of even x, then of odd x).  Rows s - 2 .. s + 1 sit in four
// split slots, row s + 2 lands by cp.async in a fifth; rows -1 and R are the
// recomputed colour-0 halo (the same site-keyed draws as in the neighbouring
// item), so items never exchange data.
//
// All four bytes of a word are active sites.  Sites 0 and 1 of word w use
// lanes (0, 1) and (2, 3) of Philox block g0 = (y L / 2 + 4 w) / 2 (acceptance
// draw, proposal draw), sites 2 and 3 those of block g0 + 1.  Per word, byte-
// parallel for states below 8:
//  * the proposals s' = (s + 1 + mulhi(u1, q - 1)) mod q: the four offsets
//    packed into one word, s + offset + 1 (at most 2q - 1) reduced through the
//    sign bit of (that + 128 - q);
//  * (a ^ b) + 7 has bit 3 set exactly when a != b, so a flag 8 [a != b] costs
//    three operations and never carries; over the four neighbour words (up,
//    down, the other half, the other half shifted by one site)
//    32 + sum 8 [!= s'] - sum 8 [!= s] = 8 (n_same(s) - n_same(s') + 4) is
//    the byte offset of the site's 8-byte table entry (index d + 4 for the
//    energy change J d);
//  * an accepted site takes its proposal (xor with s ^ s' in its byte) and
//    adds its table delta (the change of the equal-bond count).
// State counts are taken on the finished rows from bit-plane products in
// per-byte counters; the item holding row 0 subtracts the old counts, so
// `delta` receives the change.
//
// LAYOUT (kSrcSplit, kDstSplit) as in the Ising strip kernel: within a call
// of several sweeps the ping-pong buffer holds the strip lattices' rows as
// their two halves (even-x states, then odd-x states), so a landed row is a
// ring slot as it is and a finished row is stored without re-interleaving.
constexpr uint32_t kOnes = 0x01010101u;

// Every byte replaced by copies of its top bit (prmt with sign replication).
__device__ __forceinline__ uint32_t byte_signs(uint32_t v) {
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(r) : "r"(v));
    return r;
}

// If u <= thr: w ^= (xm & m) (the site takes its proposal) and acc += delta
// (an add with an unused carry-out, as in the Ising accept_site).
__device__ __forceinline__ void potts_accept(uint32_t &w, int &acc, uint32_t u, uint2 e,
                                             uint32_t xm, uint32_t m) {
    asm("{\n\t.reg .pred p;\n\t"
        "setp.le.u32 p, %2, %3;\n\t"
        "@p lop3.b32 %0, %0, %4, %5, 0x78;\n\t"
        "@p add.cc.u32 %1, %1, %6;\n\t}"
        : "+r"(w), "+r"(acc)
        : "r"(u), "r"(e.x), "r"(xm), "r"(m), "r"(e.y));
}

__device__ __forceinline__ uint32_t pair_flags(uint32_t a, uint32_t b) {
    return ((a ^ b) + 0x07070707u) & 0x08080808u;
}

// Per-byte counters of the bit planes of the states in the words a and b.
// QB = 2: h = (b0, b1, b0 b1); QB = 3: h = (b0, b1, b0 b1, b2, b0 b2, b1 b2,
// b0 b1 b2), bk the bit k of a state.  drain_counts turns them into the counts
// of the states 1 .. 2^QB - 1 by inclusion-exclusion (state 0 is the rest).
template <int QB>
__device__ __forceinline__ void count_planes(uint32_t a, uint32_t b, uint32_t (&h)[(1 << QB) - 1]) {
    const uint32_t a1 = a >> 1, b1 = b >> 1;
    const uint32_t a01 = a & a1, b01 = b & b1;
    h[0] += (a & kOnes) + (b & kOnes);
    h[1] += (a1 & kOnes) + (b1 & kOnes);
    h[2] += (a01 & kOnes) + (b01 & kOnes);
    if constexpr (QB > 2) {
        const uint32_t a2 = a >> 2, b2 = b >> 2;
        h[3] += (a2 & kOnes) + (b2 & kOnes);
        h[4] += (a & a2 & kOnes) + (b & b2 & kOnes);
        h[5] += (a1 & a2 & kOnes) + (b1 & b2 & kOnes);
        h[6] += (a01 & a2 & kOnes) + (b01 & b2 & kOnes);
    }
}

// Per-byte plane counters -> the warp's state counts in shared memory
// (tot[k - 1] += n_k; lane 0 writes).
template <int QB>
__device__ __forceinline__ void drain_counts(uint32_t (&h)[(1 << QB) - 1], uint32_t *tot, int lane) {
    uint32_t T[(1 << QB) - 1];
#pragma unroll
    for (int k = 0; k < (1 << QB) - 1; ++k) {
        T[k] = __reduce_add_sync(0xFFFFFFFFu, __dp4a(h[k], kOnes, 0u));
        h[k] = 0u;
    }
    if (lane == 0) {
        if constexpr (QB == 2) {
            tot[0] += T[0] - T[2];                    // state 1: b0 only
            tot[1] += T[1] - T[2];                    // state 2: b1 only
            tot[2] += T[2];                           // state 3
        } else {
            const uint32_t p0 = T[0], p1 = T[1], p01 = T[2], p2 = T[3], p02 = T[4], p12 = T[5], p012 = T[6];
            tot[0] += p0 - p01 - p02 + p012;          // 1
            tot[1] += p1 - p01 - p12 + p012;          // 2
            tot[2] += p01 - p012;                     // 3
            tot[3] += p2 - p02 - p12 + p012;          // 4
            tot[4] += p02 - p012;                     // 5
            tot[5] += p12 - p012;                     // 6
            tot[6] += p012;                           // 7
        }
    }
}

namespace psplit {

// Raw row (L state bytes) at src -> its two halves at dst (dst != src).
__device__ __forceinline__ void split_row(uint32_t src, uint32_t dst, int L, int lane) {
#pragma unroll 1
    for (int k = lane; k < (L >> 4); k += 32) {
        const Words<4> v = ldw<4>(src, k);
        Words<2> e, o;
        e.w[0] = prmt(v.w[0], v.w[1], 0x6420u), e.w[1] = prmt(v.w[2], v.w[3], 0x6420u);
        o.w[0] = prmt(v.w[0], v.w[1], 0x7531u), o.w[1] = prmt(v.w[2], v.w[3], 0x7531u);
        stw<2>(dst, k, e);
        stw<2>(dst + (uint32_t)(L >> 1), k, o);
    }
}

struct Walk {
    const uint4 *S;
    uint4 *D;
    uint32_t ring;   // shared address of this warp's 5 * L bytes: 4 split rows + landing
    int L, r0, nrows, lane;
    uint32_t q1, vadd, qq;
    PhiloxPrefix P0, P1;
    uint32_t tab_cnt, tab_halo;
};

// Metropolis update of the active words `act` (see the section comment);
// `edge` is the other-half word just outside the chunk (before it for p = 0,
// after it for p = 1); blocks g + 2 i, g + 2 i + 1 serve word i.
template <int NW>
__device__ __forceinline__ void update(Words<NW> &act, const Words<NW> &oth, uint32_t edge, const Words<NW> &up,
                                       const Words<NW> &dn, uint32_t g, const PhiloxPrefix &PP,
                                       const PhiloxKeys &rk, int p, uint32_t selH, const Walk &x, uint32_t stab,
                                       int &acc) {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const uint32_t nb = p ? (i + 1 < NW ? oth.w[i + 1] : edge) : (i > 0 ? oth.w[i - 1] : edge);
        const uint32_t H = prmt(oth.w[i], nb, selH);
        const uint32_t S = act.w[i];
        const uint4 ra = philox_from_prefix(g + 2u * (uint32_t)i, PP, rk);
        const uint4 rb = philox_from_prefix(g + 2u * (uint32_t)i + 1u, PP, rk);
        const uint32_t m01 = prmt(__umulhi(ra.y, x.q1), __umulhi(ra.w, x.q1), 0x0040u);
        const uint32_t m23 = prmt(__umulhi(rb.y, x.q1), __umulhi(rb.w, x.q1), 0x0040u);
        const uint32_t M = prmt(m01, m23, 0x5410u);
        const uint32_t raw = S + M + kOnes;
        const uint32_t E = byte_signs(S + M + x.vadd);   // 0xFF where raw >= q
        const uint32_t SP = raw - (E & x.qq);
        const uint32_t K = 0x20202020u + pair_flags(up.w[i], SP) + pair_flags(dn.w[i], SP) +
                           pair_flags(oth.w[i], SP) + pair_flags(H, SP) - pair_flags(up.w[i], S) -
                           pair_flags(dn.w[i], S) - pair_flags(oth.w[i], S) - pair_flags(H, S);
        SPIN_CK((K & 0x07070707u) == 0u && ((K + 0x3F3F3F3Fu) & 0x80808080u) == 0u, 125);
        const uint32_t xm = S ^ SP;
        uint32_t w = S;
        potts_accept(w, acc, ra.x, lds_u2(prmt(K, stab, 0x7650u)), xm, 0x000000FFu);
        potts_accept(w, acc, ra.z, lds_u2(prmt(K, stab, 0x7651u)), xm, 0x0000FF00u);
        potts_accept(w, acc, rb.x, lds_u2(prmt(K, stab, 0x7652u)), xm, 0x00FF0000u);
        potts_accept(w, acc, rb.z, lds_u2(prmt(K, stab, 0x7653u)), xm, 0xFF000000u);
        act.w[i] = w;
    }
}

// Final row in the split form: the active half's words at half hp, the other
// half's at ho (byte offsets into the destination row).
template <int NW>
__device__ __forceinline__ void store_halves(unsigned char *Drow, int hp, int ho, int c, const Words<NW> &act,
                                             const Words<NW> &oth) {
    st_words<NW>(Drow + hp, c, act);
    st_words<NW>(Drow + ho, c, oth);
}

// Final row: halves -> row-major bytes (no conversion: states are bytes).
template <int NW>
__device__ __forceinline__ void store_row(uint4 *Drow, int c, const Words<NW> &act, const Words<NW> &oth,
                                          uint32_t sel0, uint32_t sel1) {
    uint32_t o[2 * NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        o[2 * i] = prmt(act.w[i], oth.w[i], sel0);
        o[2 * i + 1] = prmt(act.w[i], oth.w[i], sel1);
    }
    if constexpr (NW == 4) {
        Drow[2 * c] = make_uint4(o[0], o[1], o[2], o[3]);
        Drow[2 * c + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
        Drow[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// One item: rows [r0, r0 + nrows) with the recomputed halo rows r0 - 1 and
// r0 + nrows (colour 0 only, no statistics).  NW: words of a half row per
// lane chunk (2 for L = 512, else 4).  LAYOUT: row formats.
template <int NW, int QB, int LAYOUT>
__device__ void item(const Walk &x, const PhiloxKeys &rk, int &acc, uint32_t (&h)[(1 << QB) - 1], uint32_t *tot) {
    constexpr bool kSrcS = (LAYOUT & kSrcSplit) != 0, kDstS = (LAYOUT & kDstSplit) != 0;
    const int L = x.L, lane = x.lane, half = L >> 1, nw = L >> 3, nc = nw / (32 * NW);
    const uint32_t uL = (uint32_t)L;
    uint32_t q0 = x.ring + 3 * uL, q1 = x.ring, q2 = x.ring + uL, q3 = x.ring + 2 * uL;
    uint32_t land = x.ring + 4 * uL;
    if constexpr (kSrcS) {
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
        // rows -2 and -1 land in q0 (free until step -1 ends) and the landing slot
        // and are split into q1 and q2; then row 0 (via q0) into q3, while row 1
        // stays in flight in the landing slot
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
    for (int s = -1; s <= x.nrows; ++s) {
        // q0..q3 hold rows s - 2 .. s + 1
        const int yA = wrap_row(x.r0 + s, L), yB = yA == 0 ? L - 1 : yA - 1;
        const int p = yA & 1;
        const uint32_t selH = p ? 0x4321u : 0x2107u;
        const uint32_t sel0 = p ? 0x1504u : 0x5140u, sel1 = p ? 0x3726u : 0x7362u;
        const uint32_t tabA = (s >= 0 && s < x.nrows) ? x.tab_cnt : x.tab_halo;
        const int hp = p * half, ho = half - hp;
        const uint32_t gA = (uint32_t)yA * (uint32_t)(L >> 2), gB = (uint32_t)yB * (uint32_t)(L >> 2);
        uint4 *Drow = x.D + (size_t)yB * (L >> 4);
        unsigned char *Dsplit = reinterpret_cast<unsigned char *>(Drow);
        const int eoff = p ? NW : -1;
        for (int j = 0; j < nc; ++j) {
            const int c = lane + 32 * j;
            const int we = (NW * c + eoff) & (nw - 1);
            if (!SPIN_CK(4 * NW * (c + 1) <= half && we >= 0 && we < nw, 126)) continue;
            const uint32_t eA = sld1(q2 + (uint32_t)ho + 4u * (uint32_t)we);
            Words<NW> act = ldw<NW>(q2 + (uint32_t)hp, c);
            const Words<NW> oth = ldw<NW>(q2 + (uint32_t)ho, c);
            Words<NW> upA = ldw<NW>(q1 + (uint32_t)hp, c);
            const Words<NW> dnA = ldw<NW>(q3 + (uint32_t)hp, c);
            update<NW>(act, oth, eA, upA, dnA, gA + 2u * (uint32_t)(NW * c), x.P0, rk, p, selH, x, tabA, acc);
            stw<NW>(q2 + (uint32_t)hp, c, act);
            if (s >= 1) {
                const uint32_t eB = sld1(q1 + (uint32_t)ho + 4u * (uint32_t)we);
                const Words<NW> othB = ldw<NW>(q1 + (uint32_t)ho, c);
                const Words<NW> upB = ldw<NW>(q0 + (uint32_t)hp, c);
                update<NW>(upA, othB, eB, upB, act, gB + 2u * (uint32_t)(NW * c), x.P1, rk, p, selH, x,
                           x.tab_cnt, acc);
                if constexpr (kDstS)
                    store_halves<NW>(Dsplit, hp, ho, c, upA, othB);
                else
                    store_row<NW>(Drow, c, upA, othB, sel0, sel1);
#pragma unroll
                for (int i = 0; i < NW; ++i) count_planes<QB>(upA.w[i], othB.w[i], h);
            }
        }
        if ((s & 3) == 3) drain_counts<QB>(h, tot, lane);   // at most 4 steps x 16 words per byte counter
        __syncwarp();
        if (s + 2 <= x.nrows + 1) {
            cp_async_wait_all();
            __syncwarp();
            if constexpr (kSrcS) {
                // row s + 2 takes the slot of row s - 2, which lands the next row
                const uint32_t t = q0;
                q0 = land;
                land = t;
            } else {
                split_row(land, q0, L, lane);      // row s + 2 into the slot of row s - 2
                __syncwarp();
            }
            if (s + 3 <= x.nrows + 1) {
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
    drain_counts<QB>(h, tot, lane);
}

}  // namespace psplit

template <int WARPS, int QB, int LAYOUT>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) potts_strip_kernel(PottsStripArgs a) {
    constexpr int NK = (1 << QB) - 1;
    extern __shared__ __align__(16) unsigned char ring_bytes[];
    // 256-byte tables: an entry's address is the table's with byte 0 replaced
    __shared__ __align__(256) TabEntry tabs[WARPS][2][256 / sizeof(TabEntry)];
    __shared__ uint32_t tots[WARPS][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = a.state->t;
    const int gw = blockIdx.x * WARPS + warp, nw = gridDim.x * WARPS;
    uint32_t *tot = tots[warp];
    for (int it = gw; it < a.n_items; it += nw) {
        const Item w = a.items[it];
        if (!SPIN_CK((unsigned)w.lat < (unsigned)a.n_lat, 121)) continue;
        const LatDev ld = a.lats[w.lat];
        // the ring holds five rows (ring_chunks chunks of 16 bytes each), states fit QB bits
        if (!SPIN_CK((ld.L == 512 || ld.L == 1024 || ld.L == 2048) && (ld.L >> 4) <= a.ring_chunks &&
                         w.r0 >= 0 && w.nrows >= 1 && w.r0 + w.nrows <= ld.L && ld.q >= 2 && ld.q <= (1 << QB),
                     122))
            continue;
        if (lane < kTabStride) {
            const TabEntry e = a.tabs[w.lat * kTabStride + lane];
            tabs[warp][0][lane] = e;
            tabs[warp][1][lane] = TabEntry{e.thr, 0};
        }
        if (lane < 8) tot[lane] = 0u;
        __syncwarp();
        psplit::Walk x;
        x.S = reinterpret_cast<const uint4 *>(a.src + ld.offset);
        x.D = reinterpret_cast<uint4 *>(a.dst + ld.offset);
        x.ring = (uint32_t)__cvta_generic_to_shared(ring_bytes) + (uint32_t)(warp * kRing * a.ring_chunks * 16);
        x.L = ld.L;
        x.r0 = w.r0;
        x.nrows = w.nrows;
        x.lane = lane;
        x.q1 = (uint32_t)ld.q - 1u;
        x.vadd = (0x81u - (uint32_t)ld.q) * kOnes;
        x.qq = (uint32_t)ld.q * kOnes;
        x.P0 = philox_prefix(ld.rng, t, 0u, a.rk);
        x.P1 = philox_prefix(ld.rng, t, 1u, a.rk);
        x.tab_cnt = (uint32_t)__cvta_generic_to_shared(tabs[warp][0]);
        x.tab_halo = (uint32_t)__cvta_generic_to_shared(tabs[warp][1]);
        int acc = 0;
        uint32_t h[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) h[k] = 0u;
        if (ld.L == 512)
            psplit::item<2, QB, LAYOUT>(x, a.rk, acc, h, tot);
        else
            psplit::item<4, QB, LAYOUT>(x, a.rk, acc, h, tot);
        acc = (int)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)acc);
        __syncwarp();
        // lane k adds the change of statistic k (0: B_eq, 1 + k: n_k)
        long long own = 0, v = 0;
#pragma unroll
        for (int k = 0; k < NK; ++k) own += tot[k];
        if (lane >= 2 && lane < NK + 2) v = tot[lane - 2];
        if (lane == 0) v = acc;
        if (lane == 1) v = (long long)w.nrows * ld.L - own;
        const int stat = lane;                        // 0: B_eq, 1 + k: n_k
        if (stat <= ld.q && stat < a.width) {
            int64_t *dl = a.delta + (size_t)a.width * w.lat;
            if (w.r0 == 0 && stat >= 1) v -= a.cur[(size_t)a.width * w.lat + stat];
            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(dl + stat), (unsigned long long)v);
        }
        __syncwarp();
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
        const uint4 r = philox4x32_10(make_uint4(k >> 1, ld.rng, t, (uint32_t)c), k0, k1);
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
// another caller's launches need.
cudaError_t set_potts_fused_smem(size_t smem) {
    static size_t raised[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    // Raised only when the dynamic share plus the kernel's static tables exceed
    // the default 48 KB: setting the limit without need was measured to slow the
    // sweep (the tile kernel shares the SMs with the strip kernel).
    if (dev < 0 || dev >= 64 || smem <= raised[dev]) return cudaSuccess;
    size_t stat = 0;
    for (const void *k : {(const void *)potts_fused_kernel<128>, (const void *)potts_fused_kernel<256>, (const void *)potts_fused_kernel<512>}) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, k))) return e;
        stat = fa.sharedSizeBytes > stat ? fa.sharedSizeBytes : stat;
    }
    if (smem + stat <= 48 * 1024) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaFuncSetAttribute(potts_fused_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    raised[dev] = smem;
    return cudaSuccess;
}

cudaError_t launch_potts_plain(uint8_t *spins, const LatDev *, int lat, uint32_t rng, int L, int q,
                               const TabEntry *tabs, uint32_t k0, uint32_t k1,
                               const DevState *state, int64_t *delta, int width, int colour,
                               cudaStream_t s) {
    const int units = L * (L >> 4);
    potts_plain_kernel<<<(units + 255) / 256, 256, 0, s>>>(
        spins, L, rng, (uint32_t)q, tabs + lat * kTabStride, k0, k1, state,
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

static size_t potts_ring_bytes(int warps, int ring_chunks) {
    return sizeof(uint4) * (size_t)warps * kRing * (size_t)ring_chunks;
}

template <int WARPS, int QB>
static cudaError_t potts_strip_attrs() {
    const int smem = (int)strip_ring_bytes(WARPS);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potts_strip_kernel<WARPS, QB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(potts_strip_kernel<WARPS, QB, kSrcSplit>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    if ((e = cudaFuncSetAttribute(potts_strip_kernel<WARPS, QB, kDstSplit>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem)))
        return e;
    return cudaFuncSetAttribute(potts_strip_kernel<WARPS, QB, kSrcSplit | kDstSplit>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <int QB>
static cudaError_t potts_strip_attrs() {
    cudaError_t e = potts_strip_attrs<4, QB>();
    return e ? e : potts_strip_attrs<8, QB>();
}

cudaError_t occupancy_potts_strip(int *blocks_per_sm, int warps, int qbits, int ring_chunks) {
    cudaError_t e = qbits == 2 ? potts_strip_attrs<2>() : potts_strip_attrs<3>();
    if (e) return e;
    const size_t sm = potts_ring_bytes(warps, ring_chunks);
    // the four row-format instances share one body: their occupancy is alike
    if (qbits == 2)
        return warps == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, potts_strip_kernel<4, 2, 0>, 128, sm)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, potts_strip_kernel<8, 2, 0>, 256, sm);
    return warps == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, potts_strip_kernel<4, 3, 0>, 128, sm)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, potts_strip_kernel<8, 3, 0>, 256, sm);
}

template <int WARPS, int QB>
static cudaError_t launch_potts_strip_layout(const PottsStripArgs &a, int grid, int layout, cudaStream_t s) {
    const size_t sm = potts_ring_bytes(WARPS, a.ring_chunks);
    switch (layout) {
        case 0:
            potts_strip_kernel<WARPS, QB, 0><<<grid, WARPS * 32, sm, s>>>(a);
            break;
        case kSrcSplit:
            potts_strip_kernel<WARPS, QB, kSrcSplit><<<grid, WARPS * 32, sm, s>>>(a);
            break;
        case kDstSplit:
            potts_strip_kernel<WARPS, QB, kDstSplit><<<grid, WARPS * 32, sm, s>>>(a);
            break;
        case kSrcSplit | kDstSplit:
            potts_strip_kernel<WARPS, QB, kSrcSplit | kDstSplit><<<grid, WARPS * 32, sm, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_potts_strip(const PottsStripArgs &a, int grid, int warps, int qbits, int layout, cudaStream_t s) {
    if (a.ring_chunks != 32 && a.ring_chunks != 64 && a.ring_chunks != kRowChunks) return cudaErrorInvalidValue;
    if (qbits == 2 && warps == 4) return launch_potts_strip_layout<4, 2>(a, grid, layout, s);
    if (qbits == 2 && warps == 8) return launch_potts_strip_layout<8, 2>(a, grid, layout, s);
    if (qbits == 3 && warps == 4) return launch_potts_strip_layout<4, 3>(a, grid, layout, s);
    if (qbits == 3 && warps == 8) return launch_potts_strip_layout<8, 3>(a, grid, layout, s);
    return cudaErrorInvalidValue;
}

SPIN_CHECK_ACCESSOR(check_word_potts)

}  // namespace spinmc
