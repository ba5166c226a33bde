// strip.cuh -- pieces shared by the Ising and Potts strip kernels: the ring
// geometry, cp.async helpers and the site-independent head of Philox4x32-10.
//
// A strip kernel gives one warp full rows [r0, r0 + R) of one lattice with
// L = 512, 1024 or 2048 (whole 16-byte chunks per lane) and walks down them
// with rows s-2 .. s+2 in a five-slot shared-memory ring per warp.
#pragma once
#include "internal.h"

namespace spinmc {

constexpr int kRing = 5;          // row slots per warp
constexpr int kRowChunks = 128;   // 16-byte chunks per slot (L <= 2048)

// Rounds 1 and 2 of Philox4x32-10 for counter (g, lat, t, c) have one
// product each that does not depend on g; they are formed once per item.
struct PhiloxPrefix {
    uint32_t u0, u1k, v0k, v1, ck1;
};

__device__ __forceinline__ PhiloxPrefix philox_prefix(uint32_t lat, uint32_t t, uint32_t c,
                                                      const PhiloxKeys &rk) {
    PhiloxPrefix P;
    const uint64_t pb = (uint64_t)0xCD9E8D57u * t;
    P.u0 = (uint32_t)(pb >> 32) ^ lat ^ rk.k0[0];
    const uint32_t u1 = (uint32_t)pb;
    const uint64_t pa = (uint64_t)0xD2511F53u * P.u0;
    P.u1k = u1 ^ rk.k0[1];
    P.v0k = (uint32_t)(pa >> 32) ^ rk.k1[1];
    P.v1 = (uint32_t)pa;
    P.ck1 = c ^ rk.k1[0];
    return P;
}

__device__ __forceinline__ uint4 philox_from_prefix(uint32_t g, const PhiloxPrefix &P,
                                                    const PhiloxKeys &rk) {
    const uint64_t pa = (uint64_t)0xD2511F53u * g;            // round 1
    const uint32_t x2 = (uint32_t)(pa >> 32) ^ P.ck1;
    const uint64_t pb = (uint64_t)0xCD9E8D57u * x2;            // round 2
    uint32_t c0 = (uint32_t)(pb >> 32) ^ P.u1k, c1 = (uint32_t)pb;
    uint32_t c2 = (uint32_t)pa ^ P.v0k, c3 = P.v1;
#pragma unroll
    for (int r = 2; r < 10; ++r) {                              // rounds 3..10
        const uint64_t qa = (uint64_t)0xD2511F53u * c0;
        const uint64_t qb = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(qb >> 32) ^ c1 ^ rk.k0[r];
        const uint32_t n2 = (uint32_t)(qa >> 32) ^ c3 ^ rk.k1[r];
        c1 = (uint32_t)qb;
        c3 = (uint32_t)qa;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int wrap_row(int y, int L) { return y < 0 ? y + L : (y >= L ? y - L : y); }

// ---- the split form (Ising and Potts strip kernels): a ring row is stored
// as its two colour-compressed halves, sites of even x then sites of odd x.

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// NW consecutive 32-bit words of a half row (one lane's chunk).
template <int NW>
struct Words {
    uint32_t w[NW];
};

// Chunk c of a half row at a generic address (a destination row in global memory).
template <int NW>
__device__ __forceinline__ void st_words(unsigned char *half, int c, const Words<NW> &r) {
    if constexpr (NW == 4)
        reinterpret_cast<uint4 *>(half)[c] = make_uint4(r.w[0], r.w[1], r.w[2], r.w[3]);
    else
        reinterpret_cast<uint2 *>(half)[c] = make_uint2(r.w[0], r.w[1]);
}

// Ring accesses by 32-bit shared-memory address (volatile: never merged or
// moved across the warp's ring hand-offs), and cp.async of row y into the
// ring at shared address dst.
__device__ __forceinline__ uint32_t sld1(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
template <int NW>
__device__ __forceinline__ Words<NW> ldw(uint32_t half, int c) {
    Words<NW> r;
    if constexpr (NW == 4)
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.w[0]), "=r"(r.w[1]), "=r"(r.w[2]), "=r"(r.w[3]) : "r"(half + 16u * (uint32_t)c));
    else
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.w[0]), "=r"(r.w[1]) : "r"(half + 8u * (uint32_t)c));
    return r;
}
template <int NW>
__device__ __forceinline__ void stw(uint32_t half, int c, const Words<NW> &r) {
    if constexpr (NW == 4)
        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(half + 16u * (uint32_t)c), "r"(r.w[0]),
                     "r"(r.w[1]), "r"(r.w[2]), "r"(r.w[3]));
    else
        asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(half + 8u * (uint32_t)c), "r"(r.w[0]), "r"(r.w[1]));
}
__device__ __forceinline__ void issue_raw_s(uint32_t dst, const uint4 *S, int y, int L, int lane) {
    const uint4 *src = S + (size_t)y * (L >> 4);
    for (int j = lane; j < (L >> 4); j += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * (uint32_t)j), "l"(src + j)
                     : "memory");
}

// One 8-byte table entry at a shared-memory address.
__device__ __forceinline__ uint2 lds_u2(uint32_t addr) {
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

inline size_t strip_ring_bytes(int warps) { return sizeof(uint4) * (size_t)warps * kRing * kRowChunks; }

}  // namespace spinmc
