// sweep_cpm.cu -- cellular Potts copy attempts (Sec. "Cellular Potts model"
// of Farias et al., arXiv 2304.01772; Hamiltonian Eq. "h": adhesion between
// different cells over the Moore neighbourhood plus lambda (a - A)^2).
//
// Sites are coloured c = (x & 1) | ((y & 1) << 1): no two sites of one colour
// are Moore neighbours, so all sites of a colour attempt their copy at once.
// One thread handles the two sites of one Philox group (x = 4m + (c&1) and
// x + 2 in row y).  Area terms read the areas as they stood at the start of
// the sub-step.  Two area arrays and two change arrays alternate so that no
// copy is needed between sub-steps: sub-step k reads V[k%2] (the areas after
// k-1) and adds its accepted copies atomically to V[(k+1)%2] and to D[k%2];
// V[(k+1)%2] held the areas after k-2, so the sub-step also folds in
// D[(k+1)%2] (the changes of k-1) and clears it.  After sub-step k,
// V[(k+1)%2] is the areas after k.  The finalize kernel runs once per Monte
// Carlo step (statistics and the record).
// Acceptance: integer dE, thr[dE] = max(floor(exp(-dE/T) 2^32), 1) - 1 built
// on the host; dE beyond the table accepts only u = 0 (probability 2^-32).
#include <algorithm>

#include "internal.h"

namespace spinmc {

namespace {

__constant__ int8_t kMooreDx[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
__constant__ int8_t kMooreDy[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

__device__ __forceinline__ int pair_index(int a, int b, int n) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * n - lo * (lo - 1) / 2 + (hi - lo);
}

// Most copy attempts pick a neighbour of the same cell and change nothing.
// A block therefore works in passes over kCpmGroupsPerThread Philox groups per
// thread: phase 1 draws the randoms, reads the site and the chosen neighbour
// and queues the attempts whose ids differ in shared memory; phase 2 spreads
// the queued attempts over all threads for the full energy change.  Attempts
// of one colour are independent (none is a Moore neighbour of another, and
// areas come from the snapshot), and the area and contact updates are integer
// additions, so the result does not depend on the order.
constexpr int kCpmThreads = 256;
constexpr int kCpmGroupsPerThread = 1;
constexpr int kCpmQueue = 2 * kCpmThreads * kCpmGroupsPerThread;

__device__ __forceinline__ int wrapc(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Shared-memory working set of one block of the sub-step.
struct CpmShared {
    int sJ[64];
    int scnt[36];                 // contact changes of this block, per type pair
    int4 queue[kCpmQueue];        // (y << 16 | x, id of the site, id copied in, u0)
    int qn;
};

// Load J and clear the block's contact counters.
__device__ __forceinline__ void cpm_block_setup(const CpmArgs &a, CpmShared &sh) {
    for (int k = threadIdx.x; k < a.n_types * a.n_types; k += blockDim.x) sh.sJ[k] = a.J[k];
    for (int k = threadIdx.x; k < 36; k += blockDim.x) sh.scnt[k] = 0;
    if (threadIdx.x == 0) sh.qn = 0;
    __syncthreads();
}

// Add the block's contact changes to out[pair] and clear them.
__device__ __forceinline__ void cpm_block_flush(const CpmArgs &a, CpmShared &sh, int64_t *out) {
    __syncthreads();
    const int npair = a.n_types * (a.n_types + 1) / 2;
    for (int k = threadIdx.x; k < npair; k += blockDim.x)
        if (sh.scnt[k]) {
            atomicAdd(reinterpret_cast<unsigned long long *>(out + k), (unsigned long long)(long long)sh.scnt[k]);
            sh.scnt[k] = 0;
        }
    __syncthreads();
}

// One colour sub-step of sweep t over this block's share of the Philox groups.
__device__ void cpm_substep_body(const CpmArgs &a, int c, uint32_t t, CpmShared &sh) {
    int *sJ = sh.sJ, *scnt = sh.scnt;
    int4 *queue = sh.queue;
    int &qn = sh.qn;
    const int nt = a.n_types;
    const int L = a.L, Lq = L >> 2;
    const int cx = c & 1, cy = c >> 1;
    const int n_groups = (L >> 1) * Lq;
    const int per_pass = kCpmThreads * kCpmGroupsPerThread;
    // fold the previous sub-step's area changes into vol_next (atomically: this
    // sub-step's copies land there at the same time) and clear them
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= a.n_cells; k += gridDim.x * blockDim.x) {
        const int d = a.dvol_prev[k];
        if (d) {
            atomicAdd(a.vol_next + k, d);
            a.dvol_prev[k] = 0;
        }
    }
    for (int base = blockIdx.x * per_pass; base < n_groups; base += gridDim.x * per_pass) {
        // phase 1: candidates (all four id loads of a thread in flight at once)
#pragma unroll
        for (int k = 0; k < kCpmGroupsPerThread; ++k) {
            const int g = base + k * kCpmThreads + (int)threadIdx.x;
            const bool live = g < n_groups;
            const int gg = live ? g : 0;
            const int yh = gg / Lq, m = gg - yh * Lq;
            const int y = 2 * yh + cy;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)gg, a.lat, t, (uint32_t)c), a.k0, a.k1);
            const int x0 = 4 * m + cx, x1 = x0 + 2;
            const int n0 = (int)(r.y >> 29), n1 = (int)(r.w >> 29);
            const int yn0 = wrapc(y + kMooreDy[n0], L), yn1 = wrapc(y + kMooreDy[n1], L);
            const int xn0 = wrapc(x0 + kMooreDx[n0], L), xn1 = wrapc(x1 + kMooreDx[n1], L);
            const int sg0 = a.ids[y * L + x0], sg1 = a.ids[y * L + x1];
            const int sp0 = a.ids[yn0 * L + xn0], sp1 = a.ids[yn1 * L + xn1];
            const unsigned nc = (unsigned)a.n_cells;
            if (live && sp0 != sg0 && (unsigned)sg0 <= nc && (unsigned)sp0 <= nc) {
                const int qi = atomicAdd(&qn, 1);
                if (SPIN_CK(qi < kCpmQueue, 131)) queue[qi] = make_int4((y << 16) | x0, sg0, sp0, (int)r.x);
            }
            if (live && sp1 != sg1 && (unsigned)sg1 <= nc && (unsigned)sp1 <= nc) {
                const int qi = atomicAdd(&qn, 1);
                if (SPIN_CK(qi < kCpmQueue, 131)) queue[qi] = make_int4((y << 16) | x1, sg1, sp1, (int)r.z);
            }
        }
        __syncthreads();
        const int n = qn;
        // phase 2: energy change and Metropolis decision of the queued attempts
        for (int e = threadIdx.x; e < n; e += kCpmThreads) {
            const int4 qe = queue[e];
            const int y = qe.x >> 16, x = qe.x & 0xFFFF, sg = qe.y, sp = qe.z;
            const uint32_t u0 = (uint32_t)qe.w;
            const int tg = a.type[sg], tp = a.type[sp];
            const int vp = a.vol_cur[sp], vg = a.vol_cur[sg];
            int nz[8], tzs[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int sz = a.ids[wrapc(y + kMooreDy[k], L) * L + wrapc(x + kMooreDx[k], L)];
                nz[k] = (unsigned)sz > (unsigned)a.n_cells ? 0 : sz;   // out-of-range ids read as medium
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) tzs[k] = a.type[nz[k]];
            long long dH = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (nz[k] != sp) dH += sJ[tp * nt + tzs[k]];
                if (nz[k] != sg) dH -= sJ[tg * nt + tzs[k]];
            }
            if (sp != 0) dH += (long long)a.lambda * (2ll * ((long long)vp - a.target) + 1);
            if (sg != 0) dH += (long long)a.lambda * (-2ll * ((long long)vg - a.target) + 1);
            bool acc;
            if (dH <= 0)
                acc = true;
            else
                acc = u0 <= (dH < a.n_thr ? a.thr[dH] : 0u);
            if (acc) {
                a.ids[y * L + x] = sp;
                atomicAdd(a.vol_next + sp, 1);
                atomicAdd(a.vol_next + sg, -1);
                atomicAdd(a.dvol_cur + sp, 1);
                atomicAdd(a.dvol_cur + sg, -1);
                if (nt <= 4) {
                    // contacts lost (by sg) and gained (by sp) per neighbour type, one byte each
                    uint32_t lost = 0, gained = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const uint32_t one = 1u << (8 * tzs[k]);
                        lost += nz[k] != sg ? one : 0u;
                        gained += nz[k] != sp ? one : 0u;
                    }
                    for (int tz = 0; tz < nt; ++tz) {
                        const int l = (int)((lost >> (8 * tz)) & 0xFFu), gn = (int)((gained >> (8 * tz)) & 0xFFu);
                        if (l) atomicAdd(scnt + pair_index(tg, tz, nt), -l);
                        if (gn) atomicAdd(scnt + pair_index(tp, tz, nt), gn);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (nz[k] != sg) atomicAdd(scnt + pair_index(tg, tzs[k], nt), -1);
                        if (nz[k] != sp) atomicAdd(scnt + pair_index(tp, tzs[k], nt), 1);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) qn = 0;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCpmThreads) cpm_substep_kernel(CpmArgs a, int c) {
    __shared__ CpmShared sh;
    cpm_block_setup(a, sh);
    cpm_substep_body(a, c, a.state->t, sh);
    cpm_block_flush(a, sh, a.delta);
}

// ---------------------------------------------------------------------------
// Persistent form: every Monte Carlo step of a call in one cooperative launch
// (all blocks resident), the four sub-steps separated by grid barriers instead
// of kernel boundaries.  Block 0 finishes step s (V2, V1, contacts, record)
// at the start of step s + 1: sub-step 0 of s + 1 only reads the areas V[0]
// that the finish reads, and its contact changes go to the other of two
// accumulators (acc[(s + 1) & 1]), so the barrier that ends sub-step 0 orders
// the finish before anything it reads is written again.

__device__ __forceinline__ uint64_t cpm_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kCpmWaitNs = 1000000000ull;   // a barrier wait gives up after 1 s

// Grid barrier: bar[0] counts arrivals, bar[1] is the generation.  Thread 0
// of each block reads the generation, arrives, and the arrival that makes the
// count `expected` (gridDim.x in use) resets the count and advances the
// generation; the others wait (bounded) for the advance.  False (for the whole
// block) if a wait ran out or another block has reported one in *err.
__device__ bool cpm_grid_sync(unsigned int *bar, int *err, unsigned int expected) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = bar + 1;
        const unsigned int gen = *vgen;
        int good = 1;
        __threadfence();
        if (atomicAdd(bar, 1u) == expected - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = cpm_ns();
            while (*vgen == gen) {
                if (cpm_ns() - t0 > kCpmWaitNs) {
                    atomicExch(err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*(volatile int *)err) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Statistics after a step (block-wide): V2, V1 from the areas, contacts
// cur += acc (acc cleared), and the record.
__device__ void cpm_finish_step(const int32_t *vol, int n_cells, int target, const StatsBufs &st, int64_t *acc,
                                int record, long long rec) {
    __shared__ long long r2[kCpmThreads / 32], r1[kCpmThreads / 32];
    long long v2 = 0, v1 = 0;
    for (int k = 1 + threadIdx.x; k <= n_cells; k += blockDim.x) {
        const long long d = (long long)vol[k] - target;
        v2 += d * d;
        v1 += d;
    }
    const int npair = st.width - 2;
    for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        st.cur[k] += acc[k];
        acc[k] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o);
        v1 += __shfl_xor_sync(0xFFFFFFFFu, v1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r2[threadIdx.x >> 5] = v2;
        r1[threadIdx.x >> 5] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a2 = 0, a1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a2 += r2[w];
            a1 += r1[w];
        }
        st.cur[npair] = a2;
        st.cur[npair + 1] = a1;
    }
    __syncthreads();
    if (record && st.cap > 0) {
        const long long slot = rec % st.cap;
        for (int k = threadIdx.x; k < st.width; k += blockDim.x) st.ring[slot * st.width + k] = st.cur[k];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCpmThreads) cpm_persistent_kernel(CpmPersistArgs p) {
    __shared__ CpmShared sh;
    CpmArgs a = p.a;
    cpm_block_setup(a, sh);
    for (int step = 0; step < p.n_steps; ++step) {
        const uint32_t t = p.t0 + (uint32_t)step;
        for (int c = 0; c < 4; ++c) {
            if (c == 0 && step > 0 && blockIdx.x == 0)
                cpm_finish_step(p.vol[0], a.n_cells, a.target, p.st, p.acc + kCpmAccStride * ((step - 1) & 1),
                                p.record, p.rec0 + step - 1);
            a.vol_cur = p.vol[c & 1];
            a.vol_next = p.vol[(c + 1) & 1];
            a.dvol_cur = p.dvol[c & 1];
            a.dvol_prev = p.dvol[(c + 1) & 1];
            cpm_substep_body(a, c, t, sh);
            cpm_block_flush(a, sh, p.acc + kCpmAccStride * (step & 1));
            if (!cpm_grid_sync(p.bar, p.err, gridDim.x)) return;
        }
    }
    if (blockIdx.x == 0 && p.n_steps > 0)
        cpm_finish_step(p.vol[0], a.n_cells, a.target, p.st, p.acc + kCpmAccStride * ((p.n_steps - 1) & 1),
                        p.record, p.rec0 + p.n_steps - 1);
}

// Self-test of the grid barrier: `rounds` barriers that complete after
// `expected` arrivals (expected > gridDim.x: they cannot complete, and every
// block must give up after the bounded wait).
__global__ void grid_barrier_probe_kernel(unsigned int *bar, int *err, unsigned int expected, int rounds) {
    for (int r = 0; r < rounds; ++r)
        if (!cpm_grid_sync(bar, err, expected)) return;
}

__global__ void cpm_advance_kernel(DevState *state, uint32_t n, int record) {
    state->t += n;
    if (record) state->n_rec += n;
}

// After the four sub-steps of a Monte Carlo step: contacts cur += delta, V2
// and V1 from the areas after the step, the record, and the step counter.
__global__ void __launch_bounds__(1024) cpm_finalize_kernel(const int32_t *vol, int n_cells, int target,
                                                            DevState *state, StatsBufs st, int record) {
    __shared__ long long r2[32], r1[32];
    long long v2 = 0, v1 = 0;
    for (int k = 1 + threadIdx.x; k <= n_cells; k += blockDim.x) {
        const long long d = (long long)vol[k] - target;
        v2 += d * d;
        v1 += d;
    }
    const int npair = st.width - 2;
    for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        st.cur[k] += st.delta[k];
        st.delta[k] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o);
        v1 += __shfl_xor_sync(0xFFFFFFFFu, v1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r2[threadIdx.x >> 5] = v2;
        r1[threadIdx.x >> 5] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a2 = 0, a1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a2 += r2[w];
            a1 += r1[w];
        }
        st.cur[npair] = a2;
        st.cur[npair + 1] = a1;
    }
    __syncthreads();
    if (record && st.cap > 0) {
        const long long slot = state->n_rec % st.cap;
        for (int k = threadIdx.x; k < st.width; k += blockDim.x)
            st.ring[slot * st.width + k] = st.cur[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        state->t += 1;
        if (record) state->n_rec += 1;
    }
}

__global__ void cpm_init_squares_kernel(int32_t *ids, int L, int n_cells, int side, int cols) {
    const int rows = (n_cells + cols - 1) / cols;
    const int x0 = (L - cols * side) / 2, y0 = (L - rows * side) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L - y0, x = i % L - x0;
        int id = 0;
        if (x >= 0 && y >= 0 && x < cols * side && y < rows * side) {
            const int cidx = (y / side) * cols + (x / side);
            if (cidx < n_cells) id = cidx + 1;
        }
        ids[i] = id;
    }
}

__global__ void cpm_volumes_kernel(const int32_t *ids, int L, int32_t *vol, int n_cells) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int id = ids[i];
        if ((unsigned)id <= (unsigned)n_cells) atomicAdd(vol + id, 1);
    }
}

__global__ void cpm_types_kernel(uint8_t *type, int n_cells, uint32_t lat, uint32_t k0, uint32_t k1) {
    for (int cidx = blockIdx.x * blockDim.x + threadIdx.x; cidx <= n_cells; cidx += gridDim.x * blockDim.x) {
        if (cidx == 0) {
            type[0] = 0;
            continue;
        }
        const uint4 r = philox4x32_10(make_uint4((uint32_t)cidx, lat, 0xFFFFFFFEu, 0u), k0, k1);
        type[cidx] = (uint8_t)(1u + (r.x >> 31));
    }
}

// ------------------------------------------------------------ batched CPM
// One block per lattice (grid-stride over the batch); ids, the two area
// arrays (snapshot and running), cell types, J and the acceptance table live
// in shared memory for all steps of the call.  Sub-step semantics are those of
// cpm_substep_kernel (snapshot areas, same Philox counters with the batch index
// as the lattice word), so each lattice follows its single-lattice chain.
constexpr int kCpmBatchThreads = 256;
constexpr int kCpmBatchSmemThr = 4096;   // larger tables stay in global memory

// Periodic index: a mask when L is a power of two, else a compare.
template <bool POW2>
__device__ __forceinline__ int wrapb(int v, int L) {
    return POW2 ? (v & (L - 1)) : (v < 0 ? v + L : (v >= L ? v - L : v));
}

template <bool POW2>
__global__ void __launch_bounds__(kCpmBatchThreads) cpm_batch_kernel(CpmBatchArgs a) {
    extern __shared__ __align__(16) int32_t csm[];
    __shared__ int4 queue[2 * kCpmBatchThreads];   // live attempts of one pass: (y << 16 | x, sg, sp, u0)
    __shared__ int qn;
    const int L = a.L, N = L * L, nc1 = a.n_cells + 1, nt = a.n_types;
    int32_t *ids = csm, *snap = csm + N, *next = snap + nc1, *Js = next + nc1;
    int32_t *cnt = Js + 64;                                   // contact counters (<= 36)
    uint32_t *thr_s = reinterpret_cast<uint32_t *>(cnt + 40);
    uint8_t *type = reinterpret_cast<uint8_t *>(thr_s + (a.n_thr <= kCpmBatchSmemThr ? a.n_thr : 0));
    const uint32_t *thr = a.n_thr <= kCpmBatchSmemThr ? thr_s : a.thr;
    const int npair = nt * (nt + 1) / 2;
    const unsigned ncu = (unsigned)a.n_cells;
    for (int k = threadIdx.x; k < nt * nt; k += blockDim.x) Js[k] = a.J[k];
    if (a.n_thr <= kCpmBatchSmemThr)
        for (int k = threadIdx.x; k < a.n_thr; k += blockDim.x) thr_s[k] = a.thr[k];
    if (threadIdx.x == 0) qn = 0;
    const int half = L / 2, ngroups = N / 8;
    for (int lat = blockIdx.x; lat < a.n_lat; lat += gridDim.x) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) ids[i] = a.ids[(size_t)lat * N + i];
        for (int c = threadIdx.x; c < nc1; c += blockDim.x) {
            snap[c] = next[c] = a.areas[(size_t)lat * nc1 + c];
            const uint8_t tp = a.types[(size_t)lat * nc1 + c];
            type[c] = tp < nt ? tp : 0;   // out-of-range types read as medium: J stays in bounds
        }
        __syncthreads();
        for (int step = 0; step < a.n_steps; ++step) {
            const uint32_t t = a.first_step + (uint32_t)step;
            for (int col = 0; col < 4; ++col) {
                const int cx = col & 1, cy = col >> 1;
                // passes of one Philox group per thread: draw and read, queue the live
                // attempts (ids differ), then spread them over the block
                for (int base = 0; base < ngroups; base += blockDim.x) {
                    const int g = base + (int)threadIdx.x;
                    if (g < ngroups) {
                        const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)lat, t, (uint32_t)col),
                                                      a.k0, a.k1);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int k = 2 * g + j, yh = k / half;
                            const int y = 2 * yh + cy, x = 2 * (k - yh * half) + cx;
                            const int nbi = (int)((j ? r.w : r.y) >> 29);
                            const int sg = ids[y * L + x];
                            const int sp = ids[wrapb<POW2>(y + kMooreDy[nbi], L) * L + wrapb<POW2>(x + kMooreDx[nbi], L)];
                            if (sp != sg && (unsigned)sg <= ncu && (unsigned)sp <= ncu) {
                                const int qi = atomicAdd(&qn, 1);
                                if (SPIN_CK(qi < 2 * kCpmBatchThreads, 132))
                                    queue[qi] = make_int4((y << 16) | x, sg, sp, (int)(j ? r.z : r.x));
                            }
                        }
                    }
                    __syncthreads();
                    const int n = qn;
                    __syncthreads();                 // every thread has read the count ...
                    if (threadIdx.x == 0) qn = 0;    // ... before it is reset for the next pass
                    for (int e = threadIdx.x; e < n; e += blockDim.x) {
                        const int4 q4 = queue[e];
                        const int y = q4.x >> 16, x = q4.x & 0xFFFF, sg = q4.y, sp = q4.z;
                        const uint32_t u0 = (uint32_t)q4.w;
                        const int tg = type[sg], tp = type[sp];
                        long long dH = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            int sz = ids[wrapb<POW2>(y + kMooreDy[q], L) * L + wrapb<POW2>(x + kMooreDx[q], L)];
                            sz = (unsigned)sz > ncu ? 0 : sz;
                            const int tz = type[sz];
                            if (sz != sp) dH += Js[tp * nt + tz];
                            if (sz != sg) dH -= Js[tg * nt + tz];
                        }
                        if (sp != 0) dH += (long long)a.lambda * (2ll * ((long long)snap[sp] - a.target) + 1);
                        if (sg != 0) dH += (long long)a.lambda * (-2ll * ((long long)snap[sg] - a.target) + 1);
                        if (dH <= 0 || u0 <= (dH < a.n_thr ? thr[dH] : 0u)) {
                            ids[y * L + x] = sp;
                            atomicAdd(next + sp, 1);
                            atomicAdd(next + sg, -1);
                        }
                    }
                    __syncthreads();
                }
                for (int c = threadIdx.x; c < nc1; c += blockDim.x) snap[c] = next[c];
                __syncthreads();
            }
            if (a.stats) {
                // statistics of the state after the step, recounted on chip
                for (int k = threadIdx.x; k < 40; k += blockDim.x) cnt[k] = 0;
                __syncthreads();
                long long v2 = 0, v1 = 0;
                for (int i = threadIdx.x; i < N; i += blockDim.x) {
                    const int y = i / L, x = i - y * L;
                    const int ia = ids[i];
                    const int ta = type[(unsigned)ia > ncu ? 0 : ia];
                    const int hx[4] = {1, -1, 0, 1}, hy[4] = {0, 1, 1, 1};
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int ib = ids[wrapb<POW2>(y + hy[d], L) * L + wrapb<POW2>(x + hx[d], L)];
                        if (ia == ib) continue;
                        const int tb = type[(unsigned)ib > ncu ? 0 : ib];
                        atomicAdd(cnt + pair_index(ta, tb, nt), 1);
                    }
                }
                for (int c = 1 + threadIdx.x; c < nc1; c += blockDim.x) {
                    const long long d = (long long)snap[c] - a.target;
                    v2 += d * d;
                    v1 += d;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v2 += __shfl_xor_sync(0xFFFFFFFFu, v2, o);
                    v1 += __shfl_xor_sync(0xFFFFFFFFu, v1, o);
                }
                __shared__ long long r2[kCpmBatchThreads / 32], r1[kCpmBatchThreads / 32];
                if ((threadIdx.x & 31) == 0) {
                    r2[threadIdx.x >> 5] = v2;
                    r1[threadIdx.x >> 5] = v1;
                }
                __syncthreads();
                int64_t *out = a.stats + ((size_t)step * a.n_lat + lat) * a.width;
                for (int k = threadIdx.x; k < npair; k += blockDim.x) out[k] = cnt[k];
                if (threadIdx.x == 0) {
                    long long s2 = 0, s1 = 0;
                    for (int w = 0; w < kCpmBatchThreads / 32; ++w) {
                        s2 += r2[w];
                        s1 += r1[w];
                    }
                    out[npair] = s2;
                    out[npair + 1] = s1;
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) a.ids[(size_t)lat * N + i] = ids[i];
        for (int c = threadIdx.x; c < nc1; c += blockDim.x) a.areas[(size_t)lat * nc1 + c] = snap[c];
        __syncthreads();
    }
}

// Batch initial state: every lattice gets the square-cell layout, its own cell
// types (Philox with the batch index, or the caller's types for all) and areas.
__global__ void cpm_batch_init_kernel(int n_lat, int L, int n_cells, int side, int cols, const uint8_t *given,
                                      uint32_t k0, uint32_t k1, int32_t *ids, uint8_t *types, int32_t *areas) {
    const int N = L * L, nc1 = n_cells + 1;
    const int rows = (n_cells + cols - 1) / cols;
    const int x0 = (L - cols * side) / 2, y0 = (L - rows * side) / 2;
    for (int lat = blockIdx.x; lat < n_lat; lat += gridDim.x) {
        for (int c = threadIdx.x; c < nc1; c += blockDim.x) {
            uint8_t tp = 0;
            if (c > 0) {
                if (given) {
                    tp = given[c];
                } else {
                    const uint4 r = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)lat, 0xFFFFFFFEu, 0u), k0, k1);
                    tp = (uint8_t)(1u + (r.x >> 31));
                }
            }
            types[(size_t)lat * nc1 + c] = tp;
            areas[(size_t)lat * nc1 + c] = 0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int y = i / L - y0, x = i % L - x0;
            int id = 0;
            if (x >= 0 && y >= 0 && x < cols * side && y < rows * side) {
                const int cidx = (y / side) * cols + (x / side);
                if (cidx < n_cells) id = cidx + 1;
            }
            ids[(size_t)lat * N + i] = id;
            atomicAdd(areas + (size_t)lat * nc1 + id, 1);
        }
        __syncthreads();
    }
}

}  // namespace

size_t cpm_batch_smem(int L, int n_cells, int n_thr) {
    const size_t nc1 = (size_t)n_cells + 1;
    return sizeof(int32_t) * ((size_t)L * L + 2 * nc1 + 64 + 40) +
           sizeof(uint32_t) * (size_t)(n_thr <= kCpmBatchSmemThr ? n_thr : 0) + ((nc1 + 15) & ~(size_t)15);
}

template <bool POW2>
static cudaError_t launch_cpm_batch_t(const CpmBatchArgs &a, size_t sm, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(cpm_batch_kernel<POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cpm_batch_kernel<POW2>, kCpmBatchThreads, sm);
    if (e) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(a.n_lat, sms * std::max(1, per_sm)));
    cpm_batch_kernel<POW2><<<grid, kCpmBatchThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cpm_batch(const CpmBatchArgs &a, cudaStream_t s) {
    const size_t sm = cpm_batch_smem(a.L, a.n_cells, a.n_thr);
    return (a.L & (a.L - 1)) == 0 ? launch_cpm_batch_t<true>(a, sm, s) : launch_cpm_batch_t<false>(a, sm, s);
}

cudaError_t launch_cpm_batch_init(int n_lat, int L, int n_cells, int side, int cols, const uint8_t *given,
                                  uint32_t k0, uint32_t k1, int32_t *ids, uint8_t *types, int32_t *areas,
                                  cudaStream_t s) {
    const int grid = n_lat < 152 * 8 ? n_lat : 152 * 8;
    cpm_batch_init_kernel<<<grid, 256, 0, s>>>(n_lat, L, n_cells, side, cols, given, k0, k1, ids, types, areas);
    return cudaGetLastError();
}

cudaError_t launch_cpm_substep(const CpmArgs &a, int colour, cudaStream_t s) {
    const int n_groups = (a.L >> 1) * (a.L >> 2);
    const int per_pass = kCpmThreads * kCpmGroupsPerThread;
    int blocks = (n_groups + per_pass - 1) / per_pass;
    if (blocks > 152 * 8) blocks = 152 * 8;
    cpm_substep_kernel<<<blocks, kCpmThreads, 0, s>>>(a, colour);
    return cudaGetLastError();
}

int cpm_persistent_grid() {
    int occ = 0, sms = 0, dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cpm_persistent_kernel, kCpmThreads, 0))
        return 0;
    return occ * sms;
}

cudaError_t launch_cpm_persistent(const CpmPersistArgs &p, int max_grid, DevState *state, cudaStream_t s) {
    const int n_groups = (p.a.L >> 1) * (p.a.L >> 2);
    const int per_pass = kCpmThreads * kCpmGroupsPerThread;
    const int grid = std::max(1, std::min(max_grid, (n_groups + per_pass - 1) / per_pass));
    cudaError_t e = cudaMemsetAsync(p.bar, 0, 2 * sizeof(unsigned int), s);
    if (e) return e;
    CpmPersistArgs q = p;
    void *args[] = {&q};
    e = cudaLaunchCooperativeKernel((const void *)cpm_persistent_kernel, dim3(grid), dim3(kCpmThreads), args, 0, s);
    if (e) return e;
    cpm_advance_kernel<<<1, 1, 0, s>>>(state, (uint32_t)p.n_steps, p.record);
    return cudaGetLastError();
}

cudaError_t launch_grid_barrier_probe(unsigned int *bar, int *err, int blocks, int missing, int rounds,
                                      cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s);
    if (e) return e;
    unsigned int expected = (unsigned int)(blocks + missing);
    void *args[] = {&bar, &err, &expected, &rounds};
    return cudaLaunchCooperativeKernel((const void *)grid_barrier_probe_kernel, dim3(blocks), dim3(kCpmThreads),
                                       args, 0, s);
}

cudaError_t launch_cpm_finalize(const int32_t *vol, int n_cells, int target, DevState *state, StatsBufs st,
                                int record, cudaStream_t s) {
    cpm_finalize_kernel<<<1, 1024, 0, s>>>(vol, n_cells, target, state, st, record);
    return cudaGetLastError();
}

cudaError_t launch_cpm_init_squares(int32_t *ids, int L, int n_cells, int side, int cols,
                                    cudaStream_t s) {
    cpm_init_squares_kernel<<<256, 256, 0, s>>>(ids, L, n_cells, side, cols);
    return cudaGetLastError();
}

cudaError_t launch_cpm_volumes(const int32_t *ids, int L, int32_t *vol, int n_cells, cudaStream_t s) {
    cpm_volumes_kernel<<<256, 256, 0, s>>>(ids, L, vol, n_cells);
    return cudaGetLastError();
}

cudaError_t launch_cpm_types(uint8_t *type, int n_cells, uint32_t lat, uint32_t k0, uint32_t k1,
                             cudaStream_t s) {
    cpm_types_kernel<<<(n_cells + 256) / 256, 256, 0, s>>>(type, n_cells, lat, k0, k1);
    return cudaGetLastError();
}

SPIN_CHECK_ACCESSOR(check_word_cpm)

}  // namespace spinmc
