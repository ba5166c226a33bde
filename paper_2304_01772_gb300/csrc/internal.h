// internal.h -- device data layouts and kernel launch wrappers shared by the
// CUDA translation units and the host side of libspinmc.so.  Not installed.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace spinmc {

// One lattice as the kernels see it.
struct LatDev {
    uint64_t offset;  // element offset in the spin buffers
    int32_t L;
    int32_t q;        // Potts states (2 for Ising)
    int32_t fast;     // 1: L % 16 == 0 and offset % 16 == 0 -> vectorised kernels
    int32_t geom;     // 0: square lattice, 1: triangular, 2: first and second neighbours (Ising)
    uint32_t rng;     // lattice word of the lattice's Philox counters
    uint32_t pad;
};

// One work item of the batched sweep: rows [r0, r0 + nrows) of lattice `lat`.
// whole = 1: the item is the entire lattice (no halo, periodic in shared memory).
struct Item {
    int32_t lat;
    int32_t r0;
    int32_t nrows;
    int32_t whole;
};

// Acceptance table entry: accept a draw u iff u <= thr; `delta` is the packed
// change of the statistics on acceptance (Ising: dB * 65536 + dM; Potts: dB_eq).
struct __align__(8) TabEntry {
    uint32_t thr;
    int32_t delta;
};
constexpr int kTabStride = 16;     // entries per lattice (Ising uses 10, Potts 9)
// First-and-second-neighbour Ising: thresholds per lattice indexed
// cdown * 25 + d1 * 5 + d2 (d1, d2 = down spins among the four nearest and
// the four diagonal neighbours).
constexpr int kNnnTab = 50;
// Per-lattice doubles of the observables and estimator kernels:
// J, h, N, beta (Ising) or q (Potts), J2.
constexpr int kLatParams = 5;

// Device-side counters advanced by the finalize kernels (so that captured
// graphs need no per-sweep parameters).
struct DevState {
    uint32_t t;        // sweep index of the next sweep
    int32_t substep;   // CPM colour within the current step
    int64_t n_rec;     // records written so far
};

// Counters of one sweep.  Ising: delta[l][0..1] = (dM, dB); Potts:
// delta[l][0..q] = (dB_eq, dn_0..); CPM: delta[0][pair] = contact changes.
struct StatsBufs {
    int64_t *cur;      // [n_lat][width] statistics of the current state
    int64_t *delta;    // [n_lat][width] accumulated changes of the running sweep
    int64_t *ring;     // [cap][n_lat][width] records
    int32_t cap;       // ring capacity (sweeps)
    int32_t width;
    int32_t n_lat;
    int32_t pad;
};

#ifdef __CUDACC__
// ------------------------------------------------------------------ SPIN_CHECK
// Builds with -DSPIN_CHECK (libspinmc_check.so) check work-list entries,
// shared-memory indices and table addresses before they are used.  A failed
// check records its code in this translation unit's check word (the first
// failure wins); the caller skips the access and the kernel carries on, so
// nothing traps.  spin_check_status reads and clears the words.  Other builds
// compile every check to `true`.
#ifdef SPIN_CHECK
static __device__ unsigned int g_check_word = 0u;
__device__ __forceinline__ bool spin_ck(bool ok, unsigned code) {
    if (!ok) atomicCAS(&g_check_word, 0u, code);
    return ok;
}
#define SPIN_CK(cond, code) spin_ck((cond), (code))
#define SPIN_CHECK_ACCESSOR(fn)                                                              \
    cudaError_t fn(unsigned *word, bool clear) {                                             \
        cudaError_t e = cudaMemcpyFromSymbol(word, g_check_word, sizeof(unsigned));          \
        const unsigned zero = 0u;                                                            \
        if (!e && clear) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(unsigned));      \
        return e;                                                                            \
    }
#else
#define SPIN_CK(cond, code) true
#define SPIN_CHECK_ACCESSOR(fn)                \
    cudaError_t fn(unsigned *word, bool) {     \
        *word = 0u;                            \
        return cudaSuccess;                    \
    }
#endif
// Dynamic shared memory of the running launch, in bytes.
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11.  Multipliers 0xD2511F53 / 0xCD9E8D57,
// Weyl key increments 0x9E3779B9 / 0xBB67AE85, ten rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    }
    return c;
}
#endif  // __CUDACC__

// Philox round keys (key + r * Weyl constant, r = 0..9), passed in the kernel
// parameters so that every round reads its key from the constant bank.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys r;
    for (int i = 0; i < 10; ++i) {
        r.k0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
        r.k1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
    }
    return r;
}

// -------------------------------------------------------------- launch wrappers
// All return cudaGetLastError() after the launch.
struct IsingSweepArgs {
    const Item *items;
    int n_items;
    const LatDev *lats;
    const TabEntry *tabs;
    const int8_t *src;
    int8_t *dst;
    uint32_t k0, k1;
    const DevState *state;
    int64_t *delta;   // [n_lat][2]
    PhiloxKeys rk;
    int n_lat;        // entries of lats (work-list checks of SPIN_CHECK builds)
    // strip kernel, layouts with kSrcBits / kDstBits: one bit per spin (1 = -1),
    // element e at bit e % 32 of word e / 32 (the bit-packed host format)
    const uint32_t *src_bits;
    uint32_t *dst_bits;
};

cudaError_t launch_ising_fused(const IsingSweepArgs &a, int grid, int threads, size_t smem,
                               cudaStream_t s);
// Row formats of the strip kernels' global rows (`layout` bits).  0: the
// interface's rows (Ising int8 +1 = 0x01, -1 = 0xFF; Potts uint8 states);
// kSrcSplit: the source rows are in the kernel's split form (the even-x half
// of a row, then the odd-x half; Ising one byte 8 [s < 0] per site, Potts the
// state bytes); kDstSplit: the destination rows are written in it.
constexpr int kSrcSplit = 1, kDstSplit = 2;
// Strip kernel only: kSrcBits: the strip lattices' source rows are read from
// src_bits (one bit per spin; lattice offsets multiples of 128) instead of
// src; kDstBits: each finished row is also written to dst_bits, beside its
// int8 row in dst.  Used together, for a sweep between two bit-packed
// transfers (spin_sweep_packed).
constexpr int kSrcBits = 4, kDstBits = 8;
// Warp-per-row-strip kernel for L in {512, 1024, 2048}; items are row blocks.
cudaError_t launch_ising_strip(const IsingSweepArgs &a, int grid, int warps, int layout, cudaStream_t s);
cudaError_t launch_ising_plain(int8_t *spins, const LatDev *lat_dev, int lat, uint32_t rng, int L,
                               const TabEntry *tabs, uint32_t k0, uint32_t k1,
                               const DevState *state, int64_t *delta, int colour, cudaStream_t s);
// Lattices whose side is not a multiple of 16: two passes, src -> dst (colour 0,
// other sites copied) and dst in place (colour 1).  lat_ids: device list.
// Triangular-lattice Ising (geometry 1), one colour of three over the listed
// lattices: colour 0 reads src and writes dst (copying the other sites),
// colours 1 and 2 work in place on dst.
cudaError_t launch_ising_tri(const int8_t *src, int8_t *dst, const int32_t *lat_ids, int n, int maxL,
                             const LatDev *lats, const TabEntry *tabs, uint32_t k0, uint32_t k1,
                             const DevState *state, int64_t *delta, int colour, cudaStream_t s);
cudaError_t launch_ising_generic(const int8_t *src, int8_t *dst, const int32_t *lat_ids, int n,
                                 int maxL, const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                 uint32_t k1, const DevState *state, int64_t *delta, int colour,
                                 cudaStream_t s);
// Resident form: one CTA per lattice (all lattices vectorisable, L*L <= 64 KB),
// n_sweeps sweeps in one launch, in place; then the device counters advance.
struct ResidentArgs {
    int8_t *spins;
    const LatDev *lats;
    const TabEntry *tabs;
    uint32_t k0, k1;
    uint32_t t0;
    int n_sweeps;
    long long rec0;
    int record;
    StatsBufs st;
    PhiloxKeys rk;   // round keys of (k0, k1)
};
cudaError_t launch_ising_resident(const ResidentArgs &a, int n_lat, int threads, size_t smem,
                                  DevState *state, cudaStream_t s);
// The same for batches made only of triangular lattices (L <= 240).
cudaError_t launch_ising_tri_resident(const ResidentArgs &a, int n_lat, size_t smem, DevState *state,
                                      cudaStream_t s);
// Ising with first and second neighbours (geometry 2; a context holds only
// such lattices, statistics (M, B, B2)), one colour of four over all lattices:
// colour 0 reads src and writes dst (each thread also copies the three other
// sites of its 2x2 block), colours 1..3 work in place on dst.  thr: [n][kNnnTab].
cudaError_t launch_ising_nnn(const int8_t *src, int8_t *dst, int n, int maxL, const LatDev *lats,
                             const uint32_t *thr, uint32_t k0, uint32_t k1, const DevState *state,
                             int64_t *delta, int colour, cudaStream_t s);
// Resident form of the same (L <= 256; a.tabs unused).
cudaError_t launch_ising_nnn_resident(const ResidentArgs &a, const uint32_t *thr, int n_lat, size_t smem,
                                      DevState *state, cudaStream_t s);
cudaError_t launch_init_random(void *spins, int model, const LatDev *lats, int n_lat, int maxL,
                               uint32_t k0, uint32_t k1, cudaStream_t s);
// XOR of every word of the Philox blocks for counters (g, lat, t, c),
// g in [g0, g0 + n), into *out (zeroed first).
cudaError_t launch_philox_xor(uint32_t g0, uint32_t n, uint32_t lat, uint32_t t, uint32_t c,
                              uint32_t k0, uint32_t k1, uint32_t *out, cudaStream_t s);
// Check words of the translation units with SPIN_CHECK sites (always 0 in
// other builds); clear = reset after reading.
cudaError_t check_word_ising(unsigned *word, bool clear);
cudaError_t check_word_potts(unsigned *word, bool clear);
cudaError_t check_word_cpm(unsigned *word, bool clear);
cudaError_t check_word_stats(unsigned *word, bool clear);

struct PottsSweepArgs {
    const Item *items;
    int n_items;
    const LatDev *lats;
    const TabEntry *tabs;
    const uint8_t *src;
    uint8_t *dst;
    uint32_t k0, k1;
    const DevState *state;
    int64_t *delta;   // [n_lat][width]
    int width;
    int n_lat;        // entries of lats (work-list checks of SPIN_CHECK builds)
};
cudaError_t launch_potts_fused(const PottsSweepArgs &a, int grid, int threads, size_t smem,
                               cudaStream_t s);
// Warp-per-row-strip kernel for q <= 8 and L in {512, 1024, 2048}.  `delta`
// receives the change of every statistic; the state counts are counted on the
// new rows, and the item holding row 0 subtracts `cur` (the old counts).
struct PottsStripArgs {
    const Item *items;
    int n_items;
    const LatDev *lats;
    const TabEntry *tabs;
    const uint8_t *src;
    uint8_t *dst;
    const DevState *state;
    int64_t *delta;       // [n_lat][width]
    const int64_t *cur;   // [n_lat][width]
    int width;
    int ring_chunks;      // 16-byte chunks per ring slot: L / 16 of the widest strip lattice
    PhiloxKeys rk;
    int n_lat;            // entries of lats (work-list checks of SPIN_CHECK builds)
};
// qbits: 2 for q <= 4, 3 for q <= 8.
cudaError_t launch_potts_strip(const PottsStripArgs &a, int grid, int warps, int qbits, int layout, cudaStream_t s);
cudaError_t occupancy_potts_strip(int *blocks_per_sm, int warps, int qbits, int ring_chunks);
cudaError_t launch_potts_plain(uint8_t *spins, const LatDev *lat_dev, int lat, uint32_t rng, int L, int q,
                               const TabEntry *tabs, uint32_t k0, uint32_t k1,
                               const DevState *state, int64_t *delta, int width, int colour,
                               cudaStream_t s);
cudaError_t launch_potts_generic(const uint8_t *src, uint8_t *dst, const int32_t *lat_ids, int n,
                                 int maxL, const LatDev *lats, const TabEntry *tabs, uint32_t k0,
                                 uint32_t k1, const DevState *state, int64_t *delta, int width,
                                 int colour, cudaStream_t s);

struct CpmArgs {
    int32_t *ids;
    int L;
    uint32_t lat;
    const uint8_t *type;     // [n_cells + 1]
    const int32_t *J;        // [n_types][n_types]
    int n_types;
    int n_cells;             // ids outside [0, n_cells] are left alone
    int lambda, target;
    const int32_t *vol_cur;  // snapshot areas: the areas after the previous sub-step
    int32_t *vol_next;       // becomes the areas after this sub-step (see sweep_cpm.cu)
    int32_t *dvol_cur;       // this sub-step's area changes (zero on entry)
    int32_t *dvol_prev;      // the previous sub-step's area changes, folded into vol_next and cleared
    const uint32_t *thr;     // thr[dE] for dE in [0, n_thr); beyond: 0
    int n_thr;
    uint32_t k0, k1;
    const DevState *state;
    int64_t *delta;          // [pairs] contact changes
};
cudaError_t launch_cpm_substep(const CpmArgs &a, int colour, cudaStream_t s);
// Persistent form: n_steps Monte Carlo steps in one cooperative launch (grid
// barriers between sub-steps), then the device counters advance.  a.vol_*,
// a.dvol_* and a.state are unused; contact changes go to acc[step & 1]
// ([2][kCpmAccStride] int64, zero on entry and on return); bar: two words,
// cleared by the launcher; err: set to 1 if a barrier wait ran out.
constexpr int kCpmAccStride = 64;
struct CpmPersistArgs {
    CpmArgs a;
    int32_t *vol[2];
    int32_t *dvol[2];
    int n_steps;
    uint32_t t0;
    long long rec0;
    int record;
    StatsBufs st;
    int64_t *acc;
    unsigned int *bar;
    int *err;
};
// Blocks that a cooperative launch of the persistent kernel may use (0: the
// device has no cooperative launch).
int cpm_persistent_grid();
cudaError_t launch_cpm_persistent(const CpmPersistArgs &p, int max_grid, DevState *state, cudaStream_t s);
// Cooperative launch of `blocks` blocks running `rounds` grid barriers of the
// persistent form that wait for blocks + missing arrivals (err: set to 1 when
// a wait gives up).
cudaError_t launch_grid_barrier_probe(unsigned int *bar, int *err, int blocks, int missing, int rounds,
                                      cudaStream_t s);

// Differentiable Monte Carlo (Alg. 2): relaxed sweeps with one coupling per
// bond.  spins [n_lat][L*L]; J [n_lat][2][L*L] (right, down bonds); tape
// [n_lat][2 n_sweeps][L*L/2] (old values of each sub-step's active sites).
struct DmcArgs {
    int n_lat, L, n_sweeps;
    uint32_t first_sweep;
    float beta, h, alpha;
    uint32_t k0, k1;
    float *spins;           // forward: in/out; backward: the state after the last sub-step
    const float *J;
    float *tape;            // forward: out; backward: in
    float *grad_spins;      // backward: in dL/ds after, out dL/ds before
    float *grad_J;          // backward: out
};
size_t dmc_forward_smem(int L);
size_t dmc_backward_smem(int L);
cudaError_t launch_dmc_forward(const DmcArgs &a, cudaStream_t s);
cudaError_t launch_dmc_backward(const DmcArgs &a, cudaStream_t s);
cudaError_t launch_dmc_loss(int n_lat, int N, const float *spins, const float *target, float *grad,
                            double *loss, cudaStream_t s);
cudaError_t launch_dmc_discretize(int64_t n, float *spins, cudaStream_t s);
cudaError_t launch_dmc_energy(int n_lat, int L, const float *J, const float *spins, float h, float *grad,
                              double *energy, cudaStream_t s);
cudaError_t launch_dmc_spin_step(int64_t n, float *spins, const float *grad, float eta, cudaStream_t s);
// After the four colour sub-steps of a CPM Monte Carlo step: contacts
// cur += delta, V2 / V1 from the areas after the step, record, t += 1.
cudaError_t launch_cpm_finalize(const int32_t *vol, int n_cells, int target, DevState *state, StatsBufs st,
                                int record, cudaStream_t s);
cudaError_t launch_cpm_init_squares(int32_t *ids, int L, int n_cells, int side, int cols,
                                    cudaStream_t s);
cudaError_t launch_cpm_volumes(const int32_t *ids, int L, int32_t *vol, int n_cells,
                               cudaStream_t s);

// Statistics of the current state of every lattice -> out[n_lat][width].
cudaError_t launch_stats_from_state(const void *spins, int model, const LatDev *lats, int n_lat,
                                    int maxL, int width, const uint8_t *cpm_type, int cpm_ntypes,
                                    const int32_t *cpm_vol, int cpm_ncells, int cpm_target,
                                    int64_t *out, cudaStream_t s);
// cur += delta, delta = 0, record (if record) into ring slot n_rec % cap, t += 1.
cudaError_t launch_finalize(DevState *state, StatsBufs st, int record, cudaStream_t s);
// Moments of records [first, first + n) -> out[n_lat][n_mom].
cudaError_t launch_moments(const StatsBufs &st, int64_t first, int n, int64_t *out,
                           cudaStream_t s);
// E and M per site from records [first, first + n).
struct ObsParams {
    int model;
    int n_lat;
    int width;
    const double *lat_params;  // [n_lat][kLatParams]
    const double *cpm_J;       // [pairs]
    double cpm_lambda;
};
cudaError_t launch_observables(const StatsBufs &st, int64_t first, int n, ObsParams p,
                               int64_t *stats_out, float *E, float *M, cudaStream_t s);
// Fluctuation-estimator finaliser from moments (FP64 on the device).
struct GradParams {
    int model;
    int n_lat;
    int width;
    int observable;
    int pool;
    const double *lat_params;  // [n_lat][kLatParams]
    const double *cpm_J;       // [pairs]
    double cpm_lambda, cpm_T;
    int n_pairs;
};
cudaError_t launch_grad(const int64_t *moments, GradParams p, double *out, cudaStream_t s);

// MLP
int mlp_param_count();
cudaError_t launch_mlp_forward(const float *params, const float *mu, const float *inv_sigma,
                               const float *X, int n, float *Y, cudaStream_t s);
cudaError_t launch_mlp_backward(const float *params, const float *mu, const float *inv_sigma,
                                const float *X, const float *T, int n, float *grad, float *loss,
                                float *dX, cudaStream_t s);
cudaError_t launch_mlp_adam(float *params, const float *grad, float *m, float *v, int step,
                            float lr, float b1, float b2, float eps, cudaStream_t s);
cudaError_t launch_adam(float *params, const float *grad, float *m, float *v, int n, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s);

#ifdef __CUDACC__
// One Adam step of parameter p (Kingma & Ba) with bias corrections c1 = 1 -
// b1^t, c2 = 1 - b2^t; shared by every kernel that applies Adam so that fused
// and separate launches give identical results.
__device__ __forceinline__ void adam_element(float &p, float &m, float &v, float g, float lr, float b1, float b2,
                                             float eps, float c1, float c2) {
    const float mm = b1 * m + (1.0f - b1) * g;
    const float vv = b2 * v + (1.0f - b2) * g * g;
    m = mm;
    v = vv;
    p -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}
#endif

// Adam bias corrections for step t >= 1.
inline void adam_bias(int step, float b1, float b2, float &c1, float &c2) {
    c1 = 1.0f - powf(b1, (float)step);
    c2 = 1.0f - powf(b2, (float)step);
}

// Fused differentiable Monte Carlo iteration: forward sweeps, loss, reverse
// pass, Adam on the couplings, discretisation; tape in shared memory.
struct DmcStepArgs {
    int n_lat, L, n_sweeps;
    uint32_t first_sweep;
    float beta, h, alpha;
    uint32_t k0, k1;
    float *spins;          // in: start state; out: discretised state after the sweeps
    float *J, *m, *v;      // [n_lat][2][L*L]: couplings and Adam moments, updated
    const float *target;   // [n_lat][L*L]
    double *loss;          // [n_lat]: loss of the relaxed state
    float lr, b1, b2, eps, c1, c2;
};
size_t dmc_step_smem(int L, int n_sweeps);
// Fused spin-value iteration of the differentiable Monte Carlo (see dmc.cu).
struct DmcSpinIterArgs {
    int n_lat, L, n_sweeps;
    uint32_t first_sweep;
    float beta, h, alpha, eta;
    uint32_t k0, k1;
    float *spins;          // in: +-1 spins; out: the updated, discretised spins
    const float *J;        // [n_lat][2][L*L]
    double *energy;        // [n_lat]: energy of the discretised relaxed state
};
size_t dmc_spin_iter_smem(int L, int n_sweeps);
cudaError_t launch_dmc_spin_iter(const DmcSpinIterArgs &a, cudaStream_t s);

// Batched cellular Potts: many independent lattices of one side L, each held
// by one thread block for all sub-steps of the call.
struct CpmBatchArgs {
    int n_lat, L, n_types, n_cells, lambda, target, n_thr, width;
    uint32_t first_step;
    int n_steps;
    uint32_t k0, k1;
    int32_t *ids;            // [n_lat][L*L]
    const uint8_t *types;    // [n_lat][n_cells + 1]
    int32_t *areas;          // [n_lat][n_cells + 1]
    const int32_t *J;        // [n_types][n_types]
    const uint32_t *thr;     // [n_thr]
    int64_t *stats;          // [n_steps][n_lat][width] or null
};
size_t cpm_batch_smem(int L, int n_cells, int n_thr);
cudaError_t launch_cpm_batch(const CpmBatchArgs &a, cudaStream_t s);
cudaError_t launch_cpm_batch_init(int n_lat, int L, int n_cells, int side, int cols, const uint8_t *host_types_dev,
                                  uint32_t k0, uint32_t k1, int32_t *ids, uint8_t *types, int32_t *areas,
                                  cudaStream_t s);
cudaError_t launch_dmc_step(const DmcStepArgs &a, cudaStream_t s);

// One bit per Ising spin on the host side (bit e of words[] = element e is -1):
// unpack the lattices' elements from words (other bytes untouched), counting
// the loaded state's statistics into cur [n_lat][2] = (M, B) of square lattices
// when cur is not null / pack them into
// words (bits outside the lattices 0).  Lattice offsets are multiples of 32.
// blk: per-lattice block ranges of the launch (n_lat + 1 prefix entries,
// n_blocks = blk[n_lat]).  skip_strip: lattices of side 512, 1024 or 2048 are
// left to the strip kernel's bit layouts (unpack: their statistics are still
// counted; pack: their words are not written, nor cleared: the caller keeps
// the buffer's other words, and blk may give them no blocks).
cudaError_t launch_unpack_spins(const uint32_t *words, int8_t *spins, const LatDev *lats, int n_lat,
                                const int32_t *blk, int n_blocks, int64_t *cur, cudaStream_t s,
                                bool skip_strip = false);
cudaError_t launch_pack_spins(const int8_t *spins, uint32_t *words, size_t n_words, const LatDev *lats, int n_lat,
                              const int32_t *blk, int n_blocks, cudaStream_t s, bool skip_strip = false);

// The square-lattice resident form (launch_ising_resident) with each lattice
// split over a thread-block cluster of cs CTAs (2 or 4), CTA r holding rows
// [r L/cs, (r+1) L/cs); max_l: the largest side (a multiple of 16), which
// sizes the shared memory.
cudaError_t launch_ising_resident_cluster(const ResidentArgs &a, int n_lat, int threads, int cs, int max_l,
                                          DevState *state, cudaStream_t s);

}  // namespace spinmc
