/*
 * spinmc.h -- C ABI of libspinmc.so: batched checkerboard Metropolis sweeps of
 * 2D spin lattices (Ising, q-state Potts, cellular Potts) on one GB300 GPU,
 * their observables, the fluctuation-estimator gradient and a small BF16 MLP
 * surrogate.
 *
 * Method: "A differentiable programming framework for spin models" (Farias,
 * Schultz, Mombach, Maziero, arXiv 2304.01772).  Alg. 1 (Metropolis-Hastings
 * with the checkerboard decomposition), the Ising Hamiltonian (Sec. "Ising
 * model"), the Potts Hamiltonian and proposal (Sec. "Potts model"), the
 * cellular Potts Hamiltonian Eq. "h" and copy attempt (Sec. "Cellular Potts
 * model"), and the parameters of Sec. "Results".
 *
 * Conventions (the paper prints H = sum J s s + sum B s with J < 0
 * ferromagnetic; this library uses the equivalent standard signs):
 *   Ising  H = -J sum_<ij> s_i s_j - h sum_i s_i,   s = +-1 stored as int8.
 *   Potts  H = -J sum_<ij> delta(s_i, s_j),          s in [0, q) as uint8.
 *   CPM    H = sum_<xy Moore> J[tau(x)][tau(y)] (1 - delta) + lambda sum (a - A)^2,
 *          cell ids int32 (0 = medium, no area term), each unordered pair once.
 * Bonds are counted once.  Lattices are L x L, row-major, periodic, L even.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32
 * bits, seed high 32 bits), counter = (g, lattice word, sweep index, colour)
 * with the lattice word the lattice's index in its batch unless its
 * descriptor's lattice_id says otherwise,
 * where for a site (x, y) of colour c
 *   Ising: k = (y L + x) >> 1, g = k >> 2, draw = lane k & 3;
 *   Potts: k = (y L + x) >> 1, g = k >> 1, acceptance lane 2(k&1), choice lane 2(k&1)+1,
 *          proposal s' = (s + 1 + floor(u1 (q - 1) / 2^32)) mod q;
 *   CPM:   colour c = (x & 1) | ((y & 1) << 1), k = (y >> 1)(L/2) + (x >> 1),
 *          g = k >> 1, lanes as Potts, neighbour = u1 >> 29 in the order
 *          (-1,-1),(0,-1),(1,-1),(-1,0),(1,0),(-1,1),(0,1),(1,1).
 * Ising/Potts sweep = colour (x + y) & 1 == 0 then 1; CPM step = colours 0..3.
 * Acceptance (Alg. 1): dE <= 0 always, else u < max(floor(exp(-beta dE) 2^32), 1),
 * with dE in double: Ising 2.0*s*((double)J*n + (double)h), Potts
 * (double)J*(n_same_old - n_same_new), CPM integer dE with exp(-dE / (double)T).
 * Because every draw is a function of (seed, lattice, sweep, colour, site)
 * only, results do not depend on tiling, batching, launch form or resume.
 *
 * Ownership: spin buffers are device memory owned by the caller and borrowed
 * by the context until spin_destroy; the context owns everything else it
 * allocates (tables, a second spin buffer, statistics, work lists).  Streams
 * are the caller's (void* = cudaStream_t, NULL = legacy default stream).
 * Calls are asynchronous on the stream unless a host pointer is passed.
 *
 * Errors: every int-returning call returns SPIN_OK (0) or a negative code;
 * spin_last_error(ctx) gives a message.  No exception crosses the ABI.
 */
#ifndef SPINMC_H
#define SPINMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPIN_OK 0
#define SPIN_EINVAL (-1)   /* bad argument: odd L, q out of [2,255], non-finite beta, ... */
#define SPIN_ENOMEM (-2)   /* device or host allocation failed */
#define SPIN_ECUDA (-3)    /* a CUDA runtime call failed */
#define SPIN_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define SPIN_ESTATE (-5)   /* call not valid in the context's current state */

enum { SPIN_ISING = 0, SPIN_POTTS = 1, SPIN_CPM = 2 };

/* One lattice of a batch (host array, copied by spin_init / spin_set_params).
 * Sec. "Methods": the paper batches lattices in the B axis of a [B,C,H,W]
 * tensor; here each lattice has its own size, temperature and couplings.   */
typedef struct {
    int32_t L;            /* side, even, >= 4 (a multiple of 16 takes the vectorised kernels) */
    int32_t q;            /* Potts states in [2, 255]; ignored for Ising and CPM              */
    float beta;           /* inverse temperature 1/T (finite, >= 0); ignored for CPM          */
    float J;              /* coupling (Ising, Potts)                                          */
    float h;              /* field (Ising); must be 0 for Potts                                */
    int32_t geometry;     /* 0: square lattice, 4 neighbours (Sec. "Ising model", kernel K);
                             1: triangular lattice, 6 neighbours (x+-1, y), (x, y+-1), (x+1, y-1),
                             (x-1, y+1) on the square grid, three colours c = (x - y) mod 3 updated
                             in order; Ising only, L % 6 == 0;
                             2: square lattice with first and second neighbours (Sec. "Related
                             Work": the checkerboard serves any order of neighbourhood once a
                             site's colour differs from all its neighbours'), H = -J sum_nn s s
                             - J2 sum_diag s s - h sum s, four colours c = (x & 1) | ((y & 1) << 1)
                             updated in order, draw of site (x, y): k = (y >> 1)(L/2) + (x >> 1),
                             lane k & 3 of Philox group k >> 2; Ising only, and a context holds
                             either only such lattices or none; statistics (M, B, B2)            */
    float J2;             /* second-neighbour (diagonal) coupling, geometry 2; otherwise 0    */
    uint32_t lattice_id;  /* 0: the lattice word of this lattice's Philox counters is its
                             index in this batch; k > 0: it is k - 1.  A lattice draws the
                             same numbers (initial state included) in any batch that gives
                             it the same word, so a batch split over several contexts or
                             GPUs, each lattice given its index in the whole batch plus one,
                             runs exactly the chains of the whole batch in one context.  */
    uint64_t spin_offset; /* element offset of this lattice in the caller's spin buffer       */
} spin_lattice_desc;

/* Cellular Potts parameters (Eq. "h", Sec. "Results": types medium/light/dark,
 * symmetric adhesion table, target area, lambda, temperature k_B T).      */
typedef struct {
    int32_t n_types;          /* including the medium type 0; <= 8                      */
    int32_t lambda;           /* area stiffness (integer energy units)                   */
    int32_t target_area;      /* A, the same for every cell                              */
    int32_t n_cells;          /* cell ids 1..n_cells; id 0 is the medium                 */
    const int32_t *J_type;    /* host, n_types x n_types, symmetric, integer             */
    const uint8_t *cell_type; /* host, [n_cells + 1] types (cell_type[0] = 0), or NULL
                                 to draw 1 + (u >> 31) per cell at spin_init             */
    float T;                  /* temperature (> 0)                                        */
    int32_t init_side;        /* init_mode 2: side of the square cells                   */
    int32_t init_cols;        /* init_mode 2: cells per row of the centred block         */
    int32_t reserved;         /* must be 0                                               */
} spin_cpm_params;

typedef struct spin_ctx spin_ctx;

/* Create a context for n_lattices lattices of one model.
 * d_spins: caller's device buffer (int8 Ising, uint8 Potts, int32 CPM) that
 *   holds every lattice at its spin_offset; borrowed until spin_destroy.
 * init_mode: 0 = random state from the seed (Philox(seed; g = i >> 2, lattice,
 *   0xFFFFFFFF, 0), lane i & 3 for site i = yL + x: Ising s = u>>31 ? +1 : -1,
 *   Potts s = floor(u q / 2^32)); 1 = keep the caller's state; 2 = CPM square
 *   cells (CPM only).  cpm must be non-NULL exactly for CPM (one lattice).
 * max_record_sweeps: capacity of the per-sweep observable ring (0 = none).
 * The sweep counter starts at 0.  Returns SPIN_OK and *out, or an error.  */
int spin_init(spin_ctx **out, int32_t model, uint64_t seed, int32_t n_lattices,
              const spin_lattice_desc *lat, const spin_cpm_params *cpm, void *d_spins,
              int32_t init_mode, int32_t max_record_sweeps, void *stream);

/* Run n_sweeps sweeps (CPM: Monte Carlo steps) of every lattice (Alg. 1).
 * On return (in stream order) the caller's buffer holds the new state.
 * record != 0 appends the observables after each sweep to the ring.       */
int spin_sweep(spin_ctx *ctx, int32_t n_sweeps, int32_t record, void *stream);

/* Number of int64 statistics per lattice per sweep:
 *   Ising 2: (M = sum s, B = sum_bonds s s'); with second neighbours 3:
 *       (M, B over nearest-neighbour bonds, B2 over diagonal bonds);
 *   Potts 1+q_max: (B_eq = #equal bonds, n_0 .. n_{q_max-1});
 *   CPM n_types(n_types+1)/2 + 2: (C_ab for a <= b = #Moore contacts between
 *       different cells of types a and b, V2 = sum_cells (a-A)^2, V1 = sum_cells (a-A)). */
int spin_stats_width(const spin_ctx *ctx);

/* Number of sweeps recorded so far (records are numbered from 0). */
int64_t spin_num_records(const spin_ctx *ctx);

/* Copy records [first, first + n) of the ring.  Any output may be NULL; each
 * may be a device or a (pinned or pageable) host pointer.
 *   stats [n][n_lattices][width] int64, exact;
 *   E, M  [n][n_lattices] float: energy per site and magnetisation per site
 *   (Ising: E = -J B - J2 B2 - h M, M = sum s; Potts: E = -J B_eq,
 *   M = (q max_k n_k - N)/(q - 1); CPM: E = total H, M = adhesion energy),
 *   computed in double from the exact integers and rounded once.
 * Only the last max_record_sweeps records are held (SPIN_EINVAL otherwise). */
int spin_observables(spin_ctx *ctx, int64_t first, int32_t n, int64_t *stats, float *E,
                     float *M, void *stream);

/* Statistics of the current state, recomputed from the lattice
 * ([n_lattices][width] int64, device or host pointer). */
int spin_current_stats(spin_ctx *ctx, int64_t *stats, void *stream);

/* Exact integer moments over records [first, first + n) per lattice:
 * [n_lattices][n_mom] int64 with n_mom = 1 + w + w(w+1)/2 for w = width:
 * (count, sum_i X_i, sum_{i<=j} X_i X_j) in row-major upper-triangle order.
 * This is the adjoint reduction of the fluctuation estimator.             */
int spin_moments(spin_ctx *ctx, int64_t first, int32_t n, int64_t *moments, void *stream);
int spin_num_moments(const spin_ctx *ctx);

/* Fluctuation estimator d<O>/dtheta = <dO/dtheta> - beta (<O dH/dtheta> - <O><dH/dtheta>)
 * over records [first, first + n) (not in the paper, which differentiates
 * relaxed Monte Carlo steps, Alg. 2; this is the exact identity for a
 * Boltzmann law, evaluated from the recorded samples).  Integer moments are
 * exact; the covariance is formed in FP64 on the device.
 * Ising: observable 0 = E/N, 1 = M/N; out[l][0] = d/dJ, out[l][1] = d/dh,
 *        and with second neighbours (geometry 2) out[l][2] = d/dJ2.
 * CPM:   observable 0 = adhesion energy per site; out[0][i] = d/dJ_ab for the
 *        i-th pair a <= b, then d/dlambda, d/dA (beta = 1/T).
 * pool != 0 pools the samples of all lattices (they must share theta) and
 * writes one row.  out: device or host pointer, FP64.                    */
int spin_grad(spin_ctx *ctx, int64_t first, int32_t n, int32_t observable, int32_t pool,
              double *out, void *stream);
int spin_num_grad(const spin_ctx *ctx);

/* Expectations over records [first, first + n): out[row][0] = <E>/N and
 * out[row][1] = <M>/N in FP64 (the same E and M as spin_observables), per
 * lattice or, with pool != 0, over all lattices (one row).  Formed on the
 * device from the exact integer moments.  Ising and CPM (CPM: <H>/N and
 * the mean adhesion energy per site).  out: device or host pointer. */
int spin_expectations(spin_ctx *ctx, int64_t first, int32_t n, int32_t pool, double *out,
                      void *stream);

/* Exchange step of the gradient when the chains that share theta are spread
 * over several processes (one per GPU): each process pools the exact integer
 * moments of its lattices over records [first, first + n) into limbs
 * [n_mom][4] (int64, device): the int128 value l0 + l1 2^32 + l2 2^64 + l3 2^96
 * with l0..l2 in [0, 2^32) and l3 signed, so that an element-wise SUM over
 * processes (an all-reduce) stays exact.  spin_grad_from_limbs turns summed
 * limbs into the pooled gradient (spin_num_grad doubles) and/or the pooled
 * expectations (2 doubles), as spin_grad / spin_expectations with pool != 0
 * would over all processes' samples; theta (and, for the estimator's
 * prefactors, N and beta) is taken from lattice 0 of ctx.  Device pointers. */
int spin_pooled_limbs(spin_ctx *ctx, int64_t first, int32_t n, int64_t *limbs, void *stream);
int spin_grad_from_limbs(spin_ctx *ctx, const int64_t *limbs, int32_t observable, double *grad, double *expect,
                         void *stream);

/* Replace temperatures/couplings (L, q and offsets must not change) and
 * rebuild the acceptance tables; takes effect at the next sweep. */
int spin_set_params(spin_ctx *ctx, const spin_lattice_desc *lat, const spin_cpm_params *cpm);

/* Launch form.  mode: 0 = batched persistent work-list launch (default),
 * 1 = plain per-lattice launches (two per lattice per sweep of a simple
 * per-chunk kernel), 3 = the kernels of mode 0 launched once per lattice per
 * sweep (the row-strip kernel for L = 512, 1024, 2048, the tile kernel for
 * the other sides that are multiples of 16, each lattice cut into its own
 * items: what batching the launches saves), 2 = resident
 * (Ising only, every L a multiple of 16 and <= 256, or only triangular
 * lattices with L <= 240, or only second-neighbour lattices with L <= 256: one
 * CTA per lattice keeps it in shared memory for all sweeps of a spin_sweep
 * call, one launch; for a CPM context on a device with cooperative launch,
 * the persistent form: all Monte Carlo steps of a call in one cooperative
 * launch with bounded grid barriers between the sub-steps).
 * use_graph: capture the sweep loop in a CUDA graph.  tile_rows: work-item
 * height in rows for mode 0 (0 = keep the current value, -1 = default items:
 * about 32 KB for the tile kernel; for the Ising row-strip kernel each strip
 * lattice cut into equal row ranges, at most one item per resident warp of the
 * launch and each as small as that allows, at least 8 rows); in mode 2, the
 * CTAs per square Ising lattice: 1 (or -1) = one CTA holds the lattice, 2 or 4
 * = the lattice's rows are split over a thread-block cluster of that many CTAs
 * that exchange their edge rows through distributed shared memory after every
 * colour sub-step (for batches of fewer lattices than SMs; threads 256, 512 or
 * 1024), 0 = keep.  threads: CTA size of the tile kernel (128, 256 or 512; 0 =
 * keep) and of the square-lattice resident kernel (also 1024 there); the warp
 * row-strip kernel uses 8 warps per CTA for 512, else 4.
 * Results do not depend on any of these. */
int spin_set_launch(spin_ctx *ctx, int32_t mode, int32_t use_graph, int32_t tile_rows,
                    int32_t threads);
/* Time the launch forms and tile shapes on the current state (the state is
 * saved and restored) and keep the fastest; the choice is cached per batch
 * shape in the file named by $SPINMC_TUNE_CACHE when it is set.  A trial
 * runs sweeps_per_trial sweeps (at least 2), repeated with more sweeps (up to
 * 4096) while it lasts under about a millisecond.                          */
int spin_autotune(spin_ctx *ctx, int32_t sweeps_per_trial, void *stream);
/* Current launch form as (mode, use_graph, tile_rows, threads); in mode 2
 * tile_rows is the cluster size (0 for one CTA per lattice). */
int spin_get_launch(const spin_ctx *ctx, int32_t out[4]);

/* Copy the spins between the context's device state and host memory (the
 * span of all lattices, element type of the model).  A load also recomputes
 * the running statistics (and, for CPM, the cell areas) from the loaded
 * state, so records taken after it describe the new chain.               */
int spin_load_spins(spin_ctx *ctx, const void *host, void *stream);
int spin_store_spins(spin_ctx *ctx, void *host, void *stream);

/* The same for Ising contexts with one bit per spin on the host: bit e of the
 * packed buffer (32-bit words, bit e % 32 of word e / 32) is 1 where element e
 * of the spin span holds -1.  Every lattice's spin_offset must be a multiple of
 * 32 (the binding aligns offsets to 256); otherwise SPIN_EINVAL.  A load
 * unpacks the lattices' elements only (other bytes of the span keep their
 * values) and recomputes the running statistics; a store writes
 * spin_packed_words(ctx) words, with 0 for the bits outside the lattices.
 * Not in the paper: an eightfold smaller host transfer than int8 spins. */
int32_t spin_packed_words(const spin_ctx *ctx);
int spin_load_spins_packed(spin_ctx *ctx, const uint32_t *host, void *stream);
int spin_store_spins_packed(spin_ctx *ctx, uint32_t *host, void *stream);
/* One host-to-host job in one call: spin_load_spins_packed(host_in) (skipped
 * when host_in is NULL), spin_sweep(n_sweeps, record), then
 * spin_store_spins_packed(host_out) (skipped when host_out is NULL), with the
 * same spins, statistics, records and sweep counter as those three calls.
 * With an odd n_sweeps in launch mode 0 or 3 the loaded state is unpacked
 * into the context's ping-pong buffer, so the last sweep lands in the
 * caller's spin buffer and the copy that ends an odd spin_sweep call is not
 * needed.  One sweep with both buffers in launch mode 0 (square lattices,
 * offsets of the L = 512, 1024, 2048 lattices multiples of 128): the row-strip
 * kernel reads those lattices' rows from the uploaded bits and writes their
 * bits beside the int8 rows, and only the other lattices are unpacked and
 * packed by separate kernels.  A second packed buffer of the context holds
 * the output bits.  host_in / host_out: pinned host memory for asynchronous copies,
 * spin_packed_words(ctx) words each; asynchronous on the stream.  Errors as
 * the three calls (SPIN_EINVAL for non-Ising contexts or offsets % 32 != 0).
 * Not in the paper.                                                        */
int spin_sweep_packed(spin_ctx *ctx, const uint32_t *host_in, uint32_t *host_out, int32_t n_sweeps,
                      int32_t record, void *stream);

/* Checkpoint = (sweep counter, record count, CPM areas, spins).  With
 * host_blob == NULL, *size receives the size needed. Restoring into a
 * context of the same shape continues the chain bit-identically.       */
int spin_checkpoint(spin_ctx *ctx, void *host_blob, size_t *size, void *stream);
int spin_restore(spin_ctx *ctx, const void *host_blob, size_t size, void *stream);

/* Kernel timing for roofline measurements.  While enabled (enable != 0),
 * spin_sweep launches directly (no graph replay) and brackets each launch of
 * the main sweep kernel (the batched work-list kernel, or the per-lattice
 * kernels of the plain form) with CUDA events on the caller's stream, up to
 * max_launches launches.  spin_profile_read synchronises the stream and
 * writes, for the three kernel classes (0: shared-memory tile kernel of the
 * batched form, 1: warp row-strip kernel of the batched form for L in
 * {512, 1024, 2048}, 2: per-lattice kernels of the plain form), the summed
 * kernel time in ms (total_ms[3]) and the number of timed launches
 * (launches[3]); enabling again resets the sums.  Not in the paper:
 * measurement plumbing. */
int spin_profile(spin_ctx *ctx, int32_t enable, int32_t max_launches);
int spin_profile_read(spin_ctx *ctx, double *total_ms, int64_t *launches, void *stream);

/* Self-test of the bounded grid barrier of the CPM persistent form (failure
 * detection without a GPU fault): one cooperative launch of `blocks` blocks
 * (1 <= blocks <= the SM count) runs `rounds` barriers that complete after
 * blocks + missing arrivals (0 <= missing <= blocks).  With missing = 0 every
 * barrier completes and the call returns SPIN_OK; with missing > 0 no barrier
 * can complete, every block gives up after the bounded wait (1 s) and the call
 * returns SPIN_ETIMEOUT with the device still usable.  Synchronises the
 * stream.  SPIN_EINVAL for arguments out of range or a device without
 * cooperative launch. */
int spin_barrier_selftest(int32_t blocks, int32_t missing, int32_t rounds, void *stream);

/* The random stream by itself (the RNG paragraph above; Alg. 1 draws one
 * uniform number per proposal, and this library draws it from Philox4x32-10):
 * *out (device, 4 bytes) = XOR of all four 32-bit words of the blocks for
 * counters (g, lattice, sweep, colour), g = g0 .. g0 + n_groups - 1, under
 * seed's key.  The blocks come from the same device code as the sweeps'
 * draws, so the digest checks that code against another implementation, and
 * the call's duration bounds the rate of any sweep on this stream (an Ising
 * update consumes one word, a Potts or CPM update two).  Asynchronous.
 * SPIN_EINVAL if out is NULL or g0 + n_groups > 2^32.                        */
int spin_philox_xor(uint64_t seed, uint32_t lattice, uint32_t sweep, uint32_t colour, uint32_t g0,
                    uint32_t n_groups, uint32_t *out, void *stream);

/* Device-side bounds checks (not in the paper: a debugging aid).  The
 * library built with -DSPIN_CHECK (libspinmc_check.so, build variant "check")
 * checks every work-list entry, shared-memory ring and queue index and table
 * address in its sweep kernels before use; a failed check records a code
 * (1xx: Ising kernels, 12x: Potts, 13x: CPM, 14x: statistics) in a device
 * word, the access is skipped and nothing traps.  spin_check_status
 * synchronises the device, writes the first recorded code (0: none) to
 * *first_code, clears the words, and returns 1 in a check build, 0 in other
 * builds (whose kernels have no checks), or a negative error code.          */
int spin_check_status(uint32_t *first_code);

uint32_t spin_sweep_index(const spin_ctx *ctx);
int32_t spin_gpu_launches(const spin_ctx *ctx); /* kernels launched by the last spin_sweep */
const char *spin_last_error(const spin_ctx *ctx);
void spin_destroy(spin_ctx *ctx);
int spin_version(void);   /* 2: spin_lattice_desc carries lattice_id */

/* ------------------------------------------------------------------------
 * Allocation-free Ising sweep.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (code running inside another
 * framework's memory pool or allocator hook, processes whose device memory is
 * reserved up front, embeddings that forbid allocation after start-up).
 *
 * Runs sweeps first_sweep .. first_sweep + n_sweeps - 1 of the Ising chain
 * defined by (seed, lat) on the caller's int8 spins with the result of
 * spin_sweep (bit-identical spins and statistics), without a context and
 * without allocating: its scratch (second spin buffer, tables, work list,
 * counters) is a static device array of SPIN_NOALLOC_SCRATCH_BYTES that every
 * GPU which loads the library holds until exit.  Its launch plan is simpler
 * than a context's: lattices with L % 16 == 0 run on the tile kernel (also
 * L = 512, 1024 and 2048, which spin_sweep gives the faster row-strip
 * kernel), other even L on the per-site kernel.  Limits (SPIN_EINVAL beyond
 * them): L even in [4, 2048], n_lattices <= 4096, and the lattices' span
 * (largest spin_offset + L*L bytes) plus about 2 KB of descriptors per 64
 * lattices within the 16 MiB array -- for example three 2048^2 lattices fit,
 * four do not.
 * d_stats: NULL or device int64 [n_sweeps][n_lattices][2] = (M, B) after
 * each sweep.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture.
 * Calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  Returns SPIN_OK, SPIN_EINVAL or SPIN_ECUDA.
 * ------------------------------------------------------------------------ */
#define SPIN_NOALLOC_SCRATCH_BYTES (16u << 20)
int spin_ising_sweep_noalloc(uint64_t seed, int32_t n_lattices, const spin_lattice_desc *lat,
                             void *d_spins, uint32_t first_sweep, int32_t n_sweeps,
                             int64_t *d_stats, void *stream);

/* ------------------------------------------------------------------------
 * Batched cellular Potts model (Sec. "Cellular Potts model"; the paper's
 * cell-sorting setup: 36 cells + medium, T = 8, A = 25, lambda = 1).  Many
 * independent lattices of one side L, each run by one thread block for all
 * Monte Carlo steps of a call; caller-owned buffers, nothing allocated:
 *   ids   int32 [n_lattices][L][L] (cell ids, 0 = medium),
 *   types uint8 [n_lattices][n_cells + 1] (type of each id),
 *   areas int32 [n_lattices][n_cells + 1] (sites per id),
 *   stats int64 [n_steps][n_lattices][n_types (n_types + 1) / 2 + 2] or NULL:
 *         after every step, C_ab (a <= b, unordered Moore contacts between
 *         different cells), V2 = sum (a_c - A)^2 and V1 = sum (a_c - A),
 *   workspace: spin_cpm_batch_workspace_bytes(cpm) bytes of device memory
 *         (16-byte aligned) for J and the acceptance table.
 * A step is the four colour sub-steps of the single-lattice model, with the
 * same random numbers (the batch index is the lattice word of the counter),
 * so lattice l follows the chain of a one-lattice context with lattice index
 * l.  Limits: L % 4 == 0, 8 <= L <= 128, 1 <= n_cells < L*L,
 * n_cells + 1 <= 4096, n_types in [1, 8], J symmetric, T > 0.
 * ------------------------------------------------------------------------ */
int64_t spin_cpm_batch_workspace_bytes(const spin_cpm_params *cpm);
/* Square cells (cpm->init_side, cpm->init_cols) in every lattice, types from
 * cpm->cell_type (host, shared by all lattices) or drawn per lattice, areas. */
int spin_cpm_batch_init(uint64_t seed, int32_t n_lattices, int32_t L, const spin_cpm_params *cpm, int32_t *ids,
                        uint8_t *types, int32_t *areas, void *stream);
/* n_steps Monte Carlo steps with step indices first_step, first_step + 1, ..
 * Calls that share a workspace must be ordered on one stream.               */
int spin_cpm_batch_run(uint64_t seed, int32_t n_lattices, int32_t L, const spin_cpm_params *cpm, int32_t *ids,
                       const uint8_t *types, int32_t *areas, uint32_t first_step, int32_t n_steps, int64_t *stats,
                       void *workspace, void *stream);

/* ------------------------------------------------------------------------
 * BF16 MLP surrogate 3 -> 64 -> 64 -> 2 (ReLU) mapping (beta, J, h) to
 * (<E>/N, <M>/N).  Not in the paper.  Weights live in one device buffer
 * of spin_mlp_param_count() floats (FP32 master copy, layout W1[64][3],
 * b1[64], W2[64][64], b2[64], W3[2][64], b3[2]); the kernels round weights,
 * activations and the backward signal of the second layer to BF16 and
 * accumulate in FP32 (the 64-wide products on the tensor cores).  Inputs are
 * normalised as x' = (x - mu) * inv_sigma (mu, inv_sigma: 3 floats each,
 * device).
 * ------------------------------------------------------------------------ */
int spin_mlp_param_count(void);
/* Y[n][2] = net(X[n][3]). All pointers device. */
int spin_mlp_forward(const float *params, const float *mu, const float *inv_sigma,
                     const float *X, int32_t n, float *Y, void *stream);
/* Loss L = 1/(2n) sum |Y - T|^2; writes grad[param_count] (dL/dparams),
 * loss[1] and, if dX != NULL, dX[n][3] = dL/dX.  All pointers device.   */
int spin_mlp_backward(const float *params, const float *mu, const float *inv_sigma,
                      const float *X, const float *T, int32_t n, float *grad, float *loss,
                      float *dX, void *stream);
/* Adam (Kingma & Ba) on params with moments m, v (device), step >= 1.    */
int spin_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr,
                  float beta1, float beta2, float eps, void *stream);
/* The same Adam update on any n parameters (used for the fit of J and h). */
int spin_adam(float *params, const float *grad, float *m, float *v, int32_t n, int32_t step, float lr,
              float beta1, float beta2, float eps, void *stream);

/* ------------------------------------------------------------------------
 * Differentiable Monte Carlo (Alg. 2, Sec. "Methods"; used in Sec.
 * "Optimization of the exchange parameters" to steer an Ising lattice
 * towards a target pattern by optimising one exchange parameter per bond).
 *
 * Relaxed spins s in [-1, 1], float32.  A sweep is colour 0 then colour 1
 * of the checkerboard ((x + y) & 1); in a sub-step every site of the colour
 * takes, at once,
 *   n = sum_j J_ij s_j,   dE = 2 s (n + h),   p = exp(-beta dE) (not clipped),
 *   r = (u >> 8) * 2^-24, q = 1 / (1 + exp(-alpha (p - r))),
 *   s <- q (-s) + (1 - q) s,
 * for H = -sum_<ij> J_ij s_i s_j - h sum_i s_i.  u is the site's Philox4x32-10
 * lane in the layout of the Ising sweep: key = (seed_lo, seed_hi), counter =
 * (k >> 2, lattice, sweep, colour), lane k & 3, k = (y L + x) >> 1.  As alpha
 * grows the update becomes Metropolis with acceptance r < exp(-beta dE).
 *
 * Layouts (device, float32, 16-byte aligned, caller-owned; nothing is
 * allocated):  spins [n_lattices][L][L];  J [n_lattices][2][L][L] with
 * J[l][0][y][x] the bond (x, y)-(x+1, y) and J[l][1][y][x] the bond
 * (x, y)-(x, y+1), periodic;  tape [n_lattices][2 n_sweeps][L*L/2] (see
 * spin_dmc_tape_floats).  Limits: 8 <= L <= 64, L % 8 == 0 (one lattice per
 * thread block, held in shared memory); n_sweeps >= 1.  Return 0 or a
 * negative SPIN_E* code (SPIN_EINVAL for arguments out of range).
 * ------------------------------------------------------------------------ */
/* Floats of the tape for n_lattices x n_sweeps sweeps; negative if invalid. */
int64_t spin_dmc_tape_floats(int32_t n_lattices, int32_t L, int32_t n_sweeps);
/* n_sweeps relaxed sweeps with sweep indices first_sweep, first_sweep + 1, ..
 * on spins in place; tape receives the old values of each sub-step's active
 * sites (compressed index k order).                                         */
int spin_dmc_forward(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                     const float *J, float *spins, uint32_t first_sweep, int32_t n_sweeps,
                     float *tape, void *stream);
/* Reverse pass of the same call.  spins: the state spin_dmc_forward left
 * (read only); grad_spins: on entry dL/ds after the sweeps, on exit dL/ds
 * before them; grad_J: dL/dJ, overwritten.                                  */
int spin_dmc_backward(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                      const float *J, const float *spins, const float *tape, uint32_t first_sweep,
                      int32_t n_sweeps, float *grad_spins, float *grad_J, void *stream);
/* Pattern loss per lattice, loss[l] = sum (target - s)^2 (float64), and
 * grad_spins = -2 (target - s).                                              */
int spin_dmc_loss(int32_t n_lattices, int32_t L, const float *spins, const float *target,
                  float *grad_spins, double *loss, void *stream);
/* Discretisation of n spins: s <- -1 if s < 0 else +1.                      */
int spin_dmc_discretize(int64_t n, float *spins, void *stream);
/* Spin-value optimisation (Sec. "Optimization of the spin values"): the loss
 * is the energy itself.  energy[l] = -sum_<ij> J_ij s_i s_j - h sum_i s_i
 * (float64, each bond once); grad_spins (may be NULL) = dE/ds = -(n + h).   */
int spin_dmc_energy(int32_t n_lattices, int32_t L, float h, const float *J, const float *spins,
                    float *grad_spins, double *energy, void *stream);
/* Quantised spin-value step: s <- clip(s - eta sign(grad), -1, 1), sign(0) = 0,
 * over n spins.                                                             */
int spin_dmc_spin_step(int64_t n, float *spins, const float *grad, float eta, void *stream);
/* One spin-value iteration of the differentiable Monte Carlo in a single
 * launch, identical in result to: copy s, spin_dmc_forward on the copy,
 * spin_dmc_energy (gradient) of the relaxed copy, spin_dmc_backward to
 * dE(F(s))/ds, spin_dmc_spin_step(eta) and spin_dmc_discretize on s.  spins:
 * +-1 in, the updated discretised spins out; energy[l] (float64): the energy
 * of the discretised relaxed state.  1 <= n_sweeps <=
 * spin_dmc_spin_iter_max_sweeps(L).                                         */
int spin_dmc_spin_iter(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha, float eta,
                       uint32_t first_sweep, int32_t n_sweeps, const float *J, float *spins, double *energy,
                       void *stream);
int32_t spin_dmc_spin_iter_max_sweeps(int32_t L);
/* Largest n_sweeps spin_dmc_step accepts for side L (its tape stays in
 * shared memory); SPIN_EINVAL for an invalid L.                             */
int32_t spin_dmc_step_max_sweeps(int32_t L);
/* One whole optimisation iteration in a single launch, identical in result
 * to spin_dmc_forward + spin_dmc_loss + spin_dmc_backward + spin_adam (on J,
 * step `step`) + spin_dmc_discretize: spins (in: start state; out: the
 * discretised state), J, m, v ([n_lattices][2][L][L], Adam moments) updated
 * in place, loss[l] (float64) of the relaxed state.  target as in
 * spin_dmc_loss (16-byte aligned here).  1 <= n_sweeps <=
 * spin_dmc_step_max_sweeps(L).                                              */
int spin_dmc_step(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                  uint32_t first_sweep, int32_t n_sweeps, float *spins, float *J, float *m, float *v,
                  const float *target, double *loss, int32_t step, float lr, float beta1, float beta2,
                  float eps, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SPINMC_H */
