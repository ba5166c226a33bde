// abi.cpp -- host side of libspinmc.so: the C ABI declared in include/spinmc.h.
//
// Holds the per-context state (lattice descriptors, acceptance tables, the
// second spin buffer, statistics), validates arguments, builds the work list
// of the batched sweep, captures the sweep loop in CUDA graphs, and runs the
// autotuner.  Every step of the Monte Carlo path runs in the kernels of the
// .cu files; this file only plans and launches them.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"
#include "spinmc.h"

namespace spinmc {
cudaError_t set_ising_fused_smem(size_t smem);
cudaError_t set_potts_fused_smem(size_t smem);
cudaError_t launch_cpm_types(uint8_t *type, int n_cells, uint32_t lat, uint32_t k0, uint32_t k1,
                             cudaStream_t s);
cudaError_t launch_moments_i128(const StatsBufs &st, int64_t first, int n, void *out,
                                cudaStream_t s);
cudaError_t launch_pool_moments(const void *in, int n_lat, int n_mom, void *out, cudaStream_t s);
cudaError_t launch_i128_to_i64(const void *in, int64_t *out, int n, int *overflow, cudaStream_t s);
cudaError_t launch_i128_to_limbs(const void *in, int n, int64_t *limbs, cudaStream_t s);
cudaError_t launch_limbs_to_i128(const int64_t *limbs, int n, void *out, cudaStream_t s);
cudaError_t launch_grad_i128(const void *moments, int rows, GradParams p, double *out,
                             cudaStream_t s);
cudaError_t launch_expectations_i128(const void *moments, int rows, GradParams p, double *out,
                                     cudaStream_t s);
cudaError_t launch_copy_lattices(const void *src, void *dst, const LatDev *lats, int n_lat,
                                 int elem, cudaStream_t s);
cudaError_t occupancy_ising_strip(int *blocks_per_sm, int warps);
}  // namespace spinmc

using namespace spinmc;

namespace {

constexpr int kMaxItemBytes = 65536;   // bounds the per-thread packed counters
constexpr int kWholeMaxBytes = 16384;  // lattices up to 128 x 128 are one item
constexpr int kMaxL = 32768;

// NVTX range around one ABI call (visible in Nsight Systems timelines; no
// cost beyond two calls when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// The lattice word of a lattice's Philox counters: lattice_id - 1 when the
// caller gives one, else the lattice's index in this batch.
uint32_t rng_word(const spin_lattice_desc &d, int index) {
    return d.lattice_id ? d.lattice_id - 1u : (uint32_t)index;
}

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

}  // namespace

struct spin_ctx {
    int model = 0;
    uint64_t seed = 0;
    uint32_t k0 = 0, k1 = 0;
    int n_lat = 0;
    std::vector<spin_lattice_desc> lat;
    int maxL = 0;
    size_t elem = 1;
    // CPM
    int n_types = 0, lambda = 0, target = 0, n_cells = 0, init_side = 0, init_cols = 0;
    float T = 1.0f;
    std::vector<int32_t> Jt;
    // device buffers
    void *spins = nullptr;    // caller's
    void *spins2 = nullptr;   // ours (ping-pong partner)
    size_t span_elems = 0;
    LatDev *d_lats = nullptr;
    TabEntry *d_tabs = nullptr;
    Item *d_items = nullptr;
    int n_items = 0;
    Item *d_strip = nullptr;     // warp row-strip items (Ising, L in {512, 1024, 2048})
    int n_strip = 0, strip_grid = 0, strip_warps = 8, strip_qbits = 2, strip_chunks = 128;
    int32_t *d_generic = nullptr;
    int32_t *d_tri = nullptr;   // triangular lattices (geometry 1)
    int n_tri = 0, tri_maxL = 0;
    uint32_t *d_nnn_thr = nullptr;   // first and second neighbours (geometry 2): [n_lat][kNnnTab]
    int n_nnn = 0, nnn_maxL = 0;
    int n_generic = 0, generic_maxL = 0;
    std::vector<int> fast_ids;
    DevState *d_state = nullptr;
    StatsBufs st{};
    int width = 0;
    uint8_t *d_type = nullptr;
    int32_t *d_J = nullptr;
    int32_t *d_vol[2] = {nullptr, nullptr};   // CPM areas: [0] after a Monte Carlo step, [1] alternate
    int32_t *d_dvol[2] = {nullptr, nullptr};  // CPM area changes of the last two sub-steps
    int64_t *d_cpm_acc = nullptr;             // CPM persistent form: contact changes per step parity
    unsigned int *d_cpm_bar = nullptr;        // CPM persistent form: grid barrier words
    int cpm_grid = 0;                         // blocks of the CPM persistent form (0: unavailable)
    uint32_t *d_thr = nullptr;
    int n_thr = 0;
    double *d_latp = nullptr;   // [n_lat][kLatParams]
    double *d_cpmJ = nullptr;   // [pairs]
    void *d_scratch = nullptr;  // moments etc.
    size_t scratch_bytes = 0;
    int *d_flag = nullptr;      // [0] moment overflow, [1] a device wait gave up
    uint32_t *d_packed = nullptr;   // bit-packed transfer buffer (allocated at first use)
    uint32_t *d_packed2 = nullptr;  // second one: spin_sweep_packed's output bits
    // block ranges of the pack / unpack launches per lattice: every lattice, and
    // only the lattices below the strip sides (allocated with d_packed)
    int32_t *d_blk_all = nullptr, *d_blk_small = nullptr;
    int nblk_all = 0, nblk_small = 0;
    // host mirrors
    uint32_t t = 0;
    int64_t n_rec = 0;
    // launch form
    int mode = 0, use_graph = 1, tile_rows = 0, threads = 256;
    int cluster = 1;                      // resident form: CTAs per lattice (1, 2 or 4)
    int use_strip = 1;
    // launch mode 3: one launch per lattice, items [first, first + count) of
    // the strip list (strip = 1) or of the tile list
    struct LatRange {
        int strip, first, count;
    };
    std::vector<LatRange> per_lattice;
    int per_sm_strip = 1;
    int grid = 0;
    size_t smem = 0;
    int sm_count = 0;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side = nullptr;          // tile kernel runs here, beside the strip kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    GraphCache graphs[2][4];    // [record][two-sweep ping-pong kind: row formats at its ends]
    int last_launches = 0;
    // kernel timing (spin_profile)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_cls;
    int prof_n = 0;
    std::string err;
};

namespace {

int fail(spin_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(spin_ctx *c, cudaError_t e, const char *where) {
    return fail(c, SPIN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
    } while (0)

cudaStream_t S(void *stream) { return static_cast<cudaStream_t>(stream); }

// ---------------------------------------------------------------- tables
// Number of accepted values of a uniform uint32 draw, minus one:
// dE <= 0 -> all; else max(floor(exp(-beta dE) 2^32), 1) - 1.
uint32_t thr_from(double beta, double dE) {
    if (dE <= 0.0) return 0xFFFFFFFFu;
    double k = std::floor(std::exp(-beta * dE) * 4294967296.0);
    if (k < 1.0) k = 1.0;
    if (k > 4294967296.0) k = 4294967296.0;
    return (uint32_t)(k - 1.0);
}

void ising_table(const spin_lattice_desc &d, TabEntry *e) {
    const double beta = (double)d.beta;
    for (int c = 0; c < 2; ++c)
        for (int dn = 0; dn <= 4; ++dn) {
            const int s = c ? -1 : 1;
            const int n = 4 - 2 * dn;
            const double dE = 2.0 * (double)s * ((double)d.J * (double)n + (double)d.h);
            TabEntry &x = e[dn + 5 * c];
            x.thr = thr_from(beta, dE);
            const int dM = -2 * s, dB = -2 * s * n;
            x.delta = dB * 65536 + dM;
        }
}

// Triangular lattice: entry dn + 7 c, dn = down neighbours of six, n = 6 - 2 dn.
void tri_table(const spin_lattice_desc &d, TabEntry *e) {
    const double beta = (double)d.beta;
    for (int c = 0; c < 2; ++c)
        for (int dn = 0; dn <= 6; ++dn) {
            const int s = c ? -1 : 1;
            const int n = 6 - 2 * dn;
            const double dE = 2.0 * (double)s * ((double)d.J * (double)n + (double)d.h);
            TabEntry &x = e[dn + 7 * c];
            x.thr = thr_from(beta, dE);
            x.delta = (-2 * s * n) * 65536 + (-2 * s);
        }
}

// First and second neighbours: entry 25 cdown + 5 d1 + d2 (d1, d2 = down
// spins among the four nearest and the four diagonal neighbours).
void nnn_table(const spin_lattice_desc &d, uint32_t *thr) {
    const double beta = (double)d.beta;
    for (int c = 0; c < 2; ++c)
        for (int d1 = 0; d1 <= 4; ++d1)
            for (int d2 = 0; d2 <= 4; ++d2) {
                const int s = c ? -1 : 1;
                const int n1 = 4 - 2 * d1, n2 = 4 - 2 * d2;
                const double dE = 2.0 * (double)s * ((double)d.J * (double)n1 + (double)d.J2 * (double)n2 + (double)d.h);
                thr[25 * c + 5 * d1 + d2] = thr_from(beta, dE);
            }
}

void potts_table(const spin_lattice_desc &d, TabEntry *e) {
    const double beta = (double)d.beta;
    for (int dd = -4; dd <= 4; ++dd) {
        const double dE = (double)d.J * (double)dd;
        e[dd + 4].thr = thr_from(beta, dE);
        e[dd + 4].delta = -dd;
    }
}

int stats_width(int model, const std::vector<spin_lattice_desc> &lat, int n_types) {
    if (model == SPIN_ISING) return lat[0].geometry == 2 ? 3 : 2;   // (M, B[, B2])
    if (model == SPIN_POTTS) {
        int q = 2;
        for (auto &d : lat) q = std::max(q, d.q);
        return 1 + q;
    }
    return n_types * (n_types + 1) / 2 + 2;
}

int validate(spin_ctx *ctx, int model, int n, const spin_lattice_desc *lat,
             const spin_cpm_params *cpm) {
    if (model < 0 || model > 2) return fail(ctx, SPIN_EINVAL, "unknown model");
    if (n <= 0 || n > 65535 || !lat) return fail(ctx, SPIN_EINVAL, "n_lattices must be in [1, 65535]");
    if ((model == SPIN_CPM) != (cpm != nullptr))
        return fail(ctx, SPIN_EINVAL, "cpm parameters are required exactly for the CPM model");
    if (model == SPIN_CPM && n != 1) return fail(ctx, SPIN_EINVAL, "the CPM model takes one lattice");
    std::vector<std::pair<uint64_t, uint64_t>> spans;
    for (int i = 0; i < n; ++i) {
        const spin_lattice_desc &d = lat[i];
        char buf[160];
        if (d.L < 4 || (d.L & 1) || d.L > kMaxL) {
            snprintf(buf, sizeof buf, "lattice %d: L=%d must be even and in [4, %d]", i, d.L, kMaxL);
            return fail(ctx, SPIN_EINVAL, buf);
        }
        if (model != SPIN_CPM) {
            if (d.geometry < 0 || d.geometry > 2) return fail(ctx, SPIN_EINVAL, "geometry must be 0, 1 or 2");
            if (d.geometry == 1 && (model != SPIN_ISING || d.L % 6 != 0))
                return fail(ctx, SPIN_EINVAL, "the triangular lattice needs the Ising model and L % 6 == 0");
            if (d.geometry == 2 && model != SPIN_ISING)
                return fail(ctx, SPIN_EINVAL, "second neighbours need the Ising model");
            if ((d.geometry == 2) != (lat[0].geometry == 2))
                return fail(ctx, SPIN_EINVAL, "lattices with second neighbours cannot share a context with others");
            if (!std::isfinite(d.J2) || (d.geometry != 2 && d.J2 != 0.0f))
                return fail(ctx, SPIN_EINVAL, "J2 must be finite, and 0 unless geometry is 2");
        } else if (d.geometry != 0 || d.J2 != 0.0f) {
            return fail(ctx, SPIN_EINVAL, "CPM lattices take geometry 0 and J2 = 0");
        }
        if (model == SPIN_POTTS) {
            if (d.q < 2 || d.q > 255) {
                snprintf(buf, sizeof buf, "lattice %d: q=%d out of [2, 255]", i, d.q);
                return fail(ctx, SPIN_EINVAL, buf);
            }
            if (d.h != 0.0f) return fail(ctx, SPIN_EINVAL, "Potts lattices take no field (h must be 0)");
        }
        if (model != SPIN_CPM) {
            if (!std::isfinite(d.beta) || d.beta < 0.0f)
                return fail(ctx, SPIN_EINVAL, "beta must be finite and >= 0");
            if (!std::isfinite(d.J) || !std::isfinite(d.h))
                return fail(ctx, SPIN_EINVAL, "J and h must be finite");
        } else if (d.L % 4) {
            return fail(ctx, SPIN_EINVAL, "CPM lattices need L % 4 == 0");
        }
        spans.push_back({d.spin_offset, d.spin_offset + (uint64_t)d.L * d.L});
    }
    std::sort(spans.begin(), spans.end());
    for (size_t i = 1; i < spans.size(); ++i)
        if (spans[i].first < spans[i - 1].second) return fail(ctx, SPIN_EINVAL, "lattices overlap");
    if (cpm) {
        if (cpm->n_types < 1 || cpm->n_types > 8 || !cpm->J_type)
            return fail(ctx, SPIN_EINVAL, "CPM n_types must be in [1, 8] with a J table");
        for (int a = 0; a < cpm->n_types; ++a)
            for (int b = 0; b < cpm->n_types; ++b)
                if (cpm->J_type[a * cpm->n_types + b] != cpm->J_type[b * cpm->n_types + a])
                    return fail(ctx, SPIN_EINVAL, "CPM J table must be symmetric");
        if (!(cpm->T > 0.0f) || !std::isfinite(cpm->T)) return fail(ctx, SPIN_EINVAL, "CPM T must be > 0");
        if (cpm->n_cells < 1 || cpm->n_cells >= lat[0].L * lat[0].L)
            return fail(ctx, SPIN_EINVAL, "CPM n_cells out of range");
        if (cpm->lambda < 0 || cpm->target_area < 0) return fail(ctx, SPIN_EINVAL, "lambda and A must be >= 0");
        if (cpm->reserved != 0) return fail(ctx, SPIN_EINVAL, "reserved field must be 0");
        if (cpm->cell_type) {
            if (cpm->cell_type[0] != 0) return fail(ctx, SPIN_EINVAL, "cell_type[0] must be 0 (medium)");
            for (int c = 1; c <= cpm->n_cells; ++c)
                if (cpm->cell_type[c] >= cpm->n_types) return fail(ctx, SPIN_EINVAL, "cell type out of range");
        } else if (cpm->n_types < 3) {
            return fail(ctx, SPIN_EINVAL, "drawn cell types need n_types >= 3");
        }
    }
    return SPIN_OK;
}

int upload_tables(spin_ctx *ctx, cudaStream_t s) {
    if (ctx->model == SPIN_CPM) {
        std::vector<uint32_t> thr;
        thr.push_back(0xFFFFFFFFu);  // dE = 0 (never read: dE <= 0 accepts)
        for (int dE = 1; dE < (1 << 22); ++dE) {
            const double k = std::floor(std::exp(-(double)dE / (double)ctx->T) * 4294967296.0);
            if (k <= 1.0) break;
            thr.push_back((uint32_t)(std::min(k, 4294967296.0) - 1.0));
        }
        if (ctx->d_thr) cudaFree(ctx->d_thr);
        ctx->d_thr = nullptr;
        CK(cudaMalloc(&ctx->d_thr, sizeof(uint32_t) * thr.size()));
        CK(cudaMemcpy(ctx->d_thr, thr.data(), sizeof(uint32_t) * thr.size(), cudaMemcpyHostToDevice));
        ctx->n_thr = (int)thr.size();
        CK(cudaMemcpy(ctx->d_J, ctx->Jt.data(), sizeof(int32_t) * ctx->Jt.size(), cudaMemcpyHostToDevice));
        // observables: J per pair (a <= b)
        std::vector<double> pj;
        for (int a = 0; a < ctx->n_types; ++a)
            for (int b = a; b < ctx->n_types; ++b) pj.push_back((double)ctx->Jt[a * ctx->n_types + b]);
        CK(cudaMemcpy(ctx->d_cpmJ, pj.data(), sizeof(double) * pj.size(), cudaMemcpyHostToDevice));
        std::vector<double> lp = {0.0, 0.0, (double)ctx->lat[0].L * ctx->lat[0].L, 1.0 / (double)ctx->T, 0.0};
        CK(cudaMemcpy(ctx->d_latp, lp.data(), sizeof(double) * kLatParams, cudaMemcpyHostToDevice));
        return SPIN_OK;
    }
    std::vector<TabEntry> tab((size_t)ctx->n_lat * kTabStride, TabEntry{0u, 0});
    std::vector<double> lp((size_t)ctx->n_lat * kLatParams);
    std::vector<uint32_t> nnn(ctx->n_nnn ? (size_t)ctx->n_lat * kNnnTab : 0);
    for (int i = 0; i < ctx->n_lat; ++i) {
        const spin_lattice_desc &d = ctx->lat[i];
        if (ctx->model == SPIN_ISING && d.geometry == 1)
            tri_table(d, &tab[(size_t)i * kTabStride]);
        else if (ctx->model == SPIN_ISING)
            ising_table(d, &tab[(size_t)i * kTabStride]);
        else
            potts_table(d, &tab[(size_t)i * kTabStride]);
        if (ctx->model == SPIN_ISING && d.geometry == 2) nnn_table(d, &nnn[(size_t)i * kNnnTab]);
        double *l = &lp[(size_t)kLatParams * i];
        l[0] = d.J;
        l[1] = d.h;
        l[2] = (double)d.L * d.L;
        l[3] = ctx->model == SPIN_POTTS ? (double)d.q : (double)d.beta;
        l[4] = d.geometry == 2 ? (double)d.J2 : 0.0;
    }
    (void)s;
    CK(cudaMemcpy(ctx->d_tabs, tab.data(), sizeof(TabEntry) * tab.size(), cudaMemcpyHostToDevice));
    if (!nnn.empty())
        CK(cudaMemcpy(ctx->d_nnn_thr, nnn.data(), sizeof(uint32_t) * nnn.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_latp, lp.data(), sizeof(double) * lp.size(), cudaMemcpyHostToDevice));
    return SPIN_OK;
}

void drop_graphs(spin_ctx *ctx) {
    for (auto &r : ctx->graphs)
        for (auto &g : r) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            g.launches = 0;
        }
}

// Ising strip items: warps take items round robin, so the launch lasts as long
// as the warp with the most rows.  Items are cut so that their count fits the
// resident warps `budget` (times the rounds), each lattice into equal row
// ranges of at most the smallest per-item site count that allows, and never
// thinner than kStripMinRows (every item recomputes a halo row per colour).
constexpr int kStripRounds = 1;
constexpr int kStripMinRows = 8;

void balanced_strip_items(const spin_ctx *ctx, const std::vector<int> &ids, size_t budget,
                          std::vector<Item> &out) {
    auto pieces = [&](int L, size_t per) {
        const size_t k = ((size_t)L * L + per - 1) / per;
        return (int)std::min<size_t>(k, (size_t)std::max(1, L / kStripMinRows));
    };
    size_t lo = 1, hi = 1;
    for (int id : ids) hi = std::max(hi, (size_t)ctx->lat[id].L * ctx->lat[id].L);
    while (lo < hi) {   // smallest per-item site count whose pieces fit the budget
        const size_t mid = lo + (hi - lo) / 2;
        size_t n = 0;
        for (int id : ids) n += (size_t)pieces(ctx->lat[id].L, mid);
        if (n <= budget) hi = mid;
        else lo = mid + 1;
    }
    for (int id : ids) {
        const int L = ctx->lat[id].L, k = pieces(L, lo);
        for (int i = 0; i < k; ++i) {
            const int r0 = (int)((int64_t)i * L / k), r1 = (int)((int64_t)(i + 1) * L / k);
            out.push_back(Item{id, r0, r1 - r0, 0});
        }
    }
}

// Work list of the batched launch over the vectorisable lattices.
int plan(spin_ctx *ctx) {
    drop_graphs(ctx);
    if (ctx->model == SPIN_CPM) return SPIN_OK;
    std::vector<Item> items, strip;
    std::vector<int> strip_ids;
    size_t smem = 16, strip_bytes = 0;
    ctx->strip_qbits = 2;
    for (int id : ctx->fast_ids) {
        const int L = ctx->lat[id].L;
        const bool strip_L = L == 512 || L == 1024 || L == 2048;
        const bool potts_strip = ctx->model == SPIN_POTTS && ctx->lat[id].q <= 8;
        if (ctx->use_strip && strip_L && (ctx->model == SPIN_ISING || potts_strip)) {
            strip_ids.push_back(id);
            strip_bytes += (size_t)L * L;
            if (ctx->model == SPIN_POTTS && ctx->lat[id].q > 4) ctx->strip_qbits = 3;
            continue;
        }
        if (L * L <= kWholeMaxBytes) {
            items.push_back(Item{id, 0, L, 1});
            smem = std::max(smem, (size_t)L * L);
            continue;
        }
        int rows = ctx->tile_rows > 0 ? ctx->tile_rows : std::max(1, 32768 / L);
        rows = std::min(rows, L);
        rows = std::max(1, std::min(rows, kMaxItemBytes / L));
        for (int r0 = 0; r0 < L; r0 += rows) {
            const int nr = std::min(rows, L - r0);
            items.push_back(Item{id, r0, nr, 0});
        }
        smem = std::max(smem, (size_t)(rows + 4) * L);
    }
    // mode 3 launches lattice by lattice: keep each lattice's items together
    if (ctx->mode != 3)
        std::stable_sort(items.begin(), items.end(), [&](const Item &a, const Item &b) {
            return (size_t)a.nrows * ctx->lat[a.lat].L > (size_t)b.nrows * ctx->lat[b.lat].L;
        });
    if (ctx->d_items) cudaFree(ctx->d_items);
    ctx->d_items = nullptr;
    ctx->n_items = (int)items.size();
    if (!items.empty()) {
        CK(cudaMalloc(&ctx->d_items, sizeof(Item) * items.size()));
        CK(cudaMemcpy(ctx->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice));
    }
    if (ctx->d_strip) cudaFree(ctx->d_strip);
    ctx->d_strip = nullptr;
    ctx->n_strip = 0;
    if (!strip_ids.empty()) {
        // Ising: 8 warps per block from 512 threads; Potts (more registers,
        // measured faster with 8) from 256.
        ctx->strip_warps = ctx->threads >= (ctx->model == SPIN_ISING ? 512 : 256) ? 8 : 4;
        int per_sm = 0;
        if (ctx->model == SPIN_ISING)
            CK(occupancy_ising_strip(&per_sm, ctx->strip_warps));
        else {
            int maxL = 0;
            for (int id : strip_ids) maxL = std::max(maxL, ctx->lat[id].L);
            ctx->strip_chunks = maxL / 16;
            CK(occupancy_potts_strip(&per_sm, ctx->strip_warps, ctx->strip_qbits, ctx->strip_chunks));
        }
        // Default row blocks: 64 KB for Ising.  Potts sites cost about twice as
        // much and its batches are smaller, so its default spreads the strip
        // lattices over the resident warps in about one wave (the recomputed
        // halo costs one row per item, so items stay as tall as that allows).
        const size_t slots = (size_t)ctx->sm_count * std::max(1, per_sm) * ctx->strip_warps;
        ctx->per_sm_strip = std::max(1, per_sm);
        if (ctx->mode == 3 && ctx->model == SPIN_ISING && ctx->tile_rows <= 0) {
            // each lattice alone on the GPU: its own balanced cut
            for (int id : strip_ids) balanced_strip_items(ctx, std::vector<int>{id}, slots * kStripRounds, strip);
        } else if (ctx->model == SPIN_ISING && ctx->tile_rows <= 0) {
            balanced_strip_items(ctx, strip_ids, slots * kStripRounds, strip);
        } else {
            for (int id : strip_ids) {
                const int L = ctx->lat[id].L;
                int def_rows = 65536 / L;
                if (ctx->model == SPIN_POTTS)
                    def_rows = (int)std::min<size_t>(65536 / L, std::max<size_t>(4, (strip_bytes + slots * L - 1) / (slots * L)));
                int rows = std::max(1, std::min(L, ctx->tile_rows > 0 ? ctx->tile_rows : def_rows));
                for (int r0 = 0; r0 < L; r0 += rows) strip.push_back(Item{id, r0, std::min(rows, L - r0), 0});
            }
        }
        ctx->n_strip = (int)strip.size();
        CK(cudaMalloc(&ctx->d_strip, sizeof(Item) * strip.size()));
        CK(cudaMemcpy(ctx->d_strip, strip.data(), sizeof(Item) * strip.size(), cudaMemcpyHostToDevice));
        ctx->strip_grid = std::max(1, std::min((ctx->n_strip + ctx->strip_warps - 1) / ctx->strip_warps,
                                               ctx->sm_count * std::max(1, per_sm)));
    }
    if (smem > 200 * 1024) return fail(ctx, SPIN_EINVAL, "work item does not fit in shared memory");
    ctx->smem = smem;
    if (ctx->model == SPIN_ISING)
        CK(set_ising_fused_smem(smem));
    else if (ctx->model == SPIN_POTTS)
        CK(set_potts_fused_smem(smem));
    ctx->grid = std::max(1, std::min(ctx->n_items, ctx->sm_count * std::max(1, (int)(2048 / ctx->threads))));
    // residency bound: at most as many blocks as fit on the GPU at once
    const int per_sm_smem = (int)((228 * 1024) / (smem + 1024));
    const int per_sm_thr = 2048 / ctx->threads;
    const int per_sm = std::max(1, std::min(per_sm_smem, per_sm_thr));
    ctx->grid = std::max(1, std::min(ctx->n_items, ctx->sm_count * per_sm));
    // per-lattice ranges of both lists (items of one lattice are contiguous
    // in mode 3)
    ctx->per_lattice.clear();
    if (ctx->mode == 3) {
        auto ranges = [&](const std::vector<Item> &v, int is_strip) {
            for (int i = 0; i < (int)v.size();) {
                int j = i;
                while (j < (int)v.size() && v[j].lat == v[i].lat) ++j;
                ctx->per_lattice.push_back({is_strip, i, j - i});
                i = j;
            }
        };
        ranges(strip, 1);
        ranges(items, 0);
    }
    return SPIN_OK;
}

// Event pair around one timed kernel launch (spin_profile).
bool prof_begin(spin_ctx *ctx, cudaStream_t s, int cls) {
    if (!ctx->prof || 2 * (ctx->prof_n + 1) > (int)ctx->prof_ev.size()) return false;
    ctx->prof_cls[ctx->prof_n] = cls;
    return cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], s) == cudaSuccess;
}

void prof_end(spin_ctx *ctx, cudaStream_t s) {
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], s);
    ++ctx->prof_n;
}

// One sweep of Ising/Potts lattices, src -> dst (batched) or in place (plain).
int launch_sweep(spin_ctx *ctx, void *src, void *dst, int record, cudaStream_t s, int &launches, int layout,
                 const uint32_t *src_bits = nullptr, uint32_t *dst_bits = nullptr) {
    const int w = ctx->width;
    if (ctx->mode == 1) {
        for (int c = 0; c < 2; ++c) {
            for (int id : ctx->fast_ids) {
                const int L = ctx->lat[id].L;
                const bool timed = prof_begin(ctx, s, 2);
                if (ctx->model == SPIN_ISING)
                    CK(launch_ising_plain(static_cast<int8_t *>(src) + ctx->lat[id].spin_offset, ctx->d_lats,
                                          id, rng_word(ctx->lat[id], id), L, ctx->d_tabs, ctx->k0, ctx->k1, ctx->d_state,
                                          ctx->st.delta, c, s));
                else
                    CK(launch_potts_plain(static_cast<uint8_t *>(src) + ctx->lat[id].spin_offset, ctx->d_lats,
                                          id, rng_word(ctx->lat[id], id), L, ctx->lat[id].q, ctx->d_tabs, ctx->k0, ctx->k1,
                                          ctx->d_state, ctx->st.delta, w, c, s));
                if (timed) prof_end(ctx, s);
                ++launches;
            }
            if (ctx->n_nnn && c == 0)
                for (int nc = 0; nc < 4; ++nc) {
                    CK(launch_ising_nnn(static_cast<int8_t *>(src), static_cast<int8_t *>(src), ctx->n_nnn,
                                        ctx->nnn_maxL, ctx->d_lats, ctx->d_nnn_thr, ctx->k0, ctx->k1, ctx->d_state,
                                        ctx->st.delta, nc, s));
                    ++launches;
                }
            if (ctx->n_tri && c == 0)
                for (int tc = 0; tc < 3; ++tc) {
                    CK(launch_ising_tri(static_cast<int8_t *>(src), static_cast<int8_t *>(src), ctx->d_tri, ctx->n_tri,
                                        ctx->tri_maxL, ctx->d_lats, ctx->d_tabs, ctx->k0, ctx->k1, ctx->d_state,
                                        ctx->st.delta, tc, s));
                    ++launches;
                }
            if (ctx->n_generic) {
                if (ctx->model == SPIN_ISING)
                    CK(launch_ising_generic(static_cast<int8_t *>(src), static_cast<int8_t *>(src), ctx->d_generic,
                                            ctx->n_generic, ctx->generic_maxL, ctx->d_lats, ctx->d_tabs,
                                            ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, c, s));
                else
                    CK(launch_potts_generic(static_cast<uint8_t *>(src), static_cast<uint8_t *>(src), ctx->d_generic,
                                            ctx->n_generic, ctx->generic_maxL, ctx->d_lats, ctx->d_tabs,
                                            ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, w, c, s));
                ++launches;
            }
        }
    } else {
        for (int nc = 0; nc < 4 && ctx->n_nnn; ++nc) {
            CK(launch_ising_nnn(static_cast<int8_t *>(src), static_cast<int8_t *>(dst), ctx->n_nnn, ctx->nnn_maxL,
                                ctx->d_lats, ctx->d_nnn_thr, ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, nc, s));
            ++launches;
        }
        for (int tc = 0; tc < 3 && ctx->n_tri; ++tc) {
            CK(launch_ising_tri(static_cast<int8_t *>(src), static_cast<int8_t *>(dst), ctx->d_tri, ctx->n_tri,
                                ctx->tri_maxL, ctx->d_lats, ctx->d_tabs, ctx->k0, ctx->k1, ctx->d_state,
                                ctx->st.delta, tc, s));
            ++launches;
        }
        for (int c = 0; c < 2 && ctx->n_generic; ++c) {
            if (ctx->model == SPIN_ISING)
                CK(launch_ising_generic(static_cast<int8_t *>(src), static_cast<int8_t *>(dst), ctx->d_generic,
                                        ctx->n_generic, ctx->generic_maxL, ctx->d_lats, ctx->d_tabs,
                                        ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, c, s));
            else
                CK(launch_potts_generic(static_cast<uint8_t *>(src), static_cast<uint8_t *>(dst), ctx->d_generic,
                                        ctx->n_generic, ctx->generic_maxL, ctx->d_lats, ctx->d_tabs,
                                        ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, w, c, s));
            ++launches;
        }
        if (ctx->mode == 3) {
            // one launch per lattice of the same kernels (the plain launch
            // form of the batched kernels: what batching the launches saves)
            for (const auto &r : ctx->per_lattice) {
                const bool timed = prof_begin(ctx, s, 2);
                if (ctx->model == SPIN_ISING) {
                    IsingSweepArgs a{(r.strip ? ctx->d_strip : ctx->d_items) + r.first, r.count, ctx->d_lats,
                                     ctx->d_tabs, static_cast<const int8_t *>(src), static_cast<int8_t *>(dst),
                                     ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, philox_keys(ctx->k0, ctx->k1), ctx->n_lat};
                    if (r.strip)
                        CK(launch_ising_strip(a, std::min((r.count + ctx->strip_warps - 1) / ctx->strip_warps,
                                                          ctx->sm_count * ctx->per_sm_strip),
                                              ctx->strip_warps, layout, s));
                    else
                        CK(launch_ising_fused(a, std::min(r.count, ctx->grid), ctx->threads, ctx->smem, s));
                } else if (r.strip) {
                    PottsStripArgs a{ctx->d_strip + r.first, r.count, ctx->d_lats, ctx->d_tabs,
                                     static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst),
                                     ctx->d_state, ctx->st.delta, ctx->st.cur, w, ctx->strip_chunks,
                                     philox_keys(ctx->k0, ctx->k1), ctx->n_lat};
                    CK(launch_potts_strip(a, std::min((r.count + ctx->strip_warps - 1) / ctx->strip_warps,
                                                      ctx->sm_count * ctx->per_sm_strip),
                                          ctx->strip_warps, ctx->strip_qbits, layout, s));
                } else {
                    PottsSweepArgs a{ctx->d_items + r.first, r.count, ctx->d_lats, ctx->d_tabs,
                                     static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst),
                                     ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, w, ctx->n_lat};
                    CK(launch_potts_fused(a, std::min(r.count, ctx->grid), ctx->threads, ctx->smem, s));
                }
                if (timed) prof_end(ctx, s);
                ++launches;
            }
            CK(launch_finalize(ctx->d_state, ctx->st, record, s));
            ++launches;
            return SPIN_OK;
        }
        // The tile kernel (small lattices) and the strip kernel (L >= 512) touch
        // disjoint lattices: fork the tile kernel onto a side stream and join
        // before the finalize kernel (also inside a captured graph).
        const bool fork = ctx->n_items && ctx->n_strip && ctx->side;
        cudaStream_t ts = s;
        if (fork) {
            CK(cudaEventRecord(ctx->ev_fork, s));
            CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
            ts = ctx->side;
        }
        if (ctx->n_items) {
            const bool timed = prof_begin(ctx, ts, 0);
            if (ctx->model == SPIN_ISING) {
                IsingSweepArgs a{ctx->d_items, ctx->n_items, ctx->d_lats, ctx->d_tabs,
                                 static_cast<const int8_t *>(src), static_cast<int8_t *>(dst),
                                 ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta,
                                 philox_keys(ctx->k0, ctx->k1), ctx->n_lat};
                CK(launch_ising_fused(a, ctx->grid, ctx->threads, ctx->smem, ts));
            } else {
                PottsSweepArgs a{ctx->d_items, ctx->n_items, ctx->d_lats, ctx->d_tabs,
                                 static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst),
                                 ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta, w, ctx->n_lat};
                CK(launch_potts_fused(a, ctx->grid, ctx->threads, ctx->smem, ts));
            }
            if (timed) prof_end(ctx, ts);
            ++launches;
        }
        if (ctx->n_strip) {
            const bool timed = prof_begin(ctx, s, 1);
            if (ctx->model == SPIN_ISING) {
                IsingSweepArgs a{ctx->d_strip, ctx->n_strip, ctx->d_lats, ctx->d_tabs,
                                 static_cast<const int8_t *>(src), static_cast<int8_t *>(dst),
                                 ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta,
                                 philox_keys(ctx->k0, ctx->k1), ctx->n_lat, src_bits, dst_bits};
                CK(launch_ising_strip(a, ctx->strip_grid, ctx->strip_warps, layout, s));
            } else {
                PottsStripArgs a{ctx->d_strip, ctx->n_strip, ctx->d_lats, ctx->d_tabs,
                                 static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst),
                                 ctx->d_state, ctx->st.delta, ctx->st.cur, w, ctx->strip_chunks,
                                 philox_keys(ctx->k0, ctx->k1), ctx->n_lat};
                CK(launch_potts_strip(a, ctx->strip_grid, ctx->strip_warps, ctx->strip_qbits, layout, s));
            }
            if (timed) prof_end(ctx, s);
            ++launches;
        }
        if (fork) {
            CK(cudaEventRecord(ctx->ev_join, ctx->side));
            CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
        }
    }
    CK(launch_finalize(ctx->d_state, ctx->st, record, s));
    ++launches;
    return SPIN_OK;
}

int launch_cpm_step(spin_ctx *ctx, int record, cudaStream_t s, int &launches) {
    for (int c = 0; c < 4; ++c) {
        CpmArgs a{static_cast<int32_t *>(ctx->spins), ctx->lat[0].L, rng_word(ctx->lat[0], 0), ctx->d_type, ctx->d_J,
                  ctx->n_types, ctx->n_cells, ctx->lambda, ctx->target, ctx->d_vol[c & 1], ctx->d_vol[(c + 1) & 1],
                  ctx->d_dvol[c & 1], ctx->d_dvol[(c + 1) & 1], ctx->d_thr, ctx->n_thr, ctx->k0, ctx->k1,
                  ctx->d_state, ctx->st.delta};
        CK(launch_cpm_substep(a, c, s));
        launches += 1;
    }
    // after colour 3, d_vol[0] holds the areas after the step
    CK(launch_cpm_finalize(ctx->d_vol[0], ctx->n_cells, ctx->target, ctx->d_state, ctx->st, record, s));
    launches += 1;
    return SPIN_OK;
}

// Record `two sweeps` (A -> B -> A for the batched form) into a graph.
// Strip lattices (Ising and Potts) stay in the strip kernels' split row form
// between the sweeps of one call (ping-pong launch forms): sweep i of n reads
// split rows if i > 0 and writes them if i < n - 1, so the buffers hold the
// interface's rows whenever a call returns.
bool split_rows(const spin_ctx *ctx) {
    return (ctx->model == SPIN_ISING || ctx->model == SPIN_POTTS) && ctx->mode != 1 && ctx->n_strip > 0;
}

int sweep_layout(const spin_ctx *ctx, int i, int n) {
    return split_rows(ctx) ? (i > 0 ? kSrcSplit : 0) | (i < n - 1 ? kDstSplit : 0) : 0;
}

// Graph of two sweeps; kind bit 0: its first sweep reads split rows, bit 1:
// its second sweep writes them (the middle of the pair is always split).
int get_graph(spin_ctx *ctx, int record, int kind, GraphCache *&out) {
    GraphCache &g = ctx->graphs[record ? 1 : 0][kind & 3];
    if (!g.exec) {
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int launches = 0, rc = SPIN_OK;
        if (ctx->model == SPIN_CPM) {
            rc = launch_cpm_step(ctx, record, ctx->cap_stream, launches);
        } else if (ctx->mode == 1) {
            rc = launch_sweep(ctx, ctx->spins, ctx->spins, record, ctx->cap_stream, launches, 0);
            if (rc == SPIN_OK) rc = launch_sweep(ctx, ctx->spins, ctx->spins, record, ctx->cap_stream, launches, 0);
        } else {
            const bool sp = split_rows(ctx);
            const int l0 = sp ? ((kind & 1) ? kSrcSplit : 0) | kDstSplit : 0;
            const int l1 = sp ? kSrcSplit | ((kind & 2) ? kDstSplit : 0) : 0;
            rc = launch_sweep(ctx, ctx->spins, ctx->spins2, record, ctx->cap_stream, launches, l0);
            if (rc == SPIN_OK) rc = launch_sweep(ctx, ctx->spins2, ctx->spins, record, ctx->cap_stream, launches, l1);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc != SPIN_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        g.launches = launches;
    }
    out = &g;
    return SPIN_OK;
}

// from_tmp (n odd, launch modes 0 and 3): the state to sweep is in the
// ping-pong buffer, so the first sweep goes from it into the caller's buffer
// and the rest pair up as usual: the call ends in the caller's buffer with no
// copy.
int run_sweeps(spin_ctx *ctx, int n, int record, cudaStream_t s, bool from_tmp = false) {
    int launches = 0;
    if (ctx->model == SPIN_CPM && ctx->mode == 2) {
        CpmPersistArgs p{};
        p.a = CpmArgs{static_cast<int32_t *>(ctx->spins), ctx->lat[0].L, rng_word(ctx->lat[0], 0), ctx->d_type, ctx->d_J, ctx->n_types,
                      ctx->n_cells, ctx->lambda, ctx->target, nullptr, nullptr, nullptr, nullptr, ctx->d_thr,
                      ctx->n_thr, ctx->k0, ctx->k1, ctx->d_state, ctx->st.delta};
        p.vol[0] = ctx->d_vol[0];
        p.vol[1] = ctx->d_vol[1];
        p.dvol[0] = ctx->d_dvol[0];
        p.dvol[1] = ctx->d_dvol[1];
        p.n_steps = n;
        p.t0 = ctx->t;
        p.rec0 = (long long)ctx->n_rec;
        p.record = record;
        p.st = ctx->st;
        p.acc = ctx->d_cpm_acc;
        p.bar = ctx->d_cpm_bar;
        p.err = ctx->d_flag + 1;
        CK(launch_cpm_persistent(p, ctx->cpm_grid, ctx->d_state, s));
        ctx->last_launches = 2;
        return SPIN_OK;
    }
    if (ctx->mode == 2) {
        ResidentArgs a{static_cast<int8_t *>(ctx->spins), ctx->d_lats, ctx->d_tabs, ctx->k0, ctx->k1,
                       ctx->t, n, (long long)ctx->n_rec, record, ctx->st, philox_keys(ctx->k0, ctx->k1)};
        if (ctx->n_nnn == ctx->n_lat)
            CK(launch_ising_nnn_resident(a, ctx->d_nnn_thr, ctx->n_lat, (size_t)ctx->maxL * ctx->maxL,
                                         ctx->d_state, s));
        else if (ctx->n_tri == ctx->n_lat)
            CK(launch_ising_tri_resident(a, ctx->n_lat, (size_t)ctx->maxL * ctx->maxL, ctx->d_state, s));
        else if (ctx->cluster > 1)
            CK(launch_ising_resident_cluster(a, ctx->n_lat, ctx->threads, ctx->cluster, ctx->maxL, ctx->d_state, s));
        else
            CK(launch_ising_resident(a, ctx->n_lat, ctx->threads, (size_t)ctx->maxL * ctx->maxL,
                                     ctx->d_state, s));
        ctx->last_launches = 2;
        return SPIN_OK;
    }
    if (ctx->model == SPIN_CPM) {
        int i = 0;
        if (ctx->use_graph && !ctx->prof && n >= 1) {
            GraphCache *g = nullptr;
            int rc = get_graph(ctx, record, 0, g);
            if (rc) return rc;
            for (; i < n; ++i) {
                CK(cudaGraphLaunch(g->exec, s));
                launches += g->launches;
            }
        }
        for (; i < n; ++i) {
            int rc = launch_cpm_step(ctx, record, s, launches);
            if (rc) return rc;
        }
        ctx->last_launches = launches;
        return SPIN_OK;
    }
    int i = 0;
    if (from_tmp) {
        int rc = launch_sweep(ctx, ctx->spins2, ctx->spins, record, s, launches, sweep_layout(ctx, 0, n));
        if (rc) return rc;
        i = 1;
    }
    if (ctx->use_graph && !ctx->prof && n >= 2) {
        const bool sp = split_rows(ctx);
        for (; i + 1 < n; i += 2) {
            GraphCache *g = nullptr;
            int rc = get_graph(ctx, record, sp ? (i > 0 ? 1 : 0) | (i + 2 < n ? 2 : 0) : 0, g);
            if (rc) return rc;
            CK(cudaGraphLaunch(g->exec, s));
            launches += g->launches;
        }
    }
    for (; i < n; ++i) {
        const bool even = ((i + (from_tmp ? 1 : 0)) & 1) == 0;
        void *src = ctx->mode == 1 ? ctx->spins : (even ? ctx->spins : ctx->spins2);
        void *dst = ctx->mode == 1 ? ctx->spins : (even ? ctx->spins2 : ctx->spins);
        int rc = launch_sweep(ctx, src, dst, record, s, launches, sweep_layout(ctx, i, n));
        if (rc) return rc;
    }
    if (ctx->mode != 1 && (n & 1) && !from_tmp) {
        CK(launch_copy_lattices(ctx->spins2, ctx->spins, ctx->d_lats, ctx->n_lat, (int)ctx->elem, s));
        ++launches;
    }
    ctx->last_launches = launches;
    return SPIN_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ensure_scratch(spin_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->scratch_bytes) return SPIN_OK;
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    ctx->d_scratch = nullptr;
    ctx->scratch_bytes = 0;
    CK(cudaMalloc(&ctx->d_scratch, bytes));
    ctx->scratch_bytes = bytes;
    return SPIN_OK;
}

int check_records(spin_ctx *ctx, int64_t first, int32_t n) {
    if (n < 0 || first < 0) return fail(ctx, SPIN_EINVAL, "negative record range");
    if (first + n > ctx->n_rec) return fail(ctx, SPIN_EINVAL, "records beyond the last recorded sweep");
    if (first < ctx->n_rec - ctx->st.cap) return fail(ctx, SPIN_EINVAL, "records already overwritten in the ring");
    return SPIN_OK;
}

std::string shape_key(const spin_ctx *ctx) {
    std::ostringstream o;
    o << "m" << ctx->model << "_n" << ctx->n_lat;
    uint64_t h = 1469598103934665603ull;
    for (auto &d : ctx->lat) {
        h ^= (uint64_t)d.L * 1315423911u + (uint64_t)d.q + ((uint64_t)d.geometry << 40);
        h *= 1099511628211ull;
    }
    o << "_h" << std::hex << h;
    return o.str();
}

}  // namespace

namespace spinmc {
// Acceptance table of one Ising lattice, for the allocation-free entry point.
void build_ising_table(const spin_lattice_desc &d, TabEntry *out) { ising_table(d, out); }
}  // namespace spinmc

extern "C" {

int spin_version(void) { return 2; }

const char *spin_last_error(const spin_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int spin_stats_width(const spin_ctx *ctx) { return ctx ? ctx->width : SPIN_EINVAL; }

int64_t spin_num_records(const spin_ctx *ctx) { return ctx ? ctx->n_rec : SPIN_EINVAL; }

uint32_t spin_sweep_index(const spin_ctx *ctx) { return ctx ? ctx->t : 0u; }

int32_t spin_gpu_launches(const spin_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

int spin_num_moments(const spin_ctx *ctx) {
    if (!ctx) return SPIN_EINVAL;
    const int w = ctx->width;
    return 1 + w + w * (w + 1) / 2;
}

int spin_num_grad(const spin_ctx *ctx) {
    if (!ctx) return SPIN_EINVAL;
    return ctx->model == SPIN_ISING ? ctx->width : (ctx->model == SPIN_CPM ? ctx->width : SPIN_EINVAL);
}

void spin_destroy(spin_ctx *ctx) {
    if (!ctx) return;
    drop_graphs(ctx);
    void *bufs[] = {ctx->spins2, ctx->d_lats, ctx->d_tabs, ctx->d_items, ctx->d_strip, ctx->d_generic, ctx->d_tri,
                    ctx->d_nnn_thr,
                    ctx->d_dvol[0], ctx->d_dvol[1],
                    ctx->d_state, ctx->st.cur, ctx->st.delta, ctx->st.ring, ctx->d_type,
                    ctx->d_J, ctx->d_vol[0], ctx->d_vol[1], ctx->d_thr, ctx->d_latp,
                    ctx->d_cpmJ, ctx->d_scratch, ctx->d_flag, ctx->d_cpm_acc, ctx->d_cpm_bar, ctx->d_packed, ctx->d_packed2,
                    ctx->d_blk_all, ctx->d_blk_small};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    delete ctx;
}

int spin_init(spin_ctx **out, int32_t model, uint64_t seed, int32_t n_lattices,
              const spin_lattice_desc *lat, const spin_cpm_params *cpm, void *d_spins,
              int32_t init_mode, int32_t max_record_sweeps, void *stream) {
    Range range_("spin_init");
    if (!out) return SPIN_EINVAL;
    *out = nullptr;
    spin_ctx *ctx = new spin_ctx();
    auto bail = [&](int rc) {
        spin_destroy(ctx);
        return rc;
    };
    int rc = validate(ctx, model, n_lattices, lat, cpm);
    if (rc) {
        fprintf(stderr, "spin_init: %s\n", ctx->err.c_str());
        return bail(rc);
    }
    if (!d_spins) return bail(SPIN_EINVAL);
    if (!is_device_ptr(d_spins)) return bail(SPIN_EINVAL);
    const bool mode_ok = model == SPIN_CPM ? (init_mode == 1 || init_mode == 2)
                                           : (init_mode == 0 || init_mode == 1);
    if (!mode_ok) return bail(fail(ctx, SPIN_EINVAL, "init_mode not valid for this model"));
    if (max_record_sweeps < 0) return bail(SPIN_EINVAL);
    cudaStream_t s = S(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bail(SPIN_ECUDA);
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev);
    ctx->model = model;
    ctx->seed = seed;
    ctx->k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    ctx->k1 = (uint32_t)(seed >> 32);
    ctx->n_lat = n_lattices;
    ctx->lat.assign(lat, lat + n_lattices);
    ctx->elem = model == SPIN_CPM ? 4 : 1;
    ctx->spins = d_spins;
    if (cpm) {
        ctx->n_types = cpm->n_types;
        ctx->lambda = cpm->lambda;
        ctx->target = cpm->target_area;
        ctx->n_cells = cpm->n_cells;
        ctx->T = cpm->T;
        ctx->init_side = cpm->init_side;
        ctx->init_cols = cpm->init_cols;
        ctx->Jt.assign(cpm->J_type, cpm->J_type + cpm->n_types * cpm->n_types);
    }
    ctx->width = stats_width(model, ctx->lat, ctx->n_types);
    std::vector<LatDev> ld(n_lattices);
    std::vector<int32_t> generic, tri;
    ctx->n_nnn = 0;
    for (int i = 0; i < n_lattices; ++i) {
        const auto &d = ctx->lat[i];
        const int geom = model == SPIN_CPM ? 0 : d.geometry;
        ld[i] = LatDev{d.spin_offset, d.L, model == SPIN_POTTS ? d.q : 2,
                       (geom == 0 && d.L % 16 == 0 && d.spin_offset % 16 == 0) ? 1 : 0, geom, rng_word(d, i), 0};
        ctx->maxL = std::max(ctx->maxL, d.L);
        ctx->span_elems = std::max<size_t>(ctx->span_elems, d.spin_offset + (size_t)d.L * d.L);
        if (geom == 2) {
            ++ctx->n_nnn;
            ctx->nnn_maxL = std::max(ctx->nnn_maxL, d.L);
        } else if (geom == 1) {
            tri.push_back(i);
            ctx->tri_maxL = std::max(ctx->tri_maxL, d.L);
        } else if (ld[i].fast)
            ctx->fast_ids.push_back(i);
        else {
            generic.push_back(i);
            ctx->generic_maxL = std::max(ctx->generic_maxL, d.L);
        }
    }
    ctx->n_generic = (int)generic.size();
    ctx->n_tri = (int)tri.size();
    auto ckm = [&](cudaError_t e) { return e == cudaSuccess; };
    const size_t w = (size_t)ctx->width;
    if (!ckm(cudaMalloc(&ctx->d_lats, sizeof(LatDev) * n_lattices)) ||
        !ckm(cudaMalloc(&ctx->d_tabs, sizeof(TabEntry) * kTabStride * n_lattices)) ||
        !ckm(cudaMalloc(&ctx->d_state, sizeof(DevState))) ||
        !ckm(cudaMalloc(&ctx->st.cur, sizeof(int64_t) * w * n_lattices)) ||
        !ckm(cudaMalloc(&ctx->st.delta, sizeof(int64_t) * w * n_lattices)) ||
        !ckm(cudaMalloc(&ctx->d_latp, sizeof(double) * kLatParams * n_lattices)) ||
        !ckm(cudaMalloc(&ctx->d_cpmJ, sizeof(double) * 64)) ||
        !ckm(cudaMalloc(&ctx->d_flag, 2 * sizeof(int))) || !ckm(cudaMemset(ctx->d_flag, 0, 2 * sizeof(int))) ||
        (max_record_sweeps > 0 &&
         !ckm(cudaMalloc(&ctx->st.ring, sizeof(int64_t) * w * n_lattices * (size_t)max_record_sweeps))))
        return bail(fail(ctx, SPIN_ENOMEM, "device allocation failed"));
    if (model != SPIN_CPM && !ckm(cudaMalloc(&ctx->spins2, ctx->span_elems * ctx->elem)))
        return bail(fail(ctx, SPIN_ENOMEM, "device allocation of the second spin buffer failed"));
    if (ctx->n_generic) {
        if (!ckm(cudaMalloc(&ctx->d_generic, sizeof(int32_t) * ctx->n_generic)))
            return bail(SPIN_ENOMEM);
        if (!ckm(cudaMemcpy(ctx->d_generic, generic.data(), sizeof(int32_t) * generic.size(), cudaMemcpyHostToDevice)))
            return bail(SPIN_ECUDA);
    }
    if (ctx->n_nnn && !ckm(cudaMalloc(&ctx->d_nnn_thr, sizeof(uint32_t) * kNnnTab * n_lattices)))
        return bail(SPIN_ENOMEM);
    if (ctx->n_tri) {
        if (!ckm(cudaMalloc(&ctx->d_tri, sizeof(int32_t) * ctx->n_tri))) return bail(SPIN_ENOMEM);
        if (!ckm(cudaMemcpy(ctx->d_tri, tri.data(), sizeof(int32_t) * tri.size(), cudaMemcpyHostToDevice)))
            return bail(SPIN_ECUDA);
    }
    ctx->st.cap = max_record_sweeps;
    ctx->st.width = ctx->width;
    ctx->st.n_lat = n_lattices;
    if (cudaMemcpy(ctx->d_lats, ld.data(), sizeof(LatDev) * n_lattices, cudaMemcpyHostToDevice))
        return bail(SPIN_ECUDA);
    DevState ds{0u, 0, 0};
    if (!ckm(cudaMemset(ctx->st.delta, 0, sizeof(int64_t) * w * n_lattices)) ||
        !ckm(cudaMemcpy(ctx->d_state, &ds, sizeof ds, cudaMemcpyHostToDevice)))
        return bail(SPIN_ECUDA);
    if (model == SPIN_CPM) {
        const int nc = ctx->n_cells;
        if (!ckm(cudaMalloc(&ctx->d_type, nc + 1)) || !ckm(cudaMalloc(&ctx->d_J, sizeof(int32_t) * 64)) ||
            !ckm(cudaMalloc(&ctx->d_vol[0], sizeof(int32_t) * (nc + 1))) ||
            !ckm(cudaMalloc(&ctx->d_vol[1], sizeof(int32_t) * (nc + 1))) ||
            !ckm(cudaMalloc(&ctx->d_dvol[0], sizeof(int32_t) * (nc + 1))) ||
            !ckm(cudaMalloc(&ctx->d_dvol[1], sizeof(int32_t) * (nc + 1))) ||
            !ckm(cudaMalloc(&ctx->d_cpm_acc, sizeof(int64_t) * 2 * kCpmAccStride)) ||
            !ckm(cudaMemset(ctx->d_cpm_acc, 0, sizeof(int64_t) * 2 * kCpmAccStride)) ||
            !ckm(cudaMalloc(&ctx->d_cpm_bar, 2 * sizeof(unsigned int))))
            return bail(SPIN_ENOMEM);
        // the persistent form (one cooperative launch per call): launch mode 2
        ctx->cpm_grid = cpm_persistent_grid();
    }
    rc = upload_tables(ctx, s);
    if (rc) return bail(rc);
    // initial state
    cudaError_t e = cudaSuccess;
    if (init_mode == 0) {
        e = launch_init_random(d_spins, model, ctx->d_lats, n_lattices, ctx->maxL, ctx->k0, ctx->k1, s);
    } else if (init_mode == 2) {
        const int L = ctx->lat[0].L;
        const int rows = (ctx->n_cells + std::max(1, ctx->init_cols) - 1) / std::max(1, ctx->init_cols);
        if (ctx->init_side < 1 || ctx->init_cols < 1 || ctx->init_cols * ctx->init_side > L ||
            rows * ctx->init_side > L)
            return bail(fail(ctx, SPIN_EINVAL, "initial cell block does not fit the lattice"));
        e = launch_cpm_init_squares(static_cast<int32_t *>(d_spins) + ctx->lat[0].spin_offset, L,
                                    ctx->n_cells, ctx->init_side, ctx->init_cols, s);
    }
    if (e) return bail(cuda_fail(ctx, e, "init"));
    if (model == SPIN_CPM) {
        if (cpm->cell_type) {
            e = cudaMemcpyAsync(ctx->d_type, cpm->cell_type, ctx->n_cells + 1, cudaMemcpyHostToDevice, s);
            if (e) return bail(cuda_fail(ctx, e, "cell types"));
        } else {
            e = launch_cpm_types(ctx->d_type, ctx->n_cells, rng_word(ctx->lat[0], 0), ctx->k0, ctx->k1, s);
            if (e) return bail(cuda_fail(ctx, e, "cpm types"));
        }
        // the CPM kernels address the lattice at offset 0 of the buffer
        ctx->spins = static_cast<int32_t *>(d_spins) + ctx->lat[0].spin_offset;
        const size_t vb = sizeof(int32_t) * (ctx->n_cells + 1);
        e = cudaMemsetAsync(ctx->d_vol[0], 0, vb, s);
        if (!e) e = launch_cpm_volumes(static_cast<int32_t *>(ctx->spins), ctx->lat[0].L, ctx->d_vol[0], ctx->n_cells, s);
        if (!e) e = cudaMemcpyAsync(ctx->d_vol[1], ctx->d_vol[0], vb, cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaMemsetAsync(ctx->d_dvol[0], 0, vb, s);
        if (!e) e = cudaMemsetAsync(ctx->d_dvol[1], 0, vb, s);
        if (e) return bail(cuda_fail(ctx, e, "cpm areas"));
    }
    if (model != SPIN_CPM) {
        // keep the bytes outside the lattices identical in both buffers
        e = cudaMemcpyAsync(ctx->spins2, d_spins, ctx->span_elems * ctx->elem, cudaMemcpyDeviceToDevice, s);
        if (e) return bail(cuda_fail(ctx, e, "copy"));
    }
    e = launch_stats_from_state(ctx->spins, model, ctx->d_lats, n_lattices, ctx->maxL, ctx->width,
                                ctx->d_type, ctx->n_types, ctx->d_vol[0], ctx->n_cells, ctx->target,
                                ctx->st.cur, s);
    if (e) return bail(cuda_fail(ctx, e, "initial statistics"));
    // CPM statistics read the single lattice at offset 0 of ctx->spins
    if (model == SPIN_ISING &&
        (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess))
        return bail(fail(ctx, SPIN_ECUDA, "stream or event creation failed"));
    rc = plan(ctx);
    if (rc) return bail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(SPIN_ECUDA);
    *out = ctx;
    return SPIN_OK;
}

int spin_sweep(spin_ctx *ctx, int32_t n_sweeps, int32_t record, void *stream) {
    Range range_("spin_sweep");
    if (!ctx) return SPIN_EINVAL;
    if (n_sweeps < 0) return fail(ctx, SPIN_EINVAL, "negative sweep count");
    if ((uint64_t)ctx->t + (uint64_t)n_sweeps >= 0xFFFFFFFEull)
        return fail(ctx, SPIN_ESTATE, "sweep counter would reach the values reserved for initialisation");
    if (record && ctx->st.cap <= 0) return fail(ctx, SPIN_ESTATE, "no record ring (max_record_sweeps = 0)");
    if (n_sweeps == 0) return SPIN_OK;
    int rc = run_sweeps(ctx, n_sweeps, record ? 1 : 0, S(stream));
    if (rc) return rc;
    ctx->t += (uint32_t)n_sweeps;
    if (record) ctx->n_rec += n_sweeps;
    return SPIN_OK;
}

int spin_observables(spin_ctx *ctx, int64_t first, int32_t n, int64_t *stats, float *E, float *M,
                     void *stream) {
    Range range_("spin_observables");
    if (!ctx) return SPIN_EINVAL;
    int rc = check_records(ctx, first, n);
    if (rc) return rc;
    if (n == 0) return SPIN_OK;
    cudaStream_t s = S(stream);
    const size_t ns = (size_t)n * ctx->n_lat * ctx->width, nf = (size_t)n * ctx->n_lat;
    const bool dev_s = !stats || is_device_ptr(stats), dev_e = !E || is_device_ptr(E),
               dev_m = !M || is_device_ptr(M);
    rc = ensure_scratch(ctx, sizeof(int64_t) * ns + 2 * sizeof(float) * nf + 64);
    if (rc) return rc;
    int64_t *ts = dev_s ? stats : static_cast<int64_t *>(ctx->d_scratch);
    float *te = dev_e ? E : reinterpret_cast<float *>(static_cast<char *>(ctx->d_scratch) + sizeof(int64_t) * ns);
    float *tm = dev_m ? M : te + nf;
    ObsParams p{ctx->model, ctx->n_lat, ctx->width, ctx->d_latp, ctx->d_cpmJ, (double)ctx->lambda};
    CK(launch_observables(ctx->st, first, n, p, ts, te, tm, s));
    if (!dev_s) CK(cudaMemcpyAsync(stats, ts, sizeof(int64_t) * ns, cudaMemcpyDeviceToHost, s));
    if (!dev_e) CK(cudaMemcpyAsync(E, te, sizeof(float) * nf, cudaMemcpyDeviceToHost, s));
    if (!dev_m) CK(cudaMemcpyAsync(M, tm, sizeof(float) * nf, cudaMemcpyDeviceToHost, s));
    if (!dev_s || !dev_e || !dev_m) {
        int timed_out = 0;
        CK(cudaMemcpyAsync(&timed_out, ctx->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (timed_out) return fail(ctx, SPIN_ETIMEOUT, "a device-side wait of a sweep gave up");
    }
    return SPIN_OK;
}

int spin_current_stats(spin_ctx *ctx, int64_t *stats, void *stream) {
    if (!ctx || !stats) return SPIN_EINVAL;
    cudaStream_t s = S(stream);
    const size_t ns = (size_t)ctx->n_lat * ctx->width;
    const bool dev = is_device_ptr(stats);
    int rc = ensure_scratch(ctx, sizeof(int64_t) * ns);
    if (rc) return rc;
    int64_t *t = dev ? stats : static_cast<int64_t *>(ctx->d_scratch);
    CK(launch_stats_from_state(ctx->spins, ctx->model, ctx->d_lats, ctx->n_lat, ctx->maxL, ctx->width,
                               ctx->d_type, ctx->n_types, ctx->d_vol[0], ctx->n_cells, ctx->target, t, s));
    if (!dev) {
        CK(cudaMemcpyAsync(stats, t, sizeof(int64_t) * ns, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return SPIN_OK;
}

int spin_moments(spin_ctx *ctx, int64_t first, int32_t n, int64_t *moments, void *stream) {
    Range range_("spin_moments");
    if (!ctx || !moments) return SPIN_EINVAL;
    int rc = check_records(ctx, first, n);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const int nm = spin_num_moments(ctx);
    const size_t cnt = (size_t)nm * ctx->n_lat;
    rc = ensure_scratch(ctx, 16 * cnt + sizeof(int64_t) * cnt + 64);
    if (rc) return rc;
    CK(launch_moments_i128(ctx->st, first, n, ctx->d_scratch, s));
    const bool dev = is_device_ptr(moments);
    int64_t *t = dev ? moments : reinterpret_cast<int64_t *>(static_cast<char *>(ctx->d_scratch) + 16 * cnt);
    CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    CK(launch_i128_to_i64(ctx->d_scratch, t, (int)cnt, ctx->d_flag, s));
    int flag[2] = {0, 0};
    CK(cudaMemcpyAsync(flag, ctx->d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (!dev) CK(cudaMemcpyAsync(moments, t, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flag[1]) return fail(ctx, SPIN_ETIMEOUT, "a device-side wait of a sweep gave up");
    if (flag[0]) return fail(ctx, SPIN_EINVAL, "a moment does not fit in int64");
    return SPIN_OK;
}

int spin_grad(spin_ctx *ctx, int64_t first, int32_t n, int32_t observable, int32_t pool, double *out,
              void *stream) {
    Range range_("spin_grad");
    if (!ctx || !out) return SPIN_EINVAL;
    if (ctx->model == SPIN_POTTS) return fail(ctx, SPIN_EINVAL, "no gradient for the Potts model");
    if (ctx->model == SPIN_ISING && (observable < 0 || observable > 1))
        return fail(ctx, SPIN_EINVAL, "Ising observable must be 0 (E/N) or 1 (M/N)");
    if (ctx->model == SPIN_CPM && observable != 0) return fail(ctx, SPIN_EINVAL, "CPM observable must be 0");
    int rc = check_records(ctx, first, n);
    if (rc) return rc;
    if (n < 2) return fail(ctx, SPIN_EINVAL, "need at least two records");
    cudaStream_t s = S(stream);
    const int nm = spin_num_moments(ctx);
    const size_t cnt = (size_t)nm * ctx->n_lat;
    const int rows = pool ? 1 : ctx->n_lat;
    const int ng = spin_num_grad(ctx);
    rc = ensure_scratch(ctx, 16 * cnt + 16 * (size_t)nm + sizeof(double) * rows * ng + 64);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->d_scratch);
    CK(launch_moments_i128(ctx->st, first, n, base, s));
    const void *mom = base;
    if (pool) {
        CK(launch_pool_moments(base, ctx->n_lat, nm, base + 16 * cnt, s));
        mom = base + 16 * cnt;
    }
    GradParams p{ctx->model, ctx->n_lat, ctx->width, observable, pool ? 1 : 0, ctx->d_latp,
                 ctx->d_cpmJ, (double)ctx->lambda, (double)ctx->T, ctx->width - 2};
    const bool dev = is_device_ptr(out);
    double *t = dev ? out : reinterpret_cast<double *>(base + 16 * cnt + 16 * (size_t)nm);
    CK(launch_grad_i128(mom, rows, p, t, s));
    if (!dev) {
        CK(cudaMemcpyAsync(out, t, sizeof(double) * rows * ng, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return SPIN_OK;
}

int spin_pooled_limbs(spin_ctx *ctx, int64_t first, int32_t n, int64_t *limbs, void *stream) {
    if (!ctx || !limbs) return SPIN_EINVAL;
    if (ctx->model == SPIN_POTTS) return fail(ctx, SPIN_EINVAL, "no gradient for the Potts model");
    int rc = check_records(ctx, first, n);
    if (rc) return rc;
    if (n < 1) return fail(ctx, SPIN_EINVAL, "need at least one record");
    if (!is_device_ptr(limbs)) return fail(ctx, SPIN_EINVAL, "limbs must be device memory");
    cudaStream_t s = S(stream);
    const int nm = spin_num_moments(ctx);
    const size_t cnt = (size_t)nm * ctx->n_lat;
    rc = ensure_scratch(ctx, 16 * cnt + 16 * (size_t)nm + 64);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->d_scratch);
    CK(launch_moments_i128(ctx->st, first, n, base, s));
    CK(launch_pool_moments(base, ctx->n_lat, nm, base + 16 * cnt, s));
    CK(launch_i128_to_limbs(base + 16 * cnt, nm, limbs, s));
    return SPIN_OK;
}

int spin_grad_from_limbs(spin_ctx *ctx, const int64_t *limbs, int32_t observable, double *grad, double *expect,
                         void *stream) {
    if (!ctx || !limbs || (!grad && !expect)) return SPIN_EINVAL;
    if (ctx->model == SPIN_POTTS) return fail(ctx, SPIN_EINVAL, "no gradient for the Potts model");
    if (ctx->model == SPIN_ISING && (observable < 0 || observable > 1))
        return fail(ctx, SPIN_EINVAL, "Ising observable must be 0 (E/N) or 1 (M/N)");
    if (ctx->model == SPIN_CPM && observable != 0) return fail(ctx, SPIN_EINVAL, "CPM observable must be 0");
    if (!is_device_ptr(limbs) || (grad && !is_device_ptr(grad)) || (expect && !is_device_ptr(expect)))
        return fail(ctx, SPIN_EINVAL, "limbs and outputs must be device memory");
    cudaStream_t s = S(stream);
    const int nm = spin_num_moments(ctx);
    int rc = ensure_scratch(ctx, 16 * (size_t)nm + 64);
    if (rc) return rc;
    CK(launch_limbs_to_i128(limbs, nm, ctx->d_scratch, s));
    GradParams p{ctx->model, ctx->n_lat, ctx->width, observable, 1, ctx->d_latp, ctx->d_cpmJ, (double)ctx->lambda,
                 (double)ctx->T, ctx->width - 2};
    if (grad) CK(launch_grad_i128(ctx->d_scratch, 1, p, grad, s));
    if (expect) CK(launch_expectations_i128(ctx->d_scratch, 1, p, expect, s));
    return SPIN_OK;
}

int spin_expectations(spin_ctx *ctx, int64_t first, int32_t n, int32_t pool, double *out, void *stream) {
    if (!ctx || !out) return SPIN_EINVAL;
    if (ctx->model == SPIN_POTTS) return fail(ctx, SPIN_EINVAL, "use spin_observables for the Potts model");
    int rc = check_records(ctx, first, n);
    if (rc) return rc;
    if (n < 1) return fail(ctx, SPIN_EINVAL, "need at least one record");
    cudaStream_t s = S(stream);
    const int nm = spin_num_moments(ctx);
    const size_t cnt = (size_t)nm * ctx->n_lat;
    const int rows = pool ? 1 : ctx->n_lat;
    rc = ensure_scratch(ctx, 16 * cnt + 16 * (size_t)nm + sizeof(double) * rows * 2 + 64);
    if (rc) return rc;
    char *base = static_cast<char *>(ctx->d_scratch);
    CK(launch_moments_i128(ctx->st, first, n, base, s));
    const void *mom = base;
    if (pool) {
        CK(launch_pool_moments(base, ctx->n_lat, nm, base + 16 * cnt, s));
        mom = base + 16 * cnt;
    }
    GradParams p{ctx->model, ctx->n_lat, ctx->width, 0, pool ? 1 : 0, ctx->d_latp,
                 ctx->d_cpmJ, (double)ctx->lambda, (double)ctx->T, ctx->width - 2};
    const bool dev = is_device_ptr(out);
    double *t = dev ? out : reinterpret_cast<double *>(base + 16 * cnt + 16 * (size_t)nm);
    CK(launch_expectations_i128(mom, rows, p, t, s));
    if (!dev) {
        CK(cudaMemcpyAsync(out, t, sizeof(double) * rows * 2, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return SPIN_OK;
}

int spin_set_params(spin_ctx *ctx, const spin_lattice_desc *lat, const spin_cpm_params *cpm) {
    if (!ctx) return SPIN_EINVAL;
    if (lat) {
        if (ctx->model == SPIN_CPM) return fail(ctx, SPIN_EINVAL, "CPM contexts take only cpm parameters");
        int rc = validate(ctx, ctx->model, ctx->n_lat, lat, nullptr);
        if (rc) return rc;
        for (int i = 0; i < ctx->n_lat; ++i)
            if (lat[i].L != ctx->lat[i].L || lat[i].q != ctx->lat[i].q ||
                lat[i].spin_offset != ctx->lat[i].spin_offset || lat[i].geometry != ctx->lat[i].geometry ||
                lat[i].lattice_id != ctx->lat[i].lattice_id)
                return fail(ctx, SPIN_EINVAL, "spin_set_params may not change L, q, geometry, lattice_id or offsets");
        ctx->lat.assign(lat, lat + ctx->n_lat);
    }
    if (cpm) {
        if (ctx->model != SPIN_CPM) return fail(ctx, SPIN_EINVAL, "not a CPM context");
        for (int a = 0; a < cpm->n_types && cpm->J_type; ++a)
            for (int b = 0; b < cpm->n_types; ++b)
                if (cpm->J_type[a * cpm->n_types + b] != cpm->J_type[b * cpm->n_types + a])
                    return fail(ctx, SPIN_EINVAL, "CPM J table must be symmetric");
        if (!cpm->J_type || cpm->lambda < 0 || cpm->target_area < 0)
            return fail(ctx, SPIN_EINVAL, "bad CPM parameters");
        if (cpm->n_types != ctx->n_types || cpm->n_cells != ctx->n_cells)
            return fail(ctx, SPIN_EINVAL, "spin_set_params may not change n_types or n_cells");
        if (!(cpm->T > 0.0f)) return fail(ctx, SPIN_EINVAL, "CPM T must be > 0");
        ctx->Jt.assign(cpm->J_type, cpm->J_type + ctx->n_types * ctx->n_types);
        ctx->lambda = cpm->lambda;
        ctx->target = cpm->target_area;
        ctx->T = cpm->T;
        drop_graphs(ctx);  // lambda / A are kernel arguments
    }
    CK(cudaDeviceSynchronize());
    return upload_tables(ctx, nullptr);
}

static bool resident_ok(const spin_ctx *ctx) {
    if (ctx->model == SPIN_CPM) return ctx->cpm_grid > 0;   // the persistent cooperative form
    if (ctx->model != SPIN_ISING || ctx->n_generic) return false;
    if (ctx->n_nnn) {   // first and second neighbours (a context holds only these)
        for (const auto &d : ctx->lat)
            if (d.L > 256) return false;
        return true;
    }
    if (ctx->n_tri) {   // all triangular: the triangular resident kernel
        if (ctx->n_tri != ctx->n_lat) return false;
        for (const auto &d : ctx->lat)
            if (d.L > 240) return false;
        return true;
    }
    for (const auto &d : ctx->lat)
        if (d.L > 256) return false;
    return true;
}

int spin_set_launch(spin_ctx *ctx, int32_t mode, int32_t use_graph, int32_t tile_rows, int32_t threads) {
    if (!ctx) return SPIN_EINVAL;
    if (mode < 0 || mode > 3) return fail(ctx, SPIN_EINVAL, "launch mode must be 0, 1, 2 or 3");
    if (mode == 3 && ctx->model == SPIN_CPM) return fail(ctx, SPIN_EINVAL, "mode 3 is for Ising and Potts contexts");
    if (mode == 2 && !resident_ok(ctx))
        return fail(ctx, SPIN_EINVAL, "resident form needs Ising lattices with L % 16 == 0 and L <= 256, "
                                      "only triangular lattices with L <= 240, only second-neighbour "
                                      "lattices with L <= 256, or a CPM context on a device with "
                                      "cooperative launch");
    if (threads != 0 && threads != 128 && threads != 256 && threads != 512 && !(threads == 1024 && mode == 2))
        return fail(ctx, SPIN_EINVAL, "threads must be 128, 256 or 512 (or 1024 in the resident form)");
    if (tile_rows < -1) return fail(ctx, SPIN_EINVAL, "tile_rows must be >= -1");
    int cluster = ctx->cluster;
    if (mode == 2) {   // tile_rows: CTAs per lattice (cluster size) of the square-lattice resident form
        if (tile_rows == -1 || tile_rows == 1) cluster = 1;
        else if (tile_rows > 0) cluster = tile_rows;
        if (cluster != 1 && cluster != 2 && cluster != 4)
            return fail(ctx, SPIN_EINVAL, "the resident form takes 1, 2 or 4 CTAs per lattice");
        const int th = threads ? threads : ctx->threads;
        if (cluster > 1 && (ctx->model != SPIN_ISING || ctx->n_nnn || ctx->n_tri || th < 256))
            return fail(ctx, SPIN_EINVAL, "a cluster per lattice needs square Ising lattices and 256, 512 or "
                                          "1024 threads");
    }
    ctx->mode = mode;
    ctx->use_graph = use_graph ? 1 : 0;
    if (mode == 2) ctx->cluster = cluster;
    else if (tile_rows > 0) ctx->tile_rows = tile_rows;
    else if (tile_rows == -1) ctx->tile_rows = 0;
    if (threads) ctx->threads = threads;
    if (ctx->mode != 2 && ctx->threads > 512) ctx->threads = 512;   // 1024 exists in the resident form only
    return plan(ctx);
}

int spin_get_launch(const spin_ctx *ctx, int32_t out[4]) {
    if (!ctx || !out) return SPIN_EINVAL;
    out[0] = ctx->mode;
    out[1] = ctx->use_graph;
    out[2] = ctx->mode == 2 ? (ctx->cluster > 1 ? ctx->cluster : 0) : ctx->tile_rows;
    out[3] = ctx->threads;
    return SPIN_OK;
}

int spin_load_spins(spin_ctx *ctx, const void *host, void *stream) {
    Range range_("spin_load_spins");
    if (!ctx || !host) return SPIN_EINVAL;
    char *base = static_cast<char *>(ctx->spins);
    cudaStream_t s = S(stream);
    if (ctx->model == SPIN_CPM) {
        CK(cudaMemcpyAsync(base, host, (size_t)ctx->lat[0].L * ctx->lat[0].L * 4, cudaMemcpyHostToDevice, s));
        // the areas and the running statistics follow the loaded state
        const size_t vb = sizeof(int32_t) * (ctx->n_cells + 1);
        CK(cudaMemsetAsync(ctx->d_vol[0], 0, vb, s));
        CK(launch_cpm_volumes(static_cast<int32_t *>(ctx->spins), ctx->lat[0].L, ctx->d_vol[0], ctx->n_cells, s));
        CK(cudaMemcpyAsync(ctx->d_vol[1], ctx->d_vol[0], vb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ctx->d_dvol[0], 0, vb, s));
        CK(cudaMemsetAsync(ctx->d_dvol[1], 0, vb, s));
    } else {
        CK(cudaMemcpyAsync(base, host, ctx->span_elems * ctx->elem, cudaMemcpyHostToDevice, s));
    }
    CK(launch_stats_from_state(ctx->spins, ctx->model, ctx->d_lats, ctx->n_lat, ctx->maxL, ctx->width, ctx->d_type,
                               ctx->n_types, ctx->d_vol[0], ctx->n_cells, ctx->target, ctx->st.cur, s));
    return SPIN_OK;
}

int32_t spin_packed_words(const spin_ctx *ctx) {
    if (!ctx || ctx->model != SPIN_ISING) return SPIN_EINVAL;
    return (int32_t)((ctx->span_elems + 31) / 32);
}

static int packed_ready(spin_ctx *ctx) {
    if (ctx->model != SPIN_ISING) return fail(ctx, SPIN_EINVAL, "bit-packed transfer is for Ising contexts");
    for (const auto &d : ctx->lat)
        if (d.spin_offset % 32) return fail(ctx, SPIN_EINVAL, "bit-packed transfer needs spin_offset % 32 == 0");
    if (!ctx->d_packed && cudaMalloc(&ctx->d_packed, sizeof(uint32_t) * ((ctx->span_elems + 31) / 32)) != cudaSuccess) {
        ctx->d_packed = nullptr;
        return fail(ctx, SPIN_ENOMEM, "packed transfer buffer");
    }
    if (!ctx->d_blk_all) {
        // about 16 words per thread of a 256-thread block, at least one block per lattice
        std::vector<int32_t> all(ctx->n_lat + 1, 0), small(ctx->n_lat + 1, 0);
        for (int i = 0; i < ctx->n_lat; ++i) {
            const int L = ctx->lat[i].L;
            const int64_t words = ((int64_t)L * L + 31) / 32;
            const int b = (int)std::max<int64_t>(1, (words + 4095) / 4096);
            all[i + 1] = all[i] + b;
            small[i + 1] = small[i] + ((L == 512 || L == 1024 || L == 2048) ? 0 : b);
        }
        if (cudaMalloc(&ctx->d_blk_all, sizeof(int32_t) * all.size()) != cudaSuccess ||
            cudaMalloc(&ctx->d_blk_small, sizeof(int32_t) * small.size()) != cudaSuccess)
            return fail(ctx, SPIN_ENOMEM, "packed transfer block ranges");
        CK(cudaMemcpy(ctx->d_blk_all, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_blk_small, small.data(), sizeof(int32_t) * small.size(), cudaMemcpyHostToDevice));
        ctx->nblk_all = all.back();
        ctx->nblk_small = small.back();
    }
    return SPIN_OK;
}

static bool all_square(const spin_ctx *ctx) {
    for (const auto &d : ctx->lat)
        if (d.geometry != 0) return false;
    return true;
}

// spin_sweep_packed's one-sweep path with the strip kernel's bit layouts:
// square Ising lattices in the batched form, every strip lattice's packed rows
// on 16-byte boundaries.
static bool bits_path_ok(const spin_ctx *ctx) {
    if (ctx->model != SPIN_ISING || ctx->mode != 0 || !ctx->n_strip || !all_square(ctx)) return false;
    for (const auto &d : ctx->lat)
        if ((d.L == 512 || d.L == 1024 || d.L == 2048) && d.spin_offset % 128) return false;
    return true;
}

// Upload one bit per spin and unpack it into `target` (the caller's buffer
// or the ping-pong buffer), with the running statistics of the loaded state.
static int load_packed_into(spin_ctx *ctx, const uint32_t *host, void *target, cudaStream_t s) {
    const size_t nw = (ctx->span_elems + 31) / 32;
    CK(cudaMemcpyAsync(ctx->d_packed, host, sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, s));
    // square lattices: the statistics of the loaded state are counted from the bits
    // while unpacking; other geometries are recounted from the unpacked state
    const bool square = all_square(ctx);
    CK(launch_unpack_spins(ctx->d_packed, static_cast<int8_t *>(target), ctx->d_lats, ctx->n_lat, ctx->d_blk_all,
                           ctx->nblk_all, square ? ctx->st.cur : nullptr, s));
    if (!square)
        CK(launch_stats_from_state(target, ctx->model, ctx->d_lats, ctx->n_lat, ctx->maxL, ctx->width,
                                   ctx->d_type, ctx->n_types, ctx->d_vol[0], ctx->n_cells, ctx->target, ctx->st.cur, s));
    return SPIN_OK;
}

int spin_load_spins_packed(spin_ctx *ctx, const uint32_t *host, void *stream) {
    Range range_("spin_load_spins_packed");
    if (!ctx || !host) return SPIN_EINVAL;
    int rc = packed_ready(ctx);
    if (rc) return rc;
    return load_packed_into(ctx, host, ctx->spins, S(stream));
}

int spin_store_spins_packed(spin_ctx *ctx, uint32_t *host, void *stream) {
    Range range_("spin_store_spins_packed");
    if (!ctx || !host) return SPIN_EINVAL;
    int rc = packed_ready(ctx);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    const size_t nw = (ctx->span_elems + 31) / 32;
    CK(launch_pack_spins(static_cast<const int8_t *>(ctx->spins), ctx->d_packed, nw, ctx->d_lats, ctx->n_lat,
                         ctx->d_blk_all, ctx->nblk_all, s));
    CK(cudaMemcpyAsync(host, ctx->d_packed, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost, s));
    return SPIN_OK;
}

int spin_sweep_packed(spin_ctx *ctx, const uint32_t *host_in, uint32_t *host_out, int32_t n_sweeps, int32_t record,
                      void *stream) {
    Range range_("spin_sweep_packed");
    if (!ctx) return SPIN_EINVAL;
    int rc = packed_ready(ctx);
    if (rc) return rc;
    if (n_sweeps < 0) return fail(ctx, SPIN_EINVAL, "negative sweep count");
    if ((uint64_t)ctx->t + (uint64_t)n_sweeps >= 0xFFFFFFFEull)
        return fail(ctx, SPIN_ESTATE, "sweep counter would reach the values reserved for initialisation");
    if (record && n_sweeps > 0 && ctx->st.cap <= 0) return fail(ctx, SPIN_ESTATE, "no record ring (max_record_sweeps = 0)");
    cudaStream_t s = S(stream);
    if (host_in && host_out && n_sweeps == 1 && bits_path_ok(ctx)) {
        // One sweep between the transfers: the strip kernel reads its lattices'
        // rows from the uploaded bits and writes their bits beside the int8 rows;
        // only the other lattices are unpacked (into the ping-pong buffer, which
        // the sweep reads) and packed; the loaded state's statistics are counted
        // from all the bits.
        const size_t nw = (ctx->span_elems + 31) / 32;
        if (!ctx->d_packed2) {
            // cleared once: the words between and after the lattices are never written
            // again (the strip kernel and the pack kernel write whole lattice words only)
            if (cudaMalloc(&ctx->d_packed2, sizeof(uint32_t) * nw) != cudaSuccess) {
                ctx->d_packed2 = nullptr;
                return fail(ctx, SPIN_ENOMEM, "packed transfer buffer");
            }
            CK(cudaMemsetAsync(ctx->d_packed2, 0, sizeof(uint32_t) * nw, s));
        }
        CK(cudaMemcpyAsync(ctx->d_packed, host_in, sizeof(uint32_t) * nw, cudaMemcpyHostToDevice, s));
        CK(launch_unpack_spins(ctx->d_packed, static_cast<int8_t *>(ctx->spins2), ctx->d_lats, ctx->n_lat,
                               ctx->d_blk_all, ctx->nblk_all, ctx->st.cur, s, true));
        int launches = 0;
        rc = launch_sweep(ctx, ctx->spins2, ctx->spins, record ? 1 : 0, s, launches, kSrcBits | kDstBits,
                          ctx->d_packed, ctx->d_packed2);
        if (rc) return rc;
        ctx->last_launches = launches;
        ctx->t += 1;
        if (record) ctx->n_rec += 1;
        CK(launch_pack_spins(static_cast<const int8_t *>(ctx->spins), ctx->d_packed2, nw, ctx->d_lats, ctx->n_lat,
                             ctx->d_blk_small, ctx->nblk_small, s, true));
        CK(cudaMemcpyAsync(host_out, ctx->d_packed2, sizeof(uint32_t) * nw, cudaMemcpyDeviceToHost, s));
        return SPIN_OK;
    }
    // an odd number of sweeps in a ping-pong launch form: unpack into the
    // ping-pong buffer, so that the last sweep lands in the caller's buffer
    const bool tmp = host_in && (n_sweeps & 1) && (ctx->mode == 0 || ctx->mode == 3);
    if (host_in) {
        rc = load_packed_into(ctx, host_in, tmp ? ctx->spins2 : ctx->spins, s);
        if (rc) return rc;
    }
    if (n_sweeps > 0) {
        rc = run_sweeps(ctx, n_sweeps, record ? 1 : 0, s, tmp);
        if (rc) return rc;
        ctx->t += (uint32_t)n_sweeps;
        if (record) ctx->n_rec += n_sweeps;
    }
    if (host_out) return spin_store_spins_packed(ctx, host_out, stream);
    return SPIN_OK;
}

int spin_store_spins(spin_ctx *ctx, void *host, void *stream) {
    Range range_("spin_store_spins");
    if (!ctx || !host) return SPIN_EINVAL;
    const size_t bytes = ctx->model == SPIN_CPM ? (size_t)ctx->lat[0].L * ctx->lat[0].L * 4
                                                : ctx->span_elems * ctx->elem;
    CK(cudaMemcpyAsync(host, ctx->spins, bytes, cudaMemcpyDeviceToHost, S(stream)));
    return SPIN_OK;
}

// Blob: header | cur stats | spins span | CPM areas.
struct CkptHeader {
    uint64_t magic;
    int32_t model, n_lat, width, pad;
    uint32_t t;
    int32_t pad2;
    int64_t n_rec;
    uint64_t spin_bytes, vol_bytes;
};

int spin_checkpoint(spin_ctx *ctx, void *host_blob, size_t *size, void *stream) {
    Range range_("spin_checkpoint");
    if (!ctx || !size) return SPIN_EINVAL;
    const size_t spin_bytes = ctx->model == SPIN_CPM ? (size_t)ctx->lat[0].L * ctx->lat[0].L * 4
                                                     : ctx->span_elems * ctx->elem;
    const size_t vol_bytes = ctx->model == SPIN_CPM ? sizeof(int32_t) * (ctx->n_cells + 1) : 0;
    const size_t stat_bytes = sizeof(int64_t) * ctx->n_lat * ctx->width;
    const size_t need = sizeof(CkptHeader) + stat_bytes + spin_bytes + vol_bytes;
    if (!host_blob) {
        *size = need;
        return SPIN_OK;
    }
    if (*size < need) return fail(ctx, SPIN_EINVAL, "checkpoint buffer too small");
    cudaStream_t s = S(stream);
    CkptHeader h{0x53504E4D434B5031ull, ctx->model, ctx->n_lat, ctx->width, 0, ctx->t, 0, ctx->n_rec,
                 spin_bytes, vol_bytes};
    char *p = static_cast<char *>(host_blob);
    std::memcpy(p, &h, sizeof h);
    CK(cudaMemcpyAsync(p + sizeof h, ctx->st.cur, stat_bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(p + sizeof h + stat_bytes, ctx->spins, spin_bytes, cudaMemcpyDeviceToHost, s));
    if (vol_bytes)
        CK(cudaMemcpyAsync(p + sizeof h + stat_bytes + spin_bytes, ctx->d_vol[0], vol_bytes,
                           cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *size = need;
    return SPIN_OK;
}

int spin_restore(spin_ctx *ctx, const void *host_blob, size_t size, void *stream) {
    Range range_("spin_restore");
    if (!ctx || !host_blob || size < sizeof(CkptHeader)) return SPIN_EINVAL;
    CkptHeader h;
    std::memcpy(&h, host_blob, sizeof h);
    const size_t stat_bytes = sizeof(int64_t) * ctx->n_lat * ctx->width;
    if (h.magic != 0x53504E4D434B5031ull || h.model != ctx->model || h.n_lat != ctx->n_lat ||
        h.width != ctx->width || size < sizeof h + stat_bytes + h.spin_bytes + h.vol_bytes)
        return fail(ctx, SPIN_EINVAL, "checkpoint does not match this context");
    cudaStream_t s = S(stream);
    const char *p = static_cast<const char *>(host_blob);
    CK(cudaMemcpyAsync(ctx->st.cur, p + sizeof h, stat_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->spins, p + sizeof h + stat_bytes, h.spin_bytes, cudaMemcpyHostToDevice, s));
    if (ctx->model != SPIN_CPM)
        CK(cudaMemcpyAsync(ctx->spins2, ctx->spins, h.spin_bytes, cudaMemcpyDeviceToDevice, s));
    if (h.vol_bytes) {
        CK(cudaMemcpyAsync(ctx->d_vol[0], p + sizeof h + stat_bytes + h.spin_bytes, h.vol_bytes,
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->d_vol[1], ctx->d_vol[0], h.vol_bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ctx->d_dvol[0], 0, h.vol_bytes, s));
        CK(cudaMemsetAsync(ctx->d_dvol[1], 0, h.vol_bytes, s));
    }
    DevState ds{h.t, 0, h.n_rec};
    CK(cudaMemcpyAsync(ctx->d_state, &ds, sizeof ds, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->st.delta, 0, stat_bytes, s));
    CK(cudaStreamSynchronize(s));
    ctx->t = h.t;
    ctx->n_rec = h.n_rec;
    return SPIN_OK;
}

int spin_autotune(spin_ctx *ctx, int32_t sweeps_per_trial, void *stream) {
    Range range_("spin_autotune");
    if (!ctx) return SPIN_EINVAL;
    if (ctx->model == SPIN_CPM) return SPIN_OK;
    if (sweeps_per_trial < 2) sweeps_per_trial = 2;
    const std::string key = shape_key(ctx);
    const char *cache = std::getenv("SPINMC_TUNE_CACHE");
    if (cache) {
        std::ifstream f(cache);
        std::string k;
        int m, g, tr, th;
        while (f >> k >> m >> g >> tr >> th)
            if (k == key) return spin_set_launch(ctx, m, g, tr ? tr : -1, th);
    }
    cudaStream_t s = S(stream);
    // save the chain state; trials advance it
    size_t blob = 0;
    spin_checkpoint(ctx, nullptr, &blob, stream);
    std::vector<char> saved(blob);
    int rc = spin_checkpoint(ctx, saved.data(), &blob, stream);
    if (rc) return rc;
    struct Cand { int mode, tile, threads; };
    // batched form: CTA size (tile kernel) / warps per CTA (strip kernel: 4 for
    // 128 and 256, 8 for 512) and work-item height (0 = the default items: for
    // the Ising strip kernel one per resident warp); plain form.
    std::vector<Cand> cands;
    for (int th : {128, 256, 512})
        for (int tr : {0, 8, 16, 32, 64}) cands.push_back({0, tr, th});
    cands.push_back({1, 0, 256});
    if (resident_ok(ctx)) {
        for (int th : {128, 256, 512, 1024}) cands.push_back({2, 0, th});
        // square lattices: each lattice split over a cluster of 2 or 4 CTAs
        if (ctx->model == SPIN_ISING && !ctx->n_nnn && !ctx->n_tri)
            for (int cs : {2, 4})
                for (int th : {256, 512, 1024}) cands.push_back({2, cs, th});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Cand bc = {0, 16, 256};
    // a trial lasts at least about kMinTrialMs: short ones (small batches,
    // microseconds per sweep) are repeated with proportionally more sweeps
    constexpr float kMinTrialMs = 1.0f;
    for (const Cand &c : cands) {
        rc = spin_set_launch(ctx, c.mode, 1, c.tile ? c.tile : -1, c.threads);
        if (rc) continue;
        rc = spin_sweep(ctx, 2, 0, stream);  // warm-up, graph capture
        if (rc) return rc;
        float ms = 0.f;
        for (int n = sweeps_per_trial, k = 0;; ++k) {
            CK(cudaEventRecord(e0, s));
            rc = spin_sweep(ctx, n, 0, stream);
            if (rc) return rc;
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)n;                    // per sweep
            if (ms * n >= 0.5f * kMinTrialMs || n >= 4096 || k == 3) break;
            n = std::min(4096, ((int)(kMinTrialMs / std::max(ms, 1e-4f)) + 2) & ~1);   // even: whole graphs
        }
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rc = spin_set_launch(ctx, bc.mode, 1, bc.tile ? bc.tile : -1, bc.threads);
    if (rc) return rc;
    rc = spin_restore(ctx, saved.data(), saved.size(), stream);
    if (rc) return rc;
    if (cache) {
        std::ofstream f(cache, std::ios::app);
        f << key << " " << bc.mode << " " << 1 << " " << bc.tile << " " << bc.threads << "\n";
    }
    return SPIN_OK;
}

int spin_barrier_selftest(int32_t blocks, int32_t missing, int32_t rounds, void *stream) {
    if (blocks < 1 || missing < 0 || missing > blocks || rounds < 1) return SPIN_EINVAL;
    int dev = 0, coop = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPIN_ECUDA;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || blocks > sms) return SPIN_EINVAL;
    cudaStream_t s = S(stream);
    void *buf = nullptr;
    if (cudaMalloc(&buf, 16) != cudaSuccess) return SPIN_ENOMEM;
    unsigned int *bar = static_cast<unsigned int *>(buf);
    int *err = reinterpret_cast<int *>(bar + 2);
    int flag = 0, rc = SPIN_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
        launch_grid_barrier_probe(bar, err, blocks, missing, rounds, s) != cudaSuccess ||
        cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = SPIN_ECUDA;
    else if (flag)
        rc = SPIN_ETIMEOUT;
    cudaFree(buf);
    return rc;
}

int spin_profile(spin_ctx *ctx, int32_t enable, int32_t max_launches) {
    if (!ctx) return SPIN_EINVAL;
    if (max_launches < 0) return fail(ctx, SPIN_EINVAL, "max_launches must be >= 0");
    ctx->prof = enable != 0;
    ctx->prof_n = 0;
    if (ctx->prof) {
        while ((int)ctx->prof_ev.size() < 2 * max_launches) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            ctx->prof_ev.push_back(e);
        }
        ctx->prof_cls.assign(ctx->prof_ev.size() / 2, 0);
    }
    return SPIN_OK;
}

int spin_profile_read(spin_ctx *ctx, double *total_ms, int64_t *launches, void *stream) {
    if (!ctx || !total_ms || !launches) return SPIN_EINVAL;
    CK(cudaStreamSynchronize(S(stream)));
    for (int c = 0; c < 3; ++c) {
        total_ms[c] = 0.0;
        launches[c] = 0;
    }
    for (int i = 0; i < ctx->prof_n; ++i) {
        float ms = 0.f;
        const int c = ctx->prof_cls[i];
        if (c < 0 || c > 2) continue;
        CK(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        total_ms[c] += ms;
        launches[c] += 1;
    }
    return SPIN_OK;
}

// ------------------------------------------------------------------ batched CPM
static bool aligned16(const void *p);

static std::vector<uint32_t> cpm_thresholds(float T) {
    std::vector<uint32_t> thr;
    thr.push_back(0xFFFFFFFFu);  // dE = 0 (never read: dE <= 0 accepts)
    for (int dE = 1; dE < (1 << 22); ++dE) {
        const double k = std::floor(std::exp(-(double)dE / (double)T) * 4294967296.0);
        if (k <= 1.0) break;
        thr.push_back((uint32_t)(std::min(k, 4294967296.0) - 1.0));
    }
    return thr;
}

static int cpm_batch_check(int32_t n_lattices, int32_t L, const spin_cpm_params *cpm) {
    if (!cpm || n_lattices < 1 || L < 8 || L > 128 || L % 4) return SPIN_EINVAL;
    if (cpm->n_types < 1 || cpm->n_types > 8 || !cpm->J_type || cpm->reserved != 0) return SPIN_EINVAL;
    for (int a = 0; a < cpm->n_types; ++a)
        for (int b = 0; b < cpm->n_types; ++b)
            if (cpm->J_type[a * cpm->n_types + b] != cpm->J_type[b * cpm->n_types + a]) return SPIN_EINVAL;
    if (!(cpm->T > 0.0f) || !std::isfinite(cpm->T) || cpm->lambda < 0 || cpm->target_area < 0) return SPIN_EINVAL;
    if (cpm->n_cells < 1 || cpm->n_cells >= L * L || cpm->n_cells + 1 > 4096) return SPIN_EINVAL;
    return SPIN_OK;
}

int64_t spin_cpm_batch_workspace_bytes(const spin_cpm_params *cpm) {
    if (!cpm || !(cpm->T > 0.0f) || !std::isfinite(cpm->T)) return SPIN_EINVAL;
    return 256 + 4 * (int64_t)cpm_thresholds(cpm->T).size();
}

int spin_cpm_batch_init(uint64_t seed, int32_t n_lattices, int32_t L, const spin_cpm_params *cpm, int32_t *ids,
                        uint8_t *types, int32_t *areas, void *stream) {
    if (cpm_batch_check(n_lattices, L, cpm) || !ids || !types || !areas) return SPIN_EINVAL;
    const int rows = (cpm->n_cells + std::max(1, cpm->init_cols) - 1) / std::max(1, cpm->init_cols);
    if (cpm->init_side < 1 || cpm->init_cols < 1 || cpm->init_cols * cpm->init_side > L || rows * cpm->init_side > L)
        return SPIN_EINVAL;
    cudaStream_t s = S(stream);
    uint8_t *given = nullptr;
    if (cpm->cell_type) {
        if (cpm->cell_type[0] != 0) return SPIN_EINVAL;
        for (int c = 1; c <= cpm->n_cells; ++c)
            if (cpm->cell_type[c] >= cpm->n_types) return SPIN_EINVAL;
        // the caller's types go to lattice 0's slot first and are read from there by every lattice
        if (cudaMemcpyAsync(types, cpm->cell_type, (size_t)cpm->n_cells + 1, cudaMemcpyHostToDevice, s))
            return SPIN_ECUDA;
        given = types;
    } else if (cpm->n_types < 3) {
        return SPIN_EINVAL;
    }
    return launch_cpm_batch_init(n_lattices, L, cpm->n_cells, cpm->init_side, cpm->init_cols, given,
                                 (uint32_t)seed, (uint32_t)(seed >> 32), ids, types, areas, s) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

int spin_cpm_batch_run(uint64_t seed, int32_t n_lattices, int32_t L, const spin_cpm_params *cpm, int32_t *ids,
                       const uint8_t *types, int32_t *areas, uint32_t first_step, int32_t n_steps, int64_t *stats,
                       void *workspace, void *stream) {
    Range range_("spin_cpm_batch_run");
    if (cpm_batch_check(n_lattices, L, cpm) || !ids || !types || !areas || n_steps < 1 || !aligned16(workspace))
        return SPIN_EINVAL;
    if ((uint64_t)first_step + (uint64_t)n_steps >= 0xFFFFFFFEull) return SPIN_EINVAL;
    cudaStream_t s = S(stream);
    const std::vector<uint32_t> thr = cpm_thresholds(cpm->T);
    std::vector<int32_t> J(64, 0);
    for (int k = 0; k < cpm->n_types * cpm->n_types; ++k) J[k] = cpm->J_type[k];
    char *ws = static_cast<char *>(workspace);
    // pageable sources: the runtime has copied them when these calls return
    if (cudaMemcpyAsync(ws, J.data(), 256, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(ws + 256, thr.data(), 4 * thr.size(), cudaMemcpyHostToDevice, s))
        return SPIN_ECUDA;
    CpmBatchArgs a{n_lattices, L, cpm->n_types, cpm->n_cells, cpm->lambda, cpm->target_area, (int)thr.size(),
                   cpm->n_types * (cpm->n_types + 1) / 2 + 2, first_step, n_steps, (uint32_t)seed,
                   (uint32_t)(seed >> 32), ids, types, areas, reinterpret_cast<const int32_t *>(ws),
                   reinterpret_cast<const uint32_t *>(ws + 256), stats};
    return launch_cpm_batch(a, s) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

// ------------------------------------------------------------------ MLP
int spin_mlp_param_count(void) { return mlp_param_count(); }

int spin_mlp_forward(const float *params, const float *mu, const float *inv_sigma, const float *X,
                     int32_t n, float *Y, void *stream) {
    if (!params || !mu || !inv_sigma || !X || !Y || n < 0) return SPIN_EINVAL;
    return launch_mlp_forward(params, mu, inv_sigma, X, n, Y, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int spin_mlp_backward(const float *params, const float *mu, const float *inv_sigma, const float *X,
                      const float *T, int32_t n, float *grad, float *loss, float *dX, void *stream) {
    if (!params || !mu || !inv_sigma || !X || !T || !grad || n <= 0) return SPIN_EINVAL;
    return launch_mlp_backward(params, mu, inv_sigma, X, T, n, grad, loss, dX, S(stream)) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

int spin_adam(float *params, const float *grad, float *m, float *v, int32_t n, int32_t step, float lr,
              float beta1, float beta2, float eps, void *stream) {
    if (!params || !grad || !m || !v || step < 1 || n < 0) return SPIN_EINVAL;
    return launch_adam(params, grad, m, v, n, step, lr, beta1, beta2, eps, S(stream)) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

int spin_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr,
                  float beta1, float beta2, float eps, void *stream) {
    if (!params || !grad || !m || !v || step < 1) return SPIN_EINVAL;
    return launch_mlp_adam(params, grad, m, v, step, lr, beta1, beta2, eps, S(stream)) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

// ------------------------------------------------------------------ DMC
static bool dmc_geom_ok(int32_t n_lattices, int32_t L, int32_t n_sweeps) {
    return n_lattices >= 1 && L >= 8 && L <= 64 && L % 8 == 0 && n_sweeps >= 1 && n_sweeps <= (1 << 20);
}

static bool aligned16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

int64_t spin_dmc_tape_floats(int32_t n_lattices, int32_t L, int32_t n_sweeps) {
    if (!dmc_geom_ok(n_lattices, L, n_sweeps)) return SPIN_EINVAL;
    return (int64_t)n_lattices * 2 * n_sweeps * ((int64_t)L * L / 2);
}

static bool dmc_params_ok(float beta, float h, float alpha) {
    return std::isfinite(beta) && std::isfinite(h) && std::isfinite(alpha) && beta >= 0.0f && alpha >= 0.0f;
}

int spin_dmc_forward(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                     const float *J, float *spins, uint32_t first_sweep, int32_t n_sweeps, float *tape,
                     void *stream) {
    if (!dmc_geom_ok(n_lattices, L, n_sweeps) || !dmc_params_ok(beta, h, alpha)) return SPIN_EINVAL;
    if (!aligned16(J) || !aligned16(spins) || !aligned16(tape)) return SPIN_EINVAL;
    DmcArgs a{n_lattices, L, n_sweeps, first_sweep, beta, h, alpha, (uint32_t)seed, (uint32_t)(seed >> 32),
              spins, J, tape, nullptr, nullptr};
    return launch_dmc_forward(a, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int spin_dmc_backward(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                      const float *J, const float *spins, const float *tape, uint32_t first_sweep,
                      int32_t n_sweeps, float *grad_spins, float *grad_J, void *stream) {
    if (!dmc_geom_ok(n_lattices, L, n_sweeps) || !dmc_params_ok(beta, h, alpha)) return SPIN_EINVAL;
    if (!aligned16(J) || !aligned16(spins) || !aligned16(tape) || !aligned16(grad_spins) || !aligned16(grad_J))
        return SPIN_EINVAL;
    DmcArgs a{n_lattices, L, n_sweeps, first_sweep, beta, h, alpha, (uint32_t)seed, (uint32_t)(seed >> 32),
              const_cast<float *>(spins), J, const_cast<float *>(tape), grad_spins, grad_J};
    return launch_dmc_backward(a, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int spin_dmc_loss(int32_t n_lattices, int32_t L, const float *spins, const float *target, float *grad_spins,
                  double *loss, void *stream) {
    if (n_lattices < 1 || L < 2 || (int64_t)L * L > (1 << 30) || !spins || !target || !grad_spins || !loss)
        return SPIN_EINVAL;
    return launch_dmc_loss(n_lattices, L * L, spins, target, grad_spins, loss, S(stream)) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

int32_t spin_dmc_step_max_sweeps(int32_t L) {
    if (!dmc_geom_ok(1, L, 1)) return SPIN_EINVAL;
    const size_t budget = 226 * 1024;   // dynamic shared memory of one block, with room for the static part
    int32_t k = 0;
    while (dmc_step_smem(L, k + 1) <= budget && k < 4096) ++k;
    return k;
}

int spin_dmc_step(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha,
                  uint32_t first_sweep, int32_t n_sweeps, float *spins, float *J, float *m, float *v,
                  const float *target, double *loss, int32_t step, float lr, float beta1, float beta2, float eps,
                  void *stream) {
    Range range_("spin_dmc_step");
    if (!dmc_geom_ok(n_lattices, L, n_sweeps) || !dmc_params_ok(beta, h, alpha)) return SPIN_EINVAL;
    if (n_sweeps > spin_dmc_step_max_sweeps(L) || step < 1 || !std::isfinite(lr)) return SPIN_EINVAL;
    if (!aligned16(spins) || !aligned16(J) || !aligned16(m) || !aligned16(v) || !aligned16(target) || !loss)
        return SPIN_EINVAL;
    float c1, c2;
    adam_bias(step, beta1, beta2, c1, c2);
    DmcStepArgs a{n_lattices, L, n_sweeps, first_sweep, beta, h, alpha, (uint32_t)seed, (uint32_t)(seed >> 32),
                  spins, J, m, v, target, loss, lr, beta1, beta2, eps, c1, c2};
    return launch_dmc_step(a, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int spin_dmc_energy(int32_t n_lattices, int32_t L, float h, const float *J, const float *spins, float *grad_spins,
                    double *energy, void *stream) {
    if (!dmc_geom_ok(n_lattices, L, 1) || !std::isfinite(h) || !J || !spins || !energy) return SPIN_EINVAL;
    return launch_dmc_energy(n_lattices, L, J, spins, h, grad_spins, energy, S(stream)) == cudaSuccess ? SPIN_OK
                                                                                                    : SPIN_ECUDA;
}

int spin_dmc_spin_step(int64_t n, float *spins, const float *grad, float eta, void *stream) {
    if (n < 0 || (n > 0 && (!spins || !grad)) || !std::isfinite(eta)) return SPIN_EINVAL;
    if (n == 0) return SPIN_OK;
    return launch_dmc_spin_step(n, spins, grad, eta, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int32_t spin_dmc_spin_iter_max_sweeps(int32_t L) {
    if (!dmc_geom_ok(1, L, 1)) return SPIN_EINVAL;
    const size_t budget = 226 * 1024;
    int32_t k = 0;
    while (dmc_spin_iter_smem(L, k + 1) <= budget && k < 4096) ++k;
    return k;
}

int spin_dmc_spin_iter(uint64_t seed, int32_t n_lattices, int32_t L, float beta, float h, float alpha, float eta,
                       uint32_t first_sweep, int32_t n_sweeps, const float *J, float *spins, double *energy,
                       void *stream) {
    if (!dmc_geom_ok(n_lattices, L, n_sweeps) || !dmc_params_ok(beta, h, alpha) || !std::isfinite(eta))
        return SPIN_EINVAL;
    if (n_sweeps > spin_dmc_spin_iter_max_sweeps(L) || !aligned16(J) || !aligned16(spins) || !energy)
        return SPIN_EINVAL;
    DmcSpinIterArgs a{n_lattices, L, n_sweeps, first_sweep, beta, h, alpha, eta, (uint32_t)seed,
                      (uint32_t)(seed >> 32), spins, J, energy};
    return launch_dmc_spin_iter(a, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

int spin_check_status(uint32_t *first_code) {
    if (!first_code) return SPIN_EINVAL;
    *first_code = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return SPIN_ECUDA;
    for (auto fn : {check_word_ising, check_word_potts, check_word_cpm, check_word_stats}) {
        unsigned w = 0;
        if (fn(&w, true) != cudaSuccess) return SPIN_ECUDA;
        if (w && !*first_code) *first_code = w;
    }
#ifdef SPIN_CHECK
    return 1;
#else
    return 0;
#endif
}

int spin_philox_xor(uint64_t seed, uint32_t lattice, uint32_t sweep, uint32_t colour, uint32_t g0,
                    uint32_t n_groups, uint32_t *out, void *stream) {
    if (!out || (uint64_t)g0 + (uint64_t)n_groups > ((uint64_t)1 << 32)) return SPIN_EINVAL;
    return launch_philox_xor(g0, n_groups, lattice, sweep, colour, (uint32_t)seed, (uint32_t)(seed >> 32), out,
                             S(stream)) == cudaSuccess
               ? SPIN_OK
               : SPIN_ECUDA;
}

int spin_dmc_discretize(int64_t n, float *spins, void *stream) {
    if (n < 0 || (n > 0 && !spins)) return SPIN_EINVAL;
    if (n == 0) return SPIN_OK;
    return launch_dmc_discretize(n, spins, S(stream)) == cudaSuccess ? SPIN_OK : SPIN_ECUDA;
}

}  // extern "C"
