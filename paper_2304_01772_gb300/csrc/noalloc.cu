// noalloc.cu -- an Ising sweep entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hook, a process whose device memory is
// fully reserved up front, or an embedding that forbids allocation after
// start-up.  spin_ising_sweep_noalloc runs the Ising chain of spin_sweep
// (same Philox stream, same tables: bit-identical spins and statistics)
// without a context, on a simpler launch plan: every lattice with L % 16 == 0
// goes through the tile kernel (whole lattices up to 128^2, row blocks above),
// the others through the per-site kernel; the row-strip kernel that
// spin_sweep uses for L = 512, 1024 and 2048 is not used here, so those sizes
// run slower than through a context.  Its scratch -- the second spin buffer, the
// acceptance tables, the work list and the statistics counters -- lives in
// the file-scope array g_noalloc_scratch below, which every GPU that loads
// the library holds until the process exits.  The caller passes the spins
// (in and out) and, optionally, the statistics buffer.
//
// Host code must not pass g_noalloc_scratch to a kernel: in host code that
// name is a host-side stand-in, not a device address.  The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, by the first call made on it; that first call should come before
// any stream capture.  Every call reuses the array and finds the previous
// call's contents there, so the counters are cleared at the start of each
// call; calls that overlap on the GPU (different streams, different host
// threads) race on the array and must be serialised by the caller.
#include <mutex>

#include "internal.h"
#include "spinmc.h"

namespace spinmc {
void build_ising_table(const spin_lattice_desc &d, TabEntry *out);
cudaError_t launch_copy_lattices(const void *src, void *dst, const LatDev *lats, int n_lat,
                                 int elem, cudaStream_t s);
}  // namespace spinmc

using namespace spinmc;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPIN_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};

// Host staging for the descriptors copied into the scratch array (no heap).
constexpr int kMaxLat = 4096;
constexpr int kMaxItems = 16384;
// Largest side: a row block of the tile kernel holds 32768 / L rows plus a
// four-row halo in shared memory, which at L = 4096 (12 rows, 48 KB) exceeds
// the kernel's 47 KB without a raised limit.
constexpr int kMaxSide = 2048;
LatDev g_lat_stage[kMaxLat];
TabEntry g_tab_stage[kMaxLat * kTabStride];
Item g_item_stage[kMaxItems];
int32_t g_generic_stage[kMaxLat];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int spin_ising_sweep_noalloc(uint64_t seed, int32_t n_lattices,
                                        const spin_lattice_desc *lat, void *d_spins,
                                        uint32_t first_sweep, int32_t n_sweeps, int64_t *d_stats,
                                        void *stream) {
    if (!lat || !d_spins || n_lattices < 1 || n_lattices > kMaxLat || n_sweeps < 0)
        return SPIN_EINVAL;
    if ((uint64_t)first_sweep + (uint64_t)n_sweeps >= 0xFFFFFFFEull) return SPIN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPIN_ECUDA;
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SPIN_ECUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPIN_ECUDA;
        g_scratch_dev[dev] = ptr;
        g_sm_count[dev] = sms;
    }
    // lattices: validate, stage descriptors and tables, plan the work list
    size_t span = 0;
    int n_items = 0, n_generic = 0, maxL = 0, genL = 0;
    size_t smem = 16;
    for (int i = 0; i < n_lattices; ++i) {
        const spin_lattice_desc &d = lat[i];
        if (d.L < 4 || (d.L & 1) || d.L > kMaxSide || d.geometry != 0 || d.J2 != 0.0f) return SPIN_EINVAL;
        if (!(d.beta >= 0.0f) || !(d.beta < 3.0e38f) || !(d.J == d.J) || !(d.h == d.h)) return SPIN_EINVAL;
        const bool fast = d.L % 16 == 0 && d.spin_offset % 16 == 0;
        g_lat_stage[i] = LatDev{d.spin_offset, d.L, 2, fast ? 1 : 0, 0, d.lattice_id ? d.lattice_id - 1u : (uint32_t)i, 0};
        build_ising_table(d, g_tab_stage + (size_t)i * kTabStride);
        span = span > d.spin_offset + (size_t)d.L * d.L ? span : d.spin_offset + (size_t)d.L * d.L;
        maxL = maxL > d.L ? maxL : d.L;
        if (!fast) {
            g_generic_stage[n_generic++] = i;
            genL = genL > d.L ? genL : d.L;
            continue;
        }
        if (d.L * d.L <= 16384) {
            if (n_items >= kMaxItems) return SPIN_EINVAL;
            g_item_stage[n_items++] = Item{i, 0, d.L, 1};
            smem = smem > (size_t)d.L * d.L ? smem : (size_t)d.L * d.L;
            continue;
        }
        const int rows = d.L < 32768 / d.L ? d.L : (32768 / d.L > 0 ? 32768 / d.L : 1);
        for (int r0 = 0; r0 < d.L; r0 += rows) {
            if (n_items >= kMaxItems) return SPIN_EINVAL;
            g_item_stage[n_items++] = Item{i, r0, d.L - r0 < rows ? d.L - r0 : rows, 0};
        }
        smem = smem > (size_t)(rows + 4) * d.L ? smem : (size_t)(rows + 4) * d.L;
    }
    // the tile kernel runs without a raised shared-memory limit here: its dynamic
    // share plus its static tables must stay within the default 48 KB
    if (smem > 47 * 1024) return SPIN_EINVAL;
    // scratch layout: state | lattices | tables | items | generic ids | cur | delta | spins2
    const size_t o_lat = 256;
    const size_t o_tab = align256(o_lat + sizeof(LatDev) * n_lattices);
    const size_t o_item = align256(o_tab + sizeof(TabEntry) * kTabStride * n_lattices);
    const size_t o_gen = align256(o_item + sizeof(Item) * n_items);
    const size_t o_cur = align256(o_gen + sizeof(int32_t) * n_generic);
    const size_t o_delta = align256(o_cur + sizeof(int64_t) * 2 * n_lattices);
    const size_t o_spins2 = align256(o_delta + sizeof(int64_t) * 2 * n_lattices);
    if (o_spins2 + span > SPIN_NOALLOC_SCRATCH_BYTES) return SPIN_EINVAL;   // beyond the fixed scratch size
    if (n_sweeps == 0) return SPIN_OK;
    char *base = static_cast<char *>(g_scratch_dev[dev]);
    DevState *state = reinterpret_cast<DevState *>(base);
    LatDev *d_lats = reinterpret_cast<LatDev *>(base + o_lat);
    TabEntry *d_tabs = reinterpret_cast<TabEntry *>(base + o_tab);
    Item *d_items = reinterpret_cast<Item *>(base + o_item);
    int32_t *d_gen = reinterpret_cast<int32_t *>(base + o_gen);
    int64_t *d_cur = reinterpret_cast<int64_t *>(base + o_cur);
    int64_t *d_delta = reinterpret_cast<int64_t *>(base + o_delta);
    int8_t *spins2 = reinterpret_cast<int8_t *>(base + o_spins2);
    int8_t *spins = static_cast<int8_t *>(d_spins);
    const DevState ds{first_sweep, 0, 0};
#define NA_CK(x)                              \
    do {                                      \
        if ((x) != cudaSuccess) return SPIN_ECUDA; \
    } while (0)
    NA_CK(cudaMemcpyAsync(state, &ds, sizeof ds, cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(d_lats, g_lat_stage, sizeof(LatDev) * n_lattices, cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(d_tabs, g_tab_stage, sizeof(TabEntry) * kTabStride * n_lattices,
                          cudaMemcpyHostToDevice, s));
    if (n_items) NA_CK(cudaMemcpyAsync(d_items, g_item_stage, sizeof(Item) * n_items, cudaMemcpyHostToDevice, s));
    if (n_generic)
        NA_CK(cudaMemcpyAsync(d_gen, g_generic_stage, sizeof(int32_t) * n_generic, cudaMemcpyHostToDevice, s));
    // counters start at zero; current statistics from the state
    NA_CK(cudaMemsetAsync(d_delta, 0, sizeof(int64_t) * 2 * n_lattices, s));
    NA_CK(launch_stats_from_state(spins, 0, d_lats, n_lattices, maxL, 2, nullptr, 0, nullptr, 0, 0, d_cur, s));
    const StatsBufs st{d_cur, d_delta, d_stats, d_stats ? n_sweeps : 0, 2, n_lattices, 0};
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    const int sms = g_sm_count[dev] > 0 ? g_sm_count[dev] : 1;
    const int grid = n_items < sms * 4 ? (n_items > 0 ? n_items : 1) : sms * 4;
    for (int i = 0; i < n_sweeps; ++i) {
        const int8_t *src = (i & 1) ? spins2 : spins;
        int8_t *dst = (i & 1) ? spins : spins2;
        for (int c = 0; c < 2 && n_generic; ++c)
            NA_CK(launch_ising_generic(src, dst, d_gen, n_generic, genL, d_lats, d_tabs, k0, k1, state,
                                       d_delta, c, s));
        if (n_items) {
            IsingSweepArgs a{d_items, n_items, d_lats, d_tabs, src, dst, k0, k1, state, d_delta,
                             philox_keys(k0, k1), n_lattices};
            NA_CK(launch_ising_fused(a, grid, 256, smem, s));
        }
        NA_CK(launch_finalize(state, st, d_stats ? 1 : 0, s));
    }
    if (n_sweeps & 1) NA_CK(launch_copy_lattices(spins2, spins, d_lats, n_lattices, 1, s));
#undef NA_CK
    return SPIN_OK;
}
