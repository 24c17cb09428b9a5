// sm_report_noalloc: the report search for callers that cannot allocate
// device memory. The paper has no counterpart; this is an interface choice.
//
// The regular entry points keep their scratch (per-CTA partial counts, the
// last-CTA ticket, per-tile match counts) in a context that sm_create
// allocates with cudaMalloc. Here the same scratch lives in one file-scope
// device array of fixed size, loaded with the library, so a call allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine, no
// host heap. The kernels are the same scan kernels sm_report launches.
//
// Scratch layout (bytes of g_noalloc_scratch):
//   [0, 4)        deferred status bits; after the passes a one-thread kernel
//                 turns an expired bounded wait into *d_count = UINT64_MAX
//   [4, 8)        last-CTA ticket (must be 0 when a call starts)
//   [8, 16)       tile counter of the tile-count pass (must be 0 when a call starts)
//   [256, ..)     per-CTA, then per-range partial counts, kMaxCtas x uint64
//   [.., end)     per-(tile, warp) match counts, kMaxTiles x 8 x uint32
// kMaxTiles bounds the text: at most kMaxTiles * 16384 start positions.
#include "sm.h"
#include "sm_internal.h"
#include "sm_plan.h"

#include <cstdlib>
#include <cstring>
#include <mutex>

namespace {

constexpr uint32_t kMaxCtas = 2048;
constexpr uint32_t kMaxTiles = 16384;
constexpr size_t kPartialsOff = 256;
constexpr size_t kWarpCountsOff = kPartialsOff + sizeof(uint64_t) * kMaxCtas;
constexpr size_t kScratchBytes = kWarpCountsOff + sizeof(uint32_t) * kMaxTiles * smk::kConsumerWarps;  // 540,928 bytes

static_assert((uint64_t)kMaxTiles * smk::kTile == SM_NOALLOC_MAX_STARTS, "header limit out of date");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    std::mutex mu;
    bool ok = false;                    // set once the set-up succeeded; a failed one is retried
    cudaError_t err = cudaSuccess;
    unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    size_t max_smem = 0;
};

DeviceSetup g_setup[kMaxDevices];

// Run once per device, with that device current: find the array's device
// address (host code cannot use the symbol itself) and raise the kernels'
// shared-memory limit.
void setup_device(DeviceSetup& s, int dev) {
    void* p = nullptr;
    s.err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (s.err != cudaSuccess) return;
    s.scratch = static_cast<unsigned char*>(p);
    int v = 0;
    if ((s.err = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return;
    s.num_sms = v;
    if ((s.err = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return;
    s.max_smem = (size_t)v;
    s.err = smk::scan_prepare(s.max_smem);
    s.ok = s.err == cudaSuccess;
}

// After the passes: a bounded wait that expired leaves the count and the
// positions invalid; the caller, who has no context to ask, sees it as
// *d_count == UINT64_MAX (no real count comes near it).
__global__ void timeout_to_count_kernel(const uint32_t* __restrict__ status, uint64_t* __restrict__ d_count) {
    if (*status & smk::kStatusTimeout) *d_count = ~0ull;
}

// Test hook, read at every call: SM_NOALLOC_TEST_TIMEOUT=1 makes the scan
// never start the copy of tile 0 and gives every wait a 2 ms limit, so the
// wait expires (without a fault) and the timeout report can be checked.
bool test_timeout() {
    const char* v = std::getenv("SM_NOALLOC_TEST_TIMEOUT");
    return v && v[0] == '1';
}

}  // namespace

extern "C" sm_status sm_report_noalloc(const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                                       const uint32_t* h_pi, uint64_t* d_pos, uint64_t cap, uint64_t* d_count,
                                       sm_stream_t stream) {
    if (!d_count || (!d_text && n) || (cap && !d_pos) || !h_pat) return SM_EINVAL;
    if (m == 0 || m > SM_MAX_M) return SM_EINVAL;
    if (h_pi) {
        unsigned char seen[SM_MAX_M];
        std::memset(seen, 0, m);
        for (uint32_t j = 0; j < m; ++j) {
            if (h_pi[j] >= m || seen[h_pi[j]]) return SM_EINVAL;
            seen[h_pi[j]] = 1;
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SM_ECUDA;
    DeviceSetup& su = g_setup[dev];
    {
        std::lock_guard<std::mutex> lk(su.mu);
        if (!su.ok) setup_device(su, dev);
        if (!su.ok) return SM_ECUDA;
    }

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((uint64_t)m > n) return cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s) == cudaSuccess ? SM_OK : SM_ECUDA;
    const uint64_t nstarts = n - m + 1;
    if (nstarts > SM_NOALLOC_MAX_STARTS) return SM_EINVAL;   // text longer than the scratch covers

    // compare descriptors in the order pi, the first two peeled (no histogram)
    const uint32_t delta = (uint32_t)(reinterpret_cast<uintptr_t>(d_text) & 15u);
    uint32_t v[SM_MAX_M], qc[SM_MAX_M], groups[smk::max_groups_for(SM_MAX_M)];
    for (uint32_t j = 0; j < m; ++j) {
        const uint32_t q = h_pi ? h_pi[j] : j;
        v[j] = ((q + delta) << 8) | h_pat[q];
    }
    uint32_t ng = 0;
    const uint32_t r = smk::plan_dense(v, m, nullptr, 0, qc, groups, smk::max_groups_for(SM_MAX_M), &ng);
    if (r == 0) return SM_EINVAL;
    smk::ScanArgs a{};
    a.text = d_text;
    a.n = n;
    a.nstarts = nstarts;
    a.ntiles = (nstarts + smk::kTile - 1) / smk::kTile;
    a.m = m;
    a.r = r;
    a.ng = ng;
    a.stage_bytes = smk::stage_bytes_for(m);
    a.stages = 4;
    while (a.stages > 2 && smk::scan_smem_bytes(a.stage_bytes, a.stages, smk::kKindBytes, true) > su.max_smem)
        --a.stages;
    const size_t smem = smk::scan_smem_bytes(a.stage_bytes, a.stages, smk::kKindBytes, true);
    if (smem > su.max_smem) return SM_ENOTSUP;
    const int occ = smk::scan_occupancy(smk::kModeTileCount, smk::kKindBytes, m, smem);
    if (occ <= 0) return SM_ECUDA;
    uint64_t want = (uint64_t)su.num_sms * (uint64_t)occ;
    if (want > kMaxCtas) want = kMaxCtas;
    if (want > a.ntiles) want = a.ntiles;
    a.tiles_per_cta = (a.ntiles + want - 1) / want;
    const uint32_t grid = (uint32_t)((a.ntiles + a.tiles_per_cta - 1) / a.tiles_per_cta);
    a.status = reinterpret_cast<uint32_t*>(su.scratch);
    a.ticket = reinterpret_cast<uint32_t*>(su.scratch + 4);
    a.tile_next = reinterpret_cast<unsigned long long*>(su.scratch + 8);
    a.partials = reinterpret_cast<uint64_t*>(su.scratch + kPartialsOff);
    a.warp_counts = reinterpret_cast<uint32_t*>(su.scratch + kWarpCountsOff);
    a.one = 1;
    a.d_count = d_count;
    a.spin_ns = 1000000000ull;
    if (test_timeout()) {
        a.test_skip_copy = 1;
        a.spin_ns = 2000000ull;
    }

    // the array keeps the previous call's contents: clear status, ticket
    // and tile counter
    if (cudaMemsetAsync(su.scratch, 0, kPartialsOff, s) != cudaSuccess) return SM_ECUDA;
    if (smk::launch_scan(smk::kModeTileCount, smk::kKindBytes, grid, smem, s, a, qc, groups) != cudaSuccess) return SM_ECUDA;
    if (smk::launch_range_sums(grid, s, a.warp_counts, a.ntiles, a.tiles_per_cta, a.partials) != cudaSuccess)
        return SM_ECUDA;
    a.d_pos = d_pos;
    a.cap = cap;
    if (smk::launch_scan(smk::kModeWrite, smk::kKindBytes, grid, smem, s, a, qc, groups) != cudaSuccess) return SM_ECUDA;
    timeout_to_count_kernel<<<1, 1, 0, s>>>(a.status, d_count);
    if (cudaGetLastError() != cudaSuccess) return SM_ECUDA;
    return SM_OK;
}
