// Internal interface between the host runtime (sm_api.cu) and the kernels
// (sm_kernels.cu). Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace smk {

constexpr int kThreads = 256;            // threads per scan CTA (8 warps)
constexpr uint32_t kTile = 8192;         // start positions per tile: 8 warps x 1024
constexpr int kSmallM = 64;              // pattern capacity of the small parameter block
constexpr int kLargeM = 4096;            // pattern capacity of the large parameter block
constexpr int kMaxStages = 8;

// Deferred status bits, OR-ed into the context's device status word.
constexpr uint32_t kStatusTrunc = 1u;
constexpr uint32_t kStatusTimeout = 2u;

enum ScanMode : int {
    kModeCount = 0,      // count only: per-CTA partial counts, last CTA writes *d_count
    kModeTileCount = 1,  // as kModeCount, and per-tile counts for a later report pass
    kModeWrite = 2       // report: write ascending positions of tiles with matches
};

struct ScanArgs {
    const uint8_t* text;
    uint64_t n;
    uint64_t nstarts;        // n - m + 1
    uint64_t ntiles;         // ceil(nstarts / kTile)
    uint64_t tiles_per_cta;  // each CTA owns one contiguous range of tiles
    uint32_t m;
    uint32_t r;              // peeled compares, 1..m
    uint32_t stage_bytes;    // shared-memory bytes per pipeline stage (multiple of 128)
    uint32_t stages;         // pipeline depth, 2..kMaxStages
    uint32_t* status;        // deferred status word
    uint64_t* partials;      // per-CTA counts (scratch, grid entries)
    uint32_t* ticket;        // last-CTA ticket (scratch, zero between launches)
    uint64_t* d_count;       // result count
    uint32_t* tile_counts;   // per-tile counts (scratch, ntiles entries; report only)
    uint64_t* d_pos;         // report output
    uint64_t cap;            // report capacity
    uint64_t spin_ns;        // limit of every bounded wait, in ns
    uint32_t test_skip_copy; // test hook: 1 = never issue the first tile's copy
};

struct HistArgs {
    const uint8_t* text;
    uint64_t n;
    uint64_t* partials;      // scratch, grid x 256
    uint32_t* ticket;        // scratch
    uint64_t* d_hist;        // result, 256 entries
};

// Shared-memory bytes of one stage for patterns of length m.
inline uint32_t stage_bytes_for(uint32_t m) {
    uint32_t chunks = kTile / 16 + 2 + ((14u + m) >> 4);
    uint32_t b = chunks * 16;
    return (b + 127u) & ~127u;
}

// Header (barriers, stage descriptors, reduction slots) + the stage ring.
constexpr uint32_t kScanHeader = 512;

inline size_t scan_smem_bytes(uint32_t stage_bytes, uint32_t stages) {
    return kScanHeader + (size_t)stage_bytes * stages;
}

// Launch a scan kernel. `qc` holds m words (q << 8) | p[q] in compare order.
cudaError_t launch_scan(int mode, bool seven, uint32_t grid, size_t smem, cudaStream_t s,
                        const ScanArgs& a, const uint32_t* qc);
// Resident CTAs per SM of the scan kernel used for (m, mode, seven) with this smem.
int scan_occupancy(int mode, bool seven, uint32_t m, size_t smem);
// Raise the dynamic shared-memory limit of every scan kernel.
cudaError_t scan_prepare(size_t max_smem);

constexpr int kHistThreads = 256;
cudaError_t launch_hist(uint32_t grid, cudaStream_t s, const HistArgs& a);

}  // namespace smk
