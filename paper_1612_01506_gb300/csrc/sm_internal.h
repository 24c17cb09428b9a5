// Internal interface between the host runtime (sm_api.cpp, sm_noalloc.cu) and
// the kernels (sm_kernels.cu). Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace smk {

constexpr int kConsumerWarps = 8;                       // warps that compare
constexpr int kThreads = 32 * (kConsumerWarps + 1);     // + one producer warp
constexpr int kChunks = 4;                              // 16-start chunks per lane
constexpr uint32_t kWarpStarts = 16 * 32 * kChunks;     // 2048 start positions per consumer warp
constexpr uint32_t kTile = kWarpStarts * kConsumerWarps;  // 16384 starts per tile
constexpr int kSmallM = 64;              // pattern capacity of the small parameter block
constexpr int kLargeM = 4096;            // pattern capacity of the large parameter block
constexpr int kMaxStages = 8;

// Deferred status bits, OR-ed into the status word.
constexpr uint32_t kStatusTrunc = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Compare variants of the scan kernel: bytes (exact zero-byte test), 7-bit
// bytes (a cheaper test), and 2-bit codes of texts with at most four
// distinct symbols (code bits b1, b2 adjacent or not).
enum ScanKind : int {
    kKindBytes = 0,      // byte compares, any text
    kKindSeven = 1,      // byte compares, text and pattern below 0x80
    kKindPackedAdj = 2,  // 2-bit codes (<= 4 symbols) from adjacent symbol bits
    kKindPacked = 3,     // 2-bit codes from any two symbol bits
    kKindBinary = 4,     // 1-bit codes (<= 2 symbols)
    kKinds = 5
};
inline bool kind_packed(int kind) { return kind >= kKindPackedAdj; }

enum ScanMode : int {
    kModeCount = 0,      // count only: per-CTA partial counts, last CTA writes *d_count
    kModeTileCount = 1,  // as kModeCount, and per-(tile, warp) counts (and found bitmaps) for a
                         // report
    kModeWrite = 2,      // report: write ascending positions of tiles with matches; CTA b owns
                         // tile range b (its first rank from range_sums, else from the
                         // per-range partials of launch_range_sums)
    kModeSparse = 3,     // as kModeCount, and the per-(tile, warp) counts that are not zero
                         // and their per-range sums (both arrays zero on entry): the first
                         // pass of a report whose matches fall in few tiles, which
                         // kModeWrite then scans again
    kModes = 4
};

struct ScanArgs {
    const uint8_t* text;
    uint64_t n;
    uint64_t nstarts;        // n - m + 1
    uint64_t ntiles;         // ceil(nstarts / kTile)
    uint64_t tiles_per_cta;  // write mode: each CTA owns one contiguous range of tiles
    uint32_t m;
    uint32_t r;              // peeled compares, 1..m (dense phase)
    uint32_t stage_bytes;    // shared-memory bytes per pipeline stage (multiple of 128)
    uint32_t stages;         // pipeline depth, 2..kMaxStages
    uint32_t one;            // the value 1 (keeps an add on the multiply-add pipe)
    uint32_t ng;             // window groups of the peeled compares
    uint32_t b1, b2;         // packed kinds: the symbol bits that form the codes (binary: b1)
    uint32_t gather;         // packed kinds: 0x01041040 (see pack16)
    uint32_t packed_words;   // packed kinds: words of one packed tile buffer
    uint32_t test_skip_copy; // test hook: 1 = never issue the first tile's copy
    uint32_t* status;        // deferred status word
    uint64_t* partials;      // counting modes: per-CTA counts; write: per tile-range counts (grid entries)
    uint32_t* ticket;        // last-CTA ticket (scratch, zero between launches)
    unsigned long long* tile_next;  // next unclaimed tile of the counting modes (scratch, zero between launches)
    uint64_t* d_count;       // result count
    uint32_t* warp_counts;   // per-(tile, warp) counts (scratch, ntiles x 8; report only)
    uint32_t* bitmaps;       // report: per-(tile, warp) slots of found bits (ntiles x 8 x 64 words) or null
    uint64_t* d_pos;         // report output
    uint64_t cap;            // report capacity
    uint64_t spin_ns;        // limit of every bounded wait, in ns
    // The rescanning report. Ranges of range_tiles tiles (the write mode's
    // CTAs, at most kThreads tiles each): the sparse mode adds each nonzero
    // per-(tile, warp) count into range_sums[tile / range_tiles]; the write
    // mode takes its range's first rank from them and its tiles with matches
    // from the count words, and leaves both arrays zero again (each CTA
    // clears the count words it read, the last CTA the range sums). Null in
    // the other reports: the write mode then takes the first ranks from
    // partials (range_sum_kernel) and scans the count words as it goes.
    uint64_t* range_sums;
    uint64_t range_tiles;
};

struct HistArgs {
    const uint8_t* text;
    uint64_t n;
    uint64_t* partials;      // scratch, grid x 256
    uint32_t* ticket;        // scratch
    uint64_t* d_hist;        // result, 256 entries
};

// Shared-memory bytes of one stage for patterns of length m: the tile, the
// (m-1)-byte halo, the 0..15-byte misalignment and 32 bytes of load slack.
inline uint32_t stage_bytes_for(uint32_t m) {
    uint32_t chunks = kTile / 16 + 2 + ((14u + m) >> 4);
    uint32_t b = chunks * 16;
    return (b + 127u) & ~127u;
}

// Header (barriers, stage descriptors, reduction slots), the per-warp queues
// of 16-start chunks with surviving starts (one 4-byte entry for each of the
// warp's 128 chunks), then the stage ring.
constexpr uint32_t kScanHeader = 512;
constexpr uint32_t kQueueCap = kWarpStarts / 16;                           // entries per warp
constexpr uint32_t kQueueBytes = kConsumerWarps * kQueueCap * 4;           // 4 KiB

// Packed kinds: one tile of 2-bit codes takes a word per 16-byte unit of
// the stage buffer (1-bit codes: per 32-byte unit), plus 8 words of load
// slack; four such buffers (two rounds of two tiles) replace the survivor
// queues.
inline uint32_t packed_words_for(uint32_t stage_bytes, int kind = kKindPacked) {
    return stage_bytes / (kind == kKindBinary ? 32u : 16u) + 8;
}

// Reports: the byte kinds build each warp-tile's found bitmap in shared
// memory (64 words per warp).
constexpr uint32_t kBitmapWords = kWarpStarts / 32;
constexpr uint32_t kBitmapBytes = kConsumerWarps * kBitmapWords * 4;   // 2 KiB

// The write mode with range sums lists its range's tiles with matches in
// shared memory after the stages: per tile, its 8 warp offsets (16 bits
// each), then (tile, matches).
constexpr uint32_t kWriteList = kThreads;
constexpr size_t kWriteListBytes = (size_t)kWriteList * 24;

inline size_t scan_smem_bytes(uint32_t stage_bytes, uint32_t stages, int kind = kKindBytes, bool report = false) {
    const size_t mid = kind_packed(kind) ? (size_t)16 * packed_words_for(stage_bytes, kind)
                                         : kQueueBytes + (report ? kBitmapBytes : 0u);
    return kScanHeader + mid + (size_t)stage_bytes * stages;
}

// Launch a scan kernel. `qc` holds the m compare descriptors (e << 8) | p[q],
// e = (text address mod 16) + q, in scan order and `groups` the a.ng window
// groups of the first a.r (both as planned by plan_dense).
cudaError_t launch_scan(int mode, int kind, uint32_t grid, size_t smem, cudaStream_t s,
                        const ScanArgs& a, const uint32_t* qc, const uint32_t* groups);
// Resident CTAs per SM of the scan kernel used for (m, mode, kind) with this smem.
int scan_occupancy(int mode, int kind, uint32_t m, size_t smem);
// Raise the dynamic shared-memory limit of every scan kernel.
cudaError_t scan_prepare(size_t max_smem);

constexpr int kHistThreads = 256;
cudaError_t launch_hist(uint32_t grid, cudaStream_t s, const HistArgs& a);

// Second pass of a report: positions from the found bitmaps of the first.
struct WriteArgs {
    uint64_t ntiles;
    uint64_t tiles_per_cta;       // CTA b writes the tiles of range b
    const uint64_t* partials;     // per-range match counts of the first pass
    const uint32_t* warp_counts;  // per-(tile, warp) counts
    const uint32_t* bitmaps;      // per-(tile, warp) slots of found bits (list or bitmap form)
    uint64_t* d_pos;
    uint64_t cap;
    uint32_t* status;
    uint32_t folded;              // 1: byte-compare slots (folded lane entries); 0: coded (contiguous)
};
constexpr int kWriteThreads = 32 * kConsumerWarps;
cudaError_t launch_bitmap_write(uint32_t grid, cudaStream_t s, const WriteArgs& a);
// Resident blocks per SM of the second pass.
int bitmap_write_occupancy();
// Between the passes: partials[b] = matches in tiles [b T, (b + 1) T), one block per range.
cudaError_t launch_range_sums(uint32_t grid, cudaStream_t s, const uint32_t* warp_counts, uint64_t ntiles,
                              uint64_t tiles_per_range, uint64_t* partials);

}  // namespace smk
