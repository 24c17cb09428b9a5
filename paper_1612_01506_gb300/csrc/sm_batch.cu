// Batched counting: many patterns of uneven lengths over many texts in one
// persistent launch (the batched form of the SIMD-naive search of Tarhio,
// Holub, Giaquinta, Algorithms 2-4).
//
// Work items are (text, tile) pairs over the packed texts. A CTA owns a
// contiguous range of items; its producer warp stages each tile (plus the
// halo of the text's longest pattern) once, and the consumer warps test every
// pattern of that text against the staged tile with the same dense/sparse
// compare core as the single-pattern scan, so all patterns of a text share one
// pass over HBM. Counts gather in shared memory per pattern and are added to
// the output once per CTA.
//
// The plan (sm_batch_create) runs on the host once per batch: per-text byte
// histograms (one launch), the rarest-first order of each pattern under its
// own text's frequencies (Sec. 2.2), the peel factor, the 7-bit compare where
// the text allows it, and patterns with a symbol absent from their text are
// dropped (their count is 0). sm_batch_count is then one memset and one
// launch, and can be captured in a CUDA graph.
#include "sm.h"
#include "sm_device.cuh"
#include "sm_plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

namespace smk {
namespace {

using namespace dev;

constexpr uint32_t kMaxSlots = 4096;   // patterns one CTA counts in shared memory
constexpr uint32_t kHistChunk = 65536; // bytes per histogram work item
// A pattern whose rarest symbol has at most this frequency in its text takes
// the candidate path (expected candidates per tile <= 0.08 * 16384) ...
constexpr double kCandidateFreq = 0.08;
// ... when its text region has at least kCandidateMin such patterns: the
// symbol index of a staged tile costs about as much as the dense scan of a
// dozen patterns (measured on GB300: ~16 us per tile and CTA against
// ~1.3 us for one dense pattern), so fewer run the dense scan.
constexpr uint32_t kCandidateMin = 16;

struct BatchText {        // a text, or one group of <= kMaxSlots of its patterns
    uint64_t off;         // byte offset in the packed texts
    uint64_t n;           // length (bytes readable from off)
    uint64_t item_begin;  // first work item (tile) of this entry
    uint64_t slimit;      // only starts below this are counted (a chunk of a longer text)
    uint32_t pbeg, pmid;  // patterns [pbeg, pmid) run the dense scan ...
    uint32_t pend;        // ... and [pmid, pend) the candidate path
    uint32_t maxm;
    uint32_t mask_idx;    // 8-word mask of the candidate patterns' first symbols
    uint32_t codes;       // 0: byte compares; else 2-bit codes: bits b1 (0-7), b2 (8-15), bit 16 set
};
constexpr uint32_t kCoded = 1u << 16;

struct BatchPat {
    uint32_t qc_off;      // first compare descriptor in the qc table
    uint32_t m, r;
    uint32_t ng;          // window groups of the peeled compares (after the m compares in the qc table)
    uint32_t out;         // index of the pattern in the caller's arrays
    uint32_t seven;       // 1: text and pattern are 7-bit
    uint64_t tb;          // reports: the pattern's first per-tile counter
};

// Batched reports run the batch kernel three ways: counting; counting plus a
// count per (pattern, tile); and writing positions. Between the last two,
// batch_prefix_kernel turns each pattern's tile counts into the rank of its
// first match in every tile.
constexpr int kBatchCount = 0;
constexpr int kBatchTileCount = 1;
constexpr int kBatchWrite = 2;

// A pattern's per-tile counters: tcnt[tb .. tb + nt) (tile counts) and
// toff[tb .. tb + nt] (their exclusive prefix sums, then the total).
struct PatTiles {
    uint64_t tb;
    uint32_t nt;
    uint32_t out;         // index of the pattern in the caller's arrays
    uint64_t witem;       // the write pass's work item of the pattern's tile 0
};

struct BatchArgs {
    const uint8_t* texts;
    const uint32_t* masks;      // 8 words per entry with candidate patterns
    const BatchText* tx;        // ntx + 1 entries (the last one: item_begin = total items)
    uint32_t ntx;
    const BatchPat* pats;
    const uint32_t* qc;
    const uint64_t* cta_items;  // grid + 1: CTA b takes items [cta_items[b], cta_items[b+1])
    const uint32_t* cta_pbase;  // grid: first pattern counted by CTA b (its slot 0)
    int64_t* d_counts;
    uint32_t* tcnt;             // tile count: per-(pattern, tile) counts, zeroed by the caller
    const uint64_t* toff;       // write: per-(pattern, tile) ranks of the first match
    uint64_t* d_pos;            // write: positions of pattern `out` go to d_pos + pos_off[out] ...
    const int64_t* pos_off;     // ... at most pos_off[out + 1] - pos_off[out] of them
    const uint8_t* hit;         // write: 1 for the work items (tiles) where some pattern matches
    uint32_t stage_bytes, stages, one, nslots;
    uint32_t index_cap;         // entries of the per-tile position index (0: no index)
    uint32_t packed_words;      // words of the packed-tile buffer (0: no entry uses 2-bit codes)
    uint32_t* status;
    uint64_t spin_ns;
};

struct BatchDesc {
    uint64_t k;   // tile within the text entry
    uint32_t x;   // text entry, ~0u: no more items
    uint32_t pad;
};


template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const __grid_constant__ BatchArgs A) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + 64);
    BatchDesc* desc = reinterpret_cast<BatchDesc*>(smem + 128);
    uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + 256);   // write: [2][kConsumerWarps] warp counts
    uint32_t* queues = reinterpret_cast<uint32_t*>(smem + kScanHeader);
    uint32_t* slots = reinterpret_cast<uint32_t*>(smem + kScanHeader + kQueueBytes);
    uint8_t* after_slots = smem + kScanHeader + kQueueBytes + ((A.nslots * 4u + 127u) & ~127u);
    // per-tile position index of selected symbols: count, start, cursor, positions
    uint32_t* icnt = reinterpret_cast<uint32_t*>(after_slots);
    uint32_t* istart = icnt + 256;
    uint32_t* icur = icnt + 512;
    uint16_t* ilist = reinterpret_cast<uint16_t*>(icnt + 768);
    uint8_t* after_index = after_slots + (A.index_cap ? ((3072u + 2u * A.index_cap + 127u) & ~127u) : 0u);
    uint32_t* pbuf = reinterpret_cast<uint32_t*>(after_index);   // 2-bit codes of the staged tile
    uint8_t* bufs = after_index + ((4u * A.packed_words + 127u) & ~127u);

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t SB = A.stage_bytes, S = A.stages, one = A.one;
    const uint64_t i0 = A.cta_items[blockIdx.x], i1 = A.cta_items[blockIdx.x + 1];
    const uint32_t pbase = A.cta_pbase[blockIdx.x];

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        fence_mbar_init();
    }
    for (uint32_t i = tid; i < A.nslots; i += kThreads) slots[i] = 0;
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ---------------------------------------------------------- producer
        uint32_t x = 0;
        {   // last entry whose first item is <= i0
            uint32_t lo = 0, hi = A.ntx;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (A.tx[mid].item_begin <= i0) lo = mid; else hi = mid;
            }
            x = lo;
        }
        uint64_t cursor = i0;
        uint32_t issued = 0;
        for (uint32_t it = 0, s = 0, u = 0;; ++it) {
            if (u > 0) {
                const bool ok = __all_sync(kFull, wait_bounded(&empty[s], (u - 1) & 1u, A.spin_ns));
                if (!ok) {
                    if (lane == 0) atomicOr(A.status, kStatusTimeout);
                    break;
                }
            }
            uint8_t* buf = bufs + (size_t)s * SB;
            BatchDesc d{0, ~0u, 0};
            TileCopy cp{0, 0, 0};
            if (MODE == kBatchWrite)   // only tiles with matches are staged again
                while (cursor < i1 && !__ldg(A.hit + cursor)) ++cursor;
            if (cursor < i1) {
                const uint64_t item = cursor++;
                while (A.tx[x + 1].item_begin <= item) ++x;
                const BatchText T = A.tx[x];
                d.x = x;
                d.k = item - T.item_begin;
                const uint64_t s0 = d.k * kTile;
                cp = stage_ragged(buf, A.texts + T.off, T.n, s0, min(s0 + kTile + T.maxm - 1, T.n), lane);
            }
            __syncwarp();
            if (lane == 0) {
                desc[s] = d;
                fence_proxy_async();
                mbar_arrive_expect_tx(&full[s], cp.bytes);
                if (cp.bytes) bulk_g2s(buf + cp.dst_off, reinterpret_cast<const void*>(cp.src), cp.bytes, &full[s]);
            }
            issued = it + 1;
            if (d.x == ~0u) break;
            if (++s == S) {
                s = 0;
                ++u;
            }
        }
        if (lane == 0)
            for (uint32_t st = 0; st < S && st < issued; ++st)
                (void)wait_bounded(&full[st], ((issued - 1 - st) / S) & 1u, A.spin_ns);
        __syncwarp();
    } else {
        // ---------------------------------------------------------- consumers
        uint32_t* q = queues + warp * kQueueCap;
        const uint32_t c0 = warp * (kWarpStarts / 16) + lane;
        const uint32_t wq = warp * (kWarpStarts / 4);
        uint32_t wpar = 0;   // write: which half of wcnt the next pattern uses
        for (uint32_t s = 0, phase = 0;;) {
            const bool ok = __all_sync(kFull, wait_bounded(&full[s], phase, A.spin_ns));
            // every consumer warp leaves together (later tiles use consumer barriers)
            if (consumers_any(!ok)) {
                if (lane == 0 && !ok) atomicOr(A.status, kStatusTimeout);
                break;
            }
            const BatchDesc d = desc[s];
            if (d.x == ~0u) break;
            const uint8_t* buf = bufs + (size_t)s * SB;
            const uint4* b4 = reinterpret_cast<const uint4*>(buf);
            const uint32_t* b32 = reinterpret_cast<const uint32_t*>(buf);
            const uint64_t s0 = d.k * kTile;
            const BatchText T = A.tx[d.x];

            if (T.codes) {
                // a text of at most four symbols: the tile as 2-bit codes
                // (16 starts per word), built once for all its patterns,
                // which are all dense and planned on codes
                consumers_sync();   // the previous coded tile is no longer read
                const uint32_t b1 = T.codes & 0xFFu, b2 = (T.codes >> 8) & 0xFFu;
                const uint32_t units = SB / 16u;
                if (b2 == b1 + 1)
                    for (uint32_t u = tid; u < units; u += kConsumerWarps * 32) pbuf[u] = pack16<true>(b4[u], b1, b2, 0x01041040u);
                else
                    for (uint32_t u = tid; u < units; u += kConsumerWarps * 32) pbuf[u] = pack16<false>(b4[u], b1, b2, 0x01041040u);
                consumers_sync();
                const uint32_t* const pk[2] = {pbuf, pbuf};
                uint32_t* const nobm[2] = {nullptr, nullptr};
                const uint64_t no_out[2] = {0, 0};
                for (uint32_t p = T.pbeg; p < T.pmid; ++p) {
                    const BatchPat P = A.pats[p];
                    const uint64_t nst = min(T.n - P.m + 1, T.slimit);
                    if (s0 >= nst) continue;
                    const GlobalQC qc{A.qc + P.qc_off, P.m};
                    const uint64_t s0s[2] = {s0, 0};
                    if constexpr (MODE == kBatchWrite) {
                        const uint64_t o0 = __ldg(A.toff + P.tb + d.k);
                        if (__ldg(A.toff + P.tb + d.k + 1) == o0) continue;   // the same for every warp
                        uint32_t c = packed_tiles<false, true, 1>(pk, false, warp, lane, qc, P.m, P.r, P.ng, nst, s0s,
                                                               no_out, nullptr, 0, nobm).x;
                        c = warp_sum_u32(c);
                        uint32_t* wc = wcnt + wpar * kConsumerWarps;
                        wpar ^= 1u;
                        if (lane == 0) wc[warp] = c;
                        consumers_sync();
                        const uint32_t before = warp_sum_u32(lane < warp ? wc[lane] : 0u);
                        if (c) {
                            const int64_t pb = __ldg(A.pos_off + P.out);
                            const uint64_t cap = (uint64_t)(__ldg(A.pos_off + P.out + 1) - pb);
                            const uint64_t outs[2] = {o0 + before, 0};
                            (void)packed_tiles<true, false, 1>(pk, false, warp, lane, qc, P.m, P.r, P.ng, nst, s0s, outs,
                                                            A.d_pos + pb, cap, nobm);
                        }
                        continue;
                    }
                    uint32_t c = packed_tiles<false, true, 1>(pk, false, warp, lane, qc, P.m, P.r, P.ng, nst, s0s, no_out,
                                                           nullptr, 0, nobm).x;
                    c = warp_sum_u32(c);
                    if (lane == 0 && c) {
                        atomicAdd(&slots[p - pbase], c);
                        if (MODE == kBatchTileCount) atomicAdd(A.tcnt + P.tb + d.k, c);
                    }
                }
            }

            // dense patterns: every warp scans its 2048 starts
            for (uint32_t p = T.pbeg; p < (T.codes ? T.pbeg : T.pmid); ++p) {
                const BatchPat P = A.pats[p];
                const uint64_t nst = min(T.n - P.m + 1, T.slimit);   // the plan keeps only m <= n
                if (s0 >= nst) continue;
                const GlobalQC qc{A.qc + P.qc_off, P.m};
                if constexpr (MODE == kBatchWrite) {
                    // a tile with matches: the warps count theirs, exchange
                    // the counts, then write from their ranks (the tables of
                    // this mode hold dense patterns only)
                    const uint64_t o0 = __ldg(A.toff + P.tb + d.k);
                    if (__ldg(A.toff + P.tb + d.k + 1) == o0) continue;   // the same for every warp
                    uint32_t c = P.seven ? warp_tile<true, false, true>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r,
                                                                        P.ng, one, nst, s0, q, 0, nullptr, 0)
                                         : warp_tile<false, false, true>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r,
                                                                         P.ng, one, nst, s0, q, 0, nullptr, 0);
                    c = warp_sum_u32(c);
                    uint32_t* wc = wcnt + wpar * kConsumerWarps;
                    wpar ^= 1u;
                    if (lane == 0) wc[warp] = c;
                    consumers_sync();   // (the half written two patterns ago was read before the last sync)
                    const uint32_t before = warp_sum_u32(lane < warp ? wc[lane] : 0u);
                    if (c) {
                        const int64_t pb = __ldg(A.pos_off + P.out);
                        const uint64_t cap = (uint64_t)(__ldg(A.pos_off + P.out + 1) - pb);
                        if (P.seven)
                            warp_tile<true, true, false>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r, P.ng, one, nst,
                                                         s0, q, o0 + before, A.d_pos + pb, cap);
                        else
                            warp_tile<false, true, false>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r, P.ng, one, nst,
                                                          s0, q, o0 + before, A.d_pos + pb, cap);
                    }
                    continue;
                }
                uint32_t c;
                if (P.seven)
                    c = warp_tile<true, false, true>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r, P.ng, one, nst, s0, q,
                                                     0, nullptr, 0);
                else
                    c = warp_tile<false, false, true>(b4, b32, c0, wq, warp, lane, qc, P.m, P.r, P.ng, one, nst, s0,
                                                      q, 0, nullptr, 0);
                c = warp_sum_u32(c);
                if (lane == 0 && c) {
                    atomicAdd(&slots[p - pbase], c);
                    if (MODE == kBatchTileCount) atomicAdd(A.tcnt + P.tb + d.k, c);
                }
            }

            // candidate patterns: their first (rarest) symbol is rare in the
            // text, so the starts worth testing are read from a position index
            // of the tile, built once and shared by all of them
            if (T.pmid < T.pend) {
                const uint32_t delta = (uint32_t)((reinterpret_cast<uintptr_t>(A.texts) + T.off) & 15u);
                const uint32_t nbytes = (uint32_t)(min(s0 + kTile + T.maxm - 1, T.n) - s0);
                const uint32_t* mask = A.masks + 8u * T.mask_idx;
                const uint32_t t = tid;   // 0..255 among the consumers
                consumers_sync();         // the previous tile's index is no longer read
                icnt[t] = 0;
                consumers_sync();
                for (uint32_t i = delta + t; i < delta + nbytes; i += kConsumerWarps * 32) {
                    const uint32_t c = buf[i];
                    if ((__ldg(mask + (c >> 5)) >> (c & 31)) & 1u) atomicAdd(&icnt[c], 1u);
                }
                consumers_sync();
                if (warp == 0) {   // exclusive scan of 256 counts, 8 per lane
                    uint32_t v[8], sum = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        v[k] = icnt[lane * 8 + k];
                        sum += v[k];
                    }
                    const uint32_t ex = warp_incl_scan(sum, lane) - sum;
                    uint32_t run = ex;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        istart[lane * 8 + k] = run;
                        icur[lane * 8 + k] = run;
                        run += v[k];
                    }
                }
                consumers_sync();
                for (uint32_t i = delta + t; i < delta + nbytes; i += kConsumerWarps * 32) {
                    const uint32_t c = buf[i];
                    if ((__ldg(mask + (c >> 5)) >> (c & 31)) & 1u) ilist[atomicAdd(&icur[c], 1u)] = (uint16_t)i;
                }
                consumers_sync();
                for (uint32_t p = T.pmid + warp; p < T.pend; p += kConsumerWarps) {
                    const BatchPat P = A.pats[p];
                    const uint64_t nst = min(T.n - P.m + 1, T.slimit);
                    if (s0 >= nst) continue;
                    const int32_t valid = (int32_t)min((uint64_t)kTile, nst - s0);
                    const uint32_t* pq = A.qc + P.qc_off;
                    const uint32_t v0 = __ldg(pq);
                    const int32_t e0 = (int32_t)(v0 >> 8);
                    const uint32_t sym = v0 & 0xFFu;
                    const uint32_t lo = istart[sym], hi = lo + icnt[sym];
                    uint32_t cnt = 0;
                    for (uint32_t k = lo + lane; k < hi; k += 32) {
                        const int32_t st = (int32_t)ilist[k] - e0;   // candidate start in the tile
                        if (st < 0 || st >= valid) continue;
                        bool ok2 = true;
                        for (uint32_t j = 1; j < P.m && ok2; ++j) {
                            const uint32_t v = __ldg(pq + j);
                            ok2 = buf[st + (int32_t)(v >> 8)] == (uint8_t)(v & 0xFFu);
                        }
                        cnt += ok2;
                    }
                    cnt = warp_sum_u32(cnt);
                    if (lane == 0 && cnt) {
                        atomicAdd(&slots[p - pbase], cnt);
                        if (MODE == kBatchTileCount) atomicAdd(A.tcnt + P.tb + d.k, cnt);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == S) {
                s = 0;
                phase ^= 1u;
            }
        }
    }
    if constexpr (MODE == kBatchWrite) return;
    __syncthreads();
    for (uint32_t i = tid; i < A.nslots; i += kThreads) {
        const uint32_t v = slots[i];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(A.d_counts + A.pats[pbase + i].out), (unsigned long long)v);
    }
}

// Batched reports, between the tile-count and write passes: block b takes
// pattern pt[b] and writes the exclusive prefix sums of its tile counts and
// then their total (toff[tb + nt]); a total above the pattern's position
// capacity sets the truncation status.
constexpr uint32_t kPrefixThreads = 256;

__global__ void __launch_bounds__(kPrefixThreads) batch_prefix_kernel(const PatTiles* __restrict__ pt,
                                                                      const uint32_t* __restrict__ tcnt,
                                                                      uint64_t* __restrict__ toff,
                                                                      const int64_t* __restrict__ pos_off,
                                                                      uint8_t* __restrict__ hit, uint32_t* status) {
    __shared__ uint64_t wsum[kPrefixThreads / 32];
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PatTiles P = pt[blockIdx.x];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < P.nt; base += 4 * kPrefixThreads) {
        uint32_t v[4], sum = 0;   // thread t: tiles base + 4t .. base + 4t + 3
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t k = base + 4u * tid + i;
            v[i] = k < P.nt ? tcnt[P.tb + k] : 0u;
            sum += v[i];
        }
        const uint32_t inc = warp_incl_scan(sum, lane);
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint64_t before = carry, total = carry;
        for (uint32_t w = 0; w < kPrefixThreads / 32; ++w) {
            before += w < warp ? wsum[w] : 0u;
            total += wsum[w];
        }
        uint64_t run = before + inc - sum;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t k = base + 4u * tid + i;
            if (k < P.nt) {
                toff[P.tb + k] = run;
                if (v[i]) hit[P.witem + k] = 1;
            }
            run += v[i];
        }
        carry = total;
        __syncthreads();   // wsum is rewritten by the next round
    }
    if (tid == 0) {
        toff[P.tb + P.nt] = carry;
        if (carry > (uint64_t)(pos_off[P.out + 1] - pos_off[P.out])) atomicOr(status, kStatusTrunc);
    }
}

// Byte histograms of ranges texts[beg[x] .. end[x]): work item = (range,
// 64 KiB piece).
__global__ void __launch_bounds__(256) batch_hist_kernel(const uint8_t* texts, const int64_t* beg, const int64_t* end,
                                                         const uint64_t* chunk_begin, uint32_t ntexts,
                                                         uint64_t nchunks, unsigned long long* hist) {
    __shared__ uint32_t h[8][256];
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    for (uint64_t item = blockIdx.x; item < nchunks; item += gridDim.x) {
        for (uint32_t i = tid; i < 8 * 256; i += 256) (&h[0][0])[i] = 0;
        __syncthreads();
        uint32_t lo = 0, hi = ntexts;   // last text whose first chunk <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (chunk_begin[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t x = lo;
        const uint64_t n = (uint64_t)(end[x] - beg[x]);
        const uint64_t b0 = (item - chunk_begin[x]) * kHistChunk;
        const uint64_t b1 = min(b0 + kHistChunk, n);
        const uint8_t* t = texts + beg[x];
        for (uint64_t i = b0 + tid; i < b1; i += 256) atomicAdd(&h[warp][t[i]], 1u);
        __syncthreads();
        {
            uint32_t v = 0;
            for (int w = 0; w < 8; ++w) v += h[w][tid];
            if (v) atomicAdd(&hist[(uint64_t)x * 256 + tid], (unsigned long long)v);
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace smk

// ------------------------------------------------------------------ host

sm_status sm_fail_internal(sm_status s, const char* msg);   // defined in sm_api.cpp
int sm_ctx_device(const sm_ctx* c);
int sm_ctx_num_sms(const sm_ctx* c);
size_t sm_ctx_max_smem(const sm_ctx* c);
uint32_t* sm_ctx_status(const sm_ctx* c);
uint64_t sm_ctx_spin_ns(const sm_ctx* c);
uint32_t sm_ctx_stages(const sm_ctx* c);

namespace {

using smk::BatchArgs;
using smk::BatchPat;
using smk::BatchText;
using smk::kMaxSlots;
using smk::PatTiles;
using smk::kTile;

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Peel factor from the pattern's symbol frequencies (the single-pattern
// scan's cost model: dense compare ~100, compaction ~80, 32 words ~60).
// One pattern described for a text with byte histogram h (n bytes): the
// rarest-first order (Sec. 2.2), then either the dense scan (peeled compares
// and their window groups from plan_dense) or the candidate path (compares
// in order pi, the first being the rarest symbol).
struct PatDesc {
    BatchPat pat{};             // the dense scan
    std::vector<uint32_t> qc;   // its m compares in scan order, then its window groups
    BatchPat cpat{};            // the candidate path (when cand)
    std::vector<uint32_t> cqc;  // its m compares in the order pi
    bool cand = false;   // the rarest symbol is rare enough for the candidate path
    bool zero = false;   // a symbol never occurs in the text, or m > n: count 0
};

PatDesc describe(const uint8_t* p, uint32_t m, const uint64_t* h, uint64_t n, uint32_t delta, bool text7,
                 uint32_t out, double cand_freq = smk::kCandidateFreq, uint32_t codes = 0) {
    PatDesc d;
    d.zero = (uint64_t)m > n;
    for (uint32_t q = 0; q < m && !d.zero; ++q) d.zero = h[p[q]] == 0;
    if (d.zero) return d;
    std::vector<uint32_t> pi(m);
    std::iota(pi.begin(), pi.end(), 0u);
    std::stable_sort(pi.begin(), pi.end(), [&](uint32_t a, uint32_t b) { return h[p[a]] < h[p[b]]; });
    std::vector<uint32_t> v(m);
    if (codes) {
        // a text of at most four symbols: compares on 2-bit codes, dense
        const uint32_t b1 = codes & 0xFFu, b2 = (codes >> 8) & 0xFFu;
        std::vector<double> freq(m);
        for (uint32_t j = 0; j < m; ++j) {
            const uint32_t c = p[pi[j]];
            v[j] = ((pi[j] + delta) << 8) | ((c >> b1) & 1u) | (((c >> b2) & 1u) << 1);
            freq[j] = (double)h[c] / (double)n;
        }
        d.qc.resize(m + smk::max_packed_groups_for(m));
        uint32_t ng = 0;
        const uint32_t r = smk::plan_packed(v.data(), m, freq.data(), 0, d.qc.data(), d.qc.data() + m,
                                            smk::max_packed_groups_for(m), &ng, 2);
        d.qc.resize(m + ng);
        d.pat = BatchPat{0, m, r, ng, out, 0u};
        return d;
    }
    for (uint32_t j = 0; j < m; ++j) v[j] = ((pi[j] + delta) << 8) | p[pi[j]];
    if ((double)h[p[pi[0]]] / (double)n < cand_freq) {
        d.cand = true;
        d.cpat = BatchPat{0, m, 1, 0, out, text7 ? 1u : 0u};   // ng = 0: no peeled compares
        d.cqc = v;
    }
    d.pat = BatchPat{0, m, 1, 0, out, text7 ? 1u : 0u};
    std::vector<double> freq(m);
    for (uint32_t j = 0; j < m; ++j) freq[j] = (double)h[p[pi[j]]] / (double)n;
    // the m compares in scan order, then the window groups of the peeled ones
    d.qc.resize(m + smk::max_groups_for(m));
    uint32_t ng = 0;
    d.pat.r = smk::plan_dense(v.data(), m, freq.data(), 0, d.qc.data(), d.qc.data() + m, smk::max_groups_for(m), &ng);
    d.qc.resize(m + ng);
    d.pat.ng = ng;
    return d;
}

// Host tables of one launch.
struct Tables {
    std::vector<BatchText> tx;
    std::vector<BatchPat> pats;
    std::vector<uint32_t> qc, masks, cta_pbase;
    std::vector<uint64_t> cta_items;
    std::vector<double> cost;
    uint64_t items = 0;
    uint32_t nslots = 1, maxm = 1;
    bool need_index = false;
    bool need_pack = false;   // some entry compares 2-bit codes
    uint32_t slot_hint() const { return (uint32_t)std::min<size_t>(pats.size(), kMaxSlots); }
};

// Entries for one text region [off, off + n) counting starts below slimit:
// groups of at most kMaxSlots patterns, dense ones first. allow_cand = false
// keeps every pattern on the dense scan (the write pass of a report); tb
// (indexed by the caller's pattern index) gives each pattern's per-tile
// counters for reports; pt, when given, receives each pattern's first work
// item.
void add_text(Tables& T, uint64_t off, uint64_t n, uint64_t slimit, const std::vector<const PatDesc*>& ds,
              bool allow_cand = true, const std::vector<uint64_t>* tb = nullptr,
              std::vector<PatTiles>* pt = nullptr, uint32_t cand_min = smk::kCandidateMin, uint32_t codes = 0) {
    uint32_t ncand = 0;
    for (const PatDesc* d : ds) ncand += (!d->zero && d->cand) ? 1u : 0u;
    const bool use_cand = allow_cand && !codes && ncand >= cand_min;
    std::vector<const PatDesc*> order;
    for (const PatDesc* d : ds)
        if (!d->zero && !(use_cand && d->cand)) order.push_back(d);
    const size_t ndense = order.size();
    for (const PatDesc* d : ds)
        if (!d->zero && use_cand && d->cand) order.push_back(d);
    for (size_t g0 = 0; g0 < order.size(); g0 += kMaxSlots) {
        const size_t g1 = std::min(order.size(), g0 + kMaxSlots);
        BatchText e{off, n, 0, slimit, (uint32_t)T.pats.size(), 0, 0, 0, 0, codes};
        T.need_pack |= codes != 0;
        uint32_t mask[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool any_cand = false;
        uint32_t mn = ~0u;
        for (size_t i = g0; i < g1; ++i) {
            const PatDesc* d = order[i];
            if (i >= ndense && !any_cand) {
                e.pmid = (uint32_t)T.pats.size();
                any_cand = true;
            }
            const bool c = i >= ndense;   // candidate path
            const std::vector<uint32_t>& qc = c ? d->cqc : d->qc;
            BatchPat bp = c ? d->cpat : d->pat;
            bp.qc_off = (uint32_t)T.qc.size();
            bp.tb = tb ? (*tb)[bp.out] : 0;
            if (pt) (*pt)[bp.out].witem = T.items;   // the entry's first item (set below)
            T.qc.insert(T.qc.end(), qc.begin(), qc.end());
            if (c) mask[(qc[0] & 0xFFu) >> 5] |= 1u << (qc[0] & 31u);
            T.pats.push_back(bp);
            e.maxm = std::max(e.maxm, bp.m);
            mn = std::min(mn, bp.m);
        }
        e.pend = (uint32_t)T.pats.size();
        if (!any_cand) e.pmid = e.pend;
        if (any_cand) {
            e.mask_idx = (uint32_t)(T.masks.size() / 8);
            T.masks.insert(T.masks.end(), mask, mask + 8);
        }
        e.item_begin = T.items;
        T.items += (std::min<uint64_t>(n - mn + 1, slimit) + kTile - 1) / kTile;
        T.maxm = std::max(T.maxm, e.maxm);
        T.need_index |= any_cand;
        T.cost.push_back(1.0 + (double)(e.pmid - e.pbeg) + 0.1 * (double)(e.pend - e.pmid));
        T.tx.push_back(e);
    }
}

// Sentinel entry and CTA ranges of about equal cost (tiles x patterns), each
// counting at most kMaxSlots patterns in shared memory.
void finish(Tables& T, uint64_t want_ctas) {
    T.tx.push_back(BatchText{0, 0, T.items, 0, 0, 0, 0, 0, 0, 0});
    double total = 0;
    for (size_t e = 0; e + 1 < T.tx.size(); ++e)
        total += T.cost[e] * (double)(T.tx[e + 1].item_begin - T.tx[e].item_begin);
    const double per_cta = std::max(1.0, total / (double)std::max<uint64_t>(want_ctas, 1));
    T.cta_items.assign(1, 0);
    T.cta_pbase.clear();
    T.nslots = 1;
    for (uint64_t item = 0, e = 0; item < T.items;) {
        while (T.tx[e + 1].item_begin <= item) ++e;   // entry of the CTA's first item
        const uint32_t pb = T.tx[e].pbeg;
        double acc = 0;
        uint64_t it = item, ee = e;
        while (it < T.items) {
            while (T.tx[ee + 1].item_begin <= it) ++ee;
            if (T.tx[ee].pend - pb > kMaxSlots) break;   // pattern window full: next CTA
            acc += T.cost[ee];
            ++it;
            if (acc >= per_cta) break;
        }
        uint64_t el = e;                                // entry of the CTA's last item
        while (T.tx[el + 1].item_begin < it) ++el;
        T.cta_items.push_back(it);
        T.cta_pbase.push_back(pb);
        T.nslots = std::max(T.nslots, T.tx[el].pend - pb);
        item = it;
    }
}

struct Geometry {
    uint32_t SB = 0, stages = 2, index_cap = 0, packed_words = 0;
    int occ = 1;
    size_t smem(uint32_t nslots) const {
        const size_t ib = index_cap ? ((3072u + 2u * index_cap + 127u) & ~127u) : 0u;
        const size_t pb = (4u * packed_words + 127u) & ~127u;
        return (size_t)smk::kScanHeader + smk::kQueueBytes + ((nslots * 4u + 127u) & ~127u) + ib + pb +
               (size_t)SB * stages;
    }
};

// Shared-memory layout and residency of a launch whose patterns have length
// <= maxm and whose CTAs count at most nslots patterns each: the stage
// count is lowered while that lets more CTAs reside on an SM.
Geometry geometry(sm_ctx* ctx, uint32_t maxm, bool need_index, uint32_t nslots = kMaxSlots,
                  uint32_t stages = 0, bool need_pack = false) {
    Geometry g;
    g.SB = smk::stage_bytes_for(maxm);
    g.index_cap = need_index ? g.SB : 0u;
    g.packed_words = need_pack ? smk::packed_words_for(g.SB) : 0u;
    g.stages = stages ? stages : sm_ctx_stages(ctx);
    nslots = std::max(1u, std::min(nslots, kMaxSlots));
    while (g.stages > 2 && g.smem(nslots) > sm_ctx_max_smem(ctx)) --g.stages;
    const int ms = (int)sm_ctx_max_smem(ctx);
    cudaFuncSetAttribute(smk::batch_kernel<smk::kBatchCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms);
    cudaFuncSetAttribute(smk::batch_kernel<smk::kBatchTileCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms);
    cudaFuncSetAttribute(smk::batch_kernel<smk::kBatchWrite>, cudaFuncAttributeMaxDynamicSharedMemorySize, ms);
    auto occ_of = [&](const Geometry& x) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, smk::batch_kernel<smk::kBatchTileCount>, smk::kThreads,
                                                      x.smem(nslots));
        return o;
    };
    int occ = occ_of(g);
    while (!stages && g.stages > 2) {   // (a tuned stage count is kept)
        Geometry f = g;
        --f.stages;
        const int o2 = occ_of(f);
        if (o2 <= occ) break;
        g = f;
        occ = o2;
    }
    g.occ = std::max(occ, 1);
    return g;
}

// Byte layout of the tables in one buffer (host staging and device copy).
struct Layout {
    size_t tx = 0, pats = 0, qc = 0, ci = 0, cp = 0, masks = 0, total = 0;
};

Layout layout_of(const Tables& T) {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    Layout L;
    size_t o = 0;
    L.tx = o; o += al(T.tx.size() * sizeof(BatchText));
    L.pats = o; o += al(std::max<size_t>(T.pats.size(), 1) * sizeof(BatchPat));
    L.qc = o; o += al(std::max<size_t>(T.qc.size(), 1) * 4);
    L.ci = o; o += al(T.cta_items.size() * 8);
    L.cp = o; o += al(std::max<size_t>(T.cta_pbase.size(), 1) * 4);
    L.masks = o; o += al(std::max<size_t>(T.masks.size(), 8) * 4);
    L.total = o;
    return L;
}

void pack(const Tables& T, const Layout& L, char* h) {
    std::memcpy(h + L.tx, T.tx.data(), T.tx.size() * sizeof(BatchText));
    if (!T.pats.empty()) std::memcpy(h + L.pats, T.pats.data(), T.pats.size() * sizeof(BatchPat));
    if (!T.qc.empty()) std::memcpy(h + L.qc, T.qc.data(), T.qc.size() * 4);
    std::memcpy(h + L.ci, T.cta_items.data(), T.cta_items.size() * 8);
    if (!T.cta_pbase.empty()) std::memcpy(h + L.cp, T.cta_pbase.data(), T.cta_pbase.size() * 4);
    if (!T.masks.empty()) std::memcpy(h + L.masks, T.masks.data(), T.masks.size() * 4);
}

BatchArgs args_for(sm_ctx* ctx, const uint8_t* d_texts, const Tables& T, const Layout& L, char* d,
                   const Geometry& g) {
    BatchArgs a{};
    a.texts = d_texts;
    a.masks = reinterpret_cast<const uint32_t*>(d + L.masks);
    a.tx = reinterpret_cast<const BatchText*>(d + L.tx);
    a.ntx = (uint32_t)T.tx.size() - 1;
    a.pats = reinterpret_cast<const BatchPat*>(d + L.pats);
    a.qc = reinterpret_cast<const uint32_t*>(d + L.qc);
    a.cta_items = reinterpret_cast<const uint64_t*>(d + L.ci);
    a.cta_pbase = reinterpret_cast<const uint32_t*>(d + L.cp);
    a.stage_bytes = g.SB;
    a.stages = g.stages;
    a.one = 1;
    a.nslots = T.nslots;
    a.index_cap = g.index_cap;
    a.packed_words = g.packed_words;
    a.status = sm_ctx_status(ctx);
    a.spin_ns = sm_ctx_spin_ns(ctx);
    return a;
}

bool text_is_7bit(const uint64_t* h) {
    for (int c = 0x80; c < 256; ++c)
        if (h[c]) return false;
    return true;
}

// BatchText::codes of a text with histogram h: 2-bit codes when it has at
// most four symbols, else 0 (byte compares).
uint32_t text_codes(const uint64_t* h) {
    uint32_t b1 = 0, b2 = 0;
    return smk::packed_code_bits(h, &b1, &b2) ? (b1 | (b2 << 8) | smk::kCoded) : 0u;
}

cudaError_t launch_batch(int mode, uint32_t grid, size_t smem, cudaStream_t st, const BatchArgs& a) {
    if (!grid) return cudaSuccess;
    switch (mode) {
        case smk::kBatchCount: smk::batch_kernel<smk::kBatchCount><<<grid, smk::kThreads, smem, st>>>(a); break;
        case smk::kBatchTileCount:
            smk::batch_kernel<smk::kBatchTileCount><<<grid, smk::kThreads, smem, st>>>(a);
            break;
        default: smk::batch_kernel<smk::kBatchWrite><<<grid, smk::kThreads, smem, st>>>(a); break;
    }
    return cudaGetLastError();
}

// Per-tile counters of a report: pattern k of length m[k] over a text of
// len[k] bytes has nt = ceil((len - m + 1) / kTile) tiles (0 when m > len)
// and counters [tb, tb + nt] (toff needs one more than tcnt). Returns the
// total number of counters.
uint64_t assign_tiles(const std::vector<uint32_t>& m, const std::vector<uint64_t>& len, std::vector<PatTiles>& pt,
                      std::vector<uint64_t>& tb) {
    const size_t np = m.size();
    pt.resize(np);
    tb.resize(np);
    uint64_t o = 0;
    for (size_t k = 0; k < np; ++k) {
        const uint64_t nt = (uint64_t)m[k] > len[k] ? 0 : (len[k] - m[k] + 1 + smk::kTile - 1) / smk::kTile;
        pt[k] = PatTiles{o, (uint32_t)nt, (uint32_t)k};
        tb[k] = o;
        o += nt + 1;
    }
    return o;
}

// The three passes of a report after the tables and counters are in place:
// tile counts (and counts), per-pattern prefix sums, ordered writes.
cudaError_t run_report(const BatchArgs& a1, uint32_t g1, size_t sm1, const BatchArgs& a2, uint32_t g2, size_t sm2,
                       const PatTiles* d_pt, uint32_t npt, uint32_t* d_tcnt, uint64_t ntb, uint64_t nitems,
                       int64_t* d_counts, uint32_t ncounts, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (ncounts) e = cudaMemsetAsync(d_counts, 0, (size_t)ncounts * sizeof(int64_t), st);
    if (e == cudaSuccess && ntb) e = cudaMemsetAsync(d_tcnt, 0, ntb * sizeof(uint32_t), st);
    if (e == cudaSuccess && nitems) e = cudaMemsetAsync(const_cast<uint8_t*>(a2.hit), 0, nitems, st);
    if (e == cudaSuccess) e = launch_batch(smk::kBatchTileCount, g1, sm1, st, a1);
    if (e == cudaSuccess && npt) {
        smk::batch_prefix_kernel<<<npt, smk::kPrefixThreads, 0, st>>>(d_pt, d_tcnt, const_cast<uint64_t*>(a2.toff),
                                                                      a2.pos_off, const_cast<uint8_t*>(a2.hit),
                                                                      a2.status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_batch(smk::kBatchWrite, g2, sm2, st, a2);
    return e;
}

// Byte histograms of the ranges d_texts[beg[x] .. end[x]) (x < ntexts; ranges
// may overlap), one launch over (range, 64 KiB) work items; synchronous on st.
sm_status text_histograms(sm_ctx* ctx, const uint8_t* d_texts, const int64_t* beg, const int64_t* end,
                          uint32_t ntexts, cudaStream_t st, std::vector<uint64_t>& hist) {
    std::vector<uint64_t> chunk_begin(ntexts + 1, 0);
    for (uint32_t x = 0; x < ntexts; ++x) {
        const uint64_t n = (uint64_t)(end[x] - beg[x]);
        chunk_begin[x + 1] = chunk_begin[x] + (n + smk::kHistChunk - 1) / smk::kHistChunk;
    }
    hist.assign((size_t)ntexts * 256, 0);
    void* tmp = nullptr;
    const size_t hb = hist.size() * 8, ob = (size_t)ntexts * 8, cb = (size_t)(ntexts + 1) * 8;
    if (cudaMalloc(&tmp, hb + 2 * ob + cb) != cudaSuccess) {
        cudaGetLastError();
        return sm_fail_internal(SM_ENOMEM, "histogram workspace");
    }
    unsigned long long* d_hist = static_cast<unsigned long long*>(tmp);
    int64_t* d_beg = reinterpret_cast<int64_t*>(static_cast<char*>(tmp) + hb);
    int64_t* d_end = reinterpret_cast<int64_t*>(static_cast<char*>(tmp) + hb + ob);
    uint64_t* d_cb = reinterpret_cast<uint64_t*>(static_cast<char*>(tmp) + hb + 2 * ob);
    cudaError_t e = cudaMemsetAsync(d_hist, 0, hb, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_beg, beg, ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_end, end, ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_cb, chunk_begin.data(), cb, cudaMemcpyHostToDevice, st);
    const uint64_t nchunks = chunk_begin[ntexts];
    if (e == cudaSuccess && nchunks) {
        const uint32_t grid = (uint32_t)std::min<uint64_t>(nchunks, (uint64_t)sm_ctx_num_sms(ctx) * 8);
        smk::batch_hist_kernel<<<grid, 256, 0, st>>>(d_texts, d_beg, d_end, d_cb, ntexts, nchunks, d_hist);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist.data(), d_hist, hb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    return e == cudaSuccess ? SM_OK : sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
}

}  // namespace

// ------------------------------------------------------------------ batch

// Plan parameters the autotuner varies (defaults: the constants above and
// the context's stage count).
struct BatchParams {
    double cand_freq = smk::kCandidateFreq;
    uint32_t cand_min = smk::kCandidateMin;
    uint32_t stages = 0;
};

struct sm_batch {
    sm_ctx* ctx = nullptr;
    int device = 0;
    uint32_t npats = 0;      // caller's pattern count (size of d_counts)
    // the inputs, kept to plan again with other parameters
    const uint8_t* d_texts = nullptr;
    std::vector<int64_t> text_off, pat_off;
    std::vector<int32_t> pat_text;
    std::vector<uint8_t> pats;
    std::vector<uint64_t> hist;   // per text, 256 bins
    BatchParams params;
    uint32_t grid = 0;
    size_t smem = 0;
    BatchArgs args{};
    void* d_mem = nullptr;   // one allocation holding every table
    // reports: the write pass's tables (dense scans only) and the
    // per-(pattern, tile) counters, allocated by the first report
    uint32_t wgrid = 0;
    size_t wsmem = 0;
    BatchArgs wargs{};
    void* d_wmem = nullptr;
    const PatTiles* d_pt = nullptr;   // in d_wmem, one per caller pattern
    uint64_t ntb = 0, nitems = 0;     // counters; work items of the write pass
    uint32_t* d_tcnt = nullptr;
    uint64_t* d_toff = nullptr;
    uint8_t* d_hit = nullptr;
};

// Plans (or plans again) a batch from its kept inputs under b->params:
// descriptions, tables of both passes, device copies, launch shapes.
sm_status build_plan(sm_batch* b) {
    using namespace smk;
    sm_ctx* ctx = b->ctx;
    const uint32_t npats = b->npats, ntexts = (uint32_t)b->text_off.size() - 1;
    const int64_t* h_text_off = b->text_off.data();
    const BatchParams& P = b->params;
    std::vector<PatDesc> descs(npats);
    std::vector<uint32_t> ms(npats);
    std::vector<uint64_t> lens(npats);
    for (uint32_t k = 0; k < npats; ++k) {
        const uint32_t x = (uint32_t)b->pat_text[k];
        const uint64_t n = (uint64_t)(h_text_off[x + 1] - h_text_off[x]);
        const uint64_t* h = &b->hist[(size_t)x * 256];
        const uint32_t delta = (uint32_t)((reinterpret_cast<uintptr_t>(b->d_texts) + (uint64_t)h_text_off[x]) & 15u);
        ms[k] = (uint32_t)(b->pat_off[k + 1] - b->pat_off[k]);
        lens[k] = n;
        descs[k] = describe(b->pats.data() + b->pat_off[k], ms[k], h, n, delta, text_is_7bit(h), k, P.cand_freq,
                            text_codes(h));
    }
    std::vector<PatTiles> pt;
    std::vector<uint64_t> tb;
    const uint64_t ntb = assign_tiles(ms, lens, pt, tb);
    // tables of the counting (and tile-count) pass, and of the write pass
    std::vector<uint32_t> by_text(npats);
    std::iota(by_text.begin(), by_text.end(), 0u);
    std::stable_sort(by_text.begin(), by_text.end(),
                     [&](uint32_t a, uint32_t c) { return b->pat_text[a] < b->pat_text[c]; });
    Tables T, W;
    for (size_t kk = 0, x = 0; x < ntexts; ++x) {
        std::vector<const PatDesc*> ptrs;
        for (; kk < npats && (uint32_t)b->pat_text[by_text[kk]] == x; ++kk) ptrs.push_back(&descs[by_text[kk]]);
        const uint64_t n = (uint64_t)(h_text_off[x + 1] - h_text_off[x]);
        const uint32_t codes = text_codes(&b->hist[(size_t)x * 256]);
        add_text(T, (uint64_t)h_text_off[x], n, ~0ull, ptrs, true, &tb, nullptr, P.cand_min, codes);
        add_text(W, (uint64_t)h_text_off[x], n, ~0ull, ptrs, false, &tb, &pt, P.cand_min, codes);
    }
    const Geometry g = geometry(ctx, T.maxm, T.need_index, T.slot_hint(), P.stages, T.need_pack);
    finish(T, (uint64_t)sm_ctx_num_sms(ctx) * g.occ);
    const Geometry gw = geometry(ctx, W.maxm, false, W.slot_hint(), P.stages, W.need_pack);
    finish(W, (uint64_t)sm_ctx_num_sms(ctx) * gw.occ);

    // one allocation for each pass's tables (the write pass's also holds the
    // per-pattern counter ranges); the previous plan's are freed
    const Layout L = layout_of(T);
    const Layout LW = layout_of(W);
    const size_t pt_off = LW.total, wtotal = pt_off + std::max<size_t>(pt.size(), 1) * sizeof(PatTiles);
    std::vector<char> host(std::max(L.total, wtotal));
    if (b->d_mem || b->d_wmem) cudaDeviceSynchronize();   // no launch may still read them
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->d_wmem) cudaFree(b->d_wmem);
    b->d_mem = b->d_wmem = nullptr;
    if (b->d_hit && b->nitems != W.items) {
        cudaFree(b->d_tcnt);
        cudaFree(b->d_toff);
        cudaFree(b->d_hit);
        b->d_tcnt = nullptr;
        b->d_toff = nullptr;
        b->d_hit = nullptr;
    }
    b->ntb = ntb;
    b->nitems = W.items;
    if (cudaMalloc(&b->d_mem, L.total) != cudaSuccess || cudaMalloc(&b->d_wmem, wtotal) != cudaSuccess) {
        cudaGetLastError();
        return sm_fail_internal(SM_ENOMEM, "batch plan tables");
    }
    pack(T, L, host.data());
    cudaError_t e = cudaMemcpy(b->d_mem, host.data(), L.total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        pack(W, LW, host.data());
        if (!pt.empty()) std::memcpy(host.data() + pt_off, pt.data(), pt.size() * sizeof(PatTiles));
        e = cudaMemcpy(b->d_wmem, host.data(), wtotal, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
    b->args = args_for(ctx, b->d_texts, T, L, static_cast<char*>(b->d_mem), g);
    b->grid = (uint32_t)T.cta_pbase.size();
    b->smem = g.smem(T.nslots);
    b->wargs = args_for(ctx, b->d_texts, W, LW, static_cast<char*>(b->d_wmem), gw);
    b->wgrid = (uint32_t)W.cta_pbase.size();
    b->wsmem = gw.smem(W.nslots);
    b->d_pt = reinterpret_cast<const PatTiles*>(static_cast<char*>(b->d_wmem) + pt_off);
    return SM_OK;
}

extern "C" sm_status sm_batch_create(sm_ctx* ctx, const uint8_t* d_texts, const int64_t* h_text_off, uint32_t ntexts,
                                     const uint8_t* h_pats, const int64_t* h_pat_off, const int32_t* h_pat_text,
                                     uint32_t npats, sm_batch** out, sm_stream_t stream) {
    using namespace smk;
    if (!out) return sm_fail_internal(SM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx || !h_text_off || (npats && (!h_pats || !h_pat_off || !h_pat_text)))
        return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (ntexts == 0) return sm_fail_internal(SM_EINVAL, "no texts");
    if (h_text_off[0] != 0) return sm_fail_internal(SM_EINVAL, "h_text_off[0] must be 0");
    for (uint32_t x = 0; x < ntexts; ++x)
        if (h_text_off[x + 1] < h_text_off[x]) return sm_fail_internal(SM_EINVAL, "text offsets must not decrease");
    if (h_text_off[ntexts] && !d_texts) return sm_fail_internal(SM_EINVAL, "d_texts is NULL");
    for (uint32_t k = 0; k < npats; ++k) {
        const int64_t m = h_pat_off[k + 1] - h_pat_off[k];
        if (m < 1 || m > (int64_t)SM_MAX_M) return sm_fail_internal(SM_EINVAL, "pattern length out of range");
        if (h_pat_text[k] < 0 || (uint32_t)h_pat_text[k] >= ntexts)
            return sm_fail_internal(SM_EINVAL, "pattern refers to a missing text");
    }
    Guard guard(sm_ctx_device(ctx));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // 1. per-text histograms on the device
    std::vector<uint64_t> hist;
    const sm_status hs = text_histograms(ctx, d_texts, h_text_off, h_text_off + 1, ntexts, st, hist);
    if (hs != SM_OK) return hs;

    sm_batch* b = new sm_batch();
    b->ctx = ctx;
    b->device = sm_ctx_device(ctx);
    b->npats = npats;
    b->d_texts = d_texts;
    b->text_off.assign(h_text_off, h_text_off + ntexts + 1);
    b->pat_off.assign(h_pat_off, h_pat_off + npats + 1);
    b->pat_text.assign(h_pat_text, h_pat_text + npats);
    b->pats.assign(h_pats, h_pats + (npats ? h_pat_off[npats] : 0));
    b->hist = std::move(hist);
    const sm_status ps = build_plan(b);
    if (ps != SM_OK) {
        sm_batch_destroy(b);
        return ps;
    }
    *out = b;
    return SM_OK;
}

extern "C" sm_status sm_batch_count(sm_batch* b, int64_t* d_counts, sm_stream_t stream) {
    if (!b) return sm_fail_internal(SM_EINVAL, "batch is NULL");
    if (!d_counts && b->npats) return sm_fail_internal(SM_EINVAL, "d_counts is NULL");
    Guard g(b->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (b->npats) e = cudaMemsetAsync(d_counts, 0, (size_t)b->npats * sizeof(int64_t), st);
    if (e == cudaSuccess) {
        BatchArgs a = b->args;
        a.d_counts = d_counts;
        e = launch_batch(smk::kBatchCount, b->grid, b->smem, st, a);
    }
    return e == cudaSuccess ? SM_OK : sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
}

extern "C" sm_status sm_batch_report(sm_batch* b, int64_t* d_counts, uint64_t* d_pos, const int64_t* d_pos_off,
                                     sm_stream_t stream) {
    if (!b) return sm_fail_internal(SM_EINVAL, "batch is NULL");
    if (b->npats && (!d_counts || !d_pos_off)) return sm_fail_internal(SM_EINVAL, "d_counts or d_pos_off is NULL");
    Guard g(b->device);
    if (!b->d_tcnt && b->ntb) {   // the counters, once per batch
        if (cudaMalloc(&b->d_tcnt, b->ntb * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&b->d_toff, b->ntb * sizeof(uint64_t)) != cudaSuccess ||
            cudaMalloc(&b->d_hit, std::max<uint64_t>(b->nitems, 1)) != cudaSuccess) {
            cudaGetLastError();
            for (void* q : {(void*)b->d_tcnt, (void*)b->d_toff, (void*)b->d_hit})
                if (q) cudaFree(q);
            b->d_tcnt = nullptr;
            b->d_toff = nullptr;
            b->d_hit = nullptr;
            return sm_fail_internal(SM_ENOMEM, "report tile counters");
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    BatchArgs a1 = b->args, a2 = b->wargs;
    a1.d_counts = d_counts;
    a1.tcnt = b->d_tcnt;
    a2.toff = b->d_toff;
    a2.d_pos = d_pos;
    a2.pos_off = d_pos_off;
    a2.hit = b->d_hit;
    const cudaError_t e = run_report(a1, b->grid, b->smem, a2, b->wgrid, b->wsmem, b->d_pt, b->npats, b->d_tcnt,
                                     b->ntb, b->nitems, d_counts, b->npats, st);
    return e == cudaSuccess ? SM_OK : sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
}

extern "C" sm_status sm_batch_tune(sm_batch* b, uint32_t reps, sm_batch_tuning* best, sm_stream_t stream) {
    if (!b || !best) return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (reps < 1) reps = 1;
    Guard g(b->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t* d_counts = nullptr;
    if (cudaMalloc(&d_counts, std::max<size_t>(b->npats, 1) * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        return sm_fail_internal(SM_ENOMEM, "tuning counts");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // ms per count under the current plan: one warm-up launch, then reps
    auto time_plan = [&](float* ms) -> sm_status {
        sm_status s = sm_batch_count(b, d_counts, stream);
        if (s == SM_OK && cudaEventRecord(e0, st) != cudaSuccess) s = SM_ECUDA;
        for (uint32_t r = 0; s == SM_OK && r < reps; ++r) s = sm_batch_count(b, d_counts, stream);
        if (s == SM_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
            s = sm_fail_internal(SM_ECUDA, "tuning timer");
        *ms /= (float)reps;
        return s;
    };
    const BatchParams start = b->params;
    BatchParams top = start;
    float top_ms = 0;
    sm_status s = time_plan(&top_ms);
    for (const double f : {0.02, 0.04, 0.08, 0.16, 0.32})
        for (const uint32_t cm : {4u, 16u, 64u})
            for (const uint32_t stg : {2u, 3u, 4u}) {
                if (s != SM_OK) break;
                b->params = BatchParams{f, cm, stg};
                s = build_plan(b);
                float ms = 0;
                if (s == SM_OK) s = time_plan(&ms);
                if (s == SM_OK && ms < top_ms) {
                    top_ms = ms;
                    top = b->params;
                }
            }
    b->params = s == SM_OK ? top : start;
    const sm_status s2 = build_plan(b);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_counts);
    if (s != SM_OK) return s;
    if (s2 != SM_OK) return s2;
    best->cand_freq = (float)top.cand_freq;
    best->cand_min = top.cand_min;
    best->stages = top.stages;
    best->ms = top_ms;
    return SM_OK;
}

extern "C" void sm_batch_destroy(sm_batch* b) {
    if (!b) return;
    Guard g(b->device);
    cudaDeviceSynchronize();
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->d_wmem) cudaFree(b->d_wmem);
    if (b->d_tcnt) cudaFree(b->d_tcnt);
    if (b->d_toff) cudaFree(b->d_toff);
    if (b->d_hit) cudaFree(b->d_hit);
    delete b;
}

extern "C" sm_status sm_count_batch(sm_ctx* ctx, const uint8_t* d_texts, const int64_t* d_text_off, uint32_t ntexts,
                                    const uint8_t* d_pats, const int64_t* d_pat_off, const int32_t* d_pat_text,
                                    uint32_t npats, int64_t* d_counts, uint64_t* d_pos, const int64_t* d_pos_off,
                                    sm_stream_t stream) {
    if (!ctx || !d_text_off || ntexts == 0 || (npats && (!d_pats || !d_pat_off || !d_pat_text || !d_counts)))
        return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (d_pos && !d_pos_off) return sm_fail_internal(SM_EINVAL, "d_pos needs d_pos_off");
    Guard g(sm_ctx_device(ctx));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int64_t> text_off(ntexts + 1), pat_off(npats + 1);
    std::vector<int32_t> pat_text(npats);
    cudaError_t e = cudaMemcpyAsync(text_off.data(), d_text_off, text_off.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && npats) {
        e = cudaMemcpyAsync(pat_off.data(), d_pat_off, pat_off.size() * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pat_text.data(), d_pat_text, pat_text.size() * 4, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
    std::vector<uint8_t> pats(npats ? (size_t)std::max<int64_t>(pat_off[npats], 0) : 0);
    if (!pats.empty()) {
        e = cudaMemcpy(pats.data(), d_pats, pats.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
    }
    sm_batch* b = nullptr;
    sm_status s = sm_batch_create(ctx, d_texts, text_off.data(), ntexts, pats.data(), pat_off.data(),
                                  pat_text.data(), npats, &b, stream);
    if (s != SM_OK) return s;
    // positions: the batched report (ordered positions of every pattern into its slice of d_pos)
    s = d_pos ? sm_batch_report(b, d_counts, d_pos, d_pos_off, stream) : sm_batch_count(b, d_counts, stream);
    cudaStreamSynchronize(st);
    sm_batch_destroy(b);
    return s;
}

// ------------------------------------------------------------------ stepper
//
// Continuous batching over a device-resident text cut into chunks. Each step
// scans one chunk for every active query in one batch launch (the queries
// share the chunk's pass over HBM); a query that joins at chunk c is complete
// after one step on every chunk. Counts accumulate into the caller's
// per-query int64 counters. A step allocates nothing: its tables are built in
// one of two pinned host buffers and copied asynchronously to one of two
// device buffers, alternating, so that building step k+1 overlaps step k.

struct sm_stepper {
    sm_ctx* ctx = nullptr;
    int device = 0;
    const uint8_t* d_text = nullptr;
    uint64_t n = 0, chunk = 0;
    uint32_t nchunks = 0, max_m = 0, delta = 0;
    bool text7 = true;
    uint64_t hist[256] = {};      // the whole text's (reports, orders of the whole text)
    // chunks with the same set of symbols form a class; a query is
    // described once per class under the class's frequencies, and a chunk
    // without one of its symbols is not scanned for it
    std::vector<uint32_t> chunk_class;
    std::vector<std::vector<uint64_t>> class_hist;
    std::vector<uint64_t> class_n;
    std::vector<bool> class_text7;
    std::vector<uint32_t> class_codes;   // BatchText::codes of the class (2-bit codes or bytes)
    Geometry geo[2][2];   // steps [with the candidate index][with 2-bit codes] (any active set)
    std::unordered_map<uint32_t, std::vector<PatDesc>> queries;   // one per class
    struct Buf {
        char* d = nullptr;
        char* h = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
        bool used = false;
    } buf[2], rbuf;            // step tables (alternating); report tables
    int cur = 0;
    uint32_t* d_tcnt = nullptr;   // report counters
    uint64_t* d_toff = nullptr;
    uint64_t rcap = 0;
    uint8_t* d_hit = nullptr;     // report: tiles with matches
    uint64_t hcap = 0;
};

namespace {

// Grows a table buffer (pinned host staging and its device copy) to `need` bytes.
bool grow_buf(sm_stepper::Buf& b, size_t need) {
    if (b.cap >= need) return true;
    const size_t cap = std::max(need, 2 * b.cap);
    if (b.h) cudaFreeHost(b.h);
    if (b.d) cudaFree(b.d);
    b.h = nullptr;
    b.d = nullptr;
    b.cap = 0;
    if (cudaMallocHost(&b.h, cap) != cudaSuccess || cudaMalloc(&b.d, cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    b.cap = cap;
    return true;
}

}  // namespace

extern "C" sm_status sm_stepper_create(sm_ctx* ctx, const uint8_t* d_text, uint64_t n, uint64_t chunk_bytes,
                                       uint32_t max_m, const uint64_t* h_hist256, sm_stepper** out) {
    if (!out) return sm_fail_internal(SM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx || !h_hist256 || (!d_text && n)) return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (max_m < 1 || max_m > SM_MAX_M) return sm_fail_internal(SM_EINVAL, "max_m out of range");
    if (chunk_bytes < smk::kTile || chunk_bytes % smk::kTile)
        return sm_fail_internal(SM_EINVAL, "chunk_bytes must be a positive multiple of SM_TILE_STARTS");
    Guard g(sm_ctx_device(ctx));
    sm_stepper* s = new sm_stepper();
    s->ctx = ctx;
    s->device = sm_ctx_device(ctx);
    s->d_text = d_text;
    s->n = n;
    s->chunk = chunk_bytes;
    s->nchunks = (uint32_t)((n + chunk_bytes - 1) / chunk_bytes);
    s->max_m = max_m;
    s->delta = (uint32_t)(reinterpret_cast<uintptr_t>(d_text) & 15u);
    for (int c = 0; c < 256; ++c) s->hist[c] = h_hist256[c];
    s->text7 = text_is_7bit(s->hist);
    {   // histograms of each chunk with its halo (a query's matches in the
        // chunk can read max_m - 1 bytes past it) -> classes of chunks with
        // equal symbol sets
        std::vector<int64_t> beg(s->nchunks), end(s->nchunks);
        for (uint32_t c = 0; c < s->nchunks; ++c) {
            beg[c] = (int64_t)((uint64_t)c * chunk_bytes);
            end[c] = (int64_t)std::min<uint64_t>((uint64_t)(c + 1) * chunk_bytes + max_m - 1, n);
        }
        std::vector<int64_t> off(s->nchunks + 1);
        for (uint32_t c = 0; c <= s->nchunks; ++c) off[c] = (int64_t)std::min<uint64_t>((uint64_t)c * chunk_bytes, n);
        std::vector<uint64_t> ch;
        const sm_status hs =
            s->nchunks ? text_histograms(ctx, d_text, beg.data(), end.data(), s->nchunks, nullptr, ch) : SM_OK;
        if (hs != SM_OK) {
            delete s;
            return hs;
        }
        std::vector<std::vector<uint64_t>> keys;   // symbol-set bitmaps of the classes
        for (uint32_t c = 0; c < s->nchunks; ++c) {
            std::vector<uint64_t> key(4, 0);
            for (int b = 0; b < 256; ++b)
                if (ch[(size_t)c * 256 + b]) key[b >> 6] |= 1ull << (b & 63);
            uint32_t k = 0;
            while (k < keys.size() && keys[k] != key) ++k;
            if (k == keys.size()) {
                keys.push_back(key);
                s->class_hist.emplace_back(256, 0);
                s->class_n.push_back(0);
            }
            for (int b = 0; b < 256; ++b) s->class_hist[k][b] += ch[(size_t)c * 256 + b];
            s->class_n[k] += (uint64_t)(off[c + 1] - off[c]);
            s->chunk_class.push_back(k);
        }
        for (auto& h : s->class_hist) {
            s->class_text7.push_back(text_is_7bit(h.data()));
            s->class_codes.push_back(text_codes(h.data()));
        }
    }
    for (int ix = 0; ix < 2; ++ix)
        for (int pk = 0; pk < 2; ++pk) s->geo[ix][pk] = geometry(ctx, max_m, ix == 1, kMaxSlots, 0, pk == 1);
    for (auto* b : {&s->buf[0], &s->buf[1], &s->rbuf})
        if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            sm_stepper_destroy(s);
            return sm_fail_internal(SM_ECUDA, "event");
        }
    *out = s;
    return SM_OK;
}

extern "C" uint32_t sm_stepper_chunks(const sm_stepper* s) { return s ? s->nchunks : 0; }

extern "C" sm_status sm_stepper_admit(sm_stepper* s, uint32_t qid, const uint8_t* h_pat, uint32_t m) {
    if (!s || !h_pat) return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (m < 1 || m > s->max_m) return sm_fail_internal(SM_EINVAL, "pattern length out of range for this stepper");
    // orders under each chunk class's frequencies (counts never depend on them)
    std::vector<PatDesc>& d = s->queries[qid];
    d.clear();
    for (size_t k = 0; k < s->class_hist.size(); ++k)
        d.push_back(describe(h_pat, m, s->class_hist[k].data(), s->class_n[k], s->delta, s->class_text7[k], qid,
                             smk::kCandidateFreq, s->class_codes[k]));
    return SM_OK;
}

extern "C" sm_status sm_stepper_retire(sm_stepper* s, uint32_t qid) {
    if (!s) return sm_fail_internal(SM_EINVAL, "stepper is NULL");
    s->queries.erase(qid);
    return SM_OK;
}

extern "C" sm_status sm_stepper_steps(sm_stepper* s, const uint32_t* h_qids, const uint32_t* h_nchunks, uint32_t nq,
                                      uint32_t chunk, int64_t* d_counts, sm_stream_t stream) {
    if (!s || (nq && (!h_qids || !d_counts))) return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (chunk >= s->nchunks) return sm_fail_internal(SM_EINVAL, "chunk out of range");
    Guard g(s->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<const std::vector<PatDesc>*> qd(nq);
    uint32_t span = nq ? 1u : 0u;   // chunks scanned: the most any query asks for
    for (uint32_t i = 0; i < nq; ++i) {
        auto it = s->queries.find(h_qids[i]);
        if (it == s->queries.end()) return sm_fail_internal(SM_EINVAL, "query not admitted");
        qd[i] = &it->second;
        if (h_nchunks) {
            if (h_nchunks[i] > s->nchunks) return sm_fail_internal(SM_EINVAL, "more chunks than the text has");
            span = std::max(span, h_nchunks[i]);
        }
    }
    // one entry per chunk (chunk, chunk + 1, ... wrapping), each with the
    // queries that still want it, described for the chunk's class
    Tables T;
    std::vector<const PatDesc*> ds;
    ds.reserve(nq);
    for (uint32_t k = 0; k < span; ++k) {
        const uint32_t c = (chunk + k) % s->nchunks;
        const uint64_t off = (uint64_t)c * s->chunk;
        const uint64_t avail = s->n - off;                          // bytes from the chunk start
        const uint64_t nbytes = std::min<uint64_t>(avail, s->chunk + s->max_m - 1);
        const uint64_t slimit = std::min<uint64_t>(avail, s->chunk);
        ds.clear();
        for (uint32_t i = 0; i < nq; ++i) {
            if (h_nchunks && h_nchunks[i] <= k) continue;
            const PatDesc& d = (*qd[i])[s->chunk_class[c]];
            if (d.zero || d.pat.m > nbytes) continue;   // a symbol absent from the chunk, or no start in it
            ds.push_back(&d);
        }
        if (!ds.empty())
            add_text(T, off, nbytes, slimit, ds, true, nullptr, nullptr, smk::kCandidateMin,
                     s->class_codes[s->chunk_class[c]]);
    }
    if (T.tx.empty()) return SM_OK;
    const Geometry& geo = s->geo[T.need_index ? 1 : 0][T.need_pack ? 1 : 0];
    finish(T, (uint64_t)sm_ctx_num_sms(s->ctx) * geo.occ);
    const Layout L = layout_of(T);
    sm_stepper::Buf& b = s->buf[s->cur];
    s->cur ^= 1;
    if (b.used && cudaEventSynchronize(b.ev) != cudaSuccess) return sm_fail_internal(SM_ECUDA, "event wait");
    if (!grow_buf(b, L.total)) return sm_fail_internal(SM_ENOMEM, "stepper tables");
    pack(T, L, b.h);
    cudaError_t e = cudaMemcpyAsync(b.d, b.h, L.total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        BatchArgs a = args_for(s->ctx, s->d_text, T, L, b.d, geo);
        a.d_counts = d_counts;
        e = launch_batch(smk::kBatchCount, (uint32_t)T.cta_pbase.size(), geo.smem(T.nslots), st, a);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b.ev, st);
    b.used = true;
    return e == cudaSuccess ? SM_OK : sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
}

extern "C" sm_status sm_stepper_step(sm_stepper* s, const uint32_t* h_qids, uint32_t nq, uint32_t chunk,
                                     int64_t* d_counts, sm_stream_t stream) {
    return sm_stepper_steps(s, h_qids, nullptr, nq, chunk, d_counts, stream);
}

extern "C" sm_status sm_stepper_report(sm_stepper* s, const uint8_t* h_pats, const int64_t* h_pat_off, uint32_t nq,
                                       const int64_t* h_pos_off, uint64_t* d_pos, int64_t* d_counts,
                                       sm_stream_t stream) {
    if (!s || (nq && (!h_pats || !h_pat_off || !h_pos_off || !d_counts))) return sm_fail_internal(SM_EINVAL, "NULL argument");
    if (nq && h_pos_off[nq] > h_pos_off[0] && !d_pos) return sm_fail_internal(SM_EINVAL, "d_pos is NULL");
    for (uint32_t k = 0; k < nq; ++k) {
        const int64_t m = h_pat_off[k + 1] - h_pat_off[k];
        if (m < 1 || m > (int64_t)SM_MAX_M) return sm_fail_internal(SM_EINVAL, "pattern length out of range");
        if (h_pos_off[k + 1] < h_pos_off[k]) return sm_fail_internal(SM_EINVAL, "position offsets must not decrease");
    }
    if (!nq) return SM_OK;
    Guard g(s->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // the previous report's tables and counters are reused
    if (s->rbuf.used && cudaEventSynchronize(s->rbuf.ev) != cudaSuccess) return sm_fail_internal(SM_ECUDA, "event wait");
    std::vector<PatDesc> descs(nq);
    std::vector<const PatDesc*> ptrs(nq);
    std::vector<uint32_t> ms(nq);
    std::vector<uint64_t> lens(nq, s->n);
    for (uint32_t k = 0; k < nq; ++k) {
        ms[k] = (uint32_t)(h_pat_off[k + 1] - h_pat_off[k]);
        descs[k] = describe(h_pats + h_pat_off[k], ms[k], s->hist, s->n, s->delta, s->text7, k,
                            smk::kCandidateFreq, text_codes(s->hist));
        ptrs[k] = &descs[k];
    }
    std::vector<PatTiles> pt;
    std::vector<uint64_t> tb;
    const uint64_t ntb = assign_tiles(ms, lens, pt, tb);
    Tables T, W;
    const uint32_t codes = text_codes(s->hist);
    add_text(T, 0, s->n, ~0ull, ptrs, true, &tb, nullptr, smk::kCandidateMin, codes);
    add_text(W, 0, s->n, ~0ull, ptrs, false, &tb, &pt, smk::kCandidateMin, codes);
    const Geometry g1 = geometry(s->ctx, std::max(T.maxm, 1u), T.need_index, T.slot_hint(), 0, T.need_pack);
    finish(T, (uint64_t)sm_ctx_num_sms(s->ctx) * g1.occ);
    const Geometry g2 = geometry(s->ctx, std::max(W.maxm, 1u), false, W.slot_hint(), 0, W.need_pack);
    finish(W, (uint64_t)sm_ctx_num_sms(s->ctx) * g2.occ);
    const Layout L = layout_of(T), LW = layout_of(W);
    const size_t o_w = L.total, o_pt = o_w + LW.total, o_po = o_pt + ((pt.size() * sizeof(PatTiles) + 255) & ~(size_t)255);
    const size_t total = o_po + (size_t)(nq + 1) * sizeof(int64_t);
    if (!grow_buf(s->rbuf, total)) return sm_fail_internal(SM_ENOMEM, "report tables");
    if (s->rcap < ntb) {
        const uint64_t cap = std::max<uint64_t>(ntb, 2 * s->rcap);
        if (s->d_tcnt) cudaFree(s->d_tcnt);
        if (s->d_toff) cudaFree(s->d_toff);
        s->d_tcnt = nullptr;
        s->d_toff = nullptr;
        s->rcap = 0;
        if (cudaMalloc(&s->d_tcnt, cap * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s->d_toff, cap * sizeof(uint64_t)) != cudaSuccess) {
            cudaGetLastError();
            return sm_fail_internal(SM_ENOMEM, "report tile counters");
        }
        s->rcap = cap;
    }
    if (s->hcap < std::max<uint64_t>(W.items, 1)) {
        const uint64_t cap = std::max<uint64_t>(std::max<uint64_t>(W.items, 1), 2 * s->hcap);
        if (s->d_hit) cudaFree(s->d_hit);
        s->d_hit = nullptr;
        s->hcap = 0;
        if (cudaMalloc(&s->d_hit, cap) != cudaSuccess) {
            cudaGetLastError();
            return sm_fail_internal(SM_ENOMEM, "report tile flags");
        }
        s->hcap = cap;
    }
    char* h = s->rbuf.h;
    char* d = s->rbuf.d;
    pack(T, L, h);
    pack(W, LW, h + o_w);
    std::memcpy(h + o_pt, pt.data(), pt.size() * sizeof(PatTiles));
    for (uint32_t k = 0; k <= nq; ++k) reinterpret_cast<int64_t*>(h + o_po)[k] = h_pos_off[k] - h_pos_off[0];
    cudaError_t e = cudaMemcpyAsync(d, h, total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        BatchArgs a1 = args_for(s->ctx, s->d_text, T, L, d, g1);
        BatchArgs a2 = args_for(s->ctx, s->d_text, W, LW, d + o_w, g2);
        a1.d_counts = d_counts;
        a1.tcnt = s->d_tcnt;
        a2.toff = s->d_toff;
        a2.d_pos = d_pos ? d_pos + h_pos_off[0] : nullptr;
        a2.pos_off = reinterpret_cast<const int64_t*>(d + o_po);
        a2.hit = s->d_hit;
        e = run_report(a1, (uint32_t)T.cta_pbase.size(), g1.smem(T.nslots), a2, (uint32_t)W.cta_pbase.size(),
                       g2.smem(W.nslots), reinterpret_cast<const PatTiles*>(d + o_pt), nq, s->d_tcnt, ntb, W.items,
                       d_counts, nq, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->rbuf.ev, st);
    s->rbuf.used = true;
    return e == cudaSuccess ? SM_OK : sm_fail_internal(SM_ECUDA, cudaGetErrorString(e));
}

extern "C" void sm_stepper_destroy(sm_stepper* s) {
    if (!s) return;
    Guard g(s->device);
    cudaDeviceSynchronize();
    for (auto* b : {&s->buf[0], &s->buf[1], &s->rbuf}) {
        if (b->h) cudaFreeHost(b->h);
        if (b->d) cudaFree(b->d);
        if (b->ev) cudaEventDestroy(b->ev);
    }
    if (s->d_tcnt) cudaFree(s->d_tcnt);
    if (s->d_toff) cudaFree(s->d_toff);
    if (s->d_hit) cudaFree(s->d_hit);
    delete s;
}
