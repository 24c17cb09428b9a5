// Kernels of the SIMD-naive search (Tarhio, Holub, Giaquinta, Sec. 2), for sm_103a.
//
// scan_kernel  - Algorithms 2-4 on the GPU. A CTA runs nine warps: one
//                producer and eight consumers, over tiles of kTile = 16384
//                start positions. In the counting modes CTAs claim tiles one
//                at a time from a global counter, so that the CTAs that run
//                faster take more tiles and all finish together; in the
//                write mode CTA b owns the contiguous tile range b.
//
//   Producer (warp 8): for each tile, waits until the consumers have
//   released a ring slot (mbarrier `empty`), loads the at most 30 bytes of
//   the tile that lie outside the text's 16-byte-aligned interior, and starts
//   a 1-D TMA bulk copy (cp.async.bulk, no multicast) of the rest of the
//   tile plus its (m-1)-byte halo into the slot, completing mbarrier `full`.
//
//   Consumer warp w owns starts [2048w, 2048w + 2048) of the tile; lane l
//   owns the 16-start chunks at 2048w + 512c + 16l, c = 0..3, so each
//   16-byte shared-memory load of a warp covers 512 consecutive bytes. The
//   paper's SIMDcompare for pattern position q and symbol c is computed for
//   16 starts s at a time: two 16-byte loads cover bytes s+q .. s+q+19,
//   funnel shifts align them, and w ^ c..c is zero in exactly the bytes that
//   match. Compares are ANDed by OR-ing these XORs: one exact SWAR zero-byte
//   test of the OR leaves the AND of their results in the high bit of each
//   byte ("found", four starts per 32-bit word).
//
//   Dense phase: the first r compares (in the order pi) run for every start
//   with no zero test - the loop peeling of Sec. 2.3.
//   Sparse phase: the 16-start chunks with a surviving start are compacted,
//   in position order, into a per-warp queue in shared memory; each lane
//   then continues one chunk through compares r .. m-1 and leaves as soon as
//   the chunk's found bits are zero - the early exit of Algorithm 2, taken
//   per 16-start chunk instead of per SIMD register. popcount(found) is the
//   count (Algorithm 2); the reporting modes write the set bits' positions.
//
// hist_kernel  - byte histogram of the text (the frequencies of Sec. 2.2).
//
// Every wait on an mbarrier is bounded by a %globaltimer deadline; on expiry
// the kernel records kStatusTimeout, the producer waits (bounded) for the
// copies it started, and every warp leaves its loop.
#include "sm_device.cuh"

namespace smk {
namespace {

using namespace dev;


// Warp w's first rank within its tile, from a write-list entry's eight
// 16-bit warp offsets (a tile holds at most 16384 matches before warp 7).
__device__ __forceinline__ uint32_t warp_offset(const uint4& wo, uint32_t w) {
    const uint32_t x = w < 4 ? (w < 2 ? wo.x : wo.y) : (w < 6 ? wo.z : wo.w);
    return (x >> (16u * (w & 1u))) & 0xFFFFu;
}

struct StageDesc {
    uint64_t tile;       // kEnd: no more tiles
    uint64_t offset;     // report: output offset of the tile's first match
};

// ------------------------------------------------------------ scan kernel

#ifndef SMK_MIN_BLOCKS
#define SMK_MIN_BLOCKS 3
#endif
template <int MAXM, int MODE, int KIND>
__global__ void __launch_bounds__(kThreads, SMK_MIN_BLOCKS) scan_kernel(const __grid_constant__ ScanArgs A,
                                                        const __grid_constant__ PatArg<MAXM> P) {
    constexpr bool SEVEN = KIND == kKindSeven;
    constexpr bool PACKED = KIND >= kKindPackedAdj;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);                  // [kMaxStages]
    uint64_t* empty = reinterpret_cast<uint64_t*>(smem + 64);            // [kMaxStages]
    StageDesc* desc = reinterpret_cast<StageDesc*>(smem + 128);          // [kMaxStages]
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + 256);             // [kConsumerWarps + 1]
    uint32_t* flag = reinterpret_cast<uint32_t*>(smem + 336);
    uint32_t* queues = reinterpret_cast<uint32_t*>(smem + kScanHeader);  // [kConsumerWarps][kQueueCap]
    uint32_t* pbuf = reinterpret_cast<uint32_t*>(smem + kScanHeader);    // packed: [2][2][A.packed_words]
    uint32_t* sbms = reinterpret_cast<uint32_t*>(smem + kScanHeader + kQueueBytes);   // bytes, tile-count
    uint8_t* bufs = smem + kScanHeader +
                    (PACKED ? 16u * A.packed_words : kQueueBytes + (MODE == kModeTileCount ? kBitmapBytes : 0u));
    // write mode with range sums: the range's tiles with matches, after the stages
    uint4* wl_woff = reinterpret_cast<uint4*>(bufs + (size_t)A.stages * A.stage_bytes);   // [kWriteList]
    uint2* wl_head = reinterpret_cast<uint2*>(wl_woff + kWriteList);                    // [kWriteList]
    uint32_t* wl_n = reinterpret_cast<uint32_t*>(smem + 352);                            // [kConsumerWarps + 2]

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t SB = A.stage_bytes, S = A.stages, m = A.m, r = A.r, one = A.one;
    const uint64_t t_begin = (uint64_t)blockIdx.x * A.tiles_per_cta;
    const uint64_t t_end = min(t_begin + A.tiles_per_cta, A.ntiles);

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        fence_mbar_init();
    }
    if (MODE == kModeWrite) {
        // first rank of the range: the counts of the earlier ranges, summed
        // by all threads (block 0 sums every range instead, for the
        // truncation flag); the producer adds up the warps' sums
        const uint32_t upto = blockIdx.x == 0 ? gridDim.x : blockIdx.x;
        const uint64_t* sums = A.range_sums ? A.range_sums : A.partials;
        uint64_t v = 0;
        for (uint32_t i = tid; i < upto; i += kThreads) v += __ldcg(sums + i);
        v = warp_sum_u64(v);
        if (lane == 0) red[warp] = v;
        if (A.range_sums) {
            // thread i: tile t_begin + i -> its matches and warp offsets; the
            // tiles with matches are listed in order (warp ballots, then the
            // warps' list lengths), and their count words cleared
            const uint64_t tt = t_begin + tid;
            uint32_t tot = 0;
            uint4 wo = make_uint4(0u, 0u, 0u, 0u);
            if (tt < t_end) {
                uint4* src = reinterpret_cast<uint4*>(A.warp_counts + tt * kConsumerWarps);
                const uint4 x = __ldcg(src), y = __ldcg(src + 1);
                const uint32_t c[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
                uint32_t o[8];
#pragma unroll
                for (int w = 0; w < kConsumerWarps; ++w) {
                    o[w] = tot;
                    tot += c[w] & kCountMask;
                }
                wo = make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16), o[6] | (o[7] << 16));
                if (tot) {
                    src[0] = make_uint4(0u, 0u, 0u, 0u);
                    src[1] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
            const uint32_t bal = __ballot_sync(kFull, tot != 0u);
            if (lane == 0) wl_n[warp] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, all = 0;
            for (int w = 0; w < kConsumerWarps + 1; ++w) {
                before += w < (int)warp ? wl_n[w] : 0u;
                all += wl_n[w];
            }
            if (tot) {
                const uint32_t k = before + __popc(bal & ((1u << lane) - 1u));
                wl_woff[k] = wo;
                wl_head[k] = make_uint2((uint32_t)tt, tot);
            }
            if (tid == 0) wl_n[kConsumerWarps + 1] = all;
        }
    }
    __syncthreads();

    uint32_t my_count = 0;

    if (warp == kConsumerWarps) {
        // ---------------------------------------------------------- producer
        uint64_t cursor = t_begin, running = 0;
        if (MODE == kModeWrite) {
            uint64_t b = 0;
            for (int w = 0; w < kConsumerWarps + 1; ++w) b += red[w];
            running = blockIdx.x == 0 ? 0 : b;
            if (blockIdx.x == 0 && lane == 0 && b > A.cap) atomicOr(A.status, kStatusTrunc);
        }
        uint32_t issued = 0;
        // counting modes: the claim of the next tile is in flight while the
        // producer waits for a free slot
        unsigned long long claim = 0;
        if (MODE != kModeWrite && lane == 0) claim = atomicAdd(A.tile_next, 1ull);
        // stage s and use count u of the ring for iteration it, kept without division
        for (uint32_t it = 0, s = 0, u = 0;; ++it) {
            if (u > 0) {
                const bool ok = __all_sync(kFull, wait_bounded(&empty[s], (u - 1) & 1u, A.spin_ns));
                if (!ok) {
                    if (lane == 0) atomicOr(A.status, kStatusTimeout);
                    break;
                }
            }
            uint64_t tile = kEnd;
            uint32_t tcount = 0;
            if (MODE != kModeWrite) {
                const uint64_t t = __shfl_sync(kFull, claim, 0);
                if (t < A.ntiles) {
                    tile = t;
                    if (lane == 0) claim = atomicAdd(A.tile_next, 1ull);
                }
            } else if (A.range_sums) {
                // next entry of the range's list of tiles with matches
                // (cursor counts the entries taken)
                const uint32_t i = (uint32_t)(cursor - t_begin);
                if (i < wl_n[kConsumerWarps + 1]) {   // the list's length
                    const uint2 h = wl_head[i];
                    tile = h.x;
                    tcount = h.y;
                    ++cursor;
                }
            } else {
                // next tile with matches; lanes look at 4 tiles x 8 warp counts per step
                while (cursor < t_end) {
                    const uint64_t t = cursor + (lane >> 3);
                    uint32_t c =
                        t < t_end ? __ldcg(A.warp_counts + t * kConsumerWarps + (lane & 7u)) & kCountMask : 0u;
                    c += __shfl_xor_sync(kFull, c, 1);
                    c += __shfl_xor_sync(kFull, c, 2);
                    c += __shfl_xor_sync(kFull, c, 4);
                    const uint32_t bal = __ballot_sync(kFull, c != 0 && (lane & 7u) == 0);
                    if (bal) {
                        const int k = __ffs(bal) - 1;
                        tcount = __shfl_sync(kFull, c, k);
                        tile = cursor + (uint64_t)(k >> 3);
                        cursor = tile + 1;
                        break;
                    }
                    cursor += 4;
                }
            }
            uint8_t* buf = bufs + (size_t)s * SB;
            TileCopy cp{0, 0, 0};
            if (tile != kEnd) {
                const uint64_t s0 = tile * kTile;
                cp = stage_ragged(buf, A.text, A.n, s0, min(s0 + kTile + m - 1, A.n), lane);
            }
            __syncwarp();
            if (lane == 0) {
                desc[s].tile = tile;
                desc[s].offset = running;
                const bool skip = A.test_skip_copy && tile == 0;
                fence_proxy_async();
                mbar_arrive_expect_tx(&full[s], cp.bytes);
                if (cp.bytes && !skip)
                    bulk_g2s(buf + cp.dst_off, reinterpret_cast<const void*>(cp.src), cp.bytes, &full[s]);
            }
            issued = it + 1;
            if (tile == kEnd) break;
            running += tcount;
            if (++s == S) {
                s = 0;
                ++u;
            }
        }
        // let every copy this CTA started land before the CTA can leave: the
        // last use of each stage is use (issued - 1 - stage) / S (if any)
        if (lane == 0)
            for (uint32_t st = 0; st < S && st < issued; ++st)
                (void)wait_bounded(&full[st], ((issued - 1 - st) / S) & 1u, A.spin_ns);
        __syncwarp();
    } else if constexpr (PACKED) {
        // ------------------------------------------- consumers, 2-bit codes
        // Rounds of two tiles: every consumer thread packs its 16-byte units
        // of each tile's stage into a packed buffer and releases the stage;
        // one consumer barrier (which also agrees on leaving) makes the
        // packed tiles visible; then each warp compares its 2048 starts of
        // both tiles at once. The buffer pair of a round is rewritten two
        // rounds later, after every warp has passed the next round's
        // barrier, i.e. finished comparing.
        constexpr bool ADJ = KIND == kKindPackedAdj;
        constexpr bool BIN = KIND == kKindBinary;   // 1-bit codes
        constexpr uint32_t UB = BIN ? 32u : 16u;    // stage bytes per packed word
        const uint32_t units = SB / UB, b1 = A.b1, b2 = A.b2, gather = A.gather, PW = A.packed_words;
        const uint32_t u0 = warp * (kWarpStarts / UB) + lane;
        for (uint32_t s = 0, phase = 0, t = 0;; ++t) {   // round t: list entries 2t, 2t + 1 (write mode)
            uint32_t* pw[2] = {pbuf + (t & 1u) * 2u * PW, pbuf + (t & 1u) * 2u * PW + PW};
            StageDesc d[2] = {{kEnd, 0}, {kEnd, 0}};
            bool ok = true;
            uint32_t ss = s, ph = phase;
            for (int k = 0; k < 2; ++k) {
                ok = __all_sync(kFull, wait_bounded(&full[ss], ph, A.spin_ns));
                if (!ok) break;
                d[k] = desc[ss];
                if (d[k].tile == kEnd) break;
                const uint4* b4 = reinterpret_cast<const uint4*>(bufs + (size_t)ss * SB);
                if constexpr (BIN) {
                    uint4 x[4];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        x[2 * c] = b4[2 * (u0 + 32 * c)];
                        x[2 * c + 1] = b4[2 * (u0 + 32 * c) + 1];
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c) pw[k][u0 + 32 * c] = pack32(x[2 * c], x[2 * c + 1], b1);
                    for (uint32_t u = kTile / 32 + tid; u < units; u += kConsumerWarps * 32)
                        pw[k][u] = pack32(b4[2 * u], b4[2 * u + 1], b1);
                } else {
                    uint4 x[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) x[c] = b4[u0 + 32 * c];
#pragma unroll
                    for (int c = 0; c < 4; ++c) pw[k][u0 + 32 * c] = pack16<ADJ>(x[c], b1, b2, gather);
                    for (uint32_t u = kTile / 16 + tid; u < units; u += kConsumerWarps * 32)
                        pw[k][u] = pack16<ADJ>(b4[u], b1, b2, gather);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[ss]);
                if (++ss == S) {
                    ss = 0;
                    ph ^= 1u;
                }
            }
            if (consumers_any(!ok)) {
                if (lane == 0 && !ok) atomicOr(A.status, kStatusTimeout);
                break;
            }
            if (d[0].tile == kEnd) break;
            const bool two = d[1].tile != kEnd;
            const uint64_t s0[2] = {d[0].tile * kTile, two ? d[1].tile * kTile : 0};
            uint64_t out[2] = {0, 0};
            if (MODE == kModeWrite) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (k == 0 || two) {
                        if (A.range_sums) {
                            out[k] = d[k].offset + warp_offset(wl_woff[2 * t + k], warp);
                        } else {
                            const uint32_t cw = lane < warp
                                ? __ldcg(A.warp_counts + d[k].tile * kConsumerWarps + lane) & kCountMask : 0u;
                            out[k] = d[k].offset + warp_sum_u32(cw);
                        }
                    }
            }
            const uint32_t* const pk[2] = {pw[0], two ? pw[1] : pw[0]};
            uint32_t* const bm[2] = {
                MODE == kModeTileCount && A.bitmaps
                    ? A.bitmaps + (d[0].tile * kConsumerWarps + warp) * kBitmapWords : nullptr,
                MODE == kModeTileCount && A.bitmaps && two
                    ? A.bitmaps + (d[1].tile * kConsumerWarps + warp) * kBitmapWords : nullptr};
            uint2 c;
            uint32_t ent[2] = {0u, 0u};
            if constexpr (BIN)
                c = binary_tiles<MODE == kModeWrite, MODE != kModeWrite>(pk, two, warp, lane, ParamQC<MAXM>{&P}, m, r,
                                                                         A.ng, A.nstarts, s0, out, A.d_pos, A.cap, bm,
                                                                         ent);
            else
                c = packed_tiles<MODE == kModeWrite, MODE != kModeWrite>(pk, two, warp, lane, ParamQC<MAXM>{&P}, m, r,
                                                                         A.ng, A.nstarts, s0, out, A.d_pos, A.cap, bm,
                                                                         ent);
            if (MODE == kModeTileCount || MODE == kModeSparse) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && !two) break;
                    const uint32_t wsum = warp_sum_u32(k == 0 ? c.x : c.y);
                    if (lane == 0 && (MODE == kModeTileCount || wsum)) {
                        A.warp_counts[d[k].tile * kConsumerWarps + warp] = wsum | (ent[k] << 16);
                        if (MODE == kModeSparse && A.range_sums)
                            atomicAdd(reinterpret_cast<unsigned long long*>(A.range_sums + d[k].tile / A.range_tiles),
                                      (unsigned long long)wsum);
                    }
                }
            }
            my_count += c.x + c.y;
            if (!two) break;   // the second slot held the end mark
            s = ss;
            phase = ph;
        }
    } else {
        // ---------------------------------------------------------- consumers
        uint32_t* q = queues + warp * kQueueCap;
        const uint32_t c0 = warp * (kWarpStarts / 16) + lane;   // lane's first 16-byte chunk in the tile
        const uint32_t wq = warp * (kWarpStarts / 4);           // warp's first word in the tile
        for (uint32_t s = 0, phase = 0, li = 0;; ++li) {   // li: the tile's list entry (write mode)
            const bool ok = __all_sync(kFull, wait_bounded(&full[s], phase, A.spin_ns));
            if (!ok) {
                if (lane == 0) atomicOr(A.status, kStatusTimeout);
                break;
            }
            const StageDesc d = desc[s];
            if (d.tile == kEnd) break;
            const uint8_t* buf = bufs + (size_t)s * SB;
            const uint4* b4 = reinterpret_cast<const uint4*>(buf);
            const uint32_t* b32 = reinterpret_cast<const uint32_t*>(buf);
            const uint64_t s0 = d.tile * kTile;

            uint64_t out = 0;
            if (MODE == kModeWrite) {
                if (A.range_sums) {
                    out = d.offset + warp_offset(wl_woff[li], warp);
                } else {
                    const uint32_t cw =
                        lane < warp ? __ldcg(A.warp_counts + d.tile * kConsumerWarps + lane) & kCountMask : 0u;
                    out = d.offset + warp_sum_u32(cw);
                }
            }
            uint32_t* bm = MODE == kModeTileCount && A.bitmaps
                               ? A.bitmaps + (d.tile * kConsumerWarps + warp) * kBitmapWords : nullptr;
            uint32_t ent = 0;
            const uint32_t tile_count = warp_tile<SEVEN, MODE == kModeWrite, MODE != kModeWrite>(
                b4, b32, c0, wq, warp, lane, ParamQC<MAXM>{&P}, m, r, A.ng, one,
                A.nstarts, s0, q, out, A.d_pos, A.cap, bm, sbms + warp * kBitmapWords, &ent);

            if (MODE == kModeTileCount) {
                const uint32_t wsum = warp_sum_u32(tile_count);
                if (lane == 0) A.warp_counts[d.tile * kConsumerWarps + warp] = wsum | (ent << 16);
            } else if (MODE == kModeSparse) {
                if (__any_sync(kFull, tile_count != 0u)) {
                    const uint32_t wsum = warp_sum_u32(tile_count);
                    if (lane == 0) {
                        A.warp_counts[d.tile * kConsumerWarps + warp] = wsum;
                        if (A.range_sums)
                            atomicAdd(reinterpret_cast<unsigned long long*>(A.range_sums + d.tile / A.range_tiles),
                                      (unsigned long long)wsum);
                    }
                }
            }
            my_count += tile_count;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (++s == S) {
                s = 0;
                phase ^= 1u;
            }
        }
    }

    if (MODE == kModeWrite) {
        if (A.range_sums) {
            // every CTA has read the range sums: the last one clears them
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const uint32_t tk = atomicAdd(A.ticket, 1u);
                *flag = (tk == gridDim.x - 1) ? 1u : 0u;
            }
            __syncthreads();
            if (*flag) {
                __threadfence();
                for (uint32_t i = tid; i < gridDim.x; i += kThreads) A.range_sums[i] = 0ull;
                if (tid == 0) *A.ticket = 0u;
            }
        }
        return;
    }

    // CTA total -> partials; the last CTA to finish writes the sum and
    // clears the ticket and the tile counter for the next launch. (A
    // found-bit report then overwrites the partials with per-range counts:
    // range_sum_kernel.)
    const uint64_t ws = warp_sum_u64((uint64_t)my_count);
    if (lane == 0) red[warp] = ws;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        uint64_t tot = 0;
        for (int w = 0; w < kConsumerWarps + 1; ++w) tot += red[w];
        A.partials[blockIdx.x] = tot;
        __threadfence();
        const uint32_t t = atomicAdd(A.ticket, 1u);
        *flag = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (*flag) {
        __threadfence();
        uint64_t b = 0;
        for (uint32_t i = tid; i < gridDim.x; i += kThreads) b += __ldcg(A.partials + i);
        b = warp_sum_u64(b);
        __syncthreads();
        if (lane == 0) red[warp] = b;
        __syncthreads();
        if (tid == 0) {
            uint64_t tot = 0;
            for (int w = 0; w < kConsumerWarps + 1; ++w) tot += red[w];
            *A.d_count = tot;
            *A.ticket = 0u;
            *A.tile_next = 0ull;
        }
    }
}

// ------------------------------------------------------------ report writes

// Between the two passes of a report: block b sums the per-(tile, warp)
// counts of range b (tiles [b T, (b + 1) T), T = tiles_per_range) into
// partials[b]. The tile-count pass writes only per-warp-tile counts; a
// per-range atomic there put every warp of the GPU on the same few
// addresses (tiles are claimed in order) and cost up to 2x the scan.
__global__ void __launch_bounds__(kWriteThreads) range_sum_kernel(const uint32_t* __restrict__ warp_counts,
                                                                  uint64_t ntiles, uint64_t tiles_per_range,
                                                                  uint64_t* __restrict__ partials) {
    __shared__ uint64_t redl[kWriteThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    const uint64_t t0 = (uint64_t)blockIdx.x * tiles_per_range;
    const uint64_t t1 = min(t0 + tiles_per_range, ntiles);
    uint64_t v = 0;
    // a tile's 8 counts are two 16-byte words
    const uint4* src = reinterpret_cast<const uint4*>(warp_counts + t0 * kConsumerWarps);
    const uint64_t nv = t1 > t0 ? 2 * (t1 - t0) : 0;
    for (uint64_t i = tid; i < nv; i += kWriteThreads) {
        const uint4 x = __ldcg(src + i);
        v += (uint64_t)(((x.x & kCountMask) + (x.y & kCountMask)) + ((x.z & kCountMask) + (x.w & kCountMask)));
    }
    v = warp_sum_u64(v);
    if (lane == 0) redl[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kWriteThreads / 32; ++w) t += redl[w];
        partials[blockIdx.x] = t;
    }
}

// Second pass of a report: CTA b writes the match positions of the tiles of
// range b from the found bitmaps the tile-count pass stored (no text is
// read again). Its first rank is the sum of the earlier ranges' counts. The
// range's warp counts are read into shared memory kWalk tiles at a time and
// scanned there (tile offsets, warp offsets); then every warp turns the
// bitmaps of its own warp-tiles with matches into positions: a warp-tile
// with few matches is handled by one lane (32 at a time, each reading its
// bitmap and storing its positions in order); one with many by the whole
// warp, staged through shared memory so that the stores are coalesced, with
// the bitmaps of the next kAhead such warp-tiles in flight while it writes.
constexpr uint32_t kWalk = 256;   // tiles per pass over shared memory (one per thread)
constexpr uint32_t kAhead = 4;    // bitmaps in flight per warp
constexpr uint32_t kLaneTile = 64; // warp-tiles with at most this many matches are written by one lane
constexpr uint32_t kLaneList = 14; // ... when their slot is a list of at most this many entries (32 words)

__global__ void __launch_bounds__(kWriteThreads) bitmap_write_kernel(const __grid_constant__ WriteArgs W) {
    static_assert(kWalk == kWriteThreads, "one tile per thread");
    __shared__ uint32_t stage[kConsumerWarps][kStageWords];
    __shared__ uint32_t woff[kWalk][kConsumerWarps];  // warp offsets within the tile
    __shared__ uint32_t ttot[kWalk];                  // tile totals
    __shared__ uint32_t toff[kWalk];                  // tile offsets within the pass
    __shared__ uint64_t red[kConsumerWarps];
    __shared__ uint64_t base_s;
    __shared__ uint8_t list[kConsumerWarps][kWalk];   // per warp: its warp-tiles with matches in the pass
    __shared__ uint8_t nent[kWalk][kConsumerWarps];   // list length of each warp-tile's slot (0: bitmap)
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t t0 = (uint64_t)blockIdx.x * W.tiles_per_cta;
    const uint64_t t1 = min(t0 + W.tiles_per_cta, W.ntiles);

    // first rank of the range: the counts of the earlier ranges (block 0
    // sums all of them instead, for the truncation flag)
    const uint32_t upto = blockIdx.x == 0 ? gridDim.x : blockIdx.x;
    uint64_t v = 0;
    for (uint32_t i = tid; i < upto; i += kWriteThreads) v += __ldcg(W.partials + i);
    v = warp_sum_u64(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (tid == 0) {
        uint64_t b = 0;
        for (int w = 0; w < kConsumerWarps; ++w) b += red[w];
        base_s = blockIdx.x == 0 ? 0 : b;
        if (blockIdx.x == 0 && b > W.cap) atomicOr(W.status, kStatusTrunc);
    }
    __syncthreads();
    uint64_t base = base_s;

    uint32_t* stg = stage[warp];
    for (uint64_t p0 = t0; p0 < t1; p0 += kWalk) {
        const uint32_t np = (uint32_t)min((uint64_t)kWalk, t1 - p0);
        // thread i: tile p0 + i -> warp offsets within the tile and its total
        uint32_t tot = 0;
        if (tid < np) {
            const uint4* src = reinterpret_cast<const uint4*>(W.warp_counts + (p0 + tid) * kConsumerWarps);
            const uint4 a = __ldcg(src), b = __ldcg(src + 1);
            const uint32_t c[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) {
                woff[tid][w] = tot;
                tot += c[w] & kCountMask;
                nent[tid][w] = (uint8_t)(c[w] >> 16);
            }
            ttot[tid] = tot;
        }
        // exclusive scan of the tile totals over the pass
        const uint32_t inc = warp_incl_scan(tot, lane);
        if (lane == 31) red[warp] = inc;
        __syncthreads();
        uint32_t wbase = 0;
        for (uint32_t w = 0; w < warp; ++w) wbase += (uint32_t)red[w];
        if (tid < np) toff[tid] = wbase + inc - tot;
        uint64_t pass_tot = 0;
        for (int w = 0; w < kConsumerWarps; ++w) pass_tot += red[w];
        __syncthreads();

        // warp w: the list of its warp-tiles with matches in the pass, in
        // tile order (from ballots), then their bitmaps -> positions, the
        // bitmaps loaded kAhead entries before they are written
        auto own = [&](uint32_t k) -> uint32_t {   // matches of warp-tile (p0 + k, warp)
            return (warp + 1 < kConsumerWarps ? woff[k][warp + 1] : ttot[k]) - woff[k][warp];
        };
        // warp-tiles in list form with at most kLaneTile matches (back of the
        // list) are written by one lane each; the others (front of the list)
        // by the whole warp
        auto by_lane = [&](uint32_t k, uint32_t o) {
            return nent[k][warp] != 0 && nent[k][warp] <= kLaneList && o <= kLaneTile;
        };
        uint8_t* lst = list[warp];
        uint32_t cnt = 0, ns = 0;
        for (uint32_t c0 = 0; c0 < np; c0 += 32) {
            const uint32_t k = c0 + lane;
            const uint32_t o = k < np ? own(k) : 0u;
            const bool wl = o != 0 && !by_lane(k, o), ll = o != 0 && by_lane(k, o);
            const uint32_t bal = __ballot_sync(kFull, wl);
            const uint32_t sal = __ballot_sync(kFull, ll);
            const uint32_t lt = (1u << lane) - 1u;
            if (wl) lst[cnt + __popc(bal & lt)] = (uint8_t)k;
            if (ll) lst[kWalk - 1 - (ns + __popc(sal & lt))] = (uint8_t)k;
            cnt += __popc(bal);
            ns += __popc(sal);
        }
        __syncwarp();
        for (uint32_t g = 0; g < ns; g += 32) {
            // the lists (at most 32 words) of the next 32 warp-tiles into the
            // staging area, row i (33 words) for warp-tile i: lane 8u + q
            // copies words 4q .. 4q + 3 of warp-tile 4 st + u, so that each
            // step covers four lists and the loads of four steps are in
            // flight together; then lane i writes warp-tile i from there
            const uint32_t nb = min(32u, ns - g);
            const uint32_t q = lane & 7u;
#pragma unroll
            for (uint32_t h = 0; h < 8; h += 4) {
                uint4 v[4];
#pragma unroll
                for (uint32_t st = 0; st < 4; ++st) {
                    const uint32_t i = 4u * (h + st) + (lane >> 3);
                    v[st] = make_uint4(0u, 0u, 0u, 0u);
                    if (i < nb) {
                        const uint32_t k = lst[kWalk - 1 - (g + i)];
                        if (q < 1u + (nent[k][warp] + 1u) / 2u)
                            v[st] = __ldcg(reinterpret_cast<const uint4*>(
                                               W.bitmaps + ((p0 + k) * kConsumerWarps + warp) * kBitmapWords) + q);
                    }
                }
#pragma unroll
                for (uint32_t st = 0; st < 4; ++st) {
                    uint32_t* row = stg + 33u * (4u * (h + st) + (lane >> 3)) + 4u * q;
                    row[0] = v[st].x;
                    row[1] = v[st].y;
                    row[2] = v[st].z;
                    row[3] = v[st].w;
                }
            }
            __syncwarp();
            if (lane < nb) {
                const uint32_t k = lst[kWalk - 1 - (g + lane)];
                const uint32_t* slot = stg + 33u * lane;
                const uint64_t s0 = (p0 + k) * kTile + warp * kWarpStarts;
                uint64_t o = base + toff[k] + woff[k][warp];
                const uint32_t ne = nent[k][warp];
                const uint4 h = make_uint4(slot[0], slot[1], slot[2], slot[3]);
                auto put = [&](uint64_t p0s, uint32_t fw) {
                    while (fw) {
                        if (o < W.cap) W.d_pos[o] = p0s + (uint32_t)(__ffs(fw) - 1);
                        ++o;
                        fw &= fw - 1;
                    }
                };
                if (W.folded) {
                    // ascending is chunk row c, then lane, then start in the
                    // chunk: rows[c] = the lanes with a match in row c; a
                    // lane's entry is its rank among the lanes with a match
                    const uint32_t M = h.x;
                    uint32_t rows[4] = {0u, 0u, 0u, 0u};
                    for (uint32_t j = 0, mm = M; j < ne; ++j, mm &= mm - 1u) {
                        const uint32_t bit = mm & (0u - mm);
                        const uint32_t x = slot[4 + 2 * j], y = slot[5 + 2 * j];
                        rows[0] |= (x & 0xF0F0F0F0u) ? bit : 0u;
                        rows[1] |= (x & 0x0F0F0F0Fu) ? bit : 0u;
                        rows[2] |= (y & 0xF0F0F0F0u) ? bit : 0u;
                        rows[3] |= (y & 0x0F0F0F0Fu) ? bit : 0u;
                    }
#pragma unroll
                    for (uint32_t c = 0; c < 4; ++c) {
                        for (uint32_t mm = rows[c]; mm; mm &= mm - 1u) {
                            const uint32_t sl = (uint32_t)__ffs(mm) - 1u;
                            const uint32_t j = __popc(M & ((1u << sl) - 1u));
                            const uint32_t x = slot[4 + 2 * j + (c >> 1)];
                            put(s0 + 16u * (32u * c + sl), unfold_chunk(x, c));
                        }
                    }
                } else {
                    uint32_t mm = h.x;
                    for (uint32_t j = 0; j < ne; ++j) {
                        const uint32_t sl = (uint32_t)__ffs(mm) - 1u;
                        mm &= mm - 1u;
                        put(s0 + 64u * sl, slot[4 + 2 * j]);
                        put(s0 + 64u * sl + 32u, slot[5 + 2 * j]);
                    }
                }
            }
            __syncwarp();   // the staging area is refilled by the next group
        }
        // whole warp: lane l loads words 2l, 2l + 1 of the slot; a list is
        // spread back to its lanes by shuffles, folded entries are turned
        // into lane l's 64 starts 64l .. 64l + 63 in order
        auto load = [&](uint32_t j) -> uint2 {
            return __ldcg(reinterpret_cast<const uint2*>(W.bitmaps + ((p0 + lst[j]) * kConsumerWarps + warp) *
                                                                         kBitmapWords) + lane);
        };
        auto write = [&](uint32_t j, uint2 raw) {
            const uint32_t k = lst[j];
            const uint32_t ne = nent[k][warp];
            uint32_t ex = raw.x, ey = raw.y;
            if (ne) {
                const uint32_t M = __shfl_sync(kFull, raw.x, 0);
                const uint32_t src = 2u + __popc(M & ((1u << lane) - 1u));
                const uint32_t tx = __shfl_sync(kFull, raw.x, src & 31u), ty = __shfl_sync(kFull, raw.y, src & 31u);
                const bool has = (M >> lane) & 1u;
                ex = has ? tx : 0u;
                ey = has ? ty : 0u;
            }
            uint32_t m0 = ex, m1 = ey;
            if (W.folded) {
                // lane l's chunks 4l + i sit in entry lane (4l + i) mod 32, chunk row l / 8
                const uint32_t c = lane >> 3;
                uint32_t mk[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t src = (4u * lane + (uint32_t)i) & 31u;
                    const uint32_t xs = __shfl_sync(kFull, ex, src), ys = __shfl_sync(kFull, ey, src);
                    mk[i] = unfold_chunk((c >> 1) ? ys : xs, c);
                }
                m0 = mk[0] | (mk[1] << 16);
                m1 = mk[2] | (mk[3] << 16);
            }
            const uint32_t n = __popc(m0) + __popc(m1);
            const uint32_t inc2 = warp_incl_scan(n, lane);
            const uint32_t r0 = 64u * lane, r1 = 64u * lane + 32u;
            staged_write(stg, lane, inc2 - n, n, own(k), (p0 + k) * kTile + warp * kWarpStarts,
                         base + toff[k] + woff[k][warp], W.d_pos, W.cap, [&](auto&& cb) {
                             uint32_t kk = 0, fw = m0;
                             while (fw) {
                                 cb(kk++, r0 + (uint32_t)(__ffs(fw) - 1));
                                 fw &= fw - 1;
                             }
                             fw = m1;
                             while (fw) {
                                 cb(kk++, r1 + (uint32_t)(__ffs(fw) - 1));
                                 fw &= fw - 1;
                             }
                         });
        };
        uint2 pre[kAhead];
#pragma unroll
        for (uint32_t d = 0; d < kAhead; ++d) pre[d] = d < cnt ? load(d) : make_uint2(0u, 0u);
        for (uint32_t j = 0; j < cnt; j += kAhead) {
#pragma unroll
            for (uint32_t d = 0; d < kAhead; ++d) {
                if (j + d < cnt) {
                    const uint2 x = pre[d];
                    if (j + d + kAhead < cnt) pre[d] = load(j + d + kAhead);
                    write(j + d, x);
                }
            }
        }
        base += pass_tot;
        __syncthreads();   // the pass's tables are rewritten by the next one
    }
}

// ------------------------------------------------------------ histogram

__global__ void __launch_bounds__(kHistThreads) hist_kernel(const HistArgs A) {
    // 32 lane-private copies of the 256 bins, laid out [bin][lane] so that
    // the lanes of a warp never share a bank or an address.
    __shared__ uint32_t h[256 * 32];
    __shared__ uint32_t last;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    for (uint32_t i = tid; i < 256 * 32; i += kHistThreads) h[i] = 0;
    __syncthreads();

    const uintptr_t tb = reinterpret_cast<uintptr_t>(A.text);
    const uint64_t head = min(A.n, (uint64_t)((16u - (tb & 15u)) & 15u));
    const uint64_t nvec = (A.n - head) / 16;
    const uint64_t tail0 = head + nvec * 16;
    if (blockIdx.x == 0) {
        if (tid < head) atomicAdd(&h[A.text[tid] * 32u + lane], 1u);
        if (tail0 + tid < A.n) atomicAdd(&h[A.text[tail0 + tid] * 32u + lane], 1u);
    }
    const uint4* v = reinterpret_cast<const uint4*>(A.text + head);
    const uint64_t stride = (uint64_t)gridDim.x * kHistThreads;
    for (uint64_t k = (uint64_t)blockIdx.x * kHistThreads + tid; k < nvec; k += 2 * stride) {
        const uint4 x = __ldcs(v + k);
        const bool two = k + stride < nvec;
        const uint4 y = two ? __ldcs(v + k + stride) : make_uint4(0, 0, 0, 0);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int b = 0; b < 4; ++b) atomicAdd(&h[((w[i] >> (8 * b)) & 0xFFu) * 32u + lane], 1u);
        if (two) {
            const uint32_t z[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int b = 0; b < 4; ++b) atomicAdd(&h[((z[i] >> (8 * b)) & 0xFFu) * 32u + lane], 1u);
        }
    }
    __syncthreads();

    // thread tid owns bin tid (kHistThreads == 256)
    uint64_t s = 0;
    for (uint32_t l = 0; l < 32; ++l) s += h[tid * 32u + ((l + tid) & 31u)];
    A.partials[(uint64_t)blockIdx.x * 256 + tid] = s;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(A.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (last) {
        __threadfence();
        uint64_t t = 0;
        for (uint32_t b = 0; b < gridDim.x; ++b) t += __ldcg(A.partials + (uint64_t)b * 256 + tid);
        A.d_hist[tid] = t;
        if (tid == 0) *A.ticket = 0u;
    }
}

// ------------------------------------------------------------ dispatch

template <int MAXM, int MODE, int KIND>
cudaError_t launch_one(uint32_t grid, size_t smem, cudaStream_t st, const ScanArgs& a, const uint32_t* qc,
                       const uint32_t* groups) {
    if (a.ng > (uint32_t)PatArg<MAXM>::kGroups) return cudaErrorInvalidValue;
    PatArg<MAXM> p;
    uint32_t j = 0;
    for (; j < a.m; ++j) p.qc[j] = qc[j];
    for (; j < (uint32_t)MAXM; ++j) p.qc[j] = 0;
    for (j = 0; j < a.ng; ++j) p.grp[j] = groups[j];
    for (; j < (uint32_t)PatArg<MAXM>::kGroups; ++j) p.grp[j] = 0;
    scan_kernel<MAXM, MODE, KIND><<<grid, kThreads, smem, st>>>(a, p);
    return cudaGetLastError();
}

template <int MAXM, int MODE>
cudaError_t launch_kind(int kind, uint32_t grid, size_t smem, cudaStream_t st, const ScanArgs& a, const uint32_t* qc,
                        const uint32_t* groups) {
    switch (kind) {
        case kKindBytes: return launch_one<MAXM, MODE, kKindBytes>(grid, smem, st, a, qc, groups);
        case kKindSeven: return launch_one<MAXM, MODE, kKindSeven>(grid, smem, st, a, qc, groups);
        case kKindPackedAdj: return launch_one<MAXM, MODE, kKindPackedAdj>(grid, smem, st, a, qc, groups);
        case kKindBinary: return launch_one<MAXM, MODE, kKindBinary>(grid, smem, st, a, qc, groups);
        default: return launch_one<MAXM, MODE, kKindPacked>(grid, smem, st, a, qc, groups);
    }
}

template <int MODE, int KIND>
const void* kernel_ptr(uint32_t m) {
    if (m <= (uint32_t)kSmallM) return reinterpret_cast<const void*>(&scan_kernel<kSmallM, MODE, KIND>);
    return reinterpret_cast<const void*>(&scan_kernel<kLargeM, MODE, KIND>);
}

template <int MODE>
const void* pick_kind(int kind, uint32_t m) {
    switch (kind) {
        case kKindBytes: return kernel_ptr<MODE, kKindBytes>(m);
        case kKindSeven: return kernel_ptr<MODE, kKindSeven>(m);
        case kKindPackedAdj: return kernel_ptr<MODE, kKindPackedAdj>(m);
        case kKindBinary: return kernel_ptr<MODE, kKindBinary>(m);
        default: return kernel_ptr<MODE, kKindPacked>(m);
    }
}

const void* pick(int mode, int kind, uint32_t m) {
    switch (mode) {
        case kModeCount: return pick_kind<kModeCount>(kind, m);
        case kModeTileCount: return pick_kind<kModeTileCount>(kind, m);
        case kModeSparse: return pick_kind<kModeSparse>(kind, m);
        default: return pick_kind<kModeWrite>(kind, m);
    }
}

}  // namespace

cudaError_t launch_scan(int mode, int kind, uint32_t grid, size_t smem, cudaStream_t s, const ScanArgs& a,
                        const uint32_t* qc, const uint32_t* groups) {
    const bool small = a.m <= (uint32_t)kSmallM;
    switch (mode) {
        case kModeCount:
            return small ? launch_kind<kSmallM, kModeCount>(kind, grid, smem, s, a, qc, groups)
                         : launch_kind<kLargeM, kModeCount>(kind, grid, smem, s, a, qc, groups);
        case kModeTileCount:
            return small ? launch_kind<kSmallM, kModeTileCount>(kind, grid, smem, s, a, qc, groups)
                         : launch_kind<kLargeM, kModeTileCount>(kind, grid, smem, s, a, qc, groups);
        case kModeSparse:
            return small ? launch_kind<kSmallM, kModeSparse>(kind, grid, smem, s, a, qc, groups)
                         : launch_kind<kLargeM, kModeSparse>(kind, grid, smem, s, a, qc, groups);
        default:
            return small ? launch_kind<kSmallM, kModeWrite>(kind, grid, smem, s, a, qc, groups)
                         : launch_kind<kLargeM, kModeWrite>(kind, grid, smem, s, a, qc, groups);
    }
}

int scan_occupancy(int mode, int kind, uint32_t m, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick(mode, kind, m), kThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

int bitmap_write_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bitmap_write_kernel, kWriteThreads, 0) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t scan_prepare(size_t max_smem) {
    for (int mode = 0; mode < kModes; ++mode)
        for (int kind = 0; kind < kKinds; ++kind)
            for (uint32_t m : {1u, (uint32_t)kLargeM}) {
                cudaError_t e = cudaFuncSetAttribute(pick(mode, kind, m),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

cudaError_t launch_range_sums(uint32_t grid, cudaStream_t s, const uint32_t* warp_counts, uint64_t ntiles,
                              uint64_t tiles_per_range, uint64_t* partials) {
    range_sum_kernel<<<grid, kWriteThreads, 0, s>>>(warp_counts, ntiles, tiles_per_range, partials);
    return cudaGetLastError();
}

cudaError_t launch_bitmap_write(uint32_t grid, cudaStream_t s, const WriteArgs& a) {
    bitmap_write_kernel<<<grid, kWriteThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_hist(uint32_t grid, cudaStream_t s, const HistArgs& a) {
    hist_kernel<<<grid, kHistThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace smk

#if SMK_COUNT_COMPARES
// Profiling builds only: the early-exit counters of the scan kernels (see
// sm_device.cuh), read into out[0..3] and, with reset, cleared. Not part of
// the library's interface.
extern "C" int sm_debug_compare_stats(unsigned long long* out, int reset) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(out, smk::dev::g_cmp_stats, 4 * sizeof(unsigned long long)) != cudaSuccess) return 1;
    if (reset) {
        const unsigned long long z[4] = {0, 0, 0, 0};
        if (cudaMemcpyToSymbol(smk::dev::g_cmp_stats, z, sizeof z) != cudaSuccess) return 1;
    }
    return 0;
}
#endif
