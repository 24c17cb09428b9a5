// Device helpers shared by the scan and batch kernels: mbarrier and TMA
// wrappers, bounded waits, the SWAR byte compare and warp reductions.
// Internal to the library.
#pragma once

#include "sm_internal.h"

namespace smk {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint64_t kEnd = ~0ull;

// Early-exit counters of a profiling build (-DSMK_COUNT_COMPARES=1; off in
// the library): per 16-start chunk (2-bit codes: per 16-start word) the
// compares run in the dense phase and, for the chunks that survive it, in the
// sparse phase. [0] chunks, [1] dense compares, [2] surviving chunks, [3]
// sparse compares (cooperative ones included), summed over all launches of
// the translation unit's scan kernels until read.
#ifndef SMK_COUNT_COMPARES
#define SMK_COUNT_COMPARES 0
#endif
#if SMK_COUNT_COMPARES
static __device__ unsigned long long g_cmp_stats[4];
__device__ __forceinline__ void cmp_stats_add(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    const uint32_t v[4] = {a, b, c, d};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t w = __reduce_add_sync(kFull, v[i]);
        if ((threadIdx.x & 31u) == 0 && w) atomicAdd(&g_cmp_stats[i], (unsigned long long)w);
    }
}
#define SMK_STATS(...) __VA_ARGS__
#else
#define SMK_STATS(...)
#endif

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Test the phase; a thread whose phase is not complete may be suspended until
// it completes or about SMK_SUSPEND_NS pass (0: the hardware's own limit).
#ifndef SMK_SUSPEND_NS
#define SMK_SUSPEND_NS 20000
#endif

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
#if SMK_SUSPEND_NS > 0
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"((uint32_t)SMK_SUSPEND_NS)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
#endif
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete, at most limit_ns. Between
// polls the warp sleeps, doubling from 32 ns up to max_sleep_ns, so that a
// waiting warp takes almost no issue slots from the working ones.
#ifndef SMK_MAX_SLEEP_NS
#define SMK_MAX_SLEEP_NS 256
#endif
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                             uint32_t max_sleep_ns = SMK_MAX_SLEEP_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    uint32_t sleep = 32;
    while (!mbar_try_wait(bar, parity)) {
        if (max_sleep_ns) {
            __nanosleep(sleep);
            if (sleep < max_sleep_ns) sleep <<= 1;
        }
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Consumer-wide barrier (the 8 consumer warps, barrier 1) that also returns
// whether any consumer thread passed v = true.
__device__ __forceinline__ bool consumers_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kConsumerWarps * 32)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumerWarps * 32) : "memory");
}

// ------------------------------------------------------------ tile staging

// One tile's copy: text bytes [s0, need_end) of a text of length n at
// address tb land in a stage buffer at offset (tb mod 16), so that byte x of
// the tile sits at buf[(tb mod 16) + x - s0]. The 16-byte-aligned interior
// (never outside the text) is one TMA bulk copy; the at most 15 bytes before
// it and 15 after it are loaded by the warp's lanes here.
struct TileCopy {
    uintptr_t src;       // global source of the bulk copy (16-byte aligned)
    uint32_t dst_off;    // offset of the copy in the stage buffer (16-byte aligned)
    uint32_t bytes;      // multiple of 16, may be 0
};

__device__ __forceinline__ TileCopy stage_ragged(uint8_t* buf, const uint8_t* text, uint64_t n, uint64_t s0,
                                                 uint64_t need_end, uint32_t lane) {
    const uintptr_t tb = reinterpret_cast<uintptr_t>(text);
    const uint32_t delta = (uint32_t)(tb & 15u);
    // text indices [lo_al, hi_al) form the 16-byte aligned interior
    const int64_t lo_al = (int64_t)(((tb + 15u) & ~(uintptr_t)15u) - tb);
    const int64_t hi_al = (int64_t)((tb + n) & ~(uintptr_t)15u) - (int64_t)tb;
    const int64_t ne = (int64_t)need_end;
    const int64_t h_end = min(ne, lo_al);
    const int64_t t_beg = max((int64_t)s0, max(lo_al, max(hi_al, (int64_t)0)));
    const int64_t xh = (int64_t)s0 + lane, xt = t_beg + lane;
    if (xh < h_end) buf[delta + (xh - (int64_t)s0)] = text[xh];
    if (xt < ne) buf[delta + (xt - (int64_t)s0)] = text[xt];
    const uintptr_t g0 = (tb + s0) & ~(uintptr_t)15u;
    const uintptr_t ga = max(g0, tb + (uintptr_t)lo_al);
    const uintptr_t ge = (tb + need_end + 15u) & ~(uintptr_t)15u;
    const uintptr_t gb = min(ge, (tb + n) & ~(uintptr_t)15u);
    __threadfence_block();
    TileCopy c;
    c.src = ga;
    c.dst_off = (uint32_t)(ga - g0);
    c.bytes = gb > ga ? (uint32_t)(gb - ga) : 0u;
    return c;
}

// ------------------------------------------------------------ compare core

// A byte of x = w ^ (c..c) is zero iff that byte of w equals c. Several
// compares fold into one zero-byte test: a byte of the OR of their XORs is
// zero iff every one of them matched, so the found flags after the test are
// the AND of the flags of the separate compares.
//
// keep_zero(f, y): f & [byte of y == 0], flags in the high bit of each byte.
// General bytes: the high bit of ((y & 0x7F..) + 0x7F..) | y is set iff the
// byte is nonzero. SEVEN: every byte of y is below 0x80 (text and pattern
// are 7-bit), so y + 0x7F.. cannot carry between bytes and its high bit
// alone marks a nonzero byte. With SMK_MADD_ADD the add is a multiply-add by
// `one` (== 1) so that it issues on the multiply-add pipe instead of the
// integer pipe.
#ifndef SMK_MADD_ADD
#define SMK_MADD_ADD 1
#endif
template <bool SEVEN>
__device__ __forceinline__ uint32_t keep_zero(uint32_t f, uint32_t y, uint32_t one) {
#if SMK_MADD_ADD
    if (SEVEN) return f & ~(y * one + 0x7F7F7F7Fu);
    return f & ~(((y & 0x7F7F7F7Fu) * one + 0x7F7F7F7Fu) | y);
#else
    (void)one;
    if (SEVEN) return f & ~(y + 0x7F7F7F7Fu);
    return f & ~(((y & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | y);
#endif
}

// One compare, accumulated for the lane's NC 16-start chunks: y |= window ^
// (c..c), where the window of a start s is text bytes s+q .. s+q+3 and a, b
// hold the 16-byte units E and E + 1 of each chunk. v = (e << 8) | symbol
// with e = text misalignment + pattern position q; the caller guarantees
// E == e >> 4 and D == (e >> 2) & 3, so the word selection is static.
template <int D, int NC>
__device__ __forceinline__ void acc_loaded(const uint4 (&a)[NC], const uint4 (&b)[NC], uint32_t v,
                                           uint32_t (&y)[NC][4]) {
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
    const uint32_t sh = ((v >> 8) & 3u) << 3;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const uint32_t X[8] = {a[c].x, a[c].y, a[c].z, a[c].w, b[c].x, b[c].y, b[c].z, b[c].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) y[c][i] |= __funnelshift_r(X[D + i], X[D + i + 1], sh) ^ P;
    }
}

// As acc_loaded for a compare whose window is 4-byte aligned (e mod 4 == 0):
// the words need no shift.
template <int D, int NC>
__device__ __forceinline__ void acc_aligned(const uint4 (&a)[NC], const uint4 (&b)[NC], uint32_t v,
                                            uint32_t (&y)[NC][4]) {
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const uint32_t X[8] = {a[c].x, a[c].y, a[c].z, a[c].w, b[c].x, b[c].y, b[c].z, b[c].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) y[c][i] |= X[D + i] ^ P;
    }
}

// One compare, accumulated for a single 16-start chunk whose first start is
// at word index W of the stage buffer (any alignment class).
__device__ __forceinline__ void acc_window(const uint32_t* __restrict__ b32, uint32_t W, uint32_t v,
                                           uint32_t (&y)[4]) {
    const uint32_t e = v >> 8;
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
    const uint32_t w0 = W + (e >> 2);
    const uint32_t sh = (e & 3u) << 3;
    uint32_t t[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) t[i] = b32[w0 + i];
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] |= __funnelshift_r(t[i], t[i + 1], sh) ^ P;
}

// Sum of the found flags (bit 7 of each byte) of NC x 4 words: eight words
// fold into one before each popcount, their flags landing on distinct bits.
template <int NC>
__device__ __forceinline__ uint32_t count_flags(const uint32_t (&f)[NC][4]) {
    uint32_t total = 0;
#pragma unroll
    for (int g = 0; g < NC * 4; g += 8) {
        uint32_t x = 0;
#pragma unroll
        for (int k = 0; k < 8 && g + k < NC * 4; ++k) x |= f[(g + k) / 4][(g + k) % 4] >> k;
        total += __popc(x);
    }
    return total;
}

__device__ __forceinline__ uint32_t valid_mask(int64_t lim) {
    // high bits of the bytes whose start index (relative to the word) is < lim
    if (lim >= 4) return 0x80808080u;
    if (lim <= 0) return 0u;
    return 0x80808080u & ((1u << (8 * lim)) - 1u);
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) { return __reduce_add_sync(kFull, v); }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= (uint32_t)o) v += y;
    }
    return v;
}

template <int MAXM>
struct PatArg {
    static constexpr int kGroups = (14 + MAXM) / 16 + 1;
    uint32_t qc[MAXM];        // compare j: (e_j << 8) | p[pi(j)], e_j = (text address mod 16) + pi(j)
    uint32_t grp[kGroups];    // window groups of the peeled compares
};

// A 16-start chunk's found flags packed as in the survivor queue (word i,
// byte b at bit 8b + i) -> 16 bits in start order (start 4i + b at bit
// 4i + b): gather the nibbles, then transpose the 4 x 4 bit matrix.
__device__ __forceinline__ uint32_t chunk_mask16(uint32_t x) {
    x &= 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    uint32_t t = (x ^ (x >> 3)) & 0x0A0Au;
    x ^= t ^ (t << 3);
    t = (x ^ (x >> 6)) & 0x00CCu;
    return x ^ t ^ (t << 6);
}

// Stores one batch of a warp's match positions in rank order. The lane's n
// positions have ranks excl .. excl + n - 1 of the batch's tot and are
// base + rel; for_each(cb) calls cb(k, rel) for the lane's k-th position in
// ascending order. Positions pass through the warp's staging area stg
// (kStageWords words) slice by slice, so that consecutive lanes store
// consecutive ranks. Staged rank x sits at word x + x / 32: lanes whose
// ranks are spaced evenly (by up to 32) then write distinct banks, where the
// plain layout would put them on two. Ranks at or beyond cap (counted from
// the batch's first rank `out`) are dropped. base is a multiple of
// kWarpStarts and rel < kWarpStarts (a warp-tile's positions), so base + rel
// is base | rel: no carry into the high word.
constexpr uint32_t kStageCap = 1024;
constexpr uint32_t kStageWords = kStageCap + kStageCap / 32;

template <class ForEach>
__device__ __forceinline__ void staged_write(uint32_t* stg, uint32_t lane, uint32_t excl, uint32_t n, uint32_t tot,
                                             uint64_t base, uint64_t out, uint64_t* __restrict__ d_pos,
                                             uint64_t cap, ForEach for_each) {
    const uint32_t lo = (uint32_t)base, hi = (uint32_t)(base >> 32);
    auto pos = [&](uint32_t rel) { return ((uint64_t)hi << 32) | (lo | rel); };
    for (uint32_t p0 = 0; p0 < tot; p0 += kStageCap) {
        if (tot <= kStageCap) {   // one slice: every rank of the lane is in it
            if (n) for_each([&](uint32_t k, uint32_t rel) { stg[excl + k + ((excl + k) >> 5)] = rel; });
        } else if (n && excl < p0 + kStageCap && excl + n > p0) {
            for_each([&](uint32_t k, uint32_t rel) {
                const uint32_t rk = excl + k - p0;   // wraps to a large value below the slice
                if (rk < kStageCap) stg[rk + (rk >> 5)] = rel;
            });
        }
        __syncwarp();
        // stores of two positions (16 bytes) per lane, after one lone
        // position when the slice does not start on a 16-byte boundary
        const uint32_t cnt = min(kStageCap, tot - p0);
        const uint64_t g0 = out + p0;
        const uint32_t lead = (reinterpret_cast<uintptr_t>(d_pos + g0) & 15u) ? 1u : 0u;
        if (lead && lane == 0 && cnt && g0 < cap) d_pos[g0] = pos(stg[0]);
        for (uint32_t o = lead + 2 * lane; o < cnt; o += 64) {
            const uint64_t g = g0 + o;
            const uint64_t a = pos(stg[o + (o >> 5)]);
            if (o + 1 < cnt && g + 1 < cap) {
                const uint64_t b = pos(stg[o + 1 + ((o + 1) >> 5)]);
                *reinterpret_cast<ulonglong2*>(d_pos + g) = make_ulonglong2(a, b);
            } else if (g < cap) {
                d_pos[g] = a;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ one warp-tile

// Compare descriptors and window groups held in the kernel's parameter block.
template <int MAXM>
struct ParamQC {
    const PatArg<MAXM>* p;
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return p->qc[j]; }
    __device__ __forceinline__ uint32_t group(uint32_t g) const { return p->grp[g]; }
};

// Compare descriptors in global memory (read-only, uniform across the warp),
// the window groups after the m compares.
struct GlobalQC {
    const uint32_t* __restrict__ p;
    uint32_t m;
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return __ldg(p + j); }
    __device__ __forceinline__ uint32_t group(uint32_t g) const { return __ldg(p + m + g); }
};

// One consumer warp's 2048 starts of a staged tile against one pattern:
// Algorithms 2-4. Starts at or beyond nstarts (relative to the tile's first
// start s0) are out of range. Returns this lane's number of matches; with
// WRITE, also writes the positions in ascending order from rank `out`
// (first `cap` only). DIRECT: a count may skip the compaction when r >= m.
// bm (tile-count pass of a report): when the warp-tile has matches, its
// 2048 found bits in start order are stored to bm (64 words), built in the
// warp's shared scratch sbm (64 words).
//
// Dense phase: the r peeled compares for all 2048 starts, folded into one
// zero-byte test. They arrive in ng window groups: the two 16-byte units of
// every chunk are loaded once per group and serve all its compares, the
// 4-byte-aligned ones (no shift) first.
// Sparse phase: the 16-start chunks with a surviving start are compacted, in
// position order, into the warp's queue q (at most 128 entries of one word:
// the chunk's found bits and index); each lane then takes
// one chunk and continues with compares r .. m-1, two per zero-byte test,
// leaving as soon as the chunk's found flags are all zero - the early exit
// of Algorithm 2, taken per 16-start chunk. A chunk still alive after
// kLaneCompares compares is finished by the whole warp.
// Compares a lane takes alone in the sparse phase before the warp shares
// the rest of a surviving chunk.
constexpr uint32_t kLaneCompares = 16;

// Found bits of a warp-tile with matches, as the tile-count pass of a report
// stores them in the warp-tile's 64-word slot: one 64-bit entry per lane,
// lane l's entry in the layout of the compare kind --
//   byte compares (folded): lane l's chunks 32c + l (c = 0..3, chunk k =
//     starts 16k .. 16k + 15 of the warp-tile) as the two words the count
//     folds anyway: word h = c >> 1 has bit 7 - (4 (c & 1) + i) + 8b for
//     start 16 (32c + l) + 4i + b;
//   coded compares (contiguous): lane l's starts 64l .. 64l + 63, bit s of
//     the entry (low word first) for start 64l + s.
// List form, when at most kListMax lanes have a match: word 0 holds the
// ballot of the lanes with a match (words 1-3 are zero), and the j-th lane
// with a match (ascending) has its entry at words 4 + 2j, 5 + 2j; the slot's
// other words are not written. Bitmap form otherwise: lane l's entry at
// words 2l, 2l + 1. The per-(tile, warp) count word tells them apart:
// matches in bits 0-15, the number of list entries in bits 16-23 (0: bitmap
// form). Pass 1 only stores words it has; pass 2 reorders them into
// positions.
constexpr uint32_t kListMax = kBitmapWords / 2 - 2;   // 30
constexpr uint32_t kCountMask = 0xFFFFu;

// Lane entries (x, y) -> the warp-tile's slot in the form that fits; returns
// the list length (0: bitmap form). All lanes take part.
__device__ __forceinline__ uint32_t store_slot(uint32_t* __restrict__ bm, uint32_t lane, uint32_t x, uint32_t y) {
    const bool nz = (x | y) != 0u;
    const uint32_t bal = __ballot_sync(kFull, nz);
    const uint32_t nl = __popc(bal);
    uint2* b2 = reinterpret_cast<uint2*>(bm);
    if (nl <= kListMax) {
        if (nz) b2[2 + __popc(bal & ((1u << lane) - 1u))] = make_uint2(x, y);
        if (lane == 0) reinterpret_cast<uint4*>(bm)[0] = make_uint4(bal, 0u, 0u, 0u);
        return nl;
    }
    b2[lane] = make_uint2(x, y);
    return 0;
}

// The two folded words of a lane's NC = 4 chunks of found flags (bit 7 of
// each byte): word h ORs f[2h][i] >> i and f[2h + 1][i] >> (4 + i), whose
// flags land on distinct bits. Their popcounts sum to the lane's matches.
__device__ __forceinline__ void fold_found(const uint32_t (&f)[kChunks][4], uint32_t& x0, uint32_t& x1) {
    x0 = ((f[0][0] | (f[0][1] >> 1)) | ((f[0][2] >> 2) | (f[0][3] >> 3))) |
         (((f[1][0] >> 4) | (f[1][1] >> 5)) | ((f[1][2] >> 6) | (f[1][3] >> 7)));
    x1 = ((f[2][0] | (f[2][1] >> 1)) | ((f[2][2] >> 2) | (f[2][3] >> 3))) |
         (((f[3][0] >> 4) | (f[3][1] >> 5)) | ((f[3][2] >> 6) | (f[3][3] >> 7)));
}

// Chunk c's flags in a folded word x (x is the lane's word c >> 1) -> 16
// bits in start order (bit 4i + b for start 4i + b of the chunk).
__device__ __forceinline__ uint32_t unfold_chunk(uint32_t x, uint32_t c) {
    // nibble of byte b: bit 3 - i for start 4i + b (c odd: low nibbles)
    const uint32_t n = (c & 1u) ? (x & 0x0F0F0F0Fu) : ((x >> 4) & 0x0F0F0F0Fu);
    // reverse each nibble: bit i + 8b for start 4i + b, then transpose
    const uint32_t q = ((n & 0x01010101u) << 3) | ((n & 0x02020202u) << 1) | ((n >> 1) & 0x02020202u) |
                       ((n >> 3) & 0x01010101u);
    return chunk_mask16(q);
}

template <bool SEVEN, bool WRITE, bool DIRECT, class QC>
__device__ __forceinline__ uint32_t warp_tile(const uint4* __restrict__ b4, const uint32_t* __restrict__ b32,
                                              uint32_t c0, uint32_t wq, uint32_t warp, uint32_t lane, QC qc,
                                              uint32_t m, uint32_t r, uint32_t ng, uint32_t one,
                                              uint64_t nstarts, uint64_t s0, uint32_t* q,
                                              uint64_t out, uint64_t* __restrict__ d_pos, uint64_t cap,
                                              uint32_t* __restrict__ bm = nullptr, uint32_t* sbm = nullptr,
                                              uint32_t* ent = nullptr) {
    uint32_t f[kChunks][4];
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) f[c][i] = 0u;
    for (uint32_t g = 0, j = 0; g < ng; ++g) {
        const uint32_t gd = qc.group(g);
        const uint32_t ci = c0 + (gd & 0x1FFu);
        uint4 a[kChunks], b[kChunks];
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            a[c] = b4[ci + 32 * c];
            b[c] = b4[ci + 32 * c + 1];
        }
        // aligned compares (at most one per word class), then the others
        if (gd & (1u << 9)) acc_aligned<0>(a, b, qc(j++), f);
        if (gd & (1u << 10)) acc_aligned<1>(a, b, qc(j++), f);
        if (gd & (1u << 11)) acc_aligned<2>(a, b, qc(j++), f);
        if (gd & (1u << 12)) acc_aligned<3>(a, b, qc(j++), f);
        for (uint32_t k = (gd >> 13) & 3u; k; --k) acc_loaded<0>(a, b, qc(j++), f);
        for (uint32_t k = (gd >> 15) & 3u; k; --k) acc_loaded<1>(a, b, qc(j++), f);
        for (uint32_t k = (gd >> 17) & 3u; k; --k) acc_loaded<2>(a, b, qc(j++), f);
        for (uint32_t k = (gd >> 19) & 3u; k; --k) acc_loaded<3>(a, b, qc(j++), f);
    }
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) f[c][i] = keep_zero<SEVEN>(0x80808080u, f[c][i], one);

    if (s0 + kTile > nstarts) {   // last tile: clear starts beyond n - m
        const int64_t lim = (int64_t)(nstarts - s0) - (int64_t)(warp * kWarpStarts + lane * 16u);
#pragma unroll
        for (int c = 0; c < kChunks; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i) f[c][i] &= valid_mask(lim - (512 * c + 4 * i));
    }

    SMK_STATS(uint32_t st_sparse = 0, st_alive = 0;)
    if (DIRECT && r >= m) {
        SMK_STATS(cmp_stats_add(kChunks, kChunks * r, 0, 0);)
        // every compare peeled: the found bits are final. With bm, a
        // warp-tile with matches stores its lanes' folded words
        uint32_t x0, x1;
        fold_found(f, x0, x1);
        const uint32_t cnt = __popc(x0) + __popc(x1);
        if (bm && __any_sync(kFull, cnt != 0u)) {
            const uint32_t e = store_slot(bm, lane, x0, x1);
            if (ent) *ent = e;
        }
        return cnt;
    }

    // byte c: 1 if chunk c of this lane has a surviving start
    uint32_t alive = 0;
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
        alive |= (uint32_t)(((f[c][0] | f[c][1]) | (f[c][2] | f[c][3])) != 0u) << (8 * c);
    if (!__any_sync(kFull, alive != 0u)) {
        SMK_STATS(cmp_stats_add(kChunks, kChunks * r, 0, 0);)
        return 0;
    }

    // queue in position order: chunk 0 of all lanes, then chunk 1, ...; an
    // entry packs the chunk's 16 found bits (word i's bit 7 + 8b at bit
    // i + 8b) and its index k (bits 4-7: k mod 16, bits 12-14: k / 16)
    const uint32_t incl = warp_incl_scan(alive, lane);
    const uint32_t tot = __shfl_sync(kFull, incl, 31);
    uint32_t qn = 0;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        if ((alive >> (8 * c)) & 1u) {
            const uint32_t k = 32u * c + lane;
            q[qn + ((incl >> (8 * c)) & 0xFFu) - 1u] = ((f[c][0] >> 7) | (f[c][1] >> 6)) | ((f[c][2] >> 5) |
                                                       (f[c][3] >> 4)) | ((k & 15u) << 4) | ((k >> 4) << 12);
        }
        qn += (tot >> (8 * c)) & 0xFFu;
    }
    if (bm) {   // the lanes' folded words of the surviving chunks' final flags, from zero
        sbm[2 * lane] = 0u;
        sbm[2 * lane + 1] = 0u;
    }
    __syncwarp();

    uint32_t tile_count = 0;   // this lane's share of the warp's matches in the tile
    for (uint32_t qb = 0; qb < qn; qb += 32) {
        const uint32_t e = qb + lane;
        uint32_t g[4] = {0u, 0u, 0u, 0u}, k = 0;
        if (e < qn) {
            const uint32_t x = q[e];
            k = ((x >> 4) & 15u) | ((x >> 8) & 0x70u);
#pragma unroll
            for (int i = 0; i < 4; ++i) g[i] = (x << (7 - i)) & 0x80808080u;
        }
        const uint32_t W = wq + 4u * k;   // word index of the chunk's first start
        const uint32_t jl = min(m, r + kLaneCompares);
        SMK_STATS(st_alive += e < qn ? 1u : 0u;)
        for (uint32_t j = r; j < jl && ((g[0] | g[1]) | (g[2] | g[3])); j += 2) {
            SMK_STATS(st_sparse += min(2u, m - j);)
            uint32_t y[4] = {0u, 0u, 0u, 0u};
            acc_window(b32, W, qc(j), y);
            acc_window(b32, W, qc(min(j + 1, m - 1)), y);   // an odd tail repeats compare j
#pragma unroll
            for (int i = 0; i < 4; ++i) g[i] = keep_zero<SEVEN>(g[i], y[i], one);
        }
        // chunks still alive after kLaneCompares compares (long patterns that
        // match or nearly match): the whole warp takes the remaining
        // compares of one chunk at a time, lane l every 32nd from jl + l,
        // and ANDs the found bits across lanes
        uint32_t pend = __ballot_sync(kFull, jl < m && ((g[0] | g[1]) | (g[2] | g[3])) != 0u);
        while (pend) {
            const uint32_t src = (uint32_t)__ffs(pend) - 1u;
            pend &= pend - 1u;
            const uint32_t Ws = __shfl_sync(kFull, W, src);
            SMK_STATS(if (lane == src) st_sparse += m - jl;)
            uint32_t y[4] = {0u, 0u, 0u, 0u};
            for (uint32_t j = jl + lane; j < m; j += 32) acc_window(b32, Ws, qc(j), y);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t t = keep_zero<SEVEN>(0x80808080u, y[i], one);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t &= __shfl_xor_sync(kFull, t, o);
                if (lane == src) g[i] &= t;
            }
        }
        const uint32_t n = (__popc(g[0]) + __popc(g[1])) + (__popc(g[2]) + __popc(g[3]));
        if (bm && n) {
            // chunk k = 32c + l's flags into lane l's folded word c >> 1 (its
            // own bits; another lane may set the word's other half)
            const uint32_t sh = 4u * ((k >> 5) & 1u);
            atomicOr(&sbm[2u * (k & 31u) + (k >> 6)],
                     ((g[0] >> sh) | (g[1] >> (sh + 1))) | ((g[2] >> (sh + 2)) | (g[3] >> (sh + 3))));
        }
        if (WRITE) {
            const uint32_t inc = warp_incl_scan(n, lane);
            uint64_t rk = out + inc - n;
            const uint64_t pos0 = s0 + warp * kWarpStarts + 16u * k;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t fw = g[i];
                while (fw) {
                    const uint32_t b = (uint32_t)(__ffs(fw) - 1) >> 3;
                    if (rk < cap) d_pos[rk] = pos0 + 4u * i + b;
                    ++rk;
                    fw &= fw - 1;
                }
            }
            out += __shfl_sync(kFull, inc, 31);
        } else {
            tile_count += n;
        }
    }
    SMK_STATS(cmp_stats_add(kChunks, kChunks * r, st_alive, st_sparse);)
    __syncwarp();   // the queue is reused by the next tile; sbm is complete
    if (bm && __any_sync(kFull, tile_count != 0u)) {
        const uint32_t e = store_slot(bm, lane, sbm[2 * lane], sbm[2 * lane + 1]);
        if (ent) *ent = e;
    }
    return tile_count;
}

// ------------------------------------------------------------ packed texts

// Texts of at most four distinct symbols are compared on 2-bit codes: a
// symbol's code is its bits b1 and b2 (bit b1 -> code bit 0, b2 -> bit 1),
// two bit positions where the text's symbols all differ. 16 codes fill a
// 32-bit word, code k of packed word u being the symbol at byte 16u + k of
// the stage buffer, in bits 2k and 2k + 1.
//
// The 2-bit codes of the four bytes of w, in bits 8j .. 8j + 1 of byte j.
template <bool ADJ>
__device__ __forceinline__ uint32_t byte_codes(uint32_t w, uint32_t b1, uint32_t b2) {
    if (ADJ) return (w >> b1) & 0x03030303u;   // b2 == b1 + 1
    return ((w >> b1) & 0x01010101u) | ((w >> (b2 - 1)) & 0x02020202u);
}

// 16 bytes -> one packed word. Multiplying the byte codes by gather =
// 0x01041040 moves the code of byte j to bits 24 + 2j (the partial products
// below bit 24 sum to less than 2^24, so nothing carries into byte 3); byte
// permutes collect the four top bytes.
template <bool ADJ>
__device__ __forceinline__ uint32_t pack16(const uint4& x, uint32_t b1, uint32_t b2, uint32_t gather) {
    const uint32_t u0 = byte_codes<ADJ>(x.x, b1, b2) * gather;
    const uint32_t u1 = byte_codes<ADJ>(x.y, b1, b2) * gather;
    const uint32_t u2 = byte_codes<ADJ>(x.z, b1, b2) * gather;
    const uint32_t u3 = byte_codes<ADJ>(x.w, b1, b2) * gather;
    return __byte_perm(__byte_perm(u0, u1, 0x7373u), __byte_perm(u2, u3, 0x7373u), 0x5410u);
}

// One compare on packed words, accumulated for the lane's 64 starts (four
// packed words of 16 starts) in each of two tiles: y[t] |= window ^ (c..c),
// with a[t], b[t] the lane's packed words 4E' .. 4E' + 7 past its first in
// tile t. v = (e << 8) | code with e = text misalignment + pattern position;
// the caller guarantees E' == e >> 6 and D == (e >> 4) & 3. ALIGNED:
// e mod 16 == 0 (no shift).
template <int D, bool ALIGNED, int NT = 2>
__device__ __forceinline__ void acc_packed(const uint4 (&a)[2], const uint4 (&b)[2], uint32_t v,
                                           uint32_t (&y)[2][4]) {
    const uint32_t P = (v & 3u) * 0x55555555u;
    const uint32_t sh = ((v >> 8) & 15u) << 1;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const uint32_t X[8] = {a[t].x, a[t].y, a[t].z, a[t].w, b[t].x, b[t].y, b[t].z, b[t].w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            y[t][i] |= (ALIGNED ? X[D + i] : __funnelshift_r(X[D + i], X[D + i + 1], sh)) ^ P;
    }
}

// bit 2k of x -> bit k (k = 0..15)
__device__ __forceinline__ uint32_t compress_even(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    return (x | (x >> 8)) & 0x0000FFFFu;
}

// found bits (bit 2k of a packed word: start k) of the 2-bit fields of y
// that are zero
__device__ __forceinline__ uint32_t zero_fields(uint32_t y) { return ~(y | (y >> 1)) & 0x55555555u; }

__device__ __forceinline__ uint32_t valid_fields(int64_t lim) {
    if (lim >= 16) return 0x55555555u;
    if (lim <= 0) return 0u;
    return 0x55555555u & ((1u << (2 * lim)) - 1u);
}

// One consumer warp's 2048 starts in each of two staged tiles against one
// pattern, on the packed words pk[t] of tile t (lane l's 64 starts from
// packed word 128 warp + 4l); the second tile takes part only when `two`.
// Same algorithm as warp_tile: the dense phase runs the r peeled compares
// (window groups: E' in bits 0-8, aligned compare of class D at bit 9 + D,
// number of other compares of class D in bits 13 + 4D .. 16 + 4D) and one
// zero test; then each lane continues its surviving 16-start words through
// compares r .. m-1 with early exit. Returns the lane's matches per tile;
// with WRITE also writes tile t's positions in ascending order from rank
// out[t] (first `cap` only). bm[t] (tile-count pass of a report): when the
// warp-tile of tile t has matches, its found bitmap (64 words, start order)
// is stored there. NT = 1 takes tile 0 only (pk[1] is not read).
template <bool WRITE, bool DIRECT, int NT = 2, class QC>
__device__ __forceinline__ uint2 packed_tiles(const uint32_t* const (&pk)[2], bool two, uint32_t warp,
                                              uint32_t lane, QC qc, uint32_t m, uint32_t r, uint32_t ng,
                                              uint64_t nstarts, const uint64_t (&s0)[2], const uint64_t (&out)[2],
                                              uint64_t* __restrict__ d_pos, uint64_t cap,
                                              uint32_t* const (&bm)[2], uint32_t* ent = nullptr) {
    const uint32_t w0 = warp * 128u + lane * 4u;   // lane's first packed word
    uint32_t y[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
    for (uint32_t g = 0, j = 0; g < ng; ++g) {
        const uint32_t gd = qc.group(g);
        const uint32_t u = (w0 >> 2) + (gd & 0x1FFu);
        uint4 a[2], b[2];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint4* p4 = reinterpret_cast<const uint4*>(pk[t]);
            a[t] = p4[u];
            b[t] = p4[u + 1];
        }
        if (gd & (1u << 9)) acc_packed<0, true, NT>(a, b, qc(j++), y);
        if (gd & (1u << 10)) acc_packed<1, true, NT>(a, b, qc(j++), y);
        if (gd & (1u << 11)) acc_packed<2, true, NT>(a, b, qc(j++), y);
        if (gd & (1u << 12)) acc_packed<3, true, NT>(a, b, qc(j++), y);
        for (uint32_t k = (gd >> 13) & 15u; k; --k) acc_packed<0, false, NT>(a, b, qc(j++), y);
        for (uint32_t k = (gd >> 17) & 15u; k; --k) acc_packed<1, false, NT>(a, b, qc(j++), y);
        for (uint32_t k = (gd >> 21) & 15u; k; --k) acc_packed<2, false, NT>(a, b, qc(j++), y);
        for (uint32_t k = (gd >> 25) & 15u; k; --k) acc_packed<3, false, NT>(a, b, qc(j++), y);
    }
    uint32_t f[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
#pragma unroll
    for (int t = 0; t < NT; ++t) {
#pragma unroll
        for (int i = 0; i < 4; ++i) f[t][i] = (t == 0 || two) ? zero_fields(y[t][i]) : 0u;
        if (s0[t] + kTile > nstarts) {   // last tile: clear starts beyond n - m
            const int64_t lim = (int64_t)(nstarts - s0[t]) - (int64_t)(warp * kWarpStarts + lane * 64u);
#pragma unroll
            for (int i = 0; i < 4; ++i) f[t][i] &= valid_fields(lim - 16 * i);
        }
    }
    // surviving starts continue one compare at a time; rare when r is planned
    uint32_t any = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) any |= (f[t][0] | f[t][1]) | (f[t][2] | f[t][3]);
    SMK_STATS(uint32_t st_words = 0, st_alive = 0, st_sparse = 0;)
    SMK_STATS(for (int t = 0; t < NT; ++t) if (t == 0 || two) {
        st_words += 4;
        for (int i = 0; i < 4; ++i) st_alive += f[t][i] ? 1u : 0u;
    })
    if (!(DIRECT && r >= m) && __any_sync(kFull, any != 0u)) {
        const uint32_t jl = min(m, r + kLaneCompares);
        for (uint32_t j = r; j < jl && any; ++j) {
            const uint32_t v = qc(j);
            const uint32_t e = v >> 8;
            const uint32_t P = (v & 3u) * 0x55555555u;
            const uint32_t sh = (e & 15u) << 1;
            any = 0;
#pragma unroll
            for (int t = 0; t < NT; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (f[t][i]) {
                        SMK_STATS(++st_sparse;)
                        const uint32_t W = w0 + i + (e >> 4);
                        f[t][i] &= zero_fields(__funnelshift_r(pk[t][W], pk[t][W + 1], sh) ^ P);
                    }
                    any |= f[t][i];
                }
        }
        // words still alive: the whole warp takes the remaining compares of
        // one word at a time (lane l every 32nd from jl + l) and ANDs
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t pend = __ballot_sync(kFull, jl < m && f[t][i] != 0u);
                while (pend) {
                    const uint32_t src = (uint32_t)__ffs(pend) - 1u;
                    pend &= pend - 1u;
                    const uint32_t ws = __shfl_sync(kFull, w0, src) + i;
                    SMK_STATS(if (lane == src) st_sparse += m - jl;)
                    uint32_t y = 0;
                    for (uint32_t j = jl + lane; j < m; j += 32) {
                        const uint32_t v = qc(j);
                        const uint32_t e = v >> 8;
                        const uint32_t W = ws + (e >> 4);
                        y |= __funnelshift_r(pk[t][W], pk[t][W + 1], (e & 15u) << 1) ^ ((v & 3u) * 0x55555555u);
                    }
                    uint32_t keep = zero_fields(y);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) keep &= __shfl_xor_sync(kFull, keep, o);
                    if (lane == src) f[t][i] &= keep;
                }
            }
    }
    SMK_STATS(cmp_stats_add(st_words, st_words * r, (DIRECT && r >= m) ? 0u : st_alive, st_sparse);)
    uint32_t n[2] = {0u, 0u};
#pragma unroll
    for (int t = 0; t < NT; ++t) n[t] = __popc(f[t][0] | (f[t][1] << 1)) + __popc(f[t][2] | (f[t][3] << 1));
#pragma unroll
    for (int t = 0; t < NT; ++t)
        if (bm[t] && __any_sync(kFull, n[t] != 0u)) {
            // the warp-tile's slot: lane l's 64 starts in order (found bit
            // 2k of a packed word -> bit k)
            uint32_t c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) c[i] = compress_even(f[t][i]);
            const uint32_t e = store_slot(bm[t], lane, c[0] | (c[1] << 16), c[2] | (c[3] << 16));
            if (ent) ent[t] = e;
        }
    if (WRITE) {
        // positions in order: lanes, then words, then starts
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint32_t inc = warp_incl_scan(n[t], lane);
            uint64_t rk = out[t] + inc - n[t];
            const uint64_t pos0 = s0[t] + warp * kWarpStarts + 64u * lane;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t fw = f[t][i];
                while (fw) {
                    const uint32_t k = (uint32_t)(__ffs(fw) - 1) >> 1;
                    if (rk < cap) d_pos[rk] = pos0 + 16u * i + k;
                    ++rk;
                    fw &= fw - 1;
                }
            }
        }
    }
    return make_uint2(n[0], n[1]);
}

// ------------------------------------------------------------ binary texts

// Texts of at most two distinct symbols are compared on 1-bit codes: a
// symbol's code is its bit b1, where the two symbols differ. 32 codes fill a
// word, code k of word u being the symbol at byte 32u + k of the stage buffer,
// in bit k.
//
// Bit b1 of the four bytes of w, in bits 24 + j (byte j): the multiplier
// 0x01020408 moves byte j's bit (at 8j) to 24 + j; the other partial
// products land on distinct bits below 24 or beyond 31, so nothing carries
// into bits 24-31.
__device__ __forceinline__ uint32_t nib4(uint32_t w, uint32_t b1) { return ((w >> b1) & 0x01010101u) * 0x01020408u; }

// 32 bytes (x0: bytes 0-15, x1: bytes 16-31) -> one word of 1-bit codes.
// Byte permutes collect the nibbles of the even and the odd 4-byte groups;
// nibble k lands at bits 4k .. 4k + 3.
__device__ __forceinline__ uint32_t pack32(const uint4& x0, const uint4& x1, uint32_t b1) {
    const uint32_t n0 = nib4(x0.x, b1), n1 = nib4(x0.y, b1), n2 = nib4(x0.z, b1), n3 = nib4(x0.w, b1);
    const uint32_t n4 = nib4(x1.x, b1), n5 = nib4(x1.y, b1), n6 = nib4(x1.z, b1), n7 = nib4(x1.w, b1);
    const uint32_t lo = __byte_perm(__byte_perm(n0, n2, 0x7373u), __byte_perm(n4, n6, 0x7373u), 0x5410u);
    const uint32_t hi = __byte_perm(__byte_perm(n1, n3, 0x7373u), __byte_perm(n5, n7, 0x7373u), 0x5410u);
    return lo | (hi << 4);
}

// One compare on 1-bit codes for the lane's 64 starts (two words) in each of
// two tiles: y[t][i] |= window ^ (c..c), X[t] the lane's words 2E' .. 2E' + 3
// past its first in tile t. v = (e << 8) | code; the caller guarantees
// E' == e >> 6 and D == (e >> 5) & 1. ALIGNED: e mod 32 == 0 (no shift).
template <int D, bool ALIGNED>
__device__ __forceinline__ void acc_bin(const uint32_t (&X)[2][4], uint32_t v, uint32_t (&y)[2][2]) {
    const uint32_t P = 0u - (v & 1u);
    const uint32_t sh = (v >> 8) & 31u;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int i = 0; i < 2; ++i)
            y[t][i] |= (ALIGNED ? X[t][D + i] : __funnelshift_r(X[t][D + i], X[t][D + i + 1], sh)) ^ P;
}

__device__ __forceinline__ uint32_t valid_bits(int64_t lim) {
    if (lim >= 32) return ~0u;
    if (lim <= 0) return 0u;
    return (1u << lim) - 1u;
}

// packed_tiles for 1-bit codes: one consumer warp's 2048 starts in each of
// two staged tiles, on the words pk[t] of tile t (lane l's 64 starts are
// words 64 warp + 2l and the next). Same phases, results and outputs as
// packed_tiles; a found bit is a start, so the bitmap of a warp-tile is the
// found words themselves.
template <bool WRITE, bool DIRECT, class QC>
__device__ __forceinline__ uint2 binary_tiles(const uint32_t* const (&pk)[2], bool two, uint32_t warp,
                                              uint32_t lane, QC qc, uint32_t m, uint32_t r, uint32_t ng,
                                              uint64_t nstarts, const uint64_t (&s0)[2], const uint64_t (&out)[2],
                                              uint64_t* __restrict__ d_pos, uint64_t cap,
                                              uint32_t* const (&bm)[2], uint32_t* ent = nullptr) {
    const uint32_t w0 = warp * 64u + lane * 2u;   // lane's first word
    uint32_t y[2][2] = {{0u, 0u}, {0u, 0u}};
    for (uint32_t g = 0, j = 0; g < ng; ++g) {
        const uint32_t gd = qc.group(g);
        const uint32_t u = w0 + 2u * (gd & 0x1FFu);
        uint32_t X[2][4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint2 a = *reinterpret_cast<const uint2*>(pk[t] + u);
            const uint2 b = *reinterpret_cast<const uint2*>(pk[t] + u + 2);
            X[t][0] = a.x;
            X[t][1] = a.y;
            X[t][2] = b.x;
            X[t][3] = b.y;
        }
        if (gd & (1u << 9)) acc_bin<0, true>(X, qc(j++), y);
        if (gd & (1u << 10)) acc_bin<1, true>(X, qc(j++), y);
        for (uint32_t k = (gd >> 13) & 31u; k; --k) acc_bin<0, false>(X, qc(j++), y);
        for (uint32_t k = (gd >> 18) & 31u; k; --k) acc_bin<1, false>(X, qc(j++), y);
    }
    uint32_t f[2][2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
#pragma unroll
        for (int i = 0; i < 2; ++i) f[t][i] = (t == 0 || two) ? ~y[t][i] : 0u;
        if (s0[t] + kTile > nstarts) {   // last tile: clear starts beyond n - m
            const int64_t lim = (int64_t)(nstarts - s0[t]) - (int64_t)(warp * kWarpStarts + lane * 64u);
#pragma unroll
            for (int i = 0; i < 2; ++i) f[t][i] &= valid_bits(lim - 32 * i);
        }
    }
    uint32_t any = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) any |= f[t][0] | f[t][1];
    if (!(DIRECT && r >= m) && __any_sync(kFull, any != 0u)) {
        const uint32_t jl = min(m, r + kLaneCompares);
        for (uint32_t j = r; j < jl && any; ++j) {
            const uint32_t v = qc(j);
            const uint32_t e = v >> 8;
            const uint32_t P = 0u - (v & 1u);
            const uint32_t sh = e & 31u;
            any = 0;
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (f[t][i]) {
                        const uint32_t W = w0 + i + (e >> 5);
                        f[t][i] &= ~(__funnelshift_r(pk[t][W], pk[t][W + 1], sh) ^ P);
                    }
                    any |= f[t][i];
                }
        }
        // words still alive: the whole warp takes the remaining compares of
        // one word at a time (lane l every 32nd from jl + l) and ANDs
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                uint32_t pend = __ballot_sync(kFull, jl < m && f[t][i] != 0u);
                while (pend) {
                    const uint32_t src = (uint32_t)__ffs(pend) - 1u;
                    pend &= pend - 1u;
                    const uint32_t ws = __shfl_sync(kFull, w0, src) + i;
                    uint32_t yy = 0;
                    for (uint32_t j = jl + lane; j < m; j += 32) {
                        const uint32_t v = qc(j);
                        const uint32_t e = v >> 8;
                        const uint32_t W = ws + (e >> 5);
                        yy |= __funnelshift_r(pk[t][W], pk[t][W + 1], e & 31u) ^ (0u - (v & 1u));
                    }
                    uint32_t keep = ~yy;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) keep &= __shfl_xor_sync(kFull, keep, o);
                    if (lane == src) f[t][i] &= keep;
                }
            }
    }
    uint32_t n[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) n[t] = __popc(f[t][0]) + __popc(f[t][1]);
#pragma unroll
    for (int t = 0; t < 2; ++t)
        if (bm[t] && __any_sync(kFull, n[t] != 0u)) {   // lane l's 64 starts in order: its found words
            const uint32_t e = store_slot(bm[t], lane, f[t][0], f[t][1]);
            if (ent) ent[t] = e;
        }
    if (WRITE) {
        // positions in order: lanes, then words, then starts
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint32_t inc = warp_incl_scan(n[t], lane);
            uint64_t rk = out[t] + inc - n[t];
            const uint64_t pos0 = s0[t] + warp * kWarpStarts + 64u * lane;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                uint32_t fw = f[t][i];
                while (fw) {
                    const uint32_t k = (uint32_t)(__ffs(fw) - 1);
                    if (rk < cap) d_pos[rk] = pos0 + 32u * i + k;
                    ++rk;
                    fw &= fw - 1;
                }
            }
        }
    }
    return make_uint2(n[0], n[1]);
}

}  // namespace dev
}  // namespace smk
