// Device helpers shared by the scan and batch kernels: mbarrier and TMA
// wrappers, bounded waits, the SWAR byte compare and warp reductions.
// Internal to the library.
#pragma once

#include "sm_internal.h"

namespace smk {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint64_t kEnd = ~0ull;

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

// found &= [byte of w == byte of P], flags in the high bit of each byte.
// General bytes: exact zero-byte test of x = w ^ P: the high bit of
// ((x & 0x7F..) + 0x7F..) | x is set iff the byte is nonzero.
// SEVEN: every byte of w and P is below 0x80, so x + 0x7F.. cannot carry
// between bytes and its high bit alone marks a nonzero byte.
// With SMK_MADD_ADD the add is a multiply-add by `one` (== 1) so that it
// issues on the multiply-add pipe instead of the integer pipe.
#ifndef SMK_MADD_ADD
#define SMK_MADD_ADD 1
#endif
template <bool SEVEN>
__device__ __forceinline__ uint32_t keep_equal(uint32_t f, uint32_t w, uint32_t P, uint32_t one) {
    const uint32_t x = w ^ P;
#if SMK_MADD_ADD
    if (SEVEN) return f & ~(x * one + 0x7F7F7F7Fu);
    return f & ~(((x & 0x7F7F7F7Fu) * one + 0x7F7F7F7Fu) | x);
#else
    (void)one;
    if (SEVEN) return f & ~(x + 0x7F7F7F7Fu);
    return f & ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x);
#endif
}

template <bool SEVEN, int D>
__device__ __forceinline__ void cmp_chunk(const uint4& a, const uint4& b, uint32_t sh, uint32_t P, uint32_t one,
                                          uint32_t (&f)[4]) {
    const uint32_t X[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = keep_equal<SEVEN>(f[i], __funnelshift_r(X[D + i], X[D + i + 1], sh), P, one);
}

// One SIMDcompare for the lane's NC 16-start chunks (chunk c at index
// c0 + 32c). v = (e << 8) | symbol with e = text misalignment + pattern
// position; the caller guarantees D == (e >> 2) & 3, so the word selection is
// static. All 2*NC loads issue before the compares.
template <bool SEVEN, int D, int NC>
__device__ __forceinline__ void compare_chunks(const uint4* __restrict__ b4, uint32_t c0, uint32_t v, uint32_t one,
                                               uint32_t (&f)[NC][4]) {
    const uint32_t e = v >> 8;
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
    const uint32_t ci = c0 + (e >> 4);
    const uint32_t sh = (e & 3u) << 3;
    uint4 a[NC], b[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        a[c] = b4[ci + 32 * c];
        b[c] = b4[ci + 32 * c + 1];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) cmp_chunk<SEVEN, D>(a[c], b[c], sh, P, one, f[c]);
}

// One SIMDcompare for a single 4-start word whose first start is at word
// index `wbase` of the stage buffer.
template <bool SEVEN>
__device__ __forceinline__ uint32_t compare_word(const uint32_t* __restrict__ b32, uint32_t wbase, uint32_t v,
                                                 uint32_t one, uint32_t f) {
    const uint32_t e = v >> 8;
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
    const uint32_t W = wbase + (e >> 2);
    const uint32_t w = __funnelshift_r(b32[W], b32[W + 1], (e & 3u) << 3);
    return keep_equal<SEVEN>(f, w, P, one);
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

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

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
    uint32_t qc[MAXM];   // compare j: (e_j << 8) | p[pi(j)], e_j = (text address mod 16) + pi(j)
};

// ------------------------------------------------------------ one warp-tile

// Compare descriptors held in the kernel's parameter block.
template <int MAXM>
struct ParamQC {
    const PatArg<MAXM>* p;
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return p->qc[j]; }
};

// Compare descriptors in global memory (read-only, uniform across the warp).
struct GlobalQC {
    const uint32_t* __restrict__ p;
    __device__ __forceinline__ uint32_t operator()(uint32_t j) const { return __ldg(p + j); }
};

// One consumer warp's 2048 starts of a staged tile against one pattern:
// Algorithms 2-4 (dense peeled compares, compaction of surviving words,
// per-word early exit). Starts at or beyond nstarts (relative to the tile's
// first start s0) are out of range. Returns this lane's number of
// matches; with WRITE, also
// writes the positions in ascending order from rank `out` (first `cap` only).
// DIRECT: a count may skip the compaction when r >= m.
template <bool SEVEN, bool WRITE, bool DIRECT, class QC>
__device__ __forceinline__ uint32_t warp_tile(const uint4* __restrict__ b4, const uint32_t* __restrict__ b32,
                                              uint32_t c0, uint32_t wq, uint32_t warp, uint32_t lane, QC qc,
                                              uint32_t m, uint32_t r, uint32_t nd0, uint32_t nd1, uint32_t nd2,
                                              uint32_t nd3, uint32_t one, uint64_t nstarts, uint64_t s0, uint2* q,
                                              uint64_t out, uint64_t* __restrict__ d_pos, uint64_t cap) {
    // dense phase: r compares for all starts of the warp; the peeled
    // compares arrive grouped by word alignment (A.nd)
    uint32_t f[kChunks][4];
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) f[c][i] = 0x80808080u;
    {
        uint32_t j = 0;
        for (uint32_t k = 0; k < nd0; ++k, ++j) compare_chunks<SEVEN, 0>(b4, c0, qc(j), one, f);
        for (uint32_t k = 0; k < nd1; ++k, ++j) compare_chunks<SEVEN, 1>(b4, c0, qc(j), one, f);
        for (uint32_t k = 0; k < nd2; ++k, ++j) compare_chunks<SEVEN, 2>(b4, c0, qc(j), one, f);
        for (uint32_t k = 0; k < nd3; ++k, ++j) compare_chunks<SEVEN, 3>(b4, c0, qc(j), one, f);
    }

    if (s0 + kTile > nstarts) {   // last tile: clear starts beyond n - m
        const int64_t lim = (int64_t)(nstarts - s0) - (int64_t)(warp * kWarpStarts + lane * 16u);
#pragma unroll
        for (int c = 0; c < kChunks; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i) f[c][i] &= valid_mask(lim - (512 * c + 4 * i));
    }

    uint32_t any = 0;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) any |= (f[c][0] | f[c][1]) | (f[c][2] | f[c][3]);

    uint32_t tile_count = 0;   // this lane's share of the warp's matches in the tile
    if (DIRECT && r >= m) {
        tile_count = count_flags<kChunks>(f);
    } else if (__any_sync(kFull, any != 0u)) {
        // compact surviving words in position order: chunk 0 of all
        // lanes, then chunk 1, ... (4 bits per chunk, counts in bytes)
        uint32_t a[kChunks], packed = 0;
#pragma unroll
        for (int c = 0; c < kChunks; ++c) {
            a[c] = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) a[c] |= (f[c][i] != 0u) << i;
            packed |= (uint32_t)__popc(a[c]) << (8 * c);
        }
        const uint32_t incl = warp_incl_scan(packed, lane);
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        const uint32_t qn = (tot & 0xFFu) + ((tot >> 8) & 0xFFu) + ((tot >> 16) & 0xFFu) + (tot >> 24);

        if (qn <= kQueueCap) {
            uint32_t base = 0;
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                uint32_t p = base + ((incl >> (8 * c)) & 0xFFu) - ((packed >> (8 * c)) & 0xFFu);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (a[c] & (1u << i)) q[p++] = make_uint2(128u * c + lane * 4u + i, f[c][i]);
                base += (tot >> (8 * c)) & 0xFFu;
            }
            __syncwarp();
            // sparse phase: each lane continues one word with its own early exit
            for (uint32_t qb = 0; qb < qn; qb += 32) {
                const uint32_t e = qb + lane;
                uint32_t wi = 0, fw = 0;
                if (e < qn) {
                    const uint2 x = q[e];
                    wi = x.x;
                    fw = x.y;
                }
                for (uint32_t j = r; j < m && fw; ++j) fw = compare_word<SEVEN>(b32, wq + wi, qc(j), one, fw);
                const uint32_t k = __popc(fw);
                if (WRITE) {
                    const uint32_t inc = warp_incl_scan(k, lane);
                    uint64_t rk = out + inc - k;
                    const uint64_t pos0 = s0 + warp * kWarpStarts + 4u * wi;
                    while (fw) {
                        const uint32_t b = (uint32_t)(__ffs(fw) - 1) >> 3;
                        if (rk < cap) d_pos[rk] = pos0 + b;
                        ++rk;
                        fw &= fw - 1;
                    }
                    out += __shfl_sync(kFull, inc, 31);
                } else {
                    tile_count += k;
                }
            }
            __syncwarp();   // the queue is reused by the next tile
        } else {
            // more survivors than the queue holds: continue the remaining
            // compares for all of the warp's starts, leaving when all are dead
            for (uint32_t j = r; j < m; ++j) {
                uint32_t an = 0;
#pragma unroll
                for (int c = 0; c < kChunks; ++c) an |= (f[c][0] | f[c][1]) | (f[c][2] | f[c][3]);
                if (!__any_sync(kFull, an != 0u)) break;
                const uint32_t v = qc(j);
                switch ((v >> 10) & 3u) {
                    case 0: compare_chunks<SEVEN, 0>(b4, c0, v, one, f); break;
                    case 1: compare_chunks<SEVEN, 1>(b4, c0, v, one, f); break;
                    case 2: compare_chunks<SEVEN, 2>(b4, c0, v, one, f); break;
                    default: compare_chunks<SEVEN, 3>(b4, c0, v, one, f); break;
                }
            }
            if (WRITE) {
                // positions in order: chunk c of all lanes, words, bytes
                uint32_t kc[kChunks];
#pragma unroll
                for (int c = 0; c < kChunks; ++c)
                    kc[c] = __popc(f[c][0]) + __popc(f[c][1]) + __popc(f[c][2]) + __popc(f[c][3]);
                const uint32_t i01 = warp_incl_scan(kc[0] | (kc[1] << 16), lane);
                const uint32_t i23 = warp_incl_scan(kc[2] | (kc[3] << 16), lane);
                const uint32_t t01 = __shfl_sync(kFull, i01, 31), t23 = __shfl_sync(kFull, i23, 31);
                const uint32_t incs[4] = {i01 & 0xFFFFu, i01 >> 16, i23 & 0xFFFFu, i23 >> 16};
                const uint32_t tots[4] = {t01 & 0xFFFFu, t01 >> 16, t23 & 0xFFFFu, t23 >> 16};
                uint64_t cb = out;
#pragma unroll
                for (int c = 0; c < kChunks; ++c) {
                    uint64_t rk = cb + incs[c] - kc[c];
                    const uint64_t pos0 = s0 + warp * kWarpStarts + 512u * c + 16u * lane;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        uint32_t fw = f[c][i];
                        while (fw) {
                            const uint32_t b = (uint32_t)(__ffs(fw) - 1) >> 3;
                            if (rk < cap) d_pos[rk] = pos0 + 4u * i + b;
                            ++rk;
                            fw &= fw - 1;
                        }
                    }
                    cb += tots[c];
                }
            } else {
                tile_count += count_flags<kChunks>(f);
            }
        }
    }

    return tile_count;
}

}  // namespace dev
}  // namespace smk
