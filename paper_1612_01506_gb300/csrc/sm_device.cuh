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

}  // namespace dev
}  // namespace smk
