// Kernels of the SIMD-naive search (Tarhio, Holub, Giaquinta, Sec. 2), for sm_103a.
//
// scan_kernel  - Algorithms 2-4 on the GPU. A CTA owns a contiguous range of
//                tiles of kTile = 8192 start positions. Each tile's bytes plus
//                the (m-1)-byte halo are staged in shared memory by a 1-D TMA
//                bulk copy (cp.async.bulk) into a ring of `stages` buffers
//                completed through mbarriers. Warp w owns starts
//                [1024w, 1024w+1024) of the tile; lane l owns the two 16-start
//                chunks at 1024w + 16l and 1024w + 512 + 16l, so every 16-byte
//                shared-memory load of a warp touches 512 consecutive bytes
//                (no bank conflicts). For compare j at pattern position
//                q = pi(j) a lane loads the two 16-byte chunks covering bytes
//                s+q .. s+q+15 of its 16 starts s, aligns them with funnel
//                shifts and tests 4 bytes per 32-bit word against the
//                broadcast symbol p[q] with an exact SWAR zero-byte test. The
//                result is the paper's SIMDcompare mask for 16 starts, kept as
//                the high bit of each byte ("found"). The first r compares run
//                without the zero test (loop peeling, Sec. 2.3); later ones
//                leave when the whole warp's found masks are zero (the early
//                exit of Algorithm 2, taken per warp of 1024 starts). The
//                count is the popcount of found (Algorithm 2).
// hist_kernel  - byte histogram of the text (the frequencies of Sec. 2.2).
//
// Every wait on an mbarrier is bounded by a %globaltimer deadline; on expiry
// the kernel records kStatusTimeout, waits (bounded) for its copies in
// flight and leaves its tile loop.
#include "sm_internal.h"

namespace smk {
namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint64_t kEnd = ~0ull;

template <int MAXM>
struct PatArg {
    uint32_t qc[MAXM];   // compare j: (pi(j) << 8) | p[pi(j)]
};

struct StageDesc {
    uint64_t tile;       // kEnd: no more tiles
    uint64_t offset;     // output offset of the tile's first match (report)
};

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

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
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

// Wait for phase `parity` of `bar` to complete, at most limit_ns.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// ------------------------------------------------------------ compare core

// found &= [byte of w == byte of P] in the high bit of each byte.
// General bytes: exact zero-byte test of x = w ^ P (high bit of
// ((x & 0x7F..) + 0x7F..) | x is set iff the byte is nonzero).
// SEVEN: every byte of w and P is below 0x80, so x + 0x7F.. cannot carry
// between bytes and its high bit alone marks a nonzero byte.
template <bool SEVEN>
__device__ __forceinline__ uint32_t keep_equal(uint32_t f, uint32_t w, uint32_t P) {
    const uint32_t x = w ^ P;
    if (SEVEN) return f & ~(x + 0x7F7F7F7Fu);
    return f & ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x);
}

template <bool SEVEN, int D>
__device__ __forceinline__ void cmp_chunk(const uint4& a, const uint4& b, uint32_t sh, uint32_t P,
                                          uint32_t (&f)[4]) {
    const uint32_t X[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) f[i] = keep_equal<SEVEN>(f[i], __funnelshift_r(X[D + i], X[D + i + 1], sh), P);
}

// One SIMDcompare for the lane's two chunks: v = (q << 8) | symbol.
template <bool SEVEN>
__device__ __forceinline__ void compare2(const uint4* __restrict__ b4, uint32_t c0, uint32_t v, uint32_t delta,
                                         uint32_t (&f0)[4], uint32_t (&f1)[4]) {
    const uint32_t e = delta + (v >> 8);
    const uint32_t P = (v & 0xFFu) * 0x01010101u;
    const uint32_t ci = c0 + (e >> 4);
    const uint32_t sh = (e & 3u) << 3;
    const uint4 a0 = b4[ci], b0 = b4[ci + 1], a1 = b4[ci + 32], b1 = b4[ci + 33];
    switch ((e >> 2) & 3u) {
        case 0: cmp_chunk<SEVEN, 0>(a0, b0, sh, P, f0); cmp_chunk<SEVEN, 0>(a1, b1, sh, P, f1); break;
        case 1: cmp_chunk<SEVEN, 1>(a0, b0, sh, P, f0); cmp_chunk<SEVEN, 1>(a1, b1, sh, P, f1); break;
        case 2: cmp_chunk<SEVEN, 2>(a0, b0, sh, P, f0); cmp_chunk<SEVEN, 2>(a1, b1, sh, P, f1); break;
        default: cmp_chunk<SEVEN, 3>(a0, b0, sh, P, f0); cmp_chunk<SEVEN, 3>(a1, b1, sh, P, f1); break;
    }
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

// ------------------------------------------------------------ scan kernel

template <int MAXM, int MODE, bool SEVEN>
__global__ void __launch_bounds__(kThreads) scan_kernel(const __grid_constant__ ScanArgs A,
                                                        const __grid_constant__ PatArg<MAXM> P) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);                 // [kMaxStages]
    StageDesc* desc = reinterpret_cast<StageDesc*>(smem + 64);           // [kMaxStages]
    uint32_t* wsum = reinterpret_cast<uint32_t*>(smem + 192);            // [8]
    uint64_t* red = reinterpret_cast<uint64_t*>(smem + 224);             // [8]
    uint32_t* flag = reinterpret_cast<uint32_t*>(smem + 288);
    uint8_t* bufs = smem + kScanHeader;

    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t SB = A.stage_bytes, S = A.stages, m = A.m;
    const uint64_t t_begin = (uint64_t)blockIdx.x * A.tiles_per_cta;
    const uint64_t t_end = min(t_begin + A.tiles_per_cta, A.ntiles);
    const uintptr_t tb = reinterpret_cast<uintptr_t>(A.text);
    const uint32_t delta = (uint32_t)(tb & 15u);
    // text indices [lo_al, hi_al) are the 16-byte aligned interior reachable by TMA
    const int64_t lo_al = (int64_t)(((tb + 15u) & ~(uintptr_t)15u) - tb);
    const int64_t hi_al = (int64_t)((tb + A.n) & ~(uintptr_t)15u) - (int64_t)tb;

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Producer state, uniform in warp 0.
    uint64_t cursor = t_begin, running = 0;
    if (MODE == kModeWrite) {
        if (warp == 0) {
            uint64_t b = 0;
            for (uint32_t i = lane; i < blockIdx.x; i += 32) b += __ldcg(A.partials + i);
            running = warp_sum_u64(b);
        } else if (warp == 1 && blockIdx.x == 0) {
            uint64_t b = 0;
            for (uint32_t i = lane; i < gridDim.x; i += 32) b += __ldcg(A.partials + i);
            b = warp_sum_u64(b);
            if (lane == 0 && b > A.cap) atomicOr(A.status, kStatusTrunc);
        }
    }

    // Warp 0: choose the next tile, publish its descriptor, start its copy.
    auto issue = [&](uint32_t s) {
        uint64_t tile = kEnd;
        uint32_t tcount = 0;
        if (MODE != kModeWrite) {
            if (cursor < t_end) tile = cursor++;
        } else {
            while (cursor < t_end) {
                const uint64_t idx = cursor + lane;
                const uint32_t c = idx < t_end ? __ldcg(A.tile_counts + idx) : 0u;
                const uint32_t bal = __ballot_sync(kFull, c != 0);
                if (bal) {
                    const int k = __ffs(bal) - 1;
                    tcount = __shfl_sync(kFull, c, k);
                    tile = cursor + (uint64_t)k;
                    cursor = tile + 1;
                    break;
                }
                cursor += 32;
            }
        }
        if (lane == 0) {
            desc[s].tile = tile;
            desc[s].offset = running;
            uint32_t bytes = 0;
            uintptr_t ga = 0, g0 = 0;
            if (tile != kEnd) {
                const uint64_t s0 = tile * kTile;
                const uint64_t need_end = min(s0 + kTile + m - 1, A.n);
                g0 = (tb + s0) & ~(uintptr_t)15u;
                ga = max(g0, tb + (uintptr_t)lo_al);
                const uintptr_t ge = (tb + need_end + 15u) & ~(uintptr_t)15u;
                const uintptr_t gb = min(ge, (tb + A.n) & ~(uintptr_t)15u);
                bytes = gb > ga ? (uint32_t)(gb - ga) : 0u;
            }
            const bool skip = A.test_skip_copy && tile == 0;
            fence_proxy_async();
            mbar_arrive_expect_tx(&full[s], bytes);
            if (bytes && !skip) bulk_g2s(bufs + (size_t)s * SB + (ga - g0), reinterpret_cast<const void*>(ga), bytes,
                                         &full[s]);
        }
        running += tcount;
    };

    if (warp == 0)
        for (uint32_t s = 0; s < S; ++s) issue(s);

    uint32_t my_count = 0;
    const uint32_t c0 = warp * 64u + lane;   // lane's first 16-byte chunk in the tile

    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % S;
        const uint32_t par = (it / S) & 1u;
        const bool ok = wait_bounded(&full[s], par, A.spin_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.status, kStatusTimeout);
            // let every copy this CTA started land before leaving
            for (uint32_t k = 0; k < S; ++k) {
                const uint32_t it2 = it + k;
                (void)wait_bounded(&full[it2 % S], (it2 / S) & 1u, A.spin_ns);
            }
            break;
        }
        const StageDesc d = desc[s];
        if (d.tile == kEnd) break;

        uint8_t* buf = bufs + (size_t)s * SB;
        const uint64_t s0 = d.tile * kTile;
        const uint64_t need_end = min(s0 + kTile + m - 1, A.n);

        // bytes outside the aligned interior come in by plain loads
        const int64_t h_end = min((int64_t)need_end, lo_al);
        const int64_t t_beg = max((int64_t)s0, max(lo_al, max(hi_al, (int64_t)0)));
        const bool ragged = (int64_t)s0 < h_end || t_beg < (int64_t)need_end;
        if (ragged) {
            for (int64_t x = (int64_t)s0 + tid; x < h_end; x += kThreads) buf[delta + (x - (int64_t)s0)] = A.text[x];
            for (int64_t x = t_beg + tid; x < (int64_t)need_end; x += kThreads)
                buf[delta + (x - (int64_t)s0)] = A.text[x];
            __syncthreads();
        }

        uint32_t f0[4], f1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) f0[i] = f1[i] = 0x80808080u;
        const uint4* b4 = reinterpret_cast<const uint4*>(buf);
        uint32_t j = 0;
        for (; j < A.r; ++j) compare2<SEVEN>(b4, c0, P.qc[j], delta, f0, f1);
        for (; j < m; ++j) {
            const uint32_t any = (f0[0] | f0[1] | f0[2] | f0[3]) | (f1[0] | f1[1] | f1[2] | f1[3]);
            if (!__any_sync(kFull, any != 0)) break;
            compare2<SEVEN>(b4, c0, P.qc[j], delta, f0, f1);
        }

        const uint64_t U = min((uint64_t)kTile, A.nstarts - s0);   // valid starts in this tile
        if (U < kTile) {
            const int64_t u0 = (int64_t)(warp * 1024u + lane * 16u);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                f0[i] &= valid_mask((int64_t)U - (u0 + 4 * i));
                f1[i] &= valid_mask((int64_t)U - (u0 + 512 + 4 * i));
            }
        }

        uint32_t k0 = 0, k1 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) { k0 += __popc(f0[i]); k1 += __popc(f1[i]); }

        if (MODE != kModeWrite) {
            my_count += k0 + k1;
            if (MODE == kModeTileCount) {
                const uint32_t ws = warp_sum_u32(k0 + k1);
                if (lane == 0) wsum[warp] = ws;
            }
        } else {
            // ranks: warps in order, then chunk 0 of all lanes, then chunk 1
            uint32_t i0 = k0, i1 = k1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y0 = __shfl_up_sync(kFull, i0, o), y1 = __shfl_up_sync(kFull, i1, o);
                if (lane >= (uint32_t)o) { i0 += y0; i1 += y1; }
            }
            const uint32_t t0 = __shfl_sync(kFull, i0, 31), t1 = __shfl_sync(kFull, i1, 31);
            if (lane == 0) wsum[warp] = t0 + t1;
            __syncthreads();
            uint64_t base = d.offset;
            for (uint32_t w = 0; w < warp; ++w) base += wsum[w];
            uint64_t r0 = base + (i0 - k0), r1 = base + t0 + (i1 - k1);
            const uint64_t p0 = s0 + warp * 1024u + lane * 16u;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t f = f0[i];
                while (f) {
                    const uint32_t b = (uint32_t)(__ffs(f) - 1) >> 3;
                    if (r0 < A.cap) A.d_pos[r0] = p0 + 4 * i + b;
                    ++r0;
                    f &= f - 1;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t f = f1[i];
                while (f) {
                    const uint32_t b = (uint32_t)(__ffs(f) - 1) >> 3;
                    if (r1 < A.cap) A.d_pos[r1] = p0 + 512 + 4 * i + b;
                    ++r1;
                    f &= f - 1;
                }
            }
        }

        __syncthreads();   // everyone is done with buffer s and with wsum
        if (warp == 0) {
            if (MODE == kModeTileCount && lane == 0) {
                uint32_t tc = 0;
                for (int w = 0; w < kThreads / 32; ++w) tc += wsum[w];
                A.tile_counts[d.tile] = tc;
            }
            issue(s);
        }
    }

    if (MODE == kModeWrite) return;

    // CTA total -> partials; the last CTA to finish writes the sum.
    const uint64_t ws = warp_sum_u64((uint64_t)my_count);
    if (lane == 0) red[warp] = ws;
    __syncthreads();
    if (tid == 0) {
        uint64_t tot = 0;
        for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
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
            for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
            *A.d_count = tot;
            *A.ticket = 0u;
        }
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

template <int MAXM, int MODE, bool SEVEN>
cudaError_t launch_one(uint32_t grid, size_t smem, cudaStream_t st, const ScanArgs& a, const uint32_t* qc) {
    PatArg<MAXM> p;
    for (uint32_t j = 0; j < a.m; ++j) p.qc[j] = qc[j];
    for (uint32_t j = a.m; j < (uint32_t)MAXM; ++j) p.qc[j] = 0;
    scan_kernel<MAXM, MODE, SEVEN><<<grid, kThreads, smem, st>>>(a, p);
    return cudaGetLastError();
}

template <int MODE, bool SEVEN>
const void* kernel_ptr(uint32_t m) {
    if (m <= (uint32_t)kSmallM) return reinterpret_cast<const void*>(&scan_kernel<kSmallM, MODE, SEVEN>);
    return reinterpret_cast<const void*>(&scan_kernel<kLargeM, MODE, SEVEN>);
}

const void* pick(int mode, bool seven, uint32_t m) {
    switch (mode) {
        case kModeCount: return seven ? kernel_ptr<kModeCount, true>(m) : kernel_ptr<kModeCount, false>(m);
        case kModeTileCount:
            return seven ? kernel_ptr<kModeTileCount, true>(m) : kernel_ptr<kModeTileCount, false>(m);
        default: return seven ? kernel_ptr<kModeWrite, true>(m) : kernel_ptr<kModeWrite, false>(m);
    }
}

}  // namespace

cudaError_t launch_scan(int mode, bool seven, uint32_t grid, size_t smem, cudaStream_t s, const ScanArgs& a,
                        const uint32_t* qc) {
    const bool small = a.m <= (uint32_t)kSmallM;
#define SMK_LAUNCH(MODE)                                                                            \
    if (small) return seven ? launch_one<kSmallM, MODE, true>(grid, smem, s, a, qc)                 \
                            : launch_one<kSmallM, MODE, false>(grid, smem, s, a, qc);              \
    return seven ? launch_one<kLargeM, MODE, true>(grid, smem, s, a, qc)                            \
                 : launch_one<kLargeM, MODE, false>(grid, smem, s, a, qc);
    switch (mode) {
        case kModeCount: SMK_LAUNCH(kModeCount)
        case kModeTileCount: SMK_LAUNCH(kModeTileCount)
        default: SMK_LAUNCH(kModeWrite)
    }
#undef SMK_LAUNCH
}

int scan_occupancy(int mode, bool seven, uint32_t m, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick(mode, seven, m), kThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t scan_prepare(size_t max_smem) {
    for (int mode = 0; mode < 3; ++mode)
        for (int sv = 0; sv < 2; ++sv)
            for (uint32_t m : {1u, (uint32_t)kLargeM}) {
                cudaError_t e = cudaFuncSetAttribute(pick(mode, sv != 0, m),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

cudaError_t launch_hist(uint32_t grid, cudaStream_t s, const HistArgs& a) {
    hist_kernel<<<grid, kHistThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace smk
