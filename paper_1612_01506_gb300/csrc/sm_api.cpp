// Host runtime and C ABI of the GPU string-matching library (include/sm.h).
//
// Validates arguments, owns the per-context device workspace (status word,
// last-CTA ticket, per-CTA partial counts, per-tile counts for reports),
// plans the scan grid, chooses the kernel variant and launches. Everything
// the search computes happens in the kernels of sm_kernels.cu; the host only
// computes the comparison order (Sec. 2.2 / 2.4 of Tarhio, Holub, Giaquinta),
// which the paper also builds on the host before searching.
#include "sm.h"
#include "sm_internal.h"
#include "sm_plan.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

struct sm_ctx {
    int device = 0;
    int num_sms = 0;
    size_t max_smem = 0;
    uint32_t* d_status = nullptr;
    uint32_t* h_status = nullptr;     // pinned mirror for sm_sync
    uint32_t* d_ticket = nullptr;
    unsigned long long* d_tiles = nullptr;   // tile counter of the counting modes
    uint64_t* d_partials = nullptr;
    size_t partials_cap = 0;          // entries
    uint32_t* d_warp_counts = nullptr;
    size_t warp_counts_cap = 0;       // entries
    uint32_t* d_bitmaps = nullptr;    // report: per-(tile, warp) found bitmaps
    size_t bitmaps_cap = 0;           // words
    uint64_t* d_range_sums = nullptr; // rescanning report: matches per range of the write pass
    size_t range_sums_cap = 0;        // entries
    // d_warp_counts and d_range_sums are all zero (the rescanning report
    // leaves them so); false after they were (re)allocated, after a
    // tile-count pass wrote every count word, or after a failed launch
    bool rescan_clean = false;
    uint32_t stages = 4;
    bool stages_fixed = false;        // set by SM_KNOB_STAGES; otherwise fewer stages may raise occupancy
    uint32_t grid_override = 0;
    int write_occ = 1;                // resident blocks per SM of the report's second pass
    uint64_t spin_ns = 1000000000ull;
    uint32_t test_skip_copy = 0;
    std::unordered_map<uint64_t, int> occ;   // (mode, kind, large m, smem) -> resident CTAs per SM
    // autotuned plans per (m bucket, sigma bucket); all-zero = the defaults
    sm_tuning tune[SM_TUNE_M_BUCKETS][SM_TUNE_SIGMA_BUCKETS] = {};
};

namespace {

thread_local std::string g_err;

sm_status fail(sm_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

sm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(SM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool fault_alloc() {
    const char* f = std::getenv("SM_FAULT");
    return f && std::strcmp(f, "alloc") == 0;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
sm_status grow(T** p, size_t* cap, size_t want, const char* what) {
    if (*cap >= want) return SM_OK;
    size_t n = std::max<size_t>(want, *cap * 2);
    if (fault_alloc()) return fail(SM_ENOMEM, "injected allocation failure (%s)", what);
    if (*p) {
        cudaFree(*p);   // synchronizes with the device: no launch still uses it
        *p = nullptr;
        *cap = 0;
    }
    if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SM_ENOMEM, "cudaMalloc of %zu bytes for %s failed", n * sizeof(T), what);
    }
    *cap = n;
    return SM_OK;
}

sm_status check_pattern(const uint8_t* h_pat, uint32_t m, const uint32_t* h_pi) {
    if (m == 0) return fail(SM_EINVAL, "pattern length m must be at least 1");
    if (m > SM_MAX_M) return fail(SM_EINVAL, "pattern length %u exceeds SM_MAX_M (%u)", m, SM_MAX_M);
    if (!h_pat) return fail(SM_EINVAL, "h_pat is NULL");
    if (h_pi) {
        std::vector<uint8_t> seen(m, 0);
        for (uint32_t j = 0; j < m; ++j) {
            if (h_pi[j] >= m || seen[h_pi[j]]) return fail(SM_EINVAL, "h_pi is not a permutation of 0..m-1");
            seen[h_pi[j]] = 1;
        }
    }
    return SM_OK;
}

// Autotuning buckets (include/sm.h): ceil(log2 m), and the text's alphabet.
uint32_t m_bucket_of(uint32_t m) {
    uint32_t b = 0;
    while ((1u << b) < m) ++b;
    return b;
}

uint32_t sigma_bucket_of(const uint64_t* h) {
    uint64_t n = 0;
    uint32_t distinct = 0;
    for (int c = 0; c < 256; ++c) {
        n += h[c];
        distinct += h[c] ? 1u : 0u;
    }
    if (distinct <= 2) return 0;
    if (distinct <= 4) return 1;
    double s2 = 0;
    for (int c = 0; c < 256; ++c) {
        const double p = (double)h[c] / (double)n;
        s2 += p * p;
    }
    const double eff = 1.0 / s2;
    return eff < 12.0 ? 2u : eff < 48.0 ? 3u : 4u;
}

// A non-negative integer from the environment, or -1.
long env_uint(const char* name) {
    const char* v = std::getenv(name);
    if (!v || !*v) return -1;
    char* end = nullptr;
    const long x = std::strtol(v, &end, 10);
    return (end && *end == 0 && x >= 0) ? x : -1;
}

struct Plan {
    std::vector<uint32_t> qc;       // compare descriptors in scan order (plan_dense / plan_packed)
    std::vector<uint32_t> groups;   // window groups of the peeled compares
    uint32_t r = 1;
    int kind = smk::kKindBytes;
    uint32_t b1 = 0, b2 = 0;        // packed kinds: the code bits
    bool zero = false;   // a pattern symbol never occurs in the text
    double expect = -1;  // expected matches per start from the symbol frequencies (-1: unknown)
    bool skewed = false; // effective alphabet below half the distinct symbols (e.g. natural language)
};

// Compare descriptors (e << 8) | p[q], e = (text address mod 16) + q, in the
// order pi; the text's symbol frequencies (when the caller passes its
// histogram) pick the peeled compares and the compare kind: 1-bit codes for
// texts of at most two symbols, 2-bit codes for at most four, the 7-bit test
// for texts without bytes >= 0x80, else the general byte test.
sm_status make_plan(const uint8_t* d_text, const uint8_t* p, uint32_t m, const uint32_t* pi,
                    const sm_search_opts* o, uint64_t n, Plan* pl) {
    if (o && (o->flags & ~SM_SEARCH_BYTES)) return fail(SM_EINVAL, "unknown search flags");
    const uint32_t delta = (uint32_t)(reinterpret_cast<uintptr_t>(d_text) & 15u);
    std::vector<uint32_t> v(m);
    for (uint32_t j = 0; j < m; ++j) {
        const uint32_t q = pi ? pi[j] : j;
        v[j] = ((q + delta) << 8) | p[q];
    }
    const uint64_t* h = o ? o->h_hist256 : nullptr;
    std::vector<double> freq;
    bool packed = false, binary = false;
    if (h) {
        uint64_t high = 0;
        for (int c = 0x80; c < 256; ++c) high += h[c];
        bool pat7 = true;
        for (uint32_t q = 0; q < m; ++q) {
            if (p[q] >= 0x80) pat7 = false;
            if (h[p[q]] == 0) pl->zero = true;
        }
        pl->kind = (high == 0) && pat7 ? smk::kKindSeven : smk::kKindBytes;
        freq.resize(m);
        double lp = 0;
        for (uint32_t j = 0; j < m; ++j) {
            freq[j] = n ? (double)h[v[j] & 0xFFu] / (double)n : 1.0;
            lp += std::log(std::max(freq[j], 1e-300));
        }
        pl->expect = std::exp(std::max(lp, -700.0));
        uint64_t tot = 0;
        uint32_t distinct = 0;
        for (int c = 0; c < 256; ++c) {
            tot += h[c];
            distinct += h[c] ? 1u : 0u;
        }
        double s2 = 0;
        for (int c = 0; c < 256; ++c)
            if (h[c]) s2 += ((double)h[c] / (double)tot) * ((double)h[c] / (double)tot);
        pl->skewed = s2 > 0 && 1.0 / s2 < 0.5 * (double)distinct;
        const bool codes = !pl->zero && !(o->flags & SM_SEARCH_BYTES);
        binary = codes && smk::binary_code_bit(h, &pl->b1);
        packed = codes && !binary && smk::packed_code_bits(h, &pl->b1, &pl->b2);
    }
    pl->qc.resize(m);
    uint32_t ng = 0;
    if (binary || packed) {
        // every pattern symbol occurs in the text, so its code is defined
        for (uint32_t j = 0; j < m; ++j) {
            const uint32_t c = v[j] & 0xFFu;
            v[j] = (v[j] & ~0xFFu) | ((c >> pl->b1) & 1u) | (binary ? 0u : ((c >> pl->b2) & 1u) << 1);
        }
        pl->kind = binary ? smk::kKindBinary : pl->b2 == pl->b1 + 1 ? smk::kKindPackedAdj : smk::kKindPacked;
        pl->groups.resize(smk::max_packed_groups_for(m));
        pl->r = smk::plan_packed(v.data(), m, freq.data(), o->peel, pl->qc.data(), pl->groups.data(),
                                 (uint32_t)pl->groups.size(), &ng, binary ? 1u : 2u);
    } else {
        pl->groups.resize(smk::max_groups_for(m));
        pl->r = smk::plan_dense(v.data(), m, h ? freq.data() : nullptr, o ? o->peel : 0u, pl->qc.data(),
                                pl->groups.data(), (uint32_t)pl->groups.size(), &ng);
    }
    if (pl->r == 0) return fail(SM_EINVAL, "internal: dense plan exceeds its group capacity");
    pl->groups.resize(ng);
    return SM_OK;
}

// Which report to run: the rescan (count, then the tiles with matches again)
// when the symbol frequencies expect matches in at most one tile in 32 (each
// such tile is read and compared twice, and the CTA with the most of them
// sets the second pass's length), else the found-bits passes. On a text with
// skewed frequencies the product of the symbol frequencies underestimates
// the matches of a pattern taken from it (neighbouring symbols correlate:
// a Markov-95 text gave 45,723 matches of an m = 4 pattern where the
// frequencies expected a few hundred, and the rescan read the text twice),
// so there the estimate is taken 100 times larger. SM_REPORT=rescan or
// SM_REPORT=bits forces one of them.
bool report_rescans(const Plan& pl, uint64_t nstarts, uint64_t ntiles) {
    const char* f = std::getenv("SM_REPORT");
    if (f && std::strcmp(f, "rescan") == 0) return true;
    if (f && std::strcmp(f, "bits") == 0) return false;
    if (pl.expect < 0) return false;
    const double matches = pl.expect * (double)nstarts * (pl.skewed ? 100.0 : 1.0);
    // tiles with at least one match, matches spread at random
    const double tiles = (double)ntiles * -std::expm1(-matches / (double)ntiles);
    return tiles * 32.0 <= (double)ntiles;
}

struct Grid {
    uint32_t grid = 0, stage_bytes = 0, stages = 0;
    uint64_t ntiles = 0, per_cta = 0;
    size_t smem = 0;
};

int occupancy(sm_ctx* c, int mode, int kind, uint32_t m, size_t smem) {
    const uint64_t key = ((uint64_t)smem << 8) | ((uint64_t)mode << 4) | ((uint64_t)kind << 1) |
                         (m > (uint32_t)smk::kSmallM ? 1u : 0u);
    auto it = c->occ.find(key);
    if (it != c->occ.end()) return it->second;
    const int o = smk::scan_occupancy(mode, kind, m, smem);
    c->occ.emplace(key, o);
    return o;
}

sm_status plan_grid(sm_ctx* c, int mode, int kind, bool report, uint32_t m, uint64_t nstarts, Grid* g,
                    const sm_tuning* t = nullptr) {
    g->ntiles = (nstarts + smk::kTile - 1) / smk::kTile;
    g->stage_bytes = smk::stage_bytes_for(m);
    const bool tuned_stages = t && t->stages >= 2;
    g->stages = tuned_stages ? std::min<uint32_t>(t->stages, smk::kMaxStages) : c->stages;
    while (g->stages > 2 && smk::scan_smem_bytes(g->stage_bytes, g->stages, kind, report) > c->max_smem) --g->stages;
    g->smem = smk::scan_smem_bytes(g->stage_bytes, g->stages, kind, report);
    if (g->smem > c->max_smem) return fail(SM_ENOTSUP, "pattern too long for shared memory");
    int occ = occupancy(c, mode, kind, m, g->smem);
    if (occ <= 0) return fail(SM_ECUDA, "scan kernel cannot be resident (smem %zu)", g->smem);
    // one stage fewer is worth it when it lets another CTA reside on each SM
    while (!c->stages_fixed && !tuned_stages && g->stages > 2) {
        const size_t sm2 = smk::scan_smem_bytes(g->stage_bytes, g->stages - 1, kind, report);
        const int o2 = occupancy(c, mode, kind, m, sm2);
        if (o2 <= occ) break;
        --g->stages;
        g->smem = sm2;
        occ = o2;
    }
    uint64_t want = c->grid_override;
    if (!want) want = (uint64_t)c->num_sms * (uint64_t)(t && t->ctas_per_sm ? std::min<int>(occ, (int)t->ctas_per_sm)
                                                                             : occ);
    want = std::max<uint64_t>(1, std::min<uint64_t>(want, g->ntiles));
    g->per_cta = (g->ntiles + want - 1) / want;
    g->grid = (uint32_t)((g->ntiles + g->per_cta - 1) / g->per_cta);
    return grow(&c->d_partials, &c->partials_cap, std::max<size_t>(g->grid, 256), "partials");
}

smk::ScanArgs scan_args(sm_ctx* c, const uint8_t* d_text, uint64_t n, uint32_t m, const Plan& pl, const Grid& g,
                        uint64_t* d_count) {
    smk::ScanArgs a{};
    a.text = d_text;
    a.n = n;
    a.nstarts = n - m + 1;
    a.ntiles = g.ntiles;
    a.tiles_per_cta = g.per_cta;
    a.m = m;
    a.r = pl.r;
    a.ng = (uint32_t)pl.groups.size();
    a.b1 = pl.b1;
    a.b2 = pl.b2;
    a.gather = 0x01041040u;
    a.packed_words = smk::packed_words_for(g.stage_bytes, pl.kind);
    a.stage_bytes = g.stage_bytes;
    a.stages = g.stages;
    a.status = c->d_status;
    a.partials = c->d_partials;
    a.ticket = c->d_ticket;
    a.tile_next = c->d_tiles;
    a.d_count = d_count;
    a.warp_counts = c->d_warp_counts;
    a.one = 1;
    a.spin_ns = c->spin_ns;
    a.test_skip_copy = c->test_skip_copy;
    return a;
}

sm_status zero_count(uint64_t* d_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s);
    return e == cudaSuccess ? SM_OK : cuda_fail(e, "cudaMemsetAsync");
}

}  // namespace

// Accessors for the other translation units of the library.
sm_status sm_fail_internal(sm_status s, const char* msg) { return fail(s, "%s", msg); }
int sm_ctx_device(const sm_ctx* c) { return c->device; }
int sm_ctx_num_sms(const sm_ctx* c) { return c->num_sms; }
size_t sm_ctx_max_smem(const sm_ctx* c) { return c->max_smem; }
uint32_t* sm_ctx_status(const sm_ctx* c) { return c->d_status; }
uint64_t sm_ctx_spin_ns(const sm_ctx* c) { return c->spin_ns; }
uint32_t sm_ctx_stages(const sm_ctx* c) { return c->stages; }

extern "C" {

const char* sm_last_error(void) { return g_err.c_str(); }

const char* sm_status_string(sm_status s) {
    switch (s) {
        case SM_OK: return "SM_OK";
        case SM_EINVAL: return "SM_EINVAL";
        case SM_ENOMEM: return "SM_ENOMEM";
        case SM_ECUDA: return "SM_ECUDA";
        case SM_ETRUNC: return "SM_ETRUNC";
        case SM_ETIMEOUT: return "SM_ETIMEOUT";
        case SM_ENOTSUP: return "SM_ENOTSUP";
    }
    return "unknown";
}

sm_status sm_create(sm_ctx** out, int device) {
    if (!out) return fail(SM_EINVAL, "ctx pointer is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(SM_EINVAL, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard g(device);
    if (!g.ok) return fail(SM_ECUDA, "cudaSetDevice(%d) failed", device);
    if (fault_alloc()) return fail(SM_ENOMEM, "injected allocation failure (context)");
    const long tile = env_uint("SM_TILE"), starts = env_uint("SM_STARTS");
    if (tile >= 0 && tile != (long)smk::kTile)
        return fail(SM_ENOTSUP, "SM_TILE=%ld: the tile is fixed at %u starts by the warp geometry", tile, smk::kTile);
    if (starts >= 0 && starts != 16 * smk::kChunks)
        return fail(SM_ENOTSUP, "SM_STARTS=%ld: each thread takes %d starts (fixed by the warp geometry)", starts,
                    16 * smk::kChunks);
    sm_ctx* c = new sm_ctx();
    c->device = device;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    c->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->max_smem = (size_t)v;
    if ((e = cudaMalloc(&c->d_status, 64)) != cudaSuccess || (e = cudaMemset(c->d_status, 0, 64)) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_status, 64)) != cudaSuccess) {
        sm_destroy(c);
        return cuda_fail(e, "context allocation");
    }
    c->d_ticket = c->d_status + 8;   // second 32-byte sector of the same allocation
    c->d_tiles = reinterpret_cast<unsigned long long*>(c->d_status + 12);
    if ((e = smk::scan_prepare(c->max_smem)) != cudaSuccess) {
        sm_destroy(c);
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    c->write_occ = std::max(1, smk::bitmap_write_occupancy());
    sm_status st = grow(&c->d_partials, &c->partials_cap, (size_t)c->num_sms * 16 * 256, "partials");
    if (st != SM_OK) {
        sm_destroy(c);
        return st;
    }
    *out = c;
    return SM_OK;
}

void sm_destroy(sm_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    if (c->d_status) cudaFree(c->d_status);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_warp_counts) cudaFree(c->d_warp_counts);
    if (c->d_bitmaps) cudaFree(c->d_bitmaps);
    if (c->d_range_sums) cudaFree(c->d_range_sums);
    delete c;
}

sm_status sm_set_knob(sm_ctx* c, sm_knob knob, int64_t value) {
    if (!c) return fail(SM_EINVAL, "ctx is NULL");
    switch (knob) {
        case SM_KNOB_STAGES:
            if (value < 2 || value > smk::kMaxStages) return fail(SM_EINVAL, "stages must be 2..%d", smk::kMaxStages);
            c->stages = (uint32_t)value;
            c->stages_fixed = true;
            return SM_OK;
        case SM_KNOB_GRID:
            if (value < 0 || value > (1 << 24)) return fail(SM_EINVAL, "grid out of range");
            c->grid_override = (uint32_t)value;
            return SM_OK;
        case SM_KNOB_SPIN_NS:
            if (value < 1000) return fail(SM_EINVAL, "spin limit below 1 us");
            c->spin_ns = (uint64_t)value;
            return SM_OK;
        case SM_KNOB_TEST_SKIP_COPY:
            c->test_skip_copy = value ? 1u : 0u;
            return SM_OK;
    }
    return fail(SM_EINVAL, "unknown knob %d", (int)knob);
}

sm_status sm_sync(sm_ctx* c, sm_stream_t stream) {
    if (!c) return fail(SM_EINVAL, "ctx is NULL");
    DeviceGuard g(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sm_sync");
    const uint32_t bits = *c->h_status;
    if (bits & smk::kStatusTimeout) return fail(SM_ETIMEOUT, "a bounded device wait expired");
    if (bits & smk::kStatusTrunc) return fail(SM_ETRUNC, "a report had more matches than its capacity");
    return SM_OK;
}

sm_status sm_histogram(sm_ctx* c, const uint8_t* d_text, uint64_t n, uint64_t* d_hist256, sm_stream_t stream) {
    if (!c) return fail(SM_EINVAL, "ctx is NULL");
    if (!d_hist256) return fail(SM_EINVAL, "d_hist256 is NULL");
    if (!d_text && n) return fail(SM_EINVAL, "d_text is NULL");
    DeviceGuard g(c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(d_hist256, 0, 256 * sizeof(uint64_t), s);
        return e == cudaSuccess ? SM_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    const uint64_t per_block = (uint64_t)smk::kHistThreads * 16 * 8;
    uint64_t grid = std::min<uint64_t>((uint64_t)c->num_sms * 4, (n + per_block - 1) / per_block);
    grid = std::max<uint64_t>(grid, 1);
    sm_status st = grow(&c->d_partials, &c->partials_cap, grid * 256, "partials");
    if (st != SM_OK) return st;
    smk::HistArgs a{d_text, n, c->d_partials, c->d_ticket, d_hist256};
    cudaError_t e = smk::launch_hist((uint32_t)grid, s, a);
    return e == cudaSuccess ? SM_OK : cuda_fail(e, "histogram launch");
}

sm_status sm_order(const uint8_t* h_pat, uint32_t m, const uint64_t* h_hist256, uint32_t* h_pi) {
    if (m == 0) return fail(SM_EINVAL, "pattern length m must be at least 1");
    if (!h_pat || !h_hist256 || !h_pi) return fail(SM_EINVAL, "NULL argument");
    std::vector<uint32_t> idx(m);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](uint32_t a, uint32_t b) { return h_hist256[h_pat[a]] < h_hist256[h_pat[b]]; });
    std::copy(idx.begin(), idx.end(), h_pi);
    return SM_OK;
}

sm_status sm_order_fixed(const uint8_t* h_pat, uint32_t m, int mode, uint32_t* h_pi) {
    if (m == 0) return fail(SM_EINVAL, "pattern length m must be at least 1");
    if (!h_pi) return fail(SM_EINVAL, "h_pi is NULL");
    if (mode != SM_ORDER_H && mode != SM_ORDER_HS) return fail(SM_EINVAL, "unknown order mode %d", mode);
    if (mode == SM_ORDER_HS && !h_pat) return fail(SM_EINVAL, "h_pat is NULL");
    std::vector<uint32_t> keep, spaces;
    for (uint32_t q = 0; q < m; ++q) {
        if (mode == SM_ORDER_HS && h_pat[q] == 0x20) spaces.push_back(q);
        else keep.push_back(q);
    }
    // pi_h over `keep`: first, last, then indices 3,6,.. / 2,5,.. / 1,4,.. below the last
    std::vector<uint32_t> out;
    out.reserve(m);
    const size_t L = keep.size();
    if (L) {
        out.push_back(keep[0]);
        if (L > 1) out.push_back(keep[L - 1]);
        for (size_t first : {size_t(3), size_t(2), size_t(1)})
            for (size_t k = first; k + 1 < L; k += 3) out.push_back(keep[k]);
    }
    out.insert(out.end(), spaces.begin(), spaces.end());
    std::copy(out.begin(), out.end(), h_pi);
    return SM_OK;
}

static sm_status search(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                        const uint32_t* h_pi, const sm_search_opts* opts, uint64_t* d_pos, uint64_t cap,
                        uint64_t* d_count, sm_stream_t stream, bool report) {
    if (!c) return fail(SM_EINVAL, "ctx is NULL");
    if (!d_count) return fail(SM_EINVAL, "d_count is NULL");
    if (!d_text && n) return fail(SM_EINVAL, "d_text is NULL");
    if (report && cap && !d_pos) return fail(SM_EINVAL, "d_pos is NULL with cap > 0");
    sm_status st = check_pattern(h_pat, m, h_pi);
    if (st != SM_OK) return st;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SM_ECUDA, "cudaSetDevice(%d) failed", c->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((uint64_t)m > n) return zero_count(d_count, s);
    // the autotuned plan of the search's bucket (needs the text histogram),
    // then the environment's overrides; an explicit peel or knob wins
    sm_tuning tu{};
    if (opts && opts->h_hist256) tu = c->tune[m_bucket_of(m)][sigma_bucket_of(opts->h_hist256)];
    if (env_uint("SM_R") > 0) tu.peel = (uint32_t)env_uint("SM_R");
    if (env_uint("SM_STAGES") >= 2) tu.stages = (uint32_t)env_uint("SM_STAGES");
    if (env_uint("SM_CTAS_PER_SM") > 0) tu.ctas_per_sm = (uint32_t)env_uint("SM_CTAS_PER_SM");
    if (c->stages_fixed) tu.stages = 0;
    sm_search_opts o2{};
    if (tu.peel && !(opts && opts->peel)) {
        if (opts) o2 = *opts;
        o2.peel = tu.peel;
        opts = &o2;
    }
    Plan pl;
    st = make_plan(d_text, h_pat, m, h_pi, opts, n, &pl);
    if (st != SM_OK) return st;
    if (pl.zero) return zero_count(d_count, s);

    const uint64_t nstarts = n - m + 1;
    const uint64_t ntiles = (nstarts + smk::kTile - 1) / smk::kTile;
    const bool rescan = report && report_rescans(pl, nstarts, ntiles);
    const int mode1 = !report ? smk::kModeCount : rescan ? smk::kModeSparse : smk::kModeTileCount;
    Grid gr;
    st = plan_grid(c, mode1, pl.kind, report && !rescan, m, nstarts, &gr, &tu);
    if (st != SM_OK) return st;
    // ranges of the report's second pass: one resident wave of its blocks
    const uint64_t wranges = std::max<uint64_t>(
        1, std::min<uint64_t>(gr.ntiles, (uint64_t)c->write_occ * (uint64_t)c->num_sms));
    if (report) {
        st = grow(&c->d_partials, &c->partials_cap,
                  std::max<size_t>((size_t)std::max<uint64_t>(wranges, gr.grid), 256), "partials");
        if (st != SM_OK) return st;
        const size_t cap_before = c->warp_counts_cap;
        st = grow(&c->d_warp_counts, &c->warp_counts_cap, (size_t)gr.ntiles * smk::kConsumerWarps,
                  "per-warp tile counts");
        if (c->warp_counts_cap != cap_before) c->rescan_clean = false;
        if (st != SM_OK) return st;
        if (!rescan) {
            st = grow(&c->d_bitmaps, &c->bitmaps_cap, (size_t)gr.ntiles * smk::kConsumerWarps * smk::kBitmapWords,
                      "found bitmaps");
            if (st != SM_OK) return st;
        }
    }
    smk::ScanArgs a = scan_args(c, d_text, n, m, pl, gr, d_count);
    cudaError_t e;
    if (rescan) {
        // few tiles hold matches: count, noting the warp-tiles with matches
        // and the matches per range of the write pass, then scan those tiles
        // again and write their positions. Ranges of at most kWriteList
        // tiles (the write pass lists a range's tiles in shared memory).
        const uint64_t per_w = std::min<uint64_t>(gr.per_cta, smk::kWriteList);
        const uint64_t nranges = (gr.ntiles + per_w - 1) / per_w;
        const size_t rs_before = c->range_sums_cap;
        st = grow(&c->d_range_sums, &c->range_sums_cap, (size_t)std::max<uint64_t>(nranges, 256), "range sums");
        if (c->range_sums_cap != rs_before) c->rescan_clean = false;
        if (st != SM_OK) return st;
        // the write pass: its stages and the list, with one stage fewer as
        // long as that keeps as many CTAs resident per SM as the first pass
        auto wsmem_for = [&](uint32_t nst) {
            return smk::scan_smem_bytes(gr.stage_bytes, nst, pl.kind) + smk::kWriteListBytes;
        };
        uint32_t wstages = gr.stages;
        while (wstages > 2 && wsmem_for(wstages) > c->max_smem) --wstages;
        const int occ1 = occupancy(c, mode1, pl.kind, m, gr.smem);
        while (wstages > 2 && occupancy(c, smk::kModeWrite, pl.kind, m, wsmem_for(wstages)) < occ1) --wstages;
        const size_t wsmem = wsmem_for(wstages);
        if (wsmem > c->max_smem) return fail(SM_ENOTSUP, "pattern too long for shared memory");
        if (!c->rescan_clean) {
            e = cudaMemsetAsync(c->d_warp_counts, 0, c->warp_counts_cap * sizeof(uint32_t), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_range_sums, 0, c->range_sums_cap * sizeof(uint64_t), s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        }
        c->rescan_clean = false;   // until both launches went in
        a.range_sums = c->d_range_sums;
        a.range_tiles = per_w;
        e = smk::launch_scan(mode1, pl.kind, gr.grid, gr.smem, s, a, pl.qc.data(), pl.groups.data());
        if (e != cudaSuccess) return cuda_fail(e, "scan launch");
        a.d_pos = d_pos;
        a.cap = cap;
        a.tiles_per_cta = per_w;
        a.stages = wstages;
        e = smk::launch_scan(smk::kModeWrite, pl.kind, (uint32_t)nranges, wsmem, s, a, pl.qc.data(),
                             pl.groups.data());
        if (e != cudaSuccess) return cuda_fail(e, "report launch");
        c->rescan_clean = true;
        return SM_OK;
    }
    // the tile-count pass writes every count word of its tiles
    if (report) c->rescan_clean = false;
    // a report with matches in many tiles: the tile-count pass (per-warp-tile
    // counts and found bits), the per-range counts, then the positions from
    // the found bits
    if (report) a.bitmaps = c->d_bitmaps;
    e = smk::launch_scan(mode1, pl.kind, gr.grid, gr.smem, s, a, pl.qc.data(), pl.groups.data());
    if (e != cudaSuccess) return cuda_fail(e, "scan launch");
    if (report) {
        // the write pass: one range of tiles per block, one resident wave
        const uint64_t per = (gr.ntiles + wranges - 1) / wranges;
        const uint32_t wgrid = (uint32_t)((gr.ntiles + per - 1) / per);
        e = smk::launch_range_sums(wgrid, s, c->d_warp_counts, gr.ntiles, per, c->d_partials);
        if (e != cudaSuccess) return cuda_fail(e, "range count launch");
        smk::WriteArgs w{};
        w.ntiles = gr.ntiles;
        w.tiles_per_cta = per;
        w.partials = c->d_partials;
        w.warp_counts = c->d_warp_counts;
        w.bitmaps = c->d_bitmaps;
        w.d_pos = d_pos;
        w.cap = cap;
        w.status = c->d_status;
        w.folded = smk::kind_packed(pl.kind) ? 0u : 1u;
        e = smk::launch_bitmap_write(wgrid, s, w);
        if (e != cudaSuccess) return cuda_fail(e, "report launch");
    }
    return SM_OK;
}

sm_status sm_count(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                   const uint32_t* h_pi, uint64_t* d_count, sm_stream_t stream) {
    return search(c, d_text, n, h_pat, m, h_pi, nullptr, nullptr, 0, d_count, stream, false);
}

sm_status sm_count_ex(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                      const uint32_t* h_pi, const sm_search_opts* opts, uint64_t* d_count, sm_stream_t stream) {
    return search(c, d_text, n, h_pat, m, h_pi, opts, nullptr, 0, d_count, stream, false);
}

sm_status sm_report(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                    const uint32_t* h_pi, uint64_t* d_pos, uint64_t cap, uint64_t* d_count, sm_stream_t stream) {
    return search(c, d_text, n, h_pat, m, h_pi, nullptr, d_pos, cap, d_count, stream, true);
}

sm_status sm_report_ex(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                       const uint32_t* h_pi, const sm_search_opts* opts, uint64_t* d_pos, uint64_t cap,
                       uint64_t* d_count, sm_stream_t stream) {
    return search(c, d_text, n, h_pat, m, h_pi, opts, d_pos, cap, d_count, stream, true);
}

sm_status sm_tune_bucket(const uint64_t* h_hist256, uint32_t m, uint32_t* m_bucket, uint32_t* sigma_bucket) {
    if (!h_hist256 || !m_bucket || !sigma_bucket) return fail(SM_EINVAL, "NULL argument");
    if (m == 0 || m > SM_MAX_M) return fail(SM_EINVAL, "pattern length %u out of range", m);
    *m_bucket = m_bucket_of(m);
    *sigma_bucket = sigma_bucket_of(h_hist256);
    return SM_OK;
}

sm_status sm_tune_set(sm_ctx* c, uint32_t m_bucket, uint32_t sigma_bucket, const sm_tuning* plan) {
    if (!c) return fail(SM_EINVAL, "ctx is NULL");
    if (m_bucket >= SM_TUNE_M_BUCKETS || sigma_bucket >= SM_TUNE_SIGMA_BUCKETS)
        return fail(SM_EINVAL, "bucket (%u, %u) out of range", m_bucket, sigma_bucket);
    if (plan && (plan->peel > SM_MAX_M || (plan->stages && (plan->stages < 2 || plan->stages > smk::kMaxStages)) ||
                 plan->ctas_per_sm > 64))
        return fail(SM_EINVAL, "plan out of range");
    c->tune[m_bucket][sigma_bucket] = plan ? *plan : sm_tuning{};
    return SM_OK;
}

sm_status sm_tune_get(sm_ctx* c, uint32_t m_bucket, uint32_t sigma_bucket, sm_tuning* plan) {
    if (!c || !plan) return fail(SM_EINVAL, "NULL argument");
    if (m_bucket >= SM_TUNE_M_BUCKETS || sigma_bucket >= SM_TUNE_SIGMA_BUCKETS)
        return fail(SM_EINVAL, "bucket (%u, %u) out of range", m_bucket, sigma_bucket);
    *plan = c->tune[m_bucket][sigma_bucket];
    return SM_OK;
}

sm_status sm_tune_search(sm_ctx* c, const uint8_t* d_text, uint64_t n, const uint64_t* h_hist256,
                         const uint8_t* h_pats, const int64_t* h_pat_off, uint32_t npats, uint32_t reps,
                         sm_tuning* best, sm_stream_t stream) {
    if (!c || !d_text || !h_hist256 || !h_pats || !h_pat_off || !best || npats == 0)
        return fail(SM_EINVAL, "NULL argument or no patterns");
    if (reps < 1) reps = 1;
    uint32_t mb = 0;
    for (uint32_t k = 0; k < npats; ++k) {
        const int64_t m = h_pat_off[k + 1] - h_pat_off[k];
        if (m < 1 || m > (int64_t)SM_MAX_M || (uint64_t)m > n) return fail(SM_EINVAL, "pattern %u length", k);
        if (k == 0) mb = m_bucket_of((uint32_t)m);
        if (m_bucket_of((uint32_t)m) != mb) return fail(SM_EINVAL, "patterns of different m buckets");
    }
    const uint32_t sb = sigma_bucket_of(h_hist256);
    DeviceGuard g(c->device);
    if (!g.ok) return fail(SM_ECUDA, "cudaSetDevice(%d) failed", c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<std::vector<uint32_t>> pis(npats);
    for (uint32_t k = 0; k < npats; ++k) {
        const uint32_t m = (uint32_t)(h_pat_off[k + 1] - h_pat_off[k]);
        pis[k].resize(m);
        sm_order(h_pats + h_pat_off[k], m, h_hist256, pis[k].data());
    }
    uint64_t* d_count = nullptr;
    if (cudaMalloc(&d_count, sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SM_ENOMEM, "tuning count word");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const sm_search_opts o{0u, 0u, h_hist256};
    // the patterns in two halves [0, half) and [half, npats): a candidate
    // must win on both (with one pattern, the one half is all of them)
    const uint32_t half = npats >= 2 ? npats / 2 : npats;
    auto pass = [&](uint32_t k0, uint32_t k1) -> sm_status {
        for (uint32_t k = k0; k < k1; ++k) {
            const sm_status s = sm_count_ex(c, d_text, n, h_pats + h_pat_off[k],
                                            (uint32_t)(h_pat_off[k + 1] - h_pat_off[k]), pis[k].data(), &o,
                                            d_count, stream);
            if (s != SM_OK) return s;
        }
        return SM_OK;
    };
    // mean ms per search of a plan on each half: a warm-up pass, then the
    // fastest of reps timed passes
    auto time_half = [&](uint32_t k0, uint32_t k1, float* ms) -> sm_status {
        sm_status s = SM_OK;
        float bestp = 1e30f;
        for (uint32_t r = 0; s == SM_OK && r < reps; ++r) {
            float x = 0;
            if (cudaEventRecord(e0, st) != cudaSuccess) s = fail(SM_ECUDA, "tuning timer");
            if (s == SM_OK) s = pass(k0, k1);
            if (s == SM_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&x, e0, e1) != cudaSuccess))
                s = fail(SM_ECUDA, "tuning timer");
            bestp = std::min(bestp, x);
        }
        *ms = bestp / (float)std::max<uint32_t>(1, k1 - k0);
        return s;
    };
    auto time_plan = [&](const sm_tuning& t, float (&ms)[2]) -> sm_status {
        c->tune[mb][sb] = t;
        sm_status s = pass(0, npats);
        if (s == SM_OK) s = time_half(0, half, &ms[0]);
        ms[1] = ms[0];
        if (s == SM_OK && half < npats) s = time_half(half, npats, &ms[1]);
        return s;
    };
    auto same = [](const sm_tuning& a, const sm_tuning& b) {
        return a.peel == b.peel && a.stages == b.stages && a.ctas_per_sm == b.ctas_per_sm;
    };
    sm_tuning cur = c->tune[mb][sb];
    cur.ms = 0;
    const sm_tuning start = cur;
    float cur_ms[2] = {0, 0};
    sm_status s = time_plan(cur, cur_ms);
    auto consider = [&](sm_tuning cand) {
        if (s != SM_OK || same(cand, cur)) return;
        float ms[2] = {0, 0};
        s = time_plan(cand, ms);
        if (s == SM_OK && ms[0] < 0.98f * cur_ms[0] && ms[1] < 0.98f * cur_ms[1]) {
            cur = cand;
            cur_ms[0] = ms[0];
            cur_ms[1] = ms[1];
        }
    };
    for (uint32_t r : {0u, 1u, 2u, 3u, 4u, 5u, 6u, 7u, 8u}) {
        sm_tuning t = cur;
        t.peel = r;
        consider(t);
    }
    for (uint32_t stg : {0u, 2u, 3u, 4u, 6u}) {
        sm_tuning t = cur;
        t.stages = stg;
        consider(t);
    }
    for (uint32_t k : {0u, 1u, 2u, 3u}) {
        sm_tuning t = cur;
        t.ctas_per_sm = k;
        consider(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_count);
    c->tune[mb][sb] = s == SM_OK ? cur : start;
    if (s != SM_OK) return s;
    cur.ms = (cur_ms[0] * (float)half + cur_ms[1] * (float)(npats - half)) /
             (float)(half < npats ? npats : half);
    c->tune[mb][sb].ms = cur.ms;
    *best = cur;
    return SM_OK;
}

}  // extern "C"
