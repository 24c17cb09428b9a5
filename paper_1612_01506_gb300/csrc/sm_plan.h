// Host planning of the dense phase of the scan (loop peeling, Sec. 2.3 of
// Tarhio, Holub, Giaquinta), shared by the single-pattern and batched
// launches. Internal to the library; uses no heap memory.
//
// A compare descriptor is (e << 8) | symbol, where e = (text address mod 16)
// + pattern position is the byte offset of the compare's 4-byte window from
// the first start of a 16-start chunk. A consumer lane reads that window
// from the 16-byte units E = e >> 4 and E + 1 of each of its chunks. The
// dense phase loads those two units once per group of peeled compares that
// share E, and a compare whose window is 4-byte aligned (e mod 4 == 0) needs
// no funnel shift, so it costs half the integer instructions of the others.
//
// Which compares to peel: Sec. 2.3 peels the first r compares of the order
// pi and leaves r to tuning. With the text's symbol frequencies the planner
// also builds a second order that takes, step by step, the compare with the
// most selectivity (-log frequency) per modelled cost (aligned or not, in a
// window already loaded or not), and peels the prefix of either order with
// the lowest modelled cost. The count does not depend on which compares are
// peeled or on their order: every start is still tested at every pattern
// position until its found bit is zero.
#pragma once

#include <cmath>
#include <cstdint>

namespace smk {

// Group descriptor: window unit E in bits 0-8; bit 9 + D set when the group
// has the aligned compare of word class D = (e >> 2) & 3 (e = 16E + 4D);
// bits 13 + 2D .. 14 + 2D the number (0..3) of its other compares of class D.
constexpr uint32_t kPlanMaxPeel = 16;   // largest r the cost model chooses
constexpr uint32_t kPlanCandidates = 64;
constexpr uint32_t kPlanMaxM = 4096;    // longest pattern planned (the library's SM_MAX_M)
constexpr uint32_t kPlanWindows = 4;    // windows whose aligned compares join the greedy's pool

// A set of compare indices below kPlanMaxM (positions in the order pi).
struct PlanSet {
    uint64_t w[kPlanMaxM / 64] = {};
    bool has(uint32_t j) const { return (w[j >> 6] >> (j & 63u)) & 1u; }
    void add(uint32_t j) { w[j >> 6] |= 1ull << (j & 63u); }
};

// Window groups a pattern of length m can have: e < 16 + m, so E <= (14 + m) / 16.
constexpr uint32_t max_groups_for(uint32_t m) { return (14 + m) / 16 + 1; }

inline uint32_t group_e(uint32_t v) { return v >> 12; }
inline uint32_t word_class(uint32_t v) { return (v >> 10) & 3u; }
inline bool aligned(uint32_t v) { return ((v >> 8) & 3u) == 0; }

// Modelled time of one 2048-start warp-tile, in consumer-warp cycles measured
// per phase on GB300 (3 CTAs of 8 consumer warps per SM).
struct PlanCosts {
    double base = 550, window = 550, cmp_aligned = 190, cmp_shifted = 450;
    double zero_test = 120, compact = 480, compact_per_chunk = 10;
    double round = 350, iter = 450, iter_per_lane = 15;
};

// Modelled cost of peeling the set sel[0..k) (in: the same indices as a
// set): the dense phase, then the zero test, the compaction and the sparse
// rounds, which continue with the other compares in the order pi.
inline double plan_cost(const uint32_t* v, uint32_t m, const double* freq, const uint32_t* sel, uint32_t k,
                        const PlanSet& in) {
    const PlanCosts C;
    double cost = C.base, alive = 1.0;
    for (uint32_t a = 0; a < k; ++a) {
        bool seen = false;
        for (uint32_t b = 0; b < a; ++b) seen = seen || group_e(v[sel[b]]) == group_e(v[sel[a]]);
        cost += (seen ? 0.0 : C.window) + (aligned(v[sel[a]]) ? C.cmp_aligned : C.cmp_shifted);
        alive *= freq[sel[a]];
    }
    if (k >= m) return cost;
    cost += C.zero_test;
    // 1 - (1 - a)^n ~ 1 - exp(-n a): a warp-tile (2048 starts) with any
    // survivor, and the expected number of its 16-start chunks with one
    const double p_any = -std::expm1(-2048.0 * alive);
    const double qn = -128.0 * std::expm1(-16.0 * alive);
    if (p_any < 1e-6) return cost;
    cost += p_any * (C.compact + C.compact_per_chunk * qn);
    // sparse rounds: two compares per zero test, the rest in the order pi
    const double rounds = std::fmax(1.0, qn / 32.0);
    double a = alive;
    uint32_t iters = 0, i = 0;
    auto next = [&]() -> int64_t {
        while (i < m && in.has(i)) ++i;
        return i < m ? (int64_t)i++ : -1;
    };
    while (iters < 64) {
        const int64_t j1 = next();
        if (j1 < 0) break;
        const int64_t j2 = next();
        ++iters;
        a *= freq[j1] * (j2 >= 0 ? freq[j2] : 1.0);
        if (j2 < 0 || a < 2.44e-4) break;   // fewer than 0.5 of the 128 chunks still alive
    }
    cost += p_any * rounds * (C.round + iters * (C.iter + C.iter_per_lane * std::fmin(32.0, qn / rounds)));
    return cost;
}

// Plans the dense phase of a pattern with compare descriptors v[0..m) in
// the order pi. freq[j] is the text frequency of v[j]'s symbol (nullptr:
// unknown; then r = min(m, 2), the paper's choice for English). r_fixed > 0
// peels the first r_fixed compares of pi. Writes the m descriptors in scan
// order to qc (the r peeled ones by window, in each window the aligned ones
// by word class and then the others by word class; then the rest in the
// order pi) and the window groups to groups (one per distinct window, at
// most max_groups_for(m)). Returns r, or 0 when the groups exceed
// max_groups; *ng = number of groups.
inline uint32_t plan_dense(const uint32_t* v, uint32_t m, const double* freq, uint32_t r_fixed, uint32_t* qc,
                           uint32_t* groups, uint32_t max_groups, uint32_t* ng) {
    uint32_t sel[kPlanMaxPeel > kPlanCandidates ? kPlanMaxPeel : kPlanCandidates];
    uint32_t k = 0;
    bool implicit = false;   // a long forced peel: the first r compares of pi
    if (r_fixed || !freq) {
        const uint32_t r = r_fixed ? (r_fixed < m ? r_fixed : m) : (m < 2 ? m : 2);
        implicit = r > kPlanCandidates;
        if (implicit)
            k = r;
        else
            for (k = 0; k < r; ++k) sel[k] = k;
    } else {
        const PlanCosts C;
        const uint32_t top = m < kPlanMaxPeel ? m : kPlanMaxPeel;
        double best = 1e300;
        uint32_t cand[kPlanMaxPeel];
        // prefixes of pi
        PlanSet in;
        for (uint32_t r = 1; r <= top; ++r) {
            cand[r - 1] = r - 1;
            in.add(r - 1);
            const double c = plan_cost(v, m, freq, cand, r, in);
            if (c < best) {
                best = c;
                k = r;
                for (uint32_t a = 0; a < r; ++a) sel[a] = cand[a];
            }
        }
        // prefixes of the greedy order by information per modelled cost over
        // a pool: the kPlanCandidates rarest compares, the aligned compares
        // of the kPlanWindows windows whose aligned compares carry the most
        // information, and every compare of a window already loaded. On
        // texts whose symbols are about equally frequent the rarest compares
        // of a long pattern are spread over many windows, while one window's
        // aligned compares cost one load and no shifts.
        constexpr uint32_t kW = max_groups_for(kPlanMaxM);
        const uint32_t nwin = max_groups_for(m);
        uint16_t by_win[kW][16];   // compares of each window (j in the order pi), long patterns
        uint8_t nby[kW];
        if (m > kPlanCandidates) {
            for (uint32_t E = 0; E < nwin; ++E) nby[E] = 0;
            for (uint32_t j = 0; j < m; ++j) {
                const uint32_t E = group_e(v[j]);
                by_win[E][nby[E]++] = (uint16_t)j;
            }
        }
        uint32_t pool[kPlanCandidates + 4 * kPlanWindows], np = 0;
        const uint32_t nrare = m < kPlanCandidates ? m : kPlanCandidates;
        for (uint32_t j = 0; j < nrare; ++j) pool[np++] = j;
        if (m > kPlanCandidates) {
            double wsum[kW];
            for (uint32_t E = 0; E < nwin; ++E) {
                wsum[E] = 0.0;
                for (uint32_t t = 0; t < nby[E]; ++t)
                    if (aligned(v[by_win[E][t]])) wsum[E] += -std::log(std::fmax(freq[by_win[E][t]], 1e-300));
            }
            for (uint32_t t = 0; t < kPlanWindows; ++t) {
                int64_t pick = -1;
                for (uint32_t E = 0; E < nwin; ++E)
                    if (wsum[E] > 0.0 && (pick < 0 || wsum[E] > wsum[pick])) pick = E;
                if (pick < 0) break;
                for (uint32_t u = 0; u < nby[pick]; ++u) {
                    const uint32_t j = by_win[pick][u];
                    if (j >= kPlanCandidates && aligned(v[j])) pool[np++] = j;
                }
                wsum[pick] = 0.0;
            }
        }
        PlanSet inmask;
        uint32_t wins[kPlanMaxPeel], nw = 0;   // windows of the compares taken so far
        for (uint32_t r = 1; r <= top; ++r) {
            double best_gain = -1.0;
            uint32_t pick = 0;
            auto consider = [&](uint32_t j, bool loaded) {
                if (inmask.has(j)) return;
                const double cost = (loaded ? 0.0 : C.window) + (aligned(v[j]) ? C.cmp_aligned : C.cmp_shifted);
                const double gain = -std::log(std::fmax(freq[j], 1e-300)) / cost;
                if (gain > best_gain) {
                    best_gain = gain;
                    pick = j;
                }
            };
            for (uint32_t p = 0; p < np; ++p) {
                bool loaded = false;
                for (uint32_t w = 0; w < nw; ++w) loaded = loaded || wins[w] == group_e(v[pool[p]]);
                consider(pool[p], loaded);
            }
            if (m > kPlanCandidates)   // (shorter patterns have every compare in the pool)
                for (uint32_t w = 0; w < nw; ++w)
                    for (uint32_t u = 0; u < nby[wins[w]]; ++u) consider(by_win[wins[w]][u], true);
            if (best_gain < 0.0) break;   // every candidate is taken
            cand[r - 1] = pick;
            inmask.add(pick);
            bool known = false;
            for (uint32_t w = 0; w < nw; ++w) known = known || wins[w] == group_e(v[pick]);
            if (!known) wins[nw++] = group_e(v[pick]);
            const double c = plan_cost(v, m, freq, cand, r, inmask);
            if (c < best) {
                best = c;
                k = r;
                for (uint32_t a = 0; a < r; ++a) sel[a] = cand[a];
            }
        }
    }
    const uint32_t r = k;
    auto sel_at = [&](uint32_t a) { return implicit ? a : sel[a]; };
    // the peeled compares by window, in ascending order; in a window the
    // aligned ones by word class, then the others by word class
    uint32_t o = 0, g = 0;
    int64_t prev = -1;
    while (o < r) {
        uint32_t E = ~0u;
        for (uint32_t a = 0; a < r; ++a) {
            const uint32_t e = group_e(v[sel_at(a)]);
            if ((int64_t)e > prev && e < E) E = e;
        }
        prev = E;
        uint32_t desc = E;
        for (uint32_t pass = 0; pass < 2; ++pass)
            for (uint32_t d = 0; d < 4; ++d) {
                uint32_t cnt = 0;
                for (uint32_t a = 0; a < r; ++a) {
                    const uint32_t x = v[sel_at(a)];
                    if (group_e(x) == E && word_class(x) == d && aligned(x) == (pass == 0)) {
                        qc[o++] = x;
                        ++cnt;
                    }
                }
                desc |= pass == 0 ? (cnt << (9 + d)) : (cnt << (13 + 2 * d));
            }
        if (g >= max_groups) return 0;
        groups[g++] = desc;
    }
    // the rest in the order pi
    PlanSet taken;
    for (uint32_t a = 0; a < r && !implicit; ++a) taken.add(sel[a]);
    for (uint32_t j = 0; j < m; ++j) {
        const bool in = implicit ? j < r : taken.has(j);
        if (!in) qc[o++] = v[j];
    }
    *ng = g;
    return r;
}

// ------------------------------------------------------------ packed texts

// Bit positions b1 < b2 at which the text's symbols (at most four; hist has
// 256 bins) all differ, so that (bit b1, bit b2) is an injective 2-bit code.
// Prefers adjacent positions. False when the text has more than four
// symbols or no such pair exists.
inline bool packed_code_bits(const uint64_t* hist, uint32_t* b1, uint32_t* b2) {
    uint32_t sym[4], ns = 0;
    for (uint32_t c = 0; c < 256; ++c)
        if (hist[c]) {
            if (ns == 4) return false;
            sym[ns++] = c;
        }
    if (ns == 0) return false;
    for (uint32_t pass = 0; pass < 2; ++pass)
        for (uint32_t x = 0; x < 8; ++x)
            for (uint32_t z = x + 1; z < 8; ++z) {
                if ((pass == 0) != (z == x + 1)) continue;
                uint32_t seen = 0;
                bool ok = true;
                for (uint32_t i = 0; i < ns && ok; ++i) {
                    const uint32_t code = ((sym[i] >> x) & 1u) | (((sym[i] >> z) & 1u) << 1);
                    ok = !((seen >> code) & 1u);
                    seen |= 1u << code;
                }
                if (ok) {
                    *b1 = x;
                    *b2 = z;
                    return true;
                }
            }
    return false;
}

// Bit b1 at which the text's symbols (at most two; hist has 256 bins)
// differ, so that it is an injective 1-bit code (0 for a single symbol).
// False when the text has more than two symbols.
inline bool binary_code_bit(const uint64_t* hist, uint32_t* b1) {
    uint32_t sym[2], ns = 0;
    for (uint32_t c = 0; c < 256; ++c)
        if (hist[c]) {
            if (ns == 2) return false;
            sym[ns++] = c;
        }
    if (ns == 0) return false;
    uint32_t x = 0;
    if (ns == 2)
        while (!(((sym[0] ^ sym[1]) >> x) & 1u)) ++x;
    *b1 = x;
    return true;
}

// Packed group descriptor: window E' = e >> 6 (64 starts: four words of
// 2-bit codes, two of 1-bit codes) in bits 0-8; bit 9 + D set when the group
// has the compare of word class D (2-bit codes: D = (e >> 4) & 3, 1-bit codes:
// D = (e >> 5) & 1) that needs no shift (e mod 16 == 0, resp. e mod 32 == 0);
// then the number of its other compares of class D: 2-bit codes in bits
// 13 + 4D .. 16 + 4D (at most 15), 1-bit codes in bits 13 + 5D .. 17 + 5D
// (at most 31).
constexpr uint32_t max_packed_groups_for(uint32_t m) { return (14 + m) / 64 + 1; }

// Plans the dense phase on 2-bit codes (bits = 2) or 1-bit codes (bits = 1).
// v[j] = (e << 8) | code in the order pi, freq[j] the text frequency of its
// symbol (nullptr: unknown). A packed compare costs a few integer
// instructions per 16 (32) starts, so the first compares of pi are peeled
// until fewer than 1e-5 of the starts are expected to survive (or all m;
// r_fixed > 0 peels r_fixed). Output as for plan_dense, with packed group
// descriptors.
inline uint32_t plan_packed(const uint32_t* v, uint32_t m, const double* freq, uint32_t r_fixed, uint32_t* qc,
                            uint32_t* groups, uint32_t max_groups, uint32_t* ng, uint32_t bits = 2) {
    uint32_t r = 0;
    if (r_fixed) {
        r = r_fixed < m ? r_fixed : m;
    } else if (!freq) {
        r = m < 16 ? m : 16;
    } else {
        double alive = 1.0;
        while (r < m && r < 64 && (r < 2 || alive >= 1e-5)) alive *= freq[r++];
    }
    const uint32_t cb = bits == 1 ? 5u : 4u;                     // log2 of the starts per word
    auto win = [](uint32_t x) { return x >> 14; };               // e >> 6
    auto cls = [cb](uint32_t x) { return (x >> (8 + cb)) & ((64u >> cb) - 1u); };
    auto unshifted = [cb](uint32_t x) { return ((x >> 8) & ((1u << cb) - 1u)) == 0; };
    uint32_t o = 0, g = 0;
    int64_t prev = -1;
    while (o < r) {
        uint32_t E = ~0u;
        for (uint32_t a = 0; a < r; ++a)
            if ((int64_t)win(v[a]) > prev && win(v[a]) < E) E = win(v[a]);
        prev = E;
        uint32_t desc = E;
        for (uint32_t pass = 0; pass < 2; ++pass)
            for (uint32_t d = 0; d < 4; ++d) {
                uint32_t cnt = 0;
                for (uint32_t a = 0; a < r; ++a)
                    if (win(v[a]) == E && cls(v[a]) == d && unshifted(v[a]) == (pass == 0)) {
                        qc[o++] = v[a];
                        ++cnt;
                    }
                desc |= pass == 0 ? (cnt << (9 + d)) : (cnt << (13 + (bits == 1 ? 5u : 4u) * d));
            }
        if (g >= max_groups) return 0;
        groups[g++] = desc;
    }
    for (uint32_t j = r; j < m; ++j) qc[o++] = v[j];
    *ng = g;
    return r;
}

}  // namespace smk
