// Invariant checks of the host planner (paper_1612_01506_gb300/csrc/sm_plan.h)
// on random inputs, run on the CPU by tests/test_plan.py. The kernels read the
// planner's output as: the m compare descriptors in scan order (the r peeled
// ones first, grouped by window) and one descriptor per window group giving
// how many compares of each word class it holds. A plan that loses, repeats
// or misfiles a compare would make a GPU count wrong, so every plan is
// checked against those rules here. Prints "ok <plans checked>" or the first
// violation.
#include "sm_plan.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

using namespace smk;

static int fail(const char* what, uint32_t m, uint32_t r) {
    std::printf("FAIL %s (m=%u r=%u)\n", what, m, r);
    return 1;
}

// Byte compares: groups of plan_dense. The peeled qc[0..r) must be listed
// window by window in ascending window order; in a window the aligned
// compares (one per word class at most) by class, then the others by class,
// as the group descriptor counts them; qc must be a permutation of v.
static int check_dense(std::mt19937_64& g) {
    // lengths up to 200, or up to 4096 (long patterns, where the greedy
    // pool also takes aligned compares beyond the 64 rarest); frequencies
    // spread out, or nearly equal (a uniform text)
    const uint32_t m = 1 + (uint32_t)(g() % ((g() % 4 == 0) ? 4096 : 200));
    const uint32_t delta = (uint32_t)(g() % 16);
    const bool flat = g() % 2 == 0;
    std::vector<uint32_t> v(m), qc(m), groups(max_groups_for(m));
    std::vector<double> freq(m);
    for (uint32_t j = 0; j < m; ++j) {
        v[j] = ((j + delta) << 8) | (uint32_t)(g() % 256);
        freq[j] = flat ? 0.05 * (1.0 + 1e-3 * (double)(g() % 100)) : 1.0 / (double)(1 + g() % 300);
    }
    std::shuffle(v.begin(), v.end(), g);   // an order pi: positions in any order
    std::sort(freq.begin(), freq.end());  // rarest first
    const uint32_t r_fixed = (g() % 4 == 0) ? 1 + (uint32_t)(g() % m) : 0;
    uint32_t ng = 0;
    const uint32_t r = plan_dense(v.data(), m, (g() % 5) ? freq.data() : nullptr, r_fixed, qc.data(), groups.data(),
                                  (uint32_t)groups.size(), &ng);
    if (r == 0 || r > m) return fail("dense r out of range", m, r);
    if (r_fixed && r != (r_fixed < m ? r_fixed : m)) return fail("dense forced peel not kept", m, r);
    std::vector<uint32_t> a(v), b(qc);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return fail("dense qc is not a permutation of the compares", m, r);
    uint32_t j = 0, prevE = 0;
    for (uint32_t k = 0; k < ng; ++k) {
        const uint32_t gd = groups[k], E = gd & 0x1FFu;
        if (k && E <= prevE) return fail("dense windows not ascending", m, r);
        prevE = E;
        for (uint32_t pass = 0; pass < 2; ++pass)
            for (uint32_t D = 0; D < 4; ++D) {
                const uint32_t cnt = pass == 0 ? (gd >> (9 + D)) & 1u : (gd >> (13 + 2 * D)) & 3u;
                for (uint32_t c = 0; c < cnt; ++c, ++j) {
                    if (j >= r) return fail("dense groups hold more than r compares", m, r);
                    const uint32_t e = qc[j] >> 8;
                    if ((e >> 4) != E) return fail("dense compare outside its window", m, r);
                    if (((e >> 2) & 3u) != D) return fail("dense compare in the wrong word class", m, r);
                    if (((e & 3u) == 0) != (pass == 0)) return fail("dense aligned flag wrong", m, r);
                }
            }
    }
    if (j != r) return fail("dense groups do not cover the peeled compares", m, r);
    return 0;
}

// Coded compares: groups of plan_packed (bits = 2: 16 starts per word;
// bits = 1: 32). Same rules with the packed descriptor layout.
static int check_packed(std::mt19937_64& g, uint32_t bits) {
    const uint32_t m = 1 + (uint32_t)(g() % 600);
    const uint32_t delta = (uint32_t)(g() % 16);
    std::vector<uint32_t> v(m), qc(m), groups(max_packed_groups_for(m));
    std::vector<double> freq(m);
    for (uint32_t j = 0; j < m; ++j) {
        v[j] = ((j + delta) << 8) | (uint32_t)(g() % (bits == 1 ? 2 : 4));
        freq[j] = bits == 1 ? 0.5 : 0.25;
    }
    std::shuffle(v.begin(), v.end(), g);
    const uint32_t r_fixed = (g() % 4 == 0) ? 1 + (uint32_t)(g() % m) : 0;
    uint32_t ng = 0;
    const uint32_t r = plan_packed(v.data(), m, freq.data(), r_fixed, qc.data(), groups.data(),
                                   (uint32_t)groups.size(), &ng, bits);
    if (r == 0 || r > m) return fail("packed r out of range", m, r);
    std::vector<uint32_t> a(v), b(qc);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return fail("packed qc is not a permutation of the compares", m, r);
    const uint32_t cb = bits == 1 ? 5u : 4u, nclass = 64u >> cb, cw = bits == 1 ? 5u : 4u;
    uint32_t j = 0, prevE = 0;
    for (uint32_t k = 0; k < ng; ++k) {
        const uint32_t gd = groups[k], E = gd & 0x1FFu;
        if (k && E <= prevE) return fail("packed windows not ascending", m, r);
        prevE = E;
        for (uint32_t pass = 0; pass < 2; ++pass)
            for (uint32_t D = 0; D < nclass; ++D) {
                const uint32_t cnt = pass == 0 ? (gd >> (9 + D)) & 1u : (gd >> (13 + cw * D)) & ((1u << cw) - 1u);
                for (uint32_t c = 0; c < cnt; ++c, ++j) {
                    if (j >= r) return fail("packed groups hold more than r compares", m, r);
                    const uint32_t e = qc[j] >> 8;
                    if ((e >> 6) != E) return fail("packed compare outside its window", m, r);
                    if (((e >> cb) & (nclass - 1u)) != D) return fail("packed compare in the wrong word class", m, r);
                    if (((e & ((1u << cb) - 1u)) == 0) != (pass == 0)) return fail("packed aligned flag wrong", m, r);
                }
            }
    }
    if (j != r) return fail("packed groups do not cover the peeled compares", m, r);
    return 0;
}

// Code bits: for random sets of <= 4 (<= 2) symbols the chosen bits must
// give distinct codes; larger sets must be refused.
static int check_codes(std::mt19937_64& g) {
    const uint32_t ns = 1 + (uint32_t)(g() % 6);
    uint64_t hist[256] = {};
    uint32_t sym[6];
    for (uint32_t i = 0; i < ns; ++i) {
        uint32_t c;
        bool dup;
        do {
            c = (uint32_t)(g() % 256);
            dup = false;
            for (uint32_t k = 0; k < i; ++k) dup = dup || sym[k] == c;
        } while (dup);
        sym[i] = c;
        hist[c] = 1 + g() % 1000;
    }
    uint32_t b1 = 99, b2 = 99;
    const bool two = packed_code_bits(hist, &b1, &b2);
    if (ns > 4 && two) return fail("2-bit codes for more than four symbols", ns, 0);
    if (two) {
        if (!(b1 < b2 && b2 < 8)) return fail("2-bit code bits out of order", ns, 0);
        uint32_t seen = 0;
        for (uint32_t i = 0; i < ns; ++i) {
            const uint32_t code = ((sym[i] >> b1) & 1u) | (((sym[i] >> b2) & 1u) << 1);
            if ((seen >> code) & 1u) return fail("2-bit codes collide", ns, 0);
            seen |= 1u << code;
        }
    }
    uint32_t c1 = 99;
    const bool one = binary_code_bit(hist, &c1);
    if ((ns <= 2) != one) return fail("1-bit codes offered wrongly", ns, 0);
    if (one && ns == 2 && ((sym[0] >> c1) & 1u) == ((sym[1] >> c1) & 1u)) return fail("1-bit codes collide", ns, 0);
    return 0;
}

// Long patterns over a text whose symbols are about equally frequent: the
// order pi (by frequency) scatters the pattern positions, but the peeled
// compares must come from one 16-byte window, its aligned ones (one load and
// no shifts), as for a short pattern.
static int check_flat_long() {
    std::mt19937_64 g(7);
    for (uint32_t m : {128u, 1024u, 4096u}) {
        std::vector<uint32_t> v(m), qc(m), groups(max_groups_for(m));
        std::vector<double> freq(m);
        std::vector<uint32_t> pos(m);
        for (uint32_t j = 0; j < m; ++j) pos[j] = j;
        std::shuffle(pos.begin(), pos.end(), g);
        for (uint32_t j = 0; j < m; ++j) {
            v[j] = (pos[j] << 8) | 65u;
            freq[j] = 0.05 * (1.0 + 1e-4 * (double)j);   // rarest first, nearly equal
        }
        uint32_t ng = 0;
        const uint32_t r = plan_dense(v.data(), m, freq.data(), 0, qc.data(), groups.data(),
                                      (uint32_t)groups.size(), &ng);
        if (r < 3 || ng != 1) return fail("flat long pattern: peel not taken from one window", m, r);
        for (uint32_t a = 0; a < r; ++a)
            if (((qc[a] >> 8) & 3u) != 0) return fail("flat long pattern: a shifted compare peeled", m, r);
    }
    return 0;
}

int main(int argc, char** argv) {
    const uint64_t seed = argc > 1 ? std::strtoull(argv[1], nullptr, 10) : 1;
    const int n = argc > 2 ? std::atoi(argv[2]) : 20000;
    std::mt19937_64 g(seed);
    if (check_flat_long()) return 1;
    int checked = 0;
    for (int i = 0; i < n; ++i) {
        if (check_dense(g) || check_packed(g, 2) || check_packed(g, 1) || check_codes(g)) return 1;
        checked += 4;
    }
    std::printf("ok %d\n", checked);
    return 0;
}
