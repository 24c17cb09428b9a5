/*
 * ORACLE for exact string matching - TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously correct CPU statement of what the GPU
 * library computes. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Problem statement (Tarhio, Holub, Giaquinta, "Technology Beats Algorithms
 * (in Exact String Matching)", Sec. 1): count or report every location of a
 * pattern p of length m in a text t of length n over a finite alphabet.
 * Symbols here are bytes compared as unsigned values; indices are 0-based
 * (the paper counts from 1) and overlapping occurrences all count.
 *
 * Functions and the passage each follows:
 *   oracle_naive_count   Algorithm 1 (Naive-search), Sec. 2.1: every start i,
 *                        found <- true, AND in the m compares in position
 *                        order, leave at the first false, count if found.
 *   oracle_naive_report  The reporting version of Algorithm 1 (Sec. 2.1: emit
 *                        position i where Algorithm 1 increments the count).
 *   oracle_memcmp_count  Independent cross-check: memcmp at every start.
 *   oracle_kmp_count     Independent cross-check: Knuth-Morris-Pratt
 *                        automaton (cited in Sec. 1 as a classic solution).
 *   oracle_histogram     Symbol frequencies of the text itself (Sec. 2.2
 *                        orders compares by symbol frequency; the frequency
 *                        source read here is the searched text).
 *   oracle_order_freq    Sec. 2.2 / Algorithm 3: the order pi compares
 *                        pattern positions by increasing frequency of their
 *                        symbol; built with a standard sort (Sec. 2.2).
 *                        Equal frequencies keep ascending position.
 *   oracle_order_h       Sec. 2.4: the fixed order pi_h = p[1], p[m], p[4],
 *                        p[7], ..., p[3], p[6], ..., p[2], p[5], ... with each
 *                        position taken once.
 *   oracle_order_hs      Sec. 2.4: pi_hs - positions holding a space go last
 *                        (ascending); the other positions are ordered by the
 *                        pi_h scheme applied to their list.
 *   oracle_batch_count   Algorithm 1 applied to each (text, pattern) pair of a
 *                        packed batch.
 *   oracle_count_threads / oracle_report_threads
 *                        Algorithm 1 on start ranges split across host
 *                        threads (ranges overlap by m-1 text bytes); used to
 *                        time the CPU baseline and to check large inputs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---------------------------------------------------------------- Alg. 1 */

uint64_t oracle_naive_count(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n) {
    uint64_t count = 0;
    if (m > n) return 0;
    for (uint64_t i = 0; i + m <= n; ++i) {          /* i = 1 .. n-m+1, 0-based */
        int found = 1;
        for (uint64_t j = 0; j < m; ++j) {
            found = found && (t[i + j] == p[j]);
            if (!found) break;                        /* go to the next start */
        }
        if (found) count += 1;                        /* the counting line */
    }
    return count;
}

uint64_t oracle_naive_report(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n,
                             uint64_t* pos, uint64_t cap) {
    uint64_t count = 0;
    if (m > n) return 0;
    for (uint64_t i = 0; i + m <= n; ++i) {
        int found = 1;
        for (uint64_t j = 0; j < m; ++j) {
            found = found && (t[i + j] == p[j]);
            if (!found) break;
        }
        if (found) {                                   /* report i instead of counting */
            if (count < cap) pos[count] = i;
            count += 1;
        }
    }
    return count;
}

/* ------------------------------------------------------- cross-checks */

uint64_t oracle_memcmp_count(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n) {
    uint64_t c = 0;
    if (m > n) return 0;
    for (uint64_t i = 0; i + m <= n; ++i)
        if (memcmp(t + i, p, (size_t)m) == 0) ++c;
    return c;
}

uint64_t oracle_kmp_count(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n) {
    if (m == 0 || m > n) return m == 0 ? n + 1 : 0;
    /* fail[j] = length of the longest proper border of p[0..j] */
    uint64_t* fail = (uint64_t*)malloc(m * sizeof(uint64_t));
    if (!fail) return UINT64_MAX;
    fail[0] = 0;
    for (uint64_t j = 1, k = 0; j < m; ++j) {
        while (k > 0 && p[j] != p[k]) k = fail[k - 1];
        if (p[j] == p[k]) ++k;
        fail[j] = k;
    }
    uint64_t c = 0;
    for (uint64_t i = 0, k = 0; i < n; ++i) {
        while (k > 0 && t[i] != p[k]) k = fail[k - 1];
        if (t[i] == p[k]) ++k;
        if (k == m) { ++c; k = fail[k - 1]; }
    }
    free(fail);
    return c;
}

/* ----------------------------------------------------------- Sec. 2.2 */

void oracle_histogram(const uint8_t* t, uint64_t n, uint64_t* h256) {
    for (int c = 0; c < 256; ++c) h256[c] = 0;
    for (uint64_t x = 0; x < n; ++x) h256[t[x]] += 1;
}

typedef struct { uint64_t key; uint32_t q; } okey_t;

static int okey_cmp(const void* a, const void* b) {
    const okey_t* x = (const okey_t*)a;
    const okey_t* y = (const okey_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->q < y->q ? -1 : (x->q > y->q);
}

int oracle_order_freq(const uint8_t* p, uint32_t m, const uint64_t* h256, uint32_t* pi) {
    okey_t* k = (okey_t*)malloc((size_t)(m ? m : 1) * sizeof(okey_t));
    if (!k) return -1;
    for (uint32_t q = 0; q < m; ++q) { k[q].key = h256[p[q]]; k[q].q = q; }
    qsort(k, m, sizeof(okey_t), okey_cmp);   /* (frequency, position) is a total order */
    for (uint32_t j = 0; j < m; ++j) pi[j] = k[j].q;
    free(k);
    return 0;
}

/* ----------------------------------------------------------- Sec. 2.4 */

/* pi_h over the list pos[0..len-1]; 1-based ranks 1, len, 4, 7, .., 3, 6, .., 2, 5, .. */
static void order_h_list(const uint32_t* pos, uint32_t len, uint32_t* out) {
    uint32_t k = 0;
    if (len == 0) return;
    out[k++] = pos[0];                                 /* rank 1 */
    if (len > 1) out[k++] = pos[len - 1];              /* rank m */
    for (uint32_t r = 4; r < len; r += 3) out[k++] = pos[r - 1];   /* 4, 7, ...  */
    for (uint32_t r = 3; r < len; r += 3) out[k++] = pos[r - 1];   /* 3, 6, ...  */
    for (uint32_t r = 2; r < len; r += 3) out[k++] = pos[r - 1];   /* 2, 5, ...  */
}

int oracle_order_h(uint32_t m, uint32_t* pi) {
    uint32_t* ident = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    if (!ident) return -1;
    for (uint32_t q = 0; q < m; ++q) ident[q] = q;
    order_h_list(ident, m, pi);
    free(ident);
    return 0;
}

int oracle_order_hs(const uint8_t* p, uint32_t m, uint32_t* pi) {
    uint32_t* rest = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    if (!rest) return -1;
    uint32_t nr = 0, ns = 0;
    for (uint32_t q = 0; q < m; ++q) if (p[q] != 0x20) rest[nr++] = q;
    order_h_list(rest, nr, pi);
    for (uint32_t q = 0; q < m; ++q) if (p[q] == 0x20) pi[nr + ns++] = q;
    free(rest);
    return 0;
}

/* ------------------------------------------------------------- batches */

int oracle_batch_count(const uint8_t* texts, const int64_t* text_off, uint32_t ntexts,
                       const uint8_t* pats, const int64_t* pat_off, const int32_t* pat_text,
                       uint32_t npats, int64_t* counts) {
    for (uint32_t k = 0; k < npats; ++k) {
        int32_t x = pat_text[k];
        if (x < 0 || (uint32_t)x >= ntexts) return -1;
        const uint8_t* t = texts + text_off[x];
        uint64_t n = (uint64_t)(text_off[x + 1] - text_off[x]);
        const uint8_t* p = pats + pat_off[k];
        uint64_t m = (uint64_t)(pat_off[k + 1] - pat_off[k]);
        counts[k] = (int64_t)oracle_naive_count(p, m, t, n);
    }
    return 0;
}

/* ------------------------------------------------- threaded driver */

typedef struct {
    const uint8_t* p; uint64_t m; const uint8_t* t; uint64_t n;
    uint64_t s0, s1;          /* start range [s0, s1) */
    uint64_t count;
    uint64_t* pos; uint64_t cap;
} ojob_t;

static void* count_job(void* a) {
    ojob_t* j = (ojob_t*)a;
    uint64_t len = j->s1 - j->s0 + j->m - 1;
    j->count = j->s1 > j->s0 ? oracle_naive_count(j->p, j->m, j->t + j->s0, len) : 0;
    return NULL;
}

static void* report_job(void* a) {
    ojob_t* j = (ojob_t*)a;
    uint64_t len = j->s1 - j->s0 + j->m - 1;
    if (j->s1 <= j->s0) { j->count = 0; return NULL; }
    j->count = oracle_naive_report(j->p, j->m, j->t + j->s0, len, j->pos, j->cap);
    for (uint64_t i = 0; i < j->count && i < j->cap; ++i) j->pos[i] += j->s0;
    return NULL;
}

static int split(ojob_t* jobs, int nt, const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n) {
    if (nt < 1) nt = 1;
    if (nt > 512) nt = 512;
    uint64_t starts = (m == 0 || m > n) ? 0 : n - m + 1;
    for (int k = 0; k < nt; ++k) {
        jobs[k].p = p; jobs[k].m = m; jobs[k].t = t; jobs[k].n = n;
        jobs[k].s0 = starts * (uint64_t)k / (uint64_t)nt;
        jobs[k].s1 = starts * (uint64_t)(k + 1) / (uint64_t)nt;
        jobs[k].count = 0; jobs[k].pos = NULL; jobs[k].cap = 0;
    }
    return nt;
}

static void run(void* (*fn)(void*), ojob_t* jobs, int nt) {
    pthread_t th[512];
    int ok[512];
    for (int k = 0; k < nt; ++k) ok[k] = nt > 1 && pthread_create(&th[k], NULL, fn, &jobs[k]) == 0;
    for (int k = 0; k < nt; ++k) { if (ok[k]) pthread_join(th[k], NULL); else fn(&jobs[k]); }
}

uint64_t oracle_count_threads(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n, int threads) {
    ojob_t jobs[512];
    if (m == 0) return oracle_naive_count(p, m, t, n);
    int nt = split(jobs, threads, p, m, t, n);
    run(count_job, jobs, nt);
    uint64_t c = 0;
    for (int k = 0; k < nt; ++k) c += jobs[k].count;
    return c;
}

/* Positions ascending; writes at most cap of them and returns the full count. */
uint64_t oracle_report_threads(const uint8_t* p, uint64_t m, const uint8_t* t, uint64_t n,
                               uint64_t* pos, uint64_t cap, int threads) {
    ojob_t jobs[512];
    if (m == 0) return oracle_naive_report(p, m, t, n, pos, cap);
    int nt = split(jobs, threads, p, m, t, n);
    run(count_job, jobs, nt);
    uint64_t base = 0;
    for (int k = 0; k < nt; ++k) {
        uint64_t c = jobs[k].count;
        jobs[k].pos = pos + (base < cap ? base : cap);
        jobs[k].cap = base < cap ? (cap - base < c ? cap - base : c) : 0;
        base += c;
    }
    run(report_job, jobs, nt);
    return base;
}
