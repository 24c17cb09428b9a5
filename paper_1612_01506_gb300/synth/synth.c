/*
 * Seeded synthetic inputs for exact string matching: texts and patterns.
 *
 * This file generates bytes only. It holds none of the matching arithmetic
 * (no comparison, no counting, no ordering) and is shared by the test suite,
 * the benchmark and the serving demo as the one source of input data.
 *
 * Every random number is counter based: draw(seed, stream, i) is the
 * SplitMix64 output function (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to the state
 * key(seed, stream) + (i + 1) * GOLDEN. Any byte of any text can therefore be
 * produced independently of the others, which lets the work split across
 * threads without changing the output.
 *
 * Text families (stand-ins for the corpora of the paper's experiments):
 *   uniform  - i.i.d. symbols over a given alphabet, symbol index
 *              (hi32(draw) * sigma) >> 32.
 *   markov95 - English-like text over the 95 printable ASCII bytes
 *              0x20..0x7E: a first-order reversible Markov chain whose
 *              stationary law is Zipf(s = 1) by rank (the space at rank 1,
 *              the other 94 bytes ranked by a seeded permutation) and whose
 *              transitions favour 8 neighbours on a seeded ring, so that
 *              adjacent symbols are correlated (see mk_build). The text is
 *              cut into independent 64 KiB chunks, each starting from a
 *              stationary draw.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL
#define MK_SYMS 95
#define MK_CHUNK (64u * 1024u)

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm64_mix(sm64_mix(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t draw_k(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * GOLDEN);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t index) {
    return draw_k(stream_key(seed, stream), index);
}

/* Uniform integers in [0, range) for k consecutive counters of one stream. */
void synth_below(uint64_t* out, uint64_t k, uint64_t range, uint64_t seed, uint64_t stream) {
    uint64_t key = stream_key(seed, stream);
    for (uint64_t i = 0; i < k; ++i) {
        unsigned __int128 x = (unsigned __int128)draw_k(key, i) * range;
        out[i] = (uint64_t)(x >> 64);
    }
}

/* ------------------------------------------------------------------ threads */

typedef struct {
    uint8_t* out;
    uint64_t lo, hi;           /* uniform: byte range; markov: chunk range */
    uint64_t n;
    uint64_t key;
    const uint8_t* alpha;
    uint32_t sigma;
    const void* model;
} job_t;

static int clamp_threads(int threads, uint64_t units) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > units) threads = units ? (int)units : 1;
    return threads;
}

static void run_jobs(void* (*fn)(void*), job_t* jobs, int nt) {
    pthread_t tid[256];
    int started[256];
    for (int i = 0; i < nt; ++i)
        started[i] = (nt > 1) && pthread_create(&tid[i], NULL, fn, &jobs[i]) == 0;
    for (int i = 0; i < nt; ++i) {
        if (started[i]) pthread_join(tid[i], NULL);
        else fn(&jobs[i]);
    }
}

/* ------------------------------------------------------------------ uniform */

static void* uniform_job(void* arg) {
    job_t* j = (job_t*)arg;
    const uint64_t sigma = j->sigma;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint64_t hi32 = draw_k(j->key, i) >> 32;
        j->out[i] = j->alpha[(hi32 * sigma) >> 32];
    }
    return NULL;
}

int synth_uniform(uint8_t* out, uint64_t n, const uint8_t* alpha, uint32_t sigma,
                  uint64_t seed, uint64_t stream, int threads) {
    if (!out || !alpha || sigma == 0 || sigma > 256) return -1;
    int nt = clamp_threads(threads, (n + (1u << 20) - 1) >> 20);
    job_t jobs[256];
    uint64_t key = stream_key(seed, stream);
    for (int t = 0; t < nt; ++t) {
        jobs[t].out = out; jobs[t].key = key; jobs[t].alpha = alpha; jobs[t].sigma = sigma;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nt;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nt;
    }
    run_jobs(uniform_job, jobs, nt);
    return 0;
}

/* ------------------------------------------------------------------ markov95 */

typedef struct {
    uint64_t w[MK_SYMS];            /* Zipf target weight per symbol index */
    uint64_t rowsum[MK_SYMS];       /* row sums of E: the exact stationary weights */
    uint64_t cum[MK_SYMS];          /* inclusive prefix sums of rowsum */
    uint64_t rowcum[MK_SYMS][MK_SYMS];  /* inclusive prefix sums of each row of E */
    uint8_t  byte_of[MK_SYMS];      /* symbol index -> byte (index = byte - 0x20) */
} mk_model;

static void shuffle_u8(uint8_t* a, int len, uint64_t key) {
    for (int i = len - 1; i > 0; --i) {
        unsigned __int128 x = (unsigned __int128)draw_k(key, (uint64_t)i) * (uint64_t)(i + 1);
        int j = (int)(uint64_t)(x >> 64);
        uint8_t t = a[i]; a[i] = a[j]; a[j] = t;
    }
}

/*
 * The chain moves a -> b with probability E[a][b] / rowsum[a], where E is a
 * symmetric non-negative integer matrix. Detailed balance then holds exactly
 * with stationary law rowsum / total. E is fitted so that its row sums follow
 * Zipf(s = 1): E = diag(x) K diag(x) with K[a][b] = 1 for the 8 neighbours of
 * a on a seeded ring and 1/50 elsewhere (self included); x comes from the
 * symmetric Sinkhorn iteration x <- sqrt(x * w / (K x)), then E is scaled to
 * integers. Only +, -, *, / and sqrt are used, each correctly rounded, so the
 * table is the same on every IEEE host (built with -ffp-contract=off).
 */
static void mk_build(mk_model* M, uint64_t seed) {
    uint8_t rest[MK_SYMS - 1], ring[MK_SYMS], ring_pos[MK_SYMS];
    for (int i = 0; i < MK_SYMS - 1; ++i) rest[i] = (uint8_t)(i + 1);
    shuffle_u8(rest, MK_SYMS - 1, stream_key(seed, 0x5A49504652414E4BULL));
    for (int s = 0; s < MK_SYMS; ++s) M->byte_of[s] = (uint8_t)(0x20 + s);
    for (int rank = 0; rank < MK_SYMS; ++rank) {
        int sym = rank == 0 ? 0 : rest[rank - 1];      /* rank 1 (0-based 0) is the space */
        M->w[sym] = 0xFFFFFFFFULL / (uint64_t)(rank + 1);
    }
    for (int i = 0; i < MK_SYMS; ++i) ring[i] = (uint8_t)i;
    shuffle_u8(ring, MK_SYMS, stream_key(seed, 0x52494E474F524452ULL));
    for (int i = 0; i < MK_SYMS; ++i) ring_pos[ring[i]] = (uint8_t)i;

    double K[MK_SYMS][MK_SYMS];
    double target[MK_SYMS], x[MK_SYMS], wsum = 0.0;
    for (int a = 0; a < MK_SYMS; ++a) wsum += (double)M->w[a];
    for (int a = 0; a < MK_SYMS; ++a) { target[a] = (double)M->w[a] / wsum; x[a] = 0.1; }
    for (int a = 0; a < MK_SYMS; ++a)
        for (int b = 0; b < MK_SYMS; ++b) {
            int d = (int)ring_pos[a] - (int)ring_pos[b];
            if (d < 0) d = -d;
            if (d > MK_SYMS - d) d = MK_SYMS - d;
            K[a][b] = (d >= 1 && d <= 4) ? 1.0 : 0.02;
        }
    for (int it = 0; it < 2000; ++it) {
        for (int a = 0; a < MK_SYMS; ++a) {
            double kx = 0.0;
            for (int b = 0; b < MK_SYMS; ++b) kx += K[a][b] * x[b];
            x[a] = sqrt(x[a] * target[a] / kx);
        }
    }
    const double scale = 1099511627776.0;   /* 2^40 */
    uint64_t total = 0;
    for (int a = 0; a < MK_SYMS; ++a) {
        uint64_t acc = 0;
        for (int b = 0; b < MK_SYMS; ++b) {
            int lo = a < b ? a : b, hi = a < b ? b : a;   /* same value for (a,b) and (b,a) */
            double e = x[lo] * K[lo][hi] * x[hi] * scale;
            uint64_t ei = (uint64_t)(e + 0.5);
            if (ei == 0) ei = 1;
            acc += ei;
            M->rowcum[a][b] = acc;
        }
        M->rowsum[a] = acc;
        total += acc;
        M->cum[a] = total;
    }
}

static inline int mk_pick(const uint64_t* cum, uint64_t total, uint64_t x) {
    uint64_t target = (uint64_t)(((unsigned __int128)x * total) >> 64);   /* [0, total) */
    int lo = 0, hi = MK_SYMS - 1;
    while (lo < hi) {                      /* first index with cum > target */
        int mid = (lo + hi) >> 1;
        if (cum[mid] > target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static inline int mk_stationary(const mk_model* M, uint64_t x) {
    return mk_pick(M->cum, M->cum[MK_SYMS - 1], x);
}

static inline int mk_step(const mk_model* M, int a, uint64_t x) {
    return mk_pick(M->rowcum[a], M->rowsum[a], x);
}

static void* markov_job(void* arg) {
    job_t* j = (job_t*)arg;
    const mk_model* M = (const mk_model*)j->model;
    const uint64_t startkey = j->key ^ 0x43484E4B53545254ULL;
    for (uint64_t c = j->lo; c < j->hi; ++c) {
        uint64_t b0 = c * MK_CHUNK;
        uint64_t b1 = b0 + MK_CHUNK < j->n ? b0 + MK_CHUNK : j->n;
        int s = mk_stationary(M, draw_k(startkey, c));
        j->out[b0] = M->byte_of[s];
        for (uint64_t i = b0 + 1; i < b1; ++i) {
            s = mk_step(M, s, draw_k(j->key, i));
            j->out[i] = M->byte_of[s];
        }
    }
    return NULL;
}

int synth_markov95(uint8_t* out, uint64_t n, uint64_t seed, uint64_t stream, int threads) {
    if (!out) return -1;
    mk_model* M = (mk_model*)malloc(sizeof(mk_model));
    if (!M) return -1;
    mk_build(M, seed);
    uint64_t chunks = (n + MK_CHUNK - 1) / MK_CHUNK;
    int nt = clamp_threads(threads, chunks);
    job_t jobs[256];
    uint64_t key = stream_key(seed, stream);
    for (int t = 0; t < nt; ++t) {
        jobs[t].out = out; jobs[t].n = n; jobs[t].key = key; jobs[t].model = M;
        jobs[t].lo = chunks * (uint64_t)t / (uint64_t)nt;
        jobs[t].hi = chunks * (uint64_t)(t + 1) / (uint64_t)nt;
    }
    run_jobs(markov_job, jobs, nt);
    free(M);
    return 0;
}

/* The model's stationary weights, indexed by byte (0 outside 0x20..0x7E). */
void synth_markov95_weights(uint64_t* w256, uint64_t seed) {
    mk_model* M = (mk_model*)malloc(sizeof(mk_model));
    memset(w256, 0, 256 * sizeof(uint64_t));
    if (!M) return;
    mk_build(M, seed);
    for (int s = 0; s < MK_SYMS; ++s) w256[M->byte_of[s]] = M->rowsum[s];
    free(M);
}
