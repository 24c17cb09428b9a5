/*
 * sm.h - exact string matching on the GPU: the SIMD-naive counting search
 * of Tarhio, Holub and Giaquinta, "Technology Beats Algorithms (in Exact
 * String Matching)", re-designed for NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 1): count or report every location of a pattern p of length
 * m in a text t of length n. Symbols are bytes compared as unsigned values
 * (0x00 and 0xFF are ordinary symbols). Locations are 0-based start
 * positions s with t[s .. s+m-1] = p[0 .. m-1]; the paper counts from 1.
 * Overlapping occurrences all count (Algorithm 1 tests every start).
 *
 * Conventions shared by every call
 *   - Pointers prefixed d_ are device memory of the context's device, h_ are
 *     host memory. The caller owns all of them; the library never frees or
 *     keeps them after the call returns, and never reads t outside
 *     t[0 .. n-1]. The text may start at any byte address and have any length.
 *   - Calls that take a stream are asynchronous: they validate arguments on
 *     the host, enqueue work on the stream and return. Results are valid once
 *     the stream has reached that point. Device-side conditions found later
 *     (a truncated report, an expired bounded wait) are recorded in the
 *     context and returned by sm_sync().
 *   - A context owns the library's device workspace. Work from one context
 *     must be ordered on one stream at a time; give each concurrent stream
 *     its own context.
 *   - Calls return a status and never abort or throw. sm_last_error() gives a
 *     message for the last failure on the calling thread.
 *   - m = 0 is SM_EINVAL. m > n (including n = 0) is not an error: the count
 *     is 0, no kernel is launched, and *d_count is still written.
 *   - m may be at most SM_MAX_M.
 */
#ifndef SM_H
#define SM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t / CUstream); NULL is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st* sm_stream_t;

typedef enum sm_status {
    SM_OK = 0,
    SM_EINVAL = 1,    /* invalid argument; nothing was enqueued */
    SM_ENOMEM = 2,    /* workspace allocation failed */
    SM_ECUDA = 3,     /* a CUDA runtime call failed (message in sm_last_error) */
    SM_ETRUNC = 4,    /* from sm_sync: a report had more matches than its capacity */
    SM_ETIMEOUT = 5,  /* from sm_sync: a bounded device wait expired */
    SM_ENOTSUP = 6    /* request outside what this build supports */
} sm_status;

#define SM_MAX_M 4096u          /* longest pattern accepted */
#define SM_TILE_STARTS 16384u   /* start positions per scan tile */

typedef struct sm_ctx sm_ctx;

/* Create a context on CUDA device `device`; *ctx is NULL on failure. */
sm_status sm_create(sm_ctx** ctx, int device);

/* Release a context and its workspace. Waits for the device first. NULL is a no-op. */
void sm_destroy(sm_ctx* ctx);

/* Message for the last failing call on this thread ("" if none). Owned by the library. */
const char* sm_last_error(void);

/* Name of a status code. */
const char* sm_status_string(sm_status s);

/*
 * Wait until `stream` has finished the work enqueued so far, then return and
 * clear the context's deferred device status: SM_ETRUNC if a report since the
 * last sm_sync had count > cap, SM_ETIMEOUT if a bounded device wait expired,
 * SM_ECUDA if the stream reported an error, else SM_OK.
 */
sm_status sm_sync(sm_ctx* ctx, sm_stream_t stream);

/*
 * Tuning and test knobs of a context (they change speed, never results).
 *   SM_KNOB_STAGES        shared-memory pipeline depth of the scan, 2..8 (default 4)
 *   SM_KNOB_GRID          scan CTAs; 0 = one wave of resident CTAs (default)
 *   SM_KNOB_SPIN_NS       limit of every bounded device wait, ns (default 1e9)
 *   SM_KNOB_TEST_SKIP_COPY  test hook: 1 = the scan never starts the copy of
 *                         tile 0, so its bounded wait expires and sm_sync
 *                         reports SM_ETIMEOUT (results are then invalid)
 */
typedef enum sm_knob {
    SM_KNOB_STAGES = 1,
    SM_KNOB_GRID = 2,
    SM_KNOB_SPIN_NS = 3,
    SM_KNOB_TEST_SKIP_COPY = 4
} sm_knob;
sm_status sm_set_knob(sm_ctx* ctx, sm_knob knob, int64_t value);

/* ------------------------------------------------------------------ a1 */
/*
 * Byte histogram of the text: d_hist256[c] = #{x < n : t[x] = c}, c = 0..255.
 * Sec. 2.2 orders compares by symbol frequency; this build takes the
 * frequencies from the searched text itself (computed once per text).
 *   d_text     n bytes, device, any alignment (NULL allowed only when n = 0)
 *   d_hist256  256 x uint64, device; overwritten (not accumulated)
 */
sm_status sm_histogram(sm_ctx* ctx, const uint8_t* d_text, uint64_t n,
                       uint64_t* d_hist256, sm_stream_t stream);

/* ------------------------------------------------------------------ a2 */
/*
 * Rarest-first comparison order (Sec. 2.2, Algorithm 3): h_pi[0..m-1] is the
 * permutation of pattern positions 0..m-1 sorted by h_hist256[p[q]]
 * ascending, equal frequencies in ascending position. O(m log m) on the host
 * (Sec. 2.2); synchronous, needs no context or device.
 *   h_pat      m bytes, host;  h_hist256  256 x uint64, host;
 *   h_pi       m x uint32, host, written.
 */
sm_status sm_order(const uint8_t* h_pat, uint32_t m, const uint64_t* h_hist256,
                   uint32_t* h_pi);

/*
 * Fixed comparison orders of Sec. 2.4, needing no frequencies:
 *   mode SM_ORDER_H : pi_h  = p[1], p[m], p[4], p[7], ..., p[3], p[6], ...,
 *                             p[2], p[5], ... (1-based, each position once)
 *   mode SM_ORDER_HS: pi_hs = pi_h applied to the positions that do not hold
 *                             a space (0x20), then the space positions in
 *                             ascending order.
 * Synchronous, host only. h_pat may be NULL for SM_ORDER_H.
 */
#define SM_ORDER_H 1
#define SM_ORDER_HS 2
sm_status sm_order_fixed(const uint8_t* h_pat, uint32_t m, int mode, uint32_t* h_pi);

/* ------------------------------------------------------------ a3 - a7 */
/*
 * Options for one search; NULL selects the defaults.
 *   peel       peeling factor r of Sec. 2.3 (Algorithm 4): the first r
 *              compares of every group of starts run without the zero test.
 *              0 = choose automatically (then the peeled compares are chosen
 *              by a cost model, see below). Clamped to m. Does not change the
 *              result.
 *   flags      SM_SEARCH_BYTES: compare bytes even when coded compares
 *              apply. Other bits must be 0.
 *   h_hist256  optional host histogram of THIS text (from sm_histogram). When
 *              given, it selects the automatic peel and the peeled compares,
 *              allows a faster compare when the text has no byte >= 0x80,
 *              compares 1-bit codes (32 starts per 32-bit word) when the text
 *              has at most two distinct symbols and 2-bit codes (16 starts
 *              per word) when it has at most four, and returns a zero count
 *              without scanning when some pattern symbol never occurs in the
 *              text. A histogram that does not belong to the text gives
 *              undefined results.
 */
#define SM_SEARCH_BYTES 1u
typedef struct sm_search_opts {
    uint32_t peel;
    uint32_t flags;
    const uint64_t* h_hist256;
} sm_search_opts;

/*
 * Count the occurrences of p in t (Algorithms 2-4): *d_count =
 * #{s in [0, n-m] : t[s .. s+m-1] = p}. The scan compares pattern positions
 * in the order h_pi (NULL = positions 0..m-1), which never changes the count.
 *   d_text   n bytes, device, any alignment
 *   h_pat    m bytes, host;  h_pi  m x uint32 permutation of 0..m-1 or NULL
 *   d_count  1 x uint64, device; overwritten
 * Errors: SM_EINVAL for NULL pointers, m = 0, m > SM_MAX_M or an h_pi that
 * is not a permutation.
 */
sm_status sm_count(sm_ctx* ctx, const uint8_t* d_text, uint64_t n,
                   const uint8_t* h_pat, uint32_t m, const uint32_t* h_pi,
                   uint64_t* d_count, sm_stream_t stream);

sm_status sm_count_ex(sm_ctx* ctx, const uint8_t* d_text, uint64_t n,
                      const uint8_t* h_pat, uint32_t m, const uint32_t* h_pi,
                      const sm_search_opts* opts, uint64_t* d_count, sm_stream_t stream);

/* ------------------------------------------------------------------ a8 */
/*
 * Report the occurrences (the reporting version of Algorithm 1, Sec. 2.1):
 * d_pos[0 .. min(count, cap)-1] receives the first min(count, cap) start
 * positions in ascending order and *d_count the full count. When
 * count > cap the extra positions are dropped and the next sm_sync on this
 * context returns SM_ETRUNC.
 *   d_pos  cap x uint64, device (may be NULL when cap = 0)
 * Other arguments and errors as sm_count.
 */
sm_status sm_report(sm_ctx* ctx, const uint8_t* d_text, uint64_t n,
                    const uint8_t* h_pat, uint32_t m, const uint32_t* h_pi,
                    uint64_t* d_pos, uint64_t cap, uint64_t* d_count, sm_stream_t stream);

sm_status sm_report_ex(sm_ctx* ctx, const uint8_t* d_text, uint64_t n,
                       const uint8_t* h_pat, uint32_t m, const uint32_t* h_pi,
                       const sm_search_opts* opts, uint64_t* d_pos, uint64_t cap,
                       uint64_t* d_count, sm_stream_t stream);

/* ------------------------------------------------------------- tuning */
/*
 * Autotuned plans of the single-pattern scan. Sec. 2.3 leaves the peeling
 * factor r to tuning (and Sec. 3 finds r = 2, 3 or 5 best per text type); on
 * the GPU the pipeline depth and the CTAs per SM also change the speed
 * (never the result). A context keeps one plan per bucket:
 *   m bucket      ceil(log2 m): 0 for m = 1, 1 for m = 2, 2 for m = 3..4, ...,
 *                 12 for m = 2049..4096
 *   sigma bucket  from the text's histogram: 0 at most two distinct symbols
 *                 (1-bit codes), 1 at most four (2-bit codes), then by the
 *                 effective alphabet 1 / sum(p_c^2) of the symbol
 *                 frequencies p_c: 2 below 12, 3 below 48, 4 from 48 up
 * sm_count_ex and sm_report_ex use the plan of their bucket when they are
 * given the text's histogram; fields left 0 keep the defaults, and an
 * explicit opts->peel or sm_set_knob(SM_KNOB_STAGES / SM_KNOB_GRID) wins
 * over the plan. The environment variables SM_R (peel), SM_STAGES and
 * SM_CTAS_PER_SM override plans and defaults for every search of the
 * process. Tile size (SM_TILE_STARTS) and starts per thread (64) are fixed
 * by the kernels' warp geometry: sm_create fails with SM_ENOTSUP when
 * SM_TILE or SM_STARTS asks for other values.
 */
#define SM_TUNE_M_BUCKETS 13u
#define SM_TUNE_SIGMA_BUCKETS 5u
typedef struct sm_tuning {
    uint32_t peel;          /* peeling factor r, 0 = the planner's choice */
    uint32_t stages;        /* pipeline depth 2..8, 0 = default */
    uint32_t ctas_per_sm;   /* resident scan CTAs per SM to launch, 0 = all that fit */
    float ms;               /* sm_tune_search: mean time per search of the plan */
} sm_tuning;

/* The buckets of a search for a pattern of length m (1..SM_MAX_M) in a text
 * with host histogram h_hist256. Host only. */
sm_status sm_tune_bucket(const uint64_t* h_hist256, uint32_t m, uint32_t* m_bucket, uint32_t* sigma_bucket);

/* Install (NULL: clear) or read the plan of a bucket of this context. */
sm_status sm_tune_set(sm_ctx* ctx, uint32_t m_bucket, uint32_t sigma_bucket, const sm_tuning* plan);
sm_status sm_tune_get(sm_ctx* ctx, uint32_t m_bucket, uint32_t sigma_bucket, sm_tuning* plan);

/*
 * Time sm_count_ex over npats patterns (packed in h_pats by h_pat_off, all
 * in one m bucket) in the text d_text (n bytes, device) with histogram
 * h_hist256, each in rarest-first order: the current plan of their bucket,
 * then by coordinate descent the peel (planner, 1..8), the stages (2, 3, 4,
 * 6) and the CTAs per SM (1, 2, 3) -- a candidate replaces the best only
 * when it is at least 2 % faster on each half of the patterns (the first
 * npats / 2 and the rest), so that a plan that helps a few patterns and
 * hurts the others of the bucket is not kept. Each plan: one warm-up pass,
 * then per half reps timed passes (the fastest counts). Installs the best
 * plan for the bucket and returns it in *best. Synchronous on `stream`;
 * allocates one count word.
 */
sm_status sm_tune_search(sm_ctx* ctx, const uint8_t* d_text, uint64_t n, const uint64_t* h_hist256,
                         const uint8_t* h_pats, const int64_t* h_pat_off, uint32_t npats, uint32_t reps,
                         sm_tuning* best, sm_stream_t stream);

/* ---------------------------------------------------------------- batch */
/*
 * Batched counting: many patterns of uneven lengths over many texts, with
 * each staged text tile tested against every pattern of its text so that the
 * patterns share one pass over the text (Algorithms 2-4 applied to a batch).
 *
 * Texts are packed back to back in d_texts: text x is
 * d_texts[h_text_off[x] .. h_text_off[x+1]), h_text_off[0] = 0, offsets
 * non-decreasing. Patterns are packed in h_pats the same way with h_pat_off
 * (npats + 1 entries, lengths 1..SM_MAX_M); pattern k is searched in text
 * h_pat_text[k] (any order).
 *
 * sm_batch_create plans the batch (synchronous on `stream`, allocates device
 * tables): per-text byte histograms, each pattern's rarest-first order under
 * its own text's frequencies (Sec. 2.2) and peel factor (Sec. 2.3), 2-bit
 * codes for texts of at most four symbols; patterns with a symbol that
 * never occurs in their text, or longer than it, are not scanned (count 0). The plan keeps d_texts and reads it at every count.
 * sm_batch_count enqueues one memset and one persistent kernel that writes
 * d_counts[k] (int64, npats entries) for every pattern; it allocates nothing
 * and may be captured in a CUDA graph. sm_batch_destroy waits for the device
 * and frees the plan.
 */
typedef struct sm_batch sm_batch;
sm_status sm_batch_create(sm_ctx* ctx, const uint8_t* d_texts, const int64_t* h_text_off, uint32_t ntexts,
                          const uint8_t* h_pats, const int64_t* h_pat_off, const int32_t* h_pat_text,
                          uint32_t npats, sm_batch** out, sm_stream_t stream);
sm_status sm_batch_count(sm_batch* batch, int64_t* d_counts, sm_stream_t stream);
/*
 * sm_batch_report: the reporting version (Sec. 2.1) for the whole batch.
 * Writes d_counts[k] as sm_batch_count does and the positions of pattern k,
 * ascending, to d_pos[d_pos_off[k] .. d_pos_off[k+1]) (device int64 offsets,
 * npats + 1 entries; at most that many positions, the count stays the full
 * count, and a pattern with more sets SM_ETRUNC for sm_sync). Three passes
 * over the texts' tiles: counts per (pattern, tile), their prefix sums per
 * pattern, then the writes of the tiles with matches. The first call
 * allocates 12 bytes per (pattern, tile) in the batch; later calls allocate
 * nothing.
 */
sm_status sm_batch_report(sm_batch* batch, int64_t* d_counts, uint64_t* d_pos, const int64_t* d_pos_off,
                          sm_stream_t stream);
/*
 * sm_batch_tune: the batch's autotuner. Times sm_batch_count (one warm-up
 * and reps timed launches per plan, on `stream`) for the plan it has and for
 * every plan over a grid of parameters: the text frequency below which a
 * pattern's rarest symbol sends it to the candidate path {2, 4, 8, 16, 32 %},
 * the fewest such patterns of a text that use that path {4, 16, 64}, and the
 * pipeline stages {2, 3, 4}. Keeps the fastest plan and reports it in *best
 * (ms = its time per count). Synchronous; allocates a counts buffer and the
 * trial plans' tables. Counts never depend on the plan.
 */
typedef struct sm_batch_tuning {
    float cand_freq;
    uint32_t cand_min;
    uint32_t stages;     /* 0: the context's default */
    float ms;
} sm_batch_tuning;
sm_status sm_batch_tune(sm_batch* batch, uint32_t reps, sm_batch_tuning* best, sm_stream_t stream);
void sm_batch_destroy(sm_batch* batch);

/*
 * One-shot form with device-resident metadata: d_text_off, d_pat_off,
 * d_pat_text and the packed patterns d_pats are device arrays laid out as
 * above. Counts go to d_counts. When d_pos is not NULL, the positions of
 * pattern k are written in ascending order to d_pos[d_pos_off[k] ..
 * d_pos_off[k+1]) (at most that many; the count stays the full count), as
 * sm_batch_report does. Synchronous: copies the metadata to the host, plans,
 * runs and waits.
 */
sm_status sm_count_batch(sm_ctx* ctx, const uint8_t* d_texts, const int64_t* d_text_off, uint32_t ntexts,
                         const uint8_t* d_pats, const int64_t* d_pat_off, const int32_t* d_pat_text,
                         uint32_t npats, int64_t* d_counts, uint64_t* d_pos, const int64_t* d_pos_off,
                         sm_stream_t stream);

/* ------------------------------------------------------------- serving */
/*
 * Continuous batching over one device-resident text (the serving loop's
 * core). The text is cut into chunks of chunk_bytes (a multiple of
 * SM_TILE_STARTS); a step scans one chunk for every active query in one
 * batched launch, so concurrent queries share each pass over the text. A
 * query admitted before a step on chunk c and stepped on every chunk once
 * (in any order, e.g. c, c+1, ..., c-1) has its full count in its counter.
 *
 *   sm_stepper_create  d_text (n bytes, device, resident for the stepper's
 *                      life), queries up to max_m bytes, h_hist256 = the
 *                      text's histogram (orders, Sec. 2.2)
 *   sm_stepper_admit   describe query qid (pattern copied; m <= max_m)
 *   sm_stepper_step    add the counts of chunk `chunk` for the queries
 *                      h_qids[0..nq) into d_counts[qid] (int64, device;
 *                      the caller zeroes a counter before its first step).
 *                      Asynchronous on `stream`; allocates nothing once its
 *                      two table buffers have grown to the batch size.
 *   sm_stepper_steps   the same for several chunks in one launch: query
 *                      h_qids[i] is scanned on chunks chunk, chunk + 1, ...
 *                      (wrapping) for h_nchunks[i] of them (all queries: 1
 *                      when h_nchunks is NULL; at most the chunk count).
 *   sm_stepper_retire  forget qid.
 *   sm_stepper_report  report nq patterns (h_pats / h_pat_off packed as for
 *                      sm_batch_create) over the whole text in one batched
 *                      report: counts to d_counts[0..nq), ascending positions
 *                      of pattern k to d_pos[h_pos_off[k] .. h_pos_off[k+1])
 *                      (host offsets; at most that many, SM_ETRUNC beyond).
 *                      Asynchronous on `stream`; it first waits for the
 *                      previous report of this stepper, whose tables and
 *                      per-(pattern, tile) counters (12 bytes each) it reuses.
 * One stepper is driven from one host thread and one stream.
 */
typedef struct sm_stepper sm_stepper;
sm_status sm_stepper_create(sm_ctx* ctx, const uint8_t* d_text, uint64_t n, uint64_t chunk_bytes,
                            uint32_t max_m, const uint64_t* h_hist256, sm_stepper** out);
uint32_t sm_stepper_chunks(const sm_stepper* stepper);
sm_status sm_stepper_admit(sm_stepper* stepper, uint32_t qid, const uint8_t* h_pat, uint32_t m);
sm_status sm_stepper_step(sm_stepper* stepper, const uint32_t* h_qids, uint32_t nq, uint32_t chunk,
                          int64_t* d_counts, sm_stream_t stream);
sm_status sm_stepper_steps(sm_stepper* stepper, const uint32_t* h_qids, const uint32_t* h_nchunks, uint32_t nq,
                           uint32_t chunk, int64_t* d_counts, sm_stream_t stream);
sm_status sm_stepper_retire(sm_stepper* stepper, uint32_t qid);
sm_status sm_stepper_report(sm_stepper* stepper, const uint8_t* h_pats, const int64_t* h_pat_off, uint32_t nq,
                            const int64_t* h_pos_off, uint64_t* d_pos, int64_t* d_counts, sm_stream_t stream);
void sm_stepper_destroy(sm_stepper* stepper);

/* ------------------------------------------------------- no allocation */
/*
 * sm_report_noalloc - the report of sm_report for callers that must not
 * allocate device memory. The paper has no counterpart; this entry point
 * exists for how the library is embedded, not for the method.
 *
 * Who needs it: code that is only handed input and output buffers and may
 * not call cudaMalloc -- a plug-in inside a host framework whose caching
 * allocator already reserves the device memory (a foreign cudaMalloc can fail
 * or fragment that pool), a service that forbids allocation after start-up
 * because cudaMalloc and cudaFree can block and synchronize the device, or a
 * caller with no context object to keep. sm_report keeps its scratch in an
 * sm_ctx allocated by sm_create; this call keeps it in one fixed device array
 * that the library defines (about 528 KiB), which every GPU that loads the
 * library holds until the process exits.
 *
 * Behaviour: as sm_report with default options (identity order when h_pi is
 * NULL), on the calling thread's current device and the given stream; it
 * allocates nothing (no cudaMalloc, cudaFree or other allocating routine).
 * The first call on a device also looks up the array's device address and
 * sets kernel attributes; make that first call before any stream capture.
 * All calls share the one array and it keeps the previous call's contents
 * (the call clears what must start at zero): calls whose work overlaps on
 * the GPU -- other streams, other host threads -- race and give wrong
 * results, so order them. There is no context to hold a deferred status,
 * so device-side conditions show in *d_count once the stream has reached
 * the call:
 *   - *d_count > cap: more than cap matches; the first cap positions and the
 *     full count were written (what sm_sync reports as SM_ETRUNC);
 *   - *d_count == SM_NOALLOC_TIMEOUT (UINT64_MAX): a bounded device wait
 *     expired (a tile copy did not arrive within 1 s); the positions are
 *     invalid (what sm_sync reports as SM_ETIMEOUT).
 * Errors: SM_EINVAL as sm_report, and when the text has more than
 * SM_NOALLOC_MAX_STARTS start positions (n - m + 1), the number of tiles
 * whose per-tile counts the array holds; SM_ECUDA when a CUDA call fails
 * (a failed first-call set-up is tried again by the next call).
 */
#define SM_NOALLOC_MAX_STARTS 268435456ull   /* 16384 tiles x 16384 starts */
#define SM_NOALLOC_TIMEOUT 0xFFFFFFFFFFFFFFFFull
sm_status sm_report_noalloc(const uint8_t* d_text, uint64_t n, const uint8_t* h_pat, uint32_t m,
                            const uint32_t* h_pi, uint64_t* d_pos, uint64_t cap,
                            uint64_t* d_count, sm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SM_H */
