/*
 * oasm.h -- C ABI of the GB300 (sm_103a) Online Approximate String Matching
 * library: a dictionary of patterns is searched, within a Levenshtein
 * threshold, over many byte streams, and overlapping "shadow hits" are
 * removed on the fly by the greedy priority filter of OASM.
 *
 * Method: A. Cinti, F. M. Bianchi, A. Martino, A. Rizzi, "A novel algorithm
 * for online inexact string matching and its FPGA implementation",
 * arXiv:1712.03560.
 *   - distance: Levenshtein, unit costs (Sec. 3, Eq. 1)
 *   - hit:      substring t(i;l), l in [l_p-K, l_p+K], lev(p, t(i;l)) = k <= K
 *               (Sec. 3, Eq. 2)
 *   - filter:   priority rules R1-R3 (Sec. 4.1), validation counters and
 *               Eq. 3 (Sec. 4.2), Algorithm 1 (Sec. 4)
 *   - many patterns on one stream: MOASM, one independent filter per pattern
 *               (Sec. 6.4)
 *
 * Conventions for every call:
 *   - Return value: OASM_OK (0) or a negative OASM_E* code; oasm_last_error()
 *     gives a one-line message for the most recent failure on a context.
 *   - Pointers are host pointers unless the name says "device".  The library
 *     never keeps a caller's host pointer after a call returns.
 *   - A context is not thread-safe: calls on one context must not overlap.
 *   - All device work of a context runs on one CUDA stream (its own, or the
 *     one given in oasm_config.cuda_stream).
 */
#ifndef OASM_H
#define OASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define OASM_OK 0
#define OASM_EINVAL (-1)   /* bad argument (pattern length, threshold, id, ...) */
#define OASM_ENOMEM (-2)   /* device or pinned host memory could not be had */
#define OASM_EBUSY (-3)    /* no free stream slot */
#define OASM_ETRUNC (-4)   /* more hits are ready than `cap`; the rest stay queued */
#define OASM_ETIMEOUT (-5) /* a bounded wait on the device ran out */
#define OASM_ECUDA (-6)    /* a CUDA call failed; see oasm_last_error() */
#define OASM_ESTATE (-7)   /* call not valid in the object's current state */

/* ---- limits ----------------------------------------------------------- */
#define OASM_MAX_PATTERN_LEN 128 /* 1 <= l_p <= 128 (four 32-bit words) */
#define OASM_MAX_K 15            /* 0 <= K < l_p and K <= 15 */

typedef struct oasm_ctx oasm_ctx;

/* ---- priority rules (Sec. 4.1-4.2) -------------------------------------
 * The paper's printed rules leave some choices open; each is a field here.
 * The defaults reproduce the worked example of Sec. 4.2 exactly.          */
enum {
    /* R2/R3: a hit of the same priority as the pending one replaces it ... */
    OASM_REPLACE_CONTAINED = 0, /* ... iff it lies inside it (default) */
    OASM_REPLACE_SAME_END = 1,  /* ... iff it ends at the same symbol */
    OASM_REPLACE_NEVER = 2      /* never: the first encountered wins (R2 as worded) */
};
enum {
    OASM_ORDER_PER_START_LENGTH = 0, /* every length of a start, ascending (Alg. 1) */
    OASM_ORDER_PER_START_BEST = 1    /* only the best (min k, then shortest) of a start */
};
enum {
    OASM_ACC_SUM = 0, /* acc sums the lengths of the occurrences added (Alg. 1) */
    OASM_ACC_LAST = 1 /* acc is the length of the last occurrence added (Eq. 3 text) */
};
enum {
    OASM_CMP_GT = 0, /* lower level kept iff r(k) - acc > l(k) (Eq. 3) */
    OASM_CMP_GE = 1  /* ... iff r(k) - acc >= l(k) */
};
enum {
    OASM_OUT_FILTERED = 0, /* OASM output: the filtered occurrence set S */
    OASM_OUT_ENDS = 1,     /* Less Naive (Sec. 5.1): every end e with
                              min_i lev(p, t[i..e]) <= K, unfiltered */
    OASM_OUT_ALL_HITS = 2  /* every hit of Eq. 2, unfiltered */
};

typedef struct {
    int32_t replace; /* OASM_REPLACE_* */
    int32_t order;   /* OASM_ORDER_* */
    int32_t acc;     /* OASM_ACC_* */
    int32_t cmp;     /* OASM_CMP_* */
    int32_t output;  /* OASM_OUT_* */
} oasm_rules;

typedef struct {
    int32_t device;            /* CUDA device ordinal (default 0) */
    uint32_t max_streams;      /* stream slots (default 64) */
    uint64_t mem_budget;       /* device bytes for per-stream state; 0 = no limit
                                  beyond what the device has */
    uint32_t region_bytes;     /* scan tile length in text symbols; 0 = automatic */
    uint32_t tile_warps;       /* warps per scan block, 0..16; 0 = automatic */
    int32_t timing;            /* 1: time each kernel class with CUDA events */
    uint32_t flush_timeout_ms; /* bound on every host wait (default 600000) */
    void *cuda_stream;         /* cudaStream_t to run on; NULL = library-owned */
    int32_t myers_only;        /* 1: every pattern on the Myers/Hyyro bit-vector scan;
                                  0 (default): one-word patterns with K <= 2 use the
                                  automaton scan where a class has >= 32 of them */
    int32_t graphs;            /* 1: launch each step as a captured CUDA graph,
                                  updated in place while its shape repeats */
    uint32_t groups_per_warp;  /* lane groups (32 patterns each) a scan warp runs
                                  together in one-word classes: 1 or 2; 0 = the
                                  tuned value (1 until oasm_autotune picks) */
    uint32_t prefilter_piece;  /* 0 (default): every pattern on the forward scan.
                                  4..128: a pattern whose K + 1 pieces are all at
                                  least this many symbols long (l_p / (K + 1) >= it)
                                  is searched by the exact piece filter instead:
                                  exact matches of its pieces propose the ends that
                                  verification checks (pays off where pieces rarely
                                  match at random, e.g. long byte signatures).
                                  1: automatic, per pattern, from the expected
                                  number of piece matches (symbol frequencies of
                                  the pattern set) against the scan's cost */
    int32_t full_words;        /* 0 (default): classes of 32 or more patterns longer
                                  than 32 symbols run the cut-off scan: only each
                                  pattern's first 32 rows are computed while none
                                  of them comes within K of a match (the rows below
                                  then all exceed K), every word otherwise; same
                                  output.  1: every word at every step */
    int32_t record_order;      /* filtered output only; same records either way.
                                  0 (default): automatic.  1: the filter writes
                                  each piece's records at a position fixed by the
                                  piece's place among the sorted hits, and a scan
                                  of the counts gives the output offsets
                                  (canonical order without a record sort; needs
                                  K_max + 1 spare record slots per stream and
                                  pattern).  2: records are appended as decided,
                                  then sorted.  Automatic takes 1 unless a step's
                                  streams x patterns x (K_max + 1) exceeds its hit
                                  capacity */
} oasm_config;

/* One occurrence added to S (or, for the raw outputs, one hit/end). */
typedef struct {
    uint32_t pattern_id; /* index into the pattern array given to oasm_create */
    uint32_t k;          /* lev(p, t(start; len)) = its priority level */
    uint64_t start;      /* i: 0-based position in the stream */
    uint32_t len;        /* l; the end position is start + len - 1 */
    uint32_t stream_id;  /* the stream it was found on */
    uint64_t decided_at; /* stream position at which Algorithm 1 added it to S
                            (for the raw outputs: its end position) */
} oasm_hit;

typedef struct {
    uint64_t steps;          /* batched steps run */
    uint64_t launches;       /* kernels launched by the library */
    uint64_t text_bytes;     /* new stream bytes processed */
    uint64_t cells;          /* Sellers cells: sum over patterns of l_p x bytes */
    uint64_t word_steps;     /* bit-vector word updates of the forward scan */
    uint64_t candidates;     /* ends with min distance <= K (forward scan) */
    uint64_t hits;           /* hits of Eq. 2 handed to the filter */
    uint64_t kept;           /* records emitted */
    uint64_t reruns;         /* steps re-run after a buffer grew */
    double scan_ms;          /* with timing=1: forward scan kernels */
    double verify_ms;        /* anchored verification */
    double order_ms;         /* radix sort of hits */
    double filter_ms;        /* filter, finalize and tail update */
    double copy_ms;          /* staging copies into the device text arena */
    double step_ms;          /* whole steps, first to last kernel */
    uint64_t scan_launches;  /* forward-scan kernel launches */
    uint64_t graph_builds;   /* step graphs instantiated (cfg.graphs = 1) */
    double prefilter_ms;     /* with timing=1: the piece filter (cfg.prefilter_piece) */
    uint64_t prefilter_candidates; /* distinct (pattern, end) pairs it proposed */
    double host_plan_ms;     /* host time: planning a step and preparing its upload */
    double host_launch_ms;   /* host time: enqueueing (or capturing and updating) a step */
    double host_wait_ms;     /* host time waiting for the device to finish a step */
    double host_post_ms;     /* host time after a step: counters, records into the
                                stream queues, stream bookkeeping */
    uint64_t buffer_grows;   /* device or pinned host buffers reallocated larger
                                (each a cudaMalloc or cudaHostAlloc on the call's
                                path, and a free of the old buffer) */
    double host_copy_ms;     /* host time waiting for the copy of a step's records
                                to pinned host memory (the copy runs beside the
                                caller; this is what remained when the records were
                                first needed) */
    uint64_t record_bytes;   /* bytes of records copied to the host */
} oasm_stats;

/* Fills *cfg / *rules with the defaults described above. */
int oasm_config_default(oasm_config *cfg);
int oasm_rules_default(oasm_rules *rules);

/* Creates a context for a dictionary of n_pat patterns (MOASM, Sec. 6.4).
 *   pat[j]  host pointer to pattern j (len[j] bytes, any byte values 0-255;
 *           no symbol is reserved, unlike the FPGA's $1/$2 of Sec. 7)
 *   len[j]  l_p, 1..OASM_MAX_PATTERN_LEN
 *   k[j]    threshold K of pattern j: 0 <= K < l_p (Sec. 6.3) and <= OASM_MAX_K
 *   rules   NULL for the defaults
 *   cfg     NULL for the defaults
 *   out     receives the context
 * The patterns are copied; the caller's arrays may be freed on return.
 * Errors: OASM_EINVAL (n_pat == 0, bad length or threshold), OASM_ENOMEM,
 * OASM_ECUDA.  On error *out is NULL and nothing is leaked. */
int oasm_create(const uint8_t *const *pat, const uint32_t *len, const uint32_t *k,
                uint32_t n_pat, const oasm_rules *rules, const oasm_config *cfg,
                oasm_ctx **out);

/* Integer edit costs (a variant outside the paper, whose Eq. 1 has unit
 * costs).  Each replaces one of Eq. 1's three +1 terms:
 *   sub  a pattern symbol aligned with a different text symbol (the +delta)
 *   ins  a text symbol aligned with no pattern symbol
 *   del  a pattern symbol aligned with no text symbol
 * Every cost is an integer in 1..255.  A hit of Eq. 2 is then a substring
 * whose weighted distance k is <= K; k is its priority level in Algorithm 1,
 * which runs unchanged.  Because every cost is >= 1, a hit still has a length
 * in [l_p - K, l_p + K]. */
typedef struct {
    uint32_t sub;
    uint32_t ins;
    uint32_t del;
} oasm_costs;

/* oasm_create with integer edit costs.  costs == NULL is oasm_create (unit
 * costs, the bit-parallel scan).  A non-NULL costs, even (1, 1, 1), selects
 * the weighted path: a wave-front (anti-diagonal) dynamic program over each
 * pattern's rows in place of the bit-parallel scan, a plain dynamic program
 * in place of the bit-parallel verification, the same filter.  The piece
 * filter and the automaton classes do not apply to it (cfg->prefilter_piece
 * and cfg->myers_only are ignored).  Errors as oasm_create, plus OASM_EINVAL
 * for a cost outside 1..255. */
int oasm_create_weighted(const uint8_t *const *pat, const uint32_t *len, const uint32_t *k,
                         uint32_t n_pat, const oasm_rules *rules, const oasm_costs *costs,
                         const oasm_config *cfg, oasm_ctx **out);

/* Frees every host and device resource of the context.  Safe on NULL and on a
 * context whose creation failed half way.  Waits (bounded) for device work. */
int oasm_destroy(oasm_ctx *ctx);

/* Opens a stream: a text t that arrives in pieces (Sec. 4: "continuous
 * stream of symbols").  Each stream has its own position, its own pending
 * filter window per pattern and the last l_p + 3K - 1 symbols it saw, all
 * resident on the device.  Admission is by device memory: OASM_ENOMEM when
 * the stream's state does not fit mem_budget, OASM_EBUSY when all
 * max_streams slots are taken. */
int oasm_open_stream(oasm_ctx *ctx, uint32_t *sid);

/* Closes a stream and frees its slot; undelivered hits are dropped. */
int oasm_close_stream(oasm_ctx *ctx, uint32_t sid);

/* Batched forms for serving loops with many streams.
 *   oasm_open_streams  opens up to n streams into sids[]; *n_opened receives
 *                      how many (fewer than n when slots or the memory budget
 *                      run out; that is not an error)
 *   oasm_end_streams / oasm_close_streams  as the single-stream calls, for
 *                      each id; stop at the first invalid id (OASM_EINVAL) */
int oasm_open_streams(oasm_ctx *ctx, uint32_t n, uint32_t *sids, uint32_t *n_opened);
int oasm_end_streams(oasm_ctx *ctx, uint32_t n, const uint32_t *sids);
int oasm_close_streams(oasm_ctx *ctx, uint32_t n, const uint32_t *sids);

/* Appends n bytes (host memory) to stream sid.  The bytes are copied into
 * pinned staging memory; `chunk` may be reused when the call returns.  If
 * they lie inside a range registered with oasm_register_host, they are not
 * copied: the step reads them where they are (zero copy), and `chunk` must
 * stay unchanged until a step has consumed them.  No device work is started
 * until oasm_step / oasm_flush. */
int oasm_feed(oasm_ctx *ctx, uint32_t sid, const uint8_t *chunk, size_t n);

/* Appends many packets to many streams in one call (the ingest of a serving
 * loop): packet j is buf[off[j] .. off[j] + len[j]) for stream sid[j], all
 * host memory.  Packets of one stream are appended in array order.  The
 * bytes are copied into pinned staging before the call returns.
 * OASM_EINVAL if any sid is not open (nothing is appended then). */
int oasm_feed_many(oasm_ctx *ctx, uint32_t n, const uint32_t *sid, const uint8_t *buf,
                   const uint64_t *off, const uint32_t *len);

/* Appends n bytes that are already in device memory.  The buffer is NOT
 * copied at this call: it must stay valid and unchanged until the next
 * oasm_step or oasm_flush that processes this stream has returned. */
int oasm_feed_device(oasm_ctx *ctx, uint32_t sid, const uint8_t *dchunk, size_t n);

/* Marks the end of stream sid: at the next step its last symbols are matched
 * with truncated lengths (i + l <= n) and every pending window is decided. */
int oasm_end_stream(oasm_ctx *ctx, uint32_t sid);

/* Runs one batched step over every stream with pending input or a pending
 * end: one pass of the whole device path (stage, bit-parallel scan, anchored
 * verification, ordering, filter, emit).  Returns when the step has finished
 * on the device and its decided hits are queued on their streams. */
int oasm_step(oasm_ctx *ctx);

/* oasm_step in two halves, so that host work can overlap the device.
 * oasm_step_begin plans one step over the input pending now and launches it;
 * it returns once the step's host bytes are on the device (the host may then
 * feed more input, open and end streams, and drain earlier hits).
 * oasm_step_end waits for that step and starts the copy of its decided hits
 * to the host; it returns without waiting for that copy, which then overlaps
 * whatever the caller does next (a next oasm_step_begin included).  The hits
 * reach their streams' queues at the first call that reads a queue
 * (oasm_flush, oasm_drain, oasm_ready, oasm_close_stream, oasm_save_stream)
 * or at the next step's end, whichever comes first; the order of each
 * stream's hits is unchanged.  A call that needs a quiet context (oasm_step,
 * oasm_flush, oasm_close_stream, oasm_save_stream, oasm_restore_stream,
 * oasm_autotune) finishes a step in flight first.  oasm_step_begin returns
 * OASM_ESTATE if a step is already in flight; with no pending input it
 * launches nothing and oasm_step_end is a no-op.  Pipelined use: begin step
 * i, drain and close step i - 1's streams, open and feed step i + 1's, end
 * step i. */
int oasm_step_begin(oasm_ctx *ctx);
int oasm_step_end(oasm_ctx *ctx);

/* Returns the hits of stream sid decided so far and not yet returned, in
 * canonical order (pattern_id, decided_at, k).  If the stream has input or
 * an end that no step has processed yet, a step is run first.  With
 * end_of_stream != 0 the stream is ended first (as oasm_end_stream) and,
 * once drained, rewinds to position 0 and can be fed again.
 *   out/cap   caller's array of cap records; *n_out receives the count
 * OASM_ETRUNC when more than cap records are ready: the first cap are
 * returned, the rest stay queued for the next call. */
int oasm_flush(oasm_ctx *ctx, uint32_t sid, int end_of_stream, oasm_hit *out, size_t cap,
               size_t *n_out);

/* Returns the queued hits of every stream at once: streams in id order,
 * each stream's hits in canonical order (pattern_id, decided_at, k); no step
 * is run.  OASM_ETRUNC when more than cap are queued (the rest stay). */
int oasm_drain(oasm_ctx *ctx, oasm_hit *out, size_t cap, size_t *n_out);

/* Which patterns a context created with cfg.prefilter_piece = prefilter_piece
 * would search with the piece filter (on_filter[p] = 1) rather than the
 * forward scan (0): the same rule oasm_create applies.  Host-only (no device
 * is touched).  OASM_EINVAL for patterns or a setting oasm_create would
 * reject. */
int oasm_piece_filter_choice(const uint8_t *const *pat, const uint32_t *len, const uint32_t *k,
                             uint32_t n_pat, uint32_t prefilter_piece, uint8_t *on_filter);

/* Zero-copy input.  oasm_register_host pins [ptr, ptr + bytes) of the
 * caller's host memory and maps it for the device.  An oasm_feed_many whose
 * packets all lie in one registered range then copies nothing at the call:
 * the step's gather kernel reads the packets straight from host memory over
 * the CPU-GPU link.  The caller must not modify or free the range while
 * input from it is waiting for a step.  oasm_unregister_host (ptr as
 * registered) returns OASM_ESTATE while such input is pending; ranges still
 * registered are released by oasm_destroy.  OASM_EINVAL for an overlapping
 * range, OASM_ECUDA when the driver refuses the registration. */
int oasm_register_host(oasm_ctx *ctx, const void *ptr, size_t bytes);
int oasm_unregister_host(oasm_ctx *ctx, const void *ptr);

/* ------------------------------------------------------------ serving loop
 * A packet trace for oasm_replay: packet q arrives at t[q] seconds (sorted)
 * on external stream stream[q] (< n_streams) with payload
 * payload[off[q] .. off[q] + len[q]); last[q] = 1 marks the last packet of
 * its stream.  All arrays are the caller's and are only read. */
typedef struct {
    const double *t;
    const uint32_t *stream;
    const uint64_t *off;
    const uint32_t *len;
    const uint8_t *last;
    const uint8_t *payload;
    uint64_t n_packets;
    uint32_t n_streams;
    uint32_t reserved;
} oasm_trace;

typedef struct {
    uint64_t steps;              /* batched steps run */
    uint64_t packets;            /* packets fed */
    uint64_t bytes;              /* payload bytes fed */
    uint64_t kept;               /* hits drained (all streams) */
    uint64_t n_out;              /* hits written to the caller's array */
    uint64_t streams_admitted;
    uint64_t max_waiting_streams;
    double wall_s;               /* first arrival window to last drain */
    double step_s_sum;           /* feed + step + drain, summed over steps */
    double step_s_max;
    /* what the library did during the replay (oasm_stats differences), and
       during its slowest step (launch to results queued): steps re-run after
       a buffer grew, step graphs instantiated, buffers reallocated */
    uint64_t reruns;
    uint64_t graph_builds;
    uint64_t buffer_grows;
    uint64_t slowest_step;       /* index of the step that took step_s_max */
    uint64_t slowest_bytes;      /* its payload bytes */
    uint64_t slowest_reruns;
    uint64_t slowest_graph_builds;
    uint64_t slowest_buffer_grows;
} oasm_replay_stats;

/* Online matching of many concurrent streams (the paper's online setting,
 * Sec. 1 and 4, served with continuous batching): replays the trace against
 * the clock (realtime != 0; otherwise every packet is present at the start).
 * Each step takes the packets that have arrived, up to max_batch_bytes (at
 * least one packet), feeds them with oasm_feed_many, runs oasm_step and
 * drains every stream's decided hits with oasm_drain.  A stream is opened at
 * its first packet when a slot and the memory budget allow it, else it waits
 * (FIFO, packets held in order); the step that ingests its last packet ends
 * it, and its slot is freed after the drain.
 *   done_at   optional [n_packets]: seconds from the start of the replay to
 *             the end of the step that matched each packet
 *   out/out_cap  optional array for the drained hits, stream_id = the
 *             external stream id; more than out_cap hits: OASM_ETRUNC (the
 *             replay still completes and rs->kept counts them all)
 * OASM_EINVAL for a malformed trace, OASM_ENOMEM when no stream fits the
 * memory budget, and every error of the calls it makes. */
int oasm_replay(oasm_ctx *ctx, const oasm_trace *trace, int realtime, uint64_t max_batch_bytes,
                double *done_at, oasm_hit *out, size_t out_cap, oasm_replay_stats *rs);

/* The serving loop's calls into the library, as a table: oasm_replay binds
 * it to a context (handle = the oasm_ctx*, each entry the library call of the
 * same name).  oasm_replay_ops runs the same loop through any table with the
 * same contracts, e.g. a fake library on the host that refuses admission or
 * fails a step, to test the scheduler without a device.  Every entry but
 * get_stats (may be NULL: no library counters in the stats) must be set;
 * OASM_EINVAL otherwise. */
typedef struct {
    void *handle;
    int (*open_streams)(void *handle, uint32_t n, uint32_t *sids, uint32_t *n_opened);
    int (*feed_many)(void *handle, uint32_t n, const uint32_t *sid, const uint8_t *buf,
                     const uint64_t *off, const uint32_t *len);
    int (*end_streams)(void *handle, uint32_t n, const uint32_t *sids);
    int (*close_streams)(void *handle, uint32_t n, const uint32_t *sids);
    int (*step_begin)(void *handle);
    int (*step_end)(void *handle);
    int (*ready)(void *handle, uint32_t sid, size_t *n);
    int (*drain)(void *handle, oasm_hit *out, size_t cap, size_t *n_out);
    int (*get_stats)(void *handle, oasm_stats *st);
} oasm_serve_ops;

int oasm_replay_ops(const oasm_serve_ops *ops, const oasm_trace *trace, int realtime,
                    uint64_t max_batch_bytes, double *done_at, oasm_hit *out, size_t out_cap,
                    oasm_replay_stats *rs);

/* Number of decided hits of stream sid queued and not yet returned by
 * oasm_flush (no device work is started).  sid = OASM_ALL_STREAMS gives the
 * total over every open stream: the size oasm_drain needs. */
#define OASM_ALL_STREAMS 0xFFFFFFFFu
int oasm_ready(oasm_ctx *ctx, uint32_t sid, size_t *n);

/* ---- stream checkpoint / migration -------------------------------------
 * A stream's whole matching state is small and explicit: its position, the
 * last T symbols it saw and, per pattern, the pending window (Algorithm 1's
 * mem rows).  It can be saved and restored into a stream of another context
 * built from the same patterns, thresholds and rules (checked by a
 * fingerprint), e.g. to move a stream to another GPU or process.  Hits
 * already decided are not part of the state: flush them first.
 *   oasm_stream_state_size  bytes of a saved state for this context
 *   oasm_save_stream        OASM_ESTATE if the stream has input no step has
 *                           processed yet; OASM_ETRUNC if cap is too small
 *   oasm_restore_stream     into an open stream with no pending input;
 *                           OASM_EINVAL if the state does not fit the context */
int oasm_stream_state_size(oasm_ctx *ctx, size_t *bytes);
int oasm_save_stream(oasm_ctx *ctx, uint32_t sid, void *buf, size_t cap, size_t *n);
int oasm_restore_stream(oasm_ctx *ctx, uint32_t sid, const void *buf, size_t n);

/* Cumulative counters and (with cfg.timing = 1) per-kernel-class times. */
int oasm_get_stats(oasm_ctx *ctx, oasm_stats *st);
int oasm_reset_stats(oasm_ctx *ctx);

/* The cudaStream_t the context runs on (for timing with CUDA events). */
void *oasm_cuda_stream(oasm_ctx *ctx);

/* Message of the most recent failure on ctx ("" if none); ctx may be NULL
 * for failures of oasm_create. */
const char *oasm_last_error(oasm_ctx *ctx);

/* Static text for an OASM_E* code. */
const char *oasm_strerror(int code);

/* ---- autotuning ------------------------------------------------------
 * Times the forward scan over a sample of `n` device-resident symbols for a
 * set of tile shapes (warps per block, tile length) and keeps the fastest
 * per word-count class for this context.  `report` (may be NULL) receives a
 * one-line JSON summary of at most `report_cap` bytes. */
int oasm_autotune(oasm_ctx *ctx, const uint8_t *dsample, size_t n, char *report,
                  size_t report_cap);

/* ---- measurement utility (no counterpart in the paper) ------------------
 * Integer issue rate of `device` on a synthetic kernel (no memory traffic):
 * each thread runs eight independent chains of 15 integer operations per
 * step.  `mix` selects the operations:
 *   0  ALU pipe only: 3-input logic ops, adds, funnel shifts, byte permutes
 *   1  integer multiply-adds with register operands (the FMA pipe)
 *   2  one 32-bit column step of the forward scan in the scan's own PTX
 *      forms (7 logic ops, 1 add, 2 shifts and the table address as
 *      multiply-adds, 2 high-word multiply-adds for the score, 1 or for the
 *      candidate flag, 1 byte permute), spread over the ALU and FMA pipes as
 *      in the scan
 *   3  three pairs of cells of the weighted wave-front (oasm_create_weighted)
 *      in its forms, 5 operations a pair: a logic op, a 16x2 three-way
 *      minimum, a multiply-add, two 16x2 fused add-minimums
 * *ops_per_s receives integer operations per second over the whole GPU (best
 * of five timed launches), *ms (may be NULL) the time of that launch.
 * OASM_EINVAL for another mix or a NULL ops_per_s.
 * oasm_measure_int_peak is mix 2: the measured roofline peak of the scan. */
int oasm_measure_int_peak_mix(int device, int mix, double *ops_per_s, double *ms);
int oasm_measure_int_peak(int device, double *ops_per_s, double *ms);

/* Launch settings of one scan class, as oasm_autotune picks them (no paper
 * passage: the batched form's tile shapes).  A context has one class per
 * (word count, algorithm); oasm_get_tuning lists them in the context's
 * order, so a caller can store them (keyed by the GPU and the pattern set)
 * and give them back to a new context with the same patterns through
 * oasm_set_tuning instead of timing again. */
typedef struct {
    int32_t words;           /* W: 32-bit words per lane (rows per lane, weighted path) */
    int32_t algo;            /* 0 Myers/Hyyro, 1 + K automaton for K <= 2, 8 weighted,
                                9 Myers/Hyyro with the cut-off (multi-word classes) */
    int32_t groups_per_warp; /* 1, or 2 (one-word dictionary classes) */
    int32_t warps;           /* warps per scan block, 1..16 */
    int32_t chunk;           /* TMA text buffer bytes: 512, 1024 or 2048 */
    float region_scale;      /* region length factor, (0, 16] */
} oasm_tuning;

/* Copies the context's class settings into out[0..cap) and their count into
 * *n.  OASM_ETRUNC when cap < *n (nothing is copied then). */
int oasm_get_tuning(oasm_ctx *ctx, oasm_tuning *out, uint32_t cap, uint32_t *n);

/* Sets every class's launch settings; t[i] must name class i's words and
 * algo (as oasm_get_tuning lists them) and n the class count.  OASM_EINVAL
 * for a mismatch or a value out of range (nothing is changed then).
 * Finishes a step in flight first. */
int oasm_set_tuning(oasm_ctx *ctx, const oasm_tuning *t, uint32_t n);

/* Failure-detection self-test of the bounded device waits (no paper
 * passage: the library's own failure detection).  Launches one block that
 * polls an mbarrier at most spin_limit times; with arrive = 0 nothing
 * completes the barrier, the poll runs out and the call returns
 * OASM_ETIMEOUT, exactly as a scan whose copy never lands reports
 * OASM_ETIMEOUT.  With arrive = 1 the barrier completes: OASM_OK.  No fault,
 * trap or hang is involved; the device stays usable.  Errors: OASM_EINVAL
 * (spin_limit == 0), OASM_ENOMEM, OASM_ECUDA. */
int oasm_selftest_wait(int device, uint32_t spin_limit, int arrive);

/* ---- search without device allocation (no counterpart in the paper) ----
 * For callers that cannot call cudaMalloc: code running inside a framework
 * whose caching allocator already holds the device's memory, code under a
 * hard per-process memory cap, or code that must not trigger the implicit
 * synchronisation an allocation can cause.  This call uses only the
 * caller's buffers and one fixed scratch array in the library's device image
 * (OASM_NOALLOC_SCRATCH_BYTES, held by every GPU that loads the library until
 * the process exits).
 *
 * It reports the "Less Naive" ends of Sec. 5.1 -- every end position e where
 * min over starts i of lev(p, t[i..e]) <= K -- for up to
 * OASM_NOALLOC_MAX_PATTERNS patterns over one device-resident text, with no
 * priority filter and no streaming state: the same end positions and
 * distances as an OASM_OUT_ENDS context, in no particular order.
 *   pat/len/k  as for oasm_create (1..OASM_NOALLOC_MAX_PATTERNS patterns)
 *   d_text, n  the text, device memory
 *   d_out, cap caller's device array of cap oasm_end records
 *   n_found    host pointer: the number of ends found (may exceed cap)
 *   cuda_stream the stream to run on (NULL: the legacy default stream)
 * Runs on the calling thread's current CUDA device and returns after the
 * work has finished.  The first call on a device looks up the scratch
 * array's device address; make that first call before any stream capture.
 * Calls that overlap on the GPU share the scratch array and race.
 * Returns OASM_OK, OASM_ETRUNC (more than cap ends: the first cap written,
 * in no particular order), OASM_EINVAL (bad argument, or more than
 * OASM_NOALLOC_MAX_PATTERNS patterns), OASM_ECUDA. */
#define OASM_NOALLOC_MAX_PATTERNS 64
#define OASM_NOALLOC_SCRATCH_BYTES (1024 + OASM_NOALLOC_MAX_PATTERNS * 4096)

typedef struct {
    uint32_t pattern_id;
    uint32_t k;   /* min over starts of the distance of a substring ending here */
    uint64_t end; /* 0-based end position */
} oasm_end;

int oasm_scan_ends_noalloc(const uint8_t *const *pat, const uint32_t *len, const uint32_t *k,
                           uint32_t n_pat, const uint8_t *d_text, uint64_t n, oasm_end *d_out,
                           uint64_t cap, uint64_t *n_found, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* OASM_H */
