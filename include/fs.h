/*
 * fs.h -- C ABI of the GB300 factorization-set library.
 *
 * The library computes over the factorization set of an element n in the
 * (not necessarily minimal, coprime or ordered) generators g_1..g_d:
 *
 *     Z(n, (g_1..g_d)) = { (a_1..a_d) in N^d : a_1 g_1 + ... + a_d g_d = n }   (Sec. 1)
 *
 * by the paper's method: the lexicographic order on N^d is cut into bounded
 * slices [lo, hi) (Sec. 4), and each GPU worker walks the candidates of its
 * slice with the nextCandidate successor (Algorithm 3.1).  The consumers are
 * the ones Sec. 2 lists -- count, predicate, save (enumerate) -- plus length
 * statistics of sum a_i.  All arithmetic is exact integer arithmetic.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - n      : the element, 0 <= n, and n + max(g) <= 2^31 - 1 (else FS_E_OVERFLOW).
 * - gens   : HOST pointer to d generators, each >= 1 (a zero generator makes Z
 *            infinite: FS_E_INVAL).  Repeats, any order, common divisors are
 *            allowed (Sec. 1 footnote).  The array is read before the call
 *            returns and never kept.
 * - d      : 1 <= d <= FS_MAX_D (else FS_E_INVAL).
 * - stream : a cudaStream_t (NULL = the legacy default stream).  All device
 *            work is enqueued on it, in stream order with the caller's work.
 * - device memory passed in (dev_buf, hist_dev, dev_count) is owned by the
 *   caller and must be resident on the current device; the library never
 *   frees it.  The library owns only its internal scratch: one arena per
 *   (device, stream handle), allocated on first use, grown when needed and
 *   kept until process exit.  Calls on one stream are ordered by it; calls on
 *   different streams use different arenas and may overlap on the GPU.  (A
 *   stream handle that is destroyed and later reused by the runtime inherits
 *   its arena: destroy a stream only after its library work has completed.)
 *   Host-side entry is serialised by the library.
 * - synchronous calls (no _async suffix) return after their host outputs are
 *   written; they synchronise `stream`.
 * - errors: every call returns an fs_status and writes its outputs only on
 *   FS_OK, except FS_E_CAPACITY (see fs_enumerate).  fs_last_error() gives a
 *   one-line description of the last failure on the calling thread.
 * - there is no CPU fallback: without a usable CUDA device every call that
 *   needs the GPU returns FS_E_CUDA.
 */
#ifndef FS_H
#define FS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FS_MAX_D 16

typedef enum fs_status {
    FS_OK = 0,
    FS_E_INVAL = 1,     /* bad argument: d out of range, zero generator, n < 0, NULL pointer */
    FS_E_OVERFLOW = 2,  /* n + max g >= 2^31, int16 output that cannot hold a coordinate,
                           planner leaf-count tables ((P-1) (n+1) uint64, P = max(d,3) - 2)
                           above 8 GiB, or a query whose count may reach 2^63: the bound
                           (n + sum g)^(d-1) / ((d-1)! prod g) over the d-1 largest
                           generators is checked before any work */
    FS_E_CAPACITY = 3,  /* enumerate: more factorizations than `cap` */
    FS_E_NOMEM = 4,     /* device scratch allocation failed */
    FS_E_CUDA = 5,      /* a CUDA runtime call or kernel launch failed; no device */
    FS_E_TIMEOUT = 6,   /* a bounded device-side wait ran out */
    FS_E_NOTIMPL = 7    /* combination not implemented */
} fs_status;

/* Walk method.  PLAIN runs Algorithm 3.1 exactly: one nextCandidate step per
 * candidate, consumers filter by wasValid (Sec. 3.2-3.3).  PAIR resolves the
 * last two coordinates of every prefix in closed form: the congruence step of
 * Sec. 3.2.4 taken all the way, i.e. jump straight to the first valid value of
 * a_{d-1} and count / list the valid values of (a_{d-1}, a_d) without visiting
 * the invalid candidates between them.  Both give identical results. */
typedef enum fs_method {
    FS_METHOD_AUTO = 0,
    FS_METHOD_PLAIN = 1,
    FS_METHOD_PAIR = 2,
    /* TRIPLE: the paper's dynamic behaviour of Sec. 6.1 for the last three
     * coordinates: for every residual p <= n, tables hold the number of
     * factorizations of p over the last three generators and their length
     * range, so the walk visits only the prefixes of the first d-3
     * coordinates.  Count and min / max length only (fs_count, fs_length_stats
     * without a histogram, fs_slice_counts); needs d >= 4.  AUTO uses it for
     * those when it applies, PAIR otherwise. */
    FS_METHOD_TRIPLE = 3,
    /* QUAD: the same with tables over the last four coordinates (each table
     * entry one more strided sum of the trailing-three table), so the walk
     * visits only the prefixes of the first d-4; needs d >= 5 and n < 2^22.
     * AUTO prefers it to TRIPLE where it applies. */
    FS_METHOD_QUAD = 4
} fs_method;

typedef struct fs_config {
    int32_t method;        /* fs_method; AUTO = QUAD, else TRIPLE where they apply, else PAIR */
    int32_t keep_order;    /* 1: walk the generators in the caller's order.  0 (default):
                              walk them in descending order, which visits the fewest
                              prefixes; the result is the same set (Z does not depend on
                              the order of the generators, Sec. 1). */
    int64_t slices;        /* number of lexicographic slices [lo,hi) (Sec. 4), of equal leaf
                              counts; 0 = auto: the planner picks the count from the
                              leaves and the grid, and the last sixteenth of the slices
                              hold a sixteenth of a regular slice each (short slices at
                              the end of the walks' queue) */
    int32_t block_threads; /* threads per block; 0 = auto */
    int32_t blocks_per_sm; /* resident blocks per SM for the persistent grid; 0 = auto */
    int32_t walk;          /* fs_walk: how the order-free consumers (count, length
                              statistics, predicate, trailing-table walks) take the leaves
                              of a group of sibling runs; the results are the same */
    int32_t reserved;      /* must be 0 */
} fs_config;

/* fs_config.walk.  PACKED: each run's full 32-leaf steps with the warp on one
 * run, then the runs' remainders packed into shared steps.  LANES: lane j walks
 * sibling run j on its own, the warp stepping until the longest run is done.
 * AUTO (0): per group of sibling runs, whichever costs fewer issue slots by
 * the walk's own estimate. */
typedef enum { FS_WALK_AUTO = 0, FS_WALK_PACKED = 1, FS_WALK_LANES = 2 } fs_walk;

/* Fills *cfg with the defaults (all zero = automatic). */
void fs_config_default(fs_config* cfg);

/* Length statistics of the lengths sum_i a_i over Z (the count is exact).
 * min_len / max_len are valid only when count > 0 (both 0 otherwise). */
typedef struct fs_len_summary {
    uint64_t count;
    uint32_t min_len;
    uint32_t max_len;
} fs_len_summary;

/* A linear predicate on one factorization a, the "predicate" consumer of
 * Sec. 2.  With s = sum_i w[i] a_i (w in the caller's generator order, int64
 * arithmetic):
 *   modulus > 0 : true iff s == c (mod modulus), both sides reduced to [0, modulus)
 *   op == 0     : true iff s == c
 *   op == 1     : true iff s <= c
 *   op == 2     : true iff s >= c
 * Entries w[d..FS_MAX_D-1] are ignored.  |w[i]| <= 2^20 and |c| <= 2^60. */
typedef struct fs_predicate {
    int32_t w[FS_MAX_D];
    int64_t c;
    int32_t op;
    uint32_t modulus;
} fs_predicate;

/* --- library -------------------------------------------------------------- */

/* Static string naming a status code. */
const char* fs_status_string(int status);
/* Library version: major * 10000 + minor * 100 + patch. */
int fs_version(void);
/* One-line description of the last failed call on this thread ("" if none).
 * The pointer stays valid until the next call on this thread. */
const char* fs_last_error(void);

/* --- the four consumers (Sec. 2), synchronous ----------------------------- */

/* |Z(n, g)| -> *out_count (host).  The count consumer of Sec. 2 over all slices. */
fs_status fs_count(int64_t n, const uint32_t* gens, int d, uint64_t* out_count, void* stream);

/* Count, min and max of sum a_i -> *out (host).  hist_dev (nullable) is a
 * DEVICE array of floor(n / min g) + 1 uint64 bins; bin l receives the number of
 * factorizations of length l (overwritten, not accumulated). */
fs_status fs_length_stats(int64_t n, const uint32_t* gens, int d, fs_len_summary* out,
                          uint64_t* hist_dev, void* stream);

/* *out_bool (host) = 1 iff some factorization satisfies *pred (the predicate
 * consumer of Sec. 2), else 0.  Workers stop early once one is found. */
fs_status fs_any(int64_t n, const uint32_t* gens, int d, const fs_predicate* pred,
                 int* out_bool, void* stream);

/* Materialise Z(n, g) (the save consumer of Sec. 2) into dev_buf: a DEVICE
 * buffer of `cap` rows, row-major [count][d] in the caller's generator order,
 * each coordinate an int32 (elem_bytes == 4) or int16 (elem_bytes == 2; needs
 * floor(n / min g) <= 32767, else FS_E_OVERFLOW).  dev_buf must be 16-byte
 * aligned.  Row order: lexicographically ascending in the walk order of the
 * generators (descending generators unless cfg->keep_order), deterministic;
 * with keep_order it is lex-ascending in the caller's order.  *out_count (host)
 * = |Z|.  If |Z| > cap: returns FS_E_CAPACITY with *out_count = |Z|; the first
 * cap rows are written, the rest dropped. */
fs_status fs_enumerate(int64_t n, const uint32_t* gens, int d, void* dev_buf, uint64_t cap,
                       int elem_bytes, uint64_t* out_count, void* stream);

/* --- the same with an explicit configuration (cfg may be NULL) ----------- */

fs_status fs_count_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                      uint64_t* out_count, void* stream);
fs_status fs_length_stats_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                             fs_len_summary* out, uint64_t* hist_dev, void* stream);
fs_status fs_any_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                    const fs_predicate* pred, int* out_bool, void* stream);
fs_status fs_enumerate_ex(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                          void* dev_buf, uint64_t cap, int elem_bytes, uint64_t* out_count,
                          void* stream);

/* --- asynchronous forms: enqueue only, results stay on the device -------- */

/* Enqueues the count; *dev_count (DEVICE uint64) receives |Z| in stream order.
 * Returns after the launches; argument errors are reported synchronously. */
fs_status fs_count_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                         uint64_t* dev_count, void* stream);

/* Enqueues the length statistics (as fs_length_stats_ex): hist_dev (DEVICE,
 * nullable) receives the histogram, out_dev (DEVICE, nullable) three uint64:
 * the count, the minimum and the maximum of sum a_i (both 0 when the count is
 * 0), in stream order.  Argument errors are reported synchronously. */
fs_status fs_length_stats_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                                uint64_t* hist_dev, uint64_t* out_dev, void* stream);

/* Enqueues the enumeration into dev_buf (as fs_enumerate); *dev_count (DEVICE
 * uint64) receives |Z|.  Rows past cap are dropped; the caller compares
 * *dev_count with cap. */
fs_status fs_enumerate_async(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                             void* dev_buf, uint64_t cap, int elem_bytes, uint64_t* dev_count,
                             void* stream);

/* --- resumable cursor and streamed enumerate ------------------------------ */

/* A stream's next value depends only on its current state (Sec. 2), which is
 * why the paper's enumeration has no memory limit on the result set (Table 1
 * caption): it never needs the whole set at once.  A cursor gives the same
 * property to the library's ordered output (the row order of fs_enumerate_ex
 * for the same cfg): it plans the query and counts every slice once, then
 * produces any window of rows on demand, so a result larger than device
 * memory can be consumed piece by piece, and a consumer can stop and resume
 * at any row.
 *
 * fs_cursor_create: plans and counts (synchronises `stream` once); the cursor
 *   owns a small device allocation (the query's tables, slice states and
 *   offsets; not the rows).  elem_bytes as fs_enumerate.  PAIR walk only
 *   (FS_E_NOTIMPL for cfg->method PLAIN, TRIPLE or QUAD).
 * fs_cursor_count: |Z| (host).  fs_cursor_tell: the next row to be produced.
 * fs_cursor_slices: the number of slices the rows are cut into (host); a
 *   window touches only the slices that hold its rows.
 * fs_cursor_seek: continue from any row 0 <= row <= |Z| (FS_E_INVAL beyond).
 * fs_cursor_next: enqueues on `stream` the rows [pos, pos + m) into dev_buf
 *   (DEVICE, 16-byte aligned, room for cap rows of d elements), m = min(cap,
 *   |Z| - pos), sets *rows = m (host, known at return) and advances pos by m;
 *   m = 0 at the end.  Rows are written in stream order; calls on one cursor
 *   share its device counters, so order them on one stream (or by events).
 * fs_cursor_destroy: waits for the device and frees the cursor. */
typedef struct fs_cursor fs_cursor;
fs_status fs_cursor_create(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                           int elem_bytes, void* stream, fs_cursor** out);
fs_status fs_cursor_count(const fs_cursor* c, uint64_t* total);
fs_status fs_cursor_tell(const fs_cursor* c, uint64_t* row);
fs_status fs_cursor_slices(const fs_cursor* c, uint64_t* slices);
fs_status fs_cursor_seek(fs_cursor* c, uint64_t row);
fs_status fs_cursor_next(fs_cursor* c, void* dev_buf, uint64_t cap, uint64_t* rows, void* stream);
fs_status fs_cursor_destroy(fs_cursor* c);

/* fs_enumerate into HOST memory: the same rows and return values as
 * fs_enumerate_ex (FS_E_CAPACITY with the first cap rows written when |Z| >
 * cap), streamed through two device staging buffers of up to 128 MB: the walk
 * of one window overlaps the device-to-host copy of the previous one on a
 * second stream.  host_buf (HOST, cap rows of d elements) should be pinned
 * (cudaHostAlloc) for full bandwidth; pageable memory works but copies
 * synchronously.  Synchronous: returns after every row is in host_buf.
 * PAIR walk only, as the cursor. */
fs_status fs_enumerate_host(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                            void* host_buf, uint64_t cap, int elem_bytes, uint64_t* out_count,
                            void* stream);

/* --- slice planner (Sec. 4) ---------------------------------------------- */

/* The slices the walk uses.  A "leaf" is a prefix (a_1..a_{d-2}) of the walk
 * order with a_1 g_1 + ... + a_{d-2} g_{d-2} <= n; its two last coordinates are
 * what the PAIR method resolves in closed form.  The planner cuts the
 * lexicographic order of the leaves into `slices` ranges of (nearly) equal
 * leaf counts; slice s is the lex range [B_s, B_{s+1}) where B_s is the vector
 * (leaf, 0, 0) of its first leaf and B_slices = +infinity.
 *   order   (host, d int32, nullable): walk position k uses caller generator order[k]
 *   bounds  (host, (slices + 1) x d int32, nullable): row s = B_s in walk order;
 *           row `slices` is filled with -1 (= +infinity)
 *   leaves  (host, nullable): total number of leaves
 * For d <= 2 there is exactly one leaf (the whole set is one slice).
 * `slices` must be >= 1; slices beyond the number of leaves are empty. */
fs_status fs_plan(int64_t n, const uint32_t* gens, int d, const fs_config* cfg, int64_t slices,
                  int32_t* order, int32_t* bounds, uint64_t* leaves);

/* Per-slice counts of the slicing fs_plan describes (same cfg and slices):
 * counts (host, `slices` uint64) receives |Z intersected with slice s| from the
 * GPU walk (method per cfg). */
fs_status fs_slice_counts(int64_t n, const uint32_t* gens, int d, const fs_config* cfg,
                          int64_t slices, uint64_t* counts, void* stream);

/* --- batched queries ------------------------------------------------------ */

/* Many (n, g) queries of uneven size in one persistent walk launch.  Each
 * query is planned like a single call (its own leaf counts and pair tables)
 * and cut into slices of at most `target` leaves, where target is chosen on
 * the device from the batch's total so that the batch has about
 * `cfg->slices` work items (default: 8 per resident warp); persistent warps
 * pop the items from one device queue, so small and large queries share the
 * GPU without one launch per query. */
typedef struct fs_query {
    int64_t n;
    int32_t d;
    uint32_t gens[FS_MAX_D];
} fs_query;

typedef struct fs_result {
    uint64_t count;    /* |Z(n, g)| */
    uint32_t min_len;  /* min / max of sum a_i (FS_BATCH_LENGTHS, count > 0), else 0 */
    uint32_t max_len;
    int32_t status;    /* FS_OK, or why this query was rejected (FS_E_INVAL, FS_E_OVERFLOW) */
    int32_t pad;
} fs_result;

enum { FS_BATCH_COUNT = 0, FS_BATCH_LENGTHS = 1 };

typedef struct fs_batch fs_batch;  /* opaque; owns its device memory */

/* Validates and plans the queries (host pointer, nq >= 1), allocates the
 * batch's device memory on the current device and uploads the per-query
 * constants.  Invalid queries are kept with a non-OK status and skipped.
 * mode: FS_BATCH_COUNT or FS_BATCH_LENGTHS.  cfg (nullable): block_threads
 * (<= 256), blocks_per_sm, slices (= work items of the whole batch), method
 * (FS_METHOD_PAIR: every query walks its first d-2 levels; otherwise queries
 * with d >= 4 use the trailing-three tables of FS_METHOD_TRIPLE). */
fs_status fs_batch_create(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                          fs_batch** out);
/* Reusable batches for request loops: reserve once, then load / launch /
 * fetch / collect any number of times without allocating or synchronising.
 * fs_batch_table_bytes: host-only, the table bytes `queries` need.
 * fs_batch_reserve: room for max_queries queries and table_bytes of tables
 *   (allocates all device and pinned host memory of the batch).
 * fs_batch_load: plans the queries on the host and uploads their constants
 *   on `stream` from the batch's pinned buffer; FS_E_CAPACITY if they exceed
 *   the reservation.  Do not load again before that copy has run (order it on
 *   the same stream, or wait).
 * fs_batch_load_mode: the same, switching the batch to `mode` first (a batch
 *   reserved for FS_BATCH_LENGTHS can load count-only queries, which need no
 *   length tables and walk faster, and back); its launch shape is re-derived
 *   from the new mode's occupancy.
 * fs_batch_fetch: enqueues the copy of the results into pinned host memory.
 * fs_batch_collect: reads the fetched results; the caller waits for the
 *   stream (or an event recorded after fs_batch_fetch) first. */
fs_status fs_batch_table_bytes(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                               uint64_t* bytes);
fs_status fs_batch_reserve(int max_queries, uint64_t table_bytes, int mode, const fs_config* cfg,
                           fs_batch** out);
fs_status fs_batch_load(fs_batch* b, const fs_query* queries, int nq, void* stream);
fs_status fs_batch_load_mode(fs_batch* b, const fs_query* queries, int nq, int mode, void* stream);
fs_status fs_batch_fetch(fs_batch* b, void* stream);
fs_status fs_batch_collect(fs_batch* b, fs_result* results);
/* Enqueues one complete evaluation of the batch on `stream` (tables, plan,
 * walk); nothing is allocated and nothing synchronises, so it can be
 * repeated or captured into a CUDA graph. */
fs_status fs_batch_launch(fs_batch* b, void* stream);
/* Waits for `stream` and copies the results of the last launch into
 * results (host, nq entries).  FS_E_CUDA if the device reported a fault. */
fs_status fs_batch_results(fs_batch* b, fs_result* results, void* stream);
/* Frees the batch (waits for its work to finish). */
fs_status fs_batch_destroy(fs_batch* b);
/* create + launch + results + destroy. */
fs_status fs_batch_run(const fs_query* queries, int nq, int mode, const fs_config* cfg,
                       fs_result* results, void* stream);
/* Times the batch under a set of launch shapes and work-item counts and
 * returns the fastest configuration in *best (and its time in *best_ms,
 * nullable).  Every candidate computes the same exact results. */
fs_status fs_batch_autotune(const fs_query* queries, int nq, int mode, fs_config* best,
                            double* best_ms, void* stream);

/* Grows the scratch of `stream` on the current device to at least `bytes`
 * now (it is otherwise grown on demand, which waits for the stream's earlier
 * work and frees the old scratch).  Call before stream capture or before a
 * latency-sensitive loop. */
fs_status fs_reserve(uint64_t bytes, void* stream);

/* --- serving: a request loop with continuous batching -------------------- */

/* The paper evaluates one query at a time; this loop serves a stream of them.
 * fs_server_submit queues a request and returns at once.  A worker thread
 * admits the queued requests into `slots` reusable batches (fs_batch_reserve),
 * each on its own stream: a free slot takes up to max_batch queued requests
 * (when other batches are running it first lets the batch fill for up to
 * window_us), so requests that arrive while earlier ones are on the GPU are
 * batched and run concurrently with them.  The batch gives every request its
 * count and length range.  Two kinds of request then need device work of
 * their own (a "job"): an ENUMERATE (its rows, count * d * elem_bytes bytes)
 * and a LENGTHS request with hist = 1 (its histogram, (floor(n / min g) + 1)
 * * 8 bytes).  A COUNT or LENGTHS request whose walk would be long skips the
 * batch and runs as a job from the start (fs_count_async or
 * fs_length_stats_async on a job stream, its results read back from there):
 * one long walk would otherwise hold up the whole batch's answers.  "Long" is
 * an estimate of the leaves the batched walk visits, the lattice volume
 * prod_i (n + S) / ((i + 1) g_i) over the generators it walks (descending, all
 * but the last four for d >= 5, three for d = 4, two otherwise; S their sum),
 * against direct_leaves.  A job's bytes, exact, are admitted against the device memory
 * budget: larger than the whole budget -> FS_E_CAPACITY (count and range still
 * reported; so is a histogram whose PAIR walk would visit more than
 * hist_max_leaves leaves, |Z(n; g_1..g_{d-2}, gcd(g_{d-1}, g_d))| in descending
 * order); otherwise the job waits, in arrival order, until that many bytes
 * are free and one of `job_streams` job streams is idle, then runs there
 * (fs_enumerate_async or fs_length_stats_async), several jobs at once; its
 * output stays reserved until fs_server_release.  Results are exactly those of
 * the single-query calls.  A single query whose tables exceed table_bytes is
 * answered FS_E_CAPACITY.  Thread safety: submit / poll / release may be
 * called from any thread.  The server's batches own their memory and its jobs
 * run on streams of its own, so other library calls may run beside it. */
enum { FS_REQ_COUNT = 0, FS_REQ_LENGTHS = 1, FS_REQ_ENUMERATE = 2 };

typedef struct fs_server_config {
    uint64_t mem_budget_bytes;  /* device bytes for job outputs (rows, histograms); 0 = 1 GiB */
    uint64_t table_bytes;       /* table bytes per batch slot; 0 = 256 MiB */
    int32_t max_batch;          /* queries per batch; 0 = 512 */
    int32_t slots;              /* batches in flight; 0 = 3 */
    int32_t window_us;          /* fill window while the GPU is busy; 0 = 200 */
    int32_t job_streams;        /* jobs in flight (enumerates, histograms); 0 = 4 */
    uint64_t hist_max_leaves;   /* a histogram job whose walk visits more leaves is refused
                                   with FS_E_CAPACITY; 0 = 2^34 */
    uint64_t direct_leaves;     /* a COUNT or LENGTHS request whose walk is estimated to
                                   visit more leaves runs as a job of its own instead of in
                                   a batch; 0 = 2^24 */
} fs_server_config;

typedef struct fs_request {
    int64_t n;
    int32_t d;
    uint32_t gens[FS_MAX_D];  /* as fs_count */
    int32_t op;               /* FS_REQ_* */
    int32_t elem_bytes;       /* ENUMERATE: 2 (int16) or 4 (int32) */
    int32_t keep_order;       /* ENUMERATE: row order as fs_config.keep_order */
    int32_t hist;             /* LENGTHS: 1 = also the length histogram */
} fs_request;

typedef struct fs_response {
    uint64_t ticket;
    int32_t status;     /* FS_OK or the fs_status that rejected the request */
    int32_t op;
    uint64_t count;     /* |Z(n, g)| (also for a rejected job when it was counted) */
    uint32_t min_len;   /* LENGTHS and ENUMERATE: min / max of sum a_i when count > 0 */
    uint32_t max_len;
    void* rows;         /* FS_OK jobs, DEVICE memory owned by the server until
                           fs_server_release(ticket): ENUMERATE rows [count][d] (as
                           fs_enumerate_ex with the request's keep_order); LENGTHS with
                           hist: floor(n / min g) + 1 uint64 bins (as fs_length_stats) */
    double t_submit;    /* seconds since fs_server_create */
    double t_start;     /* when its batch was launched (the end of its queue wait);
                           a request run as a job from the start: its job's launch */
    double t_counted;   /* when its batch's results were collected (run as a job
                           from the start: when the job's results were) */
    double t_job;       /* when its job was launched (0: no job) */
    double t_done;      /* when its result was seen complete */
} fs_response;

typedef struct fs_server fs_server;  /* opaque */

/* Creates the server on the current device (cfg nullable = defaults) and
 * allocates everything it uses: the batch slots, their streams, the row
 * budget.  FS_E_NOMEM / FS_E_CUDA if that fails. */
fs_status fs_server_create(const fs_server_config* cfg, fs_server** out);
/* Queues *req (copied); *ticket (host) identifies its response.  FS_E_INVAL for
 * a bad op or elem_bytes; invalid queries are answered with their status. */
fs_status fs_server_submit(fs_server* s, const fs_request* req, uint64_t* ticket);
/* Moves up to `max` completed responses into out (host), oldest first;
 * *got = how many.  Waits up to wait_ms milliseconds when none is ready. */
fs_status fs_server_poll(fs_server* s, fs_response* out, int max, int* got, int wait_ms);
/* Returns the rows of an ENUMERATE response to the budget.  FS_E_INVAL if the
 * ticket holds no rows. */
fs_status fs_server_release(fs_server* s, uint64_t ticket);
/* Finishes every queued request, then frees the server; rows not yet released
 * are freed with it. */
fs_status fs_server_destroy(fs_server* s);

/* --- kernel timing ------------------------------------------------------ */

/* While enabled (on != 0), every kernel the library launches is bracketed by
 * CUDA events recorded on the stream it is launched on.  Used by benchmarks to
 * time individual kernels; off by default (no events recorded). */
void fs_profile_enable(int on);

/* Restricts the recording to the kernels timed under `name` (as
 * fs_profile_read reports them, e.g. "pair_enum"); NULL or "" records every
 * kernel again.  The string is copied.  Fewer events on the streams while a
 * benchmark times a whole step. */
void fs_profile_only(const char* name);

/* Collects the timings recorded since the last read (waits for their events):
 * up to `max` entries, one per kernel name, in first-launch order.  names
 * (host, max * 32 chars, NUL-terminated entries), launches (host, max) = how
 * many times that kernel ran, total_ms (host, max) = summed device time.
 * Returns the number of entries (-1 on a CUDA error). */
int fs_profile_read(char* names, uint64_t* launches, double* total_ms, int max);

/* --- allocation-free count ---------------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate device memory.  Examples: a framework
 * that owns all device memory through its own pool or budget, where a
 * cudaMalloc behind its back can fail or fragment the pool; a latency-critical
 * serving loop, where cudaMalloc / cudaFree synchronise the device and take
 * unbounded time; and code that has exhausted its memory quota.
 *
 * fs_count_noalloc enqueues the same work as fs_count_async (leaf-count and
 * pair tables, then the count walk) but takes its scratch from a static
 * device array of FS_NOALLOC_SCRATCH_BYTES inside the library instead of the
 * cudaMalloc'd arena.  It calls no cudaMalloc, cudaFree, cudaMallocHost or
 * other allocating routine.
 *   dev_count : DEVICE uint64 receiving |Z| in stream order (the caller's memory).
 *   n, gens, d, stream : as fs_count.
 * Limits and behaviour:
 * - a query whose tables need more than FS_NOALLOC_SCRATCH_BYTES
 *   ((d-3) (n+1) 8 bytes of leaf counts, plus up to 16 KB of pair table and
 *   256 KB of slice start states) is rejected with FS_E_OVERFLOW and a message
 *   naming the size, before any device work;
 * - the static array costs every device that loads this library
 *   FS_NOALLOC_SCRATCH_BYTES of memory until the process exits;
 * - the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture;
 * - every call on a device shares the one array and each call re-zeroes the
 *   counters it needs; calls whose work overlaps on the GPU (different
 *   streams, no ordering between them) race on the array and give wrong
 *   results: order them on one stream or with events;
 * - the looked-up address is kept per device for the life of the process and
 *   forgotten when a call on that device meets a CUDA error; after
 *   cudaDeviceReset on a device, no call of this library may be made on it
 *   again in this process (its cached arenas and addresses belong to the
 *   destroyed context). */
#define FS_NOALLOC_SCRATCH_BYTES (4u << 20)
fs_status fs_count_noalloc(int64_t n, const uint32_t* gens, int d, uint64_t* dev_count,
                           void* stream);

/* Number of successful device allocations (cudaMalloc) and pinned host
 * allocations (cudaMallocHost) this library has made in this process, on all
 * devices: lets a caller check that a call allocated nothing (for instance
 * fs_count_noalloc).  Null pointers are skipped.  Host-only, never fails. */
void fs_alloc_counts(uint64_t* device_allocs, uint64_t* pinned_host_allocs);

/* --- integer throughput probe ------------------------------------------- */

/* Measures the GPU-wide rate of one 32-bit integer instruction kind (0: add,
 * 1: three-input logic, 2: multiply-add) with 8 independent chains per
 * thread on every SM, timed with CUDA events on the legacy default stream:
 * the denominator of the roofline of the integer-bound walks.  *ops_per_s
 * (host) receives lane-operations per second.  Returns FS_OK, FS_E_INVAL for a
 * bad kind, FS_E_CUDA on a CUDA error. */
fs_status fs_probe_int_rate(int kind, uint32_t iters, double* ops_per_s);

/* --- host-side self test of the division helper ------------------------- */

/* Checks the library's division by an invariant divisor (Granlund-Montgomery
 * 1994, round-up multiplier) against C's / and % for divisor `div` and the
 * numerators x0, x0+1, ..., x0+count-1 (all < 2^31).  Runs on the host, needs
 * no GPU.  Returns the number of mismatches (0 = correct), -1 on bad input. */
int64_t fs_selftest_division(uint32_t div, uint32_t x0, uint32_t count);

/* The planner's split of `leaves` leaf ranks into `slices` slices (Sec. 4), as
 * the walks use it: starts (host, slices + 1 uint64) receives the first rank
 * of every slice and `leaves` last.  tail = 0: equal slices (explicit slice
 * counts); tail = 1: the split of a planner that picks its own slice count,
 * whose last sixteenth of the slices hold a sixteenth of a regular slice each.
 * Runs on the host, needs no GPU.  FS_E_INVAL for slices = 0 or a null starts. */
fs_status fs_selftest_split(uint64_t leaves, uint64_t slices, int tail, uint64_t* starts);

#ifdef __cplusplus
}
#endif

#endif /* FS_H */
