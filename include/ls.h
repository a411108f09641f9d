/* ls.h -- C ABI of the GB300 learned sort (LearnedSort 2.0 hot path).
 *
 * The method is LearnedSort 2.0 (Kristo, Vaidya, Kraska, arXiv 2107.03290):
 * a two-layer RMI of linear models predicts each key's scaled eCDF (Sec. 2);
 * keys are partitioned into fan-out buckets over two levels (Alg. 1, Alg. 2);
 * each bucket is finished by a model-based counting sort and an insertion-sort
 * touch-up (Alg. 2).  Heavily repeated keys get equality buckets (the
 * duplicate-handling device of Sec. 4.1, used here inside the partition).
 *
 * Conventions for every entry point:
 *  - Pointers named `keys` are DEVICE pointers unless the name says `host`.
 *    The caller owns them; they must stay valid until the stream work ends.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work and return without waiting unless stated otherwise.
 *  - Key order (the ordering contract): ascending IEEE 754 totalOrder for
 *    floats (-NaN < -inf < ... < -0.0 < +0.0 < ... < +inf < +NaN), unsigned
 *    order for integers.  The sorted output is therefore unique.
 *  - Synchronous errors (bad arguments, allocation failure, launch failure) are
 *    returned.  Asynchronous device errors (a bounded wait that timed out, a
 *    bounds check that failed) are recorded per call: each call has its own
 *    device status block, cleared when the call starts, and ORs it at its end
 *    into the status word of its stream, which ls_stream_status() returns and
 *    clears.  A call that fails stops its remaining work (its later kernels do
 *    nothing); the key contents are then unspecified.  An error on one stream
 *    is never reported on another (server requests have their own words).
 *  - Thread safety: calls on different streams may run concurrently; the
 *    library's scratch memory is stream-ordered.  The one exception is
 *    ls_radix_sort_u64_noalloc, whose calls share one static scratch array:
 *    callers must order those calls.
 */
#ifndef LS_H
#define LS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LS_F64 = 0, LS_U64 = 1, LS_F32 = 2, LS_U32 = 3 } ls_dtype;

typedef enum {
  LS_OK = 0,
  LS_ERR_INVALID = 1,   /* bad argument                                        */
  LS_ERR_NOMEM = 2,     /* device or pinned-host allocation failed             */
  LS_ERR_CUDA = 3,      /* CUDA runtime error (launch, copy, ...)              */
  LS_ERR_TIMEOUT = 4,   /* a bounded device wait gave up (asynchronous)        */
  LS_ERR_BUSY = 5,      /* server: admission refused (HBM budget / queue full) */
  LS_ERR_CANCELLED = 6  /* server: request cancelled or server shut down       */
} ls_status;

/* Tuning parameters.  Zero fields take the defaults (ls_default_params). */
typedef struct ls_params {
  uint32_t fanout;           /* level-0 buckets f; 0: chosen by the planner (256,
                                so level-0 and level-1 scatters write 128-byte runs;
                                Sec. 6.1 uses 1000, which stays available)          */
  uint32_t leaves;           /* RMI leaves L (Sec. 6.1: 1000)                          */
  uint32_t sample_div;       /* sample s = ceil(n / sample_div) (Sec. 6.1: 1% -> 100)  */
  uint32_t heavy_per_bucket; /* max equality buckets inside one level-0 bucket (<= 15);
                                0: chosen by the planner                              */
  uint64_t sample_max;       /* cap on s (0: none)                                     */
  uint64_t seed;             /* seed of the stratified sample offsets                  */
  uint64_t heavy_min_count;  /* a key is heavy if its expected count >= this           */
  uint32_t flags;            /* LS_FLAG_*                                              */
  uint32_t reserved[7];
} ls_params;

#define LS_FLAG_NO_HEAVY 1u  /* disable equality buckets                                */
/* The in-place variant (Sec. 4.2, Alg. 1: fragments flushed over positions
 * already read, then Defragment).  Every partitioning step works inside the
 * caller's array: the workspace holds no n-key scratch and no per-key ids,
 * only per-bucket tables, one byte per 128-byte block of keys and small
 * per-CTA leftover areas (ls_workspace_bytes gives the exact size).  Level 0
 * then uses at most 512 buckets and a split at most 256 sub-buckets.  The
 * result is the same sorted array. */
#define LS_FLAG_IN_PLACE 2u

/* Per-call statistics.  Passing a non-NULL ls_stats makes the call record CUDA
 * events and synchronize the stream before returning. */
typedef struct ls_stats {
  double ms_total;           /* device time of the whole call                 */
  double ms_train;           /* sample + sort sample + fit + heavy set        */
  double ms_hist;            /* level-0 histogram (K2)                        */
  double ms_scan;            /* level-0 look-back scan (K3)                   */
  double ms_scatter;         /* level-0 scatter (K4)                          */
  double ms_classify;        /* level-0 slot classification                   */
  double ms_level1;          /* level-1 re-partition of oversized slots       */
  double ms_fill;            /* equality / homogeneous fills                  */
  double ms_sort_small;      /* in-bucket counting sort, segments <= 2048     */
  double ms_sort_large;      /* in-bucket counting sort, segments <= 8192     */
  double ms_fallback;        /* radix fallback for unsplittable segments      */
  uint64_t sample_size;      /* s                                             */
  uint64_t sample_finite;    /* finite keys in the sample                     */
  uint32_t fanout, leaves;
  uint64_t n_heavy;          /* equality buckets                              */
  uint64_t n_ext;            /* level-0 slots (buckets + equality splits)     */
  uint64_t max_bucket;       /* largest level-0 slot that is not an equality  */
  uint64_t n_eq_keys;        /* keys placed by equality buckets               */
  uint64_t n_level1;         /* slots re-partitioned at level 1               */
  uint64_t n_segments;       /* segments finished by the counting sort        */
  uint64_t n_fallback;       /* segments finished by the radix fallback       */
  uint64_t n_fill;           /* fill jobs (equality + homogeneous segments)   */
  uint64_t n_launches;       /* kernels this call launched                    */
  uint64_t n_fallback_keys;  /* keys in segments of the radix fallback        */
  uint64_t max_fallback;     /* largest fallback segment                      */
  uint64_t n_large_keys;     /* keys in counting-sort segments > 2048         */
  uint64_t n_range;          /* segments split by key range (levels 2 and 3)  */
  uint64_t workspace_bytes;  /* device workspace the call allocated            */
} ls_stats;

/* Model export for parity checks (host buffers owned by the caller). */
typedef struct ls_model_export {
  uint32_t leaves;           /* in: capacity of the per-leaf arrays (>= L)    */
  uint32_t max_heavy;        /* in: capacity of heavy_tk                      */
  uint64_t sample_size;      /* out */
  uint64_t sample_finite;    /* out */
  double root[3];            /* out: a, c, b (root(x) = a (x - c) + b)        */
  double* leaf;              /* out: 5 per leaf: a, c, b, lo, hi (FP64 fit)   */
  uint32_t fanout;           /* in: capacity of thr (>= f0); out: f0 used      */
  uint32_t pos_max;          /* out: bucket of the largest total-order key     */
  uint64_t* thr;             /* out: f0 level-0 thresholds: thr[b] = smallest
                                total-order key whose bucket floor(F(x) f0)
                                (FP64, clamped to [0, f0-1]) is >= b; thr[0] = 0 */
  uint64_t* sorted_sample_tk;/* out (optional, NULL to skip): s total-order keys */
  uint64_t* heavy_tk;        /* out: heavy values (total-order keys), ascending */
  uint64_t n_heavy;          /* out */
  uint64_t tau;              /* out: run-length threshold used for heavies     */
} ls_model_export;

void ls_default_params(ls_params* p);
const char* ls_status_string(ls_status s);

/* Sort `n` keys of `dtype` at device pointer `keys` in place on `stream`
 * (Alg. 2 end to end).  n = 0 or 1 is a no-op.  Returns after enqueueing. */
ls_status ls_sort(void* keys, size_t n, ls_dtype dtype, void* stream);

/* ls_sort with explicit parameters (NULL: defaults) and optional statistics. */
ls_status ls_sort_ex(void* keys, size_t n, ls_dtype dtype, void* stream,
                     const ls_params* params, ls_stats* stats);

/* Bytes of device workspace that ls_sort_ex(keys, n, dtype, ..., params, ...)
 * allocates from the library's pool on the current device (0 for n < 2 or an
 * invalid dtype).  The caller's keys are not included. */
size_t ls_workspace_bytes(size_t n, ls_dtype dtype, const ls_params* params);

/* End-to-end form: `host_keys` is HOST memory (pinned or pageable).  Copies the
 * keys to the device, sorts them and copies them back; returns when the sorted
 * keys are in `host_keys`. */
ls_status ls_sort_host(void* host_keys, size_t n, ls_dtype dtype, void* stream,
                       const ls_params* params);

/* Sort `count` independent arrays (device pointers keys[i] with n[i] keys each;
 * the two arrays `keys` and `n` are HOST arrays) in one batched launch
 * sequence.  Arrays must not overlap. */
ls_status ls_sort_batch(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                        void* stream);

/* Tunables of the batched sort.  Arrays of more than 8192 keys are first
 * split by a line through their own key range into sub-buckets of about
 * split_target[c] keys, c the array's size class (0: at most 65,536 keys,
 * 1: at most 524,288, 2: larger).  0 takes the library's tuned table
 * (written by paper_2107_03290_gb300/autotune.py on a GB300). */
typedef struct ls_batch_params {
  uint32_t split_target[3];
  uint32_t reserved[5];
} ls_batch_params;

/* ls_sort_batch with explicit tunables (NULL: the tuned table). */
ls_status ls_sort_batch_ex(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                           void* stream, const ls_batch_params* params);

/* Stable argsort: perm[r] receives the position (in `keys`) of the key of
 * rank r in the ascending order of the ordering contract; equal keys keep
 * their input order, so perm is unique.  `keys` (n keys of `dtype`) is left
 * unchanged; `perm` is a DEVICE array of n uint32.  n >= 2^32: LS_ERR_INVALID.
 * The keys and their positions are packed into 64-bit composite keys (total-
 * order key, position) sorted by the learned sort itself (ls_sort on uint64):
 * one pass for 4-byte keys; two passes, low then high 32 bits of the
 * total-order key, for 8-byte keys (the payload permutation that Alg. 2 does
 * not carry, built from the same hot path).  Scratch: 8 n (4-byte keys) or
 * 16 n bytes from the library's pool, plus the inner sorts' workspace.
 * Asynchronous errors reach the stream's status word (ls_stream_status). */
ls_status ls_argsort(const void* keys, uint32_t* perm, size_t n, ls_dtype dtype, void* stream);

/* Key-value sort: sorts `keys` in place (as ls_sort) and permutes `values`
 * (n elements of value_bytes = 4 or 8 bytes, a DEVICE array) alongside; equal
 * keys keep their values in input order (stable).  Built on ls_argsort plus
 * two gathers.  n >= 2^32 or another value_bytes: LS_ERR_INVALID. */
ls_status ls_sort_pairs(void* keys, void* values, size_t n, ls_dtype dtype, uint32_t value_bytes,
                        void* stream);

/* Waits for `stream`, then returns and clears the status word of `stream`:
 * LS_ERR_TIMEOUT if a bounded device wait of a call on this stream gave up
 * since the last ls_stream_status(stream), LS_ERR_CUDA if a device bounds
 * check failed, else LS_OK.  Errors of calls on other streams are not seen.
 * (Streams are tracked in a table of 1024 entries per device; beyond that,
 * streams share status words.) */
ls_status ls_stream_status(void* stream);

/* Test hook, not for production use: later calls on `stream` give up each
 * bounded device wait after `spin_limit` polls (0: the default, 2^26), and
 * with `stall` = 1 the first tile of the level-0 look-back scan never
 * publishes its running total, so the waits of the tiles after it run out
 * (the "flag that nothing sets").  Such a call ends in bounded time; its later
 * kernels do nothing, the keys are left unspecified, every access stays in
 * bounds, and ls_stream_status(stream) returns LS_ERR_TIMEOUT.  stall = 0 and
 * spin_limit = 0 restore normal calls.  Returns LS_OK. */
ls_status ls_debug_set_wait(void* stream, uint32_t stall, uint64_t spin_limit);

/* Stage entry points (used by the kernel parity tests). */

/* Train the RMI on the sample of `keys` (sample, sort, FP64 fit, level-0
 * thresholds, heavy set) and copy the model to `out` (host).
 * Synchronizes `stream`. */
ls_status ls_train(const void* keys, size_t n, ls_dtype dtype, void* stream,
                   const ls_params* params, ls_model_export* out);

/* Train, then run the level-0 histogram kernel; copies the per-slot key
 * counts (n_ext entries, at most max_ext) to `hist_host`.  Synchronizes. */
ls_status ls_level0_histogram(const void* keys, size_t n, ls_dtype dtype, void* stream,
                              const ls_params* params, uint64_t* hist_host, size_t max_ext,
                              size_t* n_ext);

/* Sort `count` 64-bit unsigned keys at device pointer `keys` in place with
 * the library's LSD radix sort (8-bit digits, one pass per digit with a
 * decoupled look-back across tiles).  count >= 2^30: LS_ERR_INVALID. */
ls_status ls_radix_sort_u64(uint64_t* keys, size_t count, void* stream);

/* Sort `count` 64-bit unsigned keys at device pointer `keys` in place with the
 * sample sort that orders the training sample (Sec. 6.1: the model is fitted
 * to the sorted 1% sample): 2048 splitters from a sorted 8192-key evenly
 * spaced oversample, each key routed to a gap between splitters or to a
 * splitter's own value, each gap sorted in shared memory (a gap over 4096 keys
 * is sorted in chunks and merged in global memory).  Scratch (count + 2048
 * keys and 48 KB of counters) comes from the library's stream-ordered pool.
 * count >= 2^32: LS_ERR_INVALID, keys untouched. */
ls_status ls_sample_sort_u64(uint64_t* keys, size_t count, void* stream);

/* Kernels the library has enqueued since it was loaded (diagnostics). */
uint64_t ls_kernel_launches(void);

/* Largest `count` accepted by ls_radix_sort_u64_noalloc (2^20 keys). */
#define LS_NOALLOC_RADIX_MAX (1u << 20)

/* ls_radix_sort_u64 for callers that cannot allocate device memory when they
 * sort: a framework whose caching allocator already owns the GPU's memory, a
 * latency-bound loop that must stay out of the driver's allocator, or a library
 * that promises never to allocate.  The paper has no counterpart; it is a
 * service of this library.  Allocates nothing: the scratch is one static device
 * array inside the library sized for LS_NOALLOC_RADIX_MAX keys (about 10.5 MB,
 * held on every GPU that loads the library until the process exits).
 * `keys`: device pointer to `count` uint64 keys, sorted in place on `stream`.
 * count > LS_NOALLOC_RADIX_MAX: LS_ERR_INVALID, keys untouched.  The first call
 * on a device looks up the array's device address; make that first call before
 * any stream capture.  All calls share the array (it keeps the last call's
 * contents; the call clears what must start at zero): calls whose work
 * overlaps on the GPU race, so the caller must order them. */
ls_status ls_radix_sort_u64_noalloc(uint64_t* keys, size_t count, void* stream);

/* ---- serving: continuous batching of sort requests ---- */
typedef struct ls_server ls_server;

typedef struct ls_server_config {
  uint64_t hbm_budget_bytes; /* admission limit on bytes of admitted requests  */
  uint32_t max_inflight;     /* requests on the GPU at once (default 64)       */
  uint32_t max_queue;        /* waiting requests before LS_ERR_BUSY (def 4096) */
  uint32_t streams;          /* CUDA streams used for overlap (default 8)      */
  uint32_t debug_stall;      /* test hook (0 in normal use): ls_debug_set_wait's
                                `stall` for every request                        */
  uint32_t debug_spin_limit; /* test hook (0 in normal use): ls_debug_set_wait's
                                `spin_limit` for every request                   */
  uint32_t in_place;         /* 1: requests sorted by ls_sort (more than
                                LS_SERVER_BATCH_MAX keys) use LS_FLAG_IN_PLACE,
                                and admission charges their in-place workspace */
  uint32_t reserved[2];
} ls_server_config;

/* Requests of at most this many keys that are admitted together are sorted
 * by one batched launch sequence per key type; larger ones by ls_sort. */
#define LS_SERVER_BATCH_MAX (1u << 24)

typedef struct ls_request_stats {
  double queue_ms;           /* submit -> launch                              */
  double device_ms;          /* launch -> completion event                    */
  double total_ms;           /* submit -> completion                          */
  ls_status status;          /* LS_OK, or the request's device error: requests
                                sorted by one batched launch share its status  */
} ls_request_stats;

ls_status ls_server_create(const ls_server_config* cfg, ls_server** out);
/* Submit a sort of device keys (sorted in place).  Returns LS_ERR_BUSY when the
 * request exceeds the budget or the queue is full; *ticket identifies it. */
ls_status ls_server_submit(ls_server* s, void* keys, size_t n, ls_dtype dtype,
                           uint64_t* ticket);
/* As ls_server_submit, with the keys first copied from the device array `src`
 * (n keys, not overlapping `keys`) into `keys` on the server's stream; the
 * copy counts in queue and total latency but not in device_ms.  Requests of
 * at most LS_SERVER_BATCH_MAX (2^24) keys that are admitted together are
 * sorted by one batched launch sequence per key type; larger ones by the full
 * learned sort. */
ls_status ls_server_submit_from(ls_server* s, const void* src, void* keys, size_t n,
                                ls_dtype dtype, uint64_t* ticket);
/* Wait up to timeout_ms for a ticket (UINT32_MAX: forever).  Returns the
 * request's status (LS_ERR_TIMEOUT also when the wait itself timed out, in
 * which case the ticket stays valid). */
ls_status ls_server_wait(ls_server* s, uint64_t ticket, uint32_t timeout_ms,
                         ls_request_stats* st);
ls_status ls_server_destroy(ls_server* s);

#ifdef __cplusplus
}
#endif
#endif /* LS_H */
