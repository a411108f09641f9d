/* CPU oracle for the learned-sort hot path (LearnedSort 2.0, Kristo, Vaidya,
 * Kraska, arXiv 2107.03290).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA path.
 *
 * Part 1 (lso_sort) is a plain, slow LearnedSort 2.0 written from Alg. 1
 * (Partition) and Alg. 2 (LearnedSort) in FP64, with real fixed-capacity
 * fragments, Defragment, the level-1 re-partition, the homogeneous-bucket
 * skip, the model-based counting sort and the closing insertion sort.
 * Part 2 (lso_reference_sort) is the plain definition of the result: the
 * keys in ascending IEEE total order (unsigned order for integers).
 * Part 3 (lso_spec_*) restates, independently of the CUDA sources, the
 * per-key arithmetic that the GPU kernels document (sample indices, heavy
 * set, the FP64 level-0 bucket map and its thresholds, the extended-slot
 * histogram) so that single kernels can be checked.
 */
#ifndef LSO_H
#define LSO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { LSO_F64 = 0, LSO_U64 = 1, LSO_F32 = 2, LSO_U32 = 3 };

typedef struct lso_params {
  uint32_t fanout;      /* f, buckets per level (Sec. 6.1: 1000)                 */
  uint32_t leaves;      /* L, RMI leaf models (Sec. 6.1: 1000)                   */
  uint32_t sample_div;  /* sample size = ceil(n / sample_div) (Sec. 6.1: 1% => 100) */
  uint32_t frag_cap;    /* c, fragment capacity (Sec. 6.1: 100)                  */
  uint64_t sample_max;  /* 0 = no cap on the sample size                         */
  uint64_t seed;        /* seed of the stratified sample offsets                 */
  uint64_t n_small;     /* n below this: insertion sort only (not in the paper)  */
} lso_params;

typedef struct lso_trace {
  uint64_t sample_size;        /* s                                             */
  uint64_t sample_finite;      /* finite keys in the sample                     */
  uint64_t l0_fragments;       /* |S_F| after the level-0 Partition             */
  uint64_t l0_full_fragments;  /* fragments flushed full inside the main loop   */
  uint64_t homogeneous;        /* buckets + sub-buckets skipped as homogeneous  */
  uint64_t l1_partitions;      /* level-1 Partition calls                       */
  uint64_t counting_sorts;     /* sub-buckets sorted by the counting sort       */
  uint64_t insertion_moves;    /* element shifts of the final insertion sort    */
  uint64_t max_bucket;         /* largest level-0 bucket                        */
} lso_trace;

/* Model: root (3 doubles: a, c, b) and L leaves (5 doubles each: a, c, b, lo, hi).
 * F(x) = clamp(a_l * (x - c_l) + b_l, lo_l, hi_l), l = route(x). */
typedef struct lso_model {
  uint32_t leaves;
  uint64_t s;        /* sample size drawn      */
  uint64_t s_fin;    /* finite sample keys     */
  double root[3];
  double* leaf;      /* caller-owned, 5 * leaves doubles */
} lso_model;

void lso_default_params(lso_params* p);

/* LearnedSort 2.0 (Alg. 2) in place; keys: host array of n elements of dtype.
 * Returns 0, or -1 on a bad dtype. */
int lso_sort(void* keys, uint64_t n, int dtype, const lso_params* p, lso_trace* tr);

/* lso_sort with an optional given model (model == NULL: train on the sample;
 * else model->leaves must equal p->leaves) and, with touch_up == 0, without
 * the closing insertion sort: the keys are left as the level-1 partitions and
 * the counting sorts of Alg. 2 arranged them. */
int lso_sort_stages(void* keys, uint64_t n, int dtype, const lso_params* p,
                    const lso_model* model, int touch_up, lso_trace* tr);

/* Plain definition of the argsort: std::stable_sort of the positions
 * 0..n-1 by the total-order key of their keys (n < 2^32). */
int lso_reference_argsort(const void* keys, uint64_t n, int dtype, uint32_t* perm);

/* The plain definition: std::sort by the total-order key. */
int lso_reference_sort(void* keys, uint64_t n, int dtype);

/* Total-order key of one element (the ordering contract). */
uint64_t lso_total_order_key(const void* keys, uint64_t i, int dtype);

uint64_t lso_sample_size(uint64_t n, const lso_params* p);
void lso_sample_indices(uint64_t n, uint64_t s, uint64_t seed, uint64_t* idx);

/* Train the RMI on the sample of `keys` (model->leaf must hold 5*L doubles). */
int lso_train(const void* keys, uint64_t n, int dtype, const lso_params* p, lso_model* model);
/* Train on an explicit list of finite doubles already sorted ascending. */
void lso_fit_sorted(const double* xs, const uint64_t* tks, uint64_t m, uint32_t leaves,
                    lso_model* model);
double lso_predict(const lso_model* model, double x, int x_is_nan, int nan_negative);

/* Alg. 1 on a contiguous array of doubles (level p, parent bucket `parent`).
 * Writes bucket sizes (f entries) and the fragment list (owner, size) in the
 * order the fragments were written; returns the number of fragments. */
uint64_t lso_partition_f64(double* a, uint64_t m, const lso_model* model, int level,
                           uint32_t f, uint32_t c, uint64_t parent, uint64_t* sizes,
                           uint64_t* frag_owner, uint64_t* frag_size, uint64_t max_frags);
void lso_defragment_f64(double* a, uint64_t m, uint32_t f, const uint64_t* sizes,
                        const uint64_t* frag_owner, const uint64_t* frag_size, uint64_t nfrag);

/* ---- Part 3: spec functions for kernel parity (see header comment) ---- */

/* The GPU's level-0 map: bucket(x) = clamp(floor(F(x) * f0), 0, f0 - 1) with
 * the FP64 model (Alg. 1); its thresholds thr[b] = min { total-order key t :
 * bucket >= b }. */
typedef struct lso_eval {
  const lso_model* model;  /* FP64 model */
  uint32_t f0;             /* level-0 fan-out */
} lso_eval;

/* Level-0 bucket of key i: clamp(floor(F(x) * f0), 0, f0-1), FP64 model;
 * NaNs take F = 0 / 1 by sign. */
uint32_t lso_spec_bucket(const lso_eval* ev, const void* keys, uint64_t i, int dtype);
/* Level-0 thresholds (f0 entries) by bisection over the total order: thr[b] =
 * smallest total-order key whose bucket is >= b (never reached: 2^64-1 for
 * 8-byte keys, 2^32 for 4-byte keys); *pos_max = bucket of the largest key. */
void lso_spec_thresholds(const lso_eval* ev, int dtype, uint64_t* thr, uint32_t* pos_max);
/* Heavy set from a sorted (ascending tk) finite sample: values whose run
 * length is >= tau, at most per_bucket per level-0 bucket (longest runs
 * first, ties by smaller key), returned in ascending key order. */
uint64_t lso_spec_heavy(const uint64_t* sorted_tk, const void* sorted_keys, uint64_t m,
                        int dtype, uint64_t tau, uint32_t per_bucket, const lso_eval* ev,
                        uint64_t* heavy_tk_out, uint64_t max_out);
/* Level-0 extended-bucket histogram: regular bucket b owning heavy values
 * h_1<...<h_k gets 2k+1 slots (<h_1, =h_1, between, ..., >h_k). */
uint64_t lso_spec_ext_histogram(const lso_eval* ev, const void* keys, uint64_t n, int dtype,
                                const uint64_t* heavy_tk, uint64_t nheavy, uint64_t* hist_out,
                                uint64_t max_ext);

#ifdef __cplusplus
}
#endif
#endif
