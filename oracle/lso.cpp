// CPU oracle for LearnedSort 2.0 (arXiv 2107.03290).  TEST INFRASTRUCTURE ONLY:
// only the tests, the smoke check and the benchmark's CPU-baseline leg may load
// this library.  It shares no code with the CUDA path.  See lso.h.
//
// Compile with -ffp-contract=off: every fused multiply-add here is explicit.
//
// Readings of the paper taken here (the paper is silent or garbled on them):
//  * Alg. 1 "pos <- F(x) f^{1+a} - p(i f)" is read as
//    pos = clamp(floor(F(x) f^{1+p}) - p i f, 0, f-1), p the level, i the parent.
//  * Loop ranges "[0, f]" and "[0..n']" in Alg. 1/2 are half-open.
//  * In the fragment flush after the main loop of Alg. 1, "Frag[pos].clear()"
//    is read as "Frag[i].clear()".
//  * S_F records (owner, size) per fragment so that Defragment can place it.
//    Defragment is out of place: prefix sums of S_B give each bucket's start.
//  * The model (Sec. 2, Sec. 6.1: two layers, 1000 linear leaves, 1% sample)
//    returns the count of sample keys strictly below x divided by the sample
//    size (ties take the first rank); root and leaves are least-squares lines;
//    slopes are clamped to >= 0 and leaf outputs to [lo_l, hi_l] (the eCDF of
//    the leaf's first sample key and of the next leaf's) so that F is monotone.
//  * The counting-sort position of Alg. 2, "[F(x) - adj] * A.size", scales by
//    the whole array size N and is clamped to [0, n'-1]; the placement
//    decrements the running total before writing (T[--K[pos]] = x).
//  * Is-Homogeneous compares bit patterns (so -0.0 and +0.0 differ).
//  * Keys are ordered by IEEE total order: -NaN < -inf < ... < -0 < +0 < ...
//    < +inf < +NaN; unsigned order for integers.  NaN keys get F = 0 (negative)
//    or F = 1 (positive); non-finite keys are left out of the sample.
#include "lso.h"

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------- key traits
struct F64 {
  typedef double T;
  static uint64_t tk(T x) {
    uint64_t u; std::memcpy(&u, &x, 8);
    return (u >> 63) ? ~u : (u | (1ull << 63));
  }
  static bool is_nan(T x) { return std::isnan(x); }
  static bool finite(T x) { return std::isfinite(x); }
  static bool neg(T x) { return std::signbit(x); }
  static double dbl(T x) { return x; }
};
struct F32 {
  typedef float T;
  static uint64_t tk(T x) {
    uint32_t u; std::memcpy(&u, &x, 4);
    return (u >> 31) ? (uint64_t)(~u) : (uint64_t)(u | 0x80000000u);
  }
  static bool is_nan(T x) { return std::isnan(x); }
  static bool finite(T x) { return std::isfinite(x); }
  static bool neg(T x) { return std::signbit(x); }
  static double dbl(T x) { return (double)x; }
};
struct U64 {
  typedef uint64_t T;
  static uint64_t tk(T x) { return x; }
  static bool is_nan(T) { return false; }
  static bool finite(T) { return true; }
  static bool neg(T) { return false; }
  static double dbl(T x) { return (double)x; }
};
struct U32 {
  typedef uint32_t T;
  static uint64_t tk(T x) { return x; }
  static bool is_nan(T) { return false; }
  static bool finite(T) { return true; }
  static bool neg(T) { return false; }
  static double dbl(T x) { return (double)x; }
};

// ---------------------------------------------------------------- model (FP64)
inline double lin(double a, double x, double c, double b) {
  if (a == 0.0) return b;
  return std::fma(a, x - c, b);
}
inline double clampd(double v, double lo, double hi) {
  if (!(v >= lo)) return lo;
  if (v > hi) return hi;
  return v;
}
inline uint32_t leaf_of(const lso_model* m, double x) {
  const double w = (double)m->leaves * lin(m->root[0], x, m->root[1], m->root[2]);
  if (!(w >= 0.0)) return 0;
  if (w >= (double)m->leaves) return m->leaves - 1;
  return (uint32_t)std::floor(w);
}
inline double predict(const lso_model* m, double x) {
  const uint32_t l = leaf_of(m, x);
  const double* p = m->leaf + 5 * (size_t)l;
  return clampd(lin(p[0], x, p[1], p[2]), p[3], p[4]);
}

template <class K>
inline double F_of(const lso_model* m, typename K::T x) {
  if (K::is_nan(x)) return K::neg(x) ? 0.0 : 1.0;
  return predict(m, K::dbl(x));
}

inline uint64_t clamp_pos(double w, uint64_t lim) {  // floor(w) clamped to [0, lim-1]
  if (!(w >= 0.0)) return 0;
  if (w >= (double)lim) return lim - 1;
  return (uint64_t)std::floor(w);
}

// ---------------------------------------------------------------- sampling
inline uint64_t mix64(uint64_t z) {  // SplitMix64 output function
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------- Alg. 1
// Partition(A, F, p, f, c).  `bucket` maps a key to its bucket index.  `frag`
// is the pre-allocated array of f fragments of capacity c (f*c elements) and
// `fill` their current sizes; both are reused across calls.
template <class T, class BucketFn>
uint64_t partition(T* a, uint64_t m, uint32_t f, uint32_t c, BucketFn bucket,
                   std::vector<uint64_t>& S_B, std::vector<uint64_t>& F_owner,
                   std::vector<uint64_t>& F_size, uint64_t* full_in_loop,
                   std::vector<T>& frag, std::vector<uint32_t>& fill) {
  frag.resize((size_t)f * c);
  fill.assign(f, 0);
  S_B.assign(f, 0);                            // bucket sizes
  F_owner.clear(); F_size.clear();             // fragment (owner, size) list
  uint64_t w = 0;                              // write head
  uint64_t full = 0;
  for (uint64_t k = 0; k < m; ++k) {
    const T x = a[k];
    const uint64_t pos = bucket(x);            // predicted bucket
    T* fr = frag.data() + pos * c;
    fr[fill[pos]++] = x;                       // place in the bucket's fragment
    S_B[pos]++;
    if (fill[pos] == c) {                      // fragment full: copy back at w
      std::copy(fr, fr + c, a + w);
      w += c;
      F_owner.push_back(pos); F_size.push_back(c);
      fill[pos] = 0;
      ++full;
    }
  }
  for (uint32_t i = 0; i < f; ++i) {           // remaining fragments
    const uint64_t s = fill[i];
    const T* fr = frag.data() + (size_t)i * c;
    std::copy(fr, fr + s, a + w);
    F_owner.push_back(i); F_size.push_back(s);
    w += s;
    fill[i] = 0;
  }
  if (full_in_loop) *full_in_loop = full;
  return F_owner.size();
}

// Defragment(A, S_B, S_F): place sibling fragments contiguously, bucket order.
template <class T>
void defragment(T* a, uint64_t m, uint32_t f, const std::vector<uint64_t>& S_B,
                const std::vector<uint64_t>& F_owner, const std::vector<uint64_t>& F_size) {
  std::vector<uint64_t> cur(f);
  uint64_t acc = 0;
  for (uint32_t i = 0; i < f; ++i) { cur[i] = acc; acc += S_B[i]; }
  std::vector<T> tmp(m);
  uint64_t r = 0;
  for (size_t k = 0; k < F_owner.size(); ++k) {
    std::copy(a + r, a + r + F_size[k], tmp.begin() + cur[F_owner[k]]);
    cur[F_owner[k]] += F_size[k];
    r += F_size[k];
  }
  std::copy(tmp.begin(), tmp.end(), a);
}

template <class K>
bool homogeneous(const typename K::T* a, uint64_t m) {
  for (uint64_t k = 1; k < m; ++k)
    if (K::tk(a[k]) != K::tk(a[0])) return false;
  return true;
}

template <class K>
uint64_t insertion_sort(typename K::T* a, uint64_t m) {
  uint64_t moves = 0;
  for (uint64_t k = 1; k < m; ++k) {
    const typename K::T x = a[k];
    const uint64_t t = K::tk(x);
    uint64_t j = k;
    while (j > 0 && K::tk(a[j - 1]) > t) { a[j] = a[j - 1]; --j; ++moves; }
    a[j] = x;
  }
  return moves;
}

// ---------------------------------------------------------------- training
template <class K>
void train(const typename K::T* keys, uint64_t n, const lso_params* p, lso_model* model,
           std::vector<double>* xs_out) {
  const uint64_t s = lso_sample_size(n, p);
  std::vector<uint64_t> idx(s);
  lso_sample_indices(n, s, p->seed, idx.data());
  std::vector<std::pair<uint64_t, double>> smp;
  smp.reserve(s);
  for (uint64_t k = 0; k < s; ++k) {
    const typename K::T x = keys[idx[k]];
    if (K::finite(x)) smp.emplace_back(K::tk(x), K::dbl(x));
  }
  std::sort(smp.begin(), smp.end(),
            [](const std::pair<uint64_t, double>& u, const std::pair<uint64_t, double>& v) {
              return u.first < v.first;
            });
  std::vector<double> xs(smp.size());
  std::vector<uint64_t> tks(smp.size());
  for (size_t k = 0; k < smp.size(); ++k) { xs[k] = smp[k].second; tks[k] = smp[k].first; }
  model->s = s;
  lso_fit_sorted(xs.data(), tks.data(), xs.size(), p->leaves, model);
  if (xs_out) xs_out->swap(xs);
}

// ---------------------------------------------------------------- Alg. 2
// `given`: a model to use instead of training one (nullptr: train on the
// sample); `touch_up` = false stops before the closing insertion sort, so that
// the arrangement left by the level-1 partitions and the counting sorts can be
// checked on its own.
template <class K>
void learned_sort(typename K::T* A, uint64_t N, const lso_params* p, lso_trace* tr,
                  const lso_model* given = nullptr, bool touch_up = true) {
  typedef typename K::T T;
  if (N < 2) return;
  if (N < p->n_small) {
    if (!touch_up) return;
    const uint64_t mv = insertion_sort<K>(A, N);
    if (tr) tr->insertion_moves = mv;
    return;
  }
  const uint32_t f = p->fanout, c = p->frag_cap;
  std::vector<double> leafbuf(5 * (size_t)p->leaves);
  lso_model model;
  model.leaves = p->leaves;
  model.leaf = leafbuf.data();
  const lso_model* M = given;
  if (!M) {
    train<K>(A, N, p, &model, nullptr);
    if (tr) { tr->sample_size = model.s; tr->sample_finite = model.s_fin; }
    M = &model;
  }
  const double ff = (double)f;

  // Model-based partitioning, level 0.
  std::vector<T> frag;
  std::vector<uint32_t> fill;
  std::vector<uint64_t> S_B, F_owner, F_size;
  uint64_t full = 0;
  partition<T>(A, N, f, c, [&](T x) { return clamp_pos(F_of<K>(M, x) * ff, f); },
               S_B, F_owner, F_size, &full, frag, fill);
  if (tr) {
    tr->l0_fragments = F_owner.size();
    tr->l0_full_fragments = full;
    tr->max_bucket = *std::max_element(S_B.begin(), S_B.end());
  }
  defragment<T>(A, N, f, S_B, F_owner, F_size);

  // Re-partition each bucket into f sub-buckets.
  uint64_t r = 0;  // read head
  std::vector<uint64_t> S_B1, F_owner1, F_size1, Kc;
  std::vector<T> Tmp;
  for (uint32_t i = 0; i < f; ++i) {
    const uint64_t n_i = S_B[i];
    const uint64_t s = r;
    if (homogeneous<K>(A + s, n_i)) {
      if (tr) tr->homogeneous++;
      r += n_i;
      continue;
    }
    const double base = (double)i * ff;
    partition<T>(A + s, n_i, f, c,
                 [&](T x) { return clamp_pos(std::floor(F_of<K>(M, x) * ff * ff) - base, f); },
                 S_B1, F_owner1, F_size1, nullptr, frag, fill);
    defragment<T>(A + s, n_i, f, S_B1, F_owner1, F_size1);
    if (tr) tr->l1_partitions++;
    for (uint32_t j = 0; j < f; ++j) {
      const uint64_t n1 = S_B1[j];
      const uint64_t s1 = r;
      if (!homogeneous<K>(A + s1, n1)) {
        // Model-based counting sort.
        const double adj = ((double)i * ff + (double)j) / (ff * ff);
        Kc.assign(n1, 0);
        for (uint64_t k = 0; k < n1; ++k)
          Kc[clamp_pos((F_of<K>(M, A[s1 + k]) - adj) * (double)N, n1)]++;
        for (uint64_t k = 1; k < n1; ++k) Kc[k] += Kc[k - 1];
        Tmp.resize(n1);
        for (uint64_t k = 0; k < n1; ++k) {
          const uint64_t pos = clamp_pos((F_of<K>(M, A[s1 + k]) - adj) * (double)N, n1);
          Tmp[--Kc[pos]] = A[s1 + k];
        }
        std::copy(Tmp.begin(), Tmp.begin() + n1, A + s1);
        if (tr) tr->counting_sorts++;
      } else if (tr && n1 > 0) {
        tr->homogeneous++;
      }
      r += n1;
    }
  }
  // Touch-up for minor prediction errors.
  if (!touch_up) return;
  const uint64_t mv = insertion_sort<K>(A, N);
  if (tr) tr->insertion_moves = mv;
}

template <class K>
void reference_sort(typename K::T* a, uint64_t n) {
  std::sort(a, a + n, [](typename K::T u, typename K::T v) { return K::tk(u) < K::tk(v); });
}

// Stable argsort by the total-order key: positions of the keys in ascending
// order, equal keys in input order (the unique stable permutation).
template <class K>
void reference_argsort(const typename K::T* a, uint64_t n, uint32_t* perm) {
  std::vector<uint32_t> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
  std::stable_sort(idx.begin(), idx.end(),
                   [a](uint32_t u, uint32_t v) { return K::tk(a[u]) < K::tk(a[v]); });
  std::copy(idx.begin(), idx.end(), perm);
}

}  // namespace

// ============================================================================ C API
extern "C" {

void lso_default_params(lso_params* p) {
  p->fanout = 1000;
  p->leaves = 1000;
  p->sample_div = 100;
  p->frag_cap = 100;
  p->sample_max = 0;
  p->seed = 0;
  p->n_small = 64;
}

uint64_t lso_total_order_key(const void* keys, uint64_t i, int dtype) {
  switch (dtype) {
    case LSO_F64: return F64::tk(((const double*)keys)[i]);
    case LSO_U64: return ((const uint64_t*)keys)[i];
    case LSO_F32: return F32::tk(((const float*)keys)[i]);
    case LSO_U32: return ((const uint32_t*)keys)[i];
  }
  return 0;
}

uint64_t lso_sample_size(uint64_t n, const lso_params* p) {
  if (n == 0) return 0;
  uint64_t s = (n + p->sample_div - 1) / p->sample_div;
  const uint64_t floor2l = std::min<uint64_t>(n, 2ull * p->leaves);
  s = std::max(s, floor2l);
  if (p->sample_max) s = std::min(s, p->sample_max);
  return std::min(s, n);
}

// Stratified offsets: i_k = floor(k n / s) + mix64(seed ^ k) mod max(1, floor(n / s)).
void lso_sample_indices(uint64_t n, uint64_t s, uint64_t seed, uint64_t* idx) {
  const uint64_t stride = std::max<uint64_t>(1, n / s);
  for (uint64_t k = 0; k < s; ++k) {
    const uint64_t base = (uint64_t)(((unsigned __int128)k * n) / s);
    idx[k] = base + mix64(seed ^ k) % stride;
  }
}

void lso_fit_sorted(const double* xs, const uint64_t* tks, uint64_t m, uint32_t L,
                    lso_model* model) {
  model->leaves = L;
  model->s_fin = m;
  double* lf = model->leaf;
  if (m == 0) {
    model->root[0] = 0; model->root[1] = 0; model->root[2] = 0.5;
    for (uint32_t l = 0; l < L; ++l) {
      double* q = lf + 5 * (size_t)l;
      q[0] = 0; q[1] = 0; q[2] = 0.5; q[3] = 0.5; q[4] = 0.5;
    }
    if (L) lf[5 * (size_t)(L - 1) + 4] = 1.0;
    return;
  }
  // Targets: first rank of each key's run / m (count of sample keys below x).
  std::vector<double> y(m);
  uint64_t first = 0;
  for (uint64_t k = 0; k < m; ++k) {
    if (k > 0 && tks[k] != tks[k - 1]) first = k;
    y[k] = (double)first / (double)m;
  }
  // Root: least squares over all sample points, centred at the mean.
  double sx = 0, sy = 0;
  for (uint64_t k = 0; k < m; ++k) { sx += xs[k]; sy += y[k]; }
  const double mx = sx / (double)m, my = sy / (double)m;
  double sxx = 0, sxy = 0;
  for (uint64_t k = 0; k < m; ++k) {
    const double dx = xs[k] - mx;
    sxx += dx * dx;
    sxy += dx * (y[k] - my);
  }
  // zero variance (every sample key equal) gets slope 0: tested on the keys
  // themselves, since the centred sums of equal keys need not round to 0
  double a0 = (sxx > 0 && xs[m - 1] != xs[0]) ? sxy / sxx : 0.0;
  if (!(a0 >= 0) || !std::isfinite(a0) || !std::isfinite(mx)) a0 = 0.0;
  model->root[0] = a0;
  model->root[1] = std::isfinite(mx) ? mx : 0.0;
  model->root[2] = my;
  // Route the sample to the leaves; leaves are contiguous in sorted order.
  std::vector<uint64_t> beg(L, 0), end(L, 0);
  std::vector<char> seen(L, 0);
  for (uint64_t k = 0; k < m; ++k) {
    const uint32_t l = leaf_of(model, xs[k]);
    if (!seen[l]) { seen[l] = 1; beg[l] = k; }
    end[l] = k + 1;
  }
  for (uint32_t l = 0; l < L; ++l) {
    double* q = lf + 5 * (size_t)l;
    if (!seen[l]) { q[0] = 0; q[1] = 0; q[2] = -1; q[3] = -1; continue; }
    const uint64_t b = beg[l], e = end[l], cnt = e - b;
    double lx = 0, ly = 0;
    for (uint64_t k = b; k < e; ++k) { lx += xs[k]; ly += y[k]; }
    const double mxl = lx / (double)cnt, myl = ly / (double)cnt;
    double lxx = 0, lxy = 0;
    for (uint64_t k = b; k < e; ++k) {
      const double dx = xs[k] - mxl;
      lxx += dx * dx;
      lxy += dx * (y[k] - myl);
    }
    double a = (cnt >= 2 && lxx > 0 && xs[e - 1] != xs[b]) ? lxy / lxx : 0.0;
    if (!(a >= 0) || !std::isfinite(a) || !std::isfinite(mxl)) a = 0.0;
    q[0] = a;
    q[1] = std::isfinite(mxl) ? mxl : 0.0;
    q[2] = myl;
    q[3] = y[b];  // lo: eCDF of the leaf's first sample key
  }
  // Empty leaves take the next non-empty leaf's lo; hi_l = lo_{l+1}.
  double next_lo = 1.0;
  for (uint32_t l = L; l-- > 0;) {
    double* q = lf + 5 * (size_t)l;
    if (q[3] < 0) { q[3] = next_lo; q[2] = next_lo; q[0] = 0; q[1] = 0; }
    q[4] = next_lo;
    next_lo = q[3];
  }
}

double lso_predict(const lso_model* model, double x, int x_is_nan, int nan_negative) {
  if (x_is_nan) return nan_negative ? 0.0 : 1.0;
  return predict(model, x);
}

int lso_train(const void* keys, uint64_t n, int dtype, const lso_params* p, lso_model* model) {
  model->leaves = p->leaves;
  switch (dtype) {
    case LSO_F64: train<F64>((const double*)keys, n, p, model, nullptr); return 0;
    case LSO_U64: train<U64>((const uint64_t*)keys, n, p, model, nullptr); return 0;
    case LSO_F32: train<F32>((const float*)keys, n, p, model, nullptr); return 0;
    case LSO_U32: train<U32>((const uint32_t*)keys, n, p, model, nullptr); return 0;
  }
  return -1;
}

int lso_sort(void* keys, uint64_t n, int dtype, const lso_params* p, lso_trace* tr) {
  if (tr) std::memset(tr, 0, sizeof(*tr));
  switch (dtype) {
    case LSO_F64: learned_sort<F64>((double*)keys, n, p, tr); return 0;
    case LSO_U64: learned_sort<U64>((uint64_t*)keys, n, p, tr); return 0;
    case LSO_F32: learned_sort<F32>((float*)keys, n, p, tr); return 0;
    case LSO_U32: learned_sort<U32>((uint32_t*)keys, n, p, tr); return 0;
  }
  return -1;
}

int lso_sort_stages(void* keys, uint64_t n, int dtype, const lso_params* p,
                    const lso_model* model, int touch_up, lso_trace* tr) {
  if (tr) std::memset(tr, 0, sizeof(*tr));
  const bool t = touch_up != 0;
  switch (dtype) {
    case LSO_F64: learned_sort<F64>((double*)keys, n, p, tr, model, t); return 0;
    case LSO_U64: learned_sort<U64>((uint64_t*)keys, n, p, tr, model, t); return 0;
    case LSO_F32: learned_sort<F32>((float*)keys, n, p, tr, model, t); return 0;
    case LSO_U32: learned_sort<U32>((uint32_t*)keys, n, p, tr, model, t); return 0;
  }
  return -1;
}

int lso_reference_argsort(const void* keys, uint64_t n, int dtype, uint32_t* perm) {
  switch (dtype) {
    case LSO_F64: reference_argsort<F64>((const double*)keys, n, perm); return 0;
    case LSO_U64: reference_argsort<U64>((const uint64_t*)keys, n, perm); return 0;
    case LSO_F32: reference_argsort<F32>((const float*)keys, n, perm); return 0;
    case LSO_U32: reference_argsort<U32>((const uint32_t*)keys, n, perm); return 0;
  }
  return -1;
}

int lso_reference_sort(void* keys, uint64_t n, int dtype) {
  switch (dtype) {
    case LSO_F64: reference_sort<F64>((double*)keys, n); return 0;
    case LSO_U64: reference_sort<U64>((uint64_t*)keys, n); return 0;
    case LSO_F32: reference_sort<F32>((float*)keys, n); return 0;
    case LSO_U32: reference_sort<U32>((uint32_t*)keys, n); return 0;
  }
  return -1;
}

uint64_t lso_partition_f64(double* a, uint64_t m, const lso_model* model, int level, uint32_t f,
                           uint32_t c, uint64_t parent, uint64_t* sizes, uint64_t* frag_owner,
                           uint64_t* frag_size, uint64_t max_frags) {
  std::vector<uint64_t> S_B, Fo, Fs;
  std::vector<double> frag;
  std::vector<uint32_t> fill;
  const double ff = (double)f;
  if (level == 0) {
    partition<double>(a, m, f, c, [&](double x) { return clamp_pos(F_of<F64>(model, x) * ff, f); },
                      S_B, Fo, Fs, nullptr, frag, fill);
  } else {
    const double base = (double)parent * ff;
    partition<double>(a, m, f, c,
                      [&](double x) {
                        return clamp_pos(std::floor(F_of<F64>(model, x) * ff * ff) - base, f);
                      },
                      S_B, Fo, Fs, nullptr, frag, fill);
  }
  for (uint32_t i = 0; i < f; ++i) sizes[i] = S_B[i];
  const uint64_t nf = std::min<uint64_t>(max_frags, Fo.size());
  for (uint64_t k = 0; k < nf; ++k) { frag_owner[k] = Fo[k]; frag_size[k] = Fs[k]; }
  return Fo.size();
}

void lso_defragment_f64(double* a, uint64_t m, uint32_t f, const uint64_t* sizes,
                        const uint64_t* frag_owner, const uint64_t* frag_size, uint64_t nfrag) {
  std::vector<uint64_t> S_B(sizes, sizes + f), Fo(frag_owner, frag_owner + nfrag),
      Fs(frag_size, frag_size + nfrag);
  defragment<double>(a, m, f, S_B, Fo, Fs);
}

// ---------------------------------------------------------------- spec functions

// Alg. 1 at level 0: pos(x) = clamp(floor(F(x) * f0), 0, f0 - 1) with the
// FP64 model (the same expression the oracle's Partition uses).
uint32_t lso_spec_bucket(const lso_eval* ev, const void* keys, uint64_t i, int dtype) {
  const double ff = (double)ev->f0;
  double F = 0.0;
  switch (dtype) {
    case LSO_F64: F = F_of<F64>(ev->model, ((const double*)keys)[i]); break;
    case LSO_U64: F = F_of<U64>(ev->model, ((const uint64_t*)keys)[i]); break;
    case LSO_F32: F = F_of<F32>(ev->model, ((const float*)keys)[i]); break;
    case LSO_U32: F = F_of<U32>(ev->model, ((const uint32_t*)keys)[i]); break;
  }
  return (uint32_t)clamp_pos(F * ff, ev->f0);
}

// The key whose total-order key is t (inverse of lso_total_order_key).
static void key_of_tk(uint64_t t, int dtype, void* out) {
  switch (dtype) {
    case LSO_F64: {
      const uint64_t u = (t >> 63) ? (t & ~(1ull << 63)) : ~t;
      std::memcpy(out, &u, 8);
      break;
    }
    case LSO_F32: {
      const uint32_t t32 = (uint32_t)t;
      const uint32_t u = (t32 >> 31) ? (t32 & 0x7FFFFFFFu) : ~t32;
      std::memcpy(out, &u, 4);
      break;
    }
    case LSO_U64: std::memcpy(out, &t, 8); break;
    case LSO_U32: { const uint32_t x = (uint32_t)t; std::memcpy(out, &x, 4); break; }
  }
}

static uint32_t bucket_of_tk(const lso_eval* ev, uint64_t t, int dtype) {
  unsigned char buf[8];
  key_of_tk(t, dtype, buf);
  return lso_spec_bucket(ev, buf, 0, dtype);
}

void lso_spec_thresholds(const lso_eval* ev, int dtype, uint64_t* thr, uint32_t* pos_max) {
  const bool wide = dtype == LSO_F64 || dtype == LSO_U64;
  const uint64_t tmax = wide ? ~0ull : 0xFFFFFFFFull;
  const uint64_t never = wide ? ~0ull : 0x100000000ull;
  const uint32_t top = bucket_of_tk(ev, tmax, dtype);
  *pos_max = top;
  thr[0] = 0;
  for (uint32_t b = 1; b < ev->f0; ++b) {
    if (top < b) { thr[b] = never; continue; }
    uint64_t lo = 0, hi = tmax;  // smallest t with bucket(t) >= b
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (bucket_of_tk(ev, mid, dtype) >= b) hi = mid; else lo = mid + 1;
    }
    thr[b] = lo;
  }
}

uint64_t lso_spec_heavy(const uint64_t* tk, const void* keys, uint64_t m, int dtype,
                        uint64_t tau, uint32_t per_bucket, const lso_eval* ev, uint64_t* out,
                        uint64_t max_out) {
  struct Cand { uint64_t tk, len, idx; uint32_t b; };
  std::vector<Cand> cand;
  uint64_t k = 0;
  while (k < m) {
    uint64_t e = k + 1;
    while (e < m && tk[e] == tk[k]) ++e;
    if (e - k >= tau) cand.push_back({tk[k], e - k, k, lso_spec_bucket(ev, keys, k, dtype)});
    k = e;
  }
  std::vector<uint64_t> res;
  size_t a = 0;
  while (a < cand.size()) {
    size_t b = a + 1;
    while (b < cand.size() && cand[b].b == cand[a].b) ++b;
    std::vector<Cand> grp(cand.begin() + a, cand.begin() + b);
    std::sort(grp.begin(), grp.end(), [](const Cand& u, const Cand& v) {
      return u.len != v.len ? u.len > v.len : u.tk < v.tk;
    });
    if (grp.size() > per_bucket) grp.resize(per_bucket);
    std::sort(grp.begin(), grp.end(), [](const Cand& u, const Cand& v) { return u.tk < v.tk; });
    for (auto& g : grp) res.push_back(g.tk);
    a = b;
  }
  const uint64_t nout = std::min<uint64_t>(res.size(), max_out);
  for (uint64_t j = 0; j < nout; ++j) out[j] = res[j];
  return res.size();
}

uint64_t lso_spec_ext_histogram(const lso_eval* ev, const void* keys, uint64_t n, int dtype,
                                const uint64_t* heavy, uint64_t nheavy, uint64_t* hist,
                                uint64_t max_ext) {
  const uint32_t f0 = ev->f0;
  // Heavy values per bucket (heavy list is ascending, buckets non-decreasing).
  std::vector<std::vector<uint64_t>> hb(f0);
  for (uint64_t j = 0; j < nheavy; ++j) {
    // the bucket of a heavy value: evaluate it as a key of `dtype`
    const uint64_t t = heavy[j];
    const uint32_t b = bucket_of_tk(ev, t, dtype);
    hb[b].push_back(t);
  }
  std::vector<uint64_t> base(f0);
  uint64_t acc = 0;
  for (uint32_t b = 0; b < f0; ++b) { base[b] = acc; acc += 2 * hb[b].size() + 1; }
  const uint64_t next = acc;
  for (uint64_t j = 0; j < std::min(next, max_ext); ++j) hist[j] = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint32_t b = lso_spec_bucket(ev, keys, i, dtype);
    const uint64_t t = lso_total_order_key(keys, i, dtype);
    uint64_t e = base[b];
    for (uint64_t h : hb[b]) {
      if (h < t) e += 2;
      else if (h == t) { e += 1; break; }
      else break;
    }
    if (e < max_ext) hist[e]++;
  }
  return next;
}

}  // extern "C"
