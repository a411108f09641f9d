// Seeded synthetic input generators for the learned-sort tests and benchmarks.
//
// This module holds no sorting arithmetic: it only draws keys.  Both the CPU
// oracle tests and the GPU path consume its output, so nothing here may
// depend on either of them.
//
// Random numbers: SplitMix64 (Steele, Lea, Flood 2014) seeds xoshiro256**
// (Blackman & Vigna 2018).  Every chunk of CHUNK elements has its own stream,
// seeded from (seed, stream id, chunk index), so the output does not depend
// on the number of host threads.  Normals use Box-Muller with the host libm;
// Zipf ranks use the inverse CDF with binary search.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const uint64_t CHUNK = 1u << 20;

inline uint64_t splitmix64_next(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

struct Xoshiro {
  uint64_t s[4];
  Xoshiro(uint64_t seed, uint64_t stream, uint64_t chunk) {
    uint64_t sm = seed ^ (stream * 0xD1B54A32D192ED03ull) ^ (chunk * 0x8CB92BA72F3D8DD7ull);
    for (int i = 0; i < 4; ++i) s[i] = splitmix64_next(sm);
  }
  uint64_t next() {
    const uint64_t r = rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return r;
  }
  // uniform on [0,1) with 53 random bits
  double uni() { return (double)(next() >> 11) * 0x1.0p-53; }
  // uniform on (0,1]
  double uni_open0() { return (double)((next() >> 11) + 1) * 0x1.0p-53; }
  double normal() {
    const double u1 = uni_open0(), u2 = uni();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

template <class F>
void parallel_chunks(uint64_t n, F f) {
  const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 1;
  if (nt > nchunks) nt = (unsigned)std::max<uint64_t>(1, nchunks);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([=]() {
      for (uint64_t c = t; c < nchunks; c += nt) {
        const uint64_t b = c * CHUNK, e = std::min(n, b + CHUNK);
        f(c, b, e);
      }
    });
  for (auto& x : th) x.join();
}

// Zipf(s) CDF over ranks 1..k (index 0 is rank 1).
std::vector<double> zipf_cdf(uint64_t k, double s) {
  std::vector<double> cdf(k);
  double acc = 0;
  for (uint64_t i = 0; i < k; ++i) { acc += std::pow((double)(i + 1), -s); cdf[i] = acc; }
  for (uint64_t i = 0; i < k; ++i) cdf[i] /= acc;
  cdf[k - 1] = 1.0;
  return cdf;
}

inline uint64_t zipf_draw(const std::vector<double>& cdf, double u) {
  return (uint64_t)(std::upper_bound(cdf.begin(), cdf.end(), u) - cdf.begin());
}

enum { ST_MAIN = 1, ST_VALUES = 2, ST_ORDER = 3, ST_SIZES = 4 };

}  // namespace

extern "C" {

// Standard normal doubles N(mu, sigma).
void lsg_normal_f64(uint64_t seed, uint64_t n, double mu, double sigma, double* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = mu + sigma * r.normal();
  });
}

// Uniform doubles on [lo, hi).
void lsg_uniform_f64(uint64_t seed, uint64_t n, double lo, double hi, double* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = lo + (hi - lo) * r.uni();
  });
}

// Uniform 64-bit unsigned integers on [0, 2^64).
void lsg_uniform_u64(uint64_t seed, uint64_t n, uint64_t* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = r.next();
  });
}

// Uniform 32-bit unsigned integers on [0, 2^bits).
void lsg_uniform_u32(uint64_t seed, uint64_t n, int bits, uint32_t* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = (uint32_t)(r.next() >> (64 - bits));
  });
}

// Keys drawn from `k` distinct lognormal(mu, sigma) values, value j (in
// generation order) chosen with Zipf(s) weight (j+1)^-s.
void lsg_zipf_lognormal_f64(uint64_t seed, uint64_t n, uint64_t k, double s,
                            double mu, double sigma, double* out) {
  std::vector<double> vals(k);
  {
    Xoshiro r(seed, ST_VALUES, 0);
    for (uint64_t j = 0; j < k; ++j) vals[j] = std::exp(mu + sigma * r.normal());
  }
  const std::vector<double> cdf = zipf_cdf(k, s);
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = vals[zipf_draw(cdf, r.uni())];
  });
}

// Zipf(s) ranks over 1..k written as doubles (the paper's Zipf skew sweep).
void lsg_zipf_rank_f64(uint64_t seed, uint64_t n, uint64_t k, double s, double* out) {
  const std::vector<double> cdf = zipf_cdf(k, s);
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = (double)(zipf_draw(cdf, r.uni()) + 1);
  });
}

// Equal-weight mixture of N(means[j], sd^2).
void lsg_gauss_mix_f64(uint64_t seed, uint64_t n, const double* means, int m, double sd,
                       double* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) {
      const int j = (int)((r.next() >> 32) * (uint64_t)m >> 32);
      out[i] = means[j] + sd * r.normal();
    }
  });
}

// Exponential(lambda) drawn in double and rounded to float (round to nearest).
void lsg_exponential_f32(uint64_t seed, uint64_t n, double lambda, float* out) {
  parallel_chunks(n, [&](uint64_t c, uint64_t b, uint64_t e) {
    Xoshiro r(seed, ST_MAIN, c);
    for (uint64_t i = b; i < e; ++i) out[i] = (float)(-std::log(r.uni_open0()) / lambda);
  });
}

// "Timestamp-like" 32-bit keys: n / run_len runs of run_len values.  A run
// starts at a uniform base in [0, 2^32 - 2^20); each next value repeats the
// previous one with probability p_repeat, else adds a geometric gap (mean
// gap_mean, at least 1).  Then a fraction p_swap of the positions of a run is
// swapped with a partner at most `radius` positions away inside the run.  The
// runs are placed in a seeded random order.  n must be a multiple of run_len.
void lsg_timestamp_u32(uint64_t seed, uint64_t n, uint64_t run_len, double p_repeat,
                       double gap_mean, double p_swap, uint64_t radius, uint32_t* out) {
  const uint64_t runs = n / run_len;
  std::vector<uint64_t> order(runs);
  for (uint64_t i = 0; i < runs; ++i) order[i] = i;
  {
    Xoshiro r(seed, ST_ORDER, 0);
    for (uint64_t i = runs; i > 1; --i) {
      const uint64_t j = (uint64_t)(((unsigned __int128)r.next() * i) >> 64);
      std::swap(order[i - 1], order[j]);
    }
  }
  const double lq = std::log(1.0 - 1.0 / gap_mean);
  parallel_chunks(runs, [&](uint64_t, uint64_t b, uint64_t e) {
    for (uint64_t run = b; run < e; ++run) {
      Xoshiro r(seed, ST_MAIN, run);
      uint32_t* o = out + order[run] * run_len;
      uint64_t v = (r.next() >> 32) % ((1ull << 32) - (1ull << 20));
      for (uint64_t i = 0; i < run_len; ++i) {
        if (i > 0 && r.uni() >= p_repeat) {
          const uint64_t g = 1 + (uint64_t)std::floor(std::log(r.uni_open0()) / lq);
          v = std::min<uint64_t>(v + g, 0xFFFFFFFFull);
        }
        o[i] = (uint32_t)v;
      }
      for (uint64_t i = 0; i < run_len; ++i) {
        if (r.uni() < p_swap) {
          const int64_t d = (int64_t)(r.next() % (2 * radius + 1)) - (int64_t)radius;
          int64_t j = (int64_t)i + d;
          j = std::max<int64_t>(0, std::min<int64_t>((int64_t)run_len - 1, j));
          std::swap(o[i], o[j]);
        }
      }
    }
  });
}

// RootDups: A[i] = i mod floor(sqrt(n)); TwoDups: A[i] = (i*i + n/2) mod n.
// Both as doubles (the paper's duplicate-heavy synthetic sets).
void lsg_rootdups_f64(uint64_t n, double* out) {
  uint64_t r = (uint64_t)std::sqrt((double)n);
  while (r * r > n) --r;
  while ((r + 1) * (r + 1) <= n) ++r;
  if (r == 0) r = 1;
  for (uint64_t i = 0; i < n; ++i) out[i] = (double)(i % r);
}
void lsg_twodups_f64(uint64_t n, double* out) {
  for (uint64_t i = 0; i < n; ++i)
    out[i] = (double)(uint64_t)(((unsigned __int128)i * i + n / 2) % n);
}

// Array sizes for the batched workload: floor(exp(ln(median) + sigma*z))
// clipped to [lo, hi], plus a distribution id in [0, ndist) per array.
void lsg_batch_sizes(uint64_t seed, uint64_t count, double median, double sigma, uint64_t lo,
                     uint64_t hi, int ndist, uint64_t* sizes, int32_t* dist) {
  Xoshiro r(seed, ST_SIZES, 0);
  for (uint64_t i = 0; i < count; ++i) {
    const double z = r.normal();
    double v = std::floor(std::exp(std::log(median) + sigma * z));
    v = std::max((double)lo, std::min((double)hi, v));
    sizes[i] = (uint64_t)v;
    dist[i] = (int32_t)((r.next() >> 32) * (uint64_t)ndist >> 32);
  }
}

}  // extern "C"
