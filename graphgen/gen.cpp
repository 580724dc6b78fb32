// Seeded synthetic graph generators for the ChebyPower workloads.
//
// This module holds no part of the propagation method: it only turns a seed and
// a shape into an undirected simple graph in CSR form (rows sorted, duplicates
// and self-loops removed, both directions stored), plus seeded source draws.
// Both the FP64 oracle and the CUDA library consume its output; neither is
// imported here.
//
// Random numbers come from a counter-based generator: the 64-bit finaliser of
// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014; constants as published by Vigna) applied to
// key + counter * 0x9E3779B97F4A7C15.  Every draw is a pure function of
// (seed, stream, index), so the graph does not depend on the thread count and
// edges can be regenerated instead of stored.
//
// Generators:
//   * Erdos-Renyi G(n, m): m endpoint pairs drawn uniformly.
//   * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): 2^scale nodes, each edge
//     descends `scale` levels choosing quadrant (a, b, c, d); no noise.
//   * Chung-Lu: expected degree w_i proportional to (i + i0)^(-1/(gamma-1)),
//     scaled to a target mean and capped at sqrt(sum w); endpoints drawn in
//     proportion to w through a Walker/Vose alias table.
// CSR build: count both directions of every non-loop pair, scatter, sort each
// row, drop duplicates, compact.  Output row_ptr is int64, col_idx int32.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Draw number `idx` of stream `stream` under `seed`.
inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t key = mix64(seed * 0x9E3779B97F4A7C15ULL + 0xD1B54A32D192ED03ULL * (stream + 1));
  return mix64(key + (idx + 1) * 0x9E3779B97F4A7C15ULL);
}

inline double unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

// floor(u * n) for u uniform in [0, 2^64), without modulo bias beyond 2^-64.
inline uint64_t below(uint64_t x, uint64_t n) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

struct Edge { int64_t u, v; };

struct ErGen {
  int64_t n; uint64_t seed;
  Edge operator()(int64_t i) const {
    return {(int64_t)below(draw(seed, 1, 2 * (uint64_t)i), (uint64_t)n),
            (int64_t)below(draw(seed, 1, 2 * (uint64_t)i + 1), (uint64_t)n)};
  }
};

struct RmatGen {
  int scale; uint64_t seed; double a, ab, abc;
  Edge operator()(int64_t i) const {
    int64_t u = 0, v = 0;
    for (int l = 0; l < scale; ++l) {
      double r = unit(draw(seed, 2, (uint64_t)i * (uint64_t)scale + (uint64_t)l));
      int bu, bv;
      if (r < a) { bu = 0; bv = 0; }
      else if (r < ab) { bu = 0; bv = 1; }
      else if (r < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    return {u, v};
  }
};

struct AliasTable {
  std::vector<double> prob;
  std::vector<int64_t> alias;
};

// Vose's alias method: O(n) construction, deterministic given w.
AliasTable build_alias(const std::vector<double>& w) {
  int64_t n = (int64_t)w.size();
  double total = 0;
  for (double x : w) total += x;
  AliasTable t;
  t.prob.assign(n, 0.0);
  t.alias.assign(n, 0);
  std::vector<double> scaled(n);
  std::vector<int64_t> small, large;
  small.reserve(n); large.reserve(n);
  for (int64_t i = 0; i < n; ++i) {
    scaled[i] = w[i] * (double)n / total;
    if (scaled[i] < 1.0) small.push_back(i); else large.push_back(i);
  }
  while (!small.empty() && !large.empty()) {
    int64_t s = small.back(); small.pop_back();
    int64_t l = large.back(); large.pop_back();
    t.prob[s] = scaled[s];
    t.alias[s] = l;
    scaled[l] = (scaled[l] + scaled[s]) - 1.0;
    if (scaled[l] < 1.0) small.push_back(l); else large.push_back(l);
  }
  for (int64_t l : large) { t.prob[l] = 1.0; t.alias[l] = l; }
  for (int64_t s : small) { t.prob[s] = 1.0; t.alias[s] = s; }
  return t;
}

struct ChungLuGen {
  const AliasTable* t; int64_t n; uint64_t seed;
  int64_t pick(uint64_t x, uint64_t y) const {
    int64_t i = (int64_t)below(x, (uint64_t)n);
    return unit(y) < t->prob[i] ? i : t->alias[i];
  }
  Edge operator()(int64_t i) const {
    uint64_t b = 4 * (uint64_t)i;
    return {pick(draw(seed, 3, b), draw(seed, 3, b + 1)),
            pick(draw(seed, 3, b + 2), draw(seed, 3, b + 3))};
  }
};

template <class G>
int build_csr(int64_t n, int64_t m, const G& gen, int64_t** rp_out, int32_t** ci_out, int64_t* nnz_out) {
  if (n <= 0 || n > INT32_MAX || m < 0) return 1;
  std::vector<std::atomic<int64_t>> cnt(n + 1);
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u <= n; ++u) cnt[u].store(0, std::memory_order_relaxed);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < m; ++i) {
    Edge e = gen(i);
    if (e.u == e.v) continue;
    cnt[e.u].fetch_add(1, std::memory_order_relaxed);
    cnt[e.v].fetch_add(1, std::memory_order_relaxed);
  }
  std::vector<int64_t> off(n + 1);
  off[0] = 0;
  for (int64_t u = 0; u < n; ++u) off[u + 1] = off[u] + cnt[u].load(std::memory_order_relaxed);
  int64_t total = off[n];
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1));
  if (!tmp) return 2;
#pragma omp parallel for schedule(static)
  for (int64_t u = 0; u < n; ++u) cnt[u].store(off[u], std::memory_order_relaxed);
#pragma omp parallel for schedule(static, 65536)
  for (int64_t i = 0; i < m; ++i) {
    Edge e = gen(i);
    if (e.u == e.v) continue;
    tmp[cnt[e.u].fetch_add(1, std::memory_order_relaxed)] = (int32_t)e.v;
    tmp[cnt[e.v].fetch_add(1, std::memory_order_relaxed)] = (int32_t)e.u;
  }
  std::vector<int64_t> len(n);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t u = 0; u < n; ++u) {
    int32_t* b = tmp + off[u];
    int32_t* e = tmp + off[u + 1];
    std::sort(b, e);
    len[u] = std::unique(b, e) - b;
  }
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!rp) { free(tmp); return 2; }
  rp[0] = 0;
  for (int64_t u = 0; u < n; ++u) rp[u + 1] = rp[u] + len[u];
  int64_t nnz = rp[n];
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
  if (!ci) { free(tmp); free(rp); return 2; }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t u = 0; u < n; ++u) memcpy(ci + rp[u], tmp + off[u], sizeof(int32_t) * (size_t)len[u]);
  free(tmp);
  *rp_out = rp;
  *ci_out = ci;
  *nnz_out = nnz;
  return 0;
}

}  // namespace

extern "C" {

// All generators return 0 on success, 1 on bad arguments, 2 on allocation
// failure.  On success *row_ptr (n+1 int64) and *col_idx (nnz int32) are
// malloc'd and owned by the caller, who releases them with gg_free.

int gg_er(int64_t n, int64_t m, uint64_t seed, int64_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
  ErGen g{n, seed};
  return build_csr(n, m, g, row_ptr, col_idx, nnz);
}

int gg_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
            int64_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
  if (scale < 1 || scale > 30 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
  RmatGen g{scale, seed, a, a + b, a + b + c};
  return build_csr((int64_t)1 << scale, m, g, row_ptr, col_idx, nnz);
}

int gg_chung_lu(int64_t n, double mean_degree, double exponent, double i0, uint64_t seed,
                int64_t** row_ptr, int32_t** col_idx, int64_t* nnz) {
  if (n < 2 || mean_degree <= 0 || exponent <= 1.0 || i0 < 0) return 1;
  std::vector<double> w(n);
  double p = -1.0 / (exponent - 1.0), sum = 0;
  for (int64_t i = 0; i < n; ++i) { w[i] = std::pow((double)i + i0 + 1.0, p); sum += w[i]; }
  double scale = mean_degree * (double)n / sum;
  sum = 0;
  for (int64_t i = 0; i < n; ++i) { w[i] *= scale; sum += w[i]; }
  double cap = std::sqrt(sum);
  for (int64_t i = 0; i < n; ++i) w[i] = std::min(w[i], cap);
  AliasTable t = build_alias(w);
  int64_t m = (int64_t)std::llround(mean_degree * (double)n / 2.0);
  ChungLuGen g{&t, n, seed};
  return build_csr(n, m, g, row_ptr, col_idx, nnz);
}

// k distinct sources drawn uniformly from the nodes whose degree is >= 1
// (rejection on the draw index; deterministic).  Returns the number written.
int64_t gg_sources(int64_t n, const int64_t* row_ptr, int64_t k, uint64_t seed, int32_t* out) {
  int64_t got = 0;
  for (uint64_t i = 0; got < k && i < (uint64_t)(64 * (k + n)); ++i) {
    int64_t u = (int64_t)below(draw(seed, 4, i), (uint64_t)n);
    if (row_ptr[u + 1] == row_ptr[u]) continue;
    bool dup = false;
    for (int64_t j = 0; j < got; ++j) dup |= (out[j] == (int32_t)u);
    if (!dup) out[got++] = (int32_t)u;
  }
  return got;
}

// Uniform doubles in [0,1): out[i] = unit(draw(seed, stream, i)).
void gg_uniform(uint64_t seed, uint64_t stream, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) out[i] = unit(draw(seed, 16 + stream, (uint64_t)i));
}

void gg_free(void* p) { free(p); }

int gg_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
