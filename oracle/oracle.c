/*
 * FP64 CPU oracle for ChebyPower (arXiv 2412.10789) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke entry point and the benchmark's CPU-baseline leg may
 * load this file's library.  It shares no code, header, table or constant with
 * the CUDA library: it is written from the paper's definitions, plainly and
 * slowly, in double precision, compiled with -ffp-contract=off so that no FMA
 * contraction changes the rounding of the written expressions.
 *
 * Notation (Section 2.1): undirected graph G=(V,E), n nodes, CSR adjacency with
 * both directions stored, d_u = |N(u)|, P = A D^{-1}.  A node with d_u = 0 has a
 * zero column in P (the reading 1/0 := 0), so P r never reads it.
 *
 * Contents
 *   or_taylor_coeffs   zeta_k of Def. SSPPR / Def. HKPR (Section 2.1)
 *   or_cheb_coeffs     c_k of Lemma 1, by quadrature of its integral definition
 *   or_P_apply         y = P x, the pull form sum_{v in N(u)} x(v)/d_v
 *   or_power           Algorithm 1 (PwMethod), Taylor truncation N
 *   or_chebypower      Algorithm 3 (ChebyPower), fixed truncation K, start vector x
 *   or_chebypower_tol  Algorithm 3 with K chosen by the l1 stopping reading
 *   or_cheb_basis      r_k = T_k(P) x for k = 0..K (Eq. res-recurrence), for pins
 *   or_chebypush       Algorithm 4 (ChebyPush), the subset Chebyshev recurrence by pushes
 *   or_bidirectional   Algorithm 5 (ChebyPush + alpha-random walks) for SSPPR
 *   or_errors          the error measures of the error-metric definition, plus max-abs
 *
 * Threads: the only parallel loop is the row loop of or_P_apply; each row is
 * summed by one thread in CSR order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PPR 0
#define OR_HKPR 1

static const double OR_PI = 3.14159265358979323846264338327950288;

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* The GP function f on [-1, 1] (Section 3.1, text after Lemma 1):
 *   SSPPR: f(x) = alpha / (1 - (1 - alpha) x)
 *   HKPR:  f(x) = exp(-t (1 - x))                                            */
static double gp_f(int kind, double param, double x) {
  if (kind == OR_PPR) return param / (1.0 - (1.0 - param) * x);
  return exp(-param * (1.0 - x));
}

/* Taylor coefficients zeta_k, k = 0..N-1.
 *   Def. SSPPR: zeta_k = alpha (1-alpha)^k
 *   Def. HKPR:  zeta_k = e^{-t} t^k / k!   (built as a running product)      */
void or_taylor_coeffs(int kind, double param, int N, double* zeta) {
  if (kind == OR_PPR) {
    double p = 1.0;
    for (int k = 0; k < N; ++k) { zeta[k] = param * p; p *= (1.0 - param); }
  } else {
    double term = exp(-param);
    for (int k = 0; k < N; ++k) { zeta[k] = term; term = term * param / (double)(k + 1); }
  }
}

/* Lemma 1: c_k = (2/pi) int_{-1}^{1} f(x) T_k(x) / sqrt(1-x^2) dx for k >= 1 and
 * the same with 1/pi for k = 0.  With x = cos(theta) this is
 *   c_k = (2/pi) int_0^pi f(cos th) cos(k th) d th,
 * whose integrand is smooth and 2*pi-periodic, so the composite trapezoid rule on
 * M intervals of [0, pi] converges geometrically (its error is the aliased
 * coefficients c_{2M-k}, c_{2M+k}, ...).  M must exceed K by a wide margin.    */
void or_cheb_coeffs(int kind, double param, int K, int M, double* c) {
  double h = OR_PI / (double)M;
  for (int k = 0; k <= K; ++k) {
    double s = 0.0;
    for (int j = 0; j <= M; ++j) {
      double th = h * (double)j;
      double w = (j == 0 || j == M) ? 0.5 : 1.0;
      s += w * gp_f(kind, param, cos(th)) * cos((double)k * th);
    }
    double integral = s * h;
    c[k] = (k == 0 ? 1.0 : 2.0) / OR_PI * integral;
  }
}

/* d_u = |N(u)| = row_ptr[u+1] - row_ptr[u] (Section 2.1). */
static double deg_of(const int64_t* row_ptr, int64_t u) { return (double)(row_ptr[u + 1] - row_ptr[u]); }

/* y = P x with P = A D^{-1}:  y(u) = sum_{v in N(u)} A_uv x(v) / d_v.
 * In a symmetric adjacency every listed v has d_v >= 1; a CSR that lists a
 * node with an empty row (accepted only with the symmetry check off) takes
 * 1/d_v := 0 for it, the zero column of P that a degree-0 node has.            */
void or_P_apply(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* x, double* y) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t u = 0; u < n; ++u) {
    double s = 0.0;
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int64_t v = col_idx[e];
      const double d = deg_of(row_ptr, v);
      if (d > 0.0) s += x[v] / d;
    }
    y[u] = s;
  }
}

/* Algorithm 1 (PwMethod): y = 0, r_0 = x; for k = 0..N-1: y += zeta_k r_k,
 * r_{k+1} = P r_k.  Returns 0, or 2 on allocation failure.                    */
int or_power(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* x,
             const double* zeta, int N, double* y) {
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* rn = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !rn) { free(r); free(rn); return 2; }
  memcpy(r, x, sizeof(double) * (size_t)n);
  for (int64_t u = 0; u < n; ++u) y[u] = 0.0;
  for (int k = 0; k < N; ++k) {
    for (int64_t u = 0; u < n; ++u) y[u] += zeta[k] * r[u];
    or_P_apply(n, row_ptr, col_idx, r, rn);
    double* t = r; r = rn; rn = t;
  }
  free(r); free(rn);
  return 0;
}

/* Algorithm 3 (ChebyPower) with start vector x (x = e_s for the GP vector;
 * Section 5.1 uses x = D^a x' for the generalised form):
 *   y = c_0 r_0; r_0 = x; r_1 = P x; k = 1
 *   while k < K: y += c_k r_k; r_{k+1} = 2 P r_k - r_{k-1}; k += 1
 *   y += c_K r_K
 * K >= 1 is required (with K = 0 the last line would add c_0 x a second time).
 * If rnorm is not NULL, rnorm[k] = ||r_k||_1 for k = 0..K.                    */
int or_chebypower(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* x,
                  const double* c, int K, double* y, double* rnorm) {
  if (K < 1) return 1;
  double* rprev = (double*)malloc(sizeof(double) * (size_t)n);
  double* rcur = (double*)malloc(sizeof(double) * (size_t)n);
  double* pr = (double*)malloc(sizeof(double) * (size_t)n);
  if (!rprev || !rcur || !pr) { free(rprev); free(rcur); free(pr); return 2; }
  memcpy(rprev, x, sizeof(double) * (size_t)n);
  or_P_apply(n, row_ptr, col_idx, rprev, rcur);
  for (int64_t u = 0; u < n; ++u) y[u] = c[0] * rprev[u];
  if (rnorm) {
    double a = 0.0, b = 0.0;
    for (int64_t u = 0; u < n; ++u) { a += fabs(rprev[u]); b += fabs(rcur[u]); }
    rnorm[0] = a; rnorm[1] = b;
  }
  int k = 1;
  while (k < K) {
    for (int64_t u = 0; u < n; ++u) y[u] += c[k] * rcur[u];
    or_P_apply(n, row_ptr, col_idx, rcur, pr);
    double nrm = 0.0;
    for (int64_t u = 0; u < n; ++u) {
      double next = 2.0 * pr[u] - rprev[u];
      rprev[u] = rcur[u];
      rcur[u] = next;
      nrm += fabs(next);
    }
    k += 1;
    if (rnorm) rnorm[k] = nrm;
  }
  for (int64_t u = 0; u < n; ++u) y[u] += c[K] * rcur[u];
  free(rprev); free(rcur); free(pr);
  return 0;
}

/* Algorithm 4 (ChebyPush): the subset Chebyshev recurrence (Def. of the
 * subset recurrence, Eq. subset-cheby-implement) carried out by pushes:
 *   y = c_0 e_s; r_cur = P e_s; r_new = -e_s; k = 1
 *   while k < K:
 *     for every u with |r_cur(u)| > eps[k] d_u          (rule 0: the algorithm)
 *                  or r_cur(u)^2 >= eps[k] d_u         (rule 1: the decisions of
 *                                                       the worked example)
 *       y(u) += c_k r_cur(u)
 *       r_new(v) += 2 r_cur(u) / d_u for every v in N(u)
 *       r_cur(u) = -r_cur(u)
 *     swap(r_cur, r_new); k += 1
 * The pushes of one iteration write r_new only, so their order does not
 * matter.  eps[1..K-1] are the per-iteration thresholds (the algorithm sets
 * eps_k = eps_a / (4 K sum_{l=k}^K |c_l|)).  Writes y, and r_cur (= r^_K) to
 * r_out when r_out is not NULL.  Returns 0, 1 for K < 1, 2 on allocation failure. */
int or_chebypush(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t s, const double* c, int K,
                 const double* eps, int rule, double* y, double* r_out) {
  if (K < 1) return 1;
  double* ra = (double*)calloc((size_t)n, sizeof(double));
  double* rb = (double*)calloc((size_t)n, sizeof(double));
  if (!ra || !rb) { free(ra); free(rb); return 2; }
  double* rcur = ra;
  double* rnew = rb;
  for (int64_t u = 0; u < n; ++u) y[u] = 0.0;
  y[s] = c[0];
  /* r_1 = P e_s, as the pushes below move residual: 1/d_s to every node in
   * the neighbour list of s (on the undirected graphs of Section 2.1 this is
   * the column s of P; for a CSR that is not symmetric it keeps the first
   * step and the iterations one operation) */
  {
    const double ds = deg_of(row_ptr, s);
    for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) rcur[col_idx[e]] += 1.0 / ds;
  }
  rnew[s] = -1.0;
  for (int k = 1; k < K; ++k) {
    for (int64_t u = 0; u < n; ++u) {
      const double r = rcur[u], d = deg_of(row_ptr, u);
      const int push = rule == 0 ? fabs(r) > eps[k] * d : r * r >= eps[k] * d;
      if (!push) continue;
      y[u] += c[k] * r;
      for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) rnew[col_idx[e]] += 2.0 * r / d;
      rcur[u] = -r;
    }
    double* t = rcur;
    rcur = rnew;
    rnew = t;
  }
  if (r_out) memcpy(r_out, rcur, sizeof(double) * (size_t)n);
  free(ra);
  free(rb);
  return 0;
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", 2014): the state advances by the golden gamma and each output
 * is the state mixed by its finaliser.  A random walk draws from its own
 * stream, seeded from (seed, start node, walk index).                        */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t sm64_next(uint64_t* state) {
  *state += 0x9E3779B97F4A7C15ull;
  return sm64_mix(*state);
}
uint64_t or_walk_seed(uint64_t seed, int64_t v, int64_t j) {
  return sm64_mix(seed ^ sm64_mix((uint64_t)v * 0x9E3779B97F4A7C15ull + (uint64_t)j));
}

/* One alpha-random walk from v (Section "Generalizing to a Bidirectional
 * Method"): at each step it stops with probability alpha, else it moves to a
 * uniformly chosen neighbour.  Draws: u = (z >> 11) 2^-53 decides the stop
 * (u < alpha); the neighbour is the ((z' >> 32) d >> 32)-th of the row.  A
 * node without neighbours ends the walk.  Returns the node where it stops.    */
int64_t or_alpha_walk(const int64_t* row_ptr, const int32_t* col_idx, int64_t v, double alpha, uint64_t state) {
  for (;;) {
    const uint64_t z = sm64_next(&state);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    if (u < alpha || d == 0) return v;
    const uint64_t z2 = sm64_next(&state);
    v = col_idx[row_ptr[v] + (int64_t)(((z2 >> 32) * (uint64_t)d) >> 32)];
  }
}

/* Algorithm 5 (ChebyPush + RW) for SSPPR with teleport alpha:
 *   W = 2 (2 eps_r / 3 + 2) ln n / (eps_r^2 delta); r_max = sqrt(alpha) / W
 *   pi^ = ChebyPush(G, f, s, K, r_max)                   (Algorithm 4, rule 0)
 *   r = e_s - alpha^-1 [I - (1 - alpha) P] pi^
 *   for every v with |r(v)| > 0: W_v = ceil(|r(v)| W) walks from v, walk j
 *     drawing from the stream or_walk_seed(seed, v, j); pi^(u) += r(v) / W_v
 *     at the node u where it stops
 * c[0..K] are the SSPPR coefficients.  Writes pi^ to y, and (when not NULL)
 * the total number of walks to *walks.  Returns 0, 1 for bad arguments, 2 on
 * allocation failure.                                                         */
int or_bidirectional(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, int64_t s, double alpha,
                     const double* c, int K, double eps_r, double delta, uint64_t seed, double* y, int64_t* walks) {
  if (K < 1 || n < 2 || !(alpha > 0.0 && alpha < 1.0)) return 1;
  const double W = 2.0 * (2.0 * eps_r / 3.0 + 2.0) * log((double)n) / (eps_r * eps_r * delta);
  const double rmax = sqrt(alpha) / W;
  double* eps = (double*)malloc(sizeof(double) * (size_t)(K + 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* pp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!eps || !r || !pp) { free(eps); free(r); free(pp); return 2; }
  eps[0] = 0.0;
  for (int k = 1; k <= K; ++k) {
    double t = 0.0;
    for (int l = k; l <= K; ++l) t += fabs(c[l]);
    eps[k] = t > 0.0 ? rmax / (4.0 * K * t) : 0.0;
  }
  int rc = or_chebypush(n, row_ptr, col_idx, s, c, K, eps, 0, y, NULL);
  if (rc) { free(eps); free(r); free(pp); return rc; }
  or_P_apply(n, row_ptr, col_idx, y, pp);
  for (int64_t u = 0; u < n; ++u) r[u] = (u == s ? 1.0 : 0.0) - (y[u] - (1.0 - alpha) * pp[u]) / alpha;
  int64_t total = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (r[v] == 0.0) continue;
    const int64_t Wv = (int64_t)ceil(fabs(r[v]) * W);
    for (int64_t j = 0; j < Wv; ++j) {
      const int64_t u = or_alpha_walk(row_ptr, col_idx, v, alpha, or_walk_seed(seed, v, j));
      y[u] += r[v] / (double)Wv;
    }
    total += Wv;
  }
  if (walks) *walks = total;
  free(eps); free(r); free(pp);
  return 0;
}

/* Algorithm 3 with the truncation K found on the fly (the stopping reading of
 * Theorem 1 for the l1 error, with Assumption 1's constant estimated):
 *   tail(k) = sum_{l>k} |c_l| over the supplied c_0..c_Kmax (c beyond Kmax is
 *   taken as part of the supplied table, so Kmax must leave a negligible rest);
 *   C(k) = OR_C_MARGIN * max_{l<=k} ||r_l||_1;
 *   K = the smallest k >= 1 with tail(k) * C(k) <= tol, or Kmax.
 * The margin: ||r_k||_1 can still grow after k (the running maximum alone let
 * the truncation exceed tol by a few percent on power-law graphs), and the
 * first omitted term obeys ||r_{k+1}||_1 <= 2 ||P r_k||_1 + ||r_{k-1}||_1, at
 * most 3 max_{l<=k} ||r_l||_1 since P is column-stochastic; 2 is the reading.
 * Writes y, *K_out and rnorm[0..K].                                           */
#define OR_C_MARGIN 2.0
int or_chebypower_tol(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* x,
                      const double* c, int Kmax, double tol, double* y, int* K_out, double* rnorm) {
  if (Kmax < 1) return 1;
  double* tail = (double*)malloc(sizeof(double) * (size_t)(Kmax + 1));
  double* rprev = (double*)malloc(sizeof(double) * (size_t)n);
  double* rcur = (double*)malloc(sizeof(double) * (size_t)n);
  double* pr = (double*)malloc(sizeof(double) * (size_t)n);
  if (!tail || !rprev || !rcur || !pr) { free(tail); free(rprev); free(rcur); free(pr); return 2; }
  for (int k = 0; k <= Kmax; ++k) {
    double s = 0.0;
    for (int l = Kmax; l > k; --l) s += fabs(c[l]);
    tail[k] = s;
  }
  memcpy(rprev, x, sizeof(double) * (size_t)n);
  or_P_apply(n, row_ptr, col_idx, rprev, rcur);
  double n0 = 0.0, n1 = 0.0;
  for (int64_t u = 0; u < n; ++u) { n0 += fabs(rprev[u]); n1 += fabs(rcur[u]); }
  rnorm[0] = n0; rnorm[1] = n1;
  double C = n0 > n1 ? n0 : n1;
  for (int64_t u = 0; u < n; ++u) y[u] = c[0] * rprev[u] + c[1] * rcur[u];
  int k = 1;
  while (k < Kmax && tail[k] * OR_C_MARGIN * C > tol) {
    or_P_apply(n, row_ptr, col_idx, rcur, pr);
    double nrm = 0.0;
    for (int64_t u = 0; u < n; ++u) {
      double next = 2.0 * pr[u] - rprev[u];
      rprev[u] = rcur[u];
      rcur[u] = next;
      nrm += fabs(next);
    }
    k += 1;
    for (int64_t u = 0; u < n; ++u) y[u] += c[k] * rcur[u];
    rnorm[k] = nrm;
    if (nrm > C) C = nrm;
  }
  *K_out = k;
  free(tail); free(rprev); free(rcur); free(pr);
  return 0;
}

/* r_0 = x, r_1 = P x, r_{k+1} = 2 P r_k - r_{k-1} (Eq. res-recurrence);
 * R is (K+1) x n, row k = r_k.                                               */
int or_cheb_basis(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* x, int K,
                  double* R) {
  if (K < 0) return 1;
  memcpy(R, x, sizeof(double) * (size_t)n);
  if (K == 0) return 0;
  or_P_apply(n, row_ptr, col_idx, R, R + n);
  double* pr = (double*)malloc(sizeof(double) * (size_t)n);
  if (!pr) return 2;
  for (int k = 1; k < K; ++k) {
    const double* rk = R + (size_t)k * (size_t)n;
    const double* rkm1 = R + (size_t)(k - 1) * (size_t)n;
    double* rkp1 = R + (size_t)(k + 1) * (size_t)n;
    or_P_apply(n, row_ptr, col_idx, rk, pr);
    for (int64_t u = 0; u < n; ++u) rkp1[u] = 2.0 * pr[u] - rkm1[u];
  }
  free(pr);
  return 0;
}

/* Error measures (definition of the error metrics, Section 2.1):
 *   out[0] = ||y - yh||_1, out[1] = ||y - yh||_2,
 *   out[2] = max_u |y(u) - yh(u)| / d_u over nodes with d_u >= 1,
 *   out[3] = max_u |y(u) - yh(u)| (max-abs).                                  */
void or_errors(int64_t n, const int64_t* row_ptr, const double* y, const double* yh, double* out) {
  double l1 = 0.0, l2 = 0.0, dn = 0.0, mx = 0.0;
  for (int64_t u = 0; u < n; ++u) {
    double e = fabs(y[u] - yh[u]);
    l1 += e;
    l2 += e * e;
    if (e > mx) mx = e;
    double d = deg_of(row_ptr, u);
    if (d >= 1.0 && e / d > dn) dn = e / d;
  }
  out[0] = l1; out[1] = sqrt(l2); out[2] = dn; out[3] = mx;
}
