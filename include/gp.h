/*
 * gp.h -- C ABI of the GB300 ChebyPower library (graph propagation by the
 * Chebyshev power iteration of arXiv 2412.10789).
 *
 * What the library computes.  For an undirected graph G = (V, E) with n nodes,
 * adjacency A, degrees d_u and the random-walk matrix P = A D^{-1} (Section 2.1),
 * a query asks for the GP vector y = f(P) e_s (Eq. 1) of one source s, where f is
 *   SSPPR: f(x) = alpha / (1 - (1 - alpha) x), alpha in (0, 1)   (Def. SSPPR)
 *   HKPR:  f(x) = exp(-t (1 - x)), t > 0                          (Def. HKPR)
 * It evaluates the truncated Chebyshev expansion y_K = sum_{k<=K} c_k T_k(P) e_s
 * (Lemma 1, coefficients of Lemma 2 / Lemma 3) with the three-term recurrence
 * r_{k+1} = 2 P r_k - r_{k-1} (Eq. res-recurrence, Algorithm 3), accumulating
 * y += c_k r_k in the same pass.  K is the smallest k >= 1 with
 * tail(k) * 2 max_{l<=k} ||r_l||_1 <= l1_tol, tail(k) = sum_{l>k} |c_l| (Theorem 1
 * read for the l1 error with Assumption 1's constant estimated on the fly:
 * twice the largest norm so far, since ||r_k||_1 can still grow after k), or
 * a cap.  A node with d_u = 0 has a zero column in P; an isolated source
 * returns f(0) e_s.
 *
 * Conventions shared by every call.
 *  - Every call returns a gp_status; GP_OK = 0.  On error the out-parameters
 *    and caller buffers are left untouched and gp_last_error() (thread-local)
 *    describes the failure.  No C++ exception crosses the ABI.
 *  - Pointers: "host" pointers are ordinary CPU memory; "device" pointers are
 *    CUDA global memory of the current device.  Flags named *_on_device say which.
 *  - The caller keeps ownership of every array it passes in; the library copies
 *    what it needs.  Output buffers are caller-owned and written only on GP_OK.
 *  - All work runs on the stream given in gp_config.stream (NULL: a stream the
 *    library creates for the graph).  A call whose outputs are all on the device
 *    and that asks for no gp_query_info returns once the work is enqueued
 *    (stream-ordered); every other call returns after the work has finished.
 *  - Calls on one gp_graph are serialised by a lock; different graphs are
 *    independent.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_graph gp_graph; /* opaque; owned by the library */

typedef enum {
  GP_OK = 0,
  GP_EINVAL = 1,     /* an argument or the graph failed validation */
  GP_ENOMEM = 2,     /* device or host allocation failed */
  GP_ECUDA = 3,      /* a CUDA call failed (message in gp_last_error) */
  GP_EAGAIN = 4,     /* gp_poll: the query is not finished yet */
  GP_ENOTFOUND = 5,  /* gp_poll: unknown ticket */
  GP_ETIMEDOUT = 6,  /* gp_wait: the ticket did not complete within the timeout */
  GP_EBUSY = 7,      /* the serving queue is full */
  GP_ENOTSUP = 8     /* a combination of options the library does not support */
} gp_status;

typedef enum { GP_F32 = 0, GP_F64 = 1, GP_BF16 = 2, GP_F16 = 3 } gp_dtype;

typedef enum { GP_FN_PPR = 0, GP_FN_HKPR = 1 } gp_function;

typedef enum {
  GP_K_TAIL = 0,  /* stop at tail(k) * 2 max_{l<=k} ||r_l||_1 <= l1_tol (default) */
  GP_K_PAPER = 1, /* K = ceil(alpha^{-1/2} ln(1/tol)) or ceil(sqrt(t) ln(1/tol)) (Section 6) */
  GP_K_FIXED = 2  /* K = gp_request.k_fixed */
} gp_k_rule;

/* Options for a graph; gp_config_default fills the defaults. */
typedef struct {
  gp_dtype storage;        /* storage of the T_k blocks in batched / served queries:
                              GP_F32, GP_BF16 or GP_F16 (16-bit ones with the FP32
                              warm-up schedule); single queries always use GP_F32 */
  int32_t block_width;     /* B, columns per batched SpMM pass; 0 = autotune */
  int32_t autotune;        /* 1: gp_batch uses gp_autotune's width (block_width 0) and degree
                              threshold (t_heavy 0) */
  int32_t k_max;           /* hard cap on K (default 96) */
  int32_t validate_symmetry; /* 1 (default): check that every (u,v) has (v,u) */
  int32_t t_heavy;         /* rows with degree >= t_heavy are summed in pieces by several warps,
                              single and batched queries (0: only rows too long for one
                              whole-row task, > 508 entries, or the tuned threshold) */
  int32_t row_ptr_64;      /* 1: keep 64-bit row offsets even when nnz fits 32 bits (default 0) */
  int32_t precise_rows;    /* single queries on graphs with at most this many non-isolated nodes
                              keep T_k as float pairs (~48 bits) instead of FP32: FP32 rounding
                              is not damped on tiny graphs with unit-modulus eigenvalues
                              (0: default 1024; -1: never) */
  double warmup_tail;      /* a column stores Q in 16 bits only once sum_m (m+1)|c_{k+1+m}| is below
                              warmup_tail (default 1e-2) for BF16, 4 * warmup_tail for FP16, each times
                              min(1, l1_tol / 1e-4) for the column's own tolerance */
  size_t mem_budget;       /* bytes the serving loop may use for column blocks (0: 80% of free) */
  void* (*alloc)(size_t bytes, void* ctx); /* device allocator; NULL: cudaMalloc */
  void (*free)(void* ptr, void* ctx);      /* its release function */
  void* alloc_ctx;         /* passed to alloc / free */
  void* stream;            /* cudaStream_t for all work on this graph; NULL: own stream */
} gp_config;

/* Per-query report (all fields filled on GP_OK). */
typedef struct {
  int32_t K;             /* truncation degree used (number of applications of P) */
  int32_t k16_from;      /* first step stored in 16 bits (K+1 when none) */
  double tail_bound;     /* tail(K) * 2 max_{l<=K} ||r_l||_1, the l1 bound of the stop rule */
  double max_r_l1;       /* max_{l<=K} ||r_l||_1 as measured on the device */
  double ms;             /* wall time of the query inside the library, milliseconds */
} gp_query_info;

/* One query for gp_batch / gp_submit. */
typedef struct {
  int32_t function;      /* gp_function */
  int32_t source;        /* 0 <= source < n, in the caller's numbering */
  double param;          /* alpha (SSPPR) or t (HKPR) */
  double l1_tol;         /* target l1 error, in (0, 1) */
  int32_t k_rule;        /* gp_k_rule */
  int32_t k_fixed;       /* K for GP_K_FIXED */
  int32_t out_dtype;     /* GP_F64 or GP_F32 */
  int32_t y_on_device;   /* 1: y_out is device memory, 0: host memory */
  void* y_out;           /* n elements of out_dtype, caller-owned */
} gp_request;

/* Fill *cfg with the defaults listed in gp_config. */
void gp_config_default(gp_config* cfg);

/*
 * Build a device-resident graph from CSR (Section 2.1: undirected, both
 * directions stored).  row_ptr has n+1 entries (int32, or int64 when
 * row_ptr_is_64), col_idx has nnz int32 entries, degree has n int32 entries;
 * all three are on the device when inputs_on_device, else on the host.
 * Validation (GP_EINVAL on failure, with the first bad index in the message):
 * row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing; 0 <= col_idx < n; rows
 * strictly increasing (sorted, no duplicates); no self-loops;
 * degree[u] == row_ptr[u+1] - row_ptr[u] exactly; and, when
 * cfg->validate_symmetry, every (u, v) has its (v, u).  The library keeps a
 * relabelled copy (rows ordered by degree, descending, ties by id); results and
 * sources always use the caller's numbering.  cfg may be NULL.
 */
gp_status gp_graph_create(int64_t n, int64_t nnz, const void* row_ptr, int row_ptr_is_64,
                          const int32_t* col_idx, const int32_t* degree, int inputs_on_device,
                          const gp_config* cfg, gp_graph** out);

/* Release the graph and everything it owns; waits for queued work and cancels
 * pending tickets (their gp_poll then reports GP_ENOTFOUND). NULL is accepted. */
gp_status gp_graph_destroy(gp_graph* g);

/* Sizes of the graph: n, nnz, nodes with degree >= 1, the largest degree. Any
 * pointer may be NULL. */
gp_status gp_graph_info(const gp_graph* g, int64_t* n, int64_t* nnz, int64_t* n_active,
                        int64_t* max_degree);

/* Copy the stored graph back in the caller's numbering (host buffers: row_ptr
 * n+1 int64, col_idx nnz int32, degree n int32).  A lossless ingest returns the
 * input arrays bit for bit. */
gp_status gp_graph_export(const gp_graph* g, int64_t* row_ptr, int32_t* col_idx, int32_t* degree);

/*
 * SSPPR query (Def. SSPPR; Lemma 2 coefficients; Algorithm 3):
 * y_out = sum_{k<=K} c_k T_k(P) e_source, K by the GP_K_TAIL rule with l1_tol.
 * out_dtype: GP_F64 or GP_F32; y_out holds n elements (device memory when
 * y_on_device).  alpha in (0,1), l1_tol in (0,1), 0 <= source < n, else GP_EINVAL.
 * info may be NULL.
 */
gp_status gp_ppr(gp_graph* g, int32_t source, double alpha, double l1_tol, gp_dtype out_dtype,
                 void* y_out, int y_on_device, gp_query_info* info);

/* HKPR query (Def. HKPR; Lemma 3 coefficients; Algorithm 3); t > 0.  Otherwise as gp_ppr. */
gp_status gp_hkpr(gp_graph* g, int32_t source, double t, double l1_tol, gp_dtype out_dtype,
                  void* y_out, int y_on_device, gp_query_info* info);

/* A single query with every option of gp_request (k rule, fixed K). */
gp_status gp_query(gp_graph* g, const gp_request* req, gp_query_info* info);

/*
 * Baseline: Algorithm 1 (PwMethod) on the device, y = sum_{k<N} zeta_k P^k e_s
 * with zeta_k of Def. SSPPR / Def. HKPR and N the smallest count whose Taylor
 * tail sum_{k>=N} zeta_k is <= l1_tol (the tail bounds the l1 error because
 * ||P^k e_s||_1 = 1).  Same arguments as gp_ppr / gp_hkpr; info->K reports N.
 */
gp_status gp_power(gp_graph* g, int32_t function, int32_t source, double param, double l1_tol,
                   gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info);

/*
 * Batched queries: the `count` requests are packed as columns of one n x B
 * block and advanced together by a fused SpMM step (B = cfg.block_width or the
 * tuned width; more requests run as successive blocks).  Each column keeps its
 * own function, parameter, coefficients and K, and is retired when its own stop
 * rule fires.  T_k storage follows cfg.storage.  The columns accumulate the
 * SpMM and y in FP32, so an l1 error much below 1e-6 is out of their reach
 * (y alone is rounded once per step); smaller tolerances are accepted but
 * only the single-query calls (float-pair y) deliver them.  infos may be NULL,
 * else it receives `count` reports.
 */
gp_status gp_batch(gp_graph* g, int32_t count, const gp_request* reqs, gp_query_info* infos);

/*
 * Batched queries in Clenshaw's backward form of the same truncated sum
 * y_K = sum_{k<=K} c_k T_k(P) e_s (Lemma 1; the paper's Further Related Work
 * cites Clenshaw's recurrence for the stability of Chebyshev sums):
 * b_{K+1} = b_{K+2} = 0, b_k = c_k e_s + 2 P b_{k+1} - b_{k+2} for k = K..1,
 * y = c_0 e_s + P b_1 - b_2.  K must be known before the first step, so every
 * request's k_rule must be GP_K_FIXED (1 <= k_fixed <= 126) or GP_K_PAPER
 * (GP_EINVAL otherwise).  The vectors are stored in FP32 whatever
 * cfg.storage says; no pass but the last reads or writes y.  Same arguments,
 * outputs and blocking as gp_batch; infos report K and tail(K), with max_r_l1
 * = 0 (not measured).
 */
gp_status gp_batch_clenshaw(gp_graph* g, int32_t count, const gp_request* reqs, gp_query_info* infos);

/*
 * Generalized graph propagation of a feature matrix (Section "Generalizations",
 * Def. general-gp and the theorem that follows it):
 *     Z = f(D^-a A D^-b) X,  a + b = 1,  computed as  Z = D^-a f(P) D^a X,
 * with f = SSPPR (param = alpha) or HKPR (param = t).  X and Z are n x F
 * row-major FP32 arrays in the caller's node numbering, both in device memory
 * (on_device = 1) or both in host memory (0; the library stages them).  The F
 * features run as the columns of the batched engine (cfg.block_width or the
 * next power of two up to 256 per block, cfg.storage for the vectors), each
 * stopped by its own tail rule: ||D^a (z_f - z*_f)||_1 <= l1_tol ||D^a x_f||_1,
 * which bounds ||z_f - z*_f||_1 by the same amount since every d_u^a >= 1 on
 * the non-isolated nodes.  Nodes of degree 0 have a zero row and column in D^-a A D^-b
 * (0^-a read as 0), so Z[u] = f(0) X[u] there.  a must be in [0, 1].  infos
 * (nullable) receives F reports.
 */
gp_status gp_propagate(gp_graph* g, int32_t function, double param, double a, int32_t F, const float* X, float* Z,
                       int on_device, double l1_tol, gp_query_info* infos);

/*
 * ChebyPush (Algorithm 4): the local form of the method.  The subset Chebyshev
 * recurrence pushes, at iteration k, only the nodes u with
 * |r^_k(u)| > eps_k d_u, eps_k = eps_a / (4 K sum_{l=k}^K |c_l|), and returns
 * y^ = c_0 e_s + sum_{k=1}^{K-1} c_k r^_k restricted to the pushed nodes.
 * Theorem 3 bounds the degree-normalised error: max_u |y(u) - y^(u)| / d_u <
 * eps_a once the truncation is below eps_a / 2; K = 0 picks the smallest K
 * with sum_{l>=K} |c_l| <= eps_a / 2 (1 <= K <= 1024 otherwise).  The vectors
 * are FP64 on the device; the graph's first push query allocates them (three
 * n-vectors and the frontier, about 24 n + 16 (n + nnz / 2048) bytes, plus n
 * doubles of staging for host outputs) and keeps them until
 * gp_graph_destroy, so later push queries allocate nothing.  Output as in gp_ppr (out_dtype GP_F64 or GP_F32,
 * device or host).  info (nullable): K; tail_bound = sum_{l>=K} |c_l|;
 * max_r_l1 = the number of push items (frontier rows, long rows counted per
 * 2048 entries) over all iterations.
 */
gp_status gp_chebypush(gp_graph* g, int32_t function, int32_t source, double param, double eps_a, int32_t K,
                       gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info);

/*
 * The bidirectional method for SSPPR (Algorithm 5, Section "Generalizing to a
 * Bidirectional Method"): W = 2 (2 eps_r / 3 + 2) ln n / (eps_r^2 delta),
 * r_max = sqrt(alpha) / W; pi^ = ChebyPush(G, f, s, K, r_max); the residual
 * r = e_s - alpha^-1 [I - (1 - alpha) P] pi^; then ceil(|r(v)| W) alpha-random
 * walks from every v with r(v) != 0, each adding r(v) / W_v where it stops.
 * For nodes with pi(v) > delta the relative error is below eps_r with high
 * probability.  Walk j from node v draws from a SplitMix64 stream seeded by
 * (seed, v in the caller's numbering, j), so a seed fixes the result (up to
 * the rounding order of the FP64 sums).  K = 0 takes the paper's
 * K = ceil(alpha^-1/2 ln(1 / r_max)).  Output as in gp_ppr.  info (nullable):
 * K; tail_bound = r_max; max_r_l1 = the number of walks.
 */
gp_status gp_ppr_bidirectional(gp_graph* g, int32_t source, double alpha, double eps_r, double delta, int32_t K,
                               uint64_t seed, gp_dtype out_dtype, void* y_out, int y_on_device, gp_query_info* info);

/*
 * Autotuner for the batched form (the block width B and the degree threshold
 * of the chunked rows; the paper has no counterpart).  Times fused SpMM passes
 * of the column engine on this graph with CUDA events on the graph's stream,
 * for `storage` (16-bit storage: 0.45 of an FP32 warm-up pass plus 0.55 of a
 * 16-bit pass): first at each candidate width (powers of two in [8, 256];
 * widths == NULL means 8, 16, 32, 64, 128, 256) with rows of more than 508
 * entries chunked, then at the best width with the rows of degree >= 65, 129
 * or 257 chunked (summed in pieces by several warps).  Returns the width with
 * the least device time per column and pass in *best_width, the degree
 * threshold in *best_t_heavy (nullable; the value cfg.t_heavy would take), and
 * that time in microseconds in *us_per_column_pass (nullable).  The
 * default-candidate result is cached per graph structure (n, nnz and degree
 * sequence), storage and device; with cfg.autotune = 1, gp_batch uses its
 * width when cfg.block_width is 0 and its threshold when cfg.t_heavy is 0.
 * Allocates and frees one column block per trial; candidates that need more
 * than half of the free device memory are skipped (GP_EINVAL if none fits).
 */
gp_status gp_autotune(gp_graph* g, gp_dtype storage, const int32_t* widths, int32_t nwidths, int32_t* best_width,
                      int32_t* best_t_heavy, double* us_per_column_pass);

/*
 * Continuous-batching service.  gp_submit queues a request and returns a
 * ticket at once (GP_EBUSY when the queue is full).  A service thread admits
 * queued requests into free columns of the running block when a column slot and
 * the memory for its share of the block are free, advances every active column
 * one step per fused SpMM pass, retires a column when its stop rule fires
 * (writing y_out before the ticket completes) and refills the slot.  The
 * block has as many slots as the memory budget allows (cfg.mem_budget, default
 * 80% of the free device memory), at most cfg.block_width (0: with cfg.autotune
 * the width gp_autotune picks for FP32 on this graph, else 256; 512 at most),
 * a power of two; a block wider than 256 columns runs as 256-column halves,
 * each with its own pass.  With cfg.storage GP_BF16 or GP_F16 a second block of
 * the same width stores 16 bits: every request starts in the FP32 block and
 * moves to the 16-bit block once its own warm-up is over (see warmup_tail)
 * and at least one more step is certain to follow, while the FP32 block is
 * busy (its columns and the waiting requests fill more than half of it) and
 * the 16-bit block would then hold at least min(64, width / 4) columns
 * (info.k16_from reports the first term stored in 16 bits, K + 1 if none);
 * under light load a request stays in FP32.  With GP_F32 the service stores
 * FP32 only.  Admission, retirement, outputs and slot refills are decided on
 * the device every pass (a request loop in mapped host memory; each
 * iteration's launches are replayed as one CUDA graph), and a lightly loaded
 * block packs its columns so that its passes narrow.  The request's y_out must stay valid
 * until gp_poll reports completion.
 * gp_poll returns GP_OK (and fills info) once the ticket is done, GP_EAGAIN
 * before that, GP_ENOTFOUND for an unknown or already-collected ticket.
 */
gp_status gp_submit(gp_graph* g, const gp_request* req, uint64_t* ticket);
gp_status gp_poll(gp_graph* g, uint64_t ticket, gp_query_info* info);

/* Block until the ticket completes (then as gp_poll: GP_OK with info, or the
 * service's error), for at most timeout_ms milliseconds of host time: a bounded
 * host-side wait that returns GP_ETIMEDOUT when the time runs out (the ticket
 * stays queued or in flight and can be waited for again).  GP_ENOTFOUND for an
 * unknown or already-collected ticket; timeout_ms must be >= 0. */
gp_status gp_wait(gp_graph* g, uint64_t ticket, double timeout_ms, gp_query_info* info);

/* Serving statistics since the graph was created: completed queries, steps
 * run (one fused pass over each block half that has active columns), and the
 * mean number of active columns per step. */
gp_status gp_serve_stats(gp_graph* g, uint64_t* completed, uint64_t* steps, double* mean_active);

/*
 * Fixed-K SSPPR / HKPR query that allocates no memory (the paper has no
 * counterpart; this is for callers that cannot allocate device memory when
 * they query: a host framework that owns all device memory, or a loop that
 * cannot afford cudaFree's device-wide synchronisation or a failing
 * cudaMalloc).  It runs the Chebyshev recurrence for exactly K steps on the
 * caller's CSR (device pointers, int32 row_ptr and col_idx, natural order)
 * and writes n doubles to the device buffer y_out, on `stream` (cudaStream_t,
 * NULL = default stream), stream-ordered: every call only enqueues kernels
 * (the source's degree is read on the device), so it returns without waiting
 * for the GPU.  The CSR is not validated here; it must satisfy what
 * gp_graph_create checks: sorted rows without duplicates or self-loops and
 * both directions of every edge (an undirected graph, Section 2.1).  A row may
 * list a node whose own row is empty; that node contributes nothing
 * (1/d := 0).  An isolated source gives f(0) e_s.  Its scratch is one 16 MiB
 * array in device memory that every GPU loading this library holds until the
 * process exits, so n must be <= 1,048,576 (GP_EINVAL otherwise);
 * 1 <= K <= 256; t <= 1000.  All calls on a device share that array: calls that
 * overlap on the GPU race and corrupt each other.  The first call on a device
 * looks up the array's address, keeps it for the life of the process, and
 * should come before any stream capture; do not call it on a device after
 * cudaDeviceReset.
 */
gp_status gp_query_static(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                          int32_t function, int32_t source, double param, int32_t K, double* y_out,
                          void* stream);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t gp_launch_count(void);

/* Kernel timing: while enabled, the fused Chebyshev step kernels of
 * gp_ppr / gp_hkpr / gp_query / gp_batch are bracketed by CUDA events on their
 * stream; gp_profile_read returns the summed device time (ms), the launch count
 * and the algorithmic bytes (col_idx once, Q_k gathered once, Q_{k-1} read,
 * Q_{k+1} written, y read and written) of the launches that did work since the
 * last read, and resets them. */
gp_status gp_profile_enable(gp_graph* g, int on);
gp_status gp_profile_read(gp_graph* g, double* step_ms, int64_t* step_launches,
                          double* step_bytes);

const char* gp_status_string(gp_status s);
const char* gp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
