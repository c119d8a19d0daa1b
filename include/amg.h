/*
 * amg.h -- C ABI of the GB300 (sm_103a) aggregation-AMG solver for graph
 * Laplacian systems A u = f, after Brannick, "Aggregation-based aggressive
 * coarsening with polynomial smoothing".
 *
 * The operator is the bilinear form of Eq. (1):
 *     (A u, v) = sum_{e=(i,j)} w_e (u_i - u_j)(v_i - v_j) + sum_i d_i u_i v_i,
 * so A_ii = sum_j w_ij + d_i and A_ij = -w_ij.  The solver is flexible CG
 * preconditioned by the nonlinear AMLI cycle (K-cycle, W(1,1)) of Sec. 4 over
 * unsmoothed (piecewise-constant) aggregation coarse spaces (Sec. 2, Eq.
 * (coarse)), with the smoother R = q_m(A), q_m the polynomial of best uniform
 * approximation to 1/x on [lambda0, lambda1], lambda1 = ||A||_inf and lambda0 =
 * lambda1/10 by default (Sec. 3, Eq. (1x-1-min); Sec. 4).
 * Aggregates are built on the device by handshake matching (Sec. 2: a
 * matching is the simplest graph partitioning), several passes per level, or
 * by the paper's maximal independent sets of the graph of A^k (Sec. 2 steps
 * (A)-(B), option `aggregation`); coarse operators are the Galerkin products
 * P^T A P (Sec. 3 remark; Sec. 5: sums of fine entries over aggregates).  The
 * stationary AMLI W-cycle of Sec. 4 is option `cycle`.
 *
 * Conventions for every entry point:
 *  - Status codes only; nothing throws across this boundary.  After an error
 *    amg_last_error() describes it.
 *  - Input arrays are borrowed for the duration of the call and never
 *    retained; the handle owns every device buffer of the hierarchy.
 *  - "Device pointer" means memory of the current CUDA device (cudaMalloc,
 *    torch tensors on that device, managed memory).  Entry points that accept
 *    either kind say so and classify pointers with cudaPointerGetAttributes.
 *  - All work is issued on the handle's stream (see amg_setup); calls return
 *    after that work has completed unless stated otherwise.
 *  - A handle is not thread safe: calls on one handle must not overlap.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_handle_s *amg_handle;

typedef enum {
  AMG_OK = 0,
  AMG_ERR_INVALID_ARG = 1,    /* bad pointer/size/option, malformed CSR           */
  AMG_ERR_NOT_SYMMETRIC = 2,  /* pattern or weights not symmetric (exact)         */
  AMG_ERR_SELF_LOOP = 3,      /* an entry (i, i) in the graph                      */
  AMG_ERR_BAD_WEIGHT = 4,     /* w <= 0, d < 0, or a non-finite value              */
  AMG_ERR_DISCONNECTED = 5,   /* pure Laplacian not connected, or a component
                                 without any d_i > 0 (A singular beyond 1)         */
  AMG_ERR_OOM = 6,            /* device allocation failed                          */
  AMG_ERR_CUDA = 7,           /* CUDA runtime error / no usable device             */
  AMG_ERR_NOT_CONVERGED = 8,  /* max_iters reached; x and info hold the last iterate */
  AMG_ERR_BREAKDOWN = 9,      /* outer CG: d^T A d <= 0 or non-finite              */
  AMG_ERR_TIMEOUT = 10,       /* a bounded device-side wait ran out                */
  AMG_ERR_SETUP_STALL = 11    /* aggregation cannot coarsen a level of > 4096 vertices */
} amg_status;

enum { AMG_MEM_HOST = 0, AMG_MEM_DEVICE = 1 };
enum { AMG_PREC_FP64 = 0, AMG_PREC_FP32 = 1 };

/* Solver options; amg_default_options() fills the defaults listed there
 * (the paper's degree, interval, cycle and restart; matching aggregation). */
typedef struct {
  int degree;          /* m, degree of q_m (Sec. 4 uses 4); 0..16                 */
  int passes;          /* matching passes composed per level (~2^passes per
                          aggregate), 1..16; AMG_AGG_MATCHING only                 */
  int coarse_max;      /* coarsen until n_k <= coarse_max; coarsest solved densely;
                          1..4096                                                  */
  int max_levels;      /* cap on the number of levels, 1..64                       */
  int inner_iters;     /* nu: flexible-CG steps on coarse levels (2 = W-cycle), 1..8 */
  int restart;         /* outer flexible CG window cleared every `restart` its (5),
                          1..16                                                    */
  int max_iters;       /* outer iteration cap, >= 0                                */
  int precision;       /* AMG_PREC_FP64: everything in fp64.  AMG_PREC_FP32: the
                          whole preconditioner (smoother, transfers, coarse-level
                          cycles) in fp32 inside fp64 outer CG; outer residual,
                          outer dots/orthogonalisation and the coarsest dense
                          solve stay fp64                                          */
  double lambda0_ratio;/* lambda0 = ratio * ||A_k||_inf, in (0, 1) (Sec. 4: 1/10) */
  uint64_t hash_salt;  /* salt of the matching tie-break hash and of the keys of
                          AMG_AGG_MIS                                            */
  int cycle;           /* AMG_CYCLE_K: nonlinear AMLI cycle (K-cycle), inner
                          flexible CG on coarse levels.  AMG_CYCLE_AMLI:
                          stationary AMLI W-cycle (Sec. 4), a fixed polynomial
                          in B_{k+1} A_{k+1} on coarse levels: e_H =
                          q(B_{k+1} A_{k+1}) B_{k+1} r_H, q = q_{nu-1}/(1+E) with
                          q_{nu-1} the best uniform approximation to 1/t on
                          [amli_alpha, 1] and E = delta^(nu-1)(1/amli_alpha-1)/2
                          its error bound (Sec. 3), which must be < 1            */
  double amli_alpha;   /* left end of the AMLI polynomial's interval, (0, 1)     */
  double rho;          /* > 0: choose m from Eq. (bound-on-m), see
                          amg_degree_for; `degree` is then ignored              */
  int aggregation;     /* AMG_AGG_MATCHING: `passes` handshake matchings per
                          level.  AMG_AGG_MIS: Sec. 2 steps (A)-(B), one pass per
                          level: S = maximal independent set of the graph of
                          A^mis_k taken greedily in decreasing key order, key(v)
                          = ((splitmix64(salt ^ v) >> 33) + 1) << 32 | v; every
                          vertex joins its nearest root (graph distance, ties to
                          the larger key); aggregates numbered by root index   */
  int mis_k;           /* k of A^k for AMG_AGG_MIS, 1..16 (Sec. 4: 4)           */
} amg_options;

enum { AMG_CYCLE_K = 0, AMG_CYCLE_AMLI = 1 };
enum { AMG_AGG_MATCHING = 0, AMG_AGG_MIS = 1 };

/* Per-solve report (Sec. 4 reports iterations and grid/operator complexity). */
typedef struct {
  int iterations;             /* outer iterations (max over right-hand sides)      */
  int converged;              /* 1 if every right-hand side reached tol            */
  double rel_residual;        /* ||r_k|| / ||b|| of the recursive residual (max)   */
  double true_rel_residual;   /* ||b - A x|| / ||b|| recomputed at the end (max)   */
  int n_levels;
  double grid_complexity;     /* sum_k n_k / n_0                                   */
  double op_complexity;       /* sum_k nnz(A_k) / nnz(A_0), diagonal included     */
  double setup_ms;            /* wall time of amg_setup                            */
  double solve_ms;            /* wall time of this amg_solve call                  */
  double *history;            /* caller buffer (host) or NULL: ||r_k||/||b|| of the
                                 first right-hand side, k = 0, 1, ...              */
  int history_cap;
  int history_len;            /* entries written                                   */
} amg_info;

/* Fill *opt with defaults: degree 4, passes 3, coarse_max 64, max_levels 30,
 * inner_iters 2, restart 5, max_iters 500, FP64, lambda0_ratio 0.1, salt 0,
 * AMG_CYCLE_K, amli_alpha 0.25, rho 0, AMG_AGG_MATCHING, mis_k 4. */
void amg_default_options(amg_options *opt);

/* Smoother degree from Eq. (bound-on-m) (Sec. 3): the smallest m with
 * E_m = delta^m (kappa - 1)/2 <= rho and E_m < 1, where kappa =
 * 1/lambda0_ratio and delta = (sqrt(kappa) - 1)/(sqrt(kappa) + 1): the
 * smoother then damps [lambda0, lambda1] by at least rho and q_m stays
 * positive.  Returns -1 if rho <= 0, lambda0_ratio is outside (0, 1) or no
 * m <= 16 suffices.  Host only; needs no GPU. */
int amg_degree_for(double rho, double lambda0_ratio);

/*
 * Build the hierarchy on the device (Sec. 2-3; setup steps all run in CUDA
 * kernels: validation, connectivity, matching passes, Galerkin sums, lambda1
 * = ||A_k||_inf, the coarsest-level pseudo-inverse, the solve-phase layouts).
 *
 *  n            number of vertices, 1 <= n <= 2^31 - 2^16 (row indices are 32-bit)
 *  row_ptr      int64[n+1] CSR row offsets of the graph (row_ptr[0] = 0)
 *  col_idx      int32[nnz] neighbours; strictly increasing within each row;
 *               no self loops; the pattern is symmetric
 *  w            double[nnz] edge weights w_ij > 0, w_ij == w_ji exactly
 *  d            double[n] lower-order terms d_i >= 0, or NULL (pure Laplacian)
 *  opt          options or NULL for defaults
 *  mem_space    AMG_MEM_HOST: the four arrays are host memory;
 *               AMG_MEM_DEVICE: they are device pointers
 *  cuda_stream  cudaStream_t for all work of this handle (kept by the handle,
 *               not owned), or NULL for the legacy default stream
 *  out          receives the handle (NULL on failure)
 * Errors, checked in this order: AMG_ERR_INVALID_ARG (sizes, pointers,
 * options, row_ptr not monotone, column out of range or rows not strictly
 * increasing), AMG_ERR_SELF_LOOP, AMG_ERR_NOT_SYMMETRIC, AMG_ERR_BAD_WEIGHT,
 * AMG_ERR_DISCONNECTED, AMG_ERR_SETUP_STALL, AMG_ERR_OOM, AMG_ERR_CUDA.
 */
amg_status amg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *w,
                     const double *d, const amg_options *opt, int mem_space, void *cuda_stream,
                     amg_handle *out);

/*
 * Solve A x = rhs for nrhs right-hand sides by flexible CG (Sec. 4: NPCG,
 * window cleared every `restart` iterations) preconditioned by the handle's
 * cycle (option `cycle`), from x0 = 0, until ||r_k|| <= tol ||b|| (recursive
 * residual, fp64).
 *
 *  rhs, x   column j at rhs + j*ld, x + j*ld (column major, ld >= n); host or
 *           device memory (each pointer classified independently); x is
 *           output only.  For a pure Laplacian each right-hand side is first
 *           projected to zero mean (the range of A is 1-perp, Sec. 1) and x is
 *           returned with zero mean.
 *  nrhs     >= 1; several right-hand sides are solved together, the
 *           preconditioner applied to all of them in one multi-vector pass
 *  info     optional report (may be NULL)
 * Returns AMG_OK, AMG_ERR_NOT_CONVERGED (x holds the last iterate),
 * AMG_ERR_BREAKDOWN, AMG_ERR_INVALID_ARG (also when a right-hand side has a
 * NaN or infinite entry, or a norm beyond the fp64 range; x is then
 * unspecified) or AMG_ERR_CUDA.
 */
amg_status amg_solve(amg_handle h, const double *rhs, double *x, int nrhs, int64_t ld, double tol,
                     amg_info *info);

/* Release the hierarchy and every device buffer of h (NULL is a no-op). */
void amg_free(amg_handle h);

/* Description of the last error of h, or of the calling thread's last
 * failed amg_setup/amg_match when h is NULL.  Owned by the library. */
const char *amg_last_error(amg_handle h);

/* ---------------------------------------------------------------------- */
/* Introspection: copies of the device hierarchy into caller host buffers. */
/* ---------------------------------------------------------------------- */

int amg_num_levels(amg_handle h);
/* vertices of level k, -1 if k is out of range */
int64_t amg_level_n(amg_handle h, int k);
/* stored off-diagonal entries of level k (each undirected edge twice) */
int64_t amg_level_nnz(amg_handle h, int k);
/* Level k operator A_k = P^T A_{k-1} P in CSR: rowptr[n+1], col[nnz] (strictly
 * increasing per row), val[nnz] = off-diagonal a_ij = -W_ij, diag[n] = A_ii,
 * dlow[n] = the lower-order term aggregated to this level (P^T d).  Any output
 * pointer may be NULL.  Host buffers. */
amg_status amg_level_csr(amg_handle h, int k, int64_t *rowptr, int32_t *col, double *val,
                         double *diag, double *dlow);
/* Composite aggregate map level k -> k+1 (k < levels-1): agg[n_k] in [0, n_{k+1}).
 * Coarse ids rank the aggregates' smallest members (AMG_AGG_MATCHING) or their
 * roots (AMG_AGG_MIS).  Host buffer. */
amg_status amg_level_agg(amg_handle h, int k, int32_t *agg);
/* Smoother data of level k < levels-1: lambda0, lambda1 = ||A_k||_inf and the
 * m+1 Chebyshev coefficients of q_m in t = (2x - l1 - l0)/(l1 - l0), m the
 * handle's degree (amg_degree_for(rho, lambda0_ratio) when rho > 0).
 * Any output pointer may be NULL. */
amg_status amg_level_smoother(amg_handle h, int k, double *lam0, double *lam1, double *coef);

/* ---------------------------------------------------------------------- */
/* Single steps of the solve phase on one level (device fp64 vectors).     */
/* In AMG_PREC_FP32 mode the level data used are the fp32 copies; vectors */
/* are converted on entry and exit.  These run on the handle's stream and  */
/* return after completion.                                                */
/* ---------------------------------------------------------------------- */

/* y = A_k x (Eq. (1) operator on level k). */
amg_status amg_apply_spmv(amg_handle h, int k, const double *x, double *y);
/* x = q_m(A_k) r by the Chebyshev three-term recurrence T_0 = r,
 * T_1 = t(A) r, T_{j+1} = 2 t(A) T_j - T_{j-1}, x = sum_j c_j T_j (Sec. 3
 * smoother R = q_m(A)); k < levels-1. */
amg_status amg_apply_smoother(amg_handle h, int k, const double *r, double *x);
/* r_H = P_k^T s: sum over each aggregate's members (Eq. (coarse)). */
amg_status amg_apply_restrict(amg_handle h, int k, const double *s, double *rH);
/* x += P_k e_H: every vertex adds its aggregate's value (Eq. (coarse)). */
amg_status amg_apply_prolong_add(amg_handle h, int k, const double *eH, double *x);
/* x = A_c^+ b on the coarsest level (Sec. 3: pseudo-inverse), fp64. */
amg_status amg_apply_coarse_solve(amg_handle h, const double *b, double *x);
/* z = K_k(r): one application of the handle's cycle at level k (pre-smooth,
 * residual, restriction, then nu inner flexible-CG steps (AMG_CYCLE_K) or
 * the AMLI polynomial (AMG_CYCLE_AMLI) or the coarsest solve, prolongation,
 * residual, post-smooth). */
amg_status amg_apply_kcycle(amg_handle h, int k, const double *r, double *z);

/* One handshake matching pass (Sec. 2) on a device CSR graph whose entries
 * carry matching weights s (double[nnz] > 0, symmetric); edge keys are
 * (s_ij, splitmix64(salt ^ (lo << 32 | hi)), lo, hi), largest wins.
 * Outputs (device): mate[n] (-1 unmatched), agg[n] coarse ids (rank of each
 * pair's smaller vertex / singleton); *n_coarse and *rounds (host) receive the
 * coarse size and the number of proposal rounds.  1 <= n <= 2^31 - 2^16.
 * row_ptr, col_idx, s, mate and agg must be non-NULL (AMG_ERR_INVALID_ARG);
 * a round limit of 4n + 8 guards against non-symmetric or non-finite s
 * (AMG_ERR_INVALID_ARG).  stream may be NULL. */
amg_status amg_match(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *s,
                     uint64_t salt, int32_t *mate, int32_t *agg, int64_t *n_coarse, int *rounds,
                     void *cuda_stream);

/* The same matching pass as amg_match, but allocation-free.  The paper has
 * no counterpart: this entry point exists for callers that may not allocate
 * device memory themselves (their memory belongs to another allocator, such
 * as a framework's caching allocator holding the GPU's free memory, or they
 * must avoid the device-wide synchronisation of cudaFree mid-pipeline).
 * Scratch lives in one fixed device array inside the library (4 MiB per GPU
 * that loads the library, kept until the process exits), so:
 *  - n must be <= 1048576 (2^20); larger n returns AMG_ERR_INVALID_ARG;
 *  - no cudaMalloc/cudaFree or allocating library routine is called;
 *  - every call looks up that array's device address for the current device
 *    (a host-side lookup) and waits for its own work on `cuda_stream`
 *    (stream synchronisation between batches of rounds and before return);
 *  - every process holds its own copy of the array, and all calls of one
 *    process on a device share it: calls from different streams or threads
 *    of one process that overlap on the GPU race and must be serialised by
 *    the caller.
 * Arguments, outputs and results are those of amg_match. */
amg_status amg_match_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             const double *s, uint64_t salt, int32_t *mate, int32_t *agg,
                             int64_t *n_coarse, int *rounds, void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Serving (not in the paper: a request loop around amg_setup/amg_solve).  */
/*                                                                        */
/* Continuous batching on one GPU: registered graphs keep their hierarchy */
/* resident; work is admitted as soon as one of `max_active` slots and    */
/* device memory under `mem_cap_bytes` are free (idle hierarchies are     */
/* evicted least-recently-used first).  A slot takes the oldest queued    */
/* request whose graph is idle together with the other queued requests   */
/* for that graph and tolerance, up to `batch_max`, and solves them in    */
/* one multi-right-hand-side call (one sweep over the levels serves the   */
/* whole batch); solves of different graphs run concurrently on their own */
/* streams.  A lone request runs the single-right-hand-side path; a batch */
/* runs the block kernels at the smallest power-of-two width that holds   */
/* it, with per-column Krylov scalars, so every request meets its own     */
/* tolerance whatever shares its block (results alone and in a batch     */
/* agree to that tolerance, not bit for bit); with batch_max 0 or 1       */
/* requests for one graph take turns on the single-right-hand-side path   */
/* and results are bit-identical alone and in the mix.  Block buffers for */
/* batch_max columns are made at setup.  A hierarchy's size is its arena  */
/* bytes,                                                                 */
/* measured at its first setup (estimated from n and nnz before that); a  */
/* setup whose measured size does not fit beside the busy hierarchies     */
/* gives its memory back and its requests are queued again (counted in    */
/* setup_retries), so resident bytes stay under the cap; a request whose  */
/* hierarchy alone exceeds mem_cap_bytes completes with AMG_ERR_OOM.      */
/* All pointers are host memory; the server copies what it needs.         */
/* ---------------------------------------------------------------------- */

typedef struct amg_server_s *amg_server;

typedef struct {
  size_t mem_cap_bytes;  /* device bytes for resident hierarchies (>= 1 MiB) */
  int max_active;        /* concurrent solves, 1..64                         */
  int batch_max;         /* requests of one graph solved together, 0..32
                            (0, 1: no batching)                              */
  amg_options opt;       /* solver options of every request                  */
} amg_server_config;

typedef struct {
  /* resident_bytes counts resident hierarchies plus reservations of setups
   * in progress; peak_resident_bytes is the largest total of resident
   * hierarchies' measured sizes */
  size_t resident_bytes, peak_resident_bytes;
  int active, peak_active;
  int64_t queued, completed, setups, evictions;
  int64_t solves;         /* solve calls; completed / solves = mean batch size */
  int64_t setup_retries;  /* setups redone to keep resident bytes under the cap */
} amg_server_stats_t;

amg_status amg_server_create(const amg_server_config *cfg, amg_server *out);
/* register a graph (arguments as amg_setup with host memory); the hierarchy
 * is built by the first request that needs it */
amg_status amg_server_add_graph(amg_server s, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                const double *w, const double *d, int64_t *graph_id);
/* queue one right-hand side (n doubles) for graph_id; *ticket identifies it.
 * A right-hand side with a non-finite entry (or whose norm overflows) is
 * refused with AMG_ERR_INVALID_ARG. */
amg_status amg_server_submit(amg_server s, int64_t graph_id, const double *rhs, double tol, int64_t *ticket);
/* *done = 0 while the request runs; once done, copies the solution into x
 * (n doubles, may be NULL), the report into info (history not filled), the
 * submit-to-finish latency into *latency_ms, releases the ticket and returns
 * the solve's status */
amg_status amg_server_poll(amg_server s, int64_t ticket, double *x, amg_info *info, int *done,
                           double *latency_ms);
/* as amg_server_poll, blocking until the request is done; AMG_ERR_INVALID_ARG
 * if another caller takes the same ticket first */
amg_status amg_server_wait(amg_server s, int64_t ticket, double *x, amg_info *info, double *latency_ms);
amg_status amg_server_stats(amg_server s, amg_server_stats_t *out);
/* stops the workers after their current solves and frees every hierarchy;
 * requests still queued are dropped.  No other call on s may be in progress
 * (a blocked amg_server_wait included) or follow. */
void amg_server_destroy(amg_server s);

/* ---------------------------------------------------------------------- */
/* Measurement hooks.                                                      */
/* ---------------------------------------------------------------------- */

/* Enable (1) or disable (0) CUDA-event timing, during amg_solve, of every
 * launch on level 0 of the fused smoother-step kernel (the dominant kernel),
 * of the restriction and of the prolongation when it runs as its own kernel;
 * enabling resets the accumulators. */
amg_status amg_kernel_timing(amg_handle h, int enable);
/* Accumulated launches, total device milliseconds and the algorithmic bytes
 * of one launch: nnz (v + 4) + 8 (slices + 1) + 6 n v for level 0 (stored
 * values and columns, slice offsets, the diagonal, T_j, T_{j-1}, T_{j+1} and
 * x read and written once; v = 8, or 4 for AMG_PREC_FP32). */
amg_status amg_kernel_timing_read(amg_handle h, int64_t *launches, double *total_ms,
                                  double *bytes_per_launch);
/* The same for `kind` 0 (the smoother step, as amg_kernel_timing_read), 1
 * (the level-0 restriction r_H = P^T s of Eq. (coarse); bytes: its member
 * lists, s and r_H once) or 2 (the level-0 prolongation x = u + P e_H;
 * bytes: n (4 + 2 v) + n_H v).  AMG_ERR_INVALID_ARG for another kind. */
amg_status amg_kernel_timing_read_kind(amg_handle h, int kind, int64_t *launches, double *total_ms,
                                       double *bytes_per_launch);
/* Number of kernel launches issued by the last amg_setup/amg_solve on h. */
int64_t amg_launch_count(amg_handle h);

#ifdef __cplusplus
}
#endif
#endif
