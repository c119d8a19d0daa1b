/*
 * amg_oracle.h -- plain, slow, single-threaded FP64 CPU oracle for the
 * aggregation AMG solve phase of Brannick, "Aggregation-based aggressive
 * coarsening with polynomial smoothing" (flexible CG preconditioned by a
 * nonlinear AMLI / K-cycle over unsmoothed aggregation, polynomial smoother).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA library: every step here is written from the paper's definitions
 * (section / equation cited beside each function in amg_oracle.c).
 *
 * Parity unpinned: the iteration counts of the full matching-based K-cycle on
 * large graphs have no paper value to compare with (the paper's table uses a
 * different aggregation); they are pinned only through the small-graph checks
 * (exact solves, two-level operator identities) exercised by the tests.
 */
#ifndef AMG_ORACLE_H
#define AMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (same numbering as the library's) */
enum {
  ORC_OK = 0,
  ORC_ERR_INVALID_ARG = 1,
  ORC_ERR_NOT_SYMMETRIC = 2,
  ORC_ERR_SELF_LOOP = 3,
  ORC_ERR_BAD_WEIGHT = 4,
  ORC_ERR_DISCONNECTED = 5,
  ORC_ERR_OOM = 6,
  ORC_ERR_NOT_CONVERGED = 8,
  ORC_ERR_BREAKDOWN = 9,
  ORC_ERR_SETUP_STALL = 11
};

/* preconditioner choices for the outer flexible CG */
enum { ORC_PREC_KCYCLE = 0, ORC_PREC_IDENTITY = 1, ORC_PREC_EXACT = 2 };
/* multilevel cycle behind ORC_PREC_KCYCLE: the nonlinear AMLI cycle (K-cycle,
 * inner flexible CG on coarse levels) or the stationary AMLI W-cycle (a fixed
 * polynomial in B_{k+1} A_{k+1} on coarse levels), Sec. 4 */
enum { ORC_CYCLE_K = 0, ORC_CYCLE_AMLI = 1 };

typedef struct {
  int degree;          /* m, degree of the smoothing polynomial q_m          */
  int passes;          /* matching passes composed into one level             */
  int coarse_max;      /* stop coarsening once n_k <= coarse_max              */
  int max_levels;      /* hard cap on the number of levels                    */
  int inner_iters;     /* nu, inner flexible-CG steps on coarse levels        */
  int restart;         /* outer window cleared every `restart` iterations     */
  int max_iters;       /* outer iteration cap                                 */
  int precond;         /* ORC_PREC_*                                          */
  double lambda0_ratio;/* lambda0 = ratio * lambda1                           */
  uint64_t hash_salt;  /* salt of the matching tie-break hash                 */
  int cycle;           /* ORC_CYCLE_K or ORC_CYCLE_AMLI                       */
  double amli_alpha;   /* AMLI polynomial: best approximation to 1/t on
                          [amli_alpha, 1], degree nu - 1; its error
                          delta^(nu-1) (1/alpha - 1)/2 must be < 1 (0.25)     */
  double rho;          /* > 0: degree m from Eq. (bound-on-m) for damping rho;
                          `degree` is then ignored                            */
  int aggregation;     /* ORC_AGG_MATCHING (`passes` handshake matchings per
                          level) or ORC_AGG_MIS (Sec. 2: maximal independent
                          set of the graph of A^k, one pass per level)        */
  int mis_k;           /* k of A^k for ORC_AGG_MIS (Sec. 4 uses 4)            */
} orc_options;

enum { ORC_AGG_MATCHING = 0, ORC_AGG_MIS = 1 };

typedef struct {
  int iterations;
  int converged;
  double rel_residual;       /* recursive ||r_k|| / ||b||                 */
  double true_rel_residual;  /* ||b - A x|| / ||b||                       */
  int n_levels;
  double grid_complexity;
  double op_complexity;
  double *history;           /* caller buffer, ||r_k||/||b||, k = 0..    */
  int history_cap;
  int history_len;
} orc_info;

typedef struct orc_hier orc_hier;

void orc_default_options(orc_options *o);

/* ---- standalone building blocks -------------------------------------- */

/* One handshake matching pass on a weighted graph given as off-diagonal
 * CSR with positive weights w.  Outputs mate[n] (-1 = unmatched), agg[n]
 * (coarse id of each vertex), returns the number of coarse vertices; *rounds
 * receives the number of proposal rounds executed (last one adds nothing). */
/* Aggregation of Sec. 2 (steps A and B): S = the maximal independent set of
 * the graph of A^k (vertices at graph distance <= k adjacent) taken greedily
 * in decreasing key order, key(v) = ((splitmix64(salt ^ v) >> 33) + 1) << 32
 * | v; then every vertex joins its nearest root (graph distance, ties to the
 * larger root key).  Aggregates are numbered by their roots' vertex order.
 * Writes agg[n] and root[n] (1 for roots); returns the number of aggregates. */
int orc_mis_aggregate(int n, const int64_t *rowptr, const int32_t *col, int k, uint64_t salt,
                      int32_t *agg, int32_t *root);
int orc_match(int n, const int64_t *rowptr, const int32_t *col, const double *w,
              uint64_t salt, int32_t *mate, int32_t *agg, int *rounds);

/* Chebyshev coefficients c[0..m] (variable t = (2x - l1 - l0)/(l1 - l0)) of
 * the polynomial of best uniform approximation to 1/x on [l0, l1], by the
 * Remez exchange; *err = max |1/x - q_m(x)| on [l0,l1]; alt[0..m+1] receives
 * the final reference (alternation) points. Returns 0 on success. */
int orc_remez_inverse(int m, double l0, double l1, double *c, double *err, double *alt);

/* Cyclic Jacobi eigen-decomposition of a dense symmetric n x n matrix
 * (row major).  evals[n], evecs (n x n, column k = eigenvector k). */
int orc_jacobi_eigen(int n, const double *A, double *evals, double *evecs);

/* ---- hierarchy ----------------------------------------------------------- */

int orc_setup(int64_t n, const int64_t *rowptr, const int32_t *col, const double *w,
              const double *d, const orc_options *opt, orc_hier **out);
int orc_solve(orc_hier *h, const double *b, double *x, double tol, orc_info *info);
void orc_free(orc_hier *h);

int orc_num_levels(const orc_hier *h);
int64_t orc_level_n(const orc_hier *h, int k);
int64_t orc_level_nnz(const orc_hier *h, int k);  /* off-diagonal entries */
/* copy out level k: rowptr[n+1], col[nnz], val[nnz] (off-diagonal a_ij),
 * diag[n], dlow[n] (aggregated lower-order term); any pointer may be NULL */
int orc_level_csr(const orc_hier *h, int k, int64_t *rowptr, int32_t *col, double *val,
                  double *diag, double *dlow);
/* composite aggregate map of level k -> level k+1 (k < L-1) */
int orc_level_agg(const orc_hier *h, int k, int32_t *agg);
/* per-pass maps of level k: pass p map (length = size before the pass) */
int orc_level_pass_count(const orc_hier *h, int k);
int64_t orc_level_pass_n(const orc_hier *h, int k, int p);
int orc_level_pass_agg(const orc_hier *h, int k, int p, int32_t *agg);
int orc_level_lambda(const orc_hier *h, int k, double *lam0, double *lam1);
int orc_level_cheb(const orc_hier *h, int k, double *coef);

/* operations on the hierarchy (fp64, plain loops) */
int orc_spmv(const orc_hier *h, int k, const double *x, double *y);
int orc_smooth(const orc_hier *h, int k, const double *r, double *x);      /* x = q_m(A_k) r */
int orc_restrict(const orc_hier *h, int k, const double *s, double *rH);   /* rH = P^T s     */
int orc_prolong_add(const orc_hier *h, int k, const double *eH, double *x);/* x += P eH      */
int orc_coarse_solve(const orc_hier *h, const double *b, double *x);       /* x = A_c^+ b    */
int orc_kcycle(const orc_hier *h, int k, const double *r, double *x);      /* x = K_k(r)     */
int orc_amli_cycle(const orc_hier *h, int k, const double *r, double *x);  /* x = B_k r      */
/* Chebyshev coefficients (nu entries) of the AMLI polynomial on [alpha, 1] */
int orc_amli_coef(const orc_hier *h, double *coef);
/* smallest m with E_m = delta^m (kappa - 1)/2 <= rho and E_m < 1,
 * kappa = 1 / lambda0_ratio (Eq. bound-on-m); -1 if none up to 30 */
int orc_degree_for(double rho, double lambda0_ratio);
int orc_inner_fcg(const orc_hier *h, int k, const double *b, double *x);   /* nu steps       */

#ifdef __cplusplus
}
#endif
#endif
