/*
 * amg_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * amg_oracle.h).  Single threaded, no blocking, no fusion: each function
 * states the definition it follows, cited by the paper's section/equation.
 *
 * Notation (paper, Sec. 1-3):
 *   A      graph Laplacian plus lower-order term, Eq. (1):
 *          (Au,v) = sum_e w_e (du)(dv) + sum_i d_i u_i v_i,
 *          so A_ii = sum_j w_ij + d_i and A_ij = -w_ij.
 *   P      piecewise-constant prolongation of a partition into aggregates,
 *          Eq. (coarse): column l is the indicator 1_l of aggregate l.
 *   A_H    Galerkin operator P^T A P (Sec. 3, remark after the spectral
 *          equivalence): entries are sums of fine entries over aggregate pairs.
 *   q_m    polynomial of best uniform approximation to 1/x on
 *          [lambda0, lambda1], Eq. (1x-1-min); R = q_m(A) is the smoother,
 *          lambda1 = ||A||_inf, lambda0 = lambda1/10 (Sec. 4).
 *   cycle  nonlinear AMLI (K-cycle): W(1,1) with flexible CG applied
 *          recursively on coarse levels, outer flexible CG restarted every
 *          five iterations (Sec. 4).
 * Built with -ffp-contract=off so results do not depend on the host's FMA.
 */
#include "amg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 64
#define ORC_STALL_RATIO 0.95
#define ORC_STALL_MAX_COARSE 4096

typedef struct {
  int64_t n;
  int64_t *rowptr;
  int32_t *col;
  double *val;  /* off-diagonal entries a_ij = -w_ij */
  double *diag; /* A_ii */
  double *dlow; /* lower-order term d_i carried to this level */
} orc_mat;

typedef struct {
  orc_mat A;
  int32_t *agg; /* composite aggregate map to the next level */
  int64_t nH;
  int npass;
  int64_t pass_n[16];
  int32_t *pass_agg[16];
  double lam0, lam1;
  double *cheb; /* m+1 Chebyshev coefficients of q_m */
} orc_level;

struct orc_hier {
  orc_options opt;
  int L;
  orc_level lv[ORC_MAX_LEVELS];
  int pure;
  /* coarsest level: eigen-decomposition for the pseudo-inverse */
  int64_t nc;
  double *c_ev;
  double *c_U;
  /* dense eigen-decomposition of A_0 for ORC_PREC_EXACT */
  double *x_ev;
  double *x_U;
  /* stationary AMLI cycle: Chebyshev coefficients of q_{nu-1} on [alpha, 1] */
  double amli_cheb[64];
};

void orc_default_options(orc_options *o) {
  o->degree = 4;
  o->passes = 3;
  o->coarse_max = 64;
  o->max_levels = 30;
  o->inner_iters = 2;
  o->restart = 5;
  o->max_iters = 500;
  o->precond = ORC_PREC_KCYCLE;
  o->lambda0_ratio = 0.1;
  o->hash_salt = 0;
  o->cycle = ORC_CYCLE_K;
  o->amli_alpha = 0.25;
  o->rho = 0.0;
  o->aggregation = ORC_AGG_MATCHING;
  o->mis_k = 4;
}

/* ------------------------------------------------------------------ */
/* vectors                                                             */
/* ------------------------------------------------------------------ */
static double *vnew(int64_t n) { return (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)); }
static double *vzeros(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }
static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* y = A x with A = diag + off-diagonal CSR */
static void mat_spmv(const orc_mat *A, const double *x, double *y) {
  for (int64_t i = 0; i < A->n; ++i) {
    double s = A->diag[i] * x[i];
    for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) s += A->val[p] * x[A->col[p]];
    y[i] = s;
  }
}

static void mat_free(orc_mat *A) {
  free(A->rowptr);
  free(A->col);
  free(A->val);
  free(A->diag);
  free(A->dlow);
  memset(A, 0, sizeof(*A));
}

/* ------------------------------------------------------------------ */
/* input validation (order: row pointers, column range, sorted rows,   */
/* self loops, symmetry, weights, lower-order terms)                   */
/* ------------------------------------------------------------------ */
static int find_in_row(const int64_t *rowptr, const int32_t *col, int64_t row, int32_t key) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == key) return (int)(mid - rowptr[row]);
    if (col[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int validate(int64_t n, const int64_t *rowptr, const int32_t *col, const double *w,
                    const double *d) {
  if (n < 1 || !rowptr) return ORC_ERR_INVALID_ARG;
  if (rowptr[0] != 0) return ORC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return ORC_ERR_INVALID_ARG;
  int64_t nnz = rowptr[n];
  if (nnz > 0 && (!col || !w)) return ORC_ERR_INVALID_ARG;
  for (int64_t p = 0; p < nnz; ++p)
    if (col[p] < 0 || col[p] >= n) return ORC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i] + 1; p < rowptr[i + 1]; ++p)
      if (col[p] <= col[p - 1]) return ORC_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (col[p] == i) return ORC_ERR_SELF_LOOP;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int q = find_in_row(rowptr, col, col[p], (int32_t)i);
      if (q < 0 || w[rowptr[col[p]] + q] != w[p]) return ORC_ERR_NOT_SYMMETRIC;
    }
  for (int64_t p = 0; p < nnz; ++p)
    if (!(w[p] > 0.0) || !isfinite(w[p])) return ORC_ERR_BAD_WEIGHT;
  if (d)
    for (int64_t i = 0; i < n; ++i)
      if (!(d[i] >= 0.0) || !isfinite(d[i])) return ORC_ERR_BAD_WEIGHT;
  return ORC_OK;
}

/* Connectivity (Sec. 1: G is connected, so the pure Laplacian's kernel is
 * the constants).  Breadth-first search over components: a pure Laplacian
 * must be connected; with lower-order terms every component needs some d_i>0
 * for A to be nonsingular. */
static int check_components(int64_t n, const int64_t *rowptr, const int32_t *col, const double *d,
                            int pure) {
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!comp || !queue) { free(comp); free(queue); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < n; ++i) comp[i] = -1;
  int ncomp = 0, status = ORC_OK;
  for (int64_t s = 0; s < n && status == ORC_OK; ++s) {
    if (comp[s] >= 0) continue;
    int64_t head = 0, tail = 0;
    double dsum = 0.0;
    queue[tail++] = s;
    comp[s] = ncomp;
    while (head < tail) {
      int64_t v = queue[head++];
      if (d) dsum += d[v];
      for (int64_t p = rowptr[v]; p < rowptr[v + 1]; ++p)
        if (comp[col[p]] < 0) { comp[col[p]] = ncomp; queue[tail++] = col[p]; }
    }
    ++ncomp;
    if (pure && ncomp > 1) status = ORC_ERR_DISCONNECTED;
    if (!pure && !(dsum > 0.0)) status = ORC_ERR_DISCONNECTED;
  }
  free(comp);
  free(queue);
  return status;
}

/* ------------------------------------------------------------------ */
/* Matching (Sec. 2: a matching is a set of pairwise non-incident edges; */
/* each matched edge becomes a two-vertex aggregate, unmatched vertices  */
/* stay singletons).                                                     */
/*                                                                       */
/* Rule: every edge {i,j}, lo = min, hi = max, has the key               */
/*   (s_ij, h, lo, hi), h = splitmix64(salt ^ (lo << 32 | hi)),          */
/* where s_ij is the edge's matching weight (the level builder passes    */
/* the strength |a_ij| / sqrt(a_ii a_jj)),                               */
/* compared lexicographically, larger winning.  In each round every      */
/* unmatched vertex points at the unmatched neighbour across its         */
/* largest-key edge; two vertices pointing at each other are matched.    */
/* Rounds repeat until one adds no pair (the largest remaining edge is   */
/* always mutual, so the result is a maximal matching).  Coarse ids:     */
/* a vertex is a representative if it is unmatched or the smaller end of */
/* its pair; the id of an aggregate is the rank of its representative.   */
/* ------------------------------------------------------------------ */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* 1 if edge a = (wa, lo_a, hi_a) has a larger key than edge b */
static int key_greater(double wa, int64_t la, int64_t ha, double wb, int64_t lb, int64_t hb,
                       uint64_t salt) {
  if (wa != wb) return wa > wb;
  uint64_t xa = splitmix64(salt ^ (((uint64_t)la << 32) | (uint64_t)ha));
  uint64_t xb = splitmix64(salt ^ (((uint64_t)lb << 32) | (uint64_t)hb));
  if (xa != xb) return xa > xb;
  if (la != lb) return la > lb;
  return ha > hb;
}

int orc_match(int n, const int64_t *rowptr, const int32_t *col, const double *w, uint64_t salt,
              int32_t *mate, int32_t *agg, int *rounds) {
  int32_t *ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!ptr) return -1;
  for (int i = 0; i < n; ++i) mate[i] = -1;
  int nr = 0;
  for (;;) {
    ++nr;
    for (int i = 0; i < n; ++i) {
      ptr[i] = -1;
      if (mate[i] >= 0) continue;
      int best = -1;
      double bw = 0.0;
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        if (mate[j] >= 0) continue;
        int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        if (best < 0) { best = j; bw = w[p]; continue; }
        int64_t blo = i < best ? i : best, bhi = i < best ? best : i;
        if (key_greater(w[p], lo, hi, bw, blo, bhi, salt)) { best = j; bw = w[p]; }
      }
      ptr[i] = best;
    }
    int added = 0;
    for (int i = 0; i < n; ++i)
      if (ptr[i] >= 0 && ptr[ptr[i]] == i) { mate[i] = ptr[i]; ++added; }
    if (!added) break;
  }
  free(ptr);
  if (rounds) *rounds = nr;
  /* representative ranks */
  int nH = 0;
  for (int i = 0; i < n; ++i)
    if (mate[i] < 0 || i < mate[i]) agg[i] = nH++;
  for (int i = 0; i < n; ++i)
    if (mate[i] >= 0 && mate[i] < i) agg[i] = agg[mate[i]];
  return nH;
}

/* ------------------------------------------------------------------ */
/* Aggregation by a maximal independent set of the graph of A^k (Sec. 2, */
/* steps (A) and (B); Sec. 4 applies it with k = 4).                     */
/* ------------------------------------------------------------------ */
static uint64_t mis_key(uint64_t salt, int v) {
  return (((splitmix64(salt ^ (uint64_t)v) >> 33) + 1) << 32) | (uint64_t)(uint32_t)v;
}

/* breadth-first distances from src, up to depth k (-1: farther) */
static void bfs_limited(int n, const int64_t *rowptr, const int32_t *col, int src, int k, int *dist,
                        int *queue, int *visited, int *nvis) {
  int head = 0, tail = 0;
  dist[src] = 0;
  queue[tail++] = src;
  visited[(*nvis)++] = src;
  while (head < tail) {
    int u = queue[head++];
    if (dist[u] == k) continue;
    for (int64_t p = rowptr[u]; p < rowptr[u + 1]; ++p) {
      int v = col[p];
      if (dist[v] < 0) {
        dist[v] = dist[u] + 1;
        queue[tail++] = v;
        visited[(*nvis)++] = v;
      }
    }
  }
  (void)n;
}

static int cmp_key_desc(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x < y) - (x > y);
}

int orc_mis_aggregate(int n, const int64_t *rowptr, const int32_t *col, int k, uint64_t salt,
                      int32_t *agg, int32_t *root) {
  if (n < 1 || k < 1) return -1;
  uint64_t *order = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  int *dist = (int *)malloc(sizeof(int) * (size_t)n), *queue = (int *)malloc(sizeof(int) * (size_t)n);
  int *vis = (int *)malloc(sizeof(int) * (size_t)n);
  char *blocked = (char *)calloc((size_t)n, 1);
  for (int v = 0; v < n; ++v) { order[v] = mis_key(salt, v); dist[v] = -1; root[v] = 0; }
  qsort(order, (size_t)n, sizeof(uint64_t), cmp_key_desc);
  /* (A) greedy: a vertex not within distance k of an earlier root becomes one */
  for (int a = 0; a < n; ++a) {
    int v = (int)(uint32_t)order[a];
    if (blocked[v]) continue;
    root[v] = 1;
    int nvis = 0;
    bfs_limited(n, rowptr, col, v, k, dist, queue, vis, &nvis);
    for (int t = 0; t < nvis; ++t) { blocked[vis[t]] = 1; dist[vis[t]] = -1; }
  }
  /* (B) nearest root, ties to the larger key: grow all roots together one
   * layer at a time; a vertex reached in layer t takes the largest label
   * among its neighbours labelled in earlier layers */
  uint64_t *lab = (uint64_t *)calloc((size_t)n, sizeof(uint64_t));
  uint64_t *nxt = (uint64_t *)calloc((size_t)n, sizeof(uint64_t));
  for (int v = 0; v < n; ++v) if (root[v]) lab[v] = mis_key(salt, v);
  for (int layer = 1; layer <= k; ++layer) {
    memcpy(nxt, lab, sizeof(uint64_t) * (size_t)n);
    for (int v = 0; v < n; ++v) {
      if (lab[v]) continue;
      uint64_t best = 0;
      for (int64_t p = rowptr[v]; p < rowptr[v + 1]; ++p)
        if (lab[col[p]] > best) best = lab[col[p]];
      nxt[v] = best;
    }
    memcpy(lab, nxt, sizeof(uint64_t) * (size_t)n);
  }
  /* aggregate ids: roots ranked by vertex index */
  int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int nH = 0;
  for (int v = 0; v < n; ++v) rank[v] = root[v] ? nH++ : -1;
  int ok = 1;
  for (int v = 0; v < n; ++v) {
    if (!lab[v]) { ok = 0; break; } /* cannot happen: S is maximal */
    agg[v] = rank[(int)(uint32_t)lab[v]];
  }
  free(order); free(dist); free(queue); free(vis); free(blocked); free(lab); free(nxt); free(rank);
  return ok ? nH : -1;
}

/* ------------------------------------------------------------------ */
/* Galerkin operator A_H = P^T A P for piecewise-constant P (Sec. 3     */
/* remark: A_H is again a weighted graph Laplacian; Sec. 5: the triple  */
/* product reduces to sums of fine entries).  For aggregates I != J:    */
/*   W_IJ = sum_{i in I, j in J} w_ij,   d_I = sum_{i in I} d_i,        */
/*   (A_H)_IJ = -W_IJ,  (A_H)_II = sum_{J != I} W_IJ + d_I.             */
/* Sums run over members in ascending order, each member's row in CSR   */
/* order.                                                               */
/* ------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static int galerkin(const orc_mat *A, const int32_t *agg, int64_t nH, orc_mat *AH) {
  int64_t n = A->n;
  int64_t *mptr = (int64_t *)calloc((size_t)nH + 1, sizeof(int64_t));
  int64_t *mem = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)nH);
  if (!mptr || !mem || !slot) return ORC_ERR_OOM;
  for (int64_t i = 0; i < n; ++i) mptr[agg[i] + 1]++;
  for (int64_t I = 0; I < nH; ++I) mptr[I + 1] += mptr[I];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nH);
    for (int64_t I = 0; I < nH; ++I) fill[I] = mptr[I];
    for (int64_t i = 0; i < n; ++i) mem[fill[agg[i]]++] = i; /* ascending i */
    free(fill);
  }
  for (int64_t I = 0; I < nH; ++I) slot[I] = -1;
  /* pass 1: count distinct neighbouring aggregates */
  AH->n = nH;
  AH->rowptr = (int64_t *)calloc((size_t)nH + 1, sizeof(int64_t));
  int64_t maxrow = 0;
  for (int64_t I = 0; I < nH; ++I) {
    int64_t cnt = 0;
    for (int64_t m = mptr[I]; m < mptr[I + 1]; ++m) {
      int64_t i = mem[m];
      for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
        int32_t J = agg[A->col[p]];
        if (J == I || slot[J] == I) continue;
        slot[J] = I;
        ++cnt;
      }
    }
    AH->rowptr[I + 1] = AH->rowptr[I] + cnt;
    if (cnt > maxrow) maxrow = cnt;
  }
  int64_t nnzH = AH->rowptr[nH];
  AH->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnzH > 0 ? nnzH : 1));
  AH->val = (double *)malloc(sizeof(double) * (size_t)(nnzH > 0 ? nnzH : 1));
  AH->diag = vnew(nH);
  AH->dlow = vnew(nH);
  double *acc = vzeros(nH);
  int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxrow > 0 ? maxrow : 1));
  for (int64_t I = 0; I < nH; ++I) slot[I] = -1;
  /* pass 2: accumulate W_IJ, emit columns in ascending order */
  for (int64_t I = 0; I < nH; ++I) {
    int64_t cnt = 0;
    double dI = 0.0;
    for (int64_t m = mptr[I]; m < mptr[I + 1]; ++m) {
      int64_t i = mem[m];
      dI += A->dlow[i];
      for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) {
        int32_t J = agg[A->col[p]];
        if (J == I) continue;
        if (slot[J] != I) { slot[J] = I; acc[J] = 0.0; cols[cnt++] = J; }
        acc[J] += -A->val[p]; /* w_ij */
      }
    }
    qsort(cols, (size_t)cnt, sizeof(int32_t), cmp_i32);
    double wsum = 0.0;
    for (int64_t c = 0; c < cnt; ++c) {
      AH->col[AH->rowptr[I] + c] = cols[c];
      AH->val[AH->rowptr[I] + c] = -acc[cols[c]];
      wsum += acc[cols[c]];
    }
    AH->dlow[I] = dI;
    AH->diag[I] = wsum + dI;
  }
  free(acc);
  free(cols);
  free(mptr);
  free(mem);
  free(slot);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Polynomial of best uniform approximation to 1/x on [l0, l1],         */
/* Eq. (1x-1-min), computed by the Remez exchange algorithm (Remez      */
/* 1934): solve p(x_i) + (-1)^i E = 1/x_i on an m+2 point reference,    */
/* move the reference to the extrema of the error, repeat until the     */
/* error levels out.  p is held in the Chebyshev basis of               */
/* t = (2x - l1 - l0)/(l1 - l0).  Internal arithmetic in long double.   */
/* ------------------------------------------------------------------ */
typedef long double ld;

static ld cheb_sum(int m, const ld *c, ld t) {
  ld T0 = 1.0L, T1 = t, s = c[0];
  if (m >= 1) s += c[1] * T1;
  for (int j = 2; j <= m; ++j) {
    ld T2 = 2.0L * t * T1 - T0;
    s += c[j] * T2;
    T0 = T1;
    T1 = T2;
  }
  return s;
}

static ld remez_err(int m, const ld *c, ld t, ld l0, ld l1) {
  ld x = ((l1 - l0) * t + (l1 + l0)) / 2.0L;
  return 1.0L / x - cheb_sum(m, c, t);
}

static int solve_dense_ld(int N, ld *M, ld *rhs) {
  for (int k = 0; k < N; ++k) {
    int piv = k;
    for (int i = k + 1; i < N; ++i)
      if (fabsl(M[i * N + k]) > fabsl(M[piv * N + k])) piv = i;
    if (M[piv * N + k] == 0.0L) return -1;
    if (piv != k) {
      for (int j = 0; j < N; ++j) { ld t = M[k * N + j]; M[k * N + j] = M[piv * N + j]; M[piv * N + j] = t; }
      ld t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
    }
    for (int i = k + 1; i < N; ++i) {
      ld f = M[i * N + k] / M[k * N + k];
      for (int j = k; j < N; ++j) M[i * N + j] -= f * M[k * N + j];
      rhs[i] -= f * rhs[k];
    }
  }
  for (int k = N - 1; k >= 0; --k) {
    ld s = rhs[k];
    for (int j = k + 1; j < N; ++j) s -= M[k * N + j] * rhs[j];
    rhs[k] = s / M[k * N + k];
  }
  return 0;
}

/* maximise sgn * e(t) on [a, b]: dense sampling, then golden section */
static ld remez_argmax(int m, const ld *c, ld l0, ld l1, ld a, ld b, ld sgn) {
  const int S = 64;
  ld best = a, bv = sgn * remez_err(m, c, a, l0, l1);
  for (int s = 1; s <= S; ++s) {
    ld t = a + (b - a) * (ld)s / (ld)S;
    ld v = sgn * remez_err(m, c, t, l0, l1);
    if (v > bv) { bv = v; best = t; }
  }
  ld lo = best - (b - a) / S, hi = best + (b - a) / S;
  if (lo < a) lo = a;
  if (hi > b) hi = b;
  const ld g = 0.6180339887498948482L;
  for (int it = 0; it < 200 && hi - lo > 1e-18L; ++it) {
    ld x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    if (sgn * remez_err(m, c, x1, l0, l1) >= sgn * remez_err(m, c, x2, l0, l1)) hi = x2; else lo = x1;
  }
  ld mid = (lo + hi) / 2;
  ld vm = sgn * remez_err(m, c, mid, l0, l1);
  return vm >= bv ? mid : best;
}

int orc_remez_inverse(int m, double l0d, double l1d, double *cout, double *err, double *alt) {
  if (m < 0 || m > 30 || !(l0d > 0.0) || !(l1d > l0d)) return -1;
  const int N = m + 2;
  ld l0 = l0d, l1 = l1d;
  ld t[32], c[33], M[33 * 33], r[33], E = 0;
  for (int i = 0; i < N; ++i) t[i] = -cosl((ld)i * 3.14159265358979323846264338327950288L / (ld)(m + 1));
  for (int iter = 0; iter < 100; ++iter) {
    for (int i = 0; i < N; ++i) {
      ld T0 = 1.0L, T1 = t[i];
      for (int j = 0; j <= m; ++j) {
        ld Tj;
        if (j == 0) Tj = T0;
        else if (j == 1) Tj = T1;
        else { Tj = 2.0L * t[i] * T1 - T0; T0 = T1; T1 = Tj; }
        M[i * N + j] = Tj;
      }
      M[i * N + m + 1] = (i % 2 == 0) ? 1.0L : -1.0L;
      ld x = ((l1 - l0) * t[i] + (l1 + l0)) / 2.0L;
      r[i] = 1.0L / x;
    }
    if (solve_dense_ld(N, M, r)) return -2;
    for (int j = 0; j <= m; ++j) c[j] = r[j];
    E = r[m + 1];
    /* zeros of the error between consecutive reference points */
    ld z[33];
    for (int i = 0; i + 1 < N; ++i) {
      ld a = t[i], b = t[i + 1];
      ld ea = remez_err(m, c, a, l0, l1);
      for (int it = 0; it < 200 && b - a > 1e-19L; ++it) {
        ld mid = (a + b) / 2;
        ld em = remez_err(m, c, mid, l0, l1);
        if ((em > 0) == (ea > 0)) { a = mid; ea = em; } else b = mid;
      }
      z[i] = (a + b) / 2;
    }
    /* new reference: extremum of (-1)^i E-signed error on each sub-interval */
    ld tn[32], maxe = 0;
    for (int i = 0; i < N; ++i) {
      ld a = (i == 0) ? -1.0L : z[i - 1];
      ld b = (i == N - 1) ? 1.0L : z[i];
      ld sgn = ((i % 2 == 0) ? 1.0L : -1.0L) * (E >= 0 ? 1.0L : -1.0L);
      tn[i] = remez_argmax(m, c, l0, l1, a, b, sgn);
      ld e = fabsl(remez_err(m, c, tn[i], l0, l1));
      if (e > maxe) maxe = e;
    }
    for (int i = 0; i < N; ++i) t[i] = tn[i];
    if (maxe - fabsl(E) <= 1e-17L * fabsl(E) + 1e-300L) break;
  }
  for (int j = 0; j <= m; ++j) cout[j] = (double)c[j];
  if (err) *err = (double)fabsl(E);
  if (alt)
    for (int i = 0; i < N; ++i) alt[i] = (double)(((l1 - l0) * t[i] + (l1 + l0)) / 2.0L);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Cyclic Jacobi eigenvalue method (Golub & Van Loan, Sec. 8.5): sweep   */
/* over all (p, q) pairs with plane rotations that zero a_pq.            */
/* ------------------------------------------------------------------ */
int orc_jacobi_eigen(int n, const double *Ain, double *evals, double *V) {
  double *A = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!A) return -1;
  memcpy(A, Ain, sizeof(double) * (size_t)n * (size_t)n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  fro = sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        if (p != q) off += A[p * n + q] * A[p * n + q];
    if (sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
        double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
        for (int k = 0; k < n; ++k) { /* A <- A J (columns p, q) */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = cs * akp - sn * akq;
          A[k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^T A (rows p, q) */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = cs * apk - sn * aqk;
          A[q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) { /* V <- V J */
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = cs * vkp - sn * vkq;
          V[k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
  free(A);
  return 0;
}

/* x = A^+ b from an eigen-decomposition (Sec. 3: the coarse solve uses the
 * pseudo-inverse): x = sum over eigenpairs with lambda_i > 1e-12 lambda_max
 * of (u_i^T b / lambda_i) u_i. */
static void eig_pinv_apply(int64_t n, const double *ev, const double *U, const double *b, double *x) {
  double lmax = 0.0;
  for (int64_t i = 0; i < n; ++i) if (ev[i] > lmax) lmax = ev[i];
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    if (!(ev[k] > 1e-12 * lmax)) continue;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += U[i * n + k] * b[i];
    s /= ev[k];
    for (int64_t i = 0; i < n; ++i) x[i] += s * U[i * n + k];
  }
}

static double *mat_dense(const orc_mat *A) {
  int64_t n = A->n;
  double *D = vzeros(n * n);
  for (int64_t i = 0; i < n; ++i) {
    D[i * n + i] = A->diag[i];
    for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) D[i * n + A->col[p]] = A->val[p];
  }
  return D;
}

/* ------------------------------------------------------------------ */
/* setup                                                                */
/* ------------------------------------------------------------------ */
int orc_setup(int64_t n, const int64_t *rowptr, const int32_t *col, const double *w,
              const double *d, const orc_options *optin, orc_hier **out) {
  if (!out) return ORC_ERR_INVALID_ARG;
  *out = NULL;
  orc_options opt;
  if (optin) opt = *optin; else orc_default_options(&opt);
  if ((opt.aggregation != ORC_AGG_MATCHING && opt.aggregation != ORC_AGG_MIS) || opt.mis_k < 1 ||
      opt.mis_k > 16)
    return ORC_ERR_INVALID_ARG;
  if (!(opt.rho >= 0.0) || !isfinite(opt.rho) || (opt.cycle != ORC_CYCLE_K && opt.cycle != ORC_CYCLE_AMLI) ||
      !(opt.amli_alpha > 0.0 && opt.amli_alpha < 1.0))
    return ORC_ERR_INVALID_ARG;
  if (opt.rho > 0.0) {
    if (!(opt.lambda0_ratio > 0.0 && opt.lambda0_ratio < 1.0)) return ORC_ERR_INVALID_ARG;
    opt.degree = orc_degree_for(opt.rho, opt.lambda0_ratio);
    if (opt.degree < 0) return ORC_ERR_INVALID_ARG;
  }
  if (opt.degree < 0 || opt.degree > 30 || opt.passes < 1 || opt.passes > 16 || opt.coarse_max < 1 ||
      opt.max_levels < 1 || opt.inner_iters < 1 || opt.inner_iters > 60 || opt.restart < 1 || opt.max_iters < 0 ||
      !(opt.lambda0_ratio > 0.0 && opt.lambda0_ratio < 1.0))
    return ORC_ERR_INVALID_ARG;
  if (n > 2147483647LL) return ORC_ERR_INVALID_ARG;
  int st = validate(n, rowptr, col, w, d);
  if (st) return st;
  int pure = 1;
  if (d)
    for (int64_t i = 0; i < n; ++i) if (d[i] != 0.0) pure = 0;
  st = check_components(n, rowptr, col, d, pure);
  if (st) return st;

  orc_hier *h = (orc_hier *)calloc(1, sizeof(orc_hier));
  h->opt = opt;
  h->pure = pure;
  /* the AMLI polynomial q_{nu-1}: best uniform approximation to 1/t on
   * [alpha, 1] (Sec. 4 with the construction of Sec. 3 applied to the
   * preconditioned coarse operator) */
  if (opt.cycle == ORC_CYCLE_AMLI) {
    /* E = delta^(nu-1) (kappa - 1)/2, kappa = 1/alpha, bounds |1 - t q(t)| on
     * [alpha, 1] (Sec. 3 with lambda1 = 1).  E < 1 (the positivity condition)
     * and the scaling q / (1 + E) give 0 < t q(t) <= 1 there, so that by
     * induction every B_k is SPD with the spectrum of B_k A_k in (0, 1] */
    double kap = 1.0 / opt.amli_alpha, del = (sqrt(kap) - 1.0) / (sqrt(kap) + 1.0);
    double E = pow(del, (double)(opt.inner_iters - 1)) * (kap - 1.0) / 2.0;
    if (!(E < 1.0) || orc_remez_inverse(opt.inner_iters - 1, opt.amli_alpha, 1.0, h->amli_cheb, NULL, NULL)) {
      free(h);
      return ORC_ERR_INVALID_ARG;
    }
    for (int p = 0; p < opt.inner_iters; ++p) h->amli_cheb[p] /= 1.0 + E;
  }
  /* level 0: assemble A from (w, d), Eq. (1) */
  orc_mat *A0 = &h->lv[0].A;
  int64_t nnz = rowptr[n];
  A0->n = n;
  A0->rowptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  A0->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  A0->val = vnew(nnz);
  A0->diag = vnew(n);
  A0->dlow = vnew(n);
  memcpy(A0->rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1));
  if (nnz) memcpy(A0->col, col, sizeof(int32_t) * (size_t)nnz);
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) { A0->val[p] = -w[p]; s += w[p]; }
    A0->dlow[i] = d ? d[i] : 0.0;
    A0->diag[i] = s + A0->dlow[i];
  }
  int L = 1;
  while (h->lv[L - 1].A.n > opt.coarse_max && L < opt.max_levels && L < ORC_MAX_LEVELS) {
    orc_level *lv = &h->lv[L - 1];
    int64_t nk = lv->A.n;
    int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * (size_t)nk);
    for (int64_t i = 0; i < nk; ++i) comp[i] = (int32_t)i;
    orc_mat cur = lv->A; /* borrowed for the first pass */
    orc_mat next;
    int owns = 0;
    int64_t ncur = nk;
    const int npass = opt.aggregation == ORC_AGG_MIS ? 1 : opt.passes;
    lv->npass = npass;
    for (int p = 0; p < npass; ++p) {
      int64_t nc = cur.n, nzc = cur.rowptr[nc];
      int32_t *agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
      int nH;
      if (opt.aggregation == ORC_AGG_MIS) {
        int32_t *isroot = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
        nH = orc_mis_aggregate((int)nc, cur.rowptr, cur.col, opt.mis_k, opt.hash_salt, agg, isroot);
        free(isroot);
      } else {
        /* matching weight of edge (i,j): strength |a_ij| / sqrt(a_ii a_jj) */
        double *wp = vnew(nzc);
        for (int64_t i = 0; i < nc; ++i)
          for (int64_t q = cur.rowptr[i]; q < cur.rowptr[i + 1]; ++q)
            wp[q] = -cur.val[q] / sqrt(cur.diag[i] * cur.diag[cur.col[q]]);
        int32_t *mate = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc);
        nH = orc_match((int)nc, cur.rowptr, cur.col, wp, opt.hash_salt, mate, agg, NULL);
        free(wp);
        free(mate);
      }
      memset(&next, 0, sizeof(next));
      st = galerkin(&cur, agg, nH, &next);
      if (st) return st;
      for (int64_t i = 0; i < nk; ++i) comp[i] = agg[comp[i]];
      lv->pass_n[p] = nc;
      lv->pass_agg[p] = agg;
      if (owns) mat_free(&cur);
      cur = next;
      owns = 1;
      ncur = nH;
    }
    if ((double)ncur > ORC_STALL_RATIO * (double)nk) {
      /* coarsening stalled: keep level L-1 as the coarsest if small enough */
      mat_free(&cur);
      free(comp);
      for (int p = 0; p < lv->npass; ++p) { free(lv->pass_agg[p]); lv->pass_agg[p] = NULL; }
      lv->npass = 0;
      if (nk > ORC_STALL_MAX_COARSE) { h->L = L; orc_free(h); return ORC_ERR_SETUP_STALL; }
      break;
    }
    lv->agg = comp;
    lv->nH = ncur;
    h->lv[L].A = cur;
    ++L;
  }
  h->L = L;
  /* smoother interval and polynomial per non-coarsest level (Sec. 3, Sec. 4) */
  for (int k = 0; k + 1 < L; ++k) {
    orc_level *lv = &h->lv[k];
    double l1 = 0.0;
    for (int64_t i = 0; i < lv->A.n; ++i) {
      double s = fabs(lv->A.diag[i]);
      for (int64_t p = lv->A.rowptr[i]; p < lv->A.rowptr[i + 1]; ++p) s += fabs(lv->A.val[p]);
      if (s > l1) l1 = s;
    }
    lv->lam1 = l1;
    lv->lam0 = opt.lambda0_ratio * l1;
    lv->cheb = vnew(opt.degree + 1);
    if (orc_remez_inverse(opt.degree, lv->lam0, lv->lam1, lv->cheb, NULL, NULL)) {
      orc_free(h);
      return ORC_ERR_INVALID_ARG;
    }
  }
  /* coarsest level: dense eigen-decomposition for the pseudo-inverse */
  {
    orc_mat *Ac = &h->lv[L - 1].A;
    h->nc = Ac->n;
    double *D = mat_dense(Ac);
    h->c_ev = vnew(h->nc);
    h->c_U = vnew(h->nc * h->nc);
    orc_jacobi_eigen((int)h->nc, D, h->c_ev, h->c_U);
    free(D);
  }
  if (opt.precond == ORC_PREC_EXACT) {
    if (n > 3000) { orc_free(h); return ORC_ERR_INVALID_ARG; }
    double *D = mat_dense(&h->lv[0].A);
    h->x_ev = vnew(n);
    h->x_U = vnew(n * n);
    orc_jacobi_eigen((int)n, D, h->x_ev, h->x_U);
    free(D);
  }
  *out = h;
  return ORC_OK;
}

void orc_free(orc_hier *h) {
  if (!h) return;
  for (int k = 0; k < h->L; ++k) {
    mat_free(&h->lv[k].A);
    free(h->lv[k].agg);
    free(h->lv[k].cheb);
    for (int p = 0; p < h->lv[k].npass; ++p) free(h->lv[k].pass_agg[p]);
  }
  free(h->c_ev);
  free(h->c_U);
  free(h->x_ev);
  free(h->x_U);
  free(h);
}

/* ------------------------------------------------------------------ */
/* accessors                                                            */
/* ------------------------------------------------------------------ */
int orc_num_levels(const orc_hier *h) { return h ? h->L : 0; }
int64_t orc_level_n(const orc_hier *h, int k) { return (h && k >= 0 && k < h->L) ? h->lv[k].A.n : -1; }
int64_t orc_level_nnz(const orc_hier *h, int k) {
  return (h && k >= 0 && k < h->L) ? h->lv[k].A.rowptr[h->lv[k].A.n] : -1;
}
int orc_level_csr(const orc_hier *h, int k, int64_t *rowptr, int32_t *col, double *val, double *diag,
                  double *dlow) {
  if (!h || k < 0 || k >= h->L) return ORC_ERR_INVALID_ARG;
  const orc_mat *A = &h->lv[k].A;
  int64_t nnz = A->rowptr[A->n];
  if (rowptr) memcpy(rowptr, A->rowptr, sizeof(int64_t) * (size_t)(A->n + 1));
  if (col && nnz) memcpy(col, A->col, sizeof(int32_t) * (size_t)nnz);
  if (val && nnz) memcpy(val, A->val, sizeof(double) * (size_t)nnz);
  if (diag) memcpy(diag, A->diag, sizeof(double) * (size_t)A->n);
  if (dlow) memcpy(dlow, A->dlow, sizeof(double) * (size_t)A->n);
  return ORC_OK;
}
int orc_level_agg(const orc_hier *h, int k, int32_t *agg) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  memcpy(agg, h->lv[k].agg, sizeof(int32_t) * (size_t)h->lv[k].A.n);
  return ORC_OK;
}
int orc_level_pass_count(const orc_hier *h, int k) {
  return (h && k >= 0 && k + 1 < h->L) ? h->lv[k].npass : 0;
}
int64_t orc_level_pass_n(const orc_hier *h, int k, int p) {
  if (!h || k < 0 || k + 1 >= h->L || p < 0 || p >= h->lv[k].npass) return -1;
  return h->lv[k].pass_n[p];
}
int orc_level_pass_agg(const orc_hier *h, int k, int p, int32_t *agg) {
  if (!h || k < 0 || k + 1 >= h->L || p < 0 || p >= h->lv[k].npass) return ORC_ERR_INVALID_ARG;
  memcpy(agg, h->lv[k].pass_agg[p], sizeof(int32_t) * (size_t)h->lv[k].pass_n[p]);
  return ORC_OK;
}
int orc_level_lambda(const orc_hier *h, int k, double *lam0, double *lam1) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  if (lam0) *lam0 = h->lv[k].lam0;
  if (lam1) *lam1 = h->lv[k].lam1;
  return ORC_OK;
}
int orc_level_cheb(const orc_hier *h, int k, double *coef) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  memcpy(coef, h->lv[k].cheb, sizeof(double) * (size_t)(h->opt.degree + 1));
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* operations                                                           */
/* ------------------------------------------------------------------ */
int orc_spmv(const orc_hier *h, int k, const double *x, double *y) {
  if (!h || k < 0 || k >= h->L) return ORC_ERR_INVALID_ARG;
  mat_spmv(&h->lv[k].A, x, y);
  return ORC_OK;
}

/* out = t(A) v, t(x) = (2x - (l1 + l0)) / (l1 - l0) maps [l0, l1] to [-1, 1] */
static void apply_t(const orc_level *lv, const double *v, double *tmp, double *out) {
  mat_spmv(&lv->A, v, tmp);
  for (int64_t i = 0; i < lv->A.n; ++i)
    out[i] = (2.0 * tmp[i] - (lv->lam1 + lv->lam0) * v[i]) / (lv->lam1 - lv->lam0);
}

/* x = q_m(A) r by the Chebyshev three-term recurrence
 * T_0 = r, T_1 = t(A) r, T_{j+1} = 2 t(A) T_j - T_{j-1}, x = sum_j c_j T_j. */
int orc_smooth(const orc_hier *h, int k, const double *r, double *x) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  const orc_level *lv = &h->lv[k];
  int64_t n = lv->A.n;
  int m = h->opt.degree;
  for (int64_t i = 0; i < n; ++i) x[i] = lv->cheb[0] * r[i];
  if (m == 0) return ORC_OK;
  double *Tp = vnew(n), *Tc = vnew(n), *Tn = vnew(n), *tmp = vnew(n);
  memcpy(Tp, r, sizeof(double) * (size_t)n);
  apply_t(lv, r, tmp, Tc);
  for (int64_t i = 0; i < n; ++i) x[i] += lv->cheb[1] * Tc[i];
  for (int j = 2; j <= m; ++j) {
    apply_t(lv, Tc, tmp, Tn);
    for (int64_t i = 0; i < n; ++i) Tn[i] = 2.0 * Tn[i] - Tp[i];
    for (int64_t i = 0; i < n; ++i) x[i] += lv->cheb[j] * Tn[i];
    double *t = Tp; Tp = Tc; Tc = Tn; Tn = t;
  }
  free(Tp); free(Tc); free(Tn); free(tmp);
  return ORC_OK;
}

/* r_H = P^T s: sum of s over the members of each aggregate, Eq. (coarse) */
int orc_restrict(const orc_hier *h, int k, const double *s, double *rH) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  const orc_level *lv = &h->lv[k];
  for (int64_t I = 0; I < lv->nH; ++I) rH[I] = 0.0;
  for (int64_t i = 0; i < lv->A.n; ++i) rH[lv->agg[i]] += s[i];
  return ORC_OK;
}

/* x += P e_H: each vertex takes its aggregate's value, Eq. (coarse) */
int orc_prolong_add(const orc_hier *h, int k, const double *eH, double *x) {
  if (!h || k < 0 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  const orc_level *lv = &h->lv[k];
  for (int64_t i = 0; i < lv->A.n; ++i) x[i] += eH[lv->agg[i]];
  return ORC_OK;
}

int orc_coarse_solve(const orc_hier *h, const double *b, double *x) {
  if (!h) return ORC_ERR_INVALID_ARG;
  eig_pinv_apply(h->nc, h->c_ev, h->c_U, b, x);
  return ORC_OK;
}

/* K-cycle at level k < L-1 (Sec. 3 two-level steps, W(1,1) of Sec. 4):
 *   x = q_m(A) r;  s = r - A x;  r_H = P^T s;
 *   e_H = A_c^+ r_H (next level coarsest) or nu steps of flexible CG on
 *         A_{k+1} e_H = r_H preconditioned by K_{k+1};
 *   x += P e_H;  s = r - A x;  x += q_m(A) s. */
int orc_kcycle(const orc_hier *h, int k, const double *r, double *x) {
  if (!h || k < 0 || k >= h->L) return ORC_ERR_INVALID_ARG;
  if (k == h->L - 1) return orc_coarse_solve(h, r, x);
  const orc_level *lv = &h->lv[k];
  int64_t n = lv->A.n, nH = lv->nH;
  double *s = vnew(n), *y = vnew(n), *rH = vnew(nH), *eH = vnew(nH);
  orc_smooth(h, k, r, x);
  mat_spmv(&lv->A, x, s);
  for (int64_t i = 0; i < n; ++i) s[i] = r[i] - s[i];
  orc_restrict(h, k, s, rH);
  if (k + 1 == h->L - 1) orc_coarse_solve(h, rH, eH);
  else orc_inner_fcg(h, k + 1, rH, eH);
  orc_prolong_add(h, k, eH, x);
  mat_spmv(&lv->A, x, s);
  for (int64_t i = 0; i < n; ++i) s[i] = r[i] - s[i];
  orc_smooth(h, k, s, y);
  for (int64_t i = 0; i < n; ++i) x[i] += y[i];
  free(s); free(y); free(rH); free(eH);
  return ORC_OK;
}

/* nu steps of flexible CG from x = 0 on A_k x = b, preconditioned by the
 * K-cycle at level k (Sec. 4: NPCG applied recursively on coarse levels).
 * Step i: c = K_k(r); v = A c; d = c - sum_{l<i} (d_l^T v / rho_l) d_l,
 * w = v - sum_{l<i} (same) w_l; rho = d^T w; alpha = d^T r / rho;
 * x += alpha d; r -= alpha w (not after the last step).  A step with
 * rho <= 0 or non-finite ends the iteration with the current x. */
int orc_inner_fcg(const orc_hier *h, int k, const double *b, double *x) {
  if (!h || k < 1 || k + 1 >= h->L) return ORC_ERR_INVALID_ARG;
  const orc_level *lv = &h->lv[k];
  int64_t n = lv->A.n;
  int nu = h->opt.inner_iters;
  double **D = (double **)malloc(sizeof(double *) * (size_t)nu);
  double **W = (double **)malloc(sizeof(double *) * (size_t)nu);
  double *rho = (double *)malloc(sizeof(double) * (size_t)nu);
  double *r = vnew(n), *beta = (double *)malloc(sizeof(double) * (size_t)nu);
  memcpy(r, b, sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  int nd = 0;
  for (int it = 0; it < nu; ++it) {
    D[it] = vnew(n);
    W[it] = vnew(n);
    orc_kcycle(h, k, r, D[it]);
    mat_spmv(&lv->A, D[it], W[it]);
    for (int l = 0; l < nd; ++l) beta[l] = dot(n, D[l], W[it]) / rho[l];
    for (int l = 0; l < nd; ++l)
      for (int64_t i = 0; i < n; ++i) { D[it][i] -= beta[l] * D[l][i]; W[it][i] -= beta[l] * W[l][i]; }
    rho[it] = dot(n, D[it], W[it]);
    nd = it + 1;
    if (!(rho[it] > 0.0) || !isfinite(rho[it])) break;
    double alpha = dot(n, D[it], r) / rho[it];
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * D[it][i];
    if (it + 1 < nu)
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * W[it][i];
  }
  for (int l = 0; l < nd; ++l) { free(D[l]); free(W[l]); }
  free(D); free(W); free(rho); free(r); free(beta);
  return ORC_OK;
}

/* Stationary AMLI W-cycle at level k < L-1 (Sec. 4: "AMLI-cycle"): the
 * two-level steps of orc_kcycle with the coarse problem solved by a fixed
 * polynomial instead of inner flexible CG:
 *   e_H = q(B_{k+1} A_{k+1}) B_{k+1} r_H   (k+1 < L-1),  e_H = A_c^+ r_H (k+1 = L-1),
 * q = q_{nu-1} / (1 + E), q_{nu-1} the best uniform approximation to 1/t on
 * [alpha, 1] and E its error bound (see orc_setup), in the Chebyshev basis of
 * tau(t) = (2t - 1 - alpha)/(1 - alpha), evaluated by the
 * forward recurrence T_0 = B r_H, T_1 = tau(BA) T_0,
 * T_{p+1} = 2 tau(BA) T_p - T_{p-1}; each tau(BA) costs one SpMV with A_{k+1}
 * and one application of B_{k+1} (nu applications of B_{k+1} in all: a
 * W-cycle for nu = 2).  B_k is linear and symmetric. */
static void amli_coarse(const orc_hier *h, int j, const double *rH, double *eH) {
  const orc_level *lv = &h->lv[j];
  int64_t n = lv->A.n;
  int deg = h->opt.inner_iters - 1;
  double a = h->opt.amli_alpha;
  double *Tp = vnew(n), *Tc = vnew(n), *Tn = vnew(n), *v = vnew(n), *w = vnew(n);
  orc_amli_cycle(h, j, rH, Tc); /* T_0 = B r_H */
  for (int64_t i = 0; i < n; ++i) eH[i] = h->amli_cheb[0] * Tc[i];
  for (int p = 1; p <= deg; ++p) {
    /* w = B A T_{p-1}; tau(BA) T_{p-1} = (2 w - (1 + a) T_{p-1}) / (1 - a) */
    mat_spmv(&lv->A, Tc, v);
    orc_amli_cycle(h, j, v, w);
    for (int64_t i = 0; i < n; ++i) {
      double t = (2.0 * w[i] - (1.0 + a) * Tc[i]) / (1.0 - a);
      Tn[i] = (p == 1) ? t : 2.0 * t - Tp[i];
    }
    for (int64_t i = 0; i < n; ++i) eH[i] += h->amli_cheb[p] * Tn[i];
    double *t = Tp; Tp = Tc; Tc = Tn; Tn = t;
  }
  free(Tp); free(Tc); free(Tn); free(v); free(w);
}

int orc_amli_cycle(const orc_hier *h, int k, const double *r, double *x) {
  if (!h || k < 0 || k >= h->L) return ORC_ERR_INVALID_ARG;
  if (k == h->L - 1) return orc_coarse_solve(h, r, x);
  const orc_level *lv = &h->lv[k];
  int64_t n = lv->A.n, nH = lv->nH;
  double *s = vnew(n), *y = vnew(n), *rH = vnew(nH), *eH = vnew(nH);
  orc_smooth(h, k, r, x);
  mat_spmv(&lv->A, x, s);
  for (int64_t i = 0; i < n; ++i) s[i] = r[i] - s[i];
  orc_restrict(h, k, s, rH);
  if (k + 1 == h->L - 1) orc_coarse_solve(h, rH, eH);
  else amli_coarse(h, k + 1, rH, eH);
  orc_prolong_add(h, k, eH, x);
  mat_spmv(&lv->A, x, s);
  for (int64_t i = 0; i < n; ++i) s[i] = r[i] - s[i];
  orc_smooth(h, k, s, y);
  for (int64_t i = 0; i < n; ++i) x[i] += y[i];
  free(s); free(y); free(rH); free(eH);
  return ORC_OK;
}

int orc_amli_coef(const orc_hier *h, double *coef) {
  if (!h || !coef || h->opt.cycle != ORC_CYCLE_AMLI) return ORC_ERR_INVALID_ARG;
  for (int p = 0; p < h->opt.inner_iters; ++p) coef[p] = h->amli_cheb[p];
  return ORC_OK;
}

/* Eq. (bound-on-m) read as: the smallest m whose error E_m = delta^m
 * (kappa - 1)/2 of the smoother polynomial (Sec. 3) is at most rho and
 * below 1 (the positivity condition), kappa = lambda1/lambda0 */
int orc_degree_for(double rho, double lambda0_ratio) {
  if (!(rho > 0.0) || !(lambda0_ratio > 0.0 && lambda0_ratio < 1.0)) return -1;
  double kappa = 1.0 / lambda0_ratio;
  double delta = (sqrt(kappa) - 1.0) / (sqrt(kappa) + 1.0);
  for (int m = 0; m <= 30; ++m) {
    double e = pow(delta, (double)m) * (kappa - 1.0) / 2.0;
    if (e <= rho && e < 1.0) return m;
  }
  return -1;
}

/* ------------------------------------------------------------------ */
/* outer flexible CG (Sec. 4: the N-AMLI cycle preconditions NPCG on the */
/* finest level, restarted every five iterations).  Iteration k:         */
/*   z = K_0(r); d = z - sum_{j in window} (q_j^T z / rho_j) d_j;        */
/*   q = A d; rho = d^T q; alpha = d^T r / rho; x += alpha d;            */
/*   r -= alpha q; the window (d_j, q_j = A d_j, rho_j) is emptied at     */
/*   every multiple of `restart`.  Stops when ||r|| <= tol ||b||.         */
/* A pure Laplacian's right-hand side is first projected to zero mean    */
/* (its range is 1-perp, Sec. 1) and x is returned with zero mean.       */
/* ------------------------------------------------------------------ */
int orc_solve(orc_hier *h, const double *bin, double *x, double tol, orc_info *info) {
  if (!h || !bin || !x) return ORC_ERR_INVALID_ARG;
  const orc_mat *A = &h->lv[0].A;
  int64_t n = A->n;
  int R = h->opt.restart;
  double *b = vnew(n), *r = vnew(n), *z = vnew(n), *tmp = vnew(n);
  double **D = (double **)malloc(sizeof(double *) * (size_t)R);
  double **Q = (double **)malloc(sizeof(double *) * (size_t)R);
  double *rho = (double *)malloc(sizeof(double) * (size_t)R);
  double *beta = (double *)malloc(sizeof(double) * (size_t)R);
  for (int j = 0; j < R; ++j) { D[j] = vnew(n); Q[j] = vnew(n); }
  memcpy(b, bin, sizeof(double) * (size_t)n);
  if (h->pure) {
    double mean = 0.0;
    for (int64_t i = 0; i < n; ++i) mean += b[i];
    mean /= (double)n;
    for (int64_t i = 0; i < n; ++i) b[i] -= mean;
  }
  double nb = sqrt(dot(n, b, b));
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  memcpy(r, b, sizeof(double) * (size_t)n);
  int status = ORC_OK, it = 0, converged = 0, hl = 0;
  double res = (nb > 0.0) ? 1.0 : 0.0;
  if (info && info->history && info->history_cap > 0) info->history[hl++] = res;
  if (nb == 0.0) converged = 1;
  int nwin = 0;
  while (!converged && it < h->opt.max_iters) {
    if (it % R == 0) nwin = 0;
    double *d = D[nwin], *q = Q[nwin];
    if (h->opt.precond == ORC_PREC_IDENTITY) memcpy(z, r, sizeof(double) * (size_t)n);
    else if (h->opt.precond == ORC_PREC_EXACT) eig_pinv_apply(n, h->x_ev, h->x_U, r, z);
    else if (h->opt.cycle == ORC_CYCLE_AMLI) orc_amli_cycle(h, 0, r, z);
    else orc_kcycle(h, 0, r, z);
    for (int j = 0; j < nwin; ++j) beta[j] = dot(n, Q[j], z) / rho[j];
    memcpy(d, z, sizeof(double) * (size_t)n);
    for (int j = 0; j < nwin; ++j)
      for (int64_t i = 0; i < n; ++i) d[i] -= beta[j] * D[j][i];
    mat_spmv(A, d, q);
    double rh = dot(n, d, q);
    if (!(rh > 0.0) || !isfinite(rh)) { status = ORC_ERR_BREAKDOWN; break; }
    double alpha = dot(n, d, r) / rh;
    for (int64_t i = 0; i < n; ++i) { x[i] += alpha * d[i]; r[i] -= alpha * q[i]; }
    rho[nwin] = rh;
    ++nwin;
    ++it;
    res = sqrt(dot(n, r, r)) / nb;
    if (info && info->history && hl < info->history_cap) info->history[hl++] = res;
    if (res <= tol) converged = 1;
  }
  if (h->pure) {
    double mean = 0.0;
    for (int64_t i = 0; i < n; ++i) mean += x[i];
    mean /= (double)n;
    for (int64_t i = 0; i < n; ++i) x[i] -= mean;
  }
  if (status == ORC_OK && !converged) status = ORC_ERR_NOT_CONVERGED;
  if (info) {
    mat_spmv(A, x, tmp);
    double tr = 0.0;
    for (int64_t i = 0; i < n; ++i) tr += (b[i] - tmp[i]) * (b[i] - tmp[i]);
    info->iterations = it;
    info->converged = converged;
    info->rel_residual = res;
    info->true_rel_residual = nb > 0.0 ? sqrt(tr) / nb : 0.0;
    info->n_levels = h->L;
    double gs = 0.0, os = 0.0;
    for (int k = 0; k < h->L; ++k) {
      gs += (double)h->lv[k].A.n;
      os += (double)(h->lv[k].A.rowptr[h->lv[k].A.n] + h->lv[k].A.n);
    }
    info->grid_complexity = gs / (double)n;
    info->op_complexity = os / (double)(A->rowptr[n] + n);
    info->history_len = hl;
  }
  for (int j = 0; j < R; ++j) { free(D[j]); free(Q[j]); }
  free(D); free(Q); free(rho); free(beta);
  free(b); free(r); free(z); free(tmp);
  return status;
}
