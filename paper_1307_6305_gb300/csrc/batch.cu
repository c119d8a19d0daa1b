// batch.cu -- many right-hand sides solved together.
//
// The right-hand sides of one amg_solve call are processed in blocks of kb
// columns (kb a power of two <= 32), stored row major: X[i * kb + c] is
// component i of column c.  Every operator of the method then becomes its
// multi-vector form (SpMM instead of SpMV): the smoother recurrence, the
// residuals, restriction and prolongation, the dense coarse operators, and
// flexible CG with one set of Krylov scalars per column (Sec. 4).  Each
// stored matrix entry is read once per row for all kb columns and the kb
// neighbour values of a column gather are contiguous.  Columns are fully
// independent: a column that has converged (or broken down) is frozen by a
// zero step length while the others continue.
//
// One block preconditioner application is a CUDA graph replayed per outer
// iteration.  The block width kb and the thread-block size of the SpMM-type
// kernels (rows per CTA = threads / kb) are chosen by timing graph replays
// of every candidate on the first batched solve of a handle.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "block_kernels.cuh"

namespace amg {

#define BLAUNCH(h)                                                                  \
  do {                                                                              \
    ++(h)->launches;                                                                \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxBlock = 32;
constexpr int kBRed = kMaxDots * kMaxBlock;  // partial sums per CTA

// per-column scalar slots (array [slot][kb])
enum : int {
  S_RHO = 0,      // rho_j (window or inner step j), 0..15
  S_ALPHA_I = 8,  // inner alpha_i, 8..15
  S_BETA = 16,    // beta_j, 16..31
  S_STOP = 24,    // inner stop flag
  S_ALPHA = 32,   // outer alpha
  S_RR = 33,      // ||r||^2
  S_BREAK = 34,   // outer breakdown flag
  S_MEAN = 35,    // mean of b / x
  S_BB = 36,      // ||b||^2
  S_TRUE = 38,    // ||b - A x||^2
  S_FROZEN = 40   // column no longer updated
};
constexpr int kScalSlots = 48;

enum BFinKind : int { BF_STORE = 0, BF_IBETA = 1, BF_IALPHA = 2, BF_OBETA = 3, BF_OALPHA = 4, BF_MEAN = 5 };

struct BFin {
  int kind;
  int o0;
  double o1;
  double *scal;
};

template <typename T>
struct BDots {
  const T *a[kMaxDots];
  const T *b[kMaxDots];  // nullptr: 1 (k_bdots) or the computed product (k_bspmv_dots)
  int nd;
};

__device__ void bfinalize(const BFin &f, int kb, int c, const double *s, int nd) {
  double *sc = f.scal;
  auto S = [&](int slot) -> double & { return sc[slot * kb + c]; };
  switch (f.kind) {
    case BF_STORE:
      for (int q = 0; q < nd; ++q) S(f.o0 + q) = s[q];
      break;
    case BF_IBETA:
      for (int l = 0; l < nd; ++l) S(S_BETA + l) = S(S_RHO + l) != 0.0 ? s[l] / S(S_RHO + l) : 0.0;
      break;
    case BF_IALPHA: {
      const double rho = s[0], sig = s[1];
      S(S_RHO + f.o0) = rho;
      if (S(S_STOP) != 0.0 || !(rho > 0.0) || !isfinite(rho)) {
        S(S_STOP) = 1.0;
        S(S_ALPHA_I + f.o0) = 0.0;
      } else {
        S(S_ALPHA_I + f.o0) = sig / rho;
      }
      break;
    }
    case BF_OBETA:
      for (int j = 0; j < nd; ++j) S(S_BETA + j) = S(S_RHO + j) != 0.0 ? s[j] / S(S_RHO + j) : 0.0;
      break;
    case BF_OALPHA: {
      const double rho = s[0], sig = s[1];
      S(S_RHO + f.o0) = rho;
      if (S(S_FROZEN) != 0.0) {
        S(S_ALPHA) = 0.0;
      } else if (!(rho > 0.0) || !isfinite(rho)) {
        S(S_BREAK) = 1.0;
        S(S_ALPHA) = 0.0;
      } else {
        S(S_ALPHA) = sig / rho;
      }
      break;
    }
    case BF_MEAN:
      S(f.o0) = s[0] / f.o1;
      break;
  }
}

// per-column deterministic reduction: rows of the CTA in order, then CTAs in
// order in the last CTA, which finalises every column
template <int ND>
__device__ __forceinline__ void breduce(const double (&acc)[ND], int kb, double *partial, unsigned *ticket,
                                        const BFin &fin) {
  __shared__ double sh[ND][kThreads];
  __shared__ double tot[ND][kMaxBlock];
  __shared__ bool last;
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < ND; ++q) sh[q][t] = acc[q];
  __syncthreads();
  const int rows = kThreads / kb;
  if (t < ND * kb) {
    const int q = t / kb, c = t % kb;
    double v = 0.0;
    for (int r = 0; r < rows; ++r) v += sh[q][r * kb + c];
    partial[(size_t)blockIdx.x * kBRed + q * kb + c] = v;
  }
  __threadfence();
  __syncthreads();
  if (t == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  {
    // G threads per (dot, column) pair, each over every G-th CTA's partial
    // (one round of independent loads), then the G sums in thread order
    const int npair = ND * kb, G = kThreads / npair;
    double v = 0.0;
    if (t < npair * G) {
      const int p = t % npair, g = t / npair;
      const int q = p / kb, c = p % kb;
      for (unsigned b = g; b < gridDim.x; b += G) v += __ldcg(&partial[(size_t)b * kBRed + q * kb + c]);
    }
    sh[0][t] = v;
    __syncthreads();
    if (t < npair) {
      double s = 0.0;
      for (int g = 0; g < G; ++g) s += sh[0][g * npair + t];
      tot[t / kb][t % kb] = s;
    }
  }
  __syncthreads();
  if (t < kb) {
    double s[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) s[q] = tot[q][t];
    bfinalize(fin, kb, t, s, ND);
  }
  if (t == 0) *ticket = 0u;
}

// reduction kernels: blockDim = kThreads = rows x kb, thread (row, column)
template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_bdots(int n, int kb, BDots<T> spec, double *partial,
                                                    unsigned *ticket, BFin fin) {
  pdl_sync();
  const int rows = kThreads / kb, c = threadIdx.x % kb;
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  for (int i = blockIdx.x * rows + threadIdx.x / kb; i < n; i += gridDim.x * rows) {
    const int64_t idx = (int64_t)i * kb + c;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const double a = (double)spec.a[q][idx];
      acc[q] += spec.b[q] ? a * (double)spec.b[q][idx] : a;
    }
  }
  breduce<ND>(acc, kb, partial, ticket, fin);
}

template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_bspmv_dots(SellView<T> A, int kb, const T *__restrict__ X,
                                                         T *__restrict__ Y, BDots<T> spec, double *partial,
                                                         unsigned *ticket, BFin fin) {
  pdl_sync();
  const int rows = kThreads / kb, c = threadIdx.x % kb;
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  for (int i = blockIdx.x * rows + threadIdx.x / kb; i < A.n; i += gridDim.x * rows) {
    const int64_t idx = (int64_t)i * kb + c;
    const T y = sell_row_block(A, X, kb, i, c, A.diag[i] * X[idx]);
    Y[idx] = y;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const double a = spec.a[q] ? (double)spec.a[q][idx] : (double)y;
      const double b = spec.b[q] ? (double)spec.b[q][idx] : (double)y;
      acc[q] += a * b;
    }
  }
  breduce<ND>(acc, kb, partial, ticket, fin);
}

// inner step it > 0: D -= sum_l beta_l D_l, W -= sum_l beta_l W_l (per column),
// then rho = D.W, sigma = D.rin per column (BF_IALPHA)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_borth_dots(int n, int kb, T *D, T *W, BDots<T> prev,
                                                         const double *beta, const T *__restrict__ rin,
                                                         double *partial, unsigned *ticket, BFin fin) {
  pdl_sync();
  const int rows = kThreads / kb, c = threadIdx.x % kb;
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * rows + threadIdx.x / kb; i < n; i += gridDim.x * rows) {
    const int64_t idx = (int64_t)i * kb + c;
    T d = D[idx], w = W[idx];
    for (int l = 0; l < prev.nd; ++l) {
      const T bl = (T)beta[l * kb + c];
      d -= bl * prev.a[l][idx];
      w -= bl * prev.b[l][idx];
    }
    D[idx] = d;
    W[idx] = w;
    acc[0] += (double)d * (double)w;
    acc[1] += (double)d * (double)rin[idx];
  }
  breduce<2>(acc, kb, partial, ticket, fin);
}

template <typename T>
__global__ void k_binner_update(int64_t nk, int kb, int it, bool upd_r, const double *sc, const T *D,
                                const T *W, const T *rin, T *x, T *r) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nk) return;
  const int c = (int)(idx % kb);
  const double al = sc[(S_ALPHA_I + it) * kb + c];
  const bool here = sc[S_STOP * kb + c] != 0.0 && al == 0.0;
  const T a = (T)al;
  if (it == 0) x[idx] = here ? T(0) : a * D[idx];
  else if (!here) x[idx] = fma(a, D[idx], x[idx]);
  if (upd_r) r[idx] = here ? rin[idx] : rin[idx] - a * W[idx];
}

// y = z - sum_j beta_j V_j per column
template <typename T>
__global__ void k_baxpy_multi(int64_t nk, int kb, T *y, const T *z, BDots<T> V, const double *beta) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nk) return;
  const int c = (int)(idx % kb);
  T v = z[idx];
  for (int j = 0; j < V.nd; ++j) v -= (T)beta[j * kb + c] * V.a[j][idx];
  y[idx] = v;
}

// x += alpha d, r -= alpha q (columns with alpha = 0 untouched), then r.r
__global__ void __launch_bounds__(kThreads) k_bouter_update(int n, int kb, const double *sc, const double *d,
                                                            const double *q, double *x, double *r,
                                                            double *partial, unsigned *ticket, BFin fin) {
  pdl_sync();
  const int rows = kThreads / kb, c = threadIdx.x % kb;
  const double a = sc[S_ALPHA * kb + c];
  double acc[1] = {0.0};
  for (int i = blockIdx.x * rows + threadIdx.x / kb; i < n; i += gridDim.x * rows) {
    const int64_t idx = (int64_t)i * kb + c;
    double ri = r[idx];
    if (a != 0.0) {
      x[idx] = fma(a, d[idx], x[idx]);
      ri = fma(-a, q[idx], ri);
      r[idx] = ri;
    }
    acc[0] += ri * ri;
  }
  breduce<1>(acc, kb, partial, ticket, fin);
}

__global__ void k_bshift(int64_t nk, int kb, const double *src, double *dst, const double *mean) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nk) dst[idx] = src[idx] - mean[idx % kb];
}

// column-major user block (ld) <-> row-major internal block of width kb;
// columns beyond nr are zero
__global__ void k_bpack(int n, int kb, int nr, int64_t ld, const double *src, double *dst) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * kb) return;
  const int i = (int)(idx / kb), c = (int)(idx % kb);
  dst[idx] = c < nr ? src[(int64_t)c * ld + i] : 0.0;
}

__global__ void k_bunpack(int n, int kb, int nr, int64_t ld, const double *src, double *dst) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * kb) return;
  const int i = (int)(idx / kb), c = (int)(idx % kb);
  if (c < nr) dst[(int64_t)c * ld + i] = src[idx];
}

template <typename A, typename B>
__global__ void k_bconvert(int64_t n, const A *__restrict__ a, B *__restrict__ b) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
static SellView<T> bview(const amg::Level &L);
template <>
SellView<double> bview<double>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.val64, L.S.diag64};
}
template <>
SellView<float> bview<float>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.val32, L.S.diag32};
}

static inline unsigned bred_grid(int n, int kb) {
  const int rows = kThreads / kb;
  return (unsigned)std::max(1, std::min(kRedBlocks, (n + rows - 1) / rows));
}

template <typename T>
static amg_status bdots(amg_handle_s *h, int n, const BDots<T> &sp, BFin fin) {
  const int kb = h->bw_use;
  const unsigned g = bred_grid(n, kb);
  double *P = h->b_partial;
  unsigned *tk = h->b_ticket;
  cudaStream_t st = h->stream;
  switch (sp.nd) {
    case 1: AMG_TRY(plaunch(h, st, k_bdots<T, 1>, dim3(g), dim3(kThreads), n, kb, sp, P, tk, fin)); break;
    case 2: AMG_TRY(plaunch(h, st, k_bdots<T, 2>, dim3(g), dim3(kThreads), n, kb, sp, P, tk, fin)); break;
    case 3: AMG_TRY(plaunch(h, st, k_bdots<T, 3>, dim3(g), dim3(kThreads), n, kb, sp, P, tk, fin)); break;
    case 4: AMG_TRY(plaunch(h, st, k_bdots<T, 4>, dim3(g), dim3(kThreads), n, kb, sp, P, tk, fin)); break;
    default: AMG_TRY(plaunch(h, st, k_bdots<T, 8>, dim3(g), dim3(kThreads), n, kb, sp, P, tk, fin)); break;
  }
  BLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status bspmv_dots(amg_handle_s *h, const amg::Level &L, const T *X, T *Y, const BDots<T> &sp, BFin fin) {
  const int kb = h->bw_use;
  const unsigned g = bred_grid(L.n, kb);
  double *P = h->b_partial;
  unsigned *tk = h->b_ticket;
  cudaStream_t st = h->stream;
  const SellView<T> A = bview<T>(L);
  switch (sp.nd) {
    case 1: AMG_TRY(plaunch(h, st, k_bspmv_dots<T, 1>, dim3(g), dim3(kThreads), A, kb, X, Y, sp, P, tk, fin)); break;
    case 2: AMG_TRY(plaunch(h, st, k_bspmv_dots<T, 2>, dim3(g), dim3(kThreads), A, kb, X, Y, sp, P, tk, fin)); break;
    case 3: AMG_TRY(plaunch(h, st, k_bspmv_dots<T, 3>, dim3(g), dim3(kThreads), A, kb, X, Y, sp, P, tk, fin)); break;
    case 4: AMG_TRY(plaunch(h, st, k_bspmv_dots<T, 4>, dim3(g), dim3(kThreads), A, kb, X, Y, sp, P, tk, fin)); break;
    default: AMG_TRY(plaunch(h, st, k_bspmv_dots<T, 8>, dim3(g), dim3(kThreads), A, kb, X, Y, sp, P, tk, fin)); break;
  }
  BLAUNCH(h);
  return AMG_OK;
}

// X (=|+=) q_m(A_k) R on the block, SpMM-type kernels with h->b_tile threads
template <typename T>
static amg_status bsmooth_t(amg_handle_s *h, int k, const T *R, T *X, bool add) {
  amg::Level &L = h->lv[k];
  amg::BatchLevel &B = h->blv[k];
  const int kb = h->bw_use, tile = h->b_tile, m = h->opt.degree;
  const SellView<T> A = bview<T>(L);
  const T sa = (T)(2.0 / (L.lam1 - L.lam0)), ca = (T)((L.lam1 + L.lam0) / (L.lam1 - L.lam0));
  const int64_t nk = (int64_t)L.n * kb;
  cudaStream_t st = h->stream;
  const dim3 g(nblk(nk, tile)), b(tile);
  if (m == 0) {
    if (add) AMG_TRY(plaunch(h, st, k_bscale<T, true>, g, b, nk, R, X, (T)L.coef[0]));
    else AMG_TRY(plaunch(h, st, k_bscale<T, false>, g, b, nk, R, X, (T)L.coef[0]));
    BLAUNCH(h);
    return AMG_OK;
  }
  T *Ta = (T *)B.Ta, *Tb = (T *)B.Tb;
  if (add) AMG_TRY(plaunch(h, st, k_bcheb_first<T, true>, g, b, A, kb, R, Ta, X, sa, ca, (T)L.coef[0], (T)L.coef[1]));
  else AMG_TRY(plaunch(h, st, k_bcheb_first<T, false>, g, b, A, kb, R, Ta, X, sa, ca, (T)L.coef[0], (T)L.coef[1]));
  BLAUNCH(h);
  const T *Tp = R;
  T *Tc = Ta;
  for (int j = 2; j <= m; ++j) {
    T *Tn = (j == 2) ? Tb : const_cast<T *>(Tp);
    AMG_TRY(plaunch(h, st, k_bcheb_step<T>, g, b, A, kb, Tc, Tp, Tn, X, sa, ca, (T)L.coef[j]));
    BLAUNCH(h);
    Tp = Tc;
    Tc = Tn;
  }
  return AMG_OK;
}

template <typename T>
static amg_status bkcycle(amg_handle_s *h, int k, const T *R, T *X);

template <typename T>
static amg_status binner(amg_handle_s *h, int k) {
  amg::Level &L = h->lv[k];
  amg::BatchLevel &B = h->blv[k];
  const int nu = h->opt.inner_iters, kb = h->bw_use, n = L.n;
  const int64_t nk = (int64_t)n * kb;
  cudaStream_t st = h->stream;
  T *b = (T *)B.b, *x = (T *)B.x, *r = (T *)B.r;
  for (int it = 0; it < nu; ++it) {
    const T *rin = (it == 0) ? b : r;
    T *D = (T *)B.D[it], *W = (T *)B.W[it];
    AMG_TRY(bkcycle<T>(h, k, rin, D));
    if (it == 0) {
      BDots<T> sp{};
      sp.a[0] = D;
      sp.b[0] = nullptr;
      sp.a[1] = rin;
      sp.b[1] = D;
      sp.nd = 2;
      AMG_TRY(bspmv_dots<T>(h, L, D, W, sp, BFin{BF_IALPHA, 0, 0.0, B.scal}));
    } else {
      BDots<T> sp{};
      for (int l = 0; l < it; ++l) {
        sp.a[l] = (const T *)B.D[l];
        sp.b[l] = nullptr;
      }
      sp.nd = it;
      AMG_TRY(bspmv_dots<T>(h, L, D, W, sp, BFin{BF_IBETA, 0, 0.0, B.scal}));
      BDots<T> prev{};
      for (int l = 0; l < it; ++l) {
        prev.a[l] = (const T *)B.D[l];
        prev.b[l] = (const T *)B.W[l];
      }
      prev.nd = it;
      AMG_TRY(plaunch(h, st, k_borth_dots<T>, dim3(bred_grid(n, kb)), dim3(kThreads), n, kb, D, W, prev,
                      (const double *)(B.scal + S_BETA * kb), rin, h->b_partial, h->b_ticket,
                      BFin{BF_IALPHA, it, 0.0, B.scal}));
      BLAUNCH(h);
    }
    AMG_TRY(plaunch(h, st, k_binner_update<T>, dim3(nblk(nk)), dim3(kThreads), nk, kb, it, it + 1 < nu,
                    (const double *)B.scal, (const T *)D, (const T *)W, rin, x, r));
    BLAUNCH(h);
  }
  return AMG_OK;
}

// X = K_k(R) for every column: the W(1,1) nonlinear AMLI cycle in block form
template <typename T>
static amg_status bkcycle(amg_handle_s *h, int k, const T *R, T *X) {
  const int kb = h->bw_use, tile = h->b_tile;
  cudaStream_t st = h->stream;
  if (k == h->L - 1 || k == h->Bk) {
    const int n = h->lv[k].n;
    const double *M = (k == h->L - 1) ? h->Z : h->Bd;
    AMG_TRY(plaunch(h, st, k_bdense<T>, dim3(nblk((int64_t)n * kb)), dim3(kThreads), n, kb, M, R, X));
    BLAUNCH(h);
    return AMG_OK;
  }
  amg::Level &L = h->lv[k], &N = h->lv[k + 1];
  amg::BatchLevel &B = h->blv[k], &NB = h->blv[k + 1];
  const SellView<T> A = bview<T>(L);
  const int64_t nk = (int64_t)L.n * kb;
  T *U = (T *)B.u, *S = (T *)B.s;
  AMG_TRY(bsmooth_t<T>(h, k, R, U, false));
  AMG_TRY(plaunch(h, st, k_bresidual<T>, dim3(nblk(nk, tile)), dim3(tile), A, kb, (const T *)U, R, S));
  BLAUNCH(h);
  AMG_TRY(plaunch(h, st, k_brestrict<T>, dim3(nblk((int64_t)N.n * kb)), dim3(kThreads), N.n, kb, L.agg_ptr,
                  L.agg_mem, (const T *)S, (T *)NB.b, NB.scal + S_STOP * kb));
  BLAUNCH(h);
  if (k + 1 == h->L - 1) {
    AMG_TRY(plaunch(h, st, k_bdense<T>, dim3(nblk((int64_t)N.n * kb)), dim3(kThreads), N.n, kb,
                    (const double *)h->Z, (const T *)NB.b, (T *)NB.x));
    BLAUNCH(h);
  } else {
    AMG_TRY(binner<T>(h, k + 1));
  }
  AMG_TRY(plaunch(h, st, k_bprolong_residual<T>, dim3(nblk(nk, tile)), dim3(tile), A, kb, (const int *)L.agg,
                  (const T *)NB.x, (const T *)U, R, X, S));
  BLAUNCH(h);
  AMG_TRY(bsmooth_t<T>(h, k, S, X, true));
  return AMG_OK;
}

// Z = K_0(R) on the outer buffers (fp64 in and out)
static amg_status bprecondition(amg_handle_s *h) {
  const int64_t nk = h->n * (int64_t)h->bw_use;
  cudaStream_t st = h->stream;
  if (h->opt.precision == AMG_PREC_FP32) {
    AMG_TRY(plaunch(h, st, k_bconvert<double, float>, dim3(nblk(nk)), dim3(kThreads), nk, (const double *)h->bo_r,
                    (float *)h->b_r32));
    BLAUNCH(h);
    AMG_TRY(bkcycle<float>(h, 0, (const float *)h->b_r32, (float *)h->b_z32));
    AMG_TRY(plaunch(h, st, k_bconvert<float, double>, dim3(nblk(nk)), dim3(kThreads), nk, (const float *)h->b_z32,
                    h->bo_z));
    BLAUNCH(h);
    return AMG_OK;
  }
  return bkcycle<double>(h, 0, h->bo_r, h->bo_z);
}

// buffers for blocks of up to W columns (W a power of two <= kMaxBlock),
// allocated on first use and re-allocated, larger, when a later solve needs
// a wider block (the old ones are released stream-ordered and the captured
// block preconditioner, which points at them, is dropped)
static void drop_block_graphs(amg_handle_s *h) {
  if (h->bpre_exec && !h->bpre_borrowed) cudaGraphExecDestroy(h->bpre_exec);
  h->bpre_exec = nullptr;
  h->bpre_borrowed = false;
  for (cudaGraphExec_t &g : h->bfixed) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

static amg_status ensure_batch_buffers(amg_handle_s *h, int W) {
  if (h->bw >= W) return AMG_OK;
  if (h->bw) {
    drop_block_graphs(h);
    for (void *p : h->batch_blocks) h->arena.free_block(p);
    h->batch_blocks.clear();
    h->bw = 0;
    h->tuned_for = 0;
  }
  const bool f32 = h->opt.precision == AMG_PREC_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const int L = h->L, nu = h->opt.inner_iters;
  const size_t blocks_before = h->arena.blocks.size();
  h->blv.assign(L, amg::BatchLevel());
  for (int k = 0; k < L; ++k) {
    amg::BatchLevel &B = h->blv[k];
    const size_t n = (size_t)std::max(h->lv[k].n, 1) * W;
    AMG_TRY(h->arena.alloc((void **)&B.scal, sizeof(double) * kScalSlots * W));
    AMG_CUDA_TRY(cudaMemsetAsync(B.scal, 0, sizeof(double) * kScalSlots * W, h->stream));
    if (k < L - 1) {
      AMG_TRY(h->arena.alloc(&B.u, es * n));
      AMG_TRY(h->arena.alloc(&B.s, es * n));
      AMG_TRY(h->arena.alloc(&B.Ta, es * n));
      AMG_TRY(h->arena.alloc(&B.Tb, es * n));
    }
    if (k >= 1) {
      AMG_TRY(h->arena.alloc(&B.b, es * n));
      AMG_TRY(h->arena.alloc(&B.x, es * n));
    }
    if (k >= 1 && k < L - 1) {
      AMG_TRY(h->arena.alloc(&B.r, es * n));
      for (int i = 0; i < nu; ++i) {
        AMG_TRY(h->arena.alloc(&B.D[i], es * n));
        AMG_TRY(h->arena.alloc(&B.W[i], es * n));
      }
    }
  }
  const size_t n0 = (size_t)h->n * W;
  AMG_TRY(h->arena.get(&h->bo_b, n0));
  AMG_TRY(h->arena.get(&h->bo_x, n0));
  AMG_TRY(h->arena.get(&h->bo_r, n0));
  AMG_TRY(h->arena.get(&h->bo_z, n0));
  AMG_TRY(h->arena.get(&h->bo_t, n0));
  for (int j = 0; j < h->opt.restart; ++j) {
    AMG_TRY(h->arena.get(&h->boD[j], n0));
    AMG_TRY(h->arena.get(&h->boQ[j], n0));
  }
  AMG_TRY(h->arena.get(&h->bo_scal, (size_t)kScalSlots * W));
  AMG_TRY(h->arena.get(&h->b_partial, (size_t)kRedBlocks * kBRed));
  AMG_TRY(h->arena.get(&h->b_ticket, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(h->b_ticket, 0, sizeof(unsigned), h->stream));
  if (f32) {
    AMG_TRY(h->arena.alloc(&h->b_r32, sizeof(float) * n0));
    AMG_TRY(h->arena.alloc(&h->b_z32, sizeof(float) * n0));
  }
  h->batch_blocks.assign(h->arena.blocks.begin() + (ptrdiff_t)blocks_before, h->arena.blocks.end());
  if (!h->b_pinned) AMG_CUDA_TRY(cudaMallocHost((void **)&h->b_pinned, sizeof(double) * 8 * kMaxBlock));
  h->bw = W;
  return AMG_OK;
}

static amg_status capture_batch_graph(amg_handle_s *h) {
  if (h->bpre_exec && !h->bpre_borrowed) cudaGraphExecDestroy(h->bpre_exec);
  h->bpre_exec = nullptr;
  h->bpre_borrowed = false;
  if (!h->use_graph) return AMG_OK;
  if (!h->cap) AMG_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  const cudaStream_t saved = h->stream;
  const int64_t saved_launches = h->launches;
  AMG_CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  h->stream = h->cap;
  h->capturing = true;
  const amg_status s = bprecondition(h);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  h->stream = saved;
  h->capturing = false;
  h->bgraph_kernels = h->launches - saved_launches;
  h->launches = saved_launches;
  if (s != AMG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&h->bpre_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    h->bpre_exec = nullptr;
    return fail(AMG_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e2));
  }
  return AMG_OK;
}

static amg_status run_bprecondition(amg_handle_s *h) {
  if (h->bpre_exec) {
    AMG_CUDA_TRY(cudaGraphLaunch(h->bpre_exec, h->stream));
    h->launches += h->bgraph_kernels;
    return AMG_OK;
  }
  return bprecondition(h);
}

static int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// decisions already made in this process, per problem shape
static std::mutex g_tune_mu;
static std::map<std::string, std::pair<int, int>> g_tuned;

// a block shape the block kernels support: kb a power of two up to kMaxBlock,
// the row tile one of the three timed sizes
static bool valid_shape(int kb, int tile) {
  return kb >= 1 && kb <= kMaxBlock && (kb & (kb - 1)) == 0 && (tile == 128 || tile == 256 || tile == 512);
}

// Pick (block width, SpMM tile) for `nrhs` columns by timing graph replays of
// the block preconditioner; the cost compared is time per column.  The
// choice is kept per (device, n, nnz, width cap, precision, degree, passes,
// aggregation, k, nu) for the process (later handles of the same shape reuse
// it) and, with AMG_GB300_TUNE_CACHE=<file>, in a JSON file across processes
// (an entry that is not a supported shape is ignored and the shape re-timed);
// AMG_GB300_BATCH=<kb>,<tile> forces one.
static amg_status autotune(amg_handle_s *h, int nrhs) {
  const int cap = std::min(kMaxBlock, pow2_at_least(nrhs));
  // the decision depends on the hierarchy's shape: key it by the problem and
  // every option that changes the levels or the cycle
  char key[200];
  snprintf(key, sizeof(key), "d%d_n%lld_nnz%lld_r%d_p%d_m%d_s%d_a%d_k%d_nu%d", h->device, (long long)h->n,
           (long long)h->lv[0].A.nnz, cap, h->opt.precision, h->opt.degree, h->opt.passes, h->opt.aggregation,
           h->opt.mis_k, h->opt.inner_iters);
  if (h->tuned_for == cap) return AMG_OK;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      h->bw_use = it->second.first;
      h->b_tile = it->second.second;
      h->tuned_for = cap;
      h->tune_log = std::string("process cache ") + key;
      return capture_batch_graph(h);
    }
  }
  if (const char *env = getenv("AMG_GB300_BATCH")) {
    int kb = 0, tile = 0;
    if (sscanf(env, "%d,%d", &kb, &tile) == 2 && valid_shape(kb, tile)) {
      h->bw_use = kb;
      h->b_tile = tile;
      h->tuned_for = cap;
      return capture_batch_graph(h);
    }
  }
  const char *cache = getenv("AMG_GB300_TUNE_CACHE");
  if (cache) {
    if (FILE *f = fopen(cache, "r")) {
      char buf[1 << 16];
      const size_t len = fread(buf, 1, sizeof(buf) - 1, f);
      buf[len] = 0;
      fclose(f);
      const std::string want = std::string("\"") + key + "\": [";
      if (const char *p = strstr(buf, want.c_str())) {
        int kb = 0, tile = 0;
        if (sscanf(p + want.size(), "%d, %d", &kb, &tile) == 2 && valid_shape(kb, tile) && kb <= cap) {
          h->bw_use = kb;
          h->b_tile = tile;
          h->tuned_for = cap;
          h->tune_log = std::string("file cache ") + key;
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tuned[key] = {kb, tile};
          return capture_batch_graph(h);
        }
      }
    }
  }
  cudaEvent_t e0, e1;
  AMG_CUDA_TRY(cudaEventCreate(&e0));
  AMG_CUDA_TRY(cudaEventCreate(&e1));
  double best = 1e300;
  int bkb = cap, btile = 256;
  std::string log;
  AMG_CUDA_TRY(cudaMemsetAsync(h->bo_r, 0, sizeof(double) * h->n * h->bw, h->stream));
  for (int kb = std::max(1, cap / 4); kb <= cap; kb *= 2) {
    for (int tile : {128, 256, 512}) {
      h->bw_use = kb;
      h->b_tile = tile;
      AMG_TRY(capture_batch_graph(h));
      AMG_TRY(run_bprecondition(h));
      AMG_CUDA_TRY(cudaEventRecord(e0, h->stream));
      for (int rep = 0; rep < 3; ++rep) AMG_TRY(run_bprecondition(h));
      AMG_CUDA_TRY(cudaEventRecord(e1, h->stream));
      AMG_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      AMG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      const double per_col = ms / 3.0 / kb;
      char item[96];
      snprintf(item, sizeof(item), "%s(%d,%d)=%.4f", log.empty() ? "" : " ", kb, tile, per_col);
      log += item;
      if (per_col < best) {
        best = per_col;
        bkb = kb;
        btile = tile;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->bw_use = bkb;
  h->b_tile = btile;
  h->tuned_for = cap;
  h->tune_log = log;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = {bkb, btile};
  }
  if (cache) {
    // append the decision (a flat JSON object, one key per line)
    std::string body;
    if (FILE *f = fopen(cache, "r")) {
      char buf[1 << 16];
      const size_t len = fread(buf, 1, sizeof(buf) - 1, f);
      buf[len] = 0;
      fclose(f);
      body = buf;
    }
    const size_t close = body.rfind('}');
    std::string entry = std::string("  \"") + key + "\": [" + std::to_string(bkb) + ", " + std::to_string(btile) + "]";
    if (close == std::string::npos || body.find('"') == std::string::npos) body = "{\n" + entry + "\n}\n";
    else body = body.substr(0, close) + ",\n" + entry + "\n}\n";
    if (FILE *f = fopen(cache, "w")) {
      fputs(body.c_str(), f);
      fclose(f);
    }
  }
  return capture_batch_graph(h);
}

// one block of nr (<= kb) columns: outer flexible CG per column, fp64
static amg_status solve_block(amg_handle_s *h, const double *rhs, double *x, int nr, int64_t ld, double tol,
                              amg_info *info, int *iters, double *rel, double *true_rel, int *conv,
                              bool *breakdown, ColumnReport *cols) {
  const int kb = h->bw_use, n = (int)h->n, R = h->opt.restart;
  const int64_t nk = (int64_t)n * kb;
  cudaStream_t st = h->stream;
  amg::Level &L0 = h->lv[0];
  double *sc = h->bo_scal, *hp = h->b_pinned;
  AMG_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * kScalSlots * kb, st));
  AMG_TRY(plaunch(h, st, k_bpack, dim3(nblk(nk)), dim3(kThreads), n, kb, nr, ld, rhs, h->bo_b));
  BLAUNCH(h);
  if (h->pure) {
    BDots<double> sp{};
    sp.a[0] = h->bo_b;
    sp.nd = 1;
    AMG_TRY(bdots<double>(h, n, sp, BFin{BF_MEAN, S_MEAN, (double)n, sc}));
    AMG_TRY(plaunch(h, st, k_bshift, dim3(nblk(nk)), dim3(kThreads), nk, kb, (const double *)h->bo_b, h->bo_b,
                    (const double *)(sc + S_MEAN * kb)));
    BLAUNCH(h);
  }
  {
    BDots<double> sp{};
    sp.a[0] = h->bo_b;
    sp.b[0] = h->bo_b;
    sp.nd = 1;
    AMG_TRY(bdots<double>(h, n, sp, BFin{BF_STORE, S_BB, 0.0, sc}));
  }
  AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + S_BB * kb, sizeof(double) * kb, cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaMemsetAsync(h->bo_x, 0, sizeof(double) * nk, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(h->bo_r, h->bo_b, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int c = 0; c < nr; ++c)
    if (!std::isfinite(hp[c]))
      return fail(AMG_ERR_INVALID_ARG, "right-hand side " + std::to_string(c) +
                                           " has a non-finite entry or a norm beyond the fp64 range");
  std::vector<double> nb(kb), res(kb, 0.0);
  std::vector<int> done(kb, 0), brk(kb, 0), col_it(kb, 0);
  int remaining = 0;
  for (int c = 0; c < kb; ++c) {
    nb[c] = sqrt(hp[c]);
    done[c] = (c >= nr || nb[c] == 0.0);
    res[c] = nb[c] > 0.0 ? 1.0 : 0.0;
    remaining += !done[c];
    hp[kb + c] = done[c] ? 1.0 : 0.0;
  }
  AMG_CUDA_TRY(cudaMemcpyAsync(sc + S_FROZEN * kb, hp + kb, sizeof(double) * kb, cudaMemcpyHostToDevice, st));
  int hl = 0;
  if (info && info->history && info->history_cap > 0) info->history[hl++] = res[0];
  int it = 0, nwin = 0;
  while (remaining > 0 && it < h->opt.max_iters) {
    if (it % R == 0) nwin = 0;
    double *d = h->boD[nwin], *q = h->boQ[nwin];
    AMG_TRY(run_bprecondition(h));
    if (nwin > 0) {
      BDots<double> sp{};
      for (int j = 0; j < nwin; ++j) {
        sp.a[j] = h->boQ[j];
        sp.b[j] = h->bo_z;
      }
      sp.nd = nwin;
      AMG_TRY(bdots<double>(h, n, sp, BFin{BF_OBETA, 0, 0.0, sc}));
    }
    {
      BDots<double> vd{};
      for (int j = 0; j < nwin; ++j) vd.a[j] = h->boD[j];
      vd.nd = nwin;
      AMG_TRY(plaunch(h, st, k_baxpy_multi<double>, dim3(nblk(nk)), dim3(kThreads), nk, kb, d,
                      (const double *)h->bo_z, vd, (const double *)(sc + S_BETA * kb)));
      BLAUNCH(h);
    }
    {
      BDots<double> sp{};
      sp.a[0] = d;
      sp.b[0] = nullptr;  // d . (A d)
      sp.a[1] = d;
      sp.b[1] = h->bo_r;
      sp.nd = 2;
      AMG_TRY(bspmv_dots<double>(h, L0, d, q, sp, BFin{BF_OALPHA, nwin, 0.0, sc}));
    }
    AMG_TRY(plaunch(h, st, k_bouter_update, dim3(bred_grid(n, kb)), dim3(kThreads), n, kb, (const double *)sc,
                    (const double *)d, (const double *)q, h->bo_x, h->bo_r, h->b_partial, h->b_ticket,
                    BFin{BF_STORE, S_RR, 0.0, sc}));
    BLAUNCH(h);
    AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + S_RR * kb, sizeof(double) * 2 * kb, cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    ++nwin;
    ++it;
    bool changed = false;
    for (int c = 0; c < kb; ++c) {
      if (done[c]) continue;
      if (hp[kb + c] != 0.0) {  // S_BREAK row follows S_RR
        brk[c] = 1;
        done[c] = 1;
        --remaining;
        changed = true;
        continue;
      }
      res[c] = sqrt(hp[c]) / nb[c];
      col_it[c] = it;
      if (res[c] <= tol) {
        done[c] = 1;
        --remaining;
        changed = true;
      }
    }
    if (info && info->history && hl < info->history_cap && !brk[0]) info->history[hl++] = res[0];
    if (changed) {
      for (int c = 0; c < kb; ++c) hp[2 * kb + c] = done[c] ? 1.0 : 0.0;
      AMG_CUDA_TRY(cudaMemcpyAsync(sc + S_FROZEN * kb, hp + 2 * kb, sizeof(double) * kb, cudaMemcpyHostToDevice, st));
    }
  }
  if (h->pure) {
    BDots<double> sp{};
    sp.a[0] = h->bo_x;
    sp.nd = 1;
    AMG_TRY(bdots<double>(h, n, sp, BFin{BF_MEAN, S_MEAN, (double)n, sc}));
    AMG_TRY(plaunch(h, st, k_bshift, dim3(nblk(nk)), dim3(kThreads), nk, kb, (const double *)h->bo_x, h->bo_x,
                    (const double *)(sc + S_MEAN * kb)));
    BLAUNCH(h);
  }
  {
    // true residuals ||b - A x|| per column
    AMG_TRY(plaunch(h, st, k_bresidual<double>, dim3(nblk(nk)), dim3(kThreads), bview<double>(L0), kb,
                    (const double *)h->bo_x, (const double *)h->bo_b, h->bo_t));
    BLAUNCH(h);
    BDots<double> sp{};
    sp.a[0] = h->bo_t;
    sp.b[0] = h->bo_t;
    sp.nd = 1;
    AMG_TRY(bdots<double>(h, n, sp, BFin{BF_STORE, S_TRUE, 0.0, sc}));
    AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + S_TRUE * kb, sizeof(double) * kb, cudaMemcpyDeviceToHost, st));
  }
  AMG_TRY(plaunch(h, st, k_bunpack, dim3(nblk(nk)), dim3(kThreads), n, kb, nr, ld, (const double *)h->bo_x, x));
  BLAUNCH(h);
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) info->history_len = hl;
  double mrel = 0.0, mtrue = 0.0;
  int all = 1;
  bool anybrk = false;
  for (int c = 0; c < nr; ++c) {
    mrel = std::max(mrel, res[c]);
    const double tr = nb[c] > 0.0 ? sqrt(hp[c]) / nb[c] : 0.0;
    mtrue = std::max(mtrue, tr);
    all &= (done[c] && !brk[c]);
    anybrk |= brk[c] != 0;
    if (cols) {
      cols[c].iterations = col_it[c];
      cols[c].rel_residual = res[c];
      cols[c].true_rel_residual = tr;
      cols[c].converged = done[c] && !brk[c];
      cols[c].breakdown = brk[c] != 0;
    }
  }
  *iters = it;
  *rel = mrel;
  *true_rel = mtrue;
  *conv = all;
  *breakdown = anybrk;
  return AMG_OK;
}

// Buffers and the captured block preconditioner for solves at a fixed width
// (the server calls this right after a setup, so that the hierarchy's arena
// bytes include them).
// One captured block preconditioner per fixed width is kept, so that solves
// alternating between widths replay instead of re-capturing.
amg_status prepare_batched(amg_handle_s *h, int width) {
  if (!valid_shape(width, 256)) return fail(AMG_ERR_INVALID_ARG, "block width must be 1, 2, 4, 8, 16 or 32");
  AMG_TRY(ensure_batch_buffers(h, width));
  if (h->tuned_for == -width && (h->bpre_exec || !h->use_graph)) return AMG_OK;
  int slot = 0;
  while ((1 << slot) < width) ++slot;
  h->bw_use = width;
  h->b_tile = 256;
  h->tuned_for = -width;
  if (!h->use_graph) return AMG_OK;
  if (!h->bfixed[slot]) {
    AMG_TRY(capture_batch_graph(h));
    h->bfixed[slot] = h->bpre_exec;       // the cache owns it from here
    h->bfixed_kernels[slot] = h->bgraph_kernels;
  }
  h->bpre_exec = h->bfixed[slot];
  h->bpre_borrowed = true;
  h->bgraph_kernels = h->bfixed_kernels[slot];
  return AMG_OK;
}

void release_block_graphs(amg_handle_s *h) { drop_block_graphs(h); }

// Solve nrhs right-hand sides (device pointers, column major with ld) in
// blocks of the tuned width, or of a fixed width.
amg_status solve_batched(amg_handle_s *h, const double *rhs, double *x, int nrhs, int64_t ld, double tol,
                         amg_info *info, int *iters, double *rel, double *true_rel, int *conv, bool *breakdown,
                         int fixed_width, ColumnReport *cols) {
  if (fixed_width > 0) {
    // a block shape that does not depend on nrhs: every column runs the same
    // kernels at the same width whatever else shares its block
    if (!valid_shape(fixed_width, 256)) return fail(AMG_ERR_INVALID_ARG, "block width must be 1, 2, 4, 8, 16 or 32");
    AMG_TRY(prepare_batched(h, fixed_width));
  } else {
    AMG_TRY(ensure_batch_buffers(h, std::min(kMaxBlock, pow2_at_least(nrhs))));
    AMG_TRY(autotune(h, nrhs));
  }
  int mit = 0, all = 1;
  double mrel = 0.0, mtrue = 0.0;
  bool brk = false;
  for (int c0 = 0; c0 < nrhs; c0 += h->bw_use) {
    const int nr = std::min(h->bw_use, nrhs - c0);
    int it = 0, cv = 0;
    double r1 = 0.0, t1 = 0.0;
    bool b1 = false;
    AMG_TRY(solve_block(h, rhs + (int64_t)c0 * ld, x + (int64_t)c0 * ld, nr, ld, tol, c0 == 0 ? info : nullptr,
                        &it, &r1, &t1, &cv, &b1, cols ? cols + c0 : nullptr));
    mit = std::max(mit, it);
    mrel = std::max(mrel, r1);
    mtrue = std::max(mtrue, t1);
    all &= cv;
    brk |= b1;
  }
  *iters = mit;
  *rel = mrel;
  *true_rel = mtrue;
  *conv = all;
  *breakdown = brk;
  return AMG_OK;
}

}  // namespace amg
