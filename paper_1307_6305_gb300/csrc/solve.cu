// solve.cu -- solve phase: flexible CG preconditioned by the nonlinear AMLI
// cycle (K-cycle) with the polynomial smoother (Sec. 3, Sec. 4).
//
// Kernels (templated on the cycle precision T = double or float):
//   k_cheb_first / k_cheb_step : one SpMV on the SELL-32 operator fused with
//       one step of the Chebyshev three-term recurrence for q_m(A) r and the
//       accumulation x += c_j T_j (Sec. 3 smoother R = q_m(A));
//   k_residual                 : s = r - A x
//       (these two groups live in sell_kernels.cuh);
//   k_restrict / k_prolong_add : r_H = P^T s (sum over aggregate members in
//       ascending order) and x += P e_H (Eq. (coarse));
//   k_dots                     : up to kMaxDots dot products in one pass,
//       deterministic two-stage reduction whose last block also derives the
//       Krylov scalars (alpha, beta, rho) on the device;
//   k_axpy_multi / k_*_update  : Krylov vector updates reading those scalars.
// The host walks the cycle and issues launches; it reads one scalar per
// outer iteration (the residual norm for the stopping test).
#include <math.h>

#include <cmath>
#include <stdlib.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "block_kernels.cuh"
#include "sell_kernels.cuh"

namespace amg {

#define SLAUNCH(h)                                                                  \
  do {                                                                              \
    ++(h)->launches;                                                                \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)


// r_H = P^T s; `flag`, when given, is the next level's inner-CG stop flag,
// cleared here because the inner solve on r_H starts right after.  One
// thread per aggregate, members in ascending order.
template <typename T>
__global__ void k_restrict(int nH, const int *__restrict__ ptr, const int *__restrict__ mem,
                           const T *__restrict__ s, T *__restrict__ rH, double *flag) {
  pdl_sync();
  if (flag && blockIdx.x == 0 && threadIdx.x == 0) *flag = 0.0;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nH) return;
  T acc = T(0);
#pragma unroll 4
  for (int a = ptr[I]; a < ptr[I + 1]; ++a) acc += s[mem[a]];
  rH[I] = acc;
}

// The same with the member table of a matching hierarchy: at most W = 2^passes
// members per aggregate, stored column-major (member k of aggregate I at
// memw[k * nH + I], ascending, -1 after the last), so a thread issues its W
// member loads at once, coalesced across the warp, with no row-pointer load
// before them; the sum is taken in the same order as k_restrict.
template <typename T, int W>
__global__ void k_restrict_w(int nH, const int *__restrict__ memw, const T *__restrict__ s, T *__restrict__ rH,
                             double *flag) {
  pdl_sync();
  if (flag && blockIdx.x == 0 && threadIdx.x == 0) *flag = 0.0;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nH) return;
  int m[W];
#pragma unroll
  for (int k = 0; k < W; ++k) m[k] = memw[(size_t)k * nH + I];
  T v[W];
#pragma unroll
  for (int k = 0; k < W; ++k) v[k] = m[k] >= 0 ? s[m[k]] : T(0);
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (m[k] >= 0) acc += v[k];
  rH[I] = acc;
}


template <typename T>
__global__ void k_prolong_add(int n, const int *__restrict__ agg, const T *__restrict__ eH,
                              T *__restrict__ x) {
  pdl_sync();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += eH[agg[i]];
}

// x = u + P e_H (the prolonged coarse correction added to the pre-smoothed u)
// four rows per thread with 16-byte loads and stores of agg, u and x when
// all three start on a 16-byte boundary (the library's own buffers do; a
// caller's vector passed to a single-step entry point may not), the tail of
// n mod 4 rows and unaligned vectors one by one
template <typename T>
__global__ void k_prolong_set(int n, const int *__restrict__ agg, const T *__restrict__ eH,
                              const T *__restrict__ u, T *__restrict__ x) {
  pdl_sync();
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= n) return;
  const bool aligned =
      ((reinterpret_cast<uintptr_t>(agg) | reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(x)) & 15u) == 0;
  if (aligned && i0 + 3 < n) {
    const int4 a = *reinterpret_cast<const int4 *>(agg + i0);
    if constexpr (sizeof(T) == 8) {
      const double2 u0 = *reinterpret_cast<const double2 *>(u + i0);
      const double2 u1 = *reinterpret_cast<const double2 *>(u + i0 + 2);
      const double2 x0 = make_double2(u0.x + eH[a.x], u0.y + eH[a.y]);
      const double2 x1 = make_double2(u1.x + eH[a.z], u1.y + eH[a.w]);
      *reinterpret_cast<double2 *>(x + i0) = x0;
      *reinterpret_cast<double2 *>(x + i0 + 2) = x1;
    } else {
      const float4 uv = *reinterpret_cast<const float4 *>(u + i0);
      *reinterpret_cast<float4 *>(x + i0) = make_float4(uv.x + eH[a.x], uv.y + eH[a.y], uv.z + eH[a.z], uv.w + eH[a.w]);
    }
    return;
  }
  for (int i = i0; i < min(n, i0 + 4); ++i) x[i] = u[i] + eH[agg[i]];
}

template <typename A, typename B>
__global__ void k_convert(int64_t n, const A *__restrict__ a, B *__restrict__ b) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// coarsest solve: x = Z b, one warp per row, fp64
__global__ void k_dense_mv(int n, const double *__restrict__ Z, const double *__restrict__ b,
                           double *__restrict__ x) {
  pdl_sync();
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc = fma(Z[(int64_t)row * n + j], b[j], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = acc;
}

// ---------------------------------------------------------------------------
// fused dot products with on-device finalisation
// ---------------------------------------------------------------------------
enum FinKind : int {
  FIN_STORE = 0,   // scal[o0 + q] = sum_q
  FIN_IBETA = 1,   // inner: scal[16 + l] = sum_l / scal[l], l < nd
  FIN_IALPHA = 2,  // inner step o0: rho = s0, alpha = s1 / rho; stop flag scal[24]
  FIN_OBETA = 3,   // outer: scal[16 + j] = sum_j / scal[j]
  FIN_OALPHA = 4,  // outer slot o0: rho = s0, alpha = s1 / rho -> scal[32]; breakdown scal[34]
  FIN_MEAN = 5     // scal[o0] = s0 / o1 (o1 = n)
};

struct Fin {
  int kind;
  int o0;
  double o1;
  double *scal;
};

template <typename T>
struct DotSpec {
  const T *a[kMaxDots];
  const T *b[kMaxDots];  // nullptr: sum of a
  int nd;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ void finalize(const Fin &f, const double *sums, int nd) {
  double *sc = f.scal;
  switch (f.kind) {
    case FIN_STORE:
      for (int q = 0; q < nd; ++q) sc[f.o0 + q] = sums[q];
      break;
    case FIN_IBETA:
      for (int l = 0; l < nd; ++l) sc[16 + l] = sums[l] / sc[l];
      break;
    case FIN_IALPHA: {
      const double rho = sums[0], sig = sums[1];
      sc[f.o0] = rho;
      if (sc[24] != 0.0 || !(rho > 0.0) || !isfinite(rho)) {
        sc[24] = 1.0;
        sc[8 + f.o0] = 0.0;
      } else {
        sc[8 + f.o0] = sig / rho;
      }
      break;
    }
    case FIN_OBETA:
      for (int j = 0; j < nd; ++j) sc[16 + j] = sums[j] / sc[j];
      break;
    case FIN_OALPHA: {
      const double rho = sums[0], sig = sums[1];
      sc[f.o0] = rho;
      if (!(rho > 0.0) || !isfinite(rho)) {
        sc[34] = 1.0;
        sc[32] = 0.0;
      } else {
        sc[32] = sig / rho;
      }
      break;
    }
    case FIN_MEAN:
      sc[f.o0] = sums[0] / f.o1;
      break;
  }
}

// per-thread partial sums -> per-block partials -> last block folds the
// partials in block order (deterministic for a fixed grid) and finalises
// (every step of a warp shuffle tree is a full-warp FP64 add, and this part's
// FP64 pipe issues 2 lanes per clock: the block's partials go through shared
// memory and one warp adds them -- 8 sequential adds and one 5-step tree per
// dot instead of a tree in each of the 8 warps)
template <int ND>
__device__ __forceinline__ void reduce_and_finalize(const double (&acc)[ND], double *partial,
                                                    unsigned *ticket, const Fin &fin) {
  __shared__ double sh[ND][kThreads];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) v += sh[q][w * 32 + lane];
      v = warp_sum(v);
      if (lane == 0) partial[blockIdx.x * kMaxDots + q] = v;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  // the last block folds the partials with all its threads (each loads at
  // most gridDim / kThreads of them, in one round of independent loads),
  // then a fixed tree: thread partials -> warp sums -> warps in order
  double v[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) v[q] = 0.0;
#pragma unroll 4
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) {
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] += __ldcg(&partial[b * kMaxDots + q]);
  }
#pragma unroll
  for (int q = 0; q < ND; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  if (warp == 0) {
    double sums[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) t += sh[q][w * 32 + lane];
      sums[q] = warp_sum(t);
    }
    if (lane == 0) {
      finalize(fin, sums, ND);
      *ticket = 0u;
    }
  }
}

template <typename T, int ND>
__global__ void __launch_bounds__(kThreads) k_dots(int64_t n, DotSpec<T> spec, double *partial,
                                                   unsigned *ticket, Fin fin) {
  pdl_sync();
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  // E elements per thread and trip, kThreads apart (coalesced); all loads of
  // a trip are issued before the first product (a null b operand reads as 1:
  // a * 1 == a exactly).  Fewer elements per trip for many dots keep the
  // registers of a thread below 128.
  constexpr int E = ND <= 2 ? kRedElems : 2;
  for (int64_t base = (int64_t)blockIdx.x * (kThreads * E) + threadIdx.x; base < n;
       base += (int64_t)gridDim.x * (kThreads * E)) {
    T av[ND][E], bv[ND][E];
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const int64_t i = base + (int64_t)u * kThreads;
      const bool in = i < n;
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        av[q][u] = in ? spec.a[q][i] : T(0);
        bv[q][u] = (in && spec.b[q]) ? spec.b[q][i] : T(1);
      }
    }
#pragma unroll
    for (int u = 0; u < E; ++u) {
      if (base + (int64_t)u * kThreads < n) {
#pragma unroll
        for (int q = 0; q < ND; ++q) acc[q] += (double)av[q][u] * (double)bv[q][u];
      }
    }
  }
  reduce_and_finalize<ND>(acc, partial, ticket, fin);
}

// y = A x fused with ND dot products; a null operand pointer stands for y
template <typename T, int ND, int WPS>
__global__ void __launch_bounds__(kThreads) k_spmv_dots(SellView<T> A, const T *__restrict__ x,
                                                        T *__restrict__ y, DotSpec<T> spec,
                                                        double *partial, unsigned *ticket, Fin fin) {
  pdl_sync();
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  auto accumulate = [&](int i, T yi) {
    y[i] = yi;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const double a = spec.a[q] ? (double)spec.a[q][i] : (double)yi;
      const double b = spec.b[q] ? (double)spec.b[q][i] : (double)yi;
      acc[q] += a * b;
    }
  };
  if constexpr (WPS == 1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
      accumulate(i, apply_row(A, x, i));
  } else {
    __shared__ T part[kThreads / 32][32];
    const int groups = (((A.n + kSlice - 1) / kSlice) * WPS + kThreads / 32 - 1) / (kThreads / 32);
    for (int g = blockIdx.x; g < groups; g += gridDim.x) {  // block-uniform trip count
      const SplitIdx ix = split_index<WPS>(g);
      const T xi = ix.i < A.n ? x[ix.i] : T(0);
      T yi;
      if (split_row<T, WPS>(A, ix, xi, [&](int j) { return x[j]; }, yi, part)) accumulate(ix.i, yi);
      __syncthreads();  // part is rewritten by the next group
    }
  }
  reduce_and_finalize<ND>(acc, partial, ticket, fin);
}

// inner step it > 0: D -= sum_l beta_l D_l, W -= sum_l beta_l W_l, then
// rho = D.W and sigma = D.rin (FIN_IALPHA); a trip's loads are issued before
// its arithmetic
template <typename T>
__global__ void __launch_bounds__(kThreads) k_orth_dots(int64_t n, T *__restrict__ D, T *__restrict__ W,
                                                        DotSpec<T> prev, const double *beta,
                                                        const T *__restrict__ rin, double *partial,
                                                        unsigned *ticket, Fin fin) {
  pdl_sync();
  double acc[2] = {0.0, 0.0};
  for (int64_t base = (int64_t)blockIdx.x * (kThreads * kRedElems) + threadIdx.x; base < n;
       base += (int64_t)gridDim.x * (kThreads * kRedElems)) {
    T d[kRedElems], w[kRedElems], ri[kRedElems];
#pragma unroll
    for (int u = 0; u < kRedElems; ++u) {
      const int64_t i = base + (int64_t)u * kThreads;
      const bool in = i < n;
      d[u] = in ? D[i] : T(0);
      w[u] = in ? W[i] : T(0);
      ri[u] = in ? rin[i] : T(0);
    }
    for (int l = 0; l < prev.nd; ++l) {
      const T bl = (T)beta[l];
      T pa[kRedElems], pb[kRedElems];
#pragma unroll
      for (int u = 0; u < kRedElems; ++u) {
        const int64_t i = base + (int64_t)u * kThreads;
        const bool in = i < n;
        pa[u] = in ? prev.a[l][i] : T(0);
        pb[u] = in ? prev.b[l][i] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kRedElems; ++u) {
        d[u] -= bl * pa[u];
        w[u] -= bl * pb[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kRedElems; ++u) {
      const int64_t i = base + (int64_t)u * kThreads;
      if (i < n) {
        D[i] = d[u];
        W[i] = w[u];
        acc[0] += (double)d[u] * (double)w[u];
        acc[1] += (double)d[u] * (double)ri[u];
      }
    }
  }
  reduce_and_finalize<2>(acc, partial, ticket, fin);
}

// x_out = u + P e_H and s = r - A x_out in one pass: neighbours' values are
// formed on the fly as u_j + e_H[agg_j] (the same rounding as forming x_out
// first), so x_out never needs a second read
template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_prolong_residual(SellView<T> A, const int *__restrict__ agg,
                                                               const T *__restrict__ eH,
                                                               const T *__restrict__ u, const T *__restrict__ r,
                                                               T *__restrict__ xout, T *__restrict__ s) {
  pdl_sync();
  if constexpr (WPS > 1) {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const T xi = ix.i < A.n ? u[ix.i] + eH[agg[ix.i]] : T(0);
    T Ax;
    if (split_row<T, WPS>(A, ix, xi, [&](int j) { return u[j] + eH[agg[j]]; }, Ax, part)) {
      xout[ix.i] = xi;
      s[ix.i] = r[ix.i] - Ax;
    }
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const T xi = u[i] + eH[agg[i]];
  xout[i] = xi;
  const int sl = i >> 5, lane = i & 31;
  const int64_t base = A.sptr[sl];
  const int w = (int)((A.sptr[sl + 1] - base) >> 5);
  const T *__restrict__ v = A.val + base + lane;
  T acc = A.diag[i] * xi;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int64_t pos = base + lane + (int64_t)k * kSlice;
    const int j = sell_col(A, pos, i);
    acc = fma(A.stream ? __ldcs(v + k * kSlice) : v[k * kSlice], u[j] + eH[agg[j]], acc);
  }
  s[i] = r[i] - acc;
}

// y = z - sum_l beta_l V_l (beta read from the device)
template <typename T>
__global__ void k_axpy_multi(int64_t n, T *y, const T *z, DotSpec<T> V, const double *beta) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T v = z[i];
  for (int l = 0; l < V.nd; ++l) v -= (T)beta[l] * V.a[l][i];
  y[i] = v;
}

// inner flexible CG update of step `it` (scalars in sc):
//   x = alpha D (it == 0) or x += alpha D; r = rin - alpha W when `upd_r`
template <typename T>
__global__ void k_inner_update(int64_t n, int it, bool upd_r, const double *sc, const T *D,
                               const T *W, const T *rin, T *x, T *r) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool stopped_here = sc[24] != 0.0 && sc[8 + it] == 0.0;
  const T a = (T)sc[8 + it];
  if (it == 0) x[i] = stopped_here ? T(0) : a * D[i];
  else if (!stopped_here) x[i] = fma(a, D[i], x[i]);
  if (upd_r) r[i] = stopped_here ? rin[i] : rin[i] - a * W[i];
}

// outer update: x += alpha d, r -= alpha q, then r.r (a trip's loads first)
__global__ void __launch_bounds__(kThreads) k_outer_update(int64_t n, const double *sc,
                                                           const double *__restrict__ d,
                                                           const double *__restrict__ q, double *__restrict__ x,
                                                           double *__restrict__ r, double *partial,
                                                           unsigned *ticket, Fin fin) {
  pdl_sync();
  double acc[1] = {0.0};
  const double a = sc[32];
  for (int64_t base = (int64_t)blockIdx.x * (kThreads * kRedElems) + threadIdx.x; base < n;
       base += (int64_t)gridDim.x * (kThreads * kRedElems)) {
    double dv[kRedElems], qv[kRedElems], xv[kRedElems], rv[kRedElems];
#pragma unroll
    for (int u = 0; u < kRedElems; ++u) {
      const int64_t i = base + (int64_t)u * kThreads;
      const bool in = i < n;
      dv[u] = in ? d[i] : 0.0;
      qv[u] = in ? q[i] : 0.0;
      xv[u] = in ? x[i] : 0.0;
      rv[u] = in ? r[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kRedElems; ++u) {
      const int64_t i = base + (int64_t)u * kThreads;
      if (i < n) {
        x[i] = fma(a, dv[u], xv[u]);
        const double ri = fma(-a, qv[u], rv[u]);
        r[i] = ri;
        acc[0] += ri * ri;
      }
    }
  }
  reduce_and_finalize<1>(acc, partial, ticket, fin);
}

// stationary AMLI coarse correction e = sum_p c_p T_p(tau(BA)) B r:
// e = c_0 T_0 (first term)
template <typename T>
__global__ void k_amli_first(int64_t n, const T *__restrict__ T0, T *__restrict__ e, T c0) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e[i] = c0 * T0[i];
}

// one recurrence step: t = tau(BA) T_{p-1} = sA w - sB T_{p-1} with w = B A T_{p-1};
// T_p = t (p = 1) or 2 t - T_{p-2}; e += c_p T_p
template <typename T>
__global__ void k_amli_step(int64_t n, const T *__restrict__ w, const T *__restrict__ Tc,
                            const T *__restrict__ Tp, T *__restrict__ Tn, T *__restrict__ e, T sA, T sB,
                            T cp, int first) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T t = fma(sA, w[i], -sB * Tc[i]);
  const T tn = first ? t : T(2) * t - Tp[i];
  Tn[i] = tn;
  e[i] = fma(cp, tn, e[i]);
}

__global__ void k_shift(int64_t n, const double *src, double *dst, const double *mean) {
  pdl_sync();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] - *mean;
}

__global__ void k_identity(int n, double *__restrict__ X) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  X[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// host side
// blocks of a streaming reduction over n elements: trips of kRedElems
// elements per thread, at most kRedBlocks blocks (each block ends with FP64
// reduction work, so fewer, fuller blocks are cheaper on this part)
static inline unsigned red_grid(const amg_handle_s *h, int64_t n) {
  (void)h;
  const int64_t per = (int64_t)kThreads * kRedElems;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(kRedBlocks, (n + per - 1) / per));
}

// blocks of the SELL kernels: (slices x WPS) warps, kThreads / 32 per block
static inline unsigned sell_grid(int n, int wps) {
  const int64_t warps = (int64_t)((n + kSlice - 1) / kSlice) * wps;
  return (unsigned)std::max<int64_t>(1, (warps + kThreads / 32 - 1) / (kThreads / 32));
}

// Warps per slice for a level of n rows: the smallest of 1, 2, 4, 8 that
// gives at least `per_sm` warps per SM (152 SMs), so that small levels
// spread their work and their dependent loads over the GPU.  per_sm is 16
// for fp64 levels and 32 for fp32 (AMG_GB300_WPS_WARPS overrides): on the
// 128^3 hierarchy these give the 45K-row level 2 and 4 warps per slice;
// measured per solve, fp64 31.35-31.44 ms with 2 against 31.59-31.62 with 4,
// fp32 24.42-24.45 ms with 4 against 24.98-25.06 with 2 (8: +0.8-0.9 ms).
int choose_wps(int n, int per_sm) {
  const int64_t slices = (n + kSlice - 1) / kSlice;
  int w = 1;
  while (w < 8 && slices * w < (int64_t)per_sm * 152) w *= 2;
  return w;
}

// call f(std::integral_constant<int, WPS>) for the level's WPS
template <typename F>
static amg_status with_wps(int wps, F f) {
  switch (wps) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 2: return f(std::integral_constant<int, 2>{});
    default: return f(std::integral_constant<int, 1>{});
  }
}

// 16-bit column offsets serve the one-row-per-thread kernels (bandwidth-
// bound levels); the split kernels of small levels keep 32-bit columns
// (with offsets they measured slower: one more step in each entry's
// dependent load chain)
static inline const int16_t *delta_cols(const amg::Level &L) { return L.wps == 1 ? L.S.sdel : nullptr; }

template <typename T>
static SellView<T> view(const amg::Level &L);
template <>
SellView<double> view<double>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.val64, L.S.diag64, L.stream, delta_cols(L)};
}
template <>
SellView<float> view<float>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.val32, L.S.diag32, L.stream, delta_cols(L)};
}

template <typename T>
static SellView<T> smoother_view(const amg::Level &L);
template <>
SellView<double> smoother_view<double>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.sval64, L.S.sdiag64, L.stream, delta_cols(L)};
}
template <>
SellView<float> smoother_view<float>(const amg::Level &L) {
  return {L.n, L.S.sptr, L.S.scol, L.S.sval32, L.S.sdiag32, L.stream, delta_cols(L)};
}

// r_H = P^T s on level k (the fixed-width member table when the level has one)
template <typename T>
static amg_status restrict_to(amg_handle_s *h, int k, const T *s, T *rH, double *flag) {
  amg::Level &L = h->lv[k];
  cudaStream_t st = h->stream;
  const dim3 g(nblk(L.nH));
  switch (L.memw ? L.memw_width : 0) {
    case 2: AMG_TRY(plaunch(h, st, k_restrict_w<T, 2>, g, dim3(kThreads), L.nH, L.memw, s, rH, flag)); break;
    case 4: AMG_TRY(plaunch(h, st, k_restrict_w<T, 4>, g, dim3(kThreads), L.nH, L.memw, s, rH, flag)); break;
    case 8: AMG_TRY(plaunch(h, st, k_restrict_w<T, 8>, g, dim3(kThreads), L.nH, L.memw, s, rH, flag)); break;
    default: AMG_TRY(plaunch(h, st, k_restrict<T>, g, dim3(kThreads), L.nH, L.agg_ptr, L.agg_mem, s, rH, flag));
  }
  SLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status dots(amg_handle_s *h, int64_t n, const DotSpec<T> &spec, Fin fin) {
  const unsigned g = red_grid(h, n);
  double *P = h->red.partial;
  unsigned *tk = h->red.ticket;
  cudaStream_t st = h->stream;
  switch (spec.nd) {
    case 1: AMG_TRY(plaunch(h, st, k_dots<T, 1>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 2: AMG_TRY(plaunch(h, st, k_dots<T, 2>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 3: AMG_TRY(plaunch(h, st, k_dots<T, 3>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 4: AMG_TRY(plaunch(h, st, k_dots<T, 4>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 5: AMG_TRY(plaunch(h, st, k_dots<T, 5>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 6: AMG_TRY(plaunch(h, st, k_dots<T, 6>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    case 7: AMG_TRY(plaunch(h, st, k_dots<T, 7>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
    default: AMG_TRY(plaunch(h, st, k_dots<T, 8>, dim3(g), dim3(kThreads), n, spec, P, tk, fin)); break;
  }
  SLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status spmv_dots(amg_handle_s *h, int k, const T *x, T *y, const DotSpec<T> &spec, Fin fin) {
  amg::Level &L = h->lv[k];
  double *P = h->red.partial;
  unsigned *tk = h->red.ticket;
  cudaStream_t st = h->stream;
  const SellView<T> A = view<T>(L);
  if (L.wps > 1 && spec.nd <= 2) {  // the inner solve's shapes (nu = 2) take the split form
    const unsigned g = std::min<unsigned>(kRedBlocks, sell_grid(L.n, L.wps));
    AMG_TRY(with_wps(L.wps, [&](auto W) {
      constexpr int wp = decltype(W)::value;
      if (spec.nd == 1) return plaunch(h, st, k_spmv_dots<T, 1, wp>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin);
      return plaunch(h, st, k_spmv_dots<T, 2, wp>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin);
    }));
    SLAUNCH(h);
    return AMG_OK;
  }
  const unsigned g = std::min<unsigned>(kRedBlocks, sell_grid(L.n, 1));
  switch (spec.nd) {
    case 1: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 1, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 2: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 2, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 3: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 3, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 4: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 4, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 5: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 5, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 6: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 6, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    case 7: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 7, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
    default: AMG_TRY(plaunch(h, st, k_spmv_dots<T, 8, 1>, dim3(g), dim3(kThreads), A, x, y, spec, P, tk, fin)); break;
  }
  SLAUNCH(h);
  return AMG_OK;
}

// record the next timing event; `kind` is stored with the first event of a pair
static amg_status timing_record(amg_handle_s *h, cudaEvent_t *ev, int kind = 0) {
  Timing &tm = h->timing;
  if (tm.used >= tm.ev.size()) {
    cudaEvent_t e;
    AMG_CUDA_TRY(cudaEventCreate(&e));
    tm.ev.push_back(e);
  }
  if (tm.used % 2 == 0) {
    const size_t pair = tm.used / 2;
    if (tm.kind.size() <= pair) tm.kind.resize(pair + 1, 0);
    tm.kind[pair] = kind;
  }
  *ev = tm.ev[tm.used++];
  if (h->capturing) AMG_CUDA_TRY(cudaEventRecordWithFlags(*ev, h->stream, cudaEventRecordExternal));
  else AMG_CUDA_TRY(cudaEventRecord(*ev, h->stream));
  return AMG_OK;
}

// add the elapsed times of the first `count` recorded events (pairs)
static amg_status timing_accumulate(amg_handle_s *h, size_t count) {
  Timing &tm = h->timing;
  for (size_t i = 0; i + 1 < count; i += 2) {
    float ms = 0.f;
    AMG_CUDA_TRY(cudaEventElapsedTime(&ms, tm.ev[i], tm.ev[i + 1]));
    const int k = tm.kind[i / 2];
    tm.total_ms[k] += ms;
    ++tm.launches[k];
  }
  return AMG_OK;
}

static amg_status timing_flush(amg_handle_s *h) {
  Timing &tm = h->timing;
  if (!tm.used) return AMG_OK;
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  AMG_TRY(timing_accumulate(h, tm.used));
  tm.used = 0;
  return AMG_OK;
}

// x (=|+=) q_m(A_k) r
template <typename T>
static amg_status smooth(amg_handle_s *h, int k, const T *r, T *x, bool add) {
  amg::Level &L = h->lv[k];
  const int m = h->opt.degree;
  const SellView<T> S = smoother_view<T>(L);  // 2 t(A) = 2 sa A - 2 ca I
  cudaStream_t st = h->stream;
  if (m == 0) {
    if (add) AMG_TRY(plaunch(h, st, k_scale<T, true>, dim3(nblk(L.n)), dim3(kThreads), L.n, r, x, (T)L.coef[0]));
    else AMG_TRY(plaunch(h, st, k_scale<T, false>, dim3(nblk(L.n)), dim3(kThreads), L.n, r, x, (T)L.coef[0]));
    SLAUNCH(h);
    return AMG_OK;
  }
  T *Ta = (T *)L.Ta, *Tb = (T *)L.Tb;
  const dim3 grid(sell_grid(L.n, L.wps));
  AMG_TRY(with_wps(L.wps, [&](auto W) {
    constexpr int wp = decltype(W)::value;
    if (add) return plaunch(h, st, k_cheb_first<T, true, wp>, grid, dim3(kThreads), S, r, Ta, x, (T)L.coef[0], (T)L.coef[1]);
    return plaunch(h, st, k_cheb_first<T, false, wp>, grid, dim3(kThreads), S, r, Ta, x, (T)L.coef[0], (T)L.coef[1]);
  }));
  SLAUNCH(h);
  const T *Tp = r;
  T *Tc = Ta;
  const bool timed = h->timing.enabled && k == 0;
  for (int j = 2; j <= m; ++j) {
    T *Tn = (j == 2) ? Tb : const_cast<T *>(Tp);
    cudaEvent_t e0, e1;
    if (timed) AMG_TRY(timing_record(h, &e0));
    AMG_TRY(with_wps(L.wps, [&](auto W) {
      return plaunch(h, st, k_cheb_step<T, decltype(W)::value>, grid, dim3(kThreads), S, Tc, Tp, Tn, x, (T)L.coef[j]);
    }));
    SLAUNCH(h);
    if (timed) AMG_TRY(timing_record(h, &e1));
    Tp = Tc;
    Tc = Tn;
  }
  return AMG_OK;
}

template <typename T>
static amg_status residual(amg_handle_s *h, int k, const T *x, const T *r, T *s) {
  amg::Level &L = h->lv[k];
  AMG_TRY(with_wps(L.wps, [&](auto W) {
    return plaunch(h, h->stream, k_residual<T, decltype(W)::value>, dim3(sell_grid(L.n, L.wps)), dim3(kThreads),
                   view<T>(L), x, r, s);
  }));
  SLAUNCH(h);
  return AMG_OK;
}

// x = u + P e_H and s = r - A x (Sec. 3 two-level steps: coarse correction,
// then the residual the post-smoother acts on).  On levels with one warp per
// slice and many rows, x is written first by a streaming kernel and the
// residual then gathers x: the fused form gathers u_j + e_H[agg_j] per entry,
// a chain of three dependent loads, and ran at 0.56 of the copy bandwidth at
// 2.1M rows against 0.77 for the plain residual.  Small levels keep the fused
// kernel, where the extra launch would cost more than it saves.  Both forms
// compute each x_i and each row's sum in the same operations and order.
constexpr int kProlongSplitRows = 1 << 17;
// matrix bytes (stored values + columns) from which a level streams its matrix
constexpr double kStreamMatrixBytes = 64.0 * (1 << 20);

template <typename T>
static amg_status prolong_residual(amg_handle_s *h, int k, const T *eH, const T *u, const T *r, T *x, T *s) {
  amg::Level &L = h->lv[k];
  if (h->prolong_split && L.wps == 1 && L.n >= kProlongSplitRows) {
    const bool timed = h->timing.enabled && k == 0;
    cudaEvent_t e0, e1;
    if (timed) AMG_TRY(timing_record(h, &e0, 2));
    AMG_TRY(plaunch(h, h->stream, k_prolong_set<T>, dim3(nblk((L.n + 3) / 4)), dim3(kThreads), L.n, L.agg, eH, u, x));
    SLAUNCH(h);
    if (timed) AMG_TRY(timing_record(h, &e1, 2));
    return residual<T>(h, k, x, r, s);
  }
  AMG_TRY(with_wps(L.wps, [&](auto W) {
    return plaunch(h, h->stream, k_prolong_residual<T, decltype(W)::value>, dim3(sell_grid(L.n, L.wps)),
                   dim3(kThreads), view<T>(L), L.agg, eH, u, r, x, s);
  }));
  SLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status coarse_solve(amg_handle_s *h, const T *b, T *x);

template <>
amg_status coarse_solve<double>(amg_handle_s *h, const double *b, double *x) {
  AMG_TRY(plaunch(h, h->stream, k_dense_mv, dim3(nblk((int64_t)h->nc * 32)), dim3(kThreads), h->nc, h->Z, b, x));
  SLAUNCH(h);
  return AMG_OK;
}

template <>
amg_status coarse_solve<float>(amg_handle_s *h, const float *b, float *x) {
  AMG_TRY(plaunch(h, h->stream, k_convert<float, double>, dim3(nblk(h->nc)), dim3(kThreads), h->nc, b, h->cb64));
  SLAUNCH(h);
  AMG_TRY(coarse_solve<double>(h, h->cb64, h->cx64));
  AMG_TRY(plaunch(h, h->stream, k_convert<double, float>, dim3(nblk(h->nc)), dim3(kThreads), h->nc, h->cx64, x));
  SLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status kcycle(amg_handle_s *h, int k, const T *r, T *x);

// nu steps of flexible CG on level k (1 <= k < L-1) from x = 0:
// b = level k's input (r_H of level k-1), result in level k's x.  Step it:
//   D = K_k(rin);  W = A D with the dots D_l.W (l < it) -> beta_l;
//   D -= sum beta_l D_l, W -= sum beta_l W_l with rho = D.W, sigma = D.rin
//   -> alpha (for it = 0 both dots come with the SpMV);  x, r update.
template <typename T>
static amg_status inner_fcg(amg_handle_s *h, int k) {
  amg::Level &L = h->lv[k];
  const int nu = h->opt.inner_iters;
  const int64_t n = L.n;
  cudaStream_t st = h->stream;
  T *b = (T *)L.b, *x = (T *)L.x, *r = (T *)L.r;
  // the stop flag L.scal[24] was cleared by the restriction that produced b
  for (int it = 0; it < nu; ++it) {
    const T *rin = (it == 0) ? b : r;
    T *D = (T *)L.D[it], *W = (T *)L.W[it];
    AMG_TRY(kcycle<T>(h, k, rin, D));
    if (it == 0) {
      DotSpec<T> sp{};
      sp.a[0] = D;
      sp.b[0] = nullptr;  // D . (A D)
      sp.a[1] = rin;
      sp.b[1] = D;
      sp.nd = 2;
      AMG_TRY(spmv_dots<T>(h, k, D, W, sp, Fin{FIN_IALPHA, 0, 0.0, L.scal}));
    } else {
      DotSpec<T> sp{};
      for (int l = 0; l < it; ++l) {
        sp.a[l] = (const T *)L.D[l];
        sp.b[l] = nullptr;  // D_l . (A D)
      }
      sp.nd = it;
      AMG_TRY(spmv_dots<T>(h, k, D, W, sp, Fin{FIN_IBETA, 0, 0.0, L.scal}));
      DotSpec<T> prev{};
      for (int l = 0; l < it; ++l) {
        prev.a[l] = (const T *)L.D[l];
        prev.b[l] = (const T *)L.W[l];
      }
      prev.nd = it;
      AMG_TRY(plaunch(h, st, k_orth_dots<T>, dim3(red_grid(h, n)), dim3(kThreads), n, D, W, prev, L.scal + 16, rin, h->red.partial,
                                                        h->red.ticket, Fin{FIN_IALPHA, it, 0.0, L.scal}));
      SLAUNCH(h);
    }
    AMG_TRY(plaunch(h, st, k_inner_update<T>, dim3(nblk(n)), dim3(kThreads), n, it, it + 1 < nu, L.scal, D, W, rin, x, r));
    SLAUNCH(h);
  }
  return AMG_OK;
}

// x = K_k(r): W(1,1) nonlinear AMLI cycle (Sec. 3 two-level steps, Sec. 4):
//   u = q_m(A) r;  s = r - A u;  r_H = P^T s;  e_H = coarse solve or nu inner
//   flexible-CG steps;  x = u + P e_H with s = r - A x in the same pass;
//   x += q_m(A) s.
template <typename T>
static amg_status dense_two_level(amg_handle_s *h, const T *r, T *x);

template <>
amg_status dense_two_level<double>(amg_handle_s *h, const double *r, double *x) {
  const int n = h->lv[h->Bk].n;
  AMG_TRY(plaunch(h, h->stream, k_dense_mv, dim3(nblk((int64_t)n * 32)), dim3(kThreads), n, h->Bd, r, x));
  SLAUNCH(h);
  return AMG_OK;
}

template <>
amg_status dense_two_level<float>(amg_handle_s *h, const float *r, float *x) {
  const int n = h->lv[h->Bk].n;
  AMG_TRY(plaunch(h, h->stream, k_convert<float, double>, dim3(nblk(n)), dim3(kThreads), n, r, h->bb64));
  SLAUNCH(h);
  AMG_TRY(dense_two_level<double>(h, h->bb64, h->bx64));
  AMG_TRY(plaunch(h, h->stream, k_convert<double, float>, dim3(nblk(n)), dim3(kThreads), n, h->bx64, x));
  SLAUNCH(h);
  return AMG_OK;
}

template <typename T>
static amg_status kcycle(amg_handle_s *h, int k, const T *r, T *x) {
  if (k == h->L - 1) return coarse_solve<T>(h, r, x);
  if (k == h->Bk) return dense_two_level<T>(h, r, x);
  amg::Level &L = h->lv[k];
  amg::Level &N = h->lv[k + 1];
  cudaStream_t st = h->stream;
  T *s = (T *)L.s, *u = (T *)L.u;
  AMG_TRY(smooth<T>(h, k, r, u, false));
  AMG_TRY(residual<T>(h, k, u, r, s));
  {
    const bool timed = h->timing.enabled && k == 0;
    cudaEvent_t e0, e1;
    if (timed) AMG_TRY(timing_record(h, &e0, 1));
    AMG_TRY(restrict_to<T>(h, k, s, (T *)N.b, N.scal + 24));
    if (timed) AMG_TRY(timing_record(h, &e1, 1));
  }
  if (k + 1 == h->L - 1) AMG_TRY(coarse_solve<T>(h, (const T *)N.b, (T *)N.x));
  else if (k + 1 == h->leaf_k) AMG_TRY(launch_leaf(h));
  else AMG_TRY(inner_fcg<T>(h, k + 1));
  AMG_TRY(prolong_residual<T>(h, k, (const T *)N.x, u, r, x, s));
  AMG_TRY(smooth<T>(h, k, s, x, true));
  return AMG_OK;
}

// x = B_k r: the stationary AMLI W-cycle (Sec. 4).  The two-level steps of
// the K-cycle, with the coarse problem solved by the fixed polynomial
// e_H = q(B_{k+1} A_{k+1}) B_{k+1} r_H (amli_coarse) instead of inner flexible CG.
template <typename T>
static amg_status amli_coarse(amg_handle_s *h, int j);

template <typename T>
static amg_status amli_cycle(amg_handle_s *h, int k, const T *r, T *x) {
  if (k == h->L - 1) return coarse_solve<T>(h, r, x);
  if (k == h->Bk) return dense_two_level<T>(h, r, x);  // exact coarse solve below: linear, = B
  amg::Level &L = h->lv[k];
  amg::Level &N = h->lv[k + 1];
  cudaStream_t st = h->stream;
  T *s = (T *)L.s, *u = (T *)L.u;
  AMG_TRY(smooth<T>(h, k, r, u, false));
  AMG_TRY(residual<T>(h, k, u, r, s));
  AMG_TRY(restrict_to<T>(h, k, s, (T *)N.b, (double *)nullptr));
  if (k + 1 == h->L - 1) AMG_TRY(coarse_solve<T>(h, (const T *)N.b, (T *)N.x));
  else AMG_TRY(amli_coarse<T>(h, k + 1));
  AMG_TRY(prolong_residual<T>(h, k, (const T *)N.x, u, r, x, s));
  AMG_TRY(smooth<T>(h, k, s, x, true));
  return AMG_OK;
}

// level j's x = q(B_j A_j) B_j b with the Chebyshev recurrence in
// tau(BA) = (2 BA - (1 + alpha) I)/(1 - alpha): T_0 = B b, T_1 = tau T_0,
// T_{p+1} = 2 tau T_p - T_{p-1}; T_p rotates through D[p mod 3], W[0] holds
// A T, W[1] holds B A T
template <typename T>
static amg_status amli_coarse(amg_handle_s *h, int j) {
  amg::Level &L = h->lv[j];
  const int64_t n = L.n;
  const int deg = h->opt.inner_iters - 1;
  cudaStream_t st = h->stream;
  T *e = (T *)L.x, *v = (T *)L.W[0], *w = (T *)L.W[1];
  auto Tb = [&](int p) { return (T *)L.D[p % 3]; };
  AMG_TRY(amli_cycle<T>(h, j, (const T *)L.b, Tb(0)));
  AMG_TRY(plaunch(h, st, k_amli_first<T>, dim3(nblk(n)), dim3(kThreads), n, Tb(0), e, (T)h->amli_coef[0]));
  SLAUNCH(h);
  for (int p = 1; p <= deg; ++p) {
    AMG_TRY(with_wps(L.wps, [&](auto W) {
      return plaunch(h, st, k_spmv<T, decltype(W)::value>, dim3(sell_grid(L.n, L.wps)), dim3(kThreads), view<T>(L),
                     Tb(p - 1), v);
    }));
    SLAUNCH(h);
    AMG_TRY(amli_cycle<T>(h, j, v, w));
    T *Tp = p >= 2 ? Tb(p - 2) : Tb(p - 1);  // unused when p == 1
    AMG_TRY(plaunch(h, st, k_amli_step<T>, dim3(nblk(n)), dim3(kThreads), n, w, Tb(p - 1), Tp, Tb(p), e,
                    (T)h->amli_sA, (T)h->amli_sB, (T)h->amli_coef[p], p == 1 ? 1 : 0));
    SLAUNCH(h);
  }
  return AMG_OK;
}

// the handle's cycle at level k
template <typename T>
static amg_status cycle(amg_handle_s *h, int k, const T *r, T *x) {
  if (h->opt.cycle == AMG_CYCLE_AMLI) return amli_cycle<T>(h, k, r, x);
  return kcycle<T>(h, k, r, x);
}

// ---------------------------------------------------------------------------
// the level above the coarsest as one dense operator
//
// With the exact coarse solve, the W(1,1) cycle at level L-2 is linear: it is
// the symmetrised two-level preconditioner of Sec. 3,
//   B = Rbar + (I - RA) P A_H^+ P^T (I - AR),  Rbar = 2R - RAR,  R = q_m(A).
// It is visited 2^(L-2) times per outer iteration, each visit a chain of
// 2m+3 tiny dependent kernels; applying B instead is a single dense matvec.
// B is built once by running that cycle, step for step, on the identity
// block (block kernels above, fp64).
// ---------------------------------------------------------------------------
constexpr int kDenseTwoLevelMax = 1024;

static amg_status bsmooth(amg_handle_s *h, int k, int ncol, const double *R, double *X, bool add,
                          double *Ta, double *Tb) {
  amg::Level &L = h->lv[k];
  const int m = h->opt.degree;
  const SellView<double> A = view<double>(L);
  const double sa = 2.0 / (L.lam1 - L.lam0), ca = (L.lam1 + L.lam0) / (L.lam1 - L.lam0);
  const int64_t nk = (int64_t)L.n * ncol;
  cudaStream_t st = h->stream;
  if (m == 0) {
    if (add) AMG_TRY(plaunch(h, st, k_bscale<double, true>, dim3(nblk(nk)), dim3(kThreads), nk, R, X, L.coef[0]));
    else AMG_TRY(plaunch(h, st, k_bscale<double, false>, dim3(nblk(nk)), dim3(kThreads), nk, R, X, L.coef[0]));
    SLAUNCH(h);
    return AMG_OK;
  }
  if (add) AMG_TRY(plaunch(h, st, k_bcheb_first<double, true>, dim3(nblk(nk)), dim3(kThreads), A, ncol, R, Ta, X, sa, ca, L.coef[0], L.coef[1]));
  else AMG_TRY(plaunch(h, st, k_bcheb_first<double, false>, dim3(nblk(nk)), dim3(kThreads), A, ncol, R, Ta, X, sa, ca, L.coef[0], L.coef[1]));
  SLAUNCH(h);
  const double *Tp = R;
  double *Tc = Ta;
  for (int j = 2; j <= m; ++j) {
    double *Tn = (j == 2) ? Tb : const_cast<double *>(Tp);
    AMG_TRY(plaunch(h, st, k_bcheb_step<double>, dim3(nblk(nk)), dim3(kThreads), A, ncol, Tc, Tp, Tn, X, sa, ca, L.coef[j]));
    SLAUNCH(h);
    Tp = Tc;
    Tc = Tn;
  }
  return AMG_OK;
}

amg_status build_dense_two_level(amg_handle_s *h) {
  h->Bk = -1;
  if (h->L < 2) return AMG_OK;
  const int k = h->L - 2;
  amg::Level &L = h->lv[k];
  const int n = L.n, nc = h->nc;
  if (n > kDenseTwoLevelMax) return AMG_OK;
  cudaStream_t st = h->stream;
  const int64_t nn = (int64_t)n * n, cn = (int64_t)nc * n;
  double *I = nullptr, *U = nullptr, *S = nullptr, *Ta = nullptr, *Tb = nullptr, *RH = nullptr, *EH = nullptr;
  AMG_TRY(pool_alloc((void **)&I, sizeof(double) * nn, st));
  AMG_TRY(pool_alloc((void **)&U, sizeof(double) * nn, st));
  AMG_TRY(pool_alloc((void **)&S, sizeof(double) * nn, st));
  AMG_TRY(pool_alloc((void **)&Ta, sizeof(double) * nn, st));
  AMG_TRY(pool_alloc((void **)&Tb, sizeof(double) * nn, st));
  AMG_TRY(pool_alloc((void **)&RH, sizeof(double) * cn, st));
  AMG_TRY(pool_alloc((void **)&EH, sizeof(double) * cn, st));
  AMG_TRY(h->arena.get(&h->Bd, (size_t)nn));
  AMG_TRY(plaunch(h, st, k_identity, dim3(nblk(nn)), dim3(kThreads), n, I));
  SLAUNCH(h);
  const SellView<double> A = view<double>(L);
  AMG_TRY(bsmooth(h, k, n, I, U, false, Ta, Tb));                       // U = R I
  AMG_TRY(plaunch(h, st, k_bresidual<double>, dim3(nblk(nn)), dim3(kThreads), A, n, U, I, S));   // S = I - A U
  SLAUNCH(h);
  AMG_TRY(plaunch(h, st, k_brestrict<double>, dim3(nblk(cn)), dim3(kThreads), nc, n, L.agg_ptr, L.agg_mem, S, RH,
                  (double *)nullptr));
  SLAUNCH(h);
  AMG_TRY(plaunch(h, st, k_bdense<double>, dim3(nblk(cn)), dim3(kThreads), nc, n, h->Z, RH, EH));         // A_H^+ P^T S
  SLAUNCH(h);
  AMG_TRY(plaunch(h, st, k_bprolong_residual<double>, dim3(nblk(nn)), dim3(kThreads), A, n, L.agg, EH, U, I, h->Bd, S));
  SLAUNCH(h);
  AMG_TRY(bsmooth(h, k, n, S, h->Bd, true, Ta, Tb));                    // B = U + P.. + R S
  for (double *p : {I, U, S, Ta, Tb, RH, EH}) pool_free(p, st);
  h->Bk = k;
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// buffers
// ---------------------------------------------------------------------------
amg_status allocate_solve_buffers(amg_handle_s *h) {
  const bool f32 = h->opt.precision == AMG_PREC_FP32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const int L = h->L, nu = h->opt.inner_iters;
  // AMG_GB300_SPLIT=0 keeps one thread per row on every level
  const char *split_env = getenv("AMG_GB300_SPLIT");
  const bool split = !(split_env && split_env[0] == '0');
  int per_sm = f32 ? 32 : 16;
  if (const char *e = getenv("AMG_GB300_WPS_WARPS")) per_sm = std::max(1, std::min(2048, atoi(e)));
  // AMG_GB300_STREAM=0 reads every level's matrix with the default cache
  // policy (A/B timing of the streaming loads)
  const char *stream_env = getenv("AMG_GB300_STREAM");
  const bool stream_ok = !(stream_env && stream_env[0] == '0');
  // AMG_GB300_WPS=w0,w1,...: warps per slice of levels 0, 1, ... (1, 2, 4 or
  // 8; A/B timing), the rule above for levels not listed
  std::vector<int> wps_force;
  if (const char *e = getenv("AMG_GB300_WPS")) {
    for (const char *c = e; *c;) {
      const int v = atoi(c);
      wps_force.push_back((v == 1 || v == 2 || v == 4 || v == 8) ? v : 0);
      while (*c && *c != ',') ++c;
      if (*c == ',') ++c;
    }
  }
  for (int k = 0; k < L; ++k) {
    amg::Level &V = h->lv[k];
    const size_t n = (size_t)std::max(V.n, 1);
    V.wps = split ? choose_wps(V.n, per_sm) : 1;
    if (k < (int)wps_force.size() && wps_force[k] > 0) V.wps = wps_force[k];
    // one pass over the level's stored values and columns is at least the
    // size of L2: stream it (the vectors and the coarser levels stay cached)
    V.stream = stream_ok && (double)V.S.stored * (double)(es + 4) >= kStreamMatrixBytes;
    AMG_TRY(h->arena.alloc((void **)&V.scal, sizeof(double) * 64));
    if (k < L - 1 && h->opt.degree > 0) {
      // the smoother form 2 t(A) of this level (Chebyshev kernels)
      amg::Sell &S = V.S;
      const double two_sa = 4.0 / (V.lam1 - V.lam0), two_ca = 2.0 * (V.lam1 + V.lam0) / (V.lam1 - V.lam0);
      const int64_t stored = std::max<int64_t>(S.stored, 1), cnt = std::max<int64_t>(S.stored, V.n);
      if (f32) {
        AMG_TRY(h->arena.alloc((void **)&S.sval32, sizeof(float) * stored));
        AMG_TRY(h->arena.alloc((void **)&S.sdiag32, sizeof(float) * n));
        k_smoother_form<float><<<nblk(cnt), kThreads, 0, h->stream>>>(S.stored, V.n, S.val64, V.diag, two_sa, two_ca,
                                                                        S.sval32, S.sdiag32);
      } else {
        AMG_TRY(h->arena.alloc((void **)&S.sval64, sizeof(double) * stored));
        AMG_TRY(h->arena.alloc((void **)&S.sdiag64, sizeof(double) * n));
        k_smoother_form<double><<<nblk(cnt), kThreads, 0, h->stream>>>(S.stored, V.n, S.val64, V.diag, two_sa, two_ca,
                                                                         S.sval64, S.sdiag64);
      }
      SLAUNCH(h);
    }
    if (k < L - 1) {
      AMG_TRY(h->arena.alloc(&V.u, es * n));
      AMG_TRY(h->arena.alloc(&V.s, es * n));
      AMG_TRY(h->arena.alloc(&V.Ta, es * n));
      AMG_TRY(h->arena.alloc(&V.Tb, es * n));
    }
    if (k >= 1) {
      AMG_TRY(h->arena.alloc(&V.b, es * n));
      AMG_TRY(h->arena.alloc(&V.x, es * n));
    }
    if (k >= 1 && k < L - 1) {
      AMG_TRY(h->arena.alloc(&V.r, es * n));
      for (int i = 0; i < nu; ++i) {
        AMG_TRY(h->arena.alloc(&V.D[i], es * n));
        AMG_TRY(h->arena.alloc(&V.W[i], es * n));
      }
    }
  }
  const size_t n0 = (size_t)h->n;
  AMG_TRY(h->arena.get(&h->ob, n0));
  AMG_TRY(h->arena.get(&h->ox, n0));
  AMG_TRY(h->arena.get(&h->or_, n0));
  AMG_TRY(h->arena.get(&h->oz, n0));
  for (int j = 0; j < h->opt.restart; ++j) {
    AMG_TRY(h->arena.get(&h->oD[j], n0));
    AMG_TRY(h->arena.get(&h->oQ[j], n0));
  }
  AMG_TRY(h->arena.get(&h->oscal, 256));
  AMG_TRY(h->arena.get(&h->red.partial, (size_t)kRedBlocks * kMaxDots));
  AMG_TRY(h->arena.get(&h->red.ticket, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(h->red.ticket, 0, sizeof(unsigned), h->stream));
  if (f32 && h->L >= 2) {
    const size_t nb = (size_t)std::max(h->lv[h->L - 2].n, 1);
    AMG_TRY(h->arena.get(&h->bb64, nb));
    AMG_TRY(h->arena.get(&h->bx64, nb));
  }
  if (f32) {
    AMG_TRY(h->arena.get(&h->r32, n0));
    AMG_TRY(h->arena.get(&h->z32, n0));
    AMG_TRY(h->arena.get(&h->cb64, (size_t)h->nc));
    AMG_TRY(h->arena.get(&h->cx64, (size_t)h->nc));
  }
  if (!h->h_pinned) AMG_CUDA_TRY(cudaMallocHost((void **)&h->h_pinned, sizeof(double) * 64));
  return AMG_OK;
}

// z = K_0(r) in the handle's cycle precision (fp64 in, fp64 out)
static amg_status precondition(amg_handle_s *h, const double *r, double *z) {
  if (h->opt.precision == AMG_PREC_FP32) {
    const int64_t n = h->n;
    AMG_TRY(plaunch(h, h->stream, k_convert<double, float>, dim3(nblk(n)), dim3(kThreads), n, r, h->r32));
    SLAUNCH(h);
    AMG_TRY(cycle<float>(h, 0, h->r32, h->z32));
    AMG_TRY(plaunch(h, h->stream, k_convert<float, double>, dim3(nblk(n)), dim3(kThreads), n, h->z32, z));
    SLAUNCH(h);
    return AMG_OK;
  }
  return cycle<double>(h, 0, r, z);
}

// Capture z = K_0(r) on the fixed buffers (or_, oz) as a CUDA graph.  All
// Krylov scalars live on the device, so the launch sequence of one
// application is static and the graph stays valid for the handle's lifetime.
static amg_status ensure_graph(amg_handle_s *h) {
  if (!h->use_graph) return AMG_OK;
  const bool timed = h->timing.enabled;
  if (h->pre_exec && h->graph_timed == timed) return AMG_OK;
  if (h->pre_exec) {
    cudaGraphExecDestroy(h->pre_exec);
    h->pre_exec = nullptr;
  }
  if (!h->cap) AMG_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  const cudaStream_t saved = h->stream;
  const int64_t saved_launches = h->launches;
  h->timing.used = 0;
  AMG_CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  h->stream = h->cap;
  h->capturing = true;
  const amg_status s = precondition(h, h->or_, h->oz);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  h->stream = saved;
  h->capturing = false;
  h->graph_kernels = h->launches - saved_launches;
  h->launches = saved_launches;
  if (s != AMG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&h->pre_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    h->pre_exec = nullptr;
    return fail(AMG_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e2));
  }
  h->graph_timed = timed;
  h->graph_events = h->timing.used;
  h->timing.used = 0;
  return AMG_OK;
}

static amg_status run_precondition(amg_handle_s *h) {
  if (h->pre_exec) {
    AMG_CUDA_TRY(cudaGraphLaunch(h->pre_exec, h->stream));
    h->launches += h->graph_kernels;
    return AMG_OK;
  }
  return precondition(h, h->or_, h->oz);
}

// ---------------------------------------------------------------------------
// outer flexible CG (Sec. 4: NPCG on the finest level, window cleared every
// `restart` iterations), fp64
// ---------------------------------------------------------------------------
amg_status solve_one(amg_handle_s *h, const double *b_dev, double *x_dev, double tol, amg_info *info,
                     int *iters_out, double *rel_out, double *true_rel_out, int *conv_out) {
  cudaStream_t st = h->stream;
  const int64_t n = h->n;
  const int R = h->opt.restart;
  amg::Level &L0 = h->lv[0];
  const SellView<double> A0 = view<double>(L0);
  double *sc = h->oscal;
  double *hp = h->h_pinned;
  // b (projected to zero mean for a pure Laplacian)
  if (h->pure) {
    DotSpec<double> sp{};
    sp.a[0] = b_dev;
    sp.b[0] = nullptr;
    sp.nd = 1;
    AMG_TRY(dots<double>(h, n, sp, Fin{FIN_MEAN, 35, (double)n, sc}));
    AMG_TRY(plaunch(h, st, k_shift, dim3(nblk(n)), dim3(kThreads), n, b_dev, h->ob, sc + 35));
    SLAUNCH(h);
  } else {
    AMG_CUDA_TRY(cudaMemcpyAsync(h->ob, b_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  }
  {
    DotSpec<double> sp{};
    sp.a[0] = h->ob;
    sp.b[0] = h->ob;
    sp.nd = 1;
    AMG_TRY(dots<double>(h, n, sp, Fin{FIN_STORE, 36, 0.0, sc}));
  }
  AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + 36, sizeof(double), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(h->or_, h->ob, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  AMG_CUDA_TRY(cudaMemsetAsync(sc + 34, 0, sizeof(double), st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  // a NaN or infinity anywhere in b (or entries so large that ||b||^2
  // overflows) makes b^T b non-finite: refuse rather than iterate on garbage
  if (!std::isfinite(hp[0]))
    return fail(AMG_ERR_INVALID_ARG, "right-hand side has a non-finite entry or a norm beyond the fp64 range");
  const double nb = sqrt(hp[0]);
  int hl = 0;
  if (info && info->history && info->history_cap > 0) info->history[hl++] = nb > 0 ? 1.0 : 0.0;
  int it = 0, converged = (nb == 0.0), nwin = 0;
  double res = nb > 0 ? 1.0 : 0.0;
  amg_status status = AMG_OK;
  AMG_TRY(ensure_graph(h));
  if (h->timing.enabled) h->timing.used = 0;
  while (!converged && it < h->opt.max_iters) {
    const NvtxRange iter_range("outer flexible-CG iteration");
    if (it % R == 0) nwin = 0;
    double *d = h->oD[nwin], *q = h->oQ[nwin];
    AMG_TRY(run_precondition(h));
    if (nwin > 0) {
      DotSpec<double> sp{};
      for (int j = 0; j < nwin; ++j) {
        sp.a[j] = h->oQ[j];
        sp.b[j] = h->oz;
      }
      sp.nd = nwin;
      AMG_TRY(dots<double>(h, n, sp, Fin{FIN_OBETA, 0, 0.0, sc}));
    }
    {
      DotSpec<double> vd{};
      for (int j = 0; j < nwin; ++j) vd.a[j] = h->oD[j];
      vd.nd = nwin;
      AMG_TRY(plaunch(h, st, k_axpy_multi<double>, dim3(nblk(n)), dim3(kThreads), n, d, h->oz, vd, sc + 16));
      SLAUNCH(h);
    }
    // q = A d (the one-row-per-thread SpMV), then rho = d.q and sigma = d.r:
    // fused into one kernel the SpMV would run as a 608-block grid-stride
    // loop, measured slower than the two
    AMG_TRY(with_wps(L0.wps, [&](auto W) {
      return plaunch(h, st, k_spmv<double, decltype(W)::value>, dim3(sell_grid(n, L0.wps)), dim3(kThreads), A0, d, q);
    }));
    SLAUNCH(h);
    {
      DotSpec<double> sp{};
      sp.a[0] = d;
      sp.b[0] = q;
      sp.a[1] = d;
      sp.b[1] = h->or_;
      sp.nd = 2;
      AMG_TRY(dots<double>(h, n, sp, Fin{FIN_OALPHA, nwin, 0.0, sc}));
    }
    AMG_TRY(plaunch(h, st, k_outer_update, dim3(red_grid(h, n)), dim3(kThreads), n, sc, d, q, x_dev, h->or_, h->red.partial,
                                                      h->red.ticket, Fin{FIN_STORE, 33, 0.0, sc}));
    SLAUNCH(h);
    AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + 33, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (h->pre_exec && h->graph_timed) AMG_TRY(timing_accumulate(h, h->graph_events));
    if (hp[1] != 0.0) {
      status = fail(AMG_ERR_BREAKDOWN, "flexible CG breakdown: d^T A d <= 0 or non-finite");
      break;
    }
    ++nwin;
    ++it;
    res = sqrt(hp[0]) / nb;
    if (info && info->history && hl < info->history_cap) info->history[hl++] = res;
    if (res <= tol) converged = 1;
  }
  if (h->timing.enabled) AMG_TRY(timing_flush(h));
  if (h->pure) {
    DotSpec<double> sp{};
    sp.a[0] = x_dev;
    sp.b[0] = nullptr;
    sp.nd = 1;
    AMG_TRY(dots<double>(h, n, sp, Fin{FIN_MEAN, 37, (double)n, sc}));
    AMG_TRY(plaunch(h, st, k_shift, dim3(nblk(n)), dim3(kThreads), n, x_dev, x_dev, sc + 37));
    SLAUNCH(h);
  }
  // true residual ||b - A x|| / ||b||
  double true_rel = 0.0;
  if (nb > 0.0) {
    AMG_TRY(with_wps(L0.wps, [&](auto W) {
      return plaunch(h, st, k_residual<double, decltype(W)::value>, dim3(sell_grid(n, L0.wps)), dim3(kThreads), A0, x_dev,
                     h->ob, h->oz);
    }));
    SLAUNCH(h);
    DotSpec<double> sp{};
    sp.a[0] = h->oz;
    sp.b[0] = h->oz;
    sp.nd = 1;
    AMG_TRY(dots<double>(h, n, sp, Fin{FIN_STORE, 38, 0.0, sc}));
    AMG_CUDA_TRY(cudaMemcpyAsync(hp, sc + 38, sizeof(double), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    true_rel = sqrt(hp[0]) / nb;
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) info->history_len = hl;
  *iters_out = it;
  *rel_out = res;
  *true_rel_out = true_rel;
  *conv_out = converged;
  if (status == AMG_OK && !converged) status = AMG_ERR_NOT_CONVERGED;
  return status;
}

// ---------------------------------------------------------------------------
// single-step entry points (fp64 vectors in and out)
// ---------------------------------------------------------------------------
template <typename F>
static amg_status with_precision(amg_handle_s *h, int k, F &&f64_fn) {
  (void)k;
  return f64_fn();
}

static bool f32(amg_handle_s *h) { return h->opt.precision == AMG_PREC_FP32; }

// run `body(T*)` on fp32 copies of (in -> out) when the cycle is fp32
template <typename Body>
static amg_status run_conv(amg_handle_s *h, const double *in, int64_t nin, double *out, int64_t nout,
                           bool out_accumulates, Body body) {
  if (!f32(h)) return body((const void *)in, (void *)out);
  float *a = nullptr, *b = nullptr;
  AMG_TRY(pool_alloc((void **)&a, sizeof(float) * (size_t)std::max<int64_t>(nin, 1), h->stream));
  AMG_TRY(pool_alloc((void **)&b, sizeof(float) * (size_t)std::max<int64_t>(nout, 1), h->stream));
  AMG_TRY(plaunch(h, h->stream, k_convert<double, float>, dim3(nblk(nin)), dim3(kThreads), nin, in, a));
  SLAUNCH(h);
  if (out_accumulates) {
    AMG_TRY(plaunch(h, h->stream, k_convert<double, float>, dim3(nblk(nout)), dim3(kThreads), nout, out, b));
    SLAUNCH(h);
  }
  AMG_TRY(body((const void *)a, (void *)b));
  AMG_TRY(plaunch(h, h->stream, k_convert<float, double>, dim3(nblk(nout)), dim3(kThreads), nout, b, out));
  SLAUNCH(h);
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  pool_free(a, h->stream);
  pool_free(b, h->stream);
  return AMG_OK;
}

amg_status apply_spmv(amg_handle_s *h, int k, const double *x, double *y) {
  amg::Level &L = h->lv[k];
  AMG_TRY(run_conv(h, x, L.n, y, L.n, false, [&](const void *a, void *b) -> amg_status {
    AMG_TRY(with_wps(L.wps, [&](auto W) {
      constexpr int wp = decltype(W)::value;
      const dim3 g(sell_grid(L.n, L.wps));
      if (f32(h)) return plaunch(h, h->stream, k_spmv<float, wp>, g, dim3(kThreads), view<float>(L), (const float *)a, (float *)b);
      return plaunch(h, h->stream, k_spmv<double, wp>, g, dim3(kThreads), view<double>(L), (const double *)a, (double *)b);
    }));
    SLAUNCH(h);
    return AMG_OK;
  }));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status apply_smoother(amg_handle_s *h, int k, const double *r, double *x) {
  amg::Level &L = h->lv[k];
  AMG_TRY(run_conv(h, r, L.n, x, L.n, false, [&](const void *a, void *b) -> amg_status {
    if (f32(h)) return smooth<float>(h, k, (const float *)a, (float *)b, false);
    return smooth<double>(h, k, (const double *)a, (double *)b, false);
  }));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status apply_restrict(amg_handle_s *h, int k, const double *s, double *rH) {
  amg::Level &L = h->lv[k];
  AMG_TRY(run_conv(h, s, L.n, rH, L.nH, false, [&](const void *a, void *b) -> amg_status {
    if (f32(h)) return restrict_to<float>(h, k, (const float *)a, (float *)b, nullptr);
    return restrict_to<double>(h, k, (const double *)a, (double *)b, nullptr);
  }));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status apply_prolong_add(amg_handle_s *h, int k, const double *eH, double *x) {
  amg::Level &L = h->lv[k];
  AMG_TRY(run_conv(h, eH, L.nH, x, L.n, true, [&](const void *a, void *b) -> amg_status {
    if (f32(h)) AMG_TRY(plaunch(h, h->stream, k_prolong_add<float>, dim3(nblk(L.n)), dim3(kThreads), L.n, L.agg, (const float *)a, (float *)b));
    else AMG_TRY(plaunch(h, h->stream, k_prolong_add<double>, dim3(nblk(L.n)), dim3(kThreads), L.n, L.agg, (const double *)a, (double *)b));
    SLAUNCH(h);
    return AMG_OK;
  }));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status apply_coarse_solve(amg_handle_s *h, const double *b, double *x) {
  AMG_TRY(coarse_solve<double>(h, b, x));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status apply_kcycle(amg_handle_s *h, int k, const double *r, double *z) {
  amg::Level &L = h->lv[k];
  // level k >= 1 reads its input from the level's b buffer when it recurses,
  // so use dedicated copies
  AMG_TRY(run_conv(h, r, L.n, z, L.n, false, [&](const void *a, void *b) -> amg_status {
    if (f32(h)) return cycle<float>(h, k, (const float *)a, (float *)b);
    return cycle<double>(h, k, (const double *)a, (double *)b);
  }));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

}  // namespace amg
