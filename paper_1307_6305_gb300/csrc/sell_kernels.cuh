// sell_kernels.cuh -- the SELL-32 operator kernels of the solve phase: one
// SpMV fused with a step of the Chebyshev recurrence of the polynomial
// smoother q_m(A) (Sec. 3), the residual and the plain SpMV, each in a
// one-thread-per-row form and a split form for small levels (several warps
// per 32-row slice).  Included by solve.cu only.
#pragma once

#include "common.cuh"
#include "block_kernels.cuh"

namespace amg {

// ---------------------------------------------------------------------------
// SELL-32 row kernel: off-diagonal part of row `row` times x
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T sell_row(const SellView<T> &A, const T *__restrict__ x, int row, T acc) {
  const int s = row >> 5, lane = row & 31;
  const int64_t base = A.sptr[s];
  const int w = (int)((A.sptr[s + 1] - base) >> 5);
  const T *__restrict__ v = A.val + base + lane;
  // both choices are uniform over the launch
  if (A.sdel) {  // columns as 16-bit offsets from the row
    const int16_t *__restrict__ d = A.sdel + base + lane;
    if (A.stream) {
#pragma unroll 4
      for (int k = 0; k < w; ++k) acc = fma(__ldcs(v + k * kSlice), x[row + __ldcs(d + k * kSlice)], acc);
    } else {
#pragma unroll 4
      for (int k = 0; k < w; ++k) acc = fma(v[k * kSlice], x[row + d[k * kSlice]], acc);
    }
    return acc;
  }
  const int32_t *__restrict__ c = A.scol + base + lane;
  if (A.stream) {
#pragma unroll 4
    for (int k = 0; k < w; ++k) acc = fma(__ldcs(v + k * kSlice), x[__ldcs(c + k * kSlice)], acc);
  } else {
#pragma unroll 4
    for (int k = 0; k < w; ++k) acc = fma(v[k * kSlice], x[c[k * kSlice]], acc);
  }
  return acc;
}

// column of stored position pos of row `row` (either layout)
template <typename T>
__device__ __forceinline__ int sell_col(const SellView<T> &A, int64_t pos, int row) {
  return A.sdel ? row + (int)A.sdel[pos] : A.scol[pos];
}

template <typename T>
__device__ __forceinline__ T apply_row(const SellView<T> &A, const T *__restrict__ x, int row) {
  return sell_row(A, x, row, A.diag[row] * x[row]);
}

// Split rows for small levels.  With one thread per row, a row of w stored
// entries costs about w/4 dependent round trips to L2 (column index, then
// x[col]), and a level of a few thousand rows keeps only a few SMs busy on
// the slow FP64 pipe.  With WPS > 1 the stored positions of a 32-row slice
// are dealt round-robin to WPS warps (warp q takes positions q, q + WPS, ...,
// still coalesced across the slice's rows); the partial sums meet in shared
// memory and the group's first warp adds them in warp order, so the result is
// deterministic.  A block of kThreads threads holds kThreads / 32 / WPS
// slices; `group` numbers those blocks of slices.
struct SplitIdx {
  int q, s, lane, i;
};

template <int WPS>
__device__ __forceinline__ SplitIdx split_index(int group) {
  const int warp = threadIdx.x >> 5;
  SplitIdx ix;
  ix.q = warp % WPS;
  ix.lane = threadIdx.x & 31;
  ix.s = group * (kThreads / 32 / WPS) + warp / WPS;
  ix.i = ix.s * kSlice + ix.lane;
  return ix;
}

// warp q's share of row ix.i's sum, accumulated onto acc; xf(j) gives x_j
template <typename T, int WPS, typename XF>
__device__ __forceinline__ T split_partial(const SellView<T> &A, const SplitIdx &ix, T acc, XF xf) {
  if (ix.i < A.n) {
    const int64_t base = A.sptr[ix.s];
    const int w = (int)((A.sptr[ix.s + 1] - base) >> 5);
    const T *__restrict__ v = A.val + base + ix.lane;
    if (A.sdel) {
      const int16_t *__restrict__ d = A.sdel + base + ix.lane;
#pragma unroll 2
      for (int k = ix.q; k < w; k += WPS) acc = fma(v[k * kSlice], xf(ix.i + d[k * kSlice]), acc);
    } else {
      const int32_t *__restrict__ c = A.scol + base + ix.lane;
#pragma unroll 2
      for (int k = ix.q; k < w; k += WPS) acc = fma(v[k * kSlice], xf(c[k * kSlice]), acc);
    }
  }
  return acc;
}

// meet in shared memory; true in the group's first warp, which then holds
// the row's full sum in acc.  Block-uniform: every thread must call it.
template <typename T, int WPS>
__device__ __forceinline__ bool split_combine(T &acc, T (*part)[32]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  part[warp][lane] = acc;
  __syncthreads();
  const bool lead = (warp % WPS) == 0;
  if (lead) {
#pragma unroll
    for (int p = 1; p < WPS; ++p) acc += part[warp + p][lane];
  }
  return lead;
}

// row sum (diag_i x_i + sum_j a_ij x_j) of the split layout; valid in lead
// threads whose row exists (returned flag)
template <typename T, int WPS, typename XF>
__device__ __forceinline__ bool split_row(const SellView<T> &A, const SplitIdx &ix, T xi, XF xf, T &out,
                                          T (*part)[32]) {
  T acc = (ix.q == 0 && ix.i < A.n) ? A.diag[ix.i] * xi : T(0);
  acc = split_partial<T, WPS>(A, ix, acc, xf);
  const bool lead = split_combine<T, WPS>(acc, part);
  out = acc;
  return lead && ix.i < A.n;
}

// The Chebyshev kernels take the smoother form S = 2 t(A) = 2 sa A - 2 ca I
// (stored once per level), so that a recurrence step is one SpMV and one
// subtraction: T_{j+1} = S T_j - T_{j-1}, and T_1 = S r / 2 (exact halving).

// T_1 = t(A) r; x (=|+=) b0*r + b1*T_1
template <typename T, bool ADD, int WPS>
__global__ void __launch_bounds__(kThreads) k_cheb_first(SellView<T> S, const T *__restrict__ r,
                                                         T *__restrict__ T1, T *__restrict__ x, T b0, T b1) {
  pdl_sync();
  int i;
  T Sr, ri, xo = T(0);
  if constexpr (WPS == 1) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    Sr = apply_row(S, r, i);
    ri = r[i];
    if (ADD) xo = x[i];
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    i = ix.i;
    // the row's own entries, read before the row sum (they do not depend on it)
    ri = i < S.n ? r[i] : T(0);
    if (ADD && ix.q == 0 && i < S.n) xo = x[i];
    if (!split_row<T, WPS>(S, ix, ri, [&](int j) { return r[j]; }, Sr, part)) return;
  }
  const T t1 = T(0.5) * Sr;
  T1[i] = t1;
  const T inc = fma(b1, t1, b0 * ri);
  x[i] = ADD ? xo + inc : inc;
}

// T_{j+1} = S T_j - T_{j-1}; x += bj * T_{j+1}.  Tn may alias Tp.
template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_cheb_step(SellView<T> S, const T *__restrict__ Tc,
                                                        const T *Tp, T *Tn, T *__restrict__ x, T bj) {
  pdl_sync();
  int i;
  T St, tp = T(0), xo = T(0);
  if constexpr (WPS == 1) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    St = apply_row(S, Tc, i);
    tp = Tp[i];
    xo = x[i];
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    i = ix.i;
    // the row's own entries, read before the row sum (they do not depend on
    // it); Tp[i] is read before Tn[i], which may alias it, is written
    if (ix.q == 0 && i < S.n) {
      tp = Tp[i];
      xo = x[i];
    }
    const T xi = i < S.n ? Tc[i] : T(0);
    if (!split_row<T, WPS>(S, ix, xi, [&](int j) { return Tc[j]; }, St, part)) return;
  }
  const T tn = St - tp;
  Tn[i] = tn;
  x[i] = fma(bj, tn, xo);
}

// smoother form of one level: sval = 2 sa val, sdiag = 2 sa diag - 2 ca
template <typename T>
__global__ void k_smoother_form(int64_t stored, int n, const double *__restrict__ val,
                                const double *__restrict__ diag, double two_sa, double two_ca,
                                T *__restrict__ sval, T *__restrict__ sdiag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < stored) sval[e] = (T)(two_sa * val[e]);
  if (e < n) sdiag[e] = (T)(two_sa * diag[e] - two_ca);
}

template <typename T, bool ADD>
__global__ void k_scale(int n, const T *__restrict__ r, T *__restrict__ x, T b0) {
  pdl_sync();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = ADD ? x[i] + b0 * r[i] : b0 * r[i];
}

template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_residual(SellView<T> A, const T *__restrict__ x,
                                                       const T *__restrict__ r, T *__restrict__ s) {
  pdl_sync();
  if constexpr (WPS == 1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    s[i] = r[i] - apply_row(A, x, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const T xi = ix.i < A.n ? x[ix.i] : T(0);
    const T ri = (ix.q == 0 && ix.i < A.n) ? r[ix.i] : T(0);  // before the row sum
    T Ax;
    if (split_row<T, WPS>(A, ix, xi, [&](int j) { return x[j]; }, Ax, part)) s[ix.i] = ri - Ax;
  }
}

template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_spmv(SellView<T> A, const T *__restrict__ x,
                                                   T *__restrict__ y) {
  pdl_sync();
  if constexpr (WPS == 1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    y[i] = apply_row(A, x, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const T xi = ix.i < A.n ? x[ix.i] : T(0);
    T Ax;
    if (split_row<T, WPS>(A, ix, xi, [&](int j) { return x[j]; }, Ax, part)) y[ix.i] = Ax;
  }
}

}  // namespace amg
