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
// SELL-32 row kernel: off-diagonal part of row `row` times x, in two parts:
// row_prefetch reads the row's slice metadata, its diagonal and its first
// kPre stored entries (matrix data only, so it may run before pdl_wait);
// row_finish gathers x and accumulates in stored order (the same order and
// operations as a single loop).
// ---------------------------------------------------------------------------
constexpr int kPre = 4;  // stored entries per thread fetched before pdl_wait

template <typename T>
struct RowPre {
  int w = 0;                     // stored positions of the row (slice width)
  const int32_t *c = nullptr;    // the row's first column index (stride kSlice)
  const T *v = nullptr;
  T d = T(0);                    // diagonal
  int pc[kPre] = {};
  T pv[kPre] = {};
};

template <typename T>
__device__ __forceinline__ int ldc(const SellView<T> &A, const int32_t *p) {
  return A.stream ? __ldcs(p) : *p;
}
template <typename T>
__device__ __forceinline__ T ldv(const SellView<T> &A, const T *p) {
  return A.stream ? __ldcs(p) : *p;
}

template <typename T>
__device__ __forceinline__ RowPre<T> row_prefetch(const SellView<T> &A, int row) {
  RowPre<T> p;
  const int s = row >> 5, lane = row & 31;
  const int64_t base = A.sptr[s];
  p.w = (int)((A.sptr[s + 1] - base) >> 5);
  p.c = A.scol + base + lane;
  p.v = A.val + base + lane;
  p.d = A.diag[row];
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    if (k < p.w) {
      p.pc[k] = ldc(A, p.c + k * kSlice);
      p.pv[k] = ldv(A, p.v + k * kSlice);
    }
  }
  return p;
}

template <typename T>
__device__ __forceinline__ T row_finish(const SellView<T> &A, const RowPre<T> &p, const T *__restrict__ x, T acc) {
#pragma unroll
  for (int k = 0; k < kPre; ++k)
    if (k < p.w) acc = fma(p.pv[k], x[p.pc[k]], acc);
  if (A.stream) {  // uniform over the launch
#pragma unroll 4
    for (int k = kPre; k < p.w; ++k) acc = fma(__ldcs(p.v + k * kSlice), x[__ldcs(p.c + k * kSlice)], acc);
  } else {
#pragma unroll 4
    for (int k = kPre; k < p.w; ++k) acc = fma(p.v[k * kSlice], x[p.c[k * kSlice]], acc);
  }
  return acc;
}

// diag_i x_i + sum_j a_ij x_j
template <typename T>
__device__ __forceinline__ T row_apply(const SellView<T> &A, const RowPre<T> &p, const T *__restrict__ x, int row) {
  return row_finish(A, p, x, p.d * x[row]);
}

template <typename T>
__device__ __forceinline__ T sell_row(const SellView<T> &A, const T *__restrict__ x, int row, T acc) {
  return row_finish(A, row_prefetch(A, row), x, acc);
}

template <typename T>
__device__ __forceinline__ T apply_row(const SellView<T> &A, const T *__restrict__ x, int row) {
  const RowPre<T> p = row_prefetch(A, row);
  return row_finish(A, p, x, p.d * x[row]);
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

// warp q's first kPre positions (q, q + WPS, ...) and the diagonal
template <typename T, int WPS>
__device__ __forceinline__ RowPre<T> split_prefetch(const SellView<T> &A, const SplitIdx &ix) {
  RowPre<T> p;
  if (ix.i < A.n) {
    const int64_t base = A.sptr[ix.s];
    p.w = (int)((A.sptr[ix.s + 1] - base) >> 5);
    p.c = A.scol + base + ix.lane;
    p.v = A.val + base + ix.lane;
    if (ix.q == 0) p.d = A.diag[ix.i];
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int pos = ix.q + k * WPS;
      if (pos < p.w) {
        p.pc[k] = ldc(A, p.c + pos * kSlice);
        p.pv[k] = ldv(A, p.v + pos * kSlice);
      }
    }
  }
  return p;
}

// warp q's share of row ix.i's sum, accumulated onto acc; xf(j) gives x_j
template <typename T, int WPS, typename XF>
__device__ __forceinline__ T split_partial(const SellView<T> &A, const SplitIdx &ix, const RowPre<T> &p, T acc,
                                           XF xf) {
  if (ix.i < A.n) {
#pragma unroll
    for (int k = 0; k < kPre; ++k)
      if (ix.q + k * WPS < p.w) acc = fma(p.pv[k], xf(p.pc[k]), acc);
#pragma unroll 2
    for (int pos = ix.q + kPre * WPS; pos < p.w; pos += WPS)
      acc = fma(ldv(A, p.v + pos * kSlice), xf(ldc(A, p.c + pos * kSlice)), acc);
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
__device__ __forceinline__ bool split_row(const SellView<T> &A, const SplitIdx &ix, const RowPre<T> &p, T xi,
                                          XF xf, T &out, T (*part)[32]) {
  T acc = (ix.q == 0 && ix.i < A.n) ? p.d * xi : T(0);
  acc = split_partial<T, WPS>(A, ix, p, acc, xf);
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
  pdl_trigger();
  int i;
  T Sr;
  if constexpr (WPS == 1) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const RowPre<T> p = row_prefetch(S, i);
    pdl_wait();
    Sr = row_apply(S, p, r, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const RowPre<T> p = split_prefetch<T, WPS>(S, ix);
    pdl_wait();
    i = ix.i;
    const T xi = i < S.n ? r[i] : T(0);
    if (!split_row<T, WPS>(S, ix, p, xi, [&](int j) { return r[j]; }, Sr, part)) return;
  }
  const T ri = r[i];
  const T t1 = T(0.5) * Sr;
  T1[i] = t1;
  const T inc = fma(b1, t1, b0 * ri);
  x[i] = ADD ? x[i] + inc : inc;
}

// T_{j+1} = S T_j - T_{j-1}; x += bj * T_{j+1}.  Tn may alias Tp.
template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_cheb_step(SellView<T> S, const T *__restrict__ Tc,
                                                        const T *Tp, T *Tn, T *__restrict__ x, T bj) {
  pdl_trigger();
  int i;
  T St;
  if constexpr (WPS == 1) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const RowPre<T> p = row_prefetch(S, i);
    pdl_wait();
    St = row_apply(S, p, Tc, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const RowPre<T> p = split_prefetch<T, WPS>(S, ix);
    pdl_wait();
    i = ix.i;
    const T xi = i < S.n ? Tc[i] : T(0);
    if (!split_row<T, WPS>(S, ix, p, xi, [&](int j) { return Tc[j]; }, St, part)) return;
  }
  const T tn = St - Tp[i];
  Tn[i] = tn;
  x[i] = fma(bj, tn, x[i]);
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
  pdl_trigger();
  if constexpr (WPS == 1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const RowPre<T> p = row_prefetch(A, i);
    pdl_wait();
    s[i] = r[i] - row_apply(A, p, x, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const RowPre<T> p = split_prefetch<T, WPS>(A, ix);
    pdl_wait();
    const T xi = ix.i < A.n ? x[ix.i] : T(0);
    T Ax;
    if (split_row<T, WPS>(A, ix, p, xi, [&](int j) { return x[j]; }, Ax, part)) s[ix.i] = r[ix.i] - Ax;
  }
}

template <typename T, int WPS>
__global__ void __launch_bounds__(kThreads) k_spmv(SellView<T> A, const T *__restrict__ x,
                                                   T *__restrict__ y) {
  pdl_trigger();
  if constexpr (WPS == 1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const RowPre<T> p = row_prefetch(A, i);
    pdl_wait();
    y[i] = row_apply(A, p, x, i);
  } else {
    __shared__ T part[kThreads / 32][32];
    const SplitIdx ix = split_index<WPS>(blockIdx.x);
    const RowPre<T> p = split_prefetch<T, WPS>(A, ix);
    pdl_wait();
    const T xi = ix.i < A.n ? x[ix.i] : T(0);
    T Ax;
    if (split_row<T, WPS>(A, ix, p, xi, [&](int j) { return x[j]; }, Ax, part)) y[ix.i] = Ax;
  }
}

}  // namespace amg
