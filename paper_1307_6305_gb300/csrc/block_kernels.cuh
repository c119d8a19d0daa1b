// block_kernels.cuh -- device helpers shared by the single-vector and the
// multi-vector (batched right-hand sides) solve paths.
#pragma once

#include <utility>

#include "common.cuh"

namespace amg {

constexpr int kThreads = 256;
static inline unsigned nblk(int64_t n, int t = kThreads) {
  return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1);
}

// Programmatic dependent launch: wait until the preceding kernel has
// completed and its writes are visible, then let the next kernel in the
// stream be scheduled while this one runs (no-op for ordinary launches)
__device__ __forceinline__ void pdl_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch with programmatic stream serialization (PDL); arguments are
// converted to the kernel's parameter types before their addresses are taken
template <typename... KArgs>
static inline amg_status plaunch_impl(amg_handle_s *h, cudaStream_t st, void (*kern)(KArgs...), dim3 g, dim3 b,
                               KArgs... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = h->use_pdl ? 1 : 0;
  void *p[] = {(void *)&args...};
  const cudaError_t e = cudaLaunchKernelExC(&cfg, (const void *)kern, p);
  if (e != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return AMG_OK;
}

template <typename... KArgs, typename... Args>
static inline amg_status plaunch(amg_handle_s *h, cudaStream_t st, void (*kern)(KArgs...), dim3 g, dim3 b,
                          Args &&...args) {
  return plaunch_impl<KArgs...>(h, st, kern, g, b, KArgs(std::forward<Args>(args))...);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// block (multi-vector) kernels: a block X of k vectors is stored row major,
// X[i * k + c] = component i of vector c, so one thread per (row, column)
// reads each stored matrix entry once per row (broadcast) and the gathered
// neighbour values of consecutive columns are contiguous
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T sell_row_block(const SellView<T> &A, const T *__restrict__ X, int k, int row,
                                            int c, T acc) {
  const int s = row >> 5, lane = row & 31;
  const int64_t base = A.sptr[s];
  const int w = (int)((A.sptr[s + 1] - base) >> 5);
  const int32_t *__restrict__ cc = A.scol + base + lane;
  const T *__restrict__ v = A.val + base + lane;
  for (int q = 0; q < w; ++q) acc = fma(v[q * kSlice], X[(int64_t)cc[q * kSlice] * k + c], acc);
  return acc;
}

template <typename T, bool ADD>
__global__ void k_bcheb_first(SellView<T> A, int k, const T *__restrict__ R, T *__restrict__ T1,
                              T *__restrict__ X, T sa, T ca, T b0, T b1) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.n * k) return;
  const int i = (int)(idx / k), c = (int)(idx % k);
  const T ri = R[idx];
  const T Ar = sell_row_block(A, R, k, i, c, A.diag[i] * ri);
  const T t1 = fma(sa, Ar, -ca * ri);
  T1[idx] = t1;
  const T inc = fma(b1, t1, b0 * ri);
  X[idx] = ADD ? X[idx] + inc : inc;
}

template <typename T>
__global__ void k_bcheb_step(SellView<T> A, int k, const T *__restrict__ Tc, const T *Tp, T *Tn,
                             T *__restrict__ X, T sa, T ca, T bj) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.n * k) return;
  const int i = (int)(idx / k), c = (int)(idx % k);
  const T tc = Tc[idx];
  const T At = sell_row_block(A, Tc, k, i, c, A.diag[i] * tc);
  const T tn = T(2) * fma(sa, At, -ca * tc) - Tp[idx];
  Tn[idx] = tn;
  X[idx] = fma(bj, tn, X[idx]);
}

template <typename T, bool ADD>
__global__ void k_bscale(int64_t nk, const T *__restrict__ R, T *__restrict__ X, T b0) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nk) return;
  X[idx] = ADD ? X[idx] + b0 * R[idx] : b0 * R[idx];
}

template <typename T>
__global__ void k_bresidual(SellView<T> A, int k, const T *__restrict__ X, const T *__restrict__ R,
                            T *__restrict__ S) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.n * k) return;
  const int i = (int)(idx / k), c = (int)(idx % k);
  S[idx] = R[idx] - sell_row_block(A, X, k, i, c, A.diag[i] * X[idx]);
}

// RH = P^T S per column; `flags` (k entries), when given, are the next
// level's per-column inner-CG stop flags, cleared here because the inner
// solve on RH starts right after
template <typename T>
__global__ void k_brestrict(int nH, int k, const int *__restrict__ ptr, const int *__restrict__ mem,
                            const T *__restrict__ S, T *__restrict__ RH, double *flags) {
  pdl_sync();
  if (flags && blockIdx.x == 0 && threadIdx.x < k) flags[threadIdx.x] = 0.0;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nH * k) return;
  const int I = (int)(idx / k), c = (int)(idx % k);
  T acc = T(0);
  for (int a = ptr[I]; a < ptr[I + 1]; ++a) acc += S[(int64_t)mem[a] * k + c];
  RH[idx] = acc;
}

template <typename T>
__global__ void k_bprolong_residual(SellView<T> A, int k, const int *__restrict__ agg,
                                    const T *__restrict__ EH, const T *__restrict__ U,
                                    const T *__restrict__ R, T *__restrict__ X, T *__restrict__ S) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)A.n * k) return;
  const int i = (int)(idx / k), c = (int)(idx % k);
  const T xi = U[idx] + EH[(int64_t)agg[i] * k + c];
  X[idx] = xi;
  const int s = i >> 5, lane = i & 31;
  const int64_t base = A.sptr[s];
  const int w = (int)((A.sptr[s + 1] - base) >> 5);
  T acc = A.diag[i] * xi;
  for (int q = 0; q < w; ++q) {
    const int j = A.scol[base + q * kSlice + lane];
    acc = fma(A.val[base + q * kSlice + lane], U[(int64_t)j * k + c] + EH[(int64_t)agg[j] * k + c], acc);
  }
  S[idx] = R[idx] - acc;
}

// X = Z B for a dense fp64 row-major n x n matrix Z and an n x k block B
// (accumulated in fp64 whatever the block's element type)
template <typename T>
__global__ void k_bdense(int n, int k, const double *__restrict__ Z, const T *__restrict__ B,
                         T *__restrict__ X) {
  pdl_sync();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * k) return;
  const int i = (int)(idx / k), c = (int)(idx % k);
  double acc = 0.0;
  for (int j = 0; j < n; ++j) acc = fma(Z[(int64_t)i * n + j], (double)B[(int64_t)j * k + c], acc);
  X[idx] = (T)acc;
}

}  // namespace amg
