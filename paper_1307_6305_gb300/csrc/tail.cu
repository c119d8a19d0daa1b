// tail.cu -- the coarse end of the K-cycle as one persistent cluster kernel.
//
// From the first level small enough (level k0 >= 1) down to the coarsest,
// a K-cycle visit is a chain of a few dozen dependent phases over a few
// thousand rows; the W-cycle (nu = 2) visits level k 2^k times per outer
// iteration, so issued as separate kernels these levels cost hundreds of
// launch latencies per iteration.  Here the complete inner flexible-CG
// solve at level k0 (nu steps, each with its recursive K-cycle below,
// Sec. 4: NPCG applied recursively on coarse levels) runs inside ONE kernel
// launch on one thread-block cluster:
//   * phases (one Chebyshev/SpMV sweep, a restriction, an update, ...) are
//     separated by the hardware cluster barrier;
//   * dot products are reduced through distributed shared memory: every CTA
//     posts its partial into CTA 0's shared memory, and after one barrier
//     every CTA folds them in rank order, so all CTAs hold bit-identical
//     Krylov scalars without any global-memory scalar traffic;
//   * vectors written inside the kernel are read with L1-bypassing loads
//     (the CTAs of the cluster sit on different SMs);
//   * the level recursion is unrolled at compile time (no device stack).
// The arithmetic is that of the multi-kernel path in solve.cu, phase for
// phase (only the summation order of dot products differs).
#include <cooperative_groups.h>
#include <math.h>

#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace amg {

constexpr int kTailThreads = 512;
constexpr int kTailMaxCTAs = 16;
constexpr int kTailMaxDepth = 8;  // levels handled inside the kernel

template <typename T>
struct TailLevel {
  SellView<T> A;
  int n, nH;
  const int *agg, *agg_ptr, *agg_mem;
  double sa, ca;
  double coef[kMaxDegree + 1];
  T *u, *s, *Ta, *Tb;
  T *b, *x, *r;
  T *D[kMaxInner], *W[kMaxInner];
};

template <typename T>
struct TailParams {
  int k0, L, Bk, nB, nc, m, nu;
  const double *Bd, *Z;
  TailLevel<T> lv[kTailMaxDepth];  // lv[k - k0]
};

enum TailMode : int { kModeCTA = 0, kModeCluster = 1, kModeGrid = 2 };

struct TailCtx {
  cg::cluster_group cl;
  int mode;       // kModeCTA: one CTA; kModeCluster: one cluster; kModeGrid:
                  // cooperative grid, one CTA per SM, software barrier
  int rank, csize, tid, nthr;
  double *slots;  // shared [2][kTailMaxCTAs][kMaxDots]
  double *wred;   // shared [kTailThreads/32][kMaxDots]
  double *bcast;  // shared [kMaxDots]
  int phase;
  // grid mode
  unsigned *bar;        // [0] arrivals, [1] generation
  double *gpart;        // [2][gridDim][kMaxDots] partial sums
  int *err;             // set when a barrier wait runs out
  long long wait_ns;    // how long a barrier wait may last before it gives up
  int test_stall;       // test hook: wait for a generation that never comes
  bool failed;
};

// loads of vectors written inside the kernel: CTAs on different SMs do not
// share (coherent) L1 caches, so cluster and grid modes read L2 directly;
// in single-CTA mode every reader shares one L1, coherent across
// __syncthreads, and may use it
template <typename T>
__device__ __forceinline__ T ld(const TailCtx &c, const T *p) {
  return c.mode != kModeCTA ? __ldcg(p) : __ldca(p);
}

// after a failed barrier every row loop is empty and every later barrier a
// no-op, so all threads run to the end of the kernel without touching memory
__device__ __forceinline__ void tail_fail(TailCtx &c) {
  c.failed = true;
  c.tid = 0x3fffffff;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// grid-wide barrier with a bounded wait (sense by generation counter)
__device__ __noinline__ void gbar(TailCtx &c) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = c.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned target = g + 1u + (c.test_stall ? 1u : 0u);
    if (atomicAdd(c.bar, 1u) == gridDim.x - 1u) {
      atomicExch(c.bar, 0u);
      __threadfence();
      atomicAdd(c.bar + 1, 1u);
    }
    // spin without sleeping (a wake-up adds latency to every phase); every
    // 256 polls look at the clock and at the error flag another CTA may set
    int ok = 1;
    unsigned it = 0;
    const unsigned long long t0 = global_ns();
    while ((int)(*gen - target) < 0) {
      if ((++it & 255u) == 0 && (global_ns() - t0 > (unsigned long long)c.wait_ns || *(volatile int *)c.err)) {
        atomicExch(c.err, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  if (!ok_s) tail_fail(c);
}

__device__ __forceinline__ void csync(TailCtx &c) {
  if (c.failed) return;
  if (c.mode == kModeCluster) c.cl.sync();
  else if (c.mode == kModeGrid) gbar(c);
  else __syncthreads();
}

// cluster-wide sum of ND per-thread values; result identical in every CTA
template <int ND>
__device__ __noinline__ void csum(TailCtx &c, double (&v)[ND]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) c.wred[warp * kMaxDots + q] = t;
  }
  __syncthreads();
  if (c.failed) {
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] = 0.0;
    return;
  }
  if (c.mode == kModeGrid) {
    double *part = c.gpart + (size_t)c.phase * gridDim.x * kMaxDots;
    if (threadIdx.x < ND) {
      double t = 0.0;
      for (int w = 0; w < kTailThreads / 32; ++w) t += c.wred[w * kMaxDots + threadIdx.x];
      part[blockIdx.x * kMaxDots + threadIdx.x] = t;
    }
    csync(c);
    if (threadIdx.x < ND) {
      double t = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&part[b * kMaxDots + threadIdx.x]);
      c.bcast[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] = c.failed ? 0.0 : c.bcast[q];
    __syncthreads();
    c.phase ^= 1;
    return;
  }
  if (c.mode == kModeCTA) {
    if (threadIdx.x < ND) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += c.wred[w * kMaxDots + threadIdx.x];
      c.bcast[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ND; ++q) v[q] = c.bcast[q];
    __syncthreads();  // bcast and wred are reused by the next reduction
    return;
  }
  double *slots = c.slots + c.phase * kTailMaxCTAs * kMaxDots;
  if (threadIdx.x < ND) {
    double t = 0.0;
    for (int w = 0; w < kTailThreads / 32; ++w) t += c.wred[w * kMaxDots + threadIdx.x];
    double *dst = c.cl.map_shared_rank(slots, 0);
    dst[c.rank * kMaxDots + threadIdx.x] = t;
  }
  csync(c);
  if (threadIdx.x < ND) {
    const double *src = c.cl.map_shared_rank(slots, 0);
    double t = 0.0;
    for (int r = 0; r < c.csize; ++r) t += src[r * kMaxDots + threadIdx.x];
    c.bcast[threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < ND; ++q) v[q] = c.bcast[q];
  c.phase ^= 1;
  // the slots of this phase are reused two reductions later; the barrier
  // inside the next reduction orders every reader before that reuse
}

// (A x)_i; the loop is unrolled so that a row's independent L2 loads are in
// flight together instead of one dependent round trip per entry
template <typename T>
__device__ __forceinline__ T row_apply(const TailCtx &c, const SellView<T> &A, const T *x, int i) {
  const int s = i >> 5, lane = i & 31;
  const int64_t base = A.sptr[s];
  const int w = (int)((A.sptr[s + 1] - base) >> 5);
  const int32_t *col = A.scol + base + lane;
  const T *v = A.val + base + lane;
  T acc = A.diag[i] * ld(c, x + i);
#pragma unroll 8
  for (int q = 0; q < w; ++q) acc = fma(v[q * kSlice], ld(c, x + col[q * kSlice]), acc);
  return acc;
}

// x = M r for a dense fp64 row-major n x n matrix, one warp per row
template <typename T>
__device__ __noinline__ void dense_dev(TailCtx &c, int n, const double *M, const T *r, T *x) {
  const int lane = threadIdx.x & 31;
  const int gw = c.tid >> 5, nw = c.nthr >> 5;
  for (int row = gw; row < n; row += nw) {
    double acc = 0.0;
#pragma unroll 8
    for (int j = lane; j < n; j += 32) acc = fma(M[(int64_t)row * n + j], (double)ld(c, r + j), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[row] = (T)acc;
  }
  csync(c);
}

// x (=|+=) q_m(A) r on level descriptor V
template <typename T>
__device__ __noinline__ void smooth_dev(TailCtx &c, const TailLevel<T> &V, int m, const T *r, T *x, bool add) {
  const T sa = (T)V.sa, ca = (T)V.ca;
  if (m == 0) {
    for (int i = c.tid; i < V.n; i += c.nthr) {
      const T inc = (T)V.coef[0] * ld(c, r + i);
      x[i] = add ? ld(c, x + i) + inc : inc;
    }
    csync(c);
    return;
  }
  {
    const T b0 = (T)V.coef[0], b1 = (T)V.coef[1];
    for (int i = c.tid; i < V.n; i += c.nthr) {
      const T ri = ld(c, r + i);
      const T t1 = fma(sa, row_apply(c, V.A, r, i), -ca * ri);
      V.Ta[i] = t1;
      const T inc = fma(b1, t1, b0 * ri);
      x[i] = add ? ld(c, x + i) + inc : inc;
    }
    csync(c);
  }
  const T *Tp = r;
  T *Tc = V.Ta;
  for (int j = 2; j <= m; ++j) {
    T *Tn = (j == 2) ? V.Tb : const_cast<T *>(Tp);
    const T bj = (T)V.coef[j];
    for (int i = c.tid; i < V.n; i += c.nthr) {
      const T tc = ld(c, Tc + i);
      const T tn = T(2) * fma(sa, row_apply(c, V.A, Tc, i), -ca * tc) - ld(c, Tp + i);
      Tn[i] = tn;
      x[i] = fma(bj, tn, ld(c, x + i));
    }
    csync(c);
    Tp = Tc;
    Tc = Tn;
  }
}

// s = r - A u, then r_H = P^T s (members in ascending order)
template <typename T>
__device__ __noinline__ void restrict_residual_dev(TailCtx &c, const TailLevel<T> &V, const T *r, T *rH) {
  for (int i = c.tid; i < V.n; i += c.nthr) V.s[i] = ld(c, r + i) - row_apply(c, V.A, V.u, i);
  csync(c);
  for (int I = c.tid; I < V.nH; I += c.nthr) {
    T acc = T(0);
    for (int a = V.agg_ptr[I]; a < V.agg_ptr[I + 1]; ++a) acc += ld(c, V.s + V.agg_mem[a]);
    rH[I] = acc;
  }
  csync(c);
}

// x = u + P e_H and s = r - A x in one sweep
template <typename T>
__device__ __noinline__ void prolong_residual_dev(TailCtx &c, const TailLevel<T> &V, const T *eH, const T *r,
                                                 T *x) {
  for (int i = c.tid; i < V.n; i += c.nthr) {
    const T xi = ld(c, V.u + i) + ld(c, eH + V.agg[i]);
    x[i] = xi;
    const int sl = i >> 5, lane = i & 31;
    const int64_t base = V.A.sptr[sl];
    const int w = (int)((V.A.sptr[sl + 1] - base) >> 5);
    T acc = V.A.diag[i] * xi;
#pragma unroll 8
    for (int q = 0; q < w; ++q) {
      const int j = V.A.scol[base + q * kSlice + lane];
      acc = fma(V.A.val[base + q * kSlice + lane], ld(c, V.u + j) + ld(c, eH + V.agg[j]), acc);
    }
    V.s[i] = ld(c, r + i) - acc;
  }
  csync(c);
}

template <typename T, int D>
__device__ void inner_dev(TailCtx &c, const TailParams<T> &P, int k);

// x = K_k(r), the W(1,1) nonlinear AMLI cycle (same steps as solve.cu)
template <typename T, int D>
__device__ void kcycle_dev(TailCtx &c, const TailParams<T> &P, int k, const T *r, T *x) {
  if (k == P.L - 1) {
    dense_dev(c, P.nc, P.Z, r, x);
    return;
  }
  if (k == P.Bk) {
    dense_dev(c, P.nB, P.Bd, r, x);
    return;
  }
  const TailLevel<T> &V = P.lv[k - P.k0];
  const TailLevel<T> &N = P.lv[k + 1 - P.k0];
  smooth_dev(c, V, P.m, r, V.u, false);
  restrict_residual_dev(c, V, r, N.b);
  if (k + 1 == P.L - 1) {
    dense_dev(c, P.nc, P.Z, N.b, N.x);
  } else {
    if constexpr (D + 1 < kTailMaxDepth) inner_dev<T, D + 1>(c, P, k + 1);
  }
  prolong_residual_dev(c, V, N.x, r, x);
  smooth_dev(c, V, P.m, V.s, x, true);
}

// one inner flexible-CG step (it) after D = K(rin): W = A D, orthogonalise
// against the earlier directions, then alpha and the x / r update
template <typename T>
__device__ __noinline__ void inner_step_dev(TailCtx &c, const TailLevel<T> &V, int it, int nu, const T *rin,
                                            double *rho, bool &stopped) {
  T *Dc = V.D[it], *Wc = V.W[it];
  double rs[2];
  if (it == 0) {
    double acc[2] = {0.0, 0.0};
    for (int i = c.tid; i < V.n; i += c.nthr) {
      const T w = row_apply(c, V.A, Dc, i);
      Wc[i] = w;
      const double d = (double)ld(c, Dc + i);
      acc[0] += d * (double)w;
      acc[1] += (double)ld(c, rin + i) * d;
    }
    csum<2>(c, acc);
    rs[0] = acc[0];
    rs[1] = acc[1];
  } else {
    double bacc[kMaxInner];
#pragma unroll
    for (int l = 0; l < kMaxInner; ++l) bacc[l] = 0.0;
    for (int i = c.tid; i < V.n; i += c.nthr) {
      const T w = row_apply(c, V.A, Dc, i);
      Wc[i] = w;
      for (int l = 0; l < it; ++l) bacc[l] += (double)ld(c, V.D[l] + i) * (double)w;
    }
    csum<kMaxInner>(c, bacc);
    double beta[kMaxInner];
    for (int l = 0; l < it; ++l) beta[l] = bacc[l] / rho[l];
    double acc[2] = {0.0, 0.0};
    for (int i = c.tid; i < V.n; i += c.nthr) {
      T d = ld(c, Dc + i), w = ld(c, Wc + i);
      for (int l = 0; l < it; ++l) {
        const T bl = (T)beta[l];
        d -= bl * ld(c, V.D[l] + i);
        w -= bl * ld(c, V.W[l] + i);
      }
      Dc[i] = d;
      Wc[i] = w;
      acc[0] += (double)d * (double)w;
      acc[1] += (double)d * (double)ld(c, rin + i);
    }
    csum<2>(c, acc);
    rs[0] = acc[0];
    rs[1] = acc[1];
  }
  rho[it] = rs[0];
  double alpha;
  if (stopped || !(rs[0] > 0.0) || !isfinite(rs[0])) {
    stopped = true;
    alpha = 0.0;
  } else {
    alpha = rs[1] / rs[0];
  }
  const bool here = stopped && alpha == 0.0;
  const bool upd_r = it + 1 < nu;
  const T a = (T)alpha;
  for (int i = c.tid; i < V.n; i += c.nthr) {
    const T di = ld(c, Dc + i);
    if (it == 0) V.x[i] = here ? T(0) : a * di;
    else if (!here) V.x[i] = fma(a, di, ld(c, V.x + i));
    if (upd_r) V.r[i] = here ? ld(c, rin + i) : ld(c, rin + i) - a * ld(c, Wc + i);
  }
  csync(c);
}

// nu steps of flexible CG at level k from x = 0 on (b -> x), as in solve.cu
template <typename T, int D>
__device__ void inner_dev(TailCtx &c, const TailParams<T> &P, int k) {
  const TailLevel<T> &V = P.lv[k - P.k0];
  double rho[kMaxInner];
  bool stopped = false;
  for (int it = 0; it < P.nu; ++it) {
    const T *rin = (it == 0) ? V.b : V.r;
    kcycle_dev<T, D>(c, P, k, rin, V.D[it]);
    inner_step_dev<T>(c, V, it, P.nu, rin, rho, stopped);
  }
}

struct TailSync {
  unsigned *bar;
  double *gpart;
  int *err;
  long long wait_ns;
  int test_stall;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailParams<T> *__restrict__ Pg, TailSync sy) {
  __shared__ double slots[2 * kTailMaxCTAs * kMaxDots];
  __shared__ double wred[(kTailThreads / 32) * kMaxDots];
  __shared__ double bcast[kMaxDots];
  __shared__ TailParams<T> P;
  asm volatile("griddepcontrol.wait;" ::: "memory");  // predecessor launched with PDL
  // stage the descriptor block in shared memory
  {
    const int words = (int)(sizeof(TailParams<T>) / sizeof(int));
    const int *src = reinterpret_cast<const int *>(Pg);
    int *dst = reinterpret_cast<int *>(&P);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  TailCtx c{cg::this_cluster(), MODE, 0, 1, 0, 0, slots, wred, bcast, 0,
            sy.bar, sy.gpart, sy.err, sy.wait_ns, sy.test_stall, false};
  if (MODE == kModeCluster) {
    c.rank = (int)c.cl.block_rank();
    c.csize = (int)c.cl.num_blocks();
  } else if (MODE == kModeGrid) {
    c.rank = blockIdx.x;
    c.csize = gridDim.x;
  }
  c.tid = c.rank * blockDim.x + threadIdx.x;
  c.nthr = c.csize * blockDim.x;
  __syncthreads();
  csync(c);  // every CTA has started before any remote or grid-wide exchange
  inner_dev<T, 0>(c, P, P.k0);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
static void fill_params(amg_handle_s *h, TailParams<T> &P) {
  memset(&P, 0, sizeof(P));
  P.k0 = h->tail_k0;
  P.L = h->L;
  P.Bk = h->Bk;
  P.nB = h->Bk >= 0 ? h->lv[h->Bk].n : 0;
  P.nc = h->nc;
  P.m = h->opt.degree;
  P.nu = h->opt.inner_iters;
  P.Bd = h->Bd;
  P.Z = h->Z;
  for (int k = h->tail_k0; k < h->L && k - h->tail_k0 < kTailMaxDepth; ++k) {
    amg::Level &L = h->lv[k];
    TailLevel<T> &V = P.lv[k - h->tail_k0];
    if constexpr (sizeof(T) == 8) V.A = {L.n, L.S.sptr, L.S.scol, (const T *)L.S.val64, (const T *)L.S.diag64};
    else V.A = {L.n, L.S.sptr, L.S.scol, (const T *)L.S.val32, (const T *)L.S.diag32};
    V.n = L.n;
    V.nH = L.nH;
    V.agg = L.agg;
    V.agg_ptr = L.agg_ptr;
    V.agg_mem = L.agg_mem;
    if (k + 1 < h->L) {
      V.sa = 2.0 / (L.lam1 - L.lam0);
      V.ca = (L.lam1 + L.lam0) / (L.lam1 - L.lam0);
      for (int j = 0; j <= h->opt.degree; ++j) V.coef[j] = L.coef[j];
    }
    V.u = (T *)L.u;
    V.s = (T *)L.s;
    V.Ta = (T *)L.Ta;
    V.Tb = (T *)L.Tb;
    V.b = (T *)L.b;
    V.x = (T *)L.x;
    V.r = (T *)L.r;
    for (int i = 0; i < kMaxInner; ++i) {
      V.D[i] = (T *)L.D[i];
      V.W[i] = (T *)L.W[i];
    }
  }
}

template <typename T>
static amg_status prepare(amg_handle_s *h, int mode) {
  int csize = 1;
  if (mode == kModeCluster) {
    auto kern = k_tail<T, kModeCluster>;
    AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    csize = 0;
    for (int want : {16, 8, 4}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      cfg.gridDim = dim3(want);
      cfg.blockDim = dim3(kTailThreads);
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = want;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) {
        csize = want;
        break;
      }
      cudaGetLastError();
    }
    if (!csize) return fail(AMG_ERR_CUDA, "no thread-block cluster size is schedulable for the tail kernel");
  } else if (mode == kModeGrid) {
    int sms = 0, per = 0;
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tail<T, kModeGrid>, kTailThreads, 0));
    if (per < 1) return fail(AMG_ERR_CUDA, "the grid tail kernel does not fit on an SM");
    // At most one CTA per SM, so all are co-resident, as a grid barrier needs.
    // 16 CTAs measured fastest on the 128^3 hierarchy (the barrier's cost
    // grows with the CTA count faster than the tail levels' work shrinks);
    // AMG_GB300_TAIL_CTAS overrides.
    csize = std::min(sms, 16);
    if (const char *env = getenv("AMG_GB300_TAIL_CTAS")) csize = std::max(1, std::min(sms, atoi(env)));
  }
  h->tail_csize = csize;
  h->tail_mode = mode;
  TailParams<T> P;
  fill_params(h, P);
  AMG_TRY(h->arena.alloc(&h->tail_params, sizeof(P)));
  AMG_TRY(h->arena.alloc((void **)&h->tail_bar, sizeof(unsigned) * 4));
  AMG_TRY(h->arena.alloc((void **)&h->tail_err, sizeof(int) * 4));
  AMG_TRY(h->arena.alloc((void **)&h->tail_gpart, sizeof(double) * 2 * (size_t)csize * kMaxDots));
  AMG_CUDA_TRY(cudaMemsetAsync(h->tail_bar, 0, sizeof(unsigned) * 4, h->stream));
  AMG_CUDA_TRY(cudaMemsetAsync(h->tail_err, 0, sizeof(int) * 4, h->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(h->tail_params, &P, sizeof(P), cudaMemcpyHostToDevice, h->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

// Choose k0, the first level >= 1 with at most `max_rows` rows (levels down
// to the coarsest must fit the compile-time depth); -1 keeps every level on
// the multi-kernel path.  Off by default: on GB300 with the 128^3 workload
// every mode measured slower than the graph-replayed kernels (fp64 solve
// 56 ms without the tail, 88 ms with the grid mode from 8192 rows; fp32 42
// vs 77 ms) -- each in-kernel phase still costs several microseconds of
// dependent memory latency, and a single SM's 2 DFMA/clk starves the one-CTA
// and cluster modes in fp64.  AMG_GB300_TAIL_ROWS=<rows> enables it and
// AMG_GB300_TAIL_MODE selects grid (default) / cluster / cta.
amg_status prepare_tail(amg_handle_s *h) {
  h->tail_k0 = -1;
  const bool f32 = h->opt.precision == AMG_PREC_FP32;
  int max_rows = 0;
  int mode = kModeGrid;
  if (const char *env = getenv("AMG_GB300_TAIL_ROWS")) max_rows = atoi(env);
  if (const char *env = getenv("AMG_GB300_TAIL_MODE")) {
    if (!strcmp(env, "cta")) mode = kModeCTA;
    else if (!strcmp(env, "cluster")) mode = kModeCluster;
  }
  h->tail_test_stall = 0;
  if (const char *env = getenv("AMG_GB300_TAIL_TEST_STALL")) h->tail_test_stall = atoi(env);
  if (max_rows <= 0 || h->L < 3 || h->opt.cycle != AMG_CYCLE_K) return AMG_OK;
  int k0 = -1;
  for (int k = 1; k + 1 < h->L; ++k)
    if (h->lv[k].n <= max_rows) {
      k0 = k;
      break;
    }
  if (k0 < 0 || h->L - k0 > kTailMaxDepth) return AMG_OK;
  h->tail_k0 = k0;
  amg_status s = f32 ? prepare<float>(h, mode) : prepare<double>(h, mode);
  if (s != AMG_OK) h->tail_k0 = -1;
  return s;
}

template <typename T>
static amg_status launch(amg_handle_s *h) {
  TailSync sy;
  sy.bar = h->tail_bar;
  sy.gpart = h->tail_gpart;
  sy.err = h->tail_err;
  // a real barrier wait lasts microseconds: give up after 2 s (the test
  // hook, whose barrier never opens, after 5 ms)
  sy.wait_ns = h->tail_test_stall ? 5000000LL : 2000000000LL;
  sy.test_stall = h->tail_test_stall;
  const TailParams<T> *P = (const TailParams<T> *)h->tail_params;
  if (h->tail_mode == kModeCTA) {
    k_tail<T, kModeCTA><<<1, kTailThreads, 0, h->stream>>>(P, sy);
    ++h->launches;
    AMG_CUDA_TRY(cudaGetLastError());
    return AMG_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(h->tail_csize);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = h->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (h->tail_mode == kModeCluster) {
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->tail_csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tail<T, kModeCluster>, P, sy));
  } else {
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tail<T, kModeGrid>, P, sy));
  }
  ++h->launches;
  return AMG_OK;
}

amg_status launch_tail(amg_handle_s *h) {
  return h->opt.precision == AMG_PREC_FP32 ? launch<float>(h) : launch<double>(h);
}

}  // namespace amg
