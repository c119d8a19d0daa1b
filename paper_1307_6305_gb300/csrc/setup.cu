// setup.cu -- device-side setup of the aggregation hierarchy.
//
// Every step of the setup runs in the kernels below; the host only sizes
// buffers and loops over levels/passes/rounds:
//   validation and connectivity of the input graph (Eq. (1) needs a
//   connected graph for the pure Laplacian, Sec. 1);
//   assembly A_ii = sum_j w_ij + d_i, A_ij = -w_ij (Eq. (1));
//   handshake matching passes (Sec. 2: a matching is the simplest graph
//   partitioning) with the symmetric strength |a_ij|/sqrt(a_ii a_jj) as edge
//   weight and a splitmix64 hash as tie-break;
//   Galerkin A_H = P^T A P for piecewise-constant P (Sec. 3 remark, Sec. 5:
//   sums of fine entries over aggregate pairs), one pass at a time, so each
//   coarse row merges at most two fine rows;
//   lambda1 = ||A_k||_inf (Sec. 3), the Chebyshev coefficients of q_m
//   (host, closed form, a few flops), the SELL-32 solve layout and the dense
//   pseudo-inverse of the coarsest operator (Sec. 3, A_H^+).
#include <math.h>

#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace amg {

#define LAUNCH_CHECK(cnt)                                                          \
  do {                                                                             \
    if (cnt) ++*(cnt);                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)

static inline unsigned blocks_for(int64_t n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

// ---------------------------------------------------------------------------
// exclusive scan (reduce-then-scan, 2048 elements per block)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

template <typename T>
__global__ void k_scan_tile(const T *__restrict__ in, T *__restrict__ out, T *__restrict__ bsum,
                            int64_t n) {
  __shared__ T wtot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  T v[kScanPer];
  T local = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    local += v[k];
  }
  T inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wtot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T t = (lane < kScanThreads / 32) ? wtot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < kScanThreads / 32) wtot[lane] = t;
  }
  __syncthreads();
  T run = inc - local + (warp > 0 ? wtot[warp - 1] : T(0));
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = wtot[kScanThreads / 32 - 1];
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ out, const T *__restrict__ off, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += off[i / kScanTile];
}

template <typename T>
static amg_status scan_rec(const T *in, T *out, int64_t n, cudaStream_t st, T *total_dev) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb < 1) nb = 1;
  if (nb == 1) {  // one tile: its block sum is the total
    k_scan_tile<T><<<1, kScanThreads, 0, st>>>(in, out, total_dev, n);
    LAUNCH_CHECK((int64_t *)nullptr);
    return AMG_OK;
  }
  T *bsum = nullptr, *boff = nullptr;
  AMG_TRY(pool_alloc((void **)&bsum, sizeof(T) * nb, st));
  k_scan_tile<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, bsum, n);
  LAUNCH_CHECK((int64_t *)nullptr);
  AMG_TRY(pool_alloc((void **)&boff, sizeof(T) * nb, st));
  AMG_TRY(scan_rec<T>(bsum, boff, nb, st, total_dev));
  k_scan_add<T><<<blocks_for(n, 256), 256, 0, st>>>(out, boff, n);
  LAUNCH_CHECK((int64_t *)nullptr);
  pool_free(boff, st);
  pool_free(bsum, st);
  return AMG_OK;
}

// exclusive scan; the total is read back (one stream synchronisation) only
// when the caller asks for it
template <typename T>
static amg_status scan_total(const T *in, T *out, int64_t n, cudaStream_t st, int64_t *total_host) {
  T *tot = nullptr;
  AMG_TRY(pool_alloc((void **)&tot, sizeof(T), st));
  AMG_TRY(scan_rec<T>(in, out, n, st, tot));
  if (total_host) {
    T t = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&t, tot, sizeof(T), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    *total_host = (int64_t)t;
  }
  pool_free(tot, st);
  return AMG_OK;
}

amg_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st,
                              int64_t *total_host) {
  return scan_total<long long>((const long long *)in, (long long *)out, n, st, total_host);
}
amg_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st,
                              int64_t *total_host) {
  return scan_total<int>(in, out, n, st, total_host);
}

// host checks of the iterative setup loops: connectivity rounds per batch,
// matching rounds per batch (the first batch of a pass may be longer)
constexpr int kCcBatch = 3;
constexpr int kMatchBatch = 4;
constexpr int kMatchMaxBatch = 16;

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
enum : unsigned {
  F_ROWPTR = 1u, F_RANGE = 2u, F_ORDER = 4u, F_SELF = 8u, F_SYM = 16u, F_W = 32u, F_D = 64u
};

__global__ void k_check_rowptr(int64_t n, const int64_t *__restrict__ rp, unsigned *flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  bool bad = (i == 0) ? (rp[0] != 0) : (rp[i] < rp[i - 1]);
  if (bad) atomicOr(flags, F_ROWPTR);
}

__global__ void k_check_entries(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const double *__restrict__ w, const double *__restrict__ d,
                                unsigned *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned f = 0;
  const int64_t a = rp[i], b = rp[i + 1];
  for (int64_t p = a; p < b; ++p) {
    const int c = col[p];
    if (c < 0 || c >= n) f |= F_RANGE;
    else if (c == i) f |= F_SELF;
    if (p > a && c <= col[p - 1]) f |= F_ORDER;
    const double wp = w[p];
    if (!(wp > 0.0) || !isfinite(wp)) f |= F_W;
  }
  if (d) {
    const double di = d[i];
    if (!(di >= 0.0) || !isfinite(di)) f |= F_D;
  }
  if (f) atomicOr(flags, f);
}

// symmetric pattern and values: (i, j, w) needs (j, i, w) with w equal bit for bit
__global__ void k_check_symmetry(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const double *__restrict__ w, unsigned *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool bad = false;
  for (int64_t p = rp[i]; p < rp[i + 1] && !bad; ++p) {
    const int j = col[p];
    if (j < 0 || j >= n) continue;  // reported by k_check_entries (launched with this one)
    int64_t lo = rp[j], hi = rp[j + 1] - 1, hit = -1;
    while (lo <= hi) {
      int64_t mid = lo + (hi - lo) / 2;
      int c = col[mid];
      if (c == i) { hit = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (hit < 0 || w[hit] != w[p]) bad = true;
  }
  if (bad) atomicOr(flags, F_SYM);
}

// ---------------------------------------------------------------------------
// connectivity: root hooking with atomicMin + pointer jumping
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cc_root(const int *parent, int v) {
  int p = parent[v];
  while (p != v) {
    v = p;
    p = parent[v];
  }
  return v;
}

__global__ void k_cc_init(int n, int *parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = i;
}

__global__ void k_cc_hook(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          int *parent, int *changed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    int j = col[p];
    if (j <= i) continue;
    int ri = cc_root(parent, i), rj = cc_root(parent, j);
    if (ri != rj) {
      atomicMin(&parent[max(ri, rj)], min(ri, rj));
      *changed = 1;
    }
  }
}

__global__ void k_cc_jump(int n, int *parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = cc_root(parent, i);
}

// components: count roots; with lower-order terms every component needs d > 0
__global__ void k_cc_mark(int n, const int *parent, const double *d, int *posd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && d && d[i] > 0.0) posd[parent[i]] = 1;
}
__global__ void k_cc_count(int n, const int *parent, const int *posd, int pure, int *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || parent[i] != i) return;
  atomicAdd(&out[0], 1);
  if (!pure && !posd[i]) atomicAdd(&out[1], 1);
}

// ---------------------------------------------------------------------------
// assembly, Eq. (1): a_ij = -w_ij, A_ii = sum_j w_ij + d_i (row order)
// ---------------------------------------------------------------------------
__global__ void k_assemble(int n, const int64_t *__restrict__ rp, const double *__restrict__ w,
                           const double *__restrict__ d, double *__restrict__ val,
                           double *__restrict__ diag, double *__restrict__ dlow) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    val[p] = -w[p];
    s += w[p];
  }
  const double di = d ? d[i] : 0.0;
  dlow[i] = di;
  diag[i] = s + di;
}

// ---------------------------------------------------------------------------
// handshake matching
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t edge_hash(uint64_t salt, int a, int b) {
  const uint64_t lo = (uint64_t)min(a, b), hi = (uint64_t)max(a, b);
  return splitmix64(salt ^ ((lo << 32) | hi));
}

// matching weight of each stored edge: |a_ij| / sqrt(a_ii a_jj)
__global__ void k_strength(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ diag,
                           double *__restrict__ s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = diag[i];
  // chunks of entries whose loads are issued together
  constexpr int kChunk = 8;
  const int64_t end = rp[i + 1];
  for (int64_t p0 = rp[i]; p0 < end; p0 += kChunk) {
    int jj[kChunk];
    double vv[kChunk], dd[kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      const bool in = p0 + k < end;
      jj[k] = in ? col[p0 + k] : -1;
      vv[k] = in ? val[p0 + k] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kChunk; ++k) dd[k] = jj[k] >= 0 ? diag[jj[k]] : 1.0;
#pragma unroll
    for (int k = 0; k < kChunk; ++k)
      if (p0 + k < end) s[p0 + k] = -vv[k] / sqrt(di * dd[k]);
  }
}

__global__ void k_match_init(int n, int *mate) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) mate[i] = -1;
}

// each unmatched vertex points across its largest-key edge to an unmatched
// neighbour; key = (s_ij, hash, lo, hi) compared lexicographically.  `prev`
// (optional) is the previous round's count of new pairs: once a round has
// added none, the matching is maximal and later rounds do nothing.
__global__ void k_propose(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          const double *__restrict__ s, uint64_t salt, const int *__restrict__ mate,
                          int *__restrict__ ptr, const int *prev) {
  if (prev && *prev == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int best = -1;
  if (mate[i] < 0) {
    double bw = 0.0;
    uint64_t bh = 0;
    bool bh_ok = false;
    // entries are taken in stored order, in chunks whose loads (columns and
    // strengths, then the neighbours' mates) are issued together
    constexpr int kChunk = 8;
    const int64_t end = rp[i + 1];
    for (int64_t p0 = rp[i]; p0 < end; p0 += kChunk) {
      int jj[kChunk], mm[kChunk];
      double ww[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const bool in = p0 + k < end;
        jj[k] = in ? col[p0 + k] : -1;
        ww[k] = in ? s[p0 + k] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kChunk; ++k) mm[k] = jj[k] >= 0 ? mate[jj[k]] : 0;
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        const int j = jj[k];
        if (j < 0 || mm[k] >= 0) continue;
        const double wj = ww[k];
        if (best < 0) { best = j; bw = wj; bh_ok = false; continue; }
        bool take;
        if (wj != bw) {
          take = wj > bw;
        } else {
          if (!bh_ok) { bh = edge_hash(salt, i, best); bh_ok = true; }
          const uint64_t hj = edge_hash(salt, i, j);
          if (hj != bh) {
            take = hj > bh;
          } else {
            const int lj = min(i, j), hj2 = max(i, j), lb = min(i, best), hb = max(i, best);
            take = (lj != lb) ? (lj > lb) : (hj2 > hb);
          }
        }
        if (take) {
          best = j;
          bw = wj;
          bh_ok = false;
        }
      }
    }
  }
  ptr[i] = best;
}

__global__ void k_accept(int n, const int *__restrict__ ptr, int *__restrict__ mate, int *added,
                         const int *prev) {
  if (prev && *prev == 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int hit = 0;
  if (i < n) {
    const int p = ptr[i];
    if (p >= 0 && ptr[p] == i) {
      mate[i] = p;
      hit = 1;
    }
  }
  hit = __syncthreads_count(hit);
  if (threadIdx.x == 0 && hit) atomicAdd(added, hit);
}

__global__ void k_rep_flags(int n, const int *__restrict__ mate, int *__restrict__ rep) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rep[i] = (mate[i] < 0 || i < mate[i]) ? 1 : 0;
}

__global__ void k_coarse_ids(int n, const int *__restrict__ mate, const int *__restrict__ id,
                             int *__restrict__ agg, int *__restrict__ m0, int *__restrict__ m1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = mate[i];
  const bool rep = (m < 0 || i < m);
  if (rep) {
    agg[i] = id[i];
    if (m0) {
      m0[id[i]] = i;
      m1[id[i]] = m;
    }
  } else {
    agg[i] = id[m];
  }
}

// One handshake matching pass.  Rounds run in batches between host checks
// (`first_batch` rounds, then kMatchBatch): a round after one that added no
// pair is a device-side no-op (the matching is maximal), so the extra rounds
// of the last batch change nothing.  Every matched pair is counted once by
// each of its two vertices, so n_H = n - (sum of the counts) / 2 is known on
// the host without another read-back.
static amg_status match_core(cudaStream_t st, int n, const int64_t *rowptr, const int32_t *col,
                             const double *s, uint64_t salt, int32_t *mate, int32_t *agg, int *m0,
                             int *m1, int *nH_out, int *rounds_out, int64_t *launches, int first_batch) {
  int *ptr = nullptr, *added = nullptr, *rep = nullptr, *id = nullptr;
  const int maxb = std::max(kMatchBatch, std::min(first_batch, kMatchMaxBatch));
  AMG_TRY(pool_alloc((void **)&ptr, sizeof(int) * (size_t)std::max(n, 1), st));
  AMG_TRY(pool_alloc((void **)&added, sizeof(int) * (size_t)maxb, st));
  const unsigned nb = blocks_for(n, 256);
  k_match_init<<<nb, 256, 0, st>>>(n, mate);
  LAUNCH_CHECK(launches);
  int rounds = 0;
  int64_t matched = 0;  // vertices matched so far (two per pair)
  int h_added[kMatchMaxBatch];
  for (int batch = maxb;; batch = kMatchBatch) {
    AMG_CUDA_TRY(cudaMemsetAsync(added, 0, sizeof(int) * batch, st));
    for (int b = 0; b < batch; ++b) {
      const int *prev = b ? added + b - 1 : nullptr;
      k_propose<<<nb, 256, 0, st>>>(n, rowptr, col, s, salt, mate, ptr, prev);
      LAUNCH_CHECK(launches);
      k_accept<<<nb, 256, 0, st>>>(n, ptr, mate, added + b, prev);
      LAUNCH_CHECK(launches);
    }
    AMG_CUDA_TRY(cudaMemcpyAsync(h_added, added, sizeof(int) * batch, cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    bool done = false;
    for (int b = 0; b < batch; ++b) {
      ++rounds;
      matched += h_added[b];
      if (h_added[b] == 0) { done = true; break; }
    }
    if (done) break;
    if (rounds > 4 * n + 8)
      return fail(AMG_ERR_INVALID_ARG, "matching did not terminate: s must be symmetric and finite");
  }
  AMG_TRY(pool_alloc((void **)&rep, sizeof(int) * (size_t)std::max(n, 1), st));
  AMG_TRY(pool_alloc((void **)&id, sizeof(int) * (size_t)std::max(n, 1), st));
  k_rep_flags<<<nb, 256, 0, st>>>(n, mate, rep);
  LAUNCH_CHECK(launches);
  AMG_TRY(exclusive_scan_i32(rep, id, n, st, nullptr));
  if (launches) *launches += 2;
  k_coarse_ids<<<nb, 256, 0, st>>>(n, mate, id, agg, m0, m1);
  LAUNCH_CHECK(launches);
  pool_free(ptr, st);
  pool_free(added, st);
  pool_free(rep, st);
  pool_free(id, st);
  if (nH_out) *nH_out = (int)(n - matched / 2);
  if (rounds_out) *rounds_out = rounds;
  return AMG_OK;
}

amg_status match_pass(cudaStream_t st, int n, const int64_t *rowptr, const int32_t *col,
                      const double *s, uint64_t salt, int32_t *mate, int32_t *agg, int *nH_out,
                      int *rounds_out, int64_t *launches) {
  return match_core(st, n, rowptr, col, s, salt, mate, agg, nullptr, nullptr, nH_out, rounds_out,
                    launches, kMatchBatch);
}

// b[i] = a[i] widened for i < n, and b[n] = 0 (the scan's last entry)
__global__ void k_widen(int n, const int *a, int64_t *b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
  else if (i == n) b[n] = 0;
}

__global__ void k_max_abs(int n, const double *a, unsigned long long *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = (i < n) ? fabs(a[i]) : 0.0;
  if (!(v == v)) v = 1.0;  // NaN counts as non-zero (rejected earlier anyway)
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Galerkin for one matching pass: coarse row I merges the rows of its
// members m0 < m1 (m1 = -1 for a singleton).  W_IJ sums the members' entries
// in order (m0's row, then m1's row, CSR order), diag_I = sum_J W_IJ (J
// ascending) + d_I, d_I = d_m0 + d_m1.
// ---------------------------------------------------------------------------
// Members of a coarse row: the pair (m0, m1) of a matching pass (m1 = -1 for
// a singleton) or an ascending member list (ptr, mem) of an aggregation pass.
struct PairMembers {
  const int *m0, *m1;
  __device__ int count(int I) const { return m1[I] >= 0 ? 2 : 1; }
  __device__ int get(int I, int q) const { return q == 0 ? m0[I] : m1[I]; }
};
struct ListMembers {
  const int *ptr, *mem;
  __device__ int count(int I) const { return ptr[I + 1] - ptr[I]; }
  __device__ int get(int I, int q) const { return mem[ptr[I] + q]; }
};

// segment lengths len[I] of the coarse rows (len[nH] = 0 for the scan), and
// the gather's three list counters cleared on the way
template <typename M>
__global__ void k_pair_seglen(int nH, const int64_t *__restrict__ rp, M mb, int64_t *__restrict__ len,
                              int *longrows, int *huge, unsigned long long *hugeoff) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I == 0) {
    *longrows = 0;
    *huge = 0;
    *hugeoff = 0ull;
  }
  if (I == nH) len[nH] = 0;
  if (I >= nH) return;
  int64_t l = 0;
  for (int q = 0; q < mb.count(I); ++q) {
    const int v = mb.get(I, q);
    l += rp[v + 1] - rp[v];
  }
  len[I] = l;
}
// gather mapped entries of the coarse row into its segment, stable-sort by J,
// count distinct J != I.  One thread per coarse row.  Rows of up to
// kLocalSort entries keep their keys J in shared memory (the thread's own
// column of the block's key table) and write each entry straight to its
// place in the stable order: the number of entries with a smaller J, or the
// same J and an earlier gather position.  Longer rows are written in gather
// order and listed for k_gal_sort_long (up to kBlockSort entries, bitonic in
// shared memory) or k_gal_sort_huge (radix through scratch).
constexpr int kLocalSort = 64;
constexpr int kBlockSort = 8192;  // longest row sorted in shared memory (128 KB)
constexpr int kGatherThreads = 128;
template <typename M>
__global__ void __launch_bounds__(kGatherThreads)
    k_pair_gather(int nH, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                  const double *__restrict__ val, const int *__restrict__ agg, M mb,
                  const int64_t *__restrict__ seg, int *__restrict__ keyJ, double *__restrict__ kval,
                  int *__restrict__ count, int *longrows, int *huge, unsigned long long *hugeoff) {
  __shared__ int sk[kLocalSort][kGatherThreads];  // 32 KB
  const int t = threadIdx.x;
  const int I = blockIdx.x * kGatherThreads + t;
  if (I >= nH) return;
  const int64_t s0 = seg[I];
  const int64_t len = seg[I + 1] - s0;
  const int nm = mb.count(I);
  if (len <= kLocalSort) {
    int a = 0;
    for (int q = 0; q < nm; ++q) {
      const int v = mb.get(I, q);
      for (int64_t p = rp[v]; p < rp[v + 1]; ++p) sk[a++][t] = agg[col[p]];
    }
    const int n = (int)len;
    int c = 0;
    a = 0;
    for (int q = 0; q < nm; ++q) {
      const int v = mb.get(I, q);
      for (int64_t p = rp[v]; p < rp[v + 1]; ++p, ++a) {
        const int Ja = sk[a][t];
        int r = 0;
        bool first = true;
        for (int b = 0; b < n; ++b) {
          const int Jb = sk[b][t];
          const bool earlier_same = Jb == Ja && b < a;
          r += (Jb < Ja || earlier_same) ? 1 : 0;
          first = first && !earlier_same;
        }
        keyJ[s0 + r] = Ja;
        kval[s0 + r] = val[p];
        if (first && Ja != I) ++c;
      }
    }
    count[I] = c;
    return;
  }
  int64_t o = s0;
  for (int q = 0; q < nm; ++q) {
    const int v = mb.get(I, q);
    for (int64_t p = rp[v]; p < rp[v + 1]; ++p, ++o) {
      keyJ[o] = agg[col[p]];
      kval[o] = val[p];
    }
  }
  if (longrows && len <= kBlockSort) {
    // long row: sorted by k_gal_sort_long, one block per row
    longrows[1 + atomicAdd(longrows, 1)] = I;
    count[I] = 0;
    return;
  }
  if (huge) {
    // very long row: stable radix sort by k_gal_sort_huge through scratch
    const int r = atomicAdd(huge, 1);
    huge[1 + r] = I;
    hugeoff[1 + r] = atomicAdd(hugeoff, (unsigned long long)len);
    count[I] = 0;
    return;
  }
  for (int64_t a = 1; a < len; ++a) {  // stable insertion sort by J (no scratch given)
    const int kj = keyJ[s0 + a];
    const double kv = kval[s0 + a];
    int64_t b = a - 1;
    while (b >= 0 && keyJ[s0 + b] > kj) {
      keyJ[s0 + b + 1] = keyJ[s0 + b];
      kval[s0 + b + 1] = kval[s0 + b];
      --b;
    }
    keyJ[s0 + b + 1] = kj;
    kval[s0 + b + 1] = kv;
  }
  int c = 0;
  for (int64_t a = 0; a < len; ++a) {
    const int J = keyJ[s0 + a];
    if (J != I && (a == 0 || keyJ[s0 + a - 1] != J)) ++c;
  }
  count[I] = c;
}

// Rows with kLocalSort < len <= kBlockSort entries (large aggregates): one
// block per row sorts (J, gather position) with a bitonic network in shared
// memory -- the position makes the order stable, as the summation order of
// the Galerkin sums requires -- then writes the row back and counts its
// distinct J != I.  Rows come from the list filled by k_pair_gather.
constexpr int kSortThreads = 128;
constexpr int kGalSortSmem = (int)(sizeof(unsigned long long) + sizeof(double)) * kBlockSort;
__global__ void __launch_bounds__(kSortThreads) k_gal_sort_long(const int64_t *__restrict__ seg,
                                                                int *__restrict__ keyJ, double *__restrict__ kval,
                                                                int *__restrict__ count, const int *longrows) {
  extern __shared__ __align__(16) unsigned char sort_smem[];
  unsigned long long *key = reinterpret_cast<unsigned long long *>(sort_smem);
  double *v = reinterpret_cast<double *>(sort_smem + sizeof(unsigned long long) * kBlockSort);
  __shared__ int cnt;
  const int nlong = longrows[0];
  for (int r = blockIdx.x; r < nlong; r += gridDim.x) {
    const int I = longrows[1 + r];
    const int64_t s0 = seg[I];
    const int len = (int)(seg[I + 1] - s0);
    int p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int a = threadIdx.x; a < p2; a += kSortThreads) {
      if (a < len) {
        key[a] = ((unsigned long long)(unsigned)keyJ[s0 + a] << 32) | (unsigned)a;
        v[a] = kval[s0 + a];
      } else {
        key[a] = ~0ull;
        v[a] = 0.0;
      }
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int a = threadIdx.x; a < p2; a += kSortThreads) {
          const int b = a ^ stride;
          if (b > a) {
            const bool up = (a & size) == 0;
            if ((key[a] > key[b]) == up) {
              const unsigned long long tk = key[a];
              key[a] = key[b];
              key[b] = tk;
              const double tv = v[a];
              v[a] = v[b];
              v[b] = tv;
            }
          }
        }
        __syncthreads();
      }
    }
    int c = 0;
    for (int a = threadIdx.x; a < len; a += kSortThreads) {
      const int J = (int)(key[a] >> 32);
      keyJ[s0 + a] = J;
      kval[s0 + a] = v[a];
      if (J != I && (a == 0 || (int)(key[a - 1] >> 32) != J)) ++c;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) count[I] = cnt;
    __syncthreads();  // key, v and cnt are reused by the next row
  }
}

// Stable LSD radix sort, 4-bit digits, of key[0, len) (keys in [0, 2^bits))
// with an optional payload, by one block of kRadixThreads threads, through
// global scratch of the same length.  Thread t owns the t-th contiguous chunk
// and scatters it in order, so equal keys keep their order.  Ends with the
// result in key/val and a block barrier.
constexpr int kRadixThreads = 256;
__device__ void block_radix_sort(int *key, double *val, int *tk, double *tv, int len, int bits, int *cnt) {
  const int t = threadIdx.x, T = kRadixThreads;
  const int chunk = (len + T - 1) / T;
  const int a0 = min(len, t * chunk), a1 = min(len, a0 + chunk);
  int *src = key, *dst = tk;
  double *vs = val, *vd = tv;
  for (int shift = 0; shift < bits; shift += 4) {
    for (int d = 0; d < 16; ++d) cnt[d * T + t] = 0;
    for (int a = a0; a < a1; ++a) ++cnt[((src[a] >> shift) & 15) * T + t];
    __syncthreads();
    if (t < 16) {  // exclusive scan of digit t over the threads
      int run = 0;
      for (int u = 0; u < T; ++u) {
        const int c = cnt[t * T + u];
        cnt[t * T + u] = run;
        run += c;
      }
      cnt[16 * T + t] = run;  // digit total
    }
    __syncthreads();
    if (t == 0) {  // digit bases
      int run = 0;
      for (int d = 0; d < 16; ++d) {
        const int c = cnt[16 * T + d];
        cnt[16 * T + d] = run;
        run += c;
      }
    }
    __syncthreads();
    for (int a = a0; a < a1; ++a) {
      const int d = (src[a] >> shift) & 15;
      const int pos = cnt[16 * T + d] + cnt[d * T + t]++;
      dst[pos] = src[a];
      if (vs) vd[pos] = vs[a];
    }
    __syncthreads();
    int *ts = src;
    src = dst;
    dst = ts;
    double *tvv = vs;
    vs = vd;
    vd = tvv;
  }
  if (src != key) {
    for (int a = t; a < len; a += T) {
      key[a] = src[a];
      if (val) val[a] = vs[a];
    }
  }
  __syncthreads();
}

// Galerkin rows of more than kBlockSort entries (a few coarse rows of a small,
// dense level): one block per row, radix sort by J (J < nH: `bits` bits),
// then the count of distinct J != I
__global__ void __launch_bounds__(kRadixThreads) k_gal_sort_huge(const int64_t *__restrict__ seg, int *keyJ,
                                                                 double *kval, int *__restrict__ count,
                                                                 const int *huge, const unsigned long long *hugeoff,
                                                                 int *skey, double *sval, int bits) {
  __shared__ int cnt[17 * kRadixThreads];
  __shared__ int tot;
  const int nh = huge[0];
  for (int r = blockIdx.x; r < nh; r += gridDim.x) {
    const int I = huge[1 + r];
    const int64_t s0 = seg[I];
    const int len = (int)(seg[I + 1] - s0);
    int *key = keyJ + s0;
    double *val = kval + s0;
    block_radix_sort(key, val, skey + hugeoff[1 + r], sval + hugeoff[1 + r], len, bits, cnt);
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    int c = 0;
    for (int a = threadIdx.x; a < len; a += kRadixThreads)
      if (key[a] != I && (a == 0 || key[a - 1] != key[a])) ++c;
    atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) count[I] = tot;
    __syncthreads();
  }
}

static inline int bits_for(int64_t n) {  // bits of the largest value below n
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < n) ++b;
  return b;
}

template <typename M>
__global__ void k_pair_emit(int nH, const int64_t *__restrict__ seg, const int *__restrict__ keyJ,
                            const double *__restrict__ kval, const int64_t *__restrict__ rpH,
                            const double *__restrict__ dlow, M mb, int32_t *__restrict__ colH,
                            double *__restrict__ valH, double *__restrict__ diagH,
                            double *__restrict__ dlowH) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nH) return;
  const int64_t s0 = seg[I], s1 = seg[I + 1];
  int64_t o = rpH[I];
  double wsum = 0.0;
  int64_t a = s0;
  while (a < s1) {
    const int J = keyJ[a];
    double acc = 0.0;
    int64_t b = a;
    for (; b < s1 && keyJ[b] == J; ++b) acc += -kval[b];
    if (J != I) {
      colH[o] = J;
      valH[o] = -acc;
      ++o;
      wsum += acc;
    }
    a = b;
  }
  double dI = 0.0;
  for (int q = 0; q < mb.count(I); ++q) dI += dlow[mb.get(I, q)];
  dlowH[I] = dI;
  diagH[I] = wsum + dI;
}

__global__ void k_compose(int n, int *__restrict__ comp, const int *__restrict__ aggp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) comp[i] = aggp[comp[i]];
}

// aggregate membership lists (restriction): counts, then placement, then a
// per-aggregate sort so that members are ascending
__global__ void k_agg_count(int n, const int *__restrict__ agg, int *__restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_agg_place(int n, const int *__restrict__ agg, const int *__restrict__ ptr,
                            int *__restrict__ fill, int *__restrict__ mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int I = agg[i];
  mem[ptr[I] + atomicAdd(&fill[I], 1)] = i;
}
// members of each aggregate in ascending order: insertion sort by one
// thread for short lists; lists of kAggShort < len <= kBlockSort members go
// to `longlist` for k_agg_sort_long (longer ones stay with the thread)
constexpr int kAggShort = 64;
__global__ void k_agg_sort(int nH, const int *__restrict__ ptr, int *__restrict__ mem, int *longlist) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nH) return;
  const int a0 = ptr[I], a1 = ptr[I + 1];
  if (longlist && a1 - a0 > kAggShort) {  // block sorts; k_agg_sort_long takes <= 8192
    longlist[1 + atomicAdd(longlist, 1)] = I;
    return;
  }
  for (int a = a0 + 1; a < a1; ++a) {
    int v = mem[a], b = a - 1;
    while (b >= a0 && mem[b] > v) { mem[b + 1] = mem[b]; --b; }
    mem[b + 1] = v;
  }
}

// one block per long member list: bitonic sort of the (distinct) vertex ids
// for lists of up to 8192 members (longer ones: k_agg_sort_huge)
__global__ void __launch_bounds__(128) k_agg_sort_long(const int *__restrict__ ptr, int *__restrict__ mem,
                                                        const int *longlist) {
  __shared__ int key[8192];
  const int nlong = longlist[0];
  for (int r = blockIdx.x; r < nlong; r += gridDim.x) {
    const int I = longlist[1 + r];
    const int a0 = ptr[I], len = ptr[I + 1] - a0;
    if (len > 8192) continue;  // block-uniform
    int p2 = 1;
    while (p2 < len) p2 <<= 1;
    for (int a = threadIdx.x; a < p2; a += blockDim.x) key[a] = a < len ? mem[a0 + a] : 0x7fffffff;
    __syncthreads();
    for (int size = 2; size <= p2; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int a = threadIdx.x; a < p2; a += blockDim.x) {
          const int b = a ^ stride;
          if (b > a && ((key[a] > key[b]) == ((a & size) == 0))) {
            const int t = key[a];
            key[a] = key[b];
            key[b] = t;
          }
        }
        __syncthreads();
      }
    }
    for (int a = threadIdx.x; a < len; a += blockDim.x) mem[a0 + a] = key[a];
    __syncthreads();
  }
}

// member lists of more than 8192 members: one block each, radix sort of the
// vertex ids (< n: `bits` bits) through scratch[ptr[I], ptr[I+1])
__global__ void __launch_bounds__(kRadixThreads) k_agg_sort_huge(const int *__restrict__ ptr, int *mem,
                                                                 const int *longlist, int *scratch, int bits) {
  __shared__ int cnt[17 * kRadixThreads];
  const int nlong = longlist[0];
  for (int r = blockIdx.x; r < nlong; r += gridDim.x) {
    const int I = longlist[1 + r];
    const int a0 = ptr[I], len = ptr[I + 1] - a0;
    if (len <= 8192) continue;  // block-uniform
    block_radix_sort(mem + a0, nullptr, scratch + a0, nullptr, len, bits, cnt);
  }
}

// sort member lists (ptr, mem) of nH aggregates in ascending order
static amg_status sort_members(amg_handle_s *h, int n, int nH, const int *ptr, int *mem) {
  cudaStream_t st = h->stream;
  int *longlist = nullptr;
  AMG_TRY(pool_alloc((void **)&longlist, sizeof(int) * (size_t)(nH + 1), st));
  AMG_CUDA_TRY(cudaMemsetAsync(longlist, 0, sizeof(int), st));
  k_agg_sort<<<blocks_for(nH, 128), 128, 0, st>>>(nH, ptr, mem, longlist);
  LAUNCH_CHECK(&h->launches);
  k_agg_sort_long<<<std::max(1, std::min(nH, 4 * 152)), 128, 0, st>>>(ptr, mem, longlist);
  LAUNCH_CHECK(&h->launches);
  // lists of more than 8192 members (some aggregate that large); the pass
  // skips every other list
  int *scratch = nullptr;
  AMG_TRY(pool_alloc((void **)&scratch, sizeof(int) * (size_t)std::max(n, 1), st));
  k_agg_sort_huge<<<std::max(1, std::min(nH, 152)), kRadixThreads, 0, st>>>(ptr, mem, longlist, scratch,
                                                                            bits_for(n));
  LAUNCH_CHECK(&h->launches);
  pool_free(scratch, st);
  pool_free(longlist, st);
  return AMG_OK;
}

// lambda1 = ||A||_inf = max_i (|a_ii| + sum_j |a_ij|), summed in row order
__global__ void k_norm_inf(int n, const int64_t *__restrict__ rp, const double *__restrict__ val,
                           const double *__restrict__ diag, unsigned long long *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    s = fabs(diag[i]);
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += fabs(val[p]);
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

// ---------------------------------------------------------------------------
// SELL-32 conversion
// ---------------------------------------------------------------------------
// slice widths, and the largest |j - i| of the level in *maxdel
__global__ void k_sell_width(int n, int nslices, const int64_t *__restrict__ rp,
                             const int32_t *__restrict__ col, int64_t *__restrict__ slen,
                             unsigned long long *maxdel) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int row = s * kSlice + lane;
  int deg = 0;
  unsigned dmax = 0;
  if (s < nslices && row < n) {
    deg = (int)(rp[row + 1] - rp[row]);
    for (int64_t p = rp[row]; p < rp[row + 1]; ++p) {
      const int64_t d = (int64_t)col[p] - row;
      const int64_t a = d < 0 ? -d : d;
      dmax = max(dmax, a > 0xffffffffll ? 0xffffffffu : (unsigned)a);
    }
  }
  deg = __reduce_max_sync(0xffffffffu, deg);
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  if (s < nslices && lane == 0) {
    slen[s] = (int64_t)deg * kSlice;
    if (dmax) atomicMax(maxdel, (unsigned long long)dmax);
  }
}

// the SELL layout of a level; sdel (optional: every |j - i| of the level
// fits 16 bits) receives the columns as offsets from the row as well
__global__ void k_sell_fill(int n, int nslices, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const double *__restrict__ val,
                            const int64_t *__restrict__ sptr, int32_t *__restrict__ scol,
                            double *__restrict__ sval, int16_t *__restrict__ sdel) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = row >> 5, lane = row & 31;
  if (s >= nslices) return;
  const int64_t base = sptr[s];
  const int w = (int)((sptr[s + 1] - base) / kSlice);
  int k = 0;
  if (row < n) {
    for (int64_t p = rp[row]; p < rp[row + 1]; ++p, ++k) {
      scol[base + (int64_t)k * kSlice + lane] = col[p];
      sval[base + (int64_t)k * kSlice + lane] = val[p];
      if (sdel) sdel[base + (int64_t)k * kSlice + lane] = (int16_t)(col[p] - row);
    }
  }
  for (; k < w; ++k) {  // padding: zero weight on the row itself
    scol[base + (int64_t)k * kSlice + lane] = row < n ? row : 0;
    sval[base + (int64_t)k * kSlice + lane] = 0.0;
    if (sdel) sdel[base + (int64_t)k * kSlice + lane] = 0;
  }
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// coarsest level: dense A_c, shifted M = A_c + alpha 1 1^T for a pure
// Laplacian (alpha = trace / n^2), in-place Gauss-Jordan inverse (M is SPD:
// no pivoting), Z = M^{-1} - 1 1^T / (alpha n^2) = A_c^+.
// ---------------------------------------------------------------------------
__global__ void k_dense(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                        const double *__restrict__ val, const double *__restrict__ diag,
                        double shift, double *__restrict__ M) {
  int i = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) M[(int64_t)i * n + j] = shift;
  __syncthreads();
  if (threadIdx.x == 0) {
    M[(int64_t)i * n + i] += diag[i];
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) M[(int64_t)i * n + col[p]] += val[p];
  }
}

__global__ void k_trace(int n, const double *__restrict__ diag, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += diag[i];
    *out = s;
  }
}

// one Gauss-Jordan pivot step, reading Min and writing Mout
__global__ void k_gj_step(int n, int p, const double *__restrict__ Min, double *__restrict__ Mout,
                          double tiny, int *singular) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  const double piv = Min[(int64_t)p * n + p];
  if (idx == 0 && !(piv > tiny)) *singular = 1;
  const double inv = 1.0 / piv;
  double out;
  if (i == p) {
    out = (j == p) ? inv : Min[(int64_t)p * n + j] * inv;
  } else {
    const double f = Min[(int64_t)i * n + p];
    out = (j == p) ? -f * inv : fma(-f, Min[(int64_t)p * n + j] * inv, Min[(int64_t)i * n + j]);
  }
  Mout[idx] = out;
}

// all n pivot steps of k_gj_step in one block with the matrix in shared
// memory (coarsest levels of up to kGjShared rows).  Per step the pivot
// column and the scaled pivot row t_j = a_pj / a_pp are formed once, then
// every entry is replaced in place by the formula of k_gj_step (the same
// operations in the same order, so the same result); thread (ty, tx) owns
// column tx of rows ty, ty + 8, ...
constexpr int kGjThreads = 512;
constexpr int kGjShared = 64;
__global__ void __launch_bounds__(kGjThreads) k_gj_shared(int n, const double *__restrict__ Min,
                                                          double *__restrict__ Zout, double tiny,
                                                          int *singular) {
  __shared__ double a[kGjShared][kGjShared];
  __shared__ double trow[kGjShared], pcol[kGjShared];
  __shared__ double sinv;
  const int tx = threadIdx.x % kGjShared, ty = threadIdx.x / kGjShared;
  constexpr int kRowStep = kGjThreads / kGjShared;
  for (int i = ty; i < n; i += kRowStep)
    if (tx < n) a[i][tx] = Min[(int64_t)i * n + tx];
  __syncthreads();
  for (int p = 0; p < n; ++p) {
    if (threadIdx.x == 0) {
      const double piv = a[p][p];
      if (!(piv > tiny)) *singular = 1;
      sinv = 1.0 / piv;
    }
    __syncthreads();
    const double inv = sinv;
    if (threadIdx.x < n) {
      trow[threadIdx.x] = a[p][threadIdx.x] * inv;
      pcol[threadIdx.x] = a[threadIdx.x][p];
    }
    __syncthreads();
    if (tx < n) {
      for (int i = ty; i < n; i += kRowStep) {
        double out;
        if (i == p) {
          out = (tx == p) ? inv : trow[tx];
        } else {
          const double f = pcol[i];
          out = (tx == p) ? -f * inv : fma(-f, trow[tx], a[i][tx]);
        }
        a[i][tx] = out;
      }
    }
    __syncthreads();
  }
  for (int i = ty; i < n; i += kRowStep)
    if (tx < n) Zout[(int64_t)i * n + tx] = a[i][tx];
}

__global__ void k_unshift(int64_t nn, double c, double *__restrict__ Z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) Z[i] -= c;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static void closed_form_coefficients(int m, double l0, double l1, double *c) {
  // Best uniform approximation to 1/x on [l0, l1] (Eq. (1x-1-min)).  With
  // t = (2x - l1 - l0)/(l1 - l0), 1/x = 2/(l1 - l0) * 1/(t + a),
  // a = (l1 + l0)/(l1 - l0), delta = a - sqrt(a^2 - 1); the best degree-m
  // approximant of 1/(t + a) in Chebyshev form keeps the first m terms of
  // the expansion 1/(t+a) = 4 delta/(1 - delta^2) * sum' (-delta)^k T_k and
  // replaces the last by (-1)^m 4 delta^(m+1)/(1 - delta^2)^2 (equioscillation
  // with m+2 alternation points including both ends; its error level is
  // delta^m (kappa - 1)/2 / l1 as stated in Sec. 3).
  const double a = (l1 + l0) / (l1 - l0);
  const double dl = a - sqrt(a * a - 1.0);
  const double om = 1.0 - dl * dl;
  const double scale = 2.0 / (l1 - l0);
  if (m == 0) {
    c[0] = scale * 2.0 * dl * (1.0 + dl * dl) / (om * om);
    return;
  }
  c[0] = scale * 2.0 * dl / om;
  double pw = 1.0;
  for (int k = 1; k < m; ++k) {
    pw *= -dl;
    c[k] = scale * 4.0 * dl * pw / om;
  }
  pw *= -dl;
  c[m] = scale * 4.0 * dl * pw / (om * om);
}

namespace {
struct LevelBuild {
  Csr A;
  double *diag = nullptr, *dlow = nullptr;
};
}  // namespace

static amg_status alloc_persist(amg_handle_s *h, void **p, size_t bytes) {
  return h->arena.alloc(p, bytes);
}

// Galerkin A_H = P^T A P on `cur` for the aggregates given by agg and their
// members (owned temporaries in `next`); sums as documented at k_pair_gather
// the long-row sort needs 128 KB of dynamic shared memory: allowed once per
// device (function attributes are process-wide; set under a lock)
static amg_status sort_kernels_ready() {
  static std::mutex mu;
  static bool done[64];
  int dev = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(AMG_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    AMG_CUDA_TRY(cudaFuncSetAttribute(k_gal_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize, kGalSortSmem));
    done[dev] = true;
  }
  return AMG_OK;
}

template <typename M>
static amg_status galerkin(amg_handle_s *h, const LevelBuild &cur, const int *aggp, M mb, int nH,
                           LevelBuild &next) {
  cudaStream_t st = h->stream;
  const unsigned nbH = blocks_for(nH, 256);
  int64_t *seglen = nullptr, *seg = nullptr;
  AMG_TRY(pool_alloc((void **)&seglen, sizeof(int64_t) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&seg, sizeof(int64_t) * (size_t)(nH + 1), st));
  int *longrows = nullptr, *huge = nullptr;  // [0]: count, then the rows
  unsigned long long *hugeoff = nullptr;     // [0]: total length, then scratch offsets
  AMG_TRY(pool_alloc((void **)&longrows, sizeof(int) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&huge, sizeof(int) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&hugeoff, sizeof(unsigned long long) * (size_t)(nH + 1), st));
  k_pair_seglen<<<blocks_for((int64_t)nH + 1, 256), 256, 0, st>>>(nH, cur.A.rowptr, mb, seglen, longrows, huge,
                                                                   hugeoff);
  LAUNCH_CHECK(&h->launches);
  // every fine row belongs to exactly one aggregate: the segments hold the
  // fine level's entries, cur.A.nnz of them (or fewer when that is a bound)
  const int64_t segtot = cur.A.nnz;
  AMG_TRY(exclusive_scan_i64(seglen, seg, nH + 1, st, nullptr));
  int *keyJ = nullptr, *count = nullptr;
  double *kval = nullptr;
  AMG_TRY(pool_alloc((void **)&keyJ, sizeof(int) * (size_t)std::max<int64_t>(segtot, 1), st));
  AMG_TRY(pool_alloc((void **)&kval, sizeof(double) * (size_t)std::max<int64_t>(segtot, 1), st));
  AMG_TRY(pool_alloc((void **)&count, sizeof(int64_t) * (size_t)(nH + 1), st));

  k_pair_gather<<<blocks_for(nH, kGatherThreads), kGatherThreads, 0, st>>>(
      nH, cur.A.rowptr, cur.A.col, cur.A.val, aggp, mb, seg, keyJ, kval, count, longrows, huge, hugeoff);
  LAUNCH_CHECK(&h->launches);
  {
    // rows of more than kBlockSort entries, if any: their scratch is bounded
    // by the segment total, and the kernel reads their count on the device
    // (no host check; with none, every block returns at once)
    int *skey = nullptr;
    double *sval = nullptr;
    AMG_TRY(pool_alloc((void **)&skey, sizeof(int) * (size_t)std::max<int64_t>(segtot, 1), st));
    AMG_TRY(pool_alloc((void **)&sval, sizeof(double) * (size_t)std::max<int64_t>(segtot, 1), st));
    k_gal_sort_huge<<<std::max(1, std::min(nH, 152)), kRadixThreads, 0, st>>>(seg, keyJ, kval, count, huge, hugeoff,
                                                                               skey, sval, bits_for(nH));
    LAUNCH_CHECK(&h->launches);
    pool_free(skey, st);
    pool_free(sval, st);
  }
  pool_free(huge, st);
  pool_free(hugeoff, st);
  AMG_TRY(sort_kernels_ready());
  k_gal_sort_long<<<std::max(1, std::min(nH, 4 * 152)), kSortThreads, kGalSortSmem, st>>>(seg, keyJ, kval, count,
                                                                                          longrows);
  LAUNCH_CHECK(&h->launches);
  pool_free(longrows, st);
  // widen counts to int64 for the row-offset scan
  int64_t *cnt64 = nullptr;
  AMG_TRY(pool_alloc((void **)&cnt64, sizeof(int64_t) * (size_t)(nH + 1), st));
  k_widen<<<blocks_for((int64_t)nH + 1, 256), 256, 0, st>>>(nH, count, cnt64);
  LAUNCH_CHECK(&h->launches);
  next.A.n = nH;
  AMG_TRY(pool_alloc((void **)&next.A.rowptr, sizeof(int64_t) * (size_t)(nH + 1), st));
  // the coarse rows hold at most the segments' entries: allocate for that
  // bound (the exact count stays on the device, in rowptr[nH], until the
  // level is complete)
  const int64_t nnzH = segtot;
  AMG_TRY(exclusive_scan_i64(cnt64, next.A.rowptr, nH + 1, st, nullptr));
  next.A.nnz = nnzH;
  AMG_TRY(pool_alloc((void **)&next.A.col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnzH, 1), st));
  AMG_TRY(pool_alloc((void **)&next.A.val, sizeof(double) * (size_t)std::max<int64_t>(nnzH, 1), st));
  AMG_TRY(pool_alloc((void **)&next.diag, sizeof(double) * (size_t)std::max(nH, 1), st));
  AMG_TRY(pool_alloc((void **)&next.dlow, sizeof(double) * (size_t)std::max(nH, 1), st));
  k_pair_emit<<<nbH, 256, 0, st>>>(nH, seg, keyJ, kval, next.A.rowptr, cur.dlow, mb, next.A.col, next.A.val,
                                   next.diag, next.dlow);
  LAUNCH_CHECK(&h->launches);
  pool_free(seglen, st);
  pool_free(seg, st);
  pool_free(keyJ, st);
  pool_free(kval, st);
  pool_free(count, st);
  pool_free(cnt64, st);
  return AMG_OK;
}

// one matching pass + Galerkin on `cur` (owned temporaries in `next`)
static amg_status coarsen_pass(amg_handle_s *h, const LevelBuild &cur, LevelBuild &next, int *aggp,
                               int *nH_out) {
  cudaStream_t st = h->stream;
  const int n = cur.A.n;
  const unsigned nb = blocks_for(n, 256);
  double *s = nullptr;
  int *mate = nullptr;
  AMG_TRY(pool_alloc((void **)&s, sizeof(double) * (size_t)std::max<int64_t>(cur.A.nnz, 1), st));
  k_strength<<<nb, 256, 0, st>>>(n, cur.A.rowptr, cur.A.col, cur.A.val, cur.diag, s);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(pool_alloc((void **)&mate, sizeof(int) * (size_t)std::max(n, 1), st));
  int *m0 = nullptr, *m1 = nullptr;
  AMG_TRY(pool_alloc((void **)&m0, sizeof(int) * (size_t)std::max(n, 1), st));
  AMG_TRY(pool_alloc((void **)&m1, sizeof(int) * (size_t)std::max(n, 1), st));
  int nH = 0, rounds = 0;
  // passes of one hierarchy take similar numbers of rounds: the first batch
  // covers the previous pass's count (one host check per pass, usually)
  const int first_batch = h->match_rounds_hint > 0 ? h->match_rounds_hint + 1 : 8;
  AMG_TRY(match_core(st, n, cur.A.rowptr, cur.A.col, s, h->opt.hash_salt, mate, aggp, m0, m1, &nH,
                     &rounds, &h->launches, first_batch));
  h->match_rounds_hint = rounds;
  pool_free(s, st);
  pool_free(mate, st);
  AMG_TRY(galerkin(h, cur, aggp, PairMembers{m0, m1}, nH, next));
  pool_free(m0, st);
  pool_free(m1, st);
  *nH_out = nH;
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// aggregation by a maximal independent set of the graph of A^k (Sec. 2 steps
// (A) and (B); Sec. 4: k = 4).  Keys ((splitmix64(salt ^ v) >> 33) + 1) << 32
// | v are distinct and nonzero.  (A) Luby's rule with fixed keys -- an
// undecided vertex whose key is the largest among undecided vertices within
// distance k joins S, then every vertex within distance k of a new root
// leaves the undecided set -- gives the greedy set in decreasing key order.
// (B) every vertex joins its nearest root, ties to the larger key: labels
// spread one layer per round, each new vertex taking its neighbours' largest
// label.  Distances come from k rounds of pull-style propagation over the
// whole graph (no atomics, deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mis_key(uint64_t salt, int v) {
  return (((splitmix64(salt ^ (uint64_t)v) >> 33) + 1) << 32) | (uint64_t)(uint32_t)v;
}

// state: 0 undecided, 1 root, 2 covered
__global__ void k_mis_seed(int n, const int *__restrict__ state, uint64_t salt, uint64_t *__restrict__ m) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) m[v] = state[v] == 0 ? mis_key(salt, v) : 0ull;
}

// out[v] = max(in[v], max_{u in N(v)} in[u]); with keep, a nonzero in[v] stays
__global__ void k_max_spread(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int keep) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint64_t b = in[v];
  if (keep && b) {
    out[v] = b;
    return;
  }
  for (int64_t p = rp[v]; p < rp[v + 1]; ++p) b = max(b, in[col[p]]);
  out[v] = b;
}

__global__ void k_mis_pick(int n, int *__restrict__ state, uint64_t salt, const uint64_t *__restrict__ m,
                           uint64_t *__restrict__ c) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const bool pick = state[v] == 0 && m[v] == mis_key(salt, v);
  if (pick) state[v] = 1;
  c[v] = pick ? 1ull : 0ull;
}

__global__ void k_mis_cover(int n, int *__restrict__ state, const uint64_t *__restrict__ c, int *left) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (state[v] == 0) {
    if (c[v]) state[v] = 2;
    else atomicAdd(left, 1);
  }
}

__global__ void k_mis_label(int n, const int *__restrict__ state, uint64_t salt, uint64_t *__restrict__ lab,
                            int *__restrict__ isroot) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  lab[v] = state[v] == 1 ? mis_key(salt, v) : 0ull;
  isroot[v] = state[v] == 1;
}

__global__ void k_mis_agg(int n, const uint64_t *__restrict__ lab, const int *__restrict__ rank,
                          int *__restrict__ agg, int *bad) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (!lab[v]) {  // unreachable: S is maximal
    atomicExch(bad, 1);
    agg[v] = 0;
    return;
  }
  agg[v] = rank[(uint32_t)(lab[v] & 0xffffffffull)];
}

static amg_status mis_aggregate(amg_handle_s *h, int n, const int64_t *rp, const int32_t *col, int k, int *aggp,
                                int *nH_out) {
  cudaStream_t st = h->stream;
  const unsigned nb = blocks_for(n, 256);
  const uint64_t salt = h->opt.hash_salt;
  int *state = nullptr, *isroot = nullptr, *rank = nullptr, *flag = nullptr;
  uint64_t *a = nullptr, *b = nullptr;
  AMG_TRY(pool_alloc((void **)&state, sizeof(int) * (size_t)n, st));
  AMG_TRY(pool_alloc((void **)&isroot, sizeof(int) * (size_t)n, st));
  AMG_TRY(pool_alloc((void **)&rank, sizeof(int) * (size_t)n, st));
  AMG_TRY(pool_alloc((void **)&a, sizeof(uint64_t) * (size_t)n, st));
  AMG_TRY(pool_alloc((void **)&b, sizeof(uint64_t) * (size_t)n, st));
  AMG_TRY(pool_alloc((void **)&flag, sizeof(int) * 2, st));
  AMG_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(int) * (size_t)n, st));
  // k spreading rounds ping-pong between a and b; the result is in *res
  auto spread = [&](uint64_t **res, int keep) -> amg_status {
    uint64_t *src = *res, *dst = (src == a) ? b : a;
    for (int r = 0; r < k; ++r) {
      k_max_spread<<<nb, 256, 0, st>>>(n, rp, col, src, dst, keep);
      LAUNCH_CHECK(&h->launches);
      std::swap(src, dst);
    }
    *res = src;
    return AMG_OK;
  };
  // (A) every round picks at least the largest undecided key, so at most n rounds
  for (int round = 0;; ++round) {
    if (round > n) return fail(AMG_ERR_CUDA, "independent-set selection did not terminate");
    uint64_t *m = a;
    k_mis_seed<<<nb, 256, 0, st>>>(n, state, salt, m);
    LAUNCH_CHECK(&h->launches);
    AMG_TRY(spread(&m, 0));
    uint64_t *c = (m == a) ? b : a;
    k_mis_pick<<<nb, 256, 0, st>>>(n, state, salt, m, c);
    LAUNCH_CHECK(&h->launches);
    AMG_TRY(spread(&c, 0));
    AMG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_mis_cover<<<nb, 256, 0, st>>>(n, state, c, flag);
    LAUNCH_CHECK(&h->launches);
    int left = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&left, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    if (left == 0) break;
  }
  // (B) nearest root, ties to the larger key
  uint64_t *lab = a;
  k_mis_label<<<nb, 256, 0, st>>>(n, state, salt, lab, isroot);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(spread(&lab, 1));
  int nH = 0;
  {
    int64_t tot = 0;
    AMG_TRY(exclusive_scan_i32(isroot, rank, n, st, &tot));
    nH = (int)tot;
  }
  AMG_CUDA_TRY(cudaMemsetAsync(flag + 1, 0, sizeof(int), st));
  k_mis_agg<<<nb, 256, 0, st>>>(n, lab, rank, aggp, flag + 1);
  LAUNCH_CHECK(&h->launches);
  int bad = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&bad, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  for (void *p : {(void *)state, (void *)isroot, (void *)rank, (void *)a, (void *)b, (void *)flag}) pool_free(p, st);
  if (bad) return fail(AMG_ERR_CUDA, "a vertex farther than k from every root");
  *nH_out = nH;
  return AMG_OK;
}

// one aggregation pass by a maximal independent set + Galerkin on `cur`
static amg_status coarsen_mis_pass(amg_handle_s *h, const LevelBuild &cur, LevelBuild &next, int *aggp,
                                   int *nH_out) {
  cudaStream_t st = h->stream;
  const int n = cur.A.n;
  int nH = 0;
  AMG_TRY(mis_aggregate(h, n, cur.A.rowptr, cur.A.col, h->opt.mis_k, aggp, &nH));
  // member lists, ascending
  int *cnt = nullptr, *fill = nullptr, *ptr = nullptr, *mem = nullptr;
  AMG_TRY(pool_alloc((void **)&cnt, sizeof(int) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&fill, sizeof(int) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&ptr, sizeof(int) * (size_t)(nH + 1), st));
  AMG_TRY(pool_alloc((void **)&mem, sizeof(int) * (size_t)std::max(n, 1), st));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nH + 1), st));
  AMG_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)(nH + 1), st));
  k_agg_count<<<blocks_for(n, 256), 256, 0, st>>>(n, aggp, cnt);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(exclusive_scan_i32(cnt, ptr, nH + 1, st, nullptr));  // total: n
  k_agg_place<<<blocks_for(n, 256), 256, 0, st>>>(n, aggp, ptr, fill, mem);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(sort_members(h, n, nH, ptr, mem));
  AMG_TRY(galerkin(h, cur, aggp, ListMembers{ptr, mem}, nH, next));
  for (void *p : {(void *)cnt, (void *)fill, (void *)ptr, (void *)mem}) pool_free(p, st);
  *nH_out = nH;
  return AMG_OK;
}

static void free_build(LevelBuild &b, cudaStream_t st) {
  pool_free(b.A.rowptr, st);
  pool_free(b.A.col, st);
  pool_free(b.A.val, st);
  pool_free(b.diag, st);
  pool_free(b.dlow, st);
  b = LevelBuild();
}

// copy a temporary level into handle-owned memory
static amg_status persist_level(amg_handle_s *h, const LevelBuild &b, amg::Level &L) {
  cudaStream_t st = h->stream;
  L.n = b.A.n;
  L.A.n = b.A.n;
  L.A.nnz = b.A.nnz;
  AMG_TRY(alloc_persist(h, (void **)&L.A.rowptr, sizeof(int64_t) * (size_t)(b.A.n + 1)));
  AMG_TRY(alloc_persist(h, (void **)&L.A.col, sizeof(int32_t) * (size_t)std::max<int64_t>(b.A.nnz, 1)));
  AMG_TRY(alloc_persist(h, (void **)&L.A.val, sizeof(double) * (size_t)std::max<int64_t>(b.A.nnz, 1)));
  AMG_TRY(alloc_persist(h, (void **)&L.diag, sizeof(double) * (size_t)std::max(b.A.n, 1)));
  AMG_TRY(alloc_persist(h, (void **)&L.dlow, sizeof(double) * (size_t)std::max(b.A.n, 1)));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.A.rowptr, b.A.rowptr, sizeof(int64_t) * (size_t)(b.A.n + 1),
                               cudaMemcpyDeviceToDevice, st));
  if (b.A.nnz) {
    AMG_CUDA_TRY(cudaMemcpyAsync(L.A.col, b.A.col, sizeof(int32_t) * (size_t)b.A.nnz,
                                 cudaMemcpyDeviceToDevice, st));
    AMG_CUDA_TRY(cudaMemcpyAsync(L.A.val, b.A.val, sizeof(double) * (size_t)b.A.nnz,
                                 cudaMemcpyDeviceToDevice, st));
  }
  AMG_CUDA_TRY(cudaMemcpyAsync(L.diag, b.diag, sizeof(double) * (size_t)b.A.n, cudaMemcpyDeviceToDevice, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(L.dlow, b.dlow, sizeof(double) * (size_t)b.A.n, cudaMemcpyDeviceToDevice, st));
  return AMG_OK;
}

// SELL-32 layout of every level in two stages, so that one read-back serves
// all levels: (1) slice widths and their scan (slice pointers) per level,
// totals left on the device; (2) with the totals known, the padded arrays.
// levels of at least this many rows get 16-bit column offsets (when they
// fit): the levels whose solve kernels run one row per thread
constexpr int kDeltaMinRows = 1 << 17;

static amg_status build_sell_all(amg_handle_s *h, bool want32) {
  cudaStream_t st = h->stream;
  const int L = h->L;
  // AMG_GB300_DELTA=0 keeps 32-bit columns on every level (A/B timing)
  const char *delta_env = getenv("AMG_GB300_DELTA");
  const bool delta_ok = !(delta_env && delta_env[0] == '0');
  // per level: stored entries, then the largest |j - i| (device)
  int64_t *totals = nullptr;
  AMG_TRY(pool_alloc((void **)&totals, sizeof(int64_t) * (size_t)(2 * L), st));
  AMG_CUDA_TRY(cudaMemsetAsync(totals + L, 0, sizeof(int64_t) * (size_t)L, st));
  for (int k = 0; k < L; ++k) {
    amg::Level &V = h->lv[k];
    Sell &S = V.S;
    S.n = V.n;
    S.nslices = (V.n + kSlice - 1) / kSlice;
    int64_t *slen = nullptr;
    AMG_TRY(pool_alloc((void **)&slen, sizeof(int64_t) * (size_t)(S.nslices + 1), st));
    AMG_CUDA_TRY(cudaMemsetAsync(slen, 0, sizeof(int64_t) * (size_t)(S.nslices + 1), st));
    k_sell_width<<<blocks_for((int64_t)S.nslices * 32, 256), 256, 0, st>>>(
        V.n, S.nslices, V.A.rowptr, V.A.col, slen, (unsigned long long *)(totals + L + k));
    LAUNCH_CHECK(&h->launches);
    AMG_TRY(alloc_persist(h, (void **)&S.sptr, sizeof(int64_t) * (size_t)(S.nslices + 1)));
    AMG_TRY(exclusive_scan_i64(slen, S.sptr, S.nslices + 1, st, nullptr));
    AMG_CUDA_TRY(cudaMemcpyAsync(totals + k, S.sptr + S.nslices, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    pool_free(slen, st);
  }
  std::vector<int64_t> stored((size_t)(2 * L), 0);
  AMG_CUDA_TRY(cudaMemcpyAsync(stored.data(), totals, sizeof(int64_t) * (size_t)(2 * L), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  pool_free(totals, st);
  for (int k = 0; k < L; ++k) {
    amg::Level &V = h->lv[k];
    Sell &S = V.S;
    S.stored = stored[k];
    AMG_TRY(alloc_persist(h, (void **)&S.scol, sizeof(int32_t) * (size_t)std::max<int64_t>(S.stored, 1)));
    AMG_TRY(alloc_persist(h, (void **)&S.val64, sizeof(double) * (size_t)std::max<int64_t>(S.stored, 1)));
    S.sdel = nullptr;
    if (delta_ok && V.n >= kDeltaMinRows && stored[L + k] <= 32767)
      AMG_TRY(alloc_persist(h, (void **)&S.sdel, sizeof(int16_t) * (size_t)std::max<int64_t>(S.stored, 1)));
    k_sell_fill<<<blocks_for((int64_t)S.nslices * 32, 256), 256, 0, st>>>(V.n, S.nslices, V.A.rowptr, V.A.col,
                                                                           V.A.val, S.sptr, S.scol, S.val64, S.sdel);
    LAUNCH_CHECK(&h->launches);
    S.diag64 = V.diag;
    if (want32) {
      AMG_TRY(alloc_persist(h, (void **)&S.val32, sizeof(float) * (size_t)std::max<int64_t>(S.stored, 1)));
      AMG_TRY(alloc_persist(h, (void **)&S.diag32, sizeof(float) * (size_t)std::max(V.n, 1)));
      if (S.stored) {
        k_to_f32<<<blocks_for(S.stored, 256), 256, 0, st>>>(S.stored, S.val64, S.val32);
        LAUNCH_CHECK(&h->launches);
      }
      k_to_f32<<<blocks_for(V.n, 256), 256, 0, st>>>(V.n, V.diag, S.diag32);
      LAUNCH_CHECK(&h->launches);
    }
  }
  return AMG_OK;
}

// member k of aggregate I at memw[k * nH + I] (k < W), -1 after the last
__global__ void k_agg_table(int nH, int W, const int *__restrict__ ptr, const int *__restrict__ mem,
                            int *__restrict__ memw) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nH) return;
  const int a0 = ptr[I], cnt = ptr[I + 1] - a0;
  for (int k = 0; k < W; ++k) memw[(size_t)k * nH + I] = k < cnt ? mem[a0 + k] : -1;
}

static amg_status build_agg_lists(amg_handle_s *h, amg::Level &L) {
  cudaStream_t st = h->stream;
  int *cnt = nullptr, *fill = nullptr;
  AMG_TRY(pool_alloc((void **)&cnt, sizeof(int) * (size_t)(L.nH + 1), st));
  AMG_TRY(pool_alloc((void **)&fill, sizeof(int) * (size_t)(L.nH + 1), st));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(L.nH + 1), st));
  AMG_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)(L.nH + 1), st));
  k_agg_count<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.agg, cnt);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(alloc_persist(h, (void **)&L.agg_ptr, sizeof(int) * (size_t)(L.nH + 1)));
  AMG_TRY(alloc_persist(h, (void **)&L.agg_mem, sizeof(int) * (size_t)std::max(L.n, 1)));
  AMG_TRY(exclusive_scan_i32(cnt, L.agg_ptr, L.nH + 1, st, nullptr));  // total: L.n
  k_agg_place<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.agg, L.agg_ptr, fill, L.agg_mem);
  LAUNCH_CHECK(&h->launches);
  AMG_TRY(sort_members(h, L.n, L.nH, L.agg_ptr, L.agg_mem));
  pool_free(cnt, st);
  pool_free(fill, st);
  // p matching passes make aggregates of at most 2^p members
  if (h->opt.aggregation == AMG_AGG_MATCHING && h->opt.passes >= 1 && h->opt.passes <= 3) {
    L.memw_width = 1 << h->opt.passes;
    AMG_TRY(alloc_persist(h, (void **)&L.memw, sizeof(int32_t) * (size_t)L.memw_width * (size_t)std::max(L.nH, 1)));
    k_agg_table<<<blocks_for(L.nH, 256), 256, 0, st>>>(L.nH, L.memw_width, L.agg_ptr, L.agg_mem, L.memw);
    LAUNCH_CHECK(&h->launches);
  }
  return AMG_OK;
}

static amg_status build_coarsest(amg_handle_s *h) {
  cudaStream_t st = h->stream;
  amg::Level &C = h->lv[h->L - 1];
  const int n = C.n;
  h->nc = n;
  double *tr = nullptr, *M = nullptr;
  int *sing = nullptr;
  AMG_TRY(pool_alloc((void **)&tr, sizeof(double), st));
  AMG_TRY(pool_alloc((void **)&sing, sizeof(int), st));
  AMG_CUDA_TRY(cudaMemsetAsync(sing, 0, sizeof(int), st));
  k_trace<<<1, 32, 0, st>>>(n, C.diag, tr);
  LAUNCH_CHECK(&h->launches);
  double trace = 0.0;
  std::vector<double> dg(n);
  AMG_CUDA_TRY(cudaMemcpyAsync(&trace, tr, sizeof(double), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(dg.data(), C.diag, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  const double alpha = h->pure ? trace / ((double)n * (double)n) : 0.0;
  const int64_t nn = (int64_t)n * n;
  AMG_TRY(alloc_persist(h, (void **)&h->Z, sizeof(double) * (size_t)nn));
  if (h->pure && !(trace > 0.0)) {  // one isolated vertex: A = [0], A^+ = [0]
    AMG_CUDA_TRY(cudaMemsetAsync(h->Z, 0, sizeof(double) * (size_t)nn, st));
    pool_free(tr, st);
    pool_free(sing, st);
    return AMG_OK;
  }
  AMG_TRY(pool_alloc((void **)&M, sizeof(double) * (size_t)nn, st));
  k_dense<<<n, 128, 0, st>>>(n, C.A.rowptr, C.A.col, C.A.val, C.diag, alpha, M);
  LAUNCH_CHECK(&h->launches);
  double maxdiag = 0.0;
  for (double v : dg) maxdiag = std::max(maxdiag, v);
  const double tiny = 1e-13 * std::max(maxdiag, 1e-300);
  double *a = M, *b = h->Z;
  if (n <= kGjShared) {
    k_gj_shared<<<1, kGjThreads, 0, st>>>(n, M, h->Z, tiny, sing);
    LAUNCH_CHECK(&h->launches);
    a = h->Z;
  } else {
    for (int p = 0; p < n; ++p) {
      k_gj_step<<<blocks_for(nn, 256), 256, 0, st>>>(n, p, a, b, tiny, sing);
      LAUNCH_CHECK(&h->launches);
      std::swap(a, b);
    }
  }
  if (a != h->Z) AMG_CUDA_TRY(cudaMemcpyAsync(h->Z, a, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  if (h->pure) {
    k_unshift<<<blocks_for(nn, 256), 256, 0, st>>>(nn, 1.0 / (alpha * (double)n * (double)n), h->Z);
    LAUNCH_CHECK(&h->launches);
  }
  int hs = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  pool_free(M, st);
  pool_free(tr, st);
  pool_free(sing, st);
  if (hs) return fail(AMG_ERR_DISCONNECTED, "coarsest operator is singular beyond the constants");
  return AMG_OK;
}

amg_status build_hierarchy(amg_handle_s *h, int64_t n64, const int64_t *rowptr, const int32_t *col,
                           const double *w, const double *d) {
  cudaStream_t st = h->stream;
  const int n = (int)n64;
  const unsigned nb = blocks_for(n, 256);
  NvtxPhase phase(st);
  phase.next("amg_setup: validation");
  // ---- validation (order of the C ABI's error list) ----
  unsigned *flags = nullptr;
  AMG_TRY(pool_alloc((void **)&flags, sizeof(unsigned), st));
  // validation failures release the flag word before returning
  auto reject = [&](amg_status code, const char *msg) {
    pool_free(flags, st);
    return fail(code, msg);
  };
  AMG_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(unsigned), st));
  k_check_rowptr<<<blocks_for(n64 + 1, 256), 256, 0, st>>>(n64, rowptr, flags);
  LAUNCH_CHECK(&h->launches);
  unsigned hf = 0;
  int64_t nnz = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr + n64, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (hf & F_ROWPTR) return reject(AMG_ERR_INVALID_ARG, "row_ptr must start at 0 and be non-decreasing");
  if (nnz > 0 && (!col || !w)) return reject(AMG_ERR_INVALID_ARG, "col_idx and w must be non-NULL");
  // with row_ptr valid, the entry checks, the symmetry check (which skips
  // out-of-range columns) and the largest |d_i| run together; the flags are
  // then reported in the documented order
  unsigned long long *mx = nullptr;
  if (d) {
    AMG_TRY(pool_alloc((void **)&mx, sizeof(unsigned long long), st));
    AMG_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st));
  }
  k_check_entries<<<nb, 256, 0, st>>>(n, rowptr, col, w, d, flags);
  LAUNCH_CHECK(&h->launches);
  k_check_symmetry<<<nb, 256, 0, st>>>(n, rowptr, col, w, flags);
  LAUNCH_CHECK(&h->launches);
  if (d) {
    k_max_abs<<<nb, 256, 0, st>>>(n, d, mx);
    LAUNCH_CHECK(&h->launches);
  }
  unsigned long long hm = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  if (d) AMG_CUDA_TRY(cudaMemcpyAsync(&hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  pool_free(mx, st);
  if (hf & (F_RANGE | F_ORDER))
    return reject(AMG_ERR_INVALID_ARG, "column index out of range or row not strictly increasing");
  if (hf & F_SELF) return reject(AMG_ERR_SELF_LOOP, "graph has a self loop");
  if (hf & F_SYM) return reject(AMG_ERR_NOT_SYMMETRIC, "graph is not symmetric (pattern or weights)");
  if (hf & F_W) return reject(AMG_ERR_BAD_WEIGHT, "edge weights must be finite and > 0");
  if (hf & F_D) return reject(AMG_ERR_BAD_WEIGHT, "lower-order terms must be finite and >= 0");
  pool_free(flags, st);
  // pure Laplacian?  (d NULL or all zero)
  h->pure = !d || hm == 0ULL;
  phase.next("amg_setup: connectivity");
  // ---- connectivity ----
  {
    int *parent = nullptr, *changed = nullptr, *posd = nullptr, *cnt = nullptr;
    AMG_TRY(pool_alloc((void **)&parent, sizeof(int) * (size_t)n, st));
    AMG_TRY(pool_alloc((void **)&posd, sizeof(int) * (size_t)n, st));
    AMG_TRY(pool_alloc((void **)&changed, sizeof(int) * kCcBatch, st));
    AMG_TRY(pool_alloc((void **)&cnt, sizeof(int) * 2, st));
    k_cc_init<<<nb, 256, 0, st>>>(n, parent);
    LAUNCH_CHECK(&h->launches);
    // hook + jump rounds in batches between host checks: once a round hooks
    // nothing the forest is final and later rounds of the batch change nothing
    for (int it = 0;; it += kCcBatch) {
      int hc[kCcBatch] = {};
      AMG_CUDA_TRY(cudaMemsetAsync(changed, 0, sizeof(int) * kCcBatch, st));
      for (int b = 0; b < kCcBatch; ++b) {
        k_cc_hook<<<nb, 256, 0, st>>>(n, rowptr, col, parent, changed + b);
        LAUNCH_CHECK(&h->launches);
        k_cc_jump<<<nb, 256, 0, st>>>(n, parent);
        LAUNCH_CHECK(&h->launches);
      }
      AMG_CUDA_TRY(cudaMemcpyAsync(hc, changed, sizeof(int) * kCcBatch, cudaMemcpyDeviceToHost, st));
      AMG_CUDA_TRY(cudaStreamSynchronize(st));
      bool done = false;
      for (int b = 0; b < kCcBatch; ++b) done |= (hc[b] == 0);
      if (done) break;
      if (it > 64 + n) return fail(AMG_ERR_CUDA, "connectivity check did not converge");
    }
    AMG_CUDA_TRY(cudaMemsetAsync(posd, 0, sizeof(int) * (size_t)n, st));
    AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * 2, st));
    if (d) {
      k_cc_mark<<<nb, 256, 0, st>>>(n, parent, d, posd);
      LAUNCH_CHECK(&h->launches);
    }
    k_cc_count<<<nb, 256, 0, st>>>(n, parent, posd, h->pure ? 1 : 0, cnt);
    LAUNCH_CHECK(&h->launches);
    int hc[2] = {0, 0};
    AMG_CUDA_TRY(cudaMemcpyAsync(hc, cnt, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    pool_free(parent, st);
    pool_free(posd, st);
    pool_free(changed, st);
    pool_free(cnt, st);
    if (h->pure && hc[0] > 1) return fail(AMG_ERR_DISCONNECTED, "pure graph Laplacian of a disconnected graph");
    if (!h->pure && hc[1] > 0)
      return fail(AMG_ERR_DISCONNECTED, "a connected component has no positive lower-order term");
  }
  // ---- level 0 ----
  h->lv.clear();
  h->lv.emplace_back();
  {
    amg::Level &L0 = h->lv[0];
    L0.n = n;
    L0.A.n = n;
    L0.A.nnz = nnz;
    AMG_TRY(alloc_persist(h, (void **)&L0.A.rowptr, sizeof(int64_t) * (size_t)(n + 1)));
    AMG_TRY(alloc_persist(h, (void **)&L0.A.col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)));
    AMG_TRY(alloc_persist(h, (void **)&L0.A.val, sizeof(double) * (size_t)std::max<int64_t>(nnz, 1)));
    AMG_TRY(alloc_persist(h, (void **)&L0.diag, sizeof(double) * (size_t)n));
    AMG_TRY(alloc_persist(h, (void **)&L0.dlow, sizeof(double) * (size_t)n));
    AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1),
                                 cudaMemcpyDeviceToDevice, st));
    if (nnz)
      AMG_CUDA_TRY(cudaMemcpyAsync(L0.A.col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
    k_assemble<<<nb, 256, 0, st>>>(n, rowptr, w, d, L0.A.val, L0.diag, L0.dlow);
    LAUNCH_CHECK(&h->launches);
  }
  phase.next("amg_setup: coarsening (matching/independent sets + Galerkin)");
  // ---- coarsening ----
  const bool mis = h->opt.aggregation == AMG_AGG_MIS;
  const int passes = mis ? 1 : h->opt.passes;
  while (h->lv.back().n > h->opt.coarse_max && (int)h->lv.size() < h->opt.max_levels) {
    const NvtxRange level_range("amg_setup: one coarser level");
    const int k = (int)h->lv.size() - 1;
    const int nk = h->lv[k].n;
    LevelBuild cur;
    cur.A = h->lv[k].A;
    cur.diag = h->lv[k].diag;
    cur.dlow = h->lv[k].dlow;
    bool owned = false;
    int *comp = nullptr;
    AMG_TRY(pool_alloc((void **)&comp, sizeof(int) * (size_t)nk, st));
    int nH = nk;
    for (int p = 0; p < passes; ++p) {
      int *aggp = nullptr;
      AMG_TRY(pool_alloc((void **)&aggp, sizeof(int) * (size_t)std::max(cur.A.n, 1), st));
      LevelBuild next;
      if (mis) AMG_TRY(coarsen_mis_pass(h, cur, next, aggp, &nH));
      else AMG_TRY(coarsen_pass(h, cur, next, aggp, &nH));
      if (p == 0) {
        AMG_CUDA_TRY(cudaMemcpyAsync(comp, aggp, sizeof(int) * (size_t)nk, cudaMemcpyDeviceToDevice, st));
      } else {
        k_compose<<<blocks_for(nk, 256), 256, 0, st>>>(nk, comp, aggp);
        LAUNCH_CHECK(&h->launches);
      }
      pool_free(aggp, st);
      if (owned) free_build(cur, st);
      cur = next;
      owned = true;
    }
    if ((double)nH > kStallRatio * (double)nk) {
      free_build(cur, st);
      pool_free(comp, st);
      if (nk > kStallMaxCoarse) return fail(AMG_ERR_SETUP_STALL, "matching cannot coarsen a large level");
      break;
    }
    amg::Level &Lk = h->lv[k];
    Lk.nH = nH;
    AMG_TRY(alloc_persist(h, (void **)&Lk.agg, sizeof(int) * (size_t)nk));
    AMG_CUDA_TRY(cudaMemcpyAsync(Lk.agg, comp, sizeof(int) * (size_t)nk, cudaMemcpyDeviceToDevice, st));
    pool_free(comp, st);
    AMG_TRY(build_agg_lists(h, h->lv[k]));
    // the passes carried an upper bound of the entry count; the exact one is
    // read once per level
    {
      int64_t nnz_exact = 0;
      AMG_CUDA_TRY(cudaMemcpyAsync(&nnz_exact, cur.A.rowptr + cur.A.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      AMG_CUDA_TRY(cudaStreamSynchronize(st));
      cur.A.nnz = nnz_exact;
    }
    amg::Level nl;
    AMG_TRY(persist_level(h, cur, nl));
    free_build(cur, st);
    h->lv.push_back(nl);
  }
  h->L = (int)h->lv.size();
  phase.next("amg_setup: smoother intervals and coefficients");
  // ---- smoother interval and polynomial per level (Sec. 3, Sec. 4) ----
  {
    // ||A_k||_inf of every smoothing level, then one read-back
    const int nl = std::max(h->L - 1, 0);
    unsigned long long *nrm = nullptr;
    AMG_TRY(pool_alloc((void **)&nrm, sizeof(unsigned long long) * (size_t)std::max(nl, 1), st));
    AMG_CUDA_TRY(cudaMemsetAsync(nrm, 0, sizeof(unsigned long long) * (size_t)std::max(nl, 1), st));
    for (int k = 0; k < nl; ++k) {
      amg::Level &L = h->lv[k];
      k_norm_inf<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.A.rowptr, L.A.val, L.diag, nrm + k);
      LAUNCH_CHECK(&h->launches);
    }
    std::vector<unsigned long long> bits((size_t)std::max(nl, 1), 0);
    AMG_CUDA_TRY(cudaMemcpyAsync(bits.data(), nrm, sizeof(unsigned long long) * (size_t)std::max(nl, 1),
                                 cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    pool_free(nrm, st);
    for (int k = 0; k < nl; ++k) {
      amg::Level &L = h->lv[k];
      double l1;
      memcpy(&l1, &bits[k], sizeof(double));
      L.lam1 = l1;
      L.lam0 = h->opt.lambda0_ratio * l1;
      closed_form_coefficients(h->opt.degree, L.lam0, L.lam1, L.coef);
    }
  }
  if (h->opt.cycle == AMG_CYCLE_AMLI) {
    // the AMLI polynomial: best approximation of degree nu-1 to 1/t on
    // [alpha, 1], divided by 1 + E (E its error bound) so that 0 < t q(t) <= 1
    const int dg = h->opt.inner_iters - 1;
    const double al = h->opt.amli_alpha, kappa = 1.0 / al;
    const double delta = (sqrt(kappa) - 1.0) / (sqrt(kappa) + 1.0);
    const double E = pow(delta, (double)dg) * (kappa - 1.0) / 2.0;
    closed_form_coefficients(dg, al, 1.0, h->amli_coef);
    for (int p = 0; p <= dg; ++p) h->amli_coef[p] /= 1.0 + E;
    h->amli_sA = 2.0 / (1.0 - al);
    h->amli_sB = (1.0 + al) / (1.0 - al);
  }
  phase.next("amg_setup: solve layouts (SELL-32)");
  // ---- solve layouts ----
  const bool want32 = h->opt.precision == AMG_PREC_FP32;
  AMG_TRY(build_sell_all(h, want32));
  phase.next("amg_setup: coarsest pseudo-inverse");
  AMG_TRY(build_coarsest(h));
  // complexities (Sec. 4)
  double gs = 0, os = 0;
  for (auto &L : h->lv) {
    gs += L.n;
    os += (double)(L.A.nnz + L.n);
  }
  h->grid_complexity = gs / (double)n;
  h->op_complexity = os / (double)(h->lv[0].A.nnz + n);
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  return AMG_OK;
}


}  // namespace amg
