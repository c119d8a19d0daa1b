// match_noalloc.cu -- amg_match_noalloc: the handshake matching pass of
// amg_match with all of its scratch in a fixed, file-scope device array, so
// that the call never allocates device memory.
//
// Who needs this: callers whose device memory is owned by someone else and
// who therefore may not call cudaMalloc/cudaFree (or any allocating library
// routine) themselves -- for example code running under a framework's
// caching allocator that has claimed the GPU's free memory, or a pipeline
// that cannot afford the implicit device-wide synchronisation cudaFree
// performs.  They pass the inputs and outputs; everything else comes from
// g_match_scratch below.
//
// Cost of the design: every GPU that loads this library keeps the array
// (kMaxN + 1024 ints, about 4 MiB) until the process exits.  Each process
// holds its own copy, so only calls made by one process share it: calls from
// different streams or threads of one process that overlap on the GPU race
// and must be serialised by the caller.
#include "common.cuh"

namespace amg {

// kernels of the matching pass (defined in setup.cu)
__global__ void k_match_init(int n, int *mate);
__global__ void k_propose(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          const double *__restrict__ s, uint64_t salt, const int *__restrict__ mate,
                          int *__restrict__ ptr, const int *prev);
__global__ void k_accept(int n, const int *__restrict__ ptr, int *__restrict__ mate, int *added,
                         const int *prev);
__global__ void k_rep_flags(int n, const int *__restrict__ mate, int *__restrict__ rep);
__global__ void k_coarse_ids(int n, const int *__restrict__ mate, const int *__restrict__ id,
                             int *__restrict__ agg, int *__restrict__ m0, int *__restrict__ m1);

namespace {

constexpr int kMaxN = 1 << 20;              // largest graph accepted (vertices)
constexpr int kTile = 2048;                 // scan elements per block
constexpr int kMaxTiles = kMaxN / kTile;    // 512 block sums
constexpr int kBatch = 2;                   // proposal rounds between host checks
// layout (ints): [0, kMaxN) per-vertex work (proposals during the rounds,
// then representative flags scanned in place into coarse ids);
// [kMaxN, kMaxN + kMaxTiles) block sums; then kBatch round counters and the
// scan total
constexpr int kSums = kMaxN;
constexpr int kAdded = kMaxN + kMaxTiles;
constexpr int kTotal = kAdded + kBatch;
constexpr int kScratchInts = kMaxN + 1024;

static __device__ __align__(256) int g_match_scratch[kScratchInts];

// Device address of g_match_scratch in the current device's context.  Looked
// up on every call (a host-side lookup that allocates nothing): a cached
// address would dangle after cudaDeviceReset recreates the context, and would
// belong to the wrong context if the caller switches contexts on one device.
amg_status scratch_address(int **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_match_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, std::string("cudaGetSymbolAddress(g_match_scratch): ") + cudaGetErrorString(e));
  }
  *out = static_cast<int *>(p);
  return AMG_OK;
}

// in-place exclusive scan of a[0, n), n <= kMaxN, in two levels
__global__ void k_tile_scan(int *a, int n, int *sums) {
  __shared__ int wtot[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = blockIdx.x * kTile + threadIdx.x * 8;
  int v[8], local = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0;
    local += v[k];
  }
  int inc = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wtot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int t = lane < 8 ? wtot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < 8) wtot[lane] = t;
  }
  __syncthreads();
  int run = inc - local + (warp > 0 ? wtot[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (base + k < n) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 255) sums[blockIdx.x] = wtot[7];
}

// one block of kMaxTiles threads: exclusive scan of the block sums, total
__global__ void k_sums_scan(int *sums, int nb, int *total) {
  __shared__ int sh[kMaxTiles];
  const int t = threadIdx.x;
  sh[t] = t < nb ? sums[t] : 0;
  __syncthreads();
  for (int o = 1; o < kMaxTiles; o <<= 1) {
    int u = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += u;
    __syncthreads();
  }
  if (t < nb) sums[t] = sh[t] - (t < nb ? sums[t] : 0);
  if (t == kMaxTiles - 1) *total = sh[t];
}

__global__ void k_sums_add(int *a, int n, const int *sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += sums[i / kTile];
}

}  // namespace
}  // namespace amg

using namespace amg;

extern "C" amg_status amg_match_noalloc(int64_t n64, const int64_t *row_ptr, const int32_t *col_idx,
                                        const double *s, uint64_t salt, int32_t *mate, int32_t *agg,
                                        int64_t *n_coarse, int *rounds, void *cuda_stream) {
  if (n64 < 1 || !row_ptr || !mate || !agg)
    return fail(AMG_ERR_INVALID_ARG, "n, row_ptr, mate or agg invalid");
  if (!col_idx || !s) return fail(AMG_ERR_INVALID_ARG, "col_idx and s must be non-NULL");
  if (n64 > kMaxN)
    return fail(AMG_ERR_INVALID_ARG, "amg_match_noalloc: n = " + std::to_string(n64) +
                                         " exceeds the fixed scratch capacity of " + std::to_string(kMaxN) +
                                         " vertices; use amg_match");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, "no usable CUDA device");
  }
  int *scr = nullptr;
  AMG_TRY(scratch_address(&scr));
  const int n = (int)n64;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const unsigned nb = (unsigned)((n + 255) / 256);
  int *work = scr, *sums = scr + kSums, *added = scr + kAdded, *total = scr + kTotal;
  k_match_init<<<nb, 256, 0, st>>>(n, mate);
  int r = 0;
  int h_added[kBatch];
  for (;;) {
    AMG_CUDA_TRY(cudaMemsetAsync(added, 0, sizeof(int) * kBatch, st));  // counters start at zero
    for (int b = 0; b < kBatch; ++b) {
      // a round after one that added no pair returns at once on the device
      const int *prev = b ? added + b - 1 : nullptr;
      k_propose<<<nb, 256, 0, st>>>(n, row_ptr, col_idx, s, salt, mate, work, prev);
      k_accept<<<nb, 256, 0, st>>>(n, work, mate, added + b, prev);
    }
    AMG_CUDA_TRY(cudaGetLastError());
    AMG_CUDA_TRY(cudaMemcpyAsync(h_added, added, sizeof(int) * kBatch, cudaMemcpyDeviceToHost, st));
    AMG_CUDA_TRY(cudaStreamSynchronize(st));
    bool done = false;
    for (int b = 0; b < kBatch && !done; ++b) {
      ++r;
      done = (h_added[b] == 0);
    }
    if (done) break;
    if (r > 4 * n + 8)
      return fail(AMG_ERR_INVALID_ARG, "matching did not terminate: s must be symmetric and finite");
  }
  // representative flags -> coarse ids (in place) -> aggregate ids
  const int tiles = (n + kTile - 1) / kTile;
  k_rep_flags<<<nb, 256, 0, st>>>(n, mate, work);
  k_tile_scan<<<tiles, 256, 0, st>>>(work, n, sums);
  k_sums_scan<<<1, kMaxTiles, 0, st>>>(sums, tiles, total);
  k_sums_add<<<nb, 256, 0, st>>>(work, n, sums);
  k_coarse_ids<<<nb, 256, 0, st>>>(n, mate, work, agg, nullptr, nullptr);
  AMG_CUDA_TRY(cudaGetLastError());
  int nH = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&nH, total, sizeof(int), cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_coarse) *n_coarse = nH;
  if (rounds) *rounds = r;
  return AMG_OK;
}
