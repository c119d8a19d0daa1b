// common.cuh -- internal declarations of the GB300 aggregation-AMG library.
//
// Data layout in HBM (one handle = one hierarchy):
//   level k setup form : CSR of the off-diagonal entries (int64 row offsets,
//                        int32 columns, fp64 values a_ij = -W_ij), fp64
//                        diagonal and aggregated lower-order term.
//   level k solve form : SELL-32 (slices of 32 consecutive rows = one warp,
//                        column-major inside a slice, padded to the slice's
//                        longest row) of the off-diagonal part plus a separate
//                        diagonal, in fp64 and, in fp32 mode, fp32.
//   transfers          : agg[n_k] (coarse id per vertex) for prolongation and
//                        the CSR of aggregates (agg_ptr, members ascending) for
//                        restriction; no floating-point atomics anywhere.
//   coarsest level     : dense fp64 pseudo-inverse Z (n_c x n_c, row major).
//   scalars            : per-level fp64 arrays on the device; the host never
//                        reads them inside a cycle.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "amg.h"

namespace amg {

constexpr int kSlice = 32;        // SELL slice height (warp width)
constexpr int kMaxDegree = 16;    // largest smoother degree
constexpr int kMaxInner = 8;      // largest nu
constexpr int kMaxWindow = 16;    // largest outer restart window
constexpr int kMaxDots = 8;       // dots per fused reduction
constexpr int kRedBlocks = 608;   // smallest partials buffer of a reduction = 4 x 152 SMs
constexpr int kRedElems = 4;      // elements per thread of a streaming reduction
constexpr int kMaxBatchServe = 32; // largest server batch (the widest block)
constexpr int kStallMaxCoarse = 4096;
constexpr double kStallRatio = 0.95;
// largest vertex count: the one-thread-per-row kernels index rows in 32-bit
// integers over grids rounded up to whole blocks, so every thread index of a
// launch must stay below 2^31
constexpr int64_t kMaxRows = (int64_t(1) << 31) - (int64_t(1) << 16);

// ---------------------------------------------------------------------------
// error plumbing: status + message, no exceptions across the C ABI
// ---------------------------------------------------------------------------
struct Error {
  amg_status code = AMG_OK;
  std::string msg;
};

#define AMG_CUDA_TRY(expr)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      return ::amg::fail(e_ == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA, \
                         std::string(#expr) + ": " + cudaGetErrorString(e_));          \
    }                                                                                  \
  } while (0)

#define AMG_TRY(expr)                  \
  do {                                 \
    amg_status s_ = (expr);            \
    if (s_ != AMG_OK) return s_;       \
  } while (0)

amg_status fail(amg_status code, const std::string &msg);  // records thread-local error
const std::string &thread_error();

// NVTX range over a host-side phase (setup steps, outer iterations); a no-op
// unless a profiler that collects NVTX is attached
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
// consecutive phases of one function: next() closes the open range and opens
// the next one; the destructor closes the last.  With AMG_GB300_SETUP_PROFILE=1
// the stream given at construction is synchronised at every phase boundary
// and each phase's wall time is printed to stderr (diagnostics only: the
// synchronisations change the timing they measure by a little).
struct NvtxPhase {
  bool open = false;
  bool timed = false;
  cudaStream_t st = nullptr;
  const char *cur = nullptr;
  double t0 = 0.0;
  explicit NvtxPhase(cudaStream_t s = nullptr);
  void next(const char *name);
  ~NvtxPhase();
};

// ---------------------------------------------------------------------------
// device memory: one library-owned stream-ordered pool per device
// ---------------------------------------------------------------------------
struct Arena {
  cudaStream_t stream = nullptr;
  std::vector<void *> blocks;
  std::vector<size_t> sizes;
  size_t bytes = 0;
  amg_status alloc(void **p, size_t bytes);
  void free_block(void *p);  // stream-ordered release of one block
  template <typename T>
  amg_status get(T **p, size_t count) {
    return alloc(reinterpret_cast<void **>(p), count * sizeof(T));
  }
  void release();  // frees every block (stream ordered) and synchronises
};
amg_status pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);

// ---------------------------------------------------------------------------
// matrices
// ---------------------------------------------------------------------------
struct Csr {  // off-diagonal part; diagonal kept separately
  int n = 0;
  int64_t nnz = 0;
  int64_t *rowptr = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
};

struct Sell {  // SELL-32 off-diagonal part + diagonal
  int n = 0;
  int nslices = 0;
  int64_t stored = 0;  // padded entries
  int64_t *sptr = nullptr;
  int32_t *scol = nullptr;
  // the same columns as 16-bit offsets j - i from the row, on levels where
  // every stored |j - i| fits (banded numberings): 2 bytes per entry less in
  // the solve kernels; null elsewhere
  int16_t *sdel = nullptr;
  double *val64 = nullptr;
  float *val32 = nullptr;
  double *diag64 = nullptr;
  float *diag32 = nullptr;
  // the smoother's operator 2 t(A) = 2 sa A - 2 ca I on the same pattern:
  // off-diagonal values times 2 sa, diagonal 2 sa a_ii - 2 ca
  double *sval64 = nullptr, *sdiag64 = nullptr;
  float *sval32 = nullptr, *sdiag32 = nullptr;
};

template <typename T>
struct SellView {
  int n;
  const int64_t *__restrict__ sptr;
  const int32_t *__restrict__ scol;
  const T *__restrict__ val;
  const T *__restrict__ diag;
  // 1: the stored values and columns are read with the streaming
  // (evict-first) cache policy -- levels whose matrix is far larger than L2,
  // so that one pass over it does not evict the vectors and the smaller
  // levels' working sets
  int stream = 0;
  // columns as offsets from the row (Sell::sdel), or null: read scol
  const int16_t *__restrict__ sdel = nullptr;
};

struct Level {
  int n = 0;
  int wps = 1;           // warps per SELL slice in the solve kernels (1, 2, 4 or 8)
  int stream = 0;        // matrix loads with the streaming cache policy (SellView::stream)
  Csr A;                 // setup form
  double *diag = nullptr;
  double *dlow = nullptr;
  Sell S;                // solve form
  // map to the next level
  int nH = 0;
  int32_t *agg = nullptr;
  int32_t *agg_ptr = nullptr;
  int32_t *agg_mem = nullptr;
  // matching hierarchies: the members again as a fixed-width table, column
  // major ([memw_width][nH], ascending, -1 after the last), for the restriction
  int32_t *memw = nullptr;
  int memw_width = 0;
  // smoother: q_m on [lam0, lam1] in the Chebyshev basis of t(x)
  double lam0 = 0, lam1 = 0;
  double coef[kMaxDegree + 1] = {};
  // per-level device scalars and work vectors (element type = cycle precision)
  double *scal = nullptr;  // [64]
  void *u = nullptr, *s = nullptr, *Ta = nullptr, *Tb = nullptr;  // cycle scratch
  void *b = nullptr, *x = nullptr, *r = nullptr;    // inner flexible CG
  void *D[kMaxInner] = {}, *W[kMaxInner] = {};
};

// per-level buffers of the batched (multi right-hand side) path: blocks of
// up to 32 columns, row major
struct BatchLevel {
  double *scal = nullptr;  // [48][32] per-column scalars
  void *u = nullptr, *s = nullptr, *Ta = nullptr, *Tb = nullptr;
  void *b = nullptr, *x = nullptr, *r = nullptr;
  void *D[kMaxInner] = {}, *W[kMaxInner] = {};
};

// fused reduction state (deterministic two-stage: per-block partials, last
// block folds them in block order)
struct RedState {
  double *partial = nullptr;   // [kRedBlocks * kMaxDots]
  unsigned int *ticket = nullptr;
};

// CUDA-event timing of chosen level-0 launches (amg_kernel_timing): kind 0
// the fused smoother step, 1 the restriction, 2 the prolongation
constexpr int kTimedKinds = 3;
struct Timing {
  bool enabled = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> kind;        // kind of each pair (indexed by pair)
  size_t used = 0;
  int64_t launches[kTimedKinds] = {};
  double total_ms[kTimedKinds] = {};
};

struct Options {
  amg_options o;
};

}  // namespace amg

struct amg_handle_s {
  amg_options opt{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0;
  bool pure = false;
  int L = 0;
  std::vector<amg::Level> lv;
  amg::Arena arena;
  amg::RedState red;
  // coarsest pseudo-inverse
  int nc = 0;
  double *Z = nullptr;
  // outer flexible CG (fp64) on level 0
  double *ob = nullptr, *ox = nullptr, *or_ = nullptr, *oz = nullptr;
  double *oD[amg::kMaxWindow] = {}, *oQ[amg::kMaxWindow] = {};
  double *oscal = nullptr;   // [256]
  double *h_pinned = nullptr;  // host mirror of a few scalars
  // fp32 mode: level-0 fp32 buffers for the preconditioner input/output
  float *r32 = nullptr, *z32 = nullptr;
  // coarsest conversion buffers (fp32 mode)
  double *cb64 = nullptr, *cx64 = nullptr;
  // level Bk = L-2 applied as one dense operator (fp64, row major), or Bk = -1
  int Bk = -1;
  double *Bd = nullptr;
  double *bb64 = nullptr, *bx64 = nullptr;
  // stationary AMLI cycle: Chebyshev coefficients of q = q_{nu-1}/(1+E) on
  // [alpha, 1] and tau(t) = sA t - sB, sA = 2/(1-alpha), sB = (1+alpha)/(1-alpha)
  double amli_coef[amg::kMaxInner] = {};
  double amli_sA = 0.0, amli_sB = 0.0;
  // the inner solve at level leaf_k (= Bk - 1) as one cluster kernel whose
  // vectors live in shared memory (leaf.cu); -1: multi-kernel path
  int leaf_k = -1;
  int leaf_csize = 0;
  void *leaf_params = nullptr;             // host copy of the launch parameters
  void (*leaf_free)(void *) = nullptr;
  unsigned long long *leaf_prof = nullptr;  // opt-in phase profile of the leaf kernel
  // batched path (batch.cu)
  int bw = 0;                        // allocated block width (0: not yet)
  int bw_use = 32;                   // block width in use
  int b_tile = 256;                  // threads per CTA of the block SpMM kernels
  int tuned_for = 0;
  std::string tune_log;
  std::vector<amg::BatchLevel> blv;
  std::vector<void *> batch_blocks;  // arena blocks of the batched path (for re-allocation)
  double *bo_b = nullptr, *bo_x = nullptr, *bo_r = nullptr, *bo_z = nullptr, *bo_t = nullptr;
  double *boD[amg::kMaxWindow] = {}, *boQ[amg::kMaxWindow] = {};
  double *bo_scal = nullptr;
  void *b_r32 = nullptr, *b_z32 = nullptr;
  double *b_partial = nullptr;
  unsigned *b_ticket = nullptr;
  double *b_pinned = nullptr;
  cudaGraphExec_t bpre_exec = nullptr;
  bool bpre_borrowed = false;        // bpre_exec belongs to bfixed[]
  cudaGraphExec_t bfixed[6] = {};    // fixed-width block preconditioners, width 2^slot
  int64_t bfixed_kernels[6] = {};
  int64_t bgraph_kernels = 0;
  double setup_ms = 0;
  int match_rounds_hint = 0;         // rounds of the last matching pass (setup)
  double grid_complexity = 0, op_complexity = 0;
  int64_t launches = 0;
  amg::Timing timing;
  // the preconditioner application z = K_0(r) on (or_, oz) captured once as a
  // CUDA graph and replayed every outer iteration
  bool use_graph = true;
  bool use_pdl = true;              // programmatic dependent launch of solve kernels
  bool prolong_split = true;        // streaming prolongation + residual on large levels
  bool capturing = false;
  cudaStream_t cap = nullptr;       // private stream used only for capture
  cudaGraphExec_t pre_exec = nullptr;
  bool graph_timed = false;         // graph holds timing event-record nodes
  size_t graph_events = 0;          // timing events recorded by one replay
  int64_t graph_kernels = 0;        // kernel nodes per replay
  std::string err;
};

namespace amg {
// setup.cu
amg_status build_hierarchy(amg_handle_s *h, int64_t n, const int64_t *rowptr, const int32_t *col,
                           const double *w, const double *d);
amg_status match_pass(cudaStream_t st, int n, const int64_t *rowptr, const int32_t *col,
                      const double *s, uint64_t salt, int32_t *mate, int32_t *agg, int *nH,
                      int *rounds, int64_t *launches);
// solve.cu
amg_status allocate_solve_buffers(amg_handle_s *h);
amg_status build_dense_two_level(amg_handle_s *h);
// batch.cu
// outcome of one column of a multi-right-hand-side solve
struct ColumnReport {
  int iterations = 0;  // outer iterations until the column met tol (or stopped)
  double rel_residual = 0.0, true_rel_residual = 0.0;
  bool converged = false, breakdown = false;
};
// nrhs right-hand sides (device, column major with ld) in blocks of the
// autotuned width, or of `fixed_width` (1..32, a power of two) when > 0;
// `cols` (optional, nrhs entries) receives each column's outcome
amg_status solve_batched(amg_handle_s *h, const double *rhs, double *x, int nrhs, int64_t ld, double tol,
                         amg_info *info, int *iters, double *rel, double *true_rel, int *conv, bool *breakdown,
                         int fixed_width = 0, ColumnReport *cols = nullptr);
amg_status prepare_batched(amg_handle_s *h, int width);
void release_block_graphs(amg_handle_s *h);
// capi.cu: the server's batched solve: host columns in and out, staged
// through device buffers of the handle's pool
amg_status solve_host_columns(amg_handle_s *h, const double *const *rhs, double *const *x, int nr, double tol,
                              int width, ColumnReport *cols);
// leaf.cu
amg_status prepare_leaf(amg_handle_s *h);
void report_leaf_profile(amg_handle_s *h);
amg_status launch_leaf(amg_handle_s *h);
amg_status solve_one(amg_handle_s *h, const double *b_dev, double *x_dev, double tol,
                     amg_info *info, int *iters, double *rel, double *true_rel, int *converged);
amg_status apply_spmv(amg_handle_s *h, int k, const double *x, double *y);
amg_status apply_smoother(amg_handle_s *h, int k, const double *r, double *x);
amg_status apply_restrict(amg_handle_s *h, int k, const double *s, double *rH);
amg_status apply_prolong_add(amg_handle_s *h, int k, const double *eH, double *x);
amg_status apply_coarse_solve(amg_handle_s *h, const double *b, double *x);
amg_status apply_kcycle(amg_handle_s *h, int k, const double *r, double *z);
// scan.cu helpers (in setup.cu)
amg_status exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st,
                              int64_t *total_host);
amg_status exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t st,
                              int64_t *total_host);
}  // namespace amg
