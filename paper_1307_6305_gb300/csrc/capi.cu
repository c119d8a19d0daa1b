// capi.cu -- the C ABI declared in include/amg.h: argument checks, handle
// lifecycle, host/device staging, introspection and measurement hooks.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>

#include <math.h>

#include "common.cuh"

namespace amg {

static thread_local std::string t_err;

amg_status fail(amg_status code, const std::string &msg) {
  t_err = msg;
  return code;
}
const std::string &thread_error() { return t_err; }

static double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

NvtxPhase::NvtxPhase(cudaStream_t s) : st(s) {
  const char *e = getenv("AMG_GB300_SETUP_PROFILE");
  timed = e && e[0] == '1';
  if (timed) {
    cudaStreamSynchronize(st);
    t0 = wall_ms();
  }
}

void NvtxPhase::next(const char *name) {
  if (timed) {
    cudaStreamSynchronize(st);
    const double t = wall_ms();
    if (cur) fprintf(stderr, "setup phase %-62s %8.3f ms\n", cur, t - t0);
    t0 = t;
    cur = name;
  }
  if (open) nvtxRangePop();
  nvtxRangePushA(name);
  open = true;
}

NvtxPhase::~NvtxPhase() {
  if (timed && cur) {
    cudaStreamSynchronize(st);
    fprintf(stderr, "setup phase %-62s %8.3f ms\n", cur, wall_ms() - t0);
  }
  if (open) nvtxRangePop();
}

// one library-owned stream-ordered pool per device; memory is kept in the
// pool between setups (release threshold = max) so repeated setup/free
// cycles do not go back to the driver
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[128];
static bool g_pool_ok[128];

static amg_status device_pool(cudaMemPool_t *out) {
  int dev = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(AMG_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_ok[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    AMG_CUDA_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
    uint64_t thr = UINT64_MAX;
    AMG_CUDA_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool_ok[dev] = true;
  }
  *out = g_pool[dev];
  return AMG_OK;
}

// Injected allocation failure, for testing the error paths of the setup
// without a real out-of-memory condition: amg_setup arms the calling thread's
// countdown from AMG_GB300_FAIL_ALLOC=k (k >= 1) and disarms it on return;
// while armed, the k-th device allocation of the setup fails as if the pool
// were exhausted.  Nothing is injected on the device.
static thread_local int64_t t_alloc_countdown = 0;

struct AllocFailArm {
  AllocFailArm() {
    const char *e = getenv("AMG_GB300_FAIL_ALLOC");
    t_alloc_countdown = e ? std::max<long long>(0, atoll(e)) : 0;
  }
  ~AllocFailArm() { t_alloc_countdown = 0; }
};

amg_status pool_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (t_alloc_countdown > 0 && --t_alloc_countdown == 0)
    return fail(AMG_ERR_OOM, "injected allocation failure (AMG_GB300_FAIL_ALLOC) of " + std::to_string(bytes) +
                                 " bytes");
  cudaMemPool_t pool;
  AMG_TRY(device_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA,
                std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  return AMG_OK;
}

void pool_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

amg_status Arena::alloc(void **p, size_t nbytes) {
  AMG_TRY(pool_alloc(p, nbytes, stream));
  blocks.push_back(*p);
  sizes.push_back(nbytes);
  bytes += nbytes;
  return AMG_OK;
}

void Arena::free_block(void *p) {
  for (size_t i = 0; i < blocks.size(); ++i) {
    if (blocks[i] != p) continue;
    pool_free(p, stream);
    bytes -= sizes[i];
    blocks.erase(blocks.begin() + (ptrdiff_t)i);
    sizes.erase(sizes.begin() + (ptrdiff_t)i);
    return;
  }
}

void Arena::release() {
  for (void *p : blocks) pool_free(p, stream);
  blocks.clear();
  sizes.clear();
  bytes = 0;
  cudaStreamSynchronize(stream);
}

// The server's batched solve: nr host columns (n doubles each, one pointer
// per request) staged into one column-major device block, solved by the
// multi-right-hand-side path at the fixed block width `width`, and copied
// back column by column.  Runs on the handle's stream; returns after the
// copies have completed.
amg_status solve_host_columns(amg_handle_s *h, const double *const *rhs, double *const *x, int nr, double tol,
                              int width, ColumnReport *cols) {
  const int64_t n = h->n;
  const size_t col_bytes = sizeof(double) * (size_t)n, bytes = col_bytes * (size_t)nr;
  cudaStream_t st = h->stream;
  double *bd = nullptr, *xd = nullptr;
  AMG_TRY(pool_alloc((void **)&bd, bytes, st));
  amg_status s = pool_alloc((void **)&xd, bytes, st);
  for (int c = 0; c < nr && !s; ++c)
    if (cudaMemcpyAsync(bd + (size_t)c * n, rhs[c], col_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      s = fail(AMG_ERR_CUDA, "copy of a right-hand side");
  int it = 0, conv = 0;
  double rel = 0.0, tr = 0.0;
  bool brk = false;
  if (!s) s = solve_batched(h, bd, xd, nr, n, tol, nullptr, &it, &rel, &tr, &conv, &brk, width, cols);
  for (int c = 0; c < nr && !s; ++c)
    if (cudaMemcpyAsync(x[c], xd + (size_t)c * n, col_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      s = fail(AMG_ERR_CUDA, "copy of a solution");
  if (!s && cudaStreamSynchronize(st) != cudaSuccess) s = fail(AMG_ERR_CUDA, "batched solve");
  pool_free(bd, st);
  pool_free(xd, st);
  return s;
}

}  // namespace amg

using namespace amg;

namespace {

// error bound delta^m (kappa - 1)/2 of the best degree-m approximation to
// 1/t on [alpha, 1], kappa = 1/alpha (Sec. 3 with lambda1 = 1)
double amli_error(int m, double alpha) {
  const double kappa = 1.0 / alpha, delta = (sqrt(kappa) - 1.0) / (sqrt(kappa) + 1.0);
  return pow(delta, (double)m) * (kappa - 1.0) / 2.0;
}

amg_status check_options(const amg_options &o) {
  if (o.degree < 0 || o.degree > kMaxDegree) return fail(AMG_ERR_INVALID_ARG, "degree must be in [0, 16]");
  if (o.passes < 1 || o.passes > 16) return fail(AMG_ERR_INVALID_ARG, "passes must be in [1, 16]");
  if (o.coarse_max < 1 || o.coarse_max > kStallMaxCoarse)
    return fail(AMG_ERR_INVALID_ARG, "coarse_max must be in [1, 4096]");
  if (o.max_levels < 1 || o.max_levels > 64) return fail(AMG_ERR_INVALID_ARG, "max_levels must be in [1, 64]");
  if (o.inner_iters < 1 || o.inner_iters > kMaxInner) return fail(AMG_ERR_INVALID_ARG, "inner_iters must be in [1, 8]");
  if (o.restart < 1 || o.restart > kMaxWindow) return fail(AMG_ERR_INVALID_ARG, "restart must be in [1, 16]");
  if (o.max_iters < 0) return fail(AMG_ERR_INVALID_ARG, "max_iters must be >= 0");
  if (o.precision != AMG_PREC_FP64 && o.precision != AMG_PREC_FP32)
    return fail(AMG_ERR_INVALID_ARG, "precision must be AMG_PREC_FP64 or AMG_PREC_FP32");
  if (!(o.lambda0_ratio > 0.0 && o.lambda0_ratio < 1.0))
    return fail(AMG_ERR_INVALID_ARG, "lambda0_ratio must be in (0, 1)");
  if (o.aggregation != AMG_AGG_MATCHING && o.aggregation != AMG_AGG_MIS)
    return fail(AMG_ERR_INVALID_ARG, "aggregation must be AMG_AGG_MATCHING or AMG_AGG_MIS");
  if (o.mis_k < 1 || o.mis_k > 16) return fail(AMG_ERR_INVALID_ARG, "mis_k must be in [1, 16]");
  if (o.cycle != AMG_CYCLE_K && o.cycle != AMG_CYCLE_AMLI)
    return fail(AMG_ERR_INVALID_ARG, "cycle must be AMG_CYCLE_K or AMG_CYCLE_AMLI");
  if (!(o.rho >= 0.0) || !std::isfinite(o.rho)) return fail(AMG_ERR_INVALID_ARG, "rho must be >= 0");
  if (o.rho > 0.0 && amg_degree_for(o.rho, o.lambda0_ratio) < 0)
    return fail(AMG_ERR_INVALID_ARG, "no smoother degree <= 16 reaches the damping rho");
  if (o.cycle == AMG_CYCLE_AMLI) {
    if (!(o.amli_alpha > 0.0 && o.amli_alpha < 1.0))
      return fail(AMG_ERR_INVALID_ARG, "amli_alpha must be in (0, 1)");
    if (!(amli_error(o.inner_iters - 1, o.amli_alpha) < 1.0))
      return fail(AMG_ERR_INVALID_ARG,
                  "the AMLI polynomial's error on [amli_alpha, 1] is >= 1: raise amli_alpha or inner_iters");
  }
  return AMG_OK;
}

amg_status cuda_ready() {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    cudaGetLastError();
    return fail(AMG_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
  }
  return AMG_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

amg_status record(amg_handle_s *h, amg_status s) {
  if (s != AMG_OK && h) h->err = thread_error();
  return s;
}

void destroy(amg_handle_s *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  report_leaf_profile(h);
  h->arena.release();
  if (h->leaf_params && h->leaf_free) h->leaf_free(h->leaf_params);
  if (h->pre_exec) cudaGraphExecDestroy(h->pre_exec);
  release_block_graphs(h);
  if (h->b_pinned) cudaFreeHost(h->b_pinned);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (cudaEvent_t e : h->timing.ev) cudaEventDestroy(e);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // namespace

extern "C" {

void amg_default_options(amg_options *o) {
  if (!o) return;
  o->degree = 4;
  o->passes = 3;
  o->coarse_max = 64;
  o->max_levels = 30;
  o->inner_iters = 2;
  o->restart = 5;
  o->max_iters = 500;
  o->precision = AMG_PREC_FP64;
  o->lambda0_ratio = 0.1;
  o->hash_salt = 0;
  o->cycle = AMG_CYCLE_K;
  o->amli_alpha = 0.25;
  o->rho = 0.0;
  o->aggregation = AMG_AGG_MATCHING;
  o->mis_k = 4;
}

int amg_degree_for(double rho, double lambda0_ratio) {
  if (!(rho > 0.0) || !(lambda0_ratio > 0.0 && lambda0_ratio < 1.0)) return -1;
  const double kappa = 1.0 / lambda0_ratio, delta = (sqrt(kappa) - 1.0) / (sqrt(kappa) + 1.0);
  auto ok = [&](int m) {
    const double e = pow(delta, (double)m) * (kappa - 1.0) / 2.0;
    return e <= rho && e < 1.0;
  };
  // E_m <= min(rho, 1): m >= log(2 min(rho, 1) / (kappa - 1)) / log(delta);
  // then settle the rounding of the logarithms on the condition itself
  const double x = log(2.0 * std::min(rho, 1.0) / (kappa - 1.0)) / log(delta);
  int m = x > 0.0 ? (int)std::min(ceil(x), (double)kMaxDegree + 1) : 0;
  while (m > 0 && ok(m - 1)) --m;
  while (m <= kMaxDegree && !ok(m)) ++m;
  return m <= kMaxDegree ? m : -1;
}

amg_status amg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *w,
                     const double *d, const amg_options *opt, int mem_space, void *cuda_stream,
                     amg_handle *out) {
  if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > kMaxRows) return fail(AMG_ERR_INVALID_ARG, "n must be in [1, 2^31 - 2^16]");
  if (!row_ptr) return fail(AMG_ERR_INVALID_ARG, "row_ptr is NULL");
  if (mem_space != AMG_MEM_HOST && mem_space != AMG_MEM_DEVICE)
    return fail(AMG_ERR_INVALID_ARG, "mem_space must be AMG_MEM_HOST or AMG_MEM_DEVICE");
  amg_options o;
  if (opt) o = *opt; else amg_default_options(&o);
  AMG_TRY(check_options(o));
  if (o.rho > 0.0) o.degree = amg_degree_for(o.rho, o.lambda0_ratio);  // Eq. (bound-on-m)
  if (mem_space == AMG_MEM_HOST) {
    if (row_ptr[0] != 0 || row_ptr[n] < 0) return fail(AMG_ERR_INVALID_ARG, "row_ptr must start at 0 and be non-decreasing");
    if (row_ptr[n] > 0 && (!col_idx || !w)) return fail(AMG_ERR_INVALID_ARG, "col_idx and w must be non-NULL");
  }
  AMG_TRY(cuda_ready());
  const AllocFailArm fail_arm;  // AMG_GB300_FAIL_ALLOC: test hook, off unless set
  const NvtxRange setup_range("amg_setup");
  auto t0 = std::chrono::steady_clock::now();
  amg_handle_s *h = new amg_handle_s();
  h->opt = o;
  h->n = n;
  {
    // CUDA-graph replay of the preconditioner is the default; AMG_GB300_GRAPHS=0
    // issues the same kernels one by one instead (debugging, A/B timing)
    const char *env = getenv("AMG_GB300_GRAPHS");
    h->use_graph = !(env && env[0] == '0');
    // AMG_GB300_PDL=1 launches the solve kernels with programmatic dependent
    // launch (overlapping each launch with its predecessor's drain); it
    // measured neutral on the 128^3 workload, so it is off by default
    const char *pdl = getenv("AMG_GB300_PDL");
    h->use_pdl = (pdl && pdl[0] == '1');
    // AMG_GB300_PROLONG_SPLIT=0 keeps the fused prolongation-residual kernel
    // on every level (A/B timing of the two equivalent forms)
    const char *ps = getenv("AMG_GB300_PROLONG_SPLIT");
    h->prolong_split = !(ps && ps[0] == '0');
  }
  cudaGetDevice(&h->device);
  // NULL selects the legacy default stream, which orders our work after any
  // work the caller queued on it (e.g. a framework's default stream)
  h->stream = (cudaStream_t)cuda_stream;
  h->arena.stream = h->stream;
  amg_status s = AMG_OK;
  const int64_t *drp = row_ptr;
  const int32_t *dcol = col_idx;
  const double *dw = w, *dd = d;
  void *tmp[4] = {nullptr, nullptr, nullptr, nullptr};
  if (mem_space == AMG_MEM_HOST) {
    const int64_t nnz = row_ptr[n];
    s = pool_alloc(&tmp[0], sizeof(int64_t) * (size_t)(n + 1), h->stream);
    if (!s) s = pool_alloc(&tmp[1], sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1), h->stream);
    if (!s) s = pool_alloc(&tmp[2], sizeof(double) * (size_t)std::max<int64_t>(nnz, 1), h->stream);
    if (!s && d) s = pool_alloc(&tmp[3], sizeof(double) * (size_t)n, h->stream);
    if (!s) {
      cudaMemcpyAsync(tmp[0], row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, h->stream);
      if (nnz) {
        cudaMemcpyAsync(tmp[1], col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(tmp[2], w, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice, h->stream);
      }
      if (d) cudaMemcpyAsync(tmp[3], d, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) s = fail(AMG_ERR_CUDA, std::string("copy of the input: ") + cudaGetErrorString(e));
      drp = (const int64_t *)tmp[0];
      dcol = (const int32_t *)tmp[1];
      dw = (const double *)tmp[2];
      dd = d ? (const double *)tmp[3] : nullptr;
    }
  }
  if (!s) s = build_hierarchy(h, n, drp, dcol, dw, dd);
  for (void *p : tmp) pool_free(p, h->stream);
  {
    NvtxPhase ph(h->stream);
    ph.next("amg_setup: solve buffers");
    if (!s) s = allocate_solve_buffers(h);
    ph.next("amg_setup: dense two-level operator");
    if (!s) s = build_dense_two_level(h);
    ph.next("amg_setup: leaf kernel data");
    if (!s) s = prepare_leaf(h);
  }
  if (!s) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = fail(AMG_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(e));
  }
  if (s) {
    std::string msg = thread_error();
    destroy(h);
    fail(s, msg);
    return s;
  }
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return AMG_OK;
}

amg_status amg_solve(amg_handle h, const double *rhs, double *x, int nrhs, int64_t ld, double tol,
                     amg_info *info) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "handle is NULL");
  if (!rhs || !x || nrhs < 1 || ld < h->n || !(tol >= 0.0))
    return record(h, fail(AMG_ERR_INVALID_ARG, "rhs/x NULL, nrhs < 1, ld < n or tol invalid"));
  if (cudaSetDevice(h->device) != cudaSuccess) return record(h, fail(AMG_ERR_CUDA, "cudaSetDevice"));
  const NvtxRange solve_range("amg_solve");
  auto t0 = std::chrono::steady_clock::now();
  h->launches = 0;
  const bool rdev = is_device_ptr(rhs), xdev = is_device_ptr(x);
  const int64_t n = h->n;
  double *bstage = nullptr, *xstage = nullptr;
  amg_status s = AMG_OK;
  const char *benv = getenv("AMG_GB300_BATCHED");
  // the block path implements the K-cycle; AMLI-cycle handles solve column by column
  if (nrhs >= 2 && !(benv && benv[0] == '0') && h->opt.cycle == AMG_CYCLE_K) {
    // all right-hand sides together (block kernels, per-column scalars)
    const double *bd = rhs;
    double *xd = x;
    const size_t bytes = sizeof(double) * (size_t)ld * (size_t)nrhs;
    if (!rdev) s = pool_alloc((void **)&bstage, bytes, h->stream);
    if (!s && !xdev) s = pool_alloc((void **)&xstage, bytes, h->stream);
    if (!s && !rdev) {
      if (cudaMemcpyAsync(bstage, rhs, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        s = fail(AMG_ERR_CUDA, "copy of the right-hand sides");
      bd = bstage;
    }
    if (!xdev) xd = xstage;
    int it = 0, conv = 0;
    double rel = 0.0, tr = 0.0;
    bool brk = false;
    if (!s) s = solve_batched(h, bd, xd, nrhs, ld, tol, info, &it, &rel, &tr, &conv, &brk, 0, nullptr);
    if (!s && !xdev) {
      if (cudaMemcpyAsync(x, xstage, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        s = fail(AMG_ERR_CUDA, "copy of the solutions");
    }
    pool_free(bstage, h->stream);
    pool_free(xstage, h->stream);
    if (!s) {
      cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) s = fail(AMG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
    }
    if (info) {
      info->iterations = it;
      info->converged = conv;
      info->rel_residual = rel;
      info->true_rel_residual = tr;
      info->n_levels = h->L;
      info->grid_complexity = h->grid_complexity;
      info->op_complexity = h->op_complexity;
      info->setup_ms = h->setup_ms;
      info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (s) return record(h, s);
    if (brk) return record(h, fail(AMG_ERR_BREAKDOWN, "flexible CG breakdown in at least one column"));
    if (!conv) return record(h, fail(AMG_ERR_NOT_CONVERGED, "max_iters reached before tol"));
    return AMG_OK;
  }
  if (!rdev) s = pool_alloc((void **)&bstage, sizeof(double) * (size_t)n, h->stream);
  if (!s && !xdev) s = pool_alloc((void **)&xstage, sizeof(double) * (size_t)n, h->stream);
  int max_it = 0, all_conv = 1;
  double max_rel = 0.0, max_true = 0.0;
  amg_status worst = AMG_OK;
  for (int j = 0; j < nrhs && !s; ++j) {
    const double *bj = rhs + (int64_t)j * ld;
    double *xj = x + (int64_t)j * ld;
    const double *bd = bj;
    if (!rdev) {
      if (cudaMemcpyAsync(bstage, bj, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        s = fail(AMG_ERR_CUDA, "copy of the right-hand side");
        break;
      }
      bd = bstage;
    }
    double *xd = xdev ? xj : xstage;
    amg_info tmp_info;
    memset(&tmp_info, 0, sizeof(tmp_info));
    if (info && j == 0) {
      tmp_info.history = info->history;
      tmp_info.history_cap = info->history_cap;
    }
    int it = 0, conv = 0;
    double rel = 0, tr = 0;
    amg_status sj = solve_one(h, bd, xd, tol, &tmp_info, &it, &rel, &tr, &conv);
    if (sj != AMG_OK && sj != AMG_ERR_NOT_CONVERGED && sj != AMG_ERR_BREAKDOWN) {
      s = sj;
      break;
    }
    if (!xdev) {
      if (cudaMemcpyAsync(xj, xstage, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess) {
        s = fail(AMG_ERR_CUDA, "copy of the solution");
        break;
      }
    }
    if (info && j == 0) info->history_len = tmp_info.history_len;
    if (sj != AMG_OK && worst == AMG_OK) worst = sj;
    if (sj == AMG_ERR_BREAKDOWN) worst = sj;
    max_it = std::max(max_it, it);
    max_rel = std::max(max_rel, rel);
    max_true = std::max(max_true, tr);
    all_conv &= conv;
  }
  pool_free(bstage, h->stream);
  pool_free(xstage, h->stream);
  if (!s) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = fail(AMG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(e));
  }
  if (info) {
    info->iterations = max_it;
    info->converged = all_conv;
    info->rel_residual = max_rel;
    info->true_rel_residual = max_true;
    info->n_levels = h->L;
    info->grid_complexity = h->grid_complexity;
    info->op_complexity = h->op_complexity;
    info->setup_ms = h->setup_ms;
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (s) return record(h, s);
  if (worst == AMG_ERR_NOT_CONVERGED) fail(worst, "max_iters reached before tol");
  return record(h, worst);
}

void amg_free(amg_handle h) { destroy(h); }

const char *amg_last_error(amg_handle h) {
  if (h) return h->err.c_str();
  return thread_error().c_str();
}

int amg_num_levels(amg_handle h) { return h ? h->L : 0; }

int64_t amg_level_n(amg_handle h, int k) {
  if (!h || k < 0 || k >= h->L) return -1;
  return h->lv[k].n;
}

int64_t amg_level_nnz(amg_handle h, int k) {
  if (!h || k < 0 || k >= h->L) return -1;
  return h->lv[k].A.nnz;
}

amg_status amg_level_csr(amg_handle h, int k, int64_t *rowptr, int32_t *col, double *val, double *diag,
                         double *dlow) {
  if (!h || k < 0 || k >= h->L) return fail(AMG_ERR_INVALID_ARG, "level out of range");
  cudaSetDevice(h->device);
  const amg::Level &L = h->lv[k];
  cudaStream_t st = h->stream;
  if (rowptr) AMG_CUDA_TRY(cudaMemcpyAsync(rowptr, L.A.rowptr, sizeof(int64_t) * (size_t)(L.n + 1), cudaMemcpyDeviceToHost, st));
  if (col && L.A.nnz) AMG_CUDA_TRY(cudaMemcpyAsync(col, L.A.col, sizeof(int32_t) * (size_t)L.A.nnz, cudaMemcpyDeviceToHost, st));
  if (val && L.A.nnz) AMG_CUDA_TRY(cudaMemcpyAsync(val, L.A.val, sizeof(double) * (size_t)L.A.nnz, cudaMemcpyDeviceToHost, st));
  if (diag) AMG_CUDA_TRY(cudaMemcpyAsync(diag, L.diag, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost, st));
  if (dlow) AMG_CUDA_TRY(cudaMemcpyAsync(dlow, L.dlow, sizeof(double) * (size_t)L.n, cudaMemcpyDeviceToHost, st));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  return AMG_OK;
}

amg_status amg_level_agg(amg_handle h, int k, int32_t *agg) {
  if (!h || k < 0 || k + 1 >= h->L || !agg) return fail(AMG_ERR_INVALID_ARG, "level out of range");
  cudaSetDevice(h->device);
  AMG_CUDA_TRY(cudaMemcpyAsync(agg, h->lv[k].agg, sizeof(int32_t) * (size_t)h->lv[k].n, cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

amg_status amg_level_smoother(amg_handle h, int k, double *lam0, double *lam1, double *coef) {
  if (!h || k < 0 || k + 1 >= h->L) return fail(AMG_ERR_INVALID_ARG, "level out of range");
  if (lam0) *lam0 = h->lv[k].lam0;
  if (lam1) *lam1 = h->lv[k].lam1;
  if (coef) memcpy(coef, h->lv[k].coef, sizeof(double) * (size_t)(h->opt.degree + 1));
  return AMG_OK;
}

#define APPLY_GUARD(cond)                                                                  \
  do {                                                                                     \
    if (!h) return fail(AMG_ERR_INVALID_ARG, "handle is NULL");                            \
    if (!(cond)) return record(h, fail(AMG_ERR_INVALID_ARG, "level or pointer invalid"));  \
    if (cudaSetDevice(h->device) != cudaSuccess) return record(h, fail(AMG_ERR_CUDA, "cudaSetDevice")); \
  } while (0)

amg_status amg_apply_spmv(amg_handle h, int k, const double *x, double *y) {
  APPLY_GUARD(k >= 0 && k < h->L && x && y);
  return record(h, apply_spmv(h, k, x, y));
}
amg_status amg_apply_smoother(amg_handle h, int k, const double *r, double *x) {
  APPLY_GUARD(k >= 0 && k + 1 < h->L && r && x);
  return record(h, apply_smoother(h, k, r, x));
}
amg_status amg_apply_restrict(amg_handle h, int k, const double *s, double *rH) {
  APPLY_GUARD(k >= 0 && k + 1 < h->L && s && rH);
  return record(h, apply_restrict(h, k, s, rH));
}
amg_status amg_apply_prolong_add(amg_handle h, int k, const double *eH, double *x) {
  APPLY_GUARD(k >= 0 && k + 1 < h->L && eH && x);
  return record(h, apply_prolong_add(h, k, eH, x));
}
amg_status amg_apply_coarse_solve(amg_handle h, const double *b, double *x) {
  APPLY_GUARD(b && x);
  return record(h, apply_coarse_solve(h, b, x));
}
amg_status amg_apply_kcycle(amg_handle h, int k, const double *r, double *z) {
  APPLY_GUARD(k >= 0 && k < h->L && r && z);
  return record(h, apply_kcycle(h, k, r, z));
}

amg_status amg_match(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const double *s,
                     uint64_t salt, int32_t *mate, int32_t *agg, int64_t *n_coarse, int *rounds,
                     void *cuda_stream) {
  if (n < 1 || n > kMaxRows || !row_ptr || !mate || !agg)
    return fail(AMG_ERR_INVALID_ARG, "n, row_ptr, mate or agg invalid");
  if (!col_idx || !s) return fail(AMG_ERR_INVALID_ARG, "col_idx and s must be non-NULL");
  AMG_TRY(cuda_ready());
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int nH = 0, r = 0;
  AMG_TRY(match_pass(st, (int)n, row_ptr, col_idx, s, salt, mate, agg, &nH, &r, nullptr));
  AMG_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_coarse) *n_coarse = nH;
  if (rounds) *rounds = r;
  return AMG_OK;
}

amg_status amg_kernel_timing(amg_handle h, int enable) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "handle is NULL");
  h->timing.enabled = enable != 0;
  for (int k = 0; k < kTimedKinds; ++k) {
    h->timing.launches[k] = 0;
    h->timing.total_ms[k] = 0.0;
  }
  h->timing.used = 0;
  return AMG_OK;
}

amg_status amg_kernel_timing_read_kind(amg_handle h, int kind, int64_t *launches, double *total_ms,
                                       double *bytes_per_launch) {
  if (!h) return fail(AMG_ERR_INVALID_ARG, "handle is NULL");
  if (kind < 0 || kind >= kTimedKinds) return record(h, fail(AMG_ERR_INVALID_ARG, "kind must be 0, 1 or 2"));
  if (launches) *launches = h->timing.launches[kind];
  if (total_ms) *total_ms = h->timing.total_ms[kind];
  if (bytes_per_launch) {
    const amg::Level &L = h->lv[0];
    const bool f32 = h->opt.precision == AMG_PREC_FP32;
    const double vs = f32 ? 4.0 : 8.0;
    const double nnz = (double)L.A.nnz, n = (double)L.n, nH = (double)L.nH;
    if (kind == 0) {
      // one fused smoother step on level 0: the stored SELL entries (value +
      // column index, 4 bytes or a 2-byte offset) and diagonal once, the
      // gathered vector T_j once, and the row-wise vectors T_{j-1} (read),
      // T_{j+1} (write), x (read + write)
      const double cs = (L.S.sdel && L.wps == 1) ? 2.0 : 4.0;
      *bytes_per_launch = nnz * (vs + cs) + (double)(L.S.nslices + 1) * 8.0 + n * vs * 6.0;
    } else if (kind == 1) {
      // r_H = P^T s: the member lists (the fixed-width table, or offsets +
      // members), s once, r_H written
      const double lists = L.memw ? (double)L.memw_width * nH * 4.0 : (nH + 1.0) * 4.0 + n * 4.0;
      *bytes_per_launch = lists + n * vs + nH * vs;
    } else {
      // x = u + P e_H: agg and u read, x written, e_H read once
      *bytes_per_launch = n * (4.0 + 2.0 * vs) + nH * vs;
    }
  }
  return AMG_OK;
}

amg_status amg_kernel_timing_read(amg_handle h, int64_t *launches, double *total_ms,
                                  double *bytes_per_launch) {
  return amg_kernel_timing_read_kind(h, 0, launches, total_ms, bytes_per_launch);
}

int64_t amg_launch_count(amg_handle h) { return h ? h->launches : 0; }

}  // extern "C"
