// leaf.cu -- the inner flexible-CG solve at the level just above the dense
// two-level operator, as ONE thread-block-cluster kernel per call.
//
// Level k0 = Bk - 1 (a few hundred to two thousand rows) is visited 2^k0
// times per outer iteration.  Issued as separate kernels, one inner solve
// there is ~45 dependent launches whose cost is latency -- dependent L2
// round trips inside each kernel plus the launch gaps -- not work.  Here one
// launch runs the whole inner solve at k0 (nu flexible-CG steps, each
// preconditioned by the K-cycle at k0: smoothing, restriction, the inner
// solve at k0+1 preconditioned by the dense two-level operator B,
// prolongation, smoothing; Sec. 3, Sec. 4) on one cluster of C CTAs:
//   * CTA c owns a contiguous block of rows on both levels and keeps in
//     shared memory its rows of A_k0 and of the smoother form 2 t(A_k0)
//     (compact CSR, no slice padding) and its rows of B and of A_k0+1 B
//     (computed once per setup), so a coarse inner step forms D = B r and
//     W = A_k0+1 D = (A_k0+1 B) r in one phase;
//   * every vector that some phase reads at another CTA's rows is kept as a
//     copy in every CTA's shared memory; the phase that produces an entry of
//     a level-k0 vector writes it with distributed-shared-memory stores into
//     the copies of the CTAs that read that row (the owner, the owners of its
//     neighbours and of its aggregate: a per-row mask made at setup), an
//     entry of a coarse vector into every copy;
//   * a hardware cluster barrier (release/acquire) ends each phase;
//   * level-k0 dot products: each CTA posts its partial sums into every CTA's
//     slot table; after the barrier every CTA adds the C partials in rank
//     order, so all CTAs hold bit-identical Krylov scalars (the stop/breakdown
//     decisions are therefore uniform) and no global scalar traffic occurs;
//   * the coarse inner solve (level k0+1, a few hundred rows): after D and W
//     are sent to every CTA, each CTA computes the scalars and updates D, W,
//     x and r over all coarse rows itself, in the same order everywhere, so
//     its orthogonalisation and updates need no barrier of their own.
// Every cluster barrier sits in code whose trip counts come from the launch
// parameters only, so all CTAs meet the same barriers.
//
// The arithmetic is that of the multi-kernel path (solve.cu) step for step:
// the Chebyshev recurrence, the stop rule of the inner flexible CG and the
// vector updates are the same expressions in the same precision; only the
// summation order inside a row and inside a dot product differs.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace amg {

constexpr int kLeafDefaultThreads = 256;  // CTA size; 512 and 1024 are also instantiated
constexpr int kLeafMaxC = 16;
constexpr int kLeafMaxInner = 4;
constexpr int kLeafMaxRows = 2048;    // rows of level k0
constexpr int kLeafMaxCoarse = 1024;  // rows of level k0 + 1
constexpr int kLeafSlot = 8;          // doubles per CTA in a slot table
constexpr int kLeafProfSlots = 128;   // phases recorded by the opt-in profile
constexpr int kDenseLanes = 8;        // lanes per row of the dense coarse products

// shared-memory arrays, in layout order
enum LeafArr : int {
  // ---- static: fixed per setup, built once in global memory in this
  // layout (one image per CTA) and copied in by every launch ----
  // compact CSR of the owned rows of A_k0 (off-diagonal) and its diagonal,
  // and the values and diagonal of the smoother form S = 2 t(A) on the same
  // pattern (2 sa a_ij; 2 sa a_ii - 2 ca)
  A_LRP = 0, A_LCOL, A_LVAL, A_LDIAG, A_SVAL, A_SDIAG,
  // aggregate id of every row of level k0
  A_AGG,
  // destination mask of every owned row (the CTAs that read it)
  A_MASK,
  // member lists of the owned aggregates
  A_LAP, A_LAM,
  // owned rows of B and of A_k0+1 B (fp64, nH columns)
  A_BROWS, A_ABROWS,
  // ---- per launch ----
  // full copies, level k0 (n entries of T)
  A_B, A_R, A_TA, A_TB, A_U, A_S, A_D0,
  // owned rows, level k0 (R entries of T)
  A_W0 = A_D0 + kLeafMaxInner, A_XO = A_W0 + kLeafMaxInner,
  // full copies, level k0+1 (nH entries of T)
  A_HB, A_HR, A_HX, A_HD0,
  A_HW0 = A_HD0 + kLeafMaxInner,
  // dot-product slot tables [2][C][kLeafSlot] and per-warp partials
  A_SLOTS = A_HW0 + kLeafMaxInner, A_WRED,
  A_COUNT
};

template <typename T>
struct LeafParams {
  int n, nH, C, R, RH, m, nu, tpr;
  int nt;                 // threads per CTA (the kernel's template argument)
  int maxnz, maxmem;
  double two_sa, two_ca;  // smoother form: 2 sa = 4/(l1 - l0), 2 ca = 2 (l1 + l0)/(l1 - l0)
  T coef[kMaxDegree + 1];
  const int64_t *rp;
  const int32_t *col;
  const double *val, *diag;
  const int32_t *agg, *agg_ptr, *agg_mem;
  const double *B, *AB;   // B and A_k0+1 B, nH x nH row major
  // mask[i]: bit r set if CTA r reads row i of the level-k0 vectors (it owns
  // i, a neighbour of i, or the aggregate of i); null: every CTA
  const unsigned *mask;
  const T *b;
  T *x;
  // opt-in phase profile (AMG_GB300_LEAF_PROFILE=1): CTA 0 adds the SM
  // cycles of every phase (barrier to barrier) into prof[phase], and the
  // launch count into prof[kLeafProfSlots - 1]; null otherwise
  unsigned long long *prof;
  // the static arrays of every CTA: CTA c's image is the first
  // static_bytes of its shared memory, at image + c * static_bytes
  const unsigned char *image;
  unsigned static_bytes;
  unsigned off[A_COUNT];  // byte offsets into dynamic shared memory
  unsigned smem;          // bytes
};

// byte offsets of every array (16-byte aligned); identical on host and device
template <typename T>
static unsigned leaf_layout(LeafParams<T> &P) {
  size_t cnt[A_COUNT] = {};
  size_t esz[A_COUNT] = {};
  for (int a = 0; a < A_COUNT; ++a) esz[a] = sizeof(T);
  for (int a = A_B; a <= A_S; ++a) cnt[a] = P.n;
  for (int l = 0; l < P.nu; ++l) {
    cnt[A_D0 + l] = P.n;
    cnt[A_W0 + l] = P.R;
    cnt[A_HD0 + l] = P.nH;
    cnt[A_HW0 + l] = P.nH;
  }
  cnt[A_XO] = P.R;
  cnt[A_HB] = cnt[A_HR] = cnt[A_HX] = P.nH;
  cnt[A_LRP] = P.R + 1;
  esz[A_LRP] = sizeof(int);
  cnt[A_LCOL] = P.maxnz;
  esz[A_LCOL] = sizeof(int);
  cnt[A_LVAL] = P.maxnz;
  cnt[A_LDIAG] = P.R;
  cnt[A_SVAL] = P.maxnz;
  cnt[A_SDIAG] = P.R;
  cnt[A_AGG] = P.n;
  esz[A_AGG] = sizeof(int);
  cnt[A_MASK] = P.R;
  esz[A_MASK] = sizeof(unsigned);
  cnt[A_LAP] = P.RH + 1;
  esz[A_LAP] = sizeof(int);
  cnt[A_LAM] = P.maxmem;
  esz[A_LAM] = sizeof(int);
  cnt[A_BROWS] = cnt[A_ABROWS] = (size_t)P.RH * P.nH;
  esz[A_BROWS] = esz[A_ABROWS] = sizeof(double);
  cnt[A_SLOTS] = 2 * (size_t)P.C * kLeafSlot;
  esz[A_SLOTS] = sizeof(double);
  cnt[A_WRED] = (size_t)(P.nt / 32) * kLeafSlot;
  esz[A_WRED] = sizeof(double);
  size_t o = 0;
  for (int a = 0; a < A_COUNT; ++a) {
    o = (o + 15) & ~(size_t)15;
    P.off[a] = (unsigned)o;
    o += cnt[a] * esz[a];
  }
  P.smem = (unsigned)((o + 15) & ~(size_t)15);
  P.static_bytes = P.off[A_B];  // a multiple of 16: every offset is
  return P.smem;
}

// 16-byte asynchronous global -> shared copy (completion: cp.async.wait_all)
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

// The static image of CTA blockIdx.x (one block per cluster rank): its rows
// of the level-k0 operator and smoother form, the aggregate map, masks,
// member lists and its rows of B and A_k0+1 B, laid out as in shared memory.
template <typename T>
__global__ void k_leaf_image(const __grid_constant__ LeafParams<T> P, unsigned char *image) {
  unsigned char *im = image + (size_t)blockIdx.x * P.static_bytes;
  const int rank = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int n = P.n, nH = P.nH;
  const int r0 = rank * P.R, nloc = max(0, min(n, r0 + P.R) - r0), r0c = min(r0, n);
  const int h0 = rank * P.RH, nlocH = max(0, min(nH, h0 + P.RH) - h0), h0c = min(h0, nH);
  auto vec = [&](int a) { return reinterpret_cast<T *>(im + P.off[a]); };
  auto ivec = [&](int a) { return reinterpret_cast<int *>(im + P.off[a]); };
  int *lrp = ivec(A_LRP), *lcol = ivec(A_LCOL), *agg = ivec(A_AGG), *lap = ivec(A_LAP), *lam = ivec(A_LAM);
  unsigned *lmask = reinterpret_cast<unsigned *>(im + P.off[A_MASK]);
  T *lval = vec(A_LVAL), *ldiag = vec(A_LDIAG), *sval = vec(A_SVAL), *sdiag = vec(A_SDIAG);
  double *brows = reinterpret_cast<double *>(im + P.off[A_BROWS]);
  double *abrows = reinterpret_cast<double *>(im + P.off[A_ABROWS]);
  for (int i = tid; i < n; i += nt) agg[i] = P.agg[i];
  const int64_t e0 = P.rp[r0c];
  for (int li = tid; li <= nloc; li += nt) lrp[li] = (int)(P.rp[r0c + li] - e0);
  for (int li = tid; li < nloc; li += nt) {
    const double dg = P.diag[r0 + li];
    ldiag[li] = (T)dg;
    sdiag[li] = (T)(P.two_sa * dg - P.two_ca);  // as the multi-kernel path stores it
    lmask[li] = P.mask ? P.mask[r0 + li] : (1u << P.C) - 1u;
  }
  const int cnt = (int)(P.rp[r0c + nloc] - e0);
  for (int e = tid; e < cnt; e += nt) {
    lcol[e] = P.col[e0 + e];
    lval[e] = (T)P.val[e0 + e];
    sval[e] = (T)(P.two_sa * P.val[e0 + e]);
  }
  const int a0 = P.agg_ptr[h0c];
  for (int lI = tid; lI <= nlocH; lI += nt) lap[lI] = P.agg_ptr[h0c + lI] - a0;
  const int mc = P.agg_ptr[h0c + nlocH] - a0;
  for (int e = tid; e < mc; e += nt) lam[e] = P.agg_mem[a0 + e];
  for (int e = tid; e < nlocH * nH; e += nt) {
    brows[e] = P.B[(size_t)h0c * nH + e];
    abrows[e] = P.AB[(size_t)h0c * nH + e];
  }
}

template <typename T, int kLeafThreads>
__global__ void __launch_bounds__(kLeafThreads, 1) k_leaf(const __grid_constant__ LeafParams<T> P) {
  constexpr int kLeafWarps = kLeafThreads / 32;
  extern __shared__ __align__(16) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int C = P.C, n = P.n, nH = P.nH, nu = P.nu, m = P.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // owned rows [r0, r0 + nloc) and [h0, h0 + nlocH); trailing CTAs may own
  // none (r0 >= n), hence the clamped starts used for loads
  const int r0 = rank * P.R, nloc = max(0, min(n, r0 + P.R) - r0), r0c = min(r0, n);
  const int h0 = rank * P.RH, nlocH = max(0, min(nH, h0 + P.RH) - h0), h0c = min(h0, nH);

  auto vec = [&](int a) { return reinterpret_cast<T *>(sm + P.off[a]); };
  auto ivec = [&](int a) { return reinterpret_cast<int *>(sm + P.off[a]); };
  T *vb = vec(A_B), *vr = vec(A_R), *vTa = vec(A_TA), *vTb = vec(A_TB), *vu = vec(A_U), *vs = vec(A_S);
  T *xo = vec(A_XO);
  T *hb = vec(A_HB), *hr = vec(A_HR), *hx = vec(A_HX);
  int *lrp = ivec(A_LRP), *lcol = ivec(A_LCOL), *agg = ivec(A_AGG), *lap = ivec(A_LAP), *lam = ivec(A_LAM);
  T *lval = vec(A_LVAL), *ldiag = vec(A_LDIAG), *sval = vec(A_SVAL), *sdiag = vec(A_SDIAG);
  double *brows = reinterpret_cast<double *>(sm + P.off[A_BROWS]);
  double *abrows = reinterpret_cast<double *>(sm + P.off[A_ABROWS]);
  double *slots = reinterpret_cast<double *>(sm + P.off[A_SLOTS]);
  double *wred = reinterpret_cast<double *>(sm + P.off[A_WRED]);
  __shared__ double s_sc[40];
  const long long t_start = clock64();

  // ---- load: this CTA's static image (one round of 16-byte asynchronous
  // copies) and b (all rows) ----
  {
    const unsigned char *src = P.image + (size_t)rank * P.static_bytes;
    for (unsigned o = (unsigned)tid * 16u; o < P.static_bytes; o += (unsigned)kLeafThreads * 16u)
      cp_async16(sm + o, src + o);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int i = tid; i < n; i += kLeafThreads) vb[i] = P.b[i];
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  unsigned *lmask = reinterpret_cast<unsigned *>(sm + P.off[A_MASK]);
  cl.sync();  // every CTA has started and loaded before any remote store
  if (P.prof && rank == 0 && tid == 0)
    atomicAdd(&P.prof[kLeafProfSlots - 2], (unsigned long long)(clock64() - t_start));
  // cluster barrier ending a phase (with the opt-in profile: CTA 0 records
  // the phase's cycles)
  int phase = 0;
  long long t_phase = clock64();
  auto csync = [&]() {
    cl.sync();
    if (P.prof && rank == 0 && tid == 0) {
      const long long t = clock64();
      if (phase < kLeafProfSlots - 2) atomicAdd(&P.prof[phase], (unsigned long long)(t - t_phase));
      t_phase = t;
    }
    ++phase;
  };

  // ---- building blocks ----
  // write v into row i of `a` in every CTA's copy (fire-and-forget stores):
  // the coarse vectors, which the dense phases read in full
  auto put = [&](T *a, int i, T v) {
    for (int r = 0; r < C; ++r) *cl.map_shared_rank(a + i, (unsigned)r) = v;
  };
  // the same for an owned row i of a level-k0 vector, into the copies of the
  // CTAs that read that row only
  auto put0 = [&](T *a, int i, T v) {
    unsigned mk = lmask[i - r0];
    while (mk) {
      const int r = __ffs(mk) - 1;
      mk &= mk - 1u;
      *cl.map_shared_rank(a + i, (unsigned)r) = v;
    }
  };
  // sweep over the owned rows of A_k0: epi(local row, row, sum_j a_ij x_j, q).
  // The tpr lanes of a row share its entries; every lane gets the full sum,
  // but only lane q == 0 may write (a row's vectors are read and written in
  // place within one phase, e.g. x += c_j T_j, so a second writer could race
  // with a slower reader of the same row).
  // off-diagonal values `vals`: lval (A) or sval (the smoother form S)
  auto sweepv = [&](const T *vals, auto xf, auto epi) {
    const int tpr = P.tpr, q = tid & (tpr - 1), per = kLeafThreads / tpr;
    for (int base = 0; base < P.R; base += per) {
      const int li = base + tid / tpr;
      const bool ok = li < nloc;
      T acc = T(0);
      if (ok)
        for (int e = lrp[li] + q; e < lrp[li + 1]; e += tpr) acc = fma(vals[e], xf(lcol[e]), acc);
      for (int o = 1; o < tpr; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (ok) epi(li, r0 + li, acc, q);
    }
  };
  auto sweep = [&](auto xf, auto epi) { sweepv(lval, xf, epi); };
  // dot products: post this CTA's nd partial sums (nd <= kLeafSlot, static
  // register indices) to every CTA's slot table
  int sb = 0;
  // Every shuffle-add step is a full-warp FP64 add (2 lanes per clock on
  // this part), so the tree is cut short: the partials sit only in lanes
  // that are multiples of `stride` (the caller's lane grouping), and a warp
  // whose partials are all zero writes zeros without a tree.
  auto post = [&](const double (&v)[kLeafSlot], int nd, int stride) {
    bool nz = false;
#pragma unroll
    for (int q = 0; q < kLeafSlot; ++q)
      if (q < nd) nz |= v[q] != 0.0;
    const bool active = __any_sync(0xffffffffu, nz);
#pragma unroll
    for (int q = 0; q < kLeafSlot; ++q) {
      if (q < nd) {
        double t = v[q];
        if (active)
          for (int o = 16; o >= stride; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) wred[warp * kLeafSlot + q] = active ? t : 0.0;
      }
    }
    __syncthreads();
    if (tid < nd) {
      double t = 0.0;
      for (int w = 0; w < kLeafWarps; ++w) t += wred[w * kLeafSlot + tid];
      for (int r = 0; r < C; ++r)
        *cl.map_shared_rank(slots + (sb * C + rank) * kLeafSlot + tid, (unsigned)r) = t;
    }
  };
  // after the barrier: the cluster-wide sums, added in rank order by nd
  // threads (the FP64 pipe runs 2 lanes per clock: scalar work is done once
  // per CTA, not once per thread) into shared out[0, nd); then a CTA barrier
  auto fold = [&](double *out, int nd) {
    if (tid < nd) {
      double t = 0.0;
      for (int c = 0; c < C; ++c) t += slots[(sb * C + c) * kLeafSlot + tid];
      out[tid] = t;
    }
    sb ^= 1;
    __syncthreads();
  };
  // Krylov scalars of one inner flexible CG, in shared memory: rho[4],
  // alpha[4], beta[4], stop flag; sums[8] holds folded dot products
  double *const scT = s_sc, *const scH = s_sc + 16, *const sums = s_sc + 32;
  // rho_it = s0; alpha_it = s1 / rho_it unless the solve has stopped or
  // rho_it is not a positive finite number (then the stop flag is set and
  // alpha_it = 0): the rule of the multi-kernel path.  Thread 0 only.
  auto fin_alpha = [&](double *sc, int it) {
    const double r = sums[0], sg = sums[1];
    sc[it] = r;
    if (sc[12] != 0.0 || !(r > 0.0) || !isfinite(r)) {
      sc[12] = 1.0;
      sc[4 + it] = 0.0;
    } else {
      sc[4 + it] = sg / r;
    }
  };

  // x (=|+=) q_m(A) r on level k0; r is a full copy, x a full copy whose
  // owned rows are updated and which is broadcast by the last step
  auto smooth = [&](const T *r, T *x, bool add) {
    if (m == 0) {
      for (int li = tid; li < nloc; li += kLeafThreads) {
        const int i = r0 + li;
        const T inc = P.coef[0] * r[i];
        const T v = add ? x[i] + inc : inc;
        put0(x, i, v);
      }
      csync();
      return;
    }
    const T b0 = P.coef[0], b1 = P.coef[1];
    // T_1 = S r / 2, T_{j+1} = S T_j - T_{j-1} with the stored smoother form
    sweepv(sval, [&](int j) { return r[j]; },
          [&](int li, int i, T acc, int q) {
            if (q != 0) return;
            const T ri = r[i];
            const T t1 = T(0.5) * fma(sdiag[li], ri, acc);
            if (m > 1) put0(vTa, i, t1);
            const T inc = fma(b1, t1, b0 * ri);
            const T v = add ? x[i] + inc : inc;
            if (m == 1) put0(x, i, v);
            else x[i] = v;
          });
    csync();
    const T *Tp = r;
    T *Tc = vTa;
    for (int j = 2; j <= m; ++j) {
      T *Tn = (j == 2) ? vTb : const_cast<T *>(Tp);
      const T bj = P.coef[j];
      const bool last = (j == m);
      sweepv(sval, [&](int jj) { return Tc[jj]; },
            [&](int li, int i, T acc, int q) {
              if (q != 0) return;
              const T tn = fma(sdiag[li], Tc[i], acc) - Tp[i];  // Tp[i] read before Tn[i] (may alias) is written
              const T v = fma(bj, tn, x[i]);
              if (!last) put0(Tn, i, tn);
              if (last) put0(x, i, v);
              else x[i] = v;
            });
      csync();
      Tp = Tc;
      Tc = Tn;
    }
  };

  // the inner flexible CG at level k0+1 (nu steps, preconditioner B) on
  // hb; result in hx (full copy)
  // dot products over all nH coarse rows of data every CTA holds in full,
  // in a fixed order (thread I's products, then the warp tree, then warps in
  // order): every CTA gets the same bits, so no cluster exchange is needed.
  // out[q] = sum_I f(I, q) for q < nd, in shared memory; ends with a CTA
  // barrier.
  auto local_dots = [&](double *out, int nd, auto f) {
    double v[kLeafSlot] = {};
    for (int I = tid; I < nH; I += kLeafThreads) {
#pragma unroll
      for (int q = 0; q < kLeafSlot; ++q)
        if (q < nd) v[q] += f(I, q);
    }
    const bool active = __any_sync(0xffffffffu, tid < nH);
#pragma unroll
    for (int q = 0; q < kLeafSlot; ++q) {
      if (q < nd) {
        double t = v[q];
        if (active)
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) wred[warp * kLeafSlot + q] = active ? t : 0.0;
      }
    }
    __syncthreads();
    if (tid < nd) {
      double t = 0.0;
      for (int w = 0; w < kLeafWarps; ++w) t += wred[w * kLeafSlot + tid];
      out[tid] = t;
    }
    __syncthreads();
  };

  // the inner flexible CG at level k0+1 (nu steps, preconditioner B) on
  // hb; result in hx (full copy).  A step forms D = B rin and W = A D =
  // (A B) rin at the owned rows and sends both to every CTA (one cluster
  // barrier); every CTA then derives the Krylov scalars and updates D, W,
  // x and r over all nH rows itself (nH is a few hundred), identically, so
  // the orthogonalisation and the update need no further barrier.
  auto inner_coarse = [&]() {
    if (tid == 0) scH[12] = 0.0;  // stop flag
    for (int it = 0; it < nu; ++it) {
      const T *rin = (it == 0) ? hb : hr;
      T *D = vec(A_HD0 + it), *W = vec(A_HW0 + it);
      // D = B rin and W = (A B) rin at the owned rows (fp64).  kDenseLanes
      // lanes per row, 32 / kDenseLanes rows per warp: on this part the FP64
      // pipe issues 2 lanes per clock, so a shuffle-add tree over 32 lanes
      // (every step a full-warp FP64 add) costs as much as the products;
      // 3 steps that serve 4 rows at once cost a tenth of it.
      const int sub = lane / kDenseLanes, dq = lane % kDenseLanes;
      constexpr int kRowsPerPass = kLeafWarps * (32 / kDenseLanes);
      for (int base = 0; base < P.RH; base += kRowsPerPass) {
        const int lI = base + warp * (32 / kDenseLanes) + sub;
        const bool ok = lI < nlocH;
        double ad = 0.0, aw = 0.0;
        if (ok)
          for (int j = dq; j < nH; j += kDenseLanes) {
            const double rj = (double)rin[j];
            ad = fma(brows[(size_t)lI * nH + j], rj, ad);
            aw = fma(abrows[(size_t)lI * nH + j], rj, aw);
          }
        for (int o = kDenseLanes / 2; o > 0; o >>= 1) {  // within the row's lane group
          ad += __shfl_xor_sync(0xffffffffu, ad, o);
          aw += __shfl_xor_sync(0xffffffffu, aw, o);
        }
        if (ok && dq == 0) {
          const int I = h0 + lI;
          put(D, I, (T)ad);
          put(W, I, (T)aw);
        }
      }
      csync();
      if (it == 0) {
        // rho = D.W, sigma = rin.D
        local_dots(sums, 2, [&](int I, int q) {
          return q == 0 ? (double)D[I] * (double)W[I] : (double)rin[I] * (double)D[I];
        });
        if (tid == 0) fin_alpha(scH, 0);
      } else {
        // beta_l = D_l.W / rho_l; D -= sum beta_l D_l, W -= sum beta_l W_l;
        // rho = D.W, sigma = D.rin
        local_dots(sums, it, [&](int I, int l) { return (double)vec(A_HD0 + l)[I] * (double)W[I]; });
        if (tid < it) scH[8 + tid] = sums[tid] / scH[tid];
        __syncthreads();
        for (int I = tid; I < nH; I += kLeafThreads) {
          T d = D[I], w = W[I];
#pragma unroll
          for (int l = 0; l < kLeafMaxInner; ++l) {
            if (l < it) {
              const T bl = (T)scH[8 + l];
              d -= bl * vec(A_HD0 + l)[I];
              w -= bl * vec(A_HW0 + l)[I];
            }
          }
          D[I] = d;
          W[I] = w;
        }
        __syncthreads();
        local_dots(sums, 2, [&](int I, int q) {
          return q == 0 ? (double)D[I] * (double)W[I] : (double)D[I] * (double)rin[I];
        });
        if (tid == 0) fin_alpha(scH, it);
      }
      __syncthreads();
      // x = alpha D (it 0) or x += alpha D; r = rin - alpha W before another step
      const bool here = scH[12] != 0.0 && scH[4 + it] == 0.0;
      const T a = (T)scH[4 + it];
      const bool upd_r = it + 1 < nu;
      for (int I = tid; I < nH; I += kLeafThreads) {
        if (it == 0) hx[I] = here ? T(0) : a * D[I];
        else if (!here) hx[I] = fma(a, D[I], hx[I]);
        if (upd_r) hr[I] = here ? rin[I] : rin[I] - a * W[I];
      }
      __syncthreads();
    }
  };


  // x = K_k0(r): the W(1,1) cycle at level k0; r, x full copies
  auto kcycle = [&](const T *r, T *x) {
    smooth(r, vu, false);  // u = q_m(A) r
    // s = r - A u
    sweep([&](int j) { return vu[j]; },
          [&](int li, int i, T acc, int q) {
            if (q == 0) put0(vs, i, r[i] - fma(ldiag[li], vu[i], acc));
          });
    csync();
    // r_H = P^T s over the owned aggregates (members in ascending order)
    for (int lI = tid; lI < nlocH; lI += kLeafThreads) {
      T acc = T(0);
      for (int a = lap[lI]; a < lap[lI + 1]; ++a) acc += vs[lam[a]];
      put(hb, h0 + lI, acc);
    }
    csync();
    inner_coarse();
    // x = u + P e_H and s = r - A x (neighbours formed on the fly)
    sweep([&](int j) { return vu[j] + hx[agg[j]]; },
          [&](int li, int i, T acc, int q) {
            if (q != 0) return;
            const T xi = vu[i] + hx[agg[i]];
            x[i] = xi;
            put0(vs, i, r[i] - fma(ldiag[li], xi, acc));
          });
    csync();
    smooth(vs, x, true);  // x += q_m(A) s, broadcast by its last step
  };

  // ---- the inner flexible CG at level k0 ----
  if (tid == 0) scT[12] = 0.0;
  for (int it = 0; it < nu; ++it) {
    const T *rin = (it == 0) ? vb : vr;
    T *D = vec(A_D0 + it), *W = vec(A_W0 + it);
    kcycle(rin, D);
    double dv[kLeafSlot] = {};
    sweep([&](int j) { return D[j]; },
          [&](int li, int i, T acc, int q) {
            if (q != 0) return;
            const T w = fma(ldiag[li], D[i], acc);
            W[li] = w;
            if (it == 0) {
              dv[0] += (double)D[i] * (double)w;
              dv[1] += (double)rin[i] * (double)D[i];
            } else {
#pragma unroll
              for (int l = 0; l < kLeafMaxInner; ++l)
                if (l < it) dv[l] += (double)vec(A_D0 + l)[i] * (double)w;
            }
          });
    post(dv, it == 0 ? 2 : it, P.tpr);
    csync();
    fold(sums, it == 0 ? 2 : it);
    if (it == 0) {
      if (tid == 0) fin_alpha(scT, 0);
    } else {
      if (tid < it) scT[8 + tid] = sums[tid] / scT[tid];  // beta_l
      __syncthreads();
      double ev[kLeafSlot] = {};
      for (int li = tid; li < nloc; li += kLeafThreads) {
        const int i = r0 + li;
        T d = D[i], w = W[li];
#pragma unroll
        for (int l = 0; l < kLeafMaxInner; ++l) {
          if (l < it) {
            const T bl = (T)scT[8 + l];
            d -= bl * vec(A_D0 + l)[i];
            w -= bl * vec(A_W0 + l)[li];
          }
        }
        D[i] = d;
        W[li] = w;
        ev[0] += (double)d * (double)w;
        ev[1] += (double)d * (double)rin[i];
      }
      post(ev, 2, 1);
      csync();
      fold(sums, 2);
      if (tid == 0) fin_alpha(scT, it);
    }
    __syncthreads();
    const bool here = scT[12] != 0.0 && scT[4 + it] == 0.0;
    const T a = (T)scT[4 + it];
    const bool upd_r = it + 1 < nu, last = it + 1 == nu;
    for (int li = tid; li < nloc; li += kLeafThreads) {
      const int i = r0 + li;
      T xv;
      if (it == 0) xv = here ? T(0) : a * D[i];
      else xv = here ? xo[li] : fma(a, D[i], xo[li]);
      xo[li] = xv;
      if (last) P.x[i] = xv;
      if (upd_r) put0(vr, i, here ? rin[i] : rin[i] - a * W[li]);
    }
    // the last step sends nothing to other CTAs (x goes to global memory):
    // every remote store of the launch completed at an earlier barrier, so
    // the CTAs may exit without another one
    if (upd_r) csync();
  }
  if (P.prof && rank == 0 && tid == 0) atomicAdd(&P.prof[kLeafProfSlots - 1], 1ull);
}

// AB = A B for the CSR operator A (off-diagonal part + diagonal) and the
// dense row-major B, n x n: thread per entry, fp64
__global__ void k_dense_ab(int n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ diag,
                           const double *__restrict__ B, double *__restrict__ AB) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), c = (int)(idx % n);
  double acc = diag[i] * B[idx];
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = fma(val[p], B[(int64_t)col[p] * n + c], acc);
  AB[idx] = acc;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
static void *kernel_ptr(int nt) {
  if (nt == 1024) return (void *)k_leaf<T, 1024>;
  if (nt == 512) return (void *)k_leaf<T, 512>;
  return (void *)k_leaf<T, 256>;
}

// The kernel attributes are process-wide state of the function: set them
// once per device, to the largest shared-memory size the device allows, so
// that handles set up concurrently (the server's slots) never lower the
// limit under another handle's launch.
template <typename T>
static amg_status leaf_attrs(int device, int optin, int nt, bool *nonportable, int *max_dynamic) {
  static std::mutex mu;
  static bool done[64][3], np_ok[64][3];
  static int dyn[64][3];
  if (device < 0 || device >= 64) return fail(AMG_ERR_CUDA, "device index out of range");
  const int v = nt == 1024 ? 2 : (nt == 512 ? 1 : 0);
  std::lock_guard<std::mutex> lk(mu);
  bool(&done_d)[3] = done[device];
  bool(&np_d)[3] = np_ok[device];
  int(&dyn_d)[3] = dyn[device];
  if (!done_d[v]) {
    void *kern = kernel_ptr<T>(nt);
    cudaFuncAttributes fa{};
    AMG_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    dyn_d[v] = optin - (int)fa.sharedSizeBytes;  // the kernel's static shared memory counts too
    AMG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_d[v]));
    np_d[v] = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    if (!np_d[v]) cudaGetLastError();
    done_d[v] = true;
  }
  *nonportable = np_d[v];
  *max_dynamic = dyn_d[v];
  return AMG_OK;
}

// threads per CTA of the leaf kernel: AMG_GB300_LEAF_THREADS=256|512|1024
static int leaf_threads() {
  if (const char *e = getenv("AMG_GB300_LEAF_THREADS")) {
    const int v = atoi(e);
    if (v == 256 || v == 512 || v == 1024) return v;
  }
  return kLeafDefaultThreads;
}

template <typename T>
static amg_status prepare_t(amg_handle_s *h, int k0) {
  const Level &L = h->lv[k0];
  const Level &N = h->lv[k0 + 1];
  const int n = L.n, nH = N.n;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> ap(nH + 1);
  AMG_CUDA_TRY(cudaMemcpyAsync(rp.data(), L.A.rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA_TRY(cudaMemcpyAsync(ap.data(), L.agg_ptr, sizeof(int32_t) * (nH + 1), cudaMemcpyDeviceToHost, h->stream));
  AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
  int optin = 0;
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
  const int nt = leaf_threads();
  void *kern = kernel_ptr<T>(nt);
  bool nonportable = false;
  int max_dynamic = 0;
  AMG_TRY(leaf_attrs<T>(h->device, optin, nt, &nonportable, &max_dynamic));
  for (int C : {kLeafMaxC, 8, 4, 2, 1}) {
    LeafParams<T> P{};
    P.n = n;
    P.nH = nH;
    P.C = C;
    P.R = (n + C - 1) / C;
    P.RH = (nH + C - 1) / C;
    P.m = h->opt.degree;
    P.nu = h->opt.inner_iters;
    P.nt = nt;
    int tpr = 8;
    while (tpr > 1 && P.R * tpr > nt) tpr >>= 1;
    // AMG_GB300_LEAF_TPR=1|2|4|8 overrides the lanes per row on level k0
    if (const char *e = getenv("AMG_GB300_LEAF_TPR")) {
      const int v = atoi(e);
      if (v == 1 || v == 2 || v == 4 || v == 8) tpr = v;
    }
    P.tpr = tpr;
    for (int c = 0; c < C; ++c) {
      const int a = std::min(n, c * P.R), b = std::min(n, (c + 1) * P.R);
      const int aH = std::min(nH, c * P.RH), bH = std::min(nH, (c + 1) * P.RH);
      P.maxnz = std::max(P.maxnz, (int)(rp[b] - rp[a]));
      P.maxmem = std::max(P.maxmem, ap[bH] - ap[aH]);
    }
    if (leaf_layout(P) > (unsigned)max_dynamic) continue;
    if (C > 8 && !nonportable) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = P.smem;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    P.two_sa = 4.0 / (L.lam1 - L.lam0);
    P.two_ca = 2.0 * (L.lam1 + L.lam0) / (L.lam1 - L.lam0);
    for (int j = 0; j <= P.m; ++j) P.coef[j] = (T)L.coef[j];
    P.rp = L.A.rowptr;
    P.col = L.A.col;
    P.val = L.A.val;
    P.diag = L.diag;
    P.agg = L.agg;
    P.agg_ptr = L.agg_ptr;
    P.agg_mem = L.agg_mem;
    // A_k0+1 B, once per setup
    double *AB = nullptr;
    AMG_TRY(h->arena.alloc((void **)&AB, sizeof(double) * (size_t)nH * nH));
    const int64_t nn = (int64_t)nH * nH;
    k_dense_ab<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(nH, N.A.rowptr, N.A.col, N.A.val, N.diag, h->Bd,
                                                                    AB);
    AMG_CUDA_TRY(cudaGetLastError());
    ++h->launches;
    // destination masks (AMG_GB300_LEAF_MASK=0: every row to every CTA)
    P.mask = nullptr;
    const char *menv = getenv("AMG_GB300_LEAF_MASK");
    if (!(menv && menv[0] == '0')) {
      std::vector<int32_t> col((size_t)std::max<int64_t>(rp[n], 1)), agg((size_t)n);
      AMG_CUDA_TRY(cudaMemcpyAsync(col.data(), L.A.col, sizeof(int32_t) * (size_t)rp[n], cudaMemcpyDeviceToHost,
                                   h->stream));
      AMG_CUDA_TRY(cudaMemcpyAsync(agg.data(), L.agg, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, h->stream));
      AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));
      std::vector<unsigned> mk((size_t)n, 0u);
      for (int i = 0; i < n; ++i) {
        unsigned v = (1u << (i / P.R)) | (1u << (agg[i] / P.RH));
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) v |= 1u << (col[e] / P.R);  // symmetric pattern
        mk[i] = v;
      }
      unsigned *dmask = nullptr;
      AMG_TRY(h->arena.alloc((void **)&dmask, sizeof(unsigned) * (size_t)n));
      AMG_CUDA_TRY(cudaMemcpyAsync(dmask, mk.data(), sizeof(unsigned) * (size_t)n, cudaMemcpyHostToDevice, h->stream));
      AMG_CUDA_TRY(cudaStreamSynchronize(h->stream));  // mk is released on return
      P.mask = dmask;
    }
    P.B = h->Bd;
    P.AB = AB;
    P.b = (const T *)L.b;
    P.x = (T *)L.x;
    {
      unsigned char *image = nullptr;
      AMG_TRY(h->arena.alloc((void **)&image, (size_t)P.static_bytes * C));
      k_leaf_image<T><<<C, 256, 0, h->stream>>>(P, image);
      AMG_CUDA_TRY(cudaGetLastError());
      ++h->launches;
      P.image = image;
    }
    P.prof = nullptr;
    if (const char *e = getenv("AMG_GB300_LEAF_PROFILE")) {
      if (e[0] == '1') {
        AMG_TRY(h->arena.alloc((void **)&P.prof, sizeof(unsigned long long) * kLeafProfSlots));
        AMG_CUDA_TRY(cudaMemsetAsync(P.prof, 0, sizeof(unsigned long long) * kLeafProfSlots, h->stream));
        h->leaf_prof = P.prof;
      }
    }
    LeafParams<T> *hp = new LeafParams<T>(P);
    h->leaf_params = hp;
    h->leaf_free = [](void *p) { delete static_cast<LeafParams<T> *>(p); };
    h->leaf_k = k0;
    h->leaf_csize = C;
    return AMG_OK;
  }
  return AMG_OK;  // nothing fits: the multi-kernel path stays in use
}

// Use the leaf kernel for the inner solve at level Bk - 1 when the level is
// small enough for every CTA to hold its vectors in shared memory.
// AMG_GB300_LEAF=0 keeps the multi-kernel path.
amg_status prepare_leaf(amg_handle_s *h) {
  h->leaf_k = -1;
  const char *env = getenv("AMG_GB300_LEAF");
  if (env && env[0] == '0') return AMG_OK;
  const int k0 = h->Bk - 1;
  if (h->Bk < 0 || k0 < 1 || h->opt.cycle != AMG_CYCLE_K) return AMG_OK;
  if (h->opt.inner_iters > kLeafMaxInner || h->opt.degree > kMaxDegree) return AMG_OK;
  if (h->lv[k0].n > kLeafMaxRows || h->lv[k0 + 1].n > kLeafMaxCoarse) return AMG_OK;
  if (h->opt.precision == AMG_PREC_FP32) return prepare_t<float>(h, k0);
  return prepare_t<double>(h, k0);
}

template <typename T>
static amg_status launch_t(amg_handle_s *h) {
  const LeafParams<T> &P = *static_cast<const LeafParams<T> *>(h->leaf_params);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3(P.C);
  cfg.blockDim = dim3(P.nt);
  cfg.dynamicSmemBytes = P.smem;
  cfg.stream = h->stream;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (P.nt == 1024) e = cudaLaunchKernelEx(&cfg, k_leaf<T, 1024>, P);
  else if (P.nt == 512) e = cudaLaunchKernelEx(&cfg, k_leaf<T, 512>, P);
  else e = cudaLaunchKernelEx(&cfg, k_leaf<T, 256>, P);
  ++h->launches;
  if (e != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("leaf kernel launch: ") + cudaGetErrorString(e));
  return AMG_OK;
}

// The opt-in phase profile, printed to stderr (average SM cycles per launch
// of the load phase and of every barrier-to-barrier phase of CTA 0).
void report_leaf_profile(amg_handle_s *h) {
  if (!h->leaf_prof) return;
  std::vector<unsigned long long> v(kLeafProfSlots, 0);
  if (cudaMemcpy(v.data(), h->leaf_prof, sizeof(unsigned long long) * kLeafProfSlots, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return;
  const double nl = (double)std::max<unsigned long long>(v[kLeafProfSlots - 1], 1);
  fprintf(stderr, "leaf profile: %llu launches, load %.0f cycles;", v[kLeafProfSlots - 1],
          v[kLeafProfSlots - 2] / nl);
  double tot = v[kLeafProfSlots - 2] / nl;
  for (int p = 0; p < kLeafProfSlots - 2 && v[p]; ++p) {
    fprintf(stderr, " %d:%.0f", p, v[p] / nl);
    tot += v[p] / nl;
  }
  fprintf(stderr, "; total %.0f cycles\n", tot);
}

amg_status launch_leaf(amg_handle_s *h) {
  if (h->opt.precision == AMG_PREC_FP32) return launch_t<float>(h);
  return launch_t<double>(h);
}

}  // namespace amg
