// krylov.cu -- right-preconditioned Bi-CGSTAB (van der Vorst 1992) and IDR(s) (Sonneveld &
// van Gijzen 2008), the Krylov methods of Section 6.2, and restarted GMRES(m) (Saad & Schultz
// 1986; the paper's remark on testing GMRES in Section 7), run entirely on the device.
//
// FP64 vectors and inner products; the V-cycle runs in the hierarchy's precision: the vector
// entering it is written in that precision by the update kernel that produces it (fused
// precision boundary), and its FP32 output is read directly by the FP64 matvec (exact upcast).
//
// Scalars (rho, alpha, omega, norms, status) live in a device struct.  Every inner product is
// reduced in the producing kernel: per-block partials, then the last block to finish (atomic
// ticket) sums the partials in a fixed order -- deterministic -- and updates the scalars.
// One iteration is captured once into a CUDA graph and driven by a conditional WHILE node
// whose condition the last kernel of the iteration sets, so a whole solve is one graph launch.
// No kernel waits on another: there is no device-side spin anywhere.
#include <cmath>
#include <cstddef>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <type_traits>

#include "stencil.cuh"
#include "krylov_state.cuh"

namespace helm {

static double host_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---- block reductions -------------------------------------------------------------------

// Sum K values over the block; thread 0 gets the totals.  Every thread's values go through shared
// memory and one warp sums each of them (KT / 32 terms a lane, then the warp's shuffle): about 24
// FP64 additions a lane on K warps, where shuffling all K sums on every warp costs 10 K on each of
// the KT / 32 warps -- at GB300's FP64 rate as much as the products of the few points a thread
// holds.  The order of the additions is fixed, so the sums are reproducible.
template <int K>
__device__ __forceinline__ void block_sum(double2 (&v)[K]) {
  __shared__ double2 sm[K][KT];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) sm[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int k = w; k < K; k += KT / 32) {
    double2 t = sm[k][lane];
#pragma unroll
    for (int q = 1; q < KT / 32; ++q) {
      t.x += sm[k][lane + 32 * q].x;
      t.y += sm[k][lane + 32 * q].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      t.x += __shfl_down_sync(0xffffffffu, t.x, o);
      t.y += __shfl_down_sync(0xffffffffu, t.y, o);
    }
    if (lane == 0) sm[k][0] = t;  // the warp's reads of row k are done (the shuffles synchronise it)
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = sm[k][0];
  __syncthreads();
}

// Stores this block's K partial sums, then returns true in the last block to arrive, where
// `tot` holds the grand totals (summed in a fixed order) on every thread.
// vb / vg: this block's index and the number of blocks among which the sum is split (the launch's
// grid, or the instance's share of a grouped launch).
template <int K>
__device__ bool reduce_last(double2 (&v)[K], double2* partials, unsigned int* ticket, double2 (&tot)[K], int vb,
                            int vg) {
  __shared__ bool last;
  __shared__ double2 res[K];
  block_sum<K>(v);
  int G = vg;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[k * G + vb] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == (unsigned int)G - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double2 a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    a[k] = mkc<double>(0.0, 0.0);
    for (int b = threadIdx.x; b < G; b += KT) {
      double2 pv = __ldcg(&partials[k * G + b]);
      a[k].x += pv.x;
      a[k].y += pv.y;
    }
  }
  block_sum<K>(a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) res[k] = a[k];
    *ticket = 0u;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = res[k];
  return true;
}

__device__ __forceinline__ bool finite2(double2 z) { return isfinite(z.x) && isfinite(z.y); }
__device__ __forceinline__ bool is_zero(double2 z) { return z.x == 0.0 && z.y == 0.0; }

__device__ __forceinline__ void record(KrylovState* S, double rn) {
  S->rel_recur = rn;
  if (S->hist && S->matvecs >= 1 && S->matvecs <= S->maxmv) S->hist[S->matvecs - 1] = rn;
}

__device__ __forceinline__ void finish(KrylovState* S, int status) {
  S->status = status;
  S->done = 1;
}

// Element i (natural order) of a V-cycle input in the multigrid precision, stored in level 0's
// order: x-split rows for an FP32 hierarchy whose finest level is x-split.
template <typename TM>
__device__ __forceinline__ void put_mg(const KrylovState* S, void* dst, long i, double2 v) {
  if (!dst) return;
  long q = i;
  if (std::is_same<TM, float>::value) {
    const int n0 = S->xs_n0;
    if (n0) {
      const long row = i < 0x7fffffffL ? (long)((unsigned)i / (unsigned)n0) : i / n0;
      const int x = (int)(i - row * n0);
      q = row * n0 + ((x & 1) ? S->xs_h + (x >> 1) : (x >> 1));
    }
  }
  reinterpret_cast<cx<TM>*>(dst)[q] = cconv<TM, double>(v);
}

// vb_ / vg_: the block's index and the block count of the instance (see VBLK and the bodies)
#define GRID_LOOP(i, n) for (long i = vb_ * (long)KT + threadIdx.x; i < (n); i += (long)vg_ * KT)
#define VBLK                                          \
  const int vb_ = blockIdx.x, vg_ = gridDim.x;        \
  (void)vb_;                                          \
  (void)vg_

// Stencil kernels walk warp-sized chunks of grid rows: a warp takes 32 consecutive points of
// one row (fixed j, l), so its loads are coalesced, only the last chunk of a row has idle lanes,
// and the index arithmetic costs one div/mod per chunk.
#define ROW_LOOP(H, i, j, l, p)                                                              \
  for (long ch_ = (vb_ * (long)KT + threadIdx.x) >> 5, nch_ = ((H).n[0] + 31) >> 5,          \
            nc_ = nch_ * (H).n[1] * (H).n[2];                                                 \
       ch_ < nc_; ch_ += ((long)vg_ * KT) >> 5)                                               \
    for (long row_ = ch_ / nch_, once_ = 1; once_; once_ = 0)                                 \
      for (int i = (int)(ch_ - row_ * nch_) * 32 + (threadIdx.x & 31), j = (int)(row_ % (H).n[1]), \
               l = (int)(row_ / (H).n[1]);                                                    \
           i < (H).n[0]; i = (H).n[0])                                                        \
        if (const long p = i + row_ * (H).n[0]; true)

// ---- shared kernels ----------------------------------------------------------------------

// Start (or restart) from the current residual r: ||r||, shadow r^ = r, p = v = 0 and
// rho = r^H r.  first: r = b and ||b|| sets the scale of the stopping rule.
__global__ void k_start(KrylovState* S, const double2* __restrict__ b, double2* r, double2* rh,
                        double2* p, double2* v, void* rmg, int mg32, long n, int first,
                        double2* partials) {
  pdl_entry();
  VBLK;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) {
    double2 ri = first ? b[i] : r[i];
    if (first) r[i] = ri;
    if (rh) rh[i] = ri;
    if (p) { p[i] = mkc<double>(0.0, 0.0); v[i] = mkc<double>(0.0, 0.0); }
    if (rmg) { if (mg32) put_mg<float>(S, rmg, i, ri); else put_mg<double>(S, rmg, i, ri); }
    acc[0].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[0].x));
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[0], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double rr = tot[0].x;
  if (first) {
    S->bnorm = sqrt(rr);
    S->matvecs = 0; S->iters = 0;
  }
  S->done = 0; S->half = 0; S->status = HELM_ERR_MAXIT;
  S->rho = mkc<double>(rr, 0.0);
  S->rho_old = S->alpha = S->omega = mkc<double>(1.0, 0.0);
  S->beta = S->rho;  // p = v = 0, so beta only multiplies zeros on the first step
  S->k = 0; S->oldest = 0;
  S->loops = 0;
  S->rel_recur = sqrt(rr) / S->bnorm;
  if (!isfinite(rr)) finish(S, HELM_ERR_NAN);
  else if (S->bnorm == 0.0) { S->rel_recur = 0.0; finish(S, HELM_OK); }
  else if (S->matvecs >= S->maxmv) finish(S, HELM_ERR_MAXIT);
}

// r = b - H x and ||r|| / ||b|| (the FP64 true residual that certifies convergence).
template <int DIM>
__global__ void k_true_res(KrylovState* S, OpView<double> H, const double2* __restrict__ b,
                           const double2* __restrict__ x, double2* __restrict__ r, long n, double2* partials) {
  pdl_entry();
  VBLK;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  ROW_LOOP(H, i, j, l, p) {
    double2 ri = csub<double>(b[p], op_row<double, double, DIM>(H, x, i, j, l, p));
    r[p] = ri;
    acc[0].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[0].x));
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[1], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  S->rel_true = S->bnorm > 0.0 ? sqrt(tot[0].x) / S->bnorm : 0.0;
}

// Sets the WHILE condition from `done`.  At the end of the body it also counts the body
// executions and, as a guard against a logic error, stops a loop that has run more bodies than
// the matvec cap allows (status HELM_ERR_TIMEOUT) -- every live body costs at least one matvec.
__global__ void k_set_cond(cudaGraphConditionalHandle h, KrylovState* S, int in_body) {
  pdl_entry();
  if (in_body) {
    S->loops += 1;
    if (!S->done && S->loops > S->maxmv + 16) finish(S, HELM_ERR_TIMEOUT);
  }
  cudaGraphSetConditional(h, S->done ? 0u : 1u);
}

// ---- Bi-CGSTAB -----------------------------------------------------------------------------

// p = r + beta (p - omega v); its copy in multigrid precision feeds the V-cycle.
template <typename TM>
__device__ __forceinline__ void bicg_p_body(int vb_, int vg_, const KrylovState* S, const double2* __restrict__ r, double2* __restrict__ p,
                         const double2* __restrict__ v, void* pmg, long n) {
  if (S->done) return;
  const double2 beta = S->beta;
  const double2 mbw = cmul<double>(mkc<double>(-beta.x, -beta.y), S->omega);  // -beta omega
  GRID_LOOP(i, n) {
    double2 pi = cfma<double>(mbw, v[i], cfma<double>(beta, p[i], r[i]));  // r + beta (p - omega v)
    p[i] = pi;
    put_mg<TM>(S, pmg, i, pi);
  }
}
template <typename TM>
__global__ void k_bicg_p(const KrylovState* S, const double2* __restrict__ r, double2* __restrict__ p,
                         const double2* __restrict__ v, void* pmg, long n) {
  pdl_entry();
  bicg_p_body<TM>(blockIdx.x, gridDim.x, S, r, p, v, pmg, n);
}

// v = H p^ and alpha = rho / (r^H v).
template <int DIM>
__device__ __forceinline__ void bicg_v_body(int vb_, int vg_, KrylovState* S, const OpView<double>& H, const double2* __restrict__ ph,
                         const double2* __restrict__ rh, double2* __restrict__ v, long n, double2* partials) {
  if (S->done) return;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  ROW_LOOP(H, i, j, l, p) {
    double2 vi = op_row<double, double, DIM>(H, ph, i, j, l, p);
    v[p] = vi;
    acc[0] = cfmac<double>(rh[p], vi, acc[0]);
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[2], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  S->matvecs += 1;
  S->iters += 1;
  double2 rv = tot[0];
  if (!finite2(rv)) { finish(S, HELM_ERR_NAN); return; }
  if (is_zero(rv)) { finish(S, HELM_ERR_BREAKDOWN); return; }
  S->alpha = cdiv<double>(S->rho, rv);
}
template <int DIM>
__global__ void k_bicg_v(KrylovState* S, OpView<double> H, const double2* __restrict__ ph,
                         const double2* __restrict__ rh, double2* __restrict__ v, long n, double2* partials) {
  pdl_entry();
  bicg_v_body<DIM>(blockIdx.x, gridDim.x, S, H, ph, rh, v, n, partials);
}

// s = r - alpha v, ||s||; stop after the half step if ||s|| / ||b|| < tol (or at the cap).
template <typename TM>
__device__ __forceinline__ void bicg_s_body(int vb_, int vg_, KrylovState* S, const double2* __restrict__ r, const double2* __restrict__ v,
                         double2* __restrict__ sv, void* smg, long n, double2* partials) {
  if (S->done) return;
  const double2 mal = mkc<double>(-S->alpha.x, -S->alpha.y);
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) {
    double2 si = cfma<double>(mal, v[i], r[i]);  // r - alpha v
    sv[i] = si;
    put_mg<TM>(S, smg, i, si);
    acc[0].x = fma(si.x, si.x, fma(si.y, si.y, acc[0].x));
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[3], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double sn = sqrt(tot[0].x) / S->bnorm;
  record(S, sn);
  if (!isfinite(sn)) { finish(S, HELM_ERR_NAN); return; }
  if (sn < S->tol) { S->half = 1; finish(S, HELM_OK); return; }
  if (S->matvecs >= S->maxmv) { S->half = 1; finish(S, HELM_ERR_MAXIT); }
}
template <typename TM>
__global__ void k_bicg_s(KrylovState* S, const double2* __restrict__ r, const double2* __restrict__ v,
                         double2* __restrict__ sv, void* smg, long n, double2* partials) {
  pdl_entry();
  bicg_s_body<TM>(blockIdx.x, gridDim.x, S, r, v, sv, smg, n, partials);
}

// x += alpha p^ after a half-step exit.
__device__ __forceinline__ void bicg_xhalf_body(int vb_, int vg_, KrylovState* S, const double2* __restrict__ ph, double2* __restrict__ x, long n) {
  if (S->half != 1) return;  // 2: a grouped loop applied it in an earlier body
  double2 al = S->alpha;
  GRID_LOOP(i, n) x[i] = cfma<double>(al, ph[i], x[i]);
}
__global__ void k_bicg_xhalf(KrylovState* S, const double2* __restrict__ ph, double2* __restrict__ x, long n) {
  pdl_entry();
  bicg_xhalf_body(blockIdx.x, gridDim.x, S, ph, x, n);
}

// t = H s^, omega = (t^H s) / (t^H t).
template <int DIM>
__device__ __forceinline__ void bicg_t_body(int vb_, int vg_, KrylovState* S, const OpView<double>& H, const double2* __restrict__ sh,
                         const double2* __restrict__ sv, double2* __restrict__ t, long n, double2* partials) {
  if (S->done) return;
  double2 acc[2] = {mkc<double>(0.0, 0.0), mkc<double>(0.0, 0.0)};
  ROW_LOOP(H, i, j, l, p) {
    double2 ti = op_row<double, double, DIM>(H, sh, i, j, l, p);
    t[p] = ti;
    acc[0] = cfmac<double>(ti, sv[p], acc[0]);
    acc[1].x = fma(ti.x, ti.x, fma(ti.y, ti.y, acc[1].x));
  }
  double2 tot[2];
  if (!reduce_last<2>(acc, partials, &S->ticket[4], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  S->matvecs += 1;
  double tt = tot[1].x;
  if (!isfinite(tt) || !finite2(tot[0])) { finish(S, HELM_ERR_NAN); return; }
  if (tt == 0.0) { finish(S, HELM_ERR_BREAKDOWN); return; }
  S->omega = cscale<double>(1.0 / tt, tot[0]);
}
template <int DIM>
__global__ void k_bicg_t(KrylovState* S, OpView<double> H, const double2* __restrict__ sh,
                         const double2* __restrict__ sv, double2* __restrict__ t, long n, double2* partials) {
  pdl_entry();
  bicg_t_body<DIM>(blockIdx.x, gridDim.x, S, H, sh, sv, t, n, partials);
}

// x += alpha p^ + omega s^; r = s - omega t; ||r||, rho = r^H r and the next beta.
__device__ __forceinline__ void bicg_xr_body(int vb_, int vg_, KrylovState* S, const double2* __restrict__ ph, const double2* __restrict__ sh,
                          const double2* __restrict__ sv, const double2* __restrict__ t,
                          const double2* __restrict__ rh, double2* __restrict__ x, double2* __restrict__ r,
                          long n, double2* partials) {
  if (S->done) return;
  double2 al = S->alpha, om = S->omega;
  const double2 mom = mkc<double>(-om.x, -om.y);
  double2 acc[2] = {mkc<double>(0.0, 0.0), mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) {
    x[i] = cfma<double>(om, sh[i], cfma<double>(al, ph[i], x[i]));
    double2 ri = cfma<double>(mom, t[i], sv[i]);  // s - omega t
    r[i] = ri;
    acc[0].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[0].x));
    acc[1] = cfmac<double>(rh[i], ri, acc[1]);
  }
  double2 tot[2];
  if (!reduce_last<2>(acc, partials, &S->ticket[5], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double rn = sqrt(tot[0].x) / S->bnorm;
  record(S, rn);
  if (!isfinite(rn)) { finish(S, HELM_ERR_NAN); return; }
  if (rn < S->tol) { finish(S, HELM_OK); return; }
  if (is_zero(om)) { finish(S, HELM_ERR_BREAKDOWN); return; }
  if (S->matvecs >= S->maxmv) { finish(S, HELM_ERR_MAXIT); return; }
  double2 rho = tot[1];
  if (!finite2(rho)) { finish(S, HELM_ERR_NAN); return; }
  if (is_zero(rho)) { finish(S, HELM_ERR_BREAKDOWN); return; }
  S->rho_old = S->rho;
  S->rho = rho;
  S->beta = cmul<double>(cdiv<double>(rho, S->rho_old), cdiv<double>(S->alpha, om));
}
__global__ void k_bicg_xr(KrylovState* S, const double2* __restrict__ ph, const double2* __restrict__ sh,
                          const double2* __restrict__ sv, const double2* __restrict__ t,
                          const double2* __restrict__ rh, double2* __restrict__ x, double2* __restrict__ r,
                          long n, double2* partials) {
  pdl_entry();
  bicg_xr_body(blockIdx.x, gridDim.x, S, ph, sh, sv, t, rh, x, r, n, partials);
}

// ---- grouped Bi-CGSTAB: one launch per kernel for many instances ---------------------------
// The blocks of a grouped launch walk its work list (group_visit): virtual block vb of instance d is
// block vb of d's own G-block launch, so every point, partial sum and reduction order is the one
// the instance has alone.

template <typename TM>
__global__ void kg_bicg_p(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    // the loop body runs for this instance: count it (the single-instance loop does this in its
    // condition kernel)
    if (vb == 0 && threadIdx.x == 0 && !g.S->done) g.S->loops += 1;
    bicg_p_body<TM>(vb, g.G, g.S, g.r, g.p, g.v, g.pmg, g.n);
  });
}

template <int DIM>
__global__ void kg_bicg_v(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    bicg_v_body<DIM>(vb, g.G, g.S, g.H, g.ph, g.rh, g.v, g.n, g.partials);
  });
}

template <typename TM>
__global__ void kg_bicg_s(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    bicg_s_body<TM>(vb, g.G, g.S, g.r, g.v, g.sv, g.smg, g.n, g.partials);
  });
}

__global__ void kg_bicg_xhalf(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    bicg_xhalf_body(vb, g.G, g.S, g.ph, g.x, g.n);
  });
}

template <int DIM>
__global__ void kg_bicg_t(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    bicg_t_body<DIM>(vb, g.G, g.S, g.H, g.sh, g.sv, g.t, g.n, g.partials);
  });
}

__global__ void kg_bicg_xr(const GroupBicg* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GroupBicg& g = A[d];
    bicg_xr_body(vb, g.G, g.S, g.ph, g.sh, g.sv, g.t, g.rh, g.x, g.r, g.n, g.partials);
  });
}

template <typename TM>
void group_krylov_launch(int which, const GroupBicg* A, const GroupList* LT, int li, int grid, cudaStream_t st) {
  switch (which) {
    case GK_P: launch_pdl(kg_bicg_p<TM>, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
    case GK_V: launch_pdl(kg_bicg_v<2>, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
    case GK_S: launch_pdl(kg_bicg_s<TM>, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
    case GK_XHALF: launch_pdl(kg_bicg_xhalf, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
    case GK_T: launch_pdl(kg_bicg_t<2>, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
    default: launch_pdl(kg_bicg_xr, dim3(grid), dim3(KT), 0, st, A, LT, li); break;
  }
}
template void group_krylov_launch<float>(int, const GroupBicg*, const GroupList*, int, int, cudaStream_t);
template void group_krylov_launch<double>(int, const GroupBicg*, const GroupList*, int, int, cudaStream_t);


// ---- IDR(s) -------------------------------------------------------------------------------

// out_i = P_i^H y for i < s (one pass over y).  Used for the shadow-space projections.
template <int S_>
__device__ __forceinline__ void proj_acc(const double2* __restrict__ P, long n, long i, double2 y, double2* acc) {
#pragma unroll
  for (int k = 0; k < S_; ++k) acc[k] = cfmac<double>(P[k * n + i], y, acc[k]);
}

// Minimal-residual start step k: t = H z, omega = (t^H r) / (t^H t).
template <int DIM>
__global__ void k_idr_mr_t(KrylovState* S, OpView<double> H, const double2* __restrict__ z,
                           const double2* __restrict__ r, double2* __restrict__ t, long n, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  double2 acc[2] = {mkc<double>(0.0, 0.0), mkc<double>(0.0, 0.0)};
  ROW_LOOP(H, i, j, l, p) {
    double2 ti = op_row<double, double, DIM>(H, z, i, j, l, p);
    t[p] = ti;
    acc[0] = cfmac<double>(ti, r[p], acc[0]);
    acc[1].x = fma(ti.x, ti.x, fma(ti.y, ti.y, acc[1].x));
  }
  double2 tot[2];
  if (!reduce_last<2>(acc, partials, &S->ticket[2], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  S->matvecs += 1;
  S->iters += 1;
  double tt = tot[1].x;
  if (!isfinite(tt)) { finish(S, HELM_ERR_NAN); return; }
  if (tt == 0.0) { finish(S, HELM_ERR_BREAKDOWN); return; }
  S->omega = cscale<double>(1.0 / tt, tot[0]);
}

// dX_k = omega z, dR_k = -omega t, x += dX_k, r += dR_k, ||r||.
template <typename TM>
__global__ void k_idr_mr_upd(KrylovState* S, int kcol, const double2* __restrict__ z, const double2* __restrict__ t,
                             double2* __restrict__ dX, double2* __restrict__ dR, double2* __restrict__ x,
                             double2* __restrict__ r, void* rmg, long n, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  double2 om = S->omega;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) {
    double2 dx = cmul<double>(om, z[i]);
    double2 dr = cmul<double>(om, t[i]);
    dr = mkc<double>(-dr.x, -dr.y);
    dX[kcol * n + i] = dx;
    dR[kcol * n + i] = dr;
    x[i] = cadd<double>(x[i], dx);
    double2 ri = cadd<double>(r[i], dr);
    r[i] = ri;
    put_mg<TM>(S, rmg, i, ri);
    acc[0].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[0].x));
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[3], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double rn = sqrt(tot[0].x) / S->bnorm;
  record(S, rn);
  if (!isfinite(rn)) { finish(S, HELM_ERR_NAN); return; }
  if (rn < S->tol) { finish(S, HELM_OK); return; }
  if (S->matvecs >= S->maxmv) finish(S, HELM_ERR_MAXIT);
}

// Projections onto the shadow space: column `col` of M = P^H dR_col, or m = P^H r (col < 0).
template <int S_>
__global__ void k_idr_proj(KrylovState* S, const double2* __restrict__ P, const double2* __restrict__ y,
                           int col, long n, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  double2 acc[S_];
#pragma unroll
  for (int k = 0; k < S_; ++k) acc[k] = mkc<double>(0.0, 0.0);
  GRID_LOOP(i, n) proj_acc<S_>(P, n, i, y[i], acc);
  double2 tot[S_];
  if (!reduce_last<S_>(acc, partials, &S->ticket[6], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  for (int k = 0; k < S_; ++k) {
    if (col >= 0) S->M[k + S_ * col] = tot[k];
    else S->m[k] = tot[k];
  }
}

// c = M^{-1} m (s x s, Gaussian elimination with partial pivoting, one thread).
__global__ void k_idr_small(KrylovState* S) {
  pdl_entry();
  if (S->done || threadIdx.x) return;
  if (S->matvecs >= S->maxmv) { finish(S, HELM_ERR_MAXIT); return; }
  int s = S->s;
  double2 A[SMAX][SMAX], b[SMAX];
  for (int i = 0; i < s; ++i) {
    b[i] = S->m[i];
    for (int j = 0; j < s; ++j) A[i][j] = S->M[i + s * j];
  }
  for (int k = 0; k < s; ++k) {
    int pv = k;
    for (int rr = k + 1; rr < s; ++rr)
      if (cabs2<double>(A[rr][k]) > cabs2<double>(A[pv][k])) pv = rr;
    if (is_zero(A[pv][k])) { finish(S, HELM_ERR_BREAKDOWN); return; }
    if (pv != k) {
      for (int j = 0; j < s; ++j) { double2 tt = A[k][j]; A[k][j] = A[pv][j]; A[pv][j] = tt; }
      double2 tt = b[k]; b[k] = b[pv]; b[pv] = tt;
    }
    for (int rr = k + 1; rr < s; ++rr) {
      double2 f = cdiv<double>(A[rr][k], A[k][k]);
      for (int j = k; j < s; ++j) A[rr][j] = csub<double>(A[rr][j], cmul<double>(f, A[k][j]));
      b[rr] = csub<double>(b[rr], cmul<double>(f, b[k]));
    }
  }
  for (int rr = s - 1; rr >= 0; --rr) {
    double2 acc = b[rr];
    for (int j = rr + 1; j < s; ++j) acc = csub<double>(acc, cmul<double>(A[rr][j], S->c[j]));
    S->c[rr] = cdiv<double>(acc, A[rr][rr]);
  }
}

// q = -dR c, v = r + q (and v in multigrid precision).
template <typename TM, int S_>
__global__ void k_idr_v(const KrylovState* S, const double2* __restrict__ dR, const double2* __restrict__ r,
                        double2* __restrict__ q, void* vmg, long n) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  double2 c[S_];
#pragma unroll
  for (int k = 0; k < S_; ++k) c[k] = S->c[k];
  GRID_LOOP(i, n) {
    double2 acc = mkc<double>(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < S_; ++k) acc = cfms<double>(dR[k * n + i], c[k], acc);
    q[i] = acc;
    put_mg<TM>(S, vmg, i, cadd<double>(r[i], acc));
  }
}

// First step of a cycle (k == 0): t = H z, omega = (t^H v) / (t^H t), v = r + q.
template <int DIM>
__global__ void k_idr_t0(KrylovState* S, OpView<double> H, const double2* __restrict__ z,
                         const double2* __restrict__ r, const double2* __restrict__ q,
                         double2* __restrict__ t, long n, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done || S->k != 0) return;
  double2 acc[2] = {mkc<double>(0.0, 0.0), mkc<double>(0.0, 0.0)};
  ROW_LOOP(H, i, j, l, p) {
    double2 ti = op_row<double, double, DIM>(H, z, i, j, l, p);
    t[p] = ti;
    acc[0] = cfmac<double>(ti, cadd<double>(r[p], q[p]), acc[0]);
    acc[1].x = fma(ti.x, ti.x, fma(ti.y, ti.y, acc[1].x));
  }
  double2 tot[2];
  if (!reduce_last<2>(acc, partials, &S->ticket[4], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double tt = tot[1].x;
  if (!isfinite(tt) || !finite2(tot[0])) { finish(S, HELM_ERR_NAN); return; }
  if (tt == 0.0) { finish(S, HELM_ERR_BREAKDOWN); return; }
  S->omega = cscale<double>(1.0 / tt, tot[0]);
}

// dX_oldest = -dX c + omega z (in place: each entry reads its row of dX before writing).
template <int S_>
__global__ void k_idr_dx(const KrylovState* S, double2* __restrict__ dX, const double2* __restrict__ z, long n) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  double2 c[S_];
#pragma unroll
  for (int k = 0; k < S_; ++k) c[k] = S->c[k];
  double2 om = S->omega;
  int o = S->oldest;
  GRID_LOOP(i, n) {
    double2 acc = cmul<double>(om, z[i]);
#pragma unroll
    for (int k = 0; k < S_; ++k) acc = cfms<double>(dX[k * n + i], c[k], acc);
    dX[o * n + i] = acc;
  }
}

// Later steps (k > 0): t = H dX_oldest.
template <int DIM>
__global__ void k_idr_tk(const KrylovState* S, OpView<double> H, const double2* __restrict__ dX,
                         double2* __restrict__ t, long n) {
  pdl_entry();
  VBLK;
  if (S->done || S->k == 0) return;
  const double2* d = dX + S->oldest * n;
  ROW_LOOP(H, i, j, l, p) {
    t[p] = op_row<double, double, DIM>(H, d, i, j, l, p);
  }
}

// dR_oldest = (k == 0 ? q - omega t : -t); r += dR_oldest; x += dX_oldest; ||r||;
// dm = P^H dR_oldest updates M and m; advance oldest and k.
template <int S_>
__global__ void k_idr_upd(KrylovState* S, const double2* __restrict__ P, double2* __restrict__ dR,
                          const double2* __restrict__ dX, const double2* __restrict__ q,
                          const double2* __restrict__ t, double2* __restrict__ x, double2* __restrict__ r,
                          long n, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  int o = S->oldest;
  bool first = S->k == 0;
  double2 om = S->omega;
  double2 acc[S_ + 1];
#pragma unroll
  for (int k = 0; k <= S_; ++k) acc[k] = mkc<double>(0.0, 0.0);
  GRID_LOOP(i, n) {
    double2 ti = t[i];
    double2 dr = first ? cfms<double>(om, ti, q[i]) : mkc<double>(-ti.x, -ti.y);
    dR[o * n + i] = dr;
    double2 ri = cadd<double>(r[i], dr);
    r[i] = ri;
    x[i] = cadd<double>(x[i], dX[o * n + i]);
    acc[S_].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[S_].x));
    proj_acc<S_>(P, n, i, dr, acc);
  }
  double2 tot[S_ + 1];
  if (!reduce_last<S_ + 1>(acc, partials, &S->ticket[5], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  S->matvecs += 1;
  S->iters += 1;
  double rn = sqrt(tot[S_].x) / S->bnorm;
  record(S, rn);
  if (!isfinite(rn)) { finish(S, HELM_ERR_NAN); return; }
  if (rn < S->tol) { finish(S, HELM_OK); return; }
  for (int k = 0; k < S_; ++k) {
    S->M[k + S_ * o] = tot[k];
    S->m[k] = cadd<double>(S->m[k], tot[k]);
  }
  S->oldest = (o + 1) % S_;
  S->k = (S->k + 1) % (S_ + 1);
}

// Modified Gram-Schmidt on the shadow vectors: h = P_i^H P_j ...
__global__ void k_dot1(KrylovState* S, const double2* __restrict__ a, const double2* __restrict__ b,
                       long n, double2* partials, double2* out) {
  pdl_entry();
  VBLK;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) acc[0] = cfmac<double>(a[i], b[i], acc[0]);
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[7], tot, vb_, vg_)) return;
  if (threadIdx.x == 0) *out = tot[0];
}
// ... P_j -= h P_i  (mode 0)  or  P_j /= sqrt(h)  (mode 1, h = P_j^H P_j)
__global__ void k_mgs_upd(double2* __restrict__ pj, const double2* __restrict__ pi, const double2* h, int mode, long n) {
  pdl_entry();
  VBLK;
  double2 hv = *h;
  double sc = mode ? 1.0 / sqrt(hv.x) : 0.0;
  GRID_LOOP(i, n) {
    if (mode) pj[i] = cscale<double>(sc, pj[i]);
    else pj[i] = csub<double>(pj[i], cmul<double>(hv, pi[i]));
  }
}

// ---- GMRES(m) --------------------------------------------------------------------------------
// One loop body is one Arnoldi step j = S->k: z = M^{-1} v_j (V-cycle), w = H z, two classical
// Gram-Schmidt passes (all inner products v_i^H w first, then one update), h_{j+1,j} = ||w||,
// the complex Givens rotations that keep the Hessenberg matrix triangular, and v_{j+1} = w / h.
// The cycle ends (done) when the rotated right-hand side shows ||r|| / ||b|| < tol, at step m or
// at the matvec cap; then y solves R y = g and x += M^{-1} (V y), and the pass's true residual
// starts the next cycle.

struct GmView {
  double2 *Hs, *cs, *sn, *g, *y, *hA, *hB;  // Hs[i + (m+1) j]; cs holds reals in .x
};
__host__ __device__ inline GmView gm_view(double2* base, int m) {
  GmView v;
  v.Hs = base;
  v.cs = v.Hs + (size_t)(m + 1) * m;
  v.sn = v.cs + m;
  v.g = v.sn + m;
  v.y = v.g + m + 1;
  v.hA = v.y + m;
  v.hB = v.hA + m + 1;
  return v;
}
inline size_t gm_elems(int m) { return (size_t)(m + 1) * m + 6 * (size_t)m + 3; }

// Cycle start from r (first pass: r = b, whose norm sets the scale): beta = ||r||, g = (beta, 0..).
__global__ void k_gm_start(KrylovState* S, const double2* __restrict__ b, double2* r, long n, int first,
                           double2* partials) {
  pdl_entry();
  VBLK;
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(i, n) {
    double2 ri = first ? b[i] : r[i];
    if (first) r[i] = ri;
    acc[0].x = fma(ri.x, ri.x, fma(ri.y, ri.y, acc[0].x));
  }
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[0], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  double beta = sqrt(tot[0].x);
  if (first) {
    S->bnorm = beta;
    S->matvecs = 0; S->iters = 0;
  }
  S->done = 0; S->half = 0; S->status = HELM_ERR_MAXIT;
  S->k = 0; S->loops = 0;
  S->beta = mkc<double>(beta, 0.0);
  GmView G = gm_view(S->gm, S->gmm);
  G.g[0] = mkc<double>(beta, 0.0);
  for (int i = 1; i <= S->gmm; ++i) G.g[i] = mkc<double>(0.0, 0.0);
  S->rel_recur = S->bnorm > 0.0 ? beta / S->bnorm : 0.0;
  if (!isfinite(beta)) finish(S, HELM_ERR_NAN);
  else if (S->bnorm == 0.0) { S->rel_recur = 0.0; finish(S, HELM_OK); }
  else if (beta / S->bnorm < S->tol) finish(S, HELM_OK);
  else if (S->matvecs >= S->maxmv) finish(S, HELM_ERR_MAXIT);
}

// v_0 = r / beta, and its copy in multigrid precision (the first V-cycle's input)
template <typename TM>
__global__ void k_gm_v0(const KrylovState* S, const double2* __restrict__ r, double2* __restrict__ V, void* vmg,
                        long n) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  const double beta = S->beta.x;
  GRID_LOOP(i, n) {
    double2 v = mkc<double>(r[i].x / beta, r[i].y / beta);
    V[i] = v;
    put_mg<TM>(S, vmg, i, v);
  }
}

// w = H z (z = M^{-1} v_j)
template <int DIM>
__global__ void k_gm_w(const KrylovState* S, OpView<double> H, const double2* __restrict__ z,
                       double2* __restrict__ w, long n) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  ROW_LOOP(H, i, j, l, p) w[p] = op_row<double, double, DIM>(H, z, i, j, l, p);
}

// h_i = v_i^H w for i = 0..j: each block takes a contiguous slice of the points, so that its
// slice of w stays in cache over the chunks of 8 basis vectors; the last block to finish adds
// the per-block partials in block order (deterministic).
// The block's 8 sums of a chunk go through shared memory, one warp per sum (8 sequential terms
// per lane, then 5 shuffle levels): a slice holds only a few points per thread, and a shuffle
// reduction of all 8 sums on every lane would cost as many FP64 additions as the products.
__global__ void k_gm_dots(KrylovState* S, const double2* __restrict__ V, const double2* __restrict__ w, long n,
                          double2* partials, double2* h, int tk) {
  static_assert(KT == 256, "one warp per chunk sum");
  pdl_entry();
  if (S->done) return;
  __shared__ double2 red[8][KT];
  const int j = S->k;
  const int G = gridDim.x;
  const long L = (n + G - 1) / G;
  const long beg = blockIdx.x * L, end = beg + L < n ? beg + L : n;
  const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i0 = 0; i0 <= j; i0 += 8) {
    double2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = mkc<double>(0.0, 0.0);
    for (long p = beg + threadIdx.x; p < end; p += KT) {
      const double2 wp = w[p];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q <= j) acc[q] = cfmac<double>(V[(size_t)(i0 + q) * n + p], wp, acc[q]);
    }
    __syncthreads();  // the previous chunk's readers are done with red
#pragma unroll
    for (int q = 0; q < 8; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    double2 t = mkc<double>(0.0, 0.0);
#pragma unroll
    for (int k = lane; k < KT; k += 32) {
      t.x += red[wq][k].x;
      t.y += red[wq][k].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      t.x += __shfl_down_sync(0xffffffffu, t.x, o);
      t.y += __shfl_down_sync(0xffffffffu, t.y, o);
    }
    if (lane == 0 && i0 + wq <= j) partials[(size_t)(i0 + wq) * G + blockIdx.x] = t;
  }
  // the partials were written by lane 0 of every warp: each fences its own writes, and the block
  // barrier orders them before the ticket
  __threadfence();
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&S->ticket[tk], 1u) == (unsigned int)G - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i <= j; i += KT) {
    double2 t = mkc<double>(0.0, 0.0);
    for (int bk = 0; bk < G; ++bk) {
      double2 pv = __ldcg(&partials[(size_t)i * G + bk]);
      t.x += pv.x;
      t.y += pv.y;
    }
    h[i] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) S->ticket[tk] = 0u;
}

// End of an Arnoldi step (one thread): the new Hessenberg column h = hA + hB, the earlier
// rotations on it, the rotation that annihilates h_{j+1,j} = hn, the rotated right-hand side and
// the stopping tests.
__device__ void gm_step_end(KrylovState* S, double hn) {
  const int j = S->k, m = S->gmm;
  GmView G = gm_view(S->gm, m);
  double2* col = G.Hs + (size_t)(m + 1) * j;
  for (int i = 0; i <= j; ++i) col[i] = cadd<double>(G.hA[i], G.hB[i]);
  for (int i = 0; i < j; ++i) {
    const double c = G.cs[i].x;
    const double2 sn = G.sn[i], a = col[i], b = col[i + 1];
    col[i] = cfma<double>(sn, b, cscale<double>(c, a));                                   // c a + s b
    col[i + 1] = csub<double>(cscale<double>(c, b), cmul<double>(mkc<double>(sn.x, -sn.y), a));  // -conj(s) a + c b
  }
  const double2 a = col[j];
  const double aa = hypot(a.x, a.y);
  if (hn == 0.0) {
    G.cs[j] = mkc<double>(1.0, 0.0);
    G.sn[j] = mkc<double>(0.0, 0.0);
  } else if (aa == 0.0) {
    G.cs[j] = mkc<double>(0.0, 0.0);
    G.sn[j] = mkc<double>(1.0, 0.0);
    col[j] = mkc<double>(hn, 0.0);
  } else {
    const double t = hypot(aa, hn);
    const double2 ph = mkc<double>(a.x / aa, a.y / aa);
    G.cs[j] = mkc<double>(aa / t, 0.0);
    G.sn[j] = cscale<double>(hn / t, ph);
    col[j] = cscale<double>(t, ph);
  }
  col[j + 1] = mkc<double>(0.0, 0.0);
  const double2 sn = G.sn[j], gj = G.g[j];
  G.g[j + 1] = cmul<double>(mkc<double>(-sn.x, sn.y), gj);  // -conj(s) g_j
  G.g[j] = cscale<double>(G.cs[j].x, gj);
  S->matvecs += 1;
  S->iters += 1;
  const double est = hypot(G.g[j + 1].x, G.g[j + 1].y) / S->bnorm;
  record(S, est);
  S->hn = hn;
  S->k = j + 1;
  if (!isfinite(est) || !isfinite(hn)) finish(S, HELM_ERR_NAN);
  else if (est < S->tol || hn == 0.0) finish(S, HELM_OK);
  else if (j + 1 == m || S->matvecs >= S->maxmv) finish(S, HELM_ERR_MAXIT);
}

// w -= sum_{i<=j} h_i v_i (one Gram-Schmidt update); after the second pass (`final`) also ||w||
// and the end of the Arnoldi step.
__global__ void k_gm_sub(KrylovState* S, const double2* __restrict__ V, double2* __restrict__ w,
                         const double2* __restrict__ h, long n, int final, double2* partials) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  __shared__ double2 hs[GMRES_MMAX + 1];
  const int j = S->k;
  for (int i = threadIdx.x; i <= j; i += KT) hs[i] = h[i];
  __syncthreads();
  double2 acc[1] = {mkc<double>(0.0, 0.0)};
  GRID_LOOP(p, n) {
    double2 u = mkc<double>(0.0, 0.0);
    for (int i = 0; i <= j; ++i) u = cfma<double>(hs[i], V[(size_t)i * n + p], u);
    const double2 wp = csub<double>(w[p], u);
    w[p] = wp;
    acc[0].x = fma(wp.x, wp.x, fma(wp.y, wp.y, acc[0].x));
  }
  if (!final) return;
  double2 tot[1];
  if (!reduce_last<1>(acc, partials, &S->ticket[5], tot, vb_, vg_)) return;
  if (threadIdx.x) return;
  gm_step_end(S, sqrt(tot[0].x));
}

// v_{j+1} = w / h_{j+1,j} and its copy in multigrid precision (the next step's V-cycle input)
template <typename TM>
__global__ void k_gm_next(const KrylovState* S, const double2* __restrict__ w, double2* __restrict__ V, void* vmg,
                          long n) {
  pdl_entry();
  VBLK;
  if (S->done) return;
  const double hn = S->hn;
  double2* vk = V + (size_t)S->k * n;
  GRID_LOOP(i, n) {
    double2 v = mkc<double>(w[i].x / hn, w[i].y / hn);
    vk[i] = v;
    put_mg<TM>(S, vmg, i, v);
  }
}

// R y = g by back substitution over the k = S->k columns of the cycle (one thread)
__global__ void k_gm_y(KrylovState* S) {
  pdl_entry();
  if (threadIdx.x) return;
  const int k = S->k, m = S->gmm;
  GmView G = gm_view(S->gm, m);
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = G.g[i];
    for (int l = i + 1; l < k; ++l) acc = cfms<double>(G.Hs[i + (size_t)(m + 1) * l], G.y[l], acc);
    G.y[i] = cdiv<double>(acc, G.Hs[i + (size_t)(m + 1) * i]);
  }
}

// u = sum_{i<k} y_i v_i, written in multigrid precision as the V-cycle input (and in FP64 when
// there is no preconditioner, where it is the correction itself)
template <typename TM>
__global__ void k_gm_comb(const KrylovState* S, const double2* __restrict__ V, void* umg, double2* u64, long n) {
  pdl_entry();
  VBLK;
  __shared__ double2 ys[GMRES_MMAX];
  const int k = S->k;
  GmView G = gm_view(S->gm, S->gmm);
  for (int i = threadIdx.x; i < k; i += KT) ys[i] = G.y[i];
  __syncthreads();
  GRID_LOOP(p, n) {
    double2 u = mkc<double>(0.0, 0.0);
    for (int i = 0; i < k; ++i) u = cfma<double>(ys[i], V[(size_t)i * n + p], u);
    put_mg<TM>(S, umg, p, u);
    if (u64) u64[p] = u;
  }
}

// x += z
__global__ void k_gm_addx(const KrylovState* S, const double2* __restrict__ z, double2* __restrict__ x, long n) {
  pdl_entry();
  VBLK;
  if (S->k == 0) return;
  GRID_LOOP(i, n) x[i] = cadd<double>(x[i], z[i]);
}

// ---- host orchestration ---------------------------------------------------------------------

static helm_status ws_alloc(helm_ctx* c, Workspace* w, void** p, size_t bytes, cudaStream_t st) {
  DevBlock b;
  helm_status s = dev_alloc(p, bytes, st, &b);
  if (s != HELM_OK) {
    set_error("device allocation failed for the Krylov workspace");
    return s;
  }
  w->mem.push_back(b);
  w->bytes += bytes;
  c->bytes += bytes;
  return HELM_OK;
}

void krylov_free(helm_ctx* c, cudaStream_t st) {
  Workspace* w = c->ws;
  if (!w) return;
  if (w->loop) cudaGraphExecDestroy(w->loop);
  if (w->body) cudaGraphExecDestroy(w->body);
  if (w->body_graph) cudaGraphDestroy(w->body_graph);
  if (w->idr_init) cudaGraphExecDestroy(w->idr_init);
  if (w->loop_graph) cudaGraphDestroy(w->loop_graph);
  if (w->init_graph) cudaGraphDestroy(w->init_graph);
  dev_free_all(w->mem, st);
  c->bytes -= w->bytes;
  pinned_slot_put(w->hst);
  delete w;
  c->ws = nullptr;
}

struct Ctx {
  helm_ctx* c;
  Workspace* w;
  long n;
  bool mg32;
  bool pc;
  int dim;
  int G;
};

// one V-cycle on the precision-boundary copy `in_mg`; the result is written in FP64
template <typename TM>
static helm_status precondition(const Ctx& k, const void* in_mg, double2* out, cudaStream_t st) {
  return mg_vcycle<TM>(k.c, (const cx<TM>*)in_mg, out, true, &k.w->st->done, st);
}

template <typename TM, int DIM>
static helm_status enqueue_bicg_iter(const Ctx& k, cudaStream_t st) {
  Workspace* w = k.w;
  OpView<double> H = k.c->H.view<double>();
  helm_status s;
  // In FP32 multigrid the update kernels also write the vector in FP32 (the V-cycle input);
  // in FP64 the V-cycle reads the Krylov vector itself.
  const bool f32 = std::is_same<TM, float>::value;
  void* pcopy = f32 ? w->pmg : nullptr;
  void* scopy = f32 ? w->smg : nullptr;
  const void* pin = f32 ? (const void*)w->pmg : (const void*)w->p;
  const void* sin_ = f32 ? (const void*)w->smg : (const void*)w->sv;
  launch_pdl(k_bicg_p<TM>, dim3(k.G), dim3(KT), 0, st, w->st, w->r, w->p, w->v, pcopy, k.n);
  const double2* ph = w->p;
  if (k.pc) {
    if ((s = precondition<TM>(k, pin, w->ph, st)) != HELM_OK) return s;
    ph = w->ph;
  }
  launch_pdl(k_bicg_v<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, ph, w->rh, w->v, k.n, w->partials);
  launch_pdl(k_bicg_s<TM>, dim3(k.G), dim3(KT), 0, st, w->st, w->r, w->v, w->sv, scopy, k.n, w->partials);
  launch_pdl(k_bicg_xhalf, dim3(k.G), dim3(KT), 0, st, w->st, ph, w->x, k.n);
  const double2* sh = w->sv;
  if (k.pc) {
    if ((s = precondition<TM>(k, sin_, w->sh, st)) != HELM_OK) return s;
    sh = w->sh;
  }
  launch_pdl(k_bicg_t<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, sh, w->sv, w->t, k.n, w->partials);
  launch_pdl(k_bicg_xr, dim3(k.G), dim3(KT), 0, st, w->st, ph, sh, w->sv, w->t, w->rh, w->x, w->r, k.n, w->partials);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename TM, int DIM, int S_>
static helm_status enqueue_idr_step(const Ctx& k, cudaStream_t st) {
  Workspace* w = k.w;
  OpView<double> H = k.c->H.view<double>();
  helm_status s;
  launch_pdl(k_idr_small, dim3(1), dim3(32), 0, st, w->st);
  void* vin = w->pmg;  // v in multigrid precision (always materialised)
  launch_pdl(k_idr_v<TM, S_>, dim3(k.G), dim3(KT), 0, st, w->st, w->dR, w->r, w->q, vin, k.n);
  const double2* z = (const double2*)vin;  // identity preconditioner: TM is double
  if (k.pc) {
    if ((s = precondition<TM>(k, vin, w->ph, st)) != HELM_OK) return s;
    z = w->ph;
  }
  launch_pdl(k_idr_t0<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, z, w->r, w->q, w->t, k.n, w->partials);
  launch_pdl(k_idr_dx<S_>, dim3(k.G), dim3(KT), 0, st, w->st, w->dX, z, k.n);
  launch_pdl(k_idr_tk<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, w->dX, w->t, k.n);
  launch_pdl(k_idr_upd<S_>, dim3(k.G), dim3(KT), 0, st, w->st, w->P, w->dR, w->dX, w->q, w->t, w->x, w->r, k.n, w->partials);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename TM, int DIM, int S_>
static helm_status enqueue_idr_init(const Ctx& k, cudaStream_t st) {
  Workspace* w = k.w;
  OpView<double> H = k.c->H.view<double>();
  helm_status s;
  for (int kc = 0; kc < S_; ++kc) {
    const double2* z = (const double2*)w->pmg;
    if (k.pc) {
      if ((s = precondition<TM>(k, w->pmg, w->ph, st)) != HELM_OK) return s;
      z = w->ph;
    }
    launch_pdl(k_idr_mr_t<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, z, w->r, w->t, k.n, w->partials);
    launch_pdl(k_idr_mr_upd<TM>, dim3(k.G), dim3(KT), 0, st, w->st, kc, z, w->t, w->dX, w->dR, w->x, w->r, w->pmg, k.n, w->partials);
  }
  for (int j = 0; j < S_; ++j) launch_pdl(k_idr_proj<S_>, dim3(k.G), dim3(KT), 0, st, w->st, w->P, w->dR + (long)j * k.n, j, k.n, w->partials);
  launch_pdl(k_idr_proj<S_>, dim3(k.G), dim3(KT), 0, st, w->st, w->P, w->r, -1, k.n, w->partials);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename TM, int DIM>
static helm_status enqueue_gm_step(const Ctx& k, cudaStream_t st) {
  Workspace* w = k.w;
  OpView<double> H = k.c->H.view<double>();
  GmView G = gm_view(w->gm, w->s);
  const double2* z = (const double2*)w->pmg;  // identity preconditioner: TM is double
  if (k.pc) {
    helm_status s = precondition<TM>(k, w->pmg, w->ph, st);
    if (s != HELM_OK) return s;
    z = w->ph;
  }
  launch_pdl(k_gm_w<DIM>, dim3(k.G), dim3(KT), 0, st, w->st, H, z, w->t, k.n);
  launch_pdl(k_gm_dots, dim3(k.G), dim3(KT), 0, st, w->st, w->V, w->t, k.n, w->partials, G.hA, 2);
  launch_pdl(k_gm_sub, dim3(k.G), dim3(KT), 0, st, w->st, w->V, w->t, G.hA, k.n, 0, w->partials);
  launch_pdl(k_gm_dots, dim3(k.G), dim3(KT), 0, st, w->st, w->V, w->t, k.n, w->partials, G.hB, 3);
  launch_pdl(k_gm_sub, dim3(k.G), dim3(KT), 0, st, w->st, w->V, w->t, G.hB, k.n, 1, w->partials);
  launch_pdl(k_gm_next<TM>, dim3(k.G), dim3(KT), 0, st, w->st, w->t, w->V, w->pmg, k.n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename TM, int DIM>
static helm_status enqueue_body(const Ctx& k, int method, int s, cudaStream_t st) {
  if (method == HELM_BICGSTAB) return enqueue_bicg_iter<TM, DIM>(k, st);
  if (method == HELM_GMRES) return enqueue_gm_step<TM, DIM>(k, st);
  switch (s) {
    case 1: return enqueue_idr_step<TM, DIM, 1>(k, st);
    case 2: return enqueue_idr_step<TM, DIM, 2>(k, st);
    case 3: return enqueue_idr_step<TM, DIM, 3>(k, st);
    case 4: return enqueue_idr_step<TM, DIM, 4>(k, st);
    case 5: return enqueue_idr_step<TM, DIM, 5>(k, st);
    case 6: return enqueue_idr_step<TM, DIM, 6>(k, st);
    case 7: return enqueue_idr_step<TM, DIM, 7>(k, st);
    default: return enqueue_idr_step<TM, DIM, 8>(k, st);
  }
}

template <typename TM, int DIM>
static helm_status enqueue_init(const Ctx& k, int s, cudaStream_t st) {
  switch (s) {
    case 1: return enqueue_idr_init<TM, DIM, 1>(k, st);
    case 2: return enqueue_idr_init<TM, DIM, 2>(k, st);
    case 3: return enqueue_idr_init<TM, DIM, 3>(k, st);
    case 4: return enqueue_idr_init<TM, DIM, 4>(k, st);
    case 5: return enqueue_idr_init<TM, DIM, 5>(k, st);
    case 6: return enqueue_idr_init<TM, DIM, 6>(k, st);
    case 7: return enqueue_idr_init<TM, DIM, 7>(k, st);
    default: return enqueue_idr_init<TM, DIM, 8>(k, st);
  }
}

template <typename TM>
static helm_status enqueue_body_any(const Ctx& k, int method, int s, cudaStream_t st) {
  if (k.dim == 1) return enqueue_body<TM, 1>(k, method, s, st);
  if (k.dim == 2) return enqueue_body<TM, 2>(k, method, s, st);
  return enqueue_body<TM, 3>(k, method, s, st);
}
template <typename TM>
static helm_status enqueue_init_any(const Ctx& k, int s, cudaStream_t st) {
  if (k.dim == 1) return enqueue_init<TM, 1>(k, s, st);
  if (k.dim == 2) return enqueue_init<TM, 2>(k, s, st);
  return enqueue_init<TM, 3>(k, s, st);
}

// Captures the straight-line enqueue into a graph.
template <typename F>
static helm_status capture(cudaStream_t st, cudaGraph_t* g, F&& fn) {
  cudaStream_t cs;
  HELM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cs); return cuda_check(e, "cudaStreamBeginCapture"); }
  helm_status s = fn(cs);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (s != HELM_OK) { if (graph) cudaGraphDestroy(graph); return s; }
  if (e != cudaSuccess) return cuda_check(e, "cudaStreamEndCapture");
  *g = graph;
  (void)st;
  return HELM_OK;
}

// Loop graph: [set condition from `done`] -> WHILE(cond) { one iteration; set condition }.
template <typename TM>
static helm_status build_loop(const Ctx& k, int method, int s) {
  Workspace* w = k.w;
  cudaGraph_t g;
  HELM_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaGraphConditionalHandleCreate"); }
  // head node: sets the condition from the current state
  cudaKernelNodeParams kp = {};
  int head_flag = 0;
  void* args[3] = {&h, &w->st, &head_flag};
  kp.func = (void*)k_set_cond;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  cudaGraphNode_t head;
  e = cudaGraphAddKernelNode(&head, g, nullptr, 0, &kp);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaGraphAddKernelNode"); }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, g, &head, nullptr, 1, &np);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaGraphAddNode(conditional)"); }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaStreamCreate"); }
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cs); cudaGraphDestroy(g); return cuda_check(e, "cudaStreamBeginCaptureToGraph"); }
  helm_status s2 = enqueue_body_any<TM>(k, method, s, cs);
  launch_pdl(k_set_cond, dim3(1), dim3(1), 0, cs, h, w->st, 1);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(cs, &out);
  cudaStreamDestroy(cs);
  if (s2 != HELM_OK) { cudaGraphDestroy(g); return s2; }
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaStreamEndCapture(body)"); }
  size_t nb = 0;
  cudaGraphGetNodes(body, nullptr, &nb);
  w->body_nodes = nb;
  e = cudaGraphInstantiate(&w->loop, g, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_check(e, "cudaGraphInstantiate(loop)"); }
  w->loop_graph = g;
  return HELM_OK;
}

template <typename TM>
static helm_status prepare_ws(helm_ctx* c, const helm_solve_opts* o, Ctx& k, cudaStream_t st);

// The Krylov workspace and graphs for (method, s), built on first use.  A build that fails part
// way (an allocation refused, a capture error) releases what it made, so that the next solve starts
// from nothing instead of finding an incomplete workspace.
template <typename TM>
static helm_status prepare(helm_ctx* c, const helm_solve_opts* o, Ctx& k, cudaStream_t st) {
  helm_status s = prepare_ws<TM>(c, o, k, st);
  Workspace* w = c->ws;
  if (s != HELM_OK && w && (!w->loop || (w->method == HELM_IDR && !w->idr_init))) {
    cudaStreamSynchronize(st);
    krylov_free(c, st);
  }
  return s;
}

template <typename TM>
static helm_status prepare_ws(helm_ctx* c, const helm_solve_opts* o, Ctx& k, cudaStream_t st) {
  Workspace*& w = c->ws;
  if (w && (w->method != o->method || (o->method != HELM_BICGSTAB && w->s != o->s))) {
    HELM_CUDA(cudaStreamSynchronize(st));
    krylov_free(c, st);
  }
  bool fresh = w == nullptr;
  if (fresh) {
    w = new Workspace();
    w->method = o->method;
    w->s = o->s;
    long n = c->n;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
    // a few blocks per SM: each thread then reduces several points before the (FP64, shuffle)
    // block reduction, whose cost is per thread, not per point
    w->G = grid_blocks(n, KT, sms * KRYLOV_BLOCKS_PER_SM);
    size_t v64 = sizeof(double2) * n;
    bool f32 = c->pc.kind != HELM_PC_NONE && c->pc.mg_dtype == HELM_C64;
    size_t vmg = (f32 ? sizeof(float2) : sizeof(double2)) * n;
    helm_status s;
    if ((s = ws_alloc(c, w, (void**)&w->st, sizeof(KrylovState), st)) != HELM_OK) return s;
    HELM_CUDA(cudaMemsetAsync(w->st, 0, sizeof(KrylovState), st));
    w->hst = (KrylovState*)pinned_slot_get(sizeof(KrylovState));
    if (!w->hst) { set_error("pinned host buffer"); return HELM_ERR_OOM; }
    w->nred = o->method == HELM_GMRES ? std::max(NRED, o->s + 1) : NRED;
    if ((s = ws_alloc(c, w, (void**)&w->partials, sizeof(double2) * w->nred * w->G, st)) != HELM_OK) return s;
    double2** vecs[] = {&w->x, &w->r, &w->t};
    for (auto pp : vecs) if ((s = ws_alloc(c, w, (void**)pp, v64, st)) != HELM_OK) return s;
    if ((s = ws_alloc(c, w, &w->pmg, vmg, st)) != HELM_OK) return s;
    if ((s = ws_alloc(c, w, (void**)&w->ph, v64, st)) != HELM_OK) return s;
    if (o->method == HELM_BICGSTAB) {
      double2** more[] = {&w->rh, &w->p, &w->v, &w->sv};
      for (auto pp : more) if ((s = ws_alloc(c, w, (void**)pp, v64, st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, &w->smg, vmg, st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, (void**)&w->sh, v64, st)) != HELM_OK) return s;
    } else if (o->method == HELM_GMRES) {
      if ((s = ws_alloc(c, w, (void**)&w->V, v64 * (o->s + 1), st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, (void**)&w->gm, sizeof(double2) * gm_elems(o->s), st)) != HELM_OK) return s;
    } else {
      if ((s = ws_alloc(c, w, (void**)&w->q, v64, st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, (void**)&w->P, v64 * o->s, st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, (void**)&w->dR, v64 * o->s, st)) != HELM_OK) return s;
      if ((s = ws_alloc(c, w, (void**)&w->dX, v64 * o->s, st)) != HELM_OK) return s;
    }
  }
  k.c = c;
  k.w = w;
  k.n = c->n;
  k.mg32 = c->pc.kind != HELM_PC_NONE && c->pc.mg_dtype == HELM_C64;
  k.pc = c->pc.kind != HELM_PC_NONE;
  k.dim = c->grid.dim;
  k.G = w->G;
  if (fresh) {
    helm_status s = build_loop<TM>(k, o->method, o->s);
    if (s != HELM_OK) return s;
    if (o->method == HELM_IDR) {
      s = capture(st, &w->init_graph, [&](cudaStream_t cs) { return enqueue_init_any<TM>(k, o->s, cs); });
      if (s != HELM_OK) return s;
      HELM_CUDA(cudaGraphInstantiate(&w->idr_init, w->init_graph, 0));
      size_t ni = 0;
      cudaGraphGetNodes(w->init_graph, nullptr, &ni);
      w->init_nodes = ni;
    }
  }
  if (o->host_loop && !w->body) {
    helm_status s = capture(st, &w->body_graph, [&](cudaStream_t cs) { return enqueue_body_any<TM>(k, o->method, o->s, cs); });
    if (s != HELM_OK) return s;
    HELM_CUDA(cudaGraphInstantiate(&w->body, w->body_graph, 0));
  }
  return HELM_OK;
}

static helm_status upload_shadow(const Ctx& k, const helm_solve_opts* o, cudaStream_t st) {
  Workspace* w = k.w;
  if (w->shadow_key == o->shadow) return HELM_OK;
  long n = k.n;
  HELM_CUDA(cudaMemcpyAsync(w->P, o->shadow, sizeof(double2) * n * o->s, cudaMemcpyHostToDevice, st));
  // modified Gram-Schmidt; the scalar goes through the partial-sum slot after the reductions
  double2* h = w->partials + (NRED - 1) * w->G;  // last slot, unused by k_dot1's own partials
  for (int j = 0; j < o->s; ++j) {
    double2* pj = w->P + (long)j * n;
    for (int i = 0; i < j; ++i) {
      double2* pi = w->P + (long)i * n;
      k_dot1<<<k.G, KT, 0, st>>>(w->st, pi, pj, n, w->partials, h);
      k_mgs_upd<<<k.G, KT, 0, st>>>(pj, pi, h, 0, n);
    }
    k_dot1<<<k.G, KT, 0, st>>>(w->st, pj, pj, n, w->partials, h);
    k_mgs_upd<<<k.G, KT, 0, st>>>(pj, pj, h, 1, n);
  }
  HELM_CUDA(cudaGetLastError());
  w->shadow_key = o->shadow;
  return HELM_OK;
}

// A solve in flight: begin() enqueues everything up to the readback of the statistics, poll()
// then finishes it or enqueues a true-residual restart.  A single solve, a batch and the server
// all drive solves through this object; nothing here synchronises another stream.
struct SolveJob {
  helm_ctx* c = nullptr;
  const double2* b = nullptr;
  double2* x = nullptr;
  helm_solve_opts o{};
  helm_solve_info* info = nullptr;
  cudaStream_t st = nullptr;
  Ctx k{};
  bool f32 = false, bicg = true, gm = false;
  int gm_passes = 0;  // GMRES cycles run
  int restarts = 0;
  long kernels = 0;
  long host_loops = -1;
  double t0 = 0.0;  // host clock at the start of the solve
  cudaEvent_t ev = nullptr;
  bool finished = false;
  helm_status status = HELM_OK;
};

template <typename TM>
static helm_status job_pass(SolveJob& j) {
  Workspace* w = j.k.w;
  cudaStream_t st = j.st;
  const Ctx& k = j.k;
  if (j.gm) {
    launch_pdl(k_gm_start, dim3(k.G), dim3(KT), 0, st, w->st, j.b, w->r, k.n, j.gm_passes == 0 ? 1 : 0,
               w->partials);
    launch_pdl(k_gm_v0<TM>, dim3(k.G), dim3(KT), 0, st, w->st, w->r, w->V, w->pmg, k.n);
  } else {
    void* rmg = j.bicg ? nullptr : w->pmg;  // IDR's first V-cycle input is r in multigrid precision
    launch_pdl(k_start, dim3(k.G), dim3(KT), 0, st, w->st, j.b, w->r, j.bicg ? w->rh : nullptr,
               j.bicg ? w->p : nullptr, j.bicg ? w->v : nullptr, rmg, k.mg32 ? 1 : 0, k.n,
               j.restarts == 0 ? 1 : 0, w->partials);
    if (!j.bicg) HELM_CUDA(cudaGraphLaunch(w->idr_init, st));
  }
  j.host_loops = -1;
  if (j.o.host_loop) {
    j.host_loops = 0;
    for (;;) {
      HELM_CUDA(cudaMemcpyAsync(&w->hst->done, &w->st->done, sizeof(int), cudaMemcpyDeviceToHost, st));
      HELM_CUDA(cudaStreamSynchronize(st));
      if (w->hst->done || j.host_loops > j.o.maxmv + 16) break;
      HELM_CUDA(cudaGraphLaunch(w->body, st));
      ++j.host_loops;
    }
  } else {
    HELM_CUDA(cudaGraphLaunch(w->loop, st));
  }
  if (j.gm) {  // end of the cycle: x += M^{-1} (V y)
    launch_pdl(k_gm_y, dim3(1), dim3(32), 0, st, w->st);
    launch_pdl(k_gm_comb<TM>, dim3(k.G), dim3(KT), 0, st, w->st, w->V, w->pmg, k.pc ? nullptr : w->ph, k.n);
    if (k.pc) {
      helm_status s = mg_vcycle<TM>(k.c, (const cx<TM>*)w->pmg, w->ph, true, nullptr, st);
      if (s != HELM_OK) return s;
    }
    launch_pdl(k_gm_addx, dim3(k.G), dim3(KT), 0, st, w->st, w->ph, w->x, k.n);
    ++j.gm_passes;
  }
  OpView<double> H = j.c->H.view<double>();
  switch (k.dim) {
    case 1: launch_pdl(k_true_res<1>, dim3(k.G), dim3(KT), 0, st, w->st, H, j.b, w->x, w->r, k.n, w->partials); break;
    case 2: launch_pdl(k_true_res<2>, dim3(k.G), dim3(KT), 0, st, w->st, H, j.b, w->x, w->r, k.n, w->partials); break;
    default: launch_pdl(k_true_res<3>, dim3(k.G), dim3(KT), 0, st, w->st, H, j.b, w->x, w->r, k.n, w->partials);
  }
  HELM_CUDA(cudaGetLastError());
  HELM_CUDA(cudaMemcpyAsync(w->hst, w->st, sizeof(KrylovState), cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaEventRecord(j.ev, st));
  return HELM_OK;
}

// the storage order of the V-cycle inputs the kernels write (level 0's)
static cudaError_t upload_mg_layout(const helm_ctx* c, Workspace* w, cudaStream_t st) {
  int xs[2] = {0, 0};
  if (c->pc.kind != HELM_PC_NONE && !c->lv.empty() && c->lv[0].xs) {
    xs[0] = c->lv[0].n[0];
    xs[1] = c->lv[0].xs_half();
  }
  static_assert(offsetof(KrylovState, xs_h) == offsetof(KrylovState, xs_n0) + sizeof(int), "adjacent");
  return cudaMemcpyAsync(&w->st->xs_n0, xs, sizeof(xs), cudaMemcpyHostToDevice, st);
}

template <typename TM>
static helm_status job_begin_t(SolveJob& j) {
  helm_status s = prepare<TM>(j.c, &j.o, j.k, j.st);
  if (s != HELM_OK) return s;
  Workspace* w = j.k.w;
  cudaStream_t st = j.st;
  if (j.o.method == HELM_IDR && (s = upload_shadow(j.k, &j.o, st)) != HELM_OK) return s;
  // per-solve scalars
  KrylovState init{};
  init.tol = j.o.tol;
  init.maxmv = j.o.maxmv;
  init.s = j.o.s;
  HELM_CUDA(cudaMemcpyAsync(&w->st->tol, &init.tol, sizeof(double), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(&w->st->maxmv, &init.maxmv, sizeof(int), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(&w->st->s, &init.s, sizeof(int), cudaMemcpyHostToDevice, st));
  double* hist = j.o.history;
  HELM_CUDA(cudaMemcpyAsync(&w->st->hist, &hist, sizeof(double*), cudaMemcpyHostToDevice, st));
  HELM_CUDA(upload_mg_layout(j.c, w, st));
  if (j.gm) {
    init.gmm = j.o.s;
    init.gm = w->gm;
    HELM_CUDA(cudaMemcpyAsync(&w->st->gmm, &init.gmm, sizeof(int), cudaMemcpyHostToDevice, st));
    HELM_CUDA(cudaMemcpyAsync(&w->st->gm, &init.gm, sizeof(double2*), cudaMemcpyHostToDevice, st));
    j.gm_passes = 0;
  }
  HELM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double2) * j.k.n, st));
  if (!j.ev) HELM_CUDA(cudaEventCreateWithFlags(&j.ev, cudaEventDisableTiming));
  return job_pass<TM>(j);
}

// Called once j.ev has completed: finish, or enqueue a restart from the true residual.
template <typename TM>
static helm_status job_step_t(SolveJob& j) {
  Workspace* w = j.k.w;
  const KrylovState& hs = *w->hst;
  // k_start, the loop head, loops x body, k_true_res (+ the IDR start graph)
  if (j.gm) {
    // k_gm_start, k_gm_v0, the loop head, loops x body, k_gm_y, k_gm_comb, the V-cycle (its
    // kernels are the body's minus the 7 GMRES ones), k_gm_addx, k_true_res
    long vc = j.k.pc ? (long)w->body_nodes - 7 : 0;
    if (j.host_loops >= 0) j.kernels += 6 + vc + j.host_loops * (long)(w->body_nodes - 1);
    else j.kernels += 7 + vc + (long)hs.loops * (long)w->body_nodes;
    // a cycle that ended at m steps continues; one whose estimate met tol while the true
    // residual did not counts as a restart
    bool more = false;
    if (!(hs.rel_true < j.o.tol) && hs.matvecs < j.o.maxmv) {
      if (hs.status == HELM_ERR_MAXIT) more = true;
      else if (hs.status == HELM_OK && j.restarts < j.o.max_restarts) { ++j.restarts; more = true; }
    }
    if (more) return job_pass<TM>(j);
  } else {
    if (j.host_loops >= 0) j.kernels += 2 + j.host_loops * (long)(w->body_nodes - 1) + (j.bicg ? 0 : (long)w->init_nodes);
    else j.kernels += 3 + (long)hs.loops * (long)w->body_nodes + (j.bicg ? 0 : (long)w->init_nodes);
    if (hs.status == HELM_OK && !(hs.rel_true < j.o.tol) && j.restarts < j.o.max_restarts) {
      ++j.restarts;
      return job_pass<TM>(j);
    }
  }
  HELM_CUDA(cudaMemcpyAsync(j.x, w->x, sizeof(double2) * j.k.n, cudaMemcpyDeviceToDevice, j.st));
  helm_status fs = (helm_status)hs.status;
  if (j.gm && (fs == HELM_OK || fs == HELM_ERR_MAXIT)) fs = hs.rel_true < j.o.tol ? HELM_OK : HELM_ERR_MAXIT;
  if (fs == HELM_OK && !(hs.rel_true < j.o.tol)) fs = HELM_ERR_MAXIT;
  if (j.info) {
    j.info->status = fs;
    j.info->iters = hs.iters;
    j.info->matvecs = hs.matvecs;
    j.info->restarts = j.restarts;
    j.info->rel_res_recur = hs.rel_recur;
    j.info->rel_res_true = hs.rel_true;
    j.info->kernels = j.kernels;
    j.info->vcycles = j.k.pc ? hs.matvecs + (j.gm ? j.gm_passes : 0) : 0;
    j.info->seconds = host_seconds() - j.t0;
    j.info->history_len = j.o.history ? (hs.matvecs < j.o.maxmv ? hs.matvecs : j.o.maxmv) : 0;
  }
  j.status = fs;
  j.finished = true;
  return HELM_OK;
}

// ---- helpers of the grouped solve (group.cu): one instance's part outside the grouped loop ----

template <typename TM>
static helm_status group_member_begin_t(helm_ctx* c, const helm_solve_opts* o, cudaStream_t st) {
  Ctx k{};
  helm_status s = prepare<TM>(c, o, k, st);
  if (s != HELM_OK) return s;
  Workspace* w = c->ws;
  const double tol = o->tol;
  const int maxmv = o->maxmv, sdim = o->s;
  double* hist = nullptr;
  HELM_CUDA(cudaMemcpyAsync(&w->st->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(&w->st->maxmv, &maxmv, sizeof(int), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(&w->st->s, &sdim, sizeof(int), cudaMemcpyHostToDevice, st));
  HELM_CUDA(cudaMemcpyAsync(&w->st->hist, &hist, sizeof(double*), cudaMemcpyHostToDevice, st));
  HELM_CUDA(upload_mg_layout(c, w, st));
  HELM_CUDA(cudaMemsetAsync(w->x, 0, sizeof(double2) * c->n, st));
  return HELM_OK;
}

helm_status group_member_begin(helm_ctx* c, const helm_solve_opts* o, cudaStream_t st) {
  const bool f32 = c->pc.kind != HELM_PC_NONE && c->pc.mg_dtype == HELM_C64;
  return f32 ? group_member_begin_t<float>(c, o, st) : group_member_begin_t<double>(c, o, st);
}

void group_member_start(helm_ctx* c, const double2* b, bool first, cudaStream_t st) {
  Workspace* w = c->ws;
  const bool f32 = c->pc.kind != HELM_PC_NONE && c->pc.mg_dtype == HELM_C64;
  launch_pdl(k_start, dim3(w->G), dim3(KT), 0, st, w->st, b, w->r, w->rh, w->p, w->v, (void*)nullptr,
             f32 ? 1 : 0, c->n, first ? 1 : 0, w->partials);
}

void group_member_true_res(helm_ctx* c, const double2* b, cudaStream_t st) {
  Workspace* w = c->ws;
  OpView<double> H = c->H.view<double>();
  launch_pdl(k_true_res<2>, dim3(w->G), dim3(KT), 0, st, w->st, H, b, w->x, w->r, c->n, w->partials);
  cudaMemcpyAsync(w->hst, w->st, sizeof(KrylovState), cudaMemcpyDeviceToHost, st);
}

static bool job_f32(const helm_ctx* c) { return c->pc.kind != HELM_PC_NONE && c->pc.mg_dtype == HELM_C64; }

helm_status job_begin(SolveJob& j) {
  j.t0 = host_seconds();
  j.f32 = job_f32(j.c);
  j.bicg = j.o.method == HELM_BICGSTAB;
  j.gm = j.o.method == HELM_GMRES;
  return j.f32 ? job_begin_t<float>(j) : job_begin_t<double>(j);
}

// Non-blocking when `block` is false: returns HELM_ERR_BUSY while the pass is still running.
helm_status job_poll(SolveJob& j, bool block) {
  if (j.finished) return HELM_OK;
  if (block) HELM_CUDA(cudaEventSynchronize(j.ev));
  else {
    cudaError_t e = cudaEventQuery(j.ev);
    if (e == cudaErrorNotReady) return HELM_ERR_BUSY;
    if (e != cudaSuccess) return cuda_check(e, "cudaEventQuery(solve)");
  }
  return j.f32 ? job_step_t<float>(j) : job_step_t<double>(j);
}

void job_release(SolveJob& j) {
  if (j.ev) cudaEventDestroy(j.ev);
  j.ev = nullptr;
}

SolveJob* job_new() { return new SolveJob(); }
void job_delete(SolveJob* j) { delete j; }
void job_setup(SolveJob* j, helm_ctx* c, const double2* b, double2* x, const helm_solve_opts* o,
               helm_solve_info* info, cudaStream_t st) {
  j->c = c; j->b = b; j->x = x; j->o = *o; j->info = info; j->st = st;
}
bool job_finished(const SolveJob* j) { return j->finished; }
helm_status job_status(const SolveJob* j) { return j->status; }

helm_status krylov_solve(helm_ctx* c, const double2* b, double2* x, const helm_solve_opts* o,
                         helm_solve_info* info, cudaStream_t st) {
  SolveJob j;
  j.c = c; j.b = b; j.x = x; j.o = *o; j.info = info; j.st = st;
  helm_status s = job_begin(j);
  while (s == HELM_OK && !j.finished) s = job_poll(j, true);
  job_release(j);
  if (s != HELM_OK) return s;
  HELM_CUDA(cudaStreamSynchronize(st));
  return j.status;
}

// Independent solves overlapped on the device: every instance runs on its own stream (ordered
// after the caller's stream and joined back into it), its device-resident loop needing no host
// involvement until its statistics are read.
helm_status krylov_solve_batch(helm_ctx* const* cs, const double2* const* b, double2* const* x, int n,
                               const helm_solve_opts* o, helm_solve_info* infos, cudaStream_t user) {
  std::vector<SolveJob> jobs(n);
  std::vector<cudaStream_t> streams(n, nullptr);
  // longest work first: stream priorities by the estimated work of each instance (unknowns x a
  // per-matvec cost of its method; IDR(s) does about 1.8 times Bi-CGSTAB's vector work per
  // matvec), ranked and spread over the device's priority range, the largest highest
  std::vector<int> prio(n, 0);
  {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    std::vector<std::pair<double, int>> w(n);
    for (int i = 0; i < n; ++i)
      w[i] = {(double)cs[i]->n * (o[i].method == HELM_IDR ? 1.8 : o[i].method == HELM_GMRES ? 1.0 + 0.2 * o[i].s : 1.0), i};
    std::sort(w.begin(), w.end());
    const int levels = least - greatest + 1;
    for (int r = 0; r < n; ++r) prio[w[r].second] = least - (int)((long)r * levels / (n > 0 ? n : 1));
  }
  cudaEvent_t start;
  HELM_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  helm_status s = HELM_OK;
  cudaError_t e = cudaEventRecord(start, user);
  if (e != cudaSuccess) s = cuda_check(e, "cudaEventRecord(batch)");
  for (int i = 0; i < n && s == HELM_OK; ++i) {
    e = cudaStreamCreateWithPriority(&streams[i], cudaStreamNonBlocking, prio[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(streams[i], start, 0);
    if (e != cudaSuccess) { s = cuda_check(e, "batch stream"); break; }
    SolveJob& j = jobs[i];
    j.c = cs[i]; j.b = b[i]; j.x = x[i]; j.o = o[i]; j.info = infos ? &infos[i] : nullptr; j.st = streams[i];
    if (j.o.host_loop) j.o.host_loop = 0;  // a batch always runs its loops on the device
    s = job_begin(j);
  }
  // finish every job (restarts are enqueued as their first pass completes)
  bool pending = s == HELM_OK;
  while (pending && s == HELM_OK) {
    pending = false;
    for (int i = 0; i < n && s == HELM_OK; ++i) {
      if (jobs[i].finished) continue;
      helm_status r = job_poll(jobs[i], false);
      if (r == HELM_ERR_BUSY) { pending = true; continue; }
      if (r != HELM_OK) { s = r; break; }
      if (!jobs[i].finished) pending = true;
    }
    if (pending) std::this_thread::yield();
  }
  // join the instance streams back into the caller's stream
  for (int i = 0; i < n; ++i) {
    if (!streams[i]) continue;
    if (s == HELM_OK) {
      cudaEvent_t done;
      if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(done, streams[i]);
        cudaStreamWaitEvent(user, done, 0);
        cudaEventDestroy(done);
      }
    }
    cudaStreamSynchronize(streams[i]);
    cudaStreamDestroy(streams[i]);
    job_release(jobs[i]);
  }
  cudaEventDestroy(start);
  if (s != HELM_OK) return s;
  helm_status worst = HELM_OK;
  for (int i = 0; i < n; ++i)
    if (jobs[i].status != HELM_OK && worst == HELM_OK) worst = jobs[i].status;
  return worst;
}

}  // namespace helm
