// mg.cu -- multigrid V(nu1, nu2) cycle on the preconditioner (Section 5.1; components of
// Section 6.1: damped Jacobi (omega), full-weighting restriction, bilinear/trilinear
// prolongation, rediscretised coarse operators; red-black Gauss-Seidel as second smoother;
// direct coarsest solve) and the FP64 Helmholtz matvec y = H x.
//
// Kernels take an optional `skip` flag: when it points to a non-zero word the kernel returns
// at once.  Inside a captured Krylov iteration this lets the remaining work of a converged
// solve cost one flag read per thread.
#include <type_traits>

#include "stencil.cuh"

namespace helm {

template <int DIM> struct Cfg;
template <> struct Cfg<1> { static constexpr int BX = 256, BY = 1; };
template <> struct Cfg<2> { static constexpr int BX = 32, BY = 8; };
template <> struct Cfg<3> { static constexpr int BX = 32, BY = 4; };

template <int DIM> static void cfg(const int n[3], dim3& g, dim3& b) {
  b = dim3(Cfg<DIM>::BX, Cfg<DIM>::BY, 1);
  g = dim3((n[0] + b.x - 1) / b.x, (n[1] + b.y - 1) / b.y, n[2]);
}

#define POINT_INDEX(op)                                                        \
  int i = blockIdx.x * blockDim.x + threadIdx.x;                               \
  int j = blockIdx.y * blockDim.y + threadIdx.y;                               \
  int l = blockIdx.z;                                                          \
  if (i >= (op).n[0] || j >= (op).n[1]) return;                                \
  long p = i + (long)(op).n[0] * (j + (long)(op).n[1] * l);

// y = M x, or y = f - M x when f is given.
template <typename T, int DIM>
__global__ void k_mg_apply(OpView<T> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ f,
                           cx<T>* __restrict__ y, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> v = op_row<T, T, DIM>(op, x, i, j, l, p);
  y[p] = f ? csub<T>(f[p], v) : v;
}

// One damped-Jacobi sweep un = u + omega D^{-1} (f - M u), evaluated as
// (1 - omega) u + (omega / D) (f - offdiag(u)) with the stored omega / D; u == nullptr is the
// zero guess (un = (omega / D) f).
template <typename T, int DIM>
__global__ void k_jacobi(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                         cx<T>* __restrict__ un, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> di = op.dinv[p];  // omega / D
  if (!u) {
    un[p] = cmul<T>(f[p], di);
    return;
  }
  cx<T> g = cmul<T>(csub<T>(f[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)), di);
  cx<T> u0 = u[p];
  const T om1 = T(1) - omega;
  un[p] = mkc<T>(fma(om1, u0.x, g.x), fma(om1, u0.y, g.y));
}

// Red-black Gauss-Seidel half-sweep on points with (i + j + l) % 2 == colour, in place:
// u_P = (f_P - offdiag(u)_P) / D_P.  zero_guess with colour 0 writes the red points from a
// zero guess (f / D) and zeroes the black points.
template <typename T, int DIM>
__global__ void k_rbgs(OpView<T> op, cx<T>* __restrict__ u, const cx<T>* __restrict__ f, int colour,
                       int zero_guess, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  int c = (i + j + l) & 1;
  if (zero_guess) {
    if (c == 0) u[p] = cmul<T>(f[p], op.dinv[p]);
    else u[p] = mkc<T>(T(0), T(0));
    return;
  }
  if (c != colour) return;
  u[p] = cmul<T>(csub<T>(f[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)), op.dinv[p]);
}

struct Dims { int f[3]; int c[3]; };

// Full weighting in index space: coarse unknown c gathers fine unknowns 2c, 2c+1, 2c+2 per
// axis with weights 1/4, 1/2, 1/4 (tensor product); indices past the grid are Dirichlet.
template <typename T, int DIM>
__global__ void k_restrict(Dims d, const cx<T>* __restrict__ r, cx<T>* __restrict__ fc, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  int L = blockIdx.z;
  if (I >= d.c[0] || J >= d.c[1]) return;
  const T w[3] = {T(0.25), T(0.5), T(0.25)};
  cx<T> acc = mkc<T>(T(0), T(0));
  int dl0 = DIM > 2 ? -1 : 0, dl1 = DIM > 2 ? 1 : 0;
  int dj0 = DIM > 1 ? -1 : 0, dj1 = DIM > 1 ? 1 : 0;
  for (int dl = dl0; dl <= dl1; ++dl) {
    int fl = DIM > 2 ? 2 * L + 1 + dl : 0;
    if (fl >= d.f[2]) continue;
    T wl = DIM > 2 ? w[dl + 1] : T(1);
    for (int dj = dj0; dj <= dj1; ++dj) {
      int fj = DIM > 1 ? 2 * J + 1 + dj : 0;
      if (fj >= d.f[1]) continue;
      T wj = DIM > 1 ? w[dj + 1] : T(1);
      const cx<T>* row = r + (long)d.f[0] * (fj + (long)d.f[1] * fl);
      for (int di = -1; di <= 1; ++di) {
        int fi = 2 * I + 1 + di;
        if (fi >= d.f[0]) continue;
        acc = cadd<T>(acc, cscale<T>(w[di + 1] * wj * wl, row[fi]));
      }
    }
  }
  fc[I + (long)d.c[0] * (J + (long)d.c[1] * L)] = acc;
}

// linear interpolation weights of fine index i from coarse indices (at most 2)
__device__ __forceinline__ int interp1(int i, int nc, int* ci, float* w) {
  if (i & 1) { ci[0] = (i - 1) >> 1; w[0] = 1.f; return 1; }
  int k = 0;
  if ((i >> 1) - 1 >= 0) { ci[k] = (i >> 1) - 1; w[k] = 0.5f; ++k; }
  if ((i >> 1) < nc) { ci[k] = i >> 1; w[k] = 0.5f; ++k; }
  return k;
}

// u += P ec (or u = P ec when overwrite), bilinear / trilinear interpolation.
template <typename T, int DIM>
__global__ void k_prolong(Dims d, const cx<T>* __restrict__ ec, cx<T>* __restrict__ u, int overwrite,
                          const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int l = blockIdx.z;
  if (i >= d.f[0] || j >= d.f[1]) return;
  int ci[2], cj[2] = {0, 0}, cl[2] = {0, 0};
  float wi[2], wj[2] = {1.f, 1.f}, wl[2] = {1.f, 1.f};
  int ni = interp1(i, d.c[0], ci, wi);
  int nj = DIM > 1 ? interp1(j, d.c[1], cj, wj) : 1;
  int nl = DIM > 2 ? interp1(l, d.c[2], cl, wl) : 1;
  cx<T> acc = mkc<T>(T(0), T(0));
  for (int c3 = 0; c3 < nl; ++c3)
    for (int c2 = 0; c2 < nj; ++c2)
      for (int c1 = 0; c1 < ni; ++c1) {
        T wt = (T)wi[c1] * (T)wj[c2] * (T)wl[c3];
        acc = cadd<T>(acc, cscale<T>(wt, ec[ci[c1] + (long)d.c[0] * (cj[c2] + (long)d.c[1] * cl[c3])]));
      }
  long p = i + (long)d.f[0] * (j + (long)d.f[1] * l);
  u[p] = overwrite ? acc : cadd<T>(u[p], acc);
}

// z = Ainv f, one warp per row of the dense inverse of the coarsest operator.
template <typename T>
__global__ void k_coarse(const cx<T>* __restrict__ Ainv, int n, const cx<T>* __restrict__ f,
                         cx<T>* __restrict__ z, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const cx<T>* row = Ainv + (long)warp * n;
  cx<T> acc = mkc<T>(T(0), T(0));
  for (int c = lane; c < n; c += 32) acc = cfma<T>(row[c], f[c], acc);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) z[warp] = acc;
}

// y = H x in FP64 arithmetic, x complex128 or complex64.
template <typename TX, int DIM>
__global__ void k_h_apply(OpView<double> op, const cx<TX>* __restrict__ x, double2* __restrict__ y) {
  pdl_entry();
  POINT_INDEX(op);
  y[p] = op_row<double, TX, DIM>(op, x, i, j, l, p);
}

__global__ void k_widen(const float2* __restrict__ a, double2* __restrict__ b, long n, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p < n) b[p] = cconv<double, float>(a[p]);
}

// ---- host side -------------------------------------------------------------------------

static void widen_c64(const helm_ctx*, const float2* a, double2* b, long n, const int* skip, cudaStream_t st) {
  launch_pdl(k_widen, dim3((int)((n + 255) / 256)), dim3(256), 0, st, a, b, n, skip);
}

template <typename T>
static void vcycle_unfused(helm_ctx* c, int l, const cx<T>* f, cx<T>* out, const int* skip, cudaStream_t st);

template <typename T, int DIM> struct Launch {
  static void apply(const LevelHost& L, const cx<T>* x, const cx<T>* f, cx<T>* y, const int* skip, cudaStream_t st) {
    dim3 g, b; cfg<DIM>(L.n, g, b);
    launch_pdl(k_mg_apply<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), x, f, y, skip);
  }
  static void jacobi(const LevelHost& L, const cx<T>* u, const cx<T>* f, cx<T>* un, T omega, const int* skip, cudaStream_t st) {
    dim3 g, b; cfg<DIM>(L.n, g, b);
    launch_pdl(k_jacobi<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, un, omega, skip);
  }
  static void rbgs(const LevelHost& L, cx<T>* u, const cx<T>* f, int colour, int zero, const int* skip, cudaStream_t st) {
    dim3 g, b; cfg<DIM>(L.n, g, b);
    launch_pdl(k_rbgs<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, colour, zero, skip);
  }
  static void restrict_(const LevelHost& F, const LevelHost& C, const cx<T>* r, cx<T>* fc, const int* skip, cudaStream_t st) {
    Dims d; for (int a = 0; a < 3; ++a) { d.f[a] = F.n[a]; d.c[a] = C.n[a]; }
    dim3 g, b; cfg<DIM>(C.n, g, b);
    launch_pdl(k_restrict<T, DIM>, dim3(g), dim3(b), 0, st, d, r, fc, skip);
  }
  static void prolong(const LevelHost& F, const LevelHost& C, const cx<T>* ec, cx<T>* u, int overwrite, const int* skip, cudaStream_t st) {
    Dims d; for (int a = 0; a < 3; ++a) { d.f[a] = F.n[a]; d.c[a] = C.n[a]; }
    dim3 g, b; cfg<DIM>(F.n, g, b);
    launch_pdl(k_prolong<T, DIM>, dim3(g), dim3(b), 0, st, d, ec, u, overwrite, skip);
  }
};

template <typename T> struct Ops {
  const LevelHost& L;
  int dim;
  void apply(const cx<T>* x, const cx<T>* f, cx<T>* y, const int* skip, cudaStream_t st) const {
    if (dim == 1) Launch<T, 1>::apply(L, x, f, y, skip, st);
    else if (dim == 2) Launch<T, 2>::apply(L, x, f, y, skip, st);
    else Launch<T, 3>::apply(L, x, f, y, skip, st);
  }
  void jacobi(const cx<T>* u, const cx<T>* f, cx<T>* un, T om, const int* skip, cudaStream_t st) const {
    if (dim == 1) Launch<T, 1>::jacobi(L, u, f, un, om, skip, st);
    else if (dim == 2) Launch<T, 2>::jacobi(L, u, f, un, om, skip, st);
    else Launch<T, 3>::jacobi(L, u, f, un, om, skip, st);
  }
  void rbgs(cx<T>* u, const cx<T>* f, int colour, int zero, const int* skip, cudaStream_t st) const {
    if (dim == 1) Launch<T, 1>::rbgs(L, u, f, colour, zero, skip, st);
    else if (dim == 2) Launch<T, 2>::rbgs(L, u, f, colour, zero, skip, st);
    else Launch<T, 3>::rbgs(L, u, f, colour, zero, skip, st);
  }
};

template <typename T>
static void restrict_any(const LevelHost& F, const LevelHost& C, const cx<T>* r, cx<T>* fc, const int* skip, cudaStream_t st) {
  if (F.dim == 1) Launch<T, 1>::restrict_(F, C, r, fc, skip, st);
  else if (F.dim == 2) Launch<T, 2>::restrict_(F, C, r, fc, skip, st);
  else Launch<T, 3>::restrict_(F, C, r, fc, skip, st);
}
template <typename T>
static void prolong_any(const LevelHost& F, const LevelHost& C, const cx<T>* ec, cx<T>* u, int ow, const int* skip, cudaStream_t st) {
  if (F.dim == 1) Launch<T, 1>::prolong(F, C, ec, u, ow, skip, st);
  else if (F.dim == 2) Launch<T, 2>::prolong(F, C, ec, u, ow, skip, st);
  else Launch<T, 3>::prolong(F, C, ec, u, ow, skip, st);
}
template <typename T>
static void coarse_solve(helm_ctx* c, const cx<T>* f, cx<T>* z, const int* skip, cudaStream_t st) {
  int n = c->nco;
  int thr = 256;
  int blocks = (n * 32 + thr - 1) / thr;
  launch_pdl(k_coarse<T>, dim3(blocks), dim3(thr), 0, st, (const cx<T>*)c->coarse_inv, n, f, z, skip);
}

// Smoothing sweeps on level L; buffers b[2] with *cur the index holding u.  zero: start from u = 0.
template <typename T>
static void smooth(helm_ctx* c, const LevelHost& L, cx<T>* b[2], int* cur, const cx<T>* f, int sweeps,
                   bool zero, const int* skip, cudaStream_t st) {
  Ops<T> op{L, L.dim};
  for (int k = 0; k < sweeps; ++k) {
    bool z0 = zero && k == 0;
    if (c->pc.smoother == HELM_SM_JACOBI) {
      op.jacobi(z0 ? nullptr : b[*cur], f, b[1 - *cur], (T)c->pc.omega, skip, st);
      *cur = 1 - *cur;
    } else {
      op.rbgs(b[*cur], f, 0, z0 ? 1 : 0, skip, st);
      op.rbgs(b[*cur], f, 1, 0, skip, st);
    }
  }
}

template <typename T>
static bool fused_applies(const helm_ctx* c, int l) {
  const helm_precond& pcf = c->pc;
  if (pcf.flags & HELM_PF_UNFUSED) return false;
  if (l >= c->tail_first) return true;
  return c->lv[l].dim == 2 && pcf.nu1 == 1 && pcf.nu2 == 1 && l < (int)c->lv.size() - 1;
}

// V-cycle on level l for M_l u = f from u = 0; the result lands in `out` (complex128 when
// out_f64, else cx<T>; only level 0 is ever asked for complex128 with T = float).
template <typename T>
static void vcycle_level(helm_ctx* c, int l, const cx<T>* f, void* out, bool out_f64, const int* skip,
                         cudaStream_t st) {
  const LevelHost& L = c->lv[l];
  int nl = (int)c->lv.size();
  if (fused_applies<T>(c, l)) {
    if (l >= c->tail_first) {  // this level and all coarser ones in one block
      tail_vcycle<T>(c, l, f, out, out_f64, skip, st);
      return;
    }
    const LevelHost& C = c->lv[l + 1];
    fused_down2d<T>(c, l, f, (cx<T>*)L.w, (cx<T>*)C.f, skip, st);
    vcycle_level<T>(c, l + 1, (const cx<T>*)C.f, C.u, false, skip, st);
    fused_up2d<T>(c, l, (const cx<T>*)L.w, (const cx<T>*)C.u, f, out, out_f64, skip, st);
    return;
  }
  if (out_f64 && !std::is_same<T, double>::value) {
    // one-kernel-per-component path: run in the multigrid precision, then widen
    vcycle_level<T>(c, l, f, c->scratch, false, skip, st);
    widen_c64(c, (const float2*)c->scratch, (double2*)out, L.ntot, skip, st);
    return;
  }
  vcycle_unfused<T>(c, l, f, (cx<T>*)out, skip, st);
}

// the one-kernel-per-component V-cycle on level l (below it, fused levels may take over)
template <typename T>
static void vcycle_unfused(helm_ctx* c, int l, const cx<T>* f, cx<T>* out, const int* skip, cudaStream_t st) {
  const LevelHost& L = c->lv[l];
  int nl = (int)c->lv.size();
  if (l == nl - 1) {
    coarse_solve<T>(c, f, out, skip, st);
    return;
  }
  const LevelHost& C = c->lv[l + 1];
  const helm_precond& pc = c->pc;
  cx<T>* b[2] = {out, (cx<T>*)L.w};
  bool jac = pc.smoother == HELM_SM_JACOBI;
  int cur = jac ? ((pc.nu1 + pc.nu2) & 1) : 0;  // so that the last Jacobi sweep writes `out`
  Ops<T> op{L, L.dim};
  cx<T>* fc = (cx<T>*)C.f;
  if (pc.nu1 > 0) {
    smooth<T>(c, L, b, &cur, f, pc.nu1, true, skip, st);
    op.apply(b[cur], f, b[1 - cur], skip, st);  // residual into the spare buffer
    restrict_any<T>(L, C, b[1 - cur], fc, skip, st);
  } else {
    restrict_any<T>(L, C, f, fc, skip, st);
  }
  vcycle_level<T>(c, l + 1, fc, C.u, false, skip, st);
  prolong_any<T>(L, C, (const cx<T>*)C.u, b[cur], pc.nu1 > 0 ? 0 : 1, skip, st);
  smooth<T>(c, L, b, &cur, f, pc.nu2, false, skip, st);
}

template <typename T>
helm_status mg_vcycle(helm_ctx* c, const cx<T>* f0, void* u0, bool u0_f64, const int* skip, cudaStream_t st) {
  vcycle_level<T>(c, 0, f0, u0, u0_f64 && !std::is_same<T, double>::value, skip, st);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}
template helm_status mg_vcycle<float>(helm_ctx*, const float2*, void*, bool, const int*, cudaStream_t);
template helm_status mg_vcycle<double>(helm_ctx*, const double2*, void*, bool, const int*, cudaStream_t);

template <typename T>
static helm_status level_op_t(helm_ctx* c, int op, int lvl, void* a, const void* bb, void* out, int count,
                              cudaStream_t st) {
  int nl = (int)c->lv.size();
  if (lvl < 0 || lvl >= nl) return HELM_ERR_ARG;
  const LevelHost& L = c->lv[lvl];
  Ops<T> o{L, L.dim};
  cx<T>* A = (cx<T>*)a;
  const cx<T>* B = (const cx<T>*)bb;
  cx<T>* O = (cx<T>*)out;
  switch (op) {
    case HELM_OP_APPLY: if (!A || !O) return HELM_ERR_ARG; o.apply(A, nullptr, O, nullptr, st); break;
    case HELM_OP_RESIDUAL: if (!A || !B || !O) return HELM_ERR_ARG; o.apply(A, B, O, nullptr, st); break;
    case HELM_OP_SMOOTH:
    case HELM_OP_SMOOTH0: {
      if (!A || !B || count < 0) return HELM_ERR_ARG;
      cx<T>* b2[2] = {A, (cx<T>*)L.w};
      int cur = 0;
      smooth<T>(c, L, b2, &cur, B, count, op == HELM_OP_SMOOTH0, nullptr, st);
      if (cur == 1) HELM_CUDA(cudaMemcpyAsync(A, L.w, sizeof(cx<T>) * L.ntot, cudaMemcpyDeviceToDevice, st));
      break;
    }
    case HELM_OP_RESTRICT: if (lvl >= nl - 1 || !A || !O) return HELM_ERR_ARG; restrict_any<T>(L, c->lv[lvl + 1], A, O, nullptr, st); break;
    case HELM_OP_PROLONG: if (lvl >= nl - 1 || !A || !B) return HELM_ERR_ARG; prolong_any<T>(L, c->lv[lvl + 1], B, A, 0, nullptr, st); break;
    case HELM_OP_COARSE: if (lvl != nl - 1 || !A || !O) return HELM_ERR_ARG; coarse_solve<T>(c, A, O, nullptr, st); break;
    case HELM_OP_DOWN:
      if (lvl >= nl - 1 || L.dim != 2 || c->pc.nu1 != 1 || !A || !B || !O) return HELM_ERR_ARG;
      fused_down2d<T>(c, lvl, B, A, O, nullptr, st);
      break;
    default: return HELM_ERR_ARG;
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status mg_level_op(helm_ctx* c, int op, int lvl, void* a, const void* b, void* out, int count,
                        cudaStream_t st) {
  if (c->pc.kind == HELM_PC_NONE) return HELM_ERR_ARG;
  if (c->pc.mg_dtype == HELM_C64) return level_op_t<float>(c, op, lvl, a, b, out, count, st);
  return level_op_t<double>(c, op, lvl, a, b, out, count, st);
}

helm_status h_apply(helm_ctx* c, bool x_is_f32, const void* x, double2* y, cudaStream_t st) {
  const LevelHost& H = c->H;
  OpView<double> v = H.view<double>();
  dim3 g, b;
  switch (H.dim) {
    case 1: cfg<1>(H.n, g, b);
      if (x_is_f32) launch_pdl(k_h_apply<float, 1>, dim3(g), dim3(b), 0, st, v, (const float2*)x, y);
      else launch_pdl(k_h_apply<double, 1>, dim3(g), dim3(b), 0, st, v, (const double2*)x, y);
      break;
    case 2: cfg<2>(H.n, g, b);
      if (x_is_f32) launch_pdl(k_h_apply<float, 2>, dim3(g), dim3(b), 0, st, v, (const float2*)x, y);
      else launch_pdl(k_h_apply<double, 2>, dim3(g), dim3(b), 0, st, v, (const double2*)x, y);
      break;
    default: cfg<3>(H.n, g, b);
      if (x_is_f32) launch_pdl(k_h_apply<float, 3>, dim3(g), dim3(b), 0, st, v, (const float2*)x, y);
      else launch_pdl(k_h_apply<double, 3>, dim3(g), dim3(b), 0, st, v, (const double2*)x, y);
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

}  // namespace helm
