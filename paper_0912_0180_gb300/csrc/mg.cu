// mg.cu -- multigrid V(nu1, nu2) cycle on the preconditioner (Section 5.1; components of
// Section 6.1: damped Jacobi (omega), full-weighting restriction, bilinear/trilinear
// prolongation, rediscretised coarse operators; red-black Gauss-Seidel as second smoother;
// direct coarsest solve) and the FP64 Helmholtz matvec y = H x.
//
// Kernels take an optional `skip` flag: when it points to a non-zero word the kernel returns
// at once.  Inside a captured Krylov iteration this lets the remaining work of a converged
// solve cost one flag read per thread.
#include <algorithm>
#include <type_traits>
#include <vector>

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
// the colour-packed kernels (rb_pair_index): n[0] pairs a row; in 2D and 3D 16 pairs and two rows
// a warp
template <int DIM> static void rb_cfg(const int n[3], dim3& g, dim3& b) {
  if (DIM == 1) {
    cfg<DIM>(n, g, b);
    return;
  }
  b = dim3(32, Cfg<DIM>::BY, 1);
  g = dim3((n[0] + 15) / 16, (n[1] + 2 * b.y - 1) / (2 * b.y), n[2]);
}

#define POINT_INDEX(op)                                                        \
  int i = blockIdx.x * blockDim.x + threadIdx.x;                               \
  int j = blockIdx.y * blockDim.y + threadIdx.y;                               \
  int l = blockIdx.z;                                                          \
  if (i >= (op).n[0] || j >= (op).n[1]) return;                                \
  long p = i + (long)(op).n[0] * (j + (long)(op).n[1] * l);

// y = M x, or y = f - M x when f is given.  XS: x, f and y are stored x-split (h = (n0 + 1) / 2).
template <typename T, int DIM, bool XS = false>
__global__ void k_mg_apply(OpView<T> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ f,
                           cx<T>* __restrict__ y, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  if (XS) {
    const int h = (op.n[0] + 1) >> 1;
    const long row = p - i, ps = row + xs_pos(i, h);
    cx<T> v = op_row_at<T, T, DIM>(op, x, i, j, l, ps, p, row + xs_pos(i - 1, h), row + xs_pos(i + 1, h));
    y[ps] = f ? csub<T>(f[ps], v) : v;
    return;
  }
  cx<T> v = op_row<T, T, DIM>(op, x, i, j, l, p);
  y[p] = f ? csub<T>(f[p], v) : v;
}

// One damped-Jacobi sweep un = u + omega D^{-1} (f - M u), evaluated as
// (1 - omega) u + (omega / D) (f - offdiag(u)) with the stored omega / D; u == nullptr is the
// zero guess (un = (omega / D) f).
template <typename T, int DIM>
__global__ void k_jacobi(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                         cx<T>* __restrict__ un, T omega, double2* __restrict__ wide, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> di = op.dinv[p];  // omega / D
  cx<T> v;
  if (!u) {
    v = cmul<T>(f[p], di);
  } else {
    cx<T> g = cmul<T>(csub<T>(f[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)), di);
    cx<T> u0 = u[p];
    const T om1 = T(1) - omega;
    v = mkc<T>(fma(om1, u0.x, g.x), fma(om1, u0.y, g.y));
  }
  if (wide) wide[p] = cconv<double, T>(v);  // the last sweep of a V-cycle that ends in complex128
  else un[p] = v;
}

// Red-black Gauss-Seidel half-sweep on the points with (i + j + l) % 2 == colour, in place:
// u_P = (f_P - offdiag(u)_P) / D_P.  Along a row the colours alternate, so the grid holds one
// thread per point of the colour (thread t of a row takes i = 2t or 2t + 1) and every lane of a
// warp does arithmetic.  zero_guess (colour 0) writes the red points from a zero guess, f / D; the
// black sweep that always follows it reads only red neighbours and writes every black point.
// `wide` (black sweeps only): also write the pair of points of this thread, widened to complex128
// in natural order.  XS (the zero-guess sweep of an x-split level only): u, f and dinv are stored
// x-split, the colour's point of thread t at t, or h + t when the colour's x indices are odd.
// Thread -> (pair t, row j) of the colour-packed kernels.  In 2D and 3D a warp takes 16 pairs --
// 32 consecutive x points from a multiple of 32, one chunk of the uniform-interior rule -- of two
// neighbouring rows, so its lanes share the formula along x (one pair per lane over 32 pairs would
// span two chunks); launched by rb_cfg.
template <int DIM>
__device__ __forceinline__ void rb_pair_index(int& t, int& j) {
  if (DIM == 1) {
    t = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    return;
  }
  t = blockIdx.x * 16 + (threadIdx.x & 15);
  j = (blockIdx.y * blockDim.y + threadIdx.y) * 2 + (threadIdx.x >> 4);
}

template <typename T, int DIM, bool XS = false>
__global__ void k_rbgs(OpView<T> op, cx<T>* __restrict__ u, const cx<T>* __restrict__ f, int colour,
                       int zero_guess, double2* __restrict__ wide, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int t, j;
  rb_pair_index<DIM>(t, j);
  int l = blockIdx.z;
  if (j >= op.n[1]) return;
  const long row = (long)op.n[0] * (j + (long)op.n[1] * l);
  const int h = (op.n[0] + 1) >> 1;
  const int par = (j + l + colour) & 1;
  const int i = 2 * t + par;
  if (i < op.n[0]) {
    const long p = XS ? row + (par ? h + t : t) : row + i;
    if (zero_guess) {
      u[p] = cmul<T>(f[p], op.dinv[p]);
      return;
    }
    // x-split levels run every other sweep in k_rbgs3z2 / k_rbgs3z; only the zero-guess sweep (no neighbours)
    // comes here for them
    if (XS) return;
    const cx<T> off = op_offdiag<T, T, DIM>(op, u, i, j, l, p);
    cx<T> v = cmul<T>(csub<T>(f[p], off), op.dinv[p]);
    u[p] = v;
    if (wide) wide[row + i] = cconv<double, T>(v);
  }
  // the other point of the pair [2t, 2t + 1] is already final; it is in the grid even when this
  // thread's point lies past an odd row end
  const int i2 = 2 * t + 1 - par;
  if (wide && i2 < op.n[0]) wide[row + i2] = cconv<double, T>(u[XS ? row + (par ? t : h + t) : row + i2]);
}

// Red-black half-sweep on an x-split 3D level, marching along z: a thread owns the pair of
// columns (2t, 2t + 1) of row j and walks the planes [l0, l0 + lz).  In plane p the colour's
// point is column cur(p) = (j + p + colour) & 1 of the pair, and the pair's other-colour value
// V(p) (column 1 - cur(p)) is the point's in-pair x neighbour and, since the colour flips from
// plane to plane, the z neighbour of the colour's points in planes p - 1 and p + 1: a window of
// three V values in registers serves both, one new load per plane.  The other x neighbour is
// the V of the adjacent thread of the row segment (a shuffle; the segment's end lanes load it),
// the y neighbours are read from the rows j -+ 1, and every neighbour enters through its axis
// table (a neighbour outside the grid has value zero; its table entry is finite).  A row is a
// segment of W lanes (W = 32 or 16); the two segments of a 16-lane warp take rows of equal parity
// (j and j + 4), so cur is uniform over the warp and each plane's step is compiled for its column.
// RESID: instead of updating u, write the residual after the zero-guess sweep to r (-offdiag(u)
// on the colour, zero on the other one).  WIDE (sweeps only): both points of the pair also written
// widened to complex128 in natural order.  Every load of plane p + 1 (f, 1/D, the y neighbours, an
// end lane's x neighbour, V(p + 2)) is issued before plane p is computed: they read the other
// colour or read-only data, which this half-sweep never writes.  IDX: the offset type (int when
// N < 2^31).
template <typename T, bool RESID, bool WIDE, int W, typename IDX>
__global__ void __launch_bounds__(128) k_rbgs3z(OpView<T> op, cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                                                cx<T>* __restrict__ r, int colour, int lz,
                                                double2* __restrict__ wide, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  constexpr int SEGS = 32 / W;  // rows per warp
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2];
  const int h = (n0 + 1) >> 1;
  const int sl = threadIdx.x % W, seg = threadIdx.x / W;
  const int t = blockIdx.x * W + sl;
  const int j = blockIdx.y * (4 * SEGS) + seg * 4 + threadIdx.y;
  const int l0 = blockIdx.z * lz, l1 = min(l0 + lz, n2);
  const cx<T> zero = mkc<T>(T(0), T(0));
  const bool row_ok = j < n1;
  const bool has0 = row_ok && 2 * t < n0, has1 = row_ok && 2 * t + 1 < n0;
  const bool ylo = j > 0, yhi = j < n1 - 1;
  const bool xlo = row_ok && t > 0 && t - 1 < h && sl == 0, xhi = row_ok && 2 * t + 2 < n0 && sl == W - 1;
  const cx<T> axm0 = has0 ? op.am[0][2 * t] : zero, axp0 = has0 ? op.ap[0][2 * t] : zero;
  const cx<T> axm1 = has1 ? op.am[0][2 * t + 1] : zero, axp1 = has1 ? op.ap[0][2 * t + 1] : zero;
  const cx<T> aym = row_ok ? op.am[1][j] : zero, ayp = row_ok ? op.ap[1][j] : zero;
  const IDX P = (IDX)n0 * n1;
  const IDX rowoff = (IDX)n0 * (row_ok ? j : 0);
  // the pair's two columns in this row (x-split positions t and h + t)
  const IDX ce = rowoff + t, co = rowoff + h + t;
  const cx<T>* const dv = op.dinv;
  auto vload = [&](int q) -> cx<T> {  // V(q): the other colour's column of plane q
    if (q < 0 || q >= n2) return zero;
    const bool odd = ((j + q + colour) & 1) == 0;
    return (odd ? has1 : has0) ? u[(odd ? co : ce) + (IDX)q * P] : zero;
  };
  // f and 1/D of the colour's point of a plane (offset oo, column C): the streams from DRAM,
  // fetched two planes ahead
  auto fd = [&](auto cc, IDX oo, cx<T>& fv, cx<T>& dvv) {
    constexpr int C = decltype(cc)::value;
    const IDX pc = (C ? co : ce) + oo;
    const bool hc = C ? has1 : has0;
    fv = !RESID && hc ? f[pc] : zero;
    dvv = !RESID && hc ? dv[pc] : zero;
  };
  // the y neighbours and an end lane's outer x neighbour (mostly cache hits), one plane ahead
  struct Nb { cx<T> ym, yp, xe; };
  auto nb = [&](auto cc, IDX oo) -> Nb {
    constexpr int C = decltype(cc)::value;
    const IDX pc = (C ? co : ce) + oo;
    const bool hc = C ? has1 : has0;
    Nb q;
    q.ym = hc && ylo ? u[pc - n0] : zero;
    q.yp = hc && yhi ? u[pc + n0] : zero;
    if (C == 0) q.xe = xlo ? u[co + oo - 1] : zero;  // column 2t - 1
    else q.xe = xhi ? u[ce + oo + 1] : zero;         // column 2t + 2
    return q;
  };
  int cur = (j + l0 + colour) & 1;
  IDX o = (IDX)l0 * P;
  cx<T> vm = vload(l0 - 1), v0 = vload(l0), vp = vload(l0 + 1), vpp = vload(l0 + 2);
  cx<T> f0, d0, f1 = zero, d1 = zero;
  Nb pre;
  if (cur) {
    fd(std::integral_constant<int, 1>(), o, f0, d0);
    if (l0 + 1 < l1) fd(std::integral_constant<int, 0>(), o + P, f1, d1);
    pre = nb(std::integral_constant<int, 1>(), o);
  } else {
    fd(std::integral_constant<int, 0>(), o, f0, d0);
    if (l0 + 1 < l1) fd(std::integral_constant<int, 1>(), o + P, f1, d1);
    pre = nb(std::integral_constant<int, 0>(), o);
  }
  auto step = [&](auto cc, int p) {
    constexpr int C = decltype(cc)::value;
    const IDX pc = (C ? co : ce) + o, po = (C ? ce : co) + o;  // the colour's point, the other one
    const bool hc = C ? has1 : has0, ho = C ? has0 : has1;
    // plane p + 2 (its colour's column is C again): f, 1/D and V(p + 3) (also column C); plane
    // p + 1: the neighbours
    cx<T> f2 = zero, d2 = zero, v3 = zero;
    if (p + 2 < l1) fd(cc, o + 2 * P, f2, d2);
    if (p + 3 < n2 && p + 1 < l1 && hc) v3 = u[pc + 3 * P];
    Nb nx = pre;
    if (p + 1 < l1) nx = nb(std::integral_constant<int, 1 - C>(), o + P);
    cx<T> xo;  // the x neighbour outside the pair
    if (C == 0) {
      xo.x = __shfl_up_sync(0xffffffffu, v0.x, 1, W);
      xo.y = __shfl_up_sync(0xffffffffu, v0.y, 1, W);
      if (sl == 0) xo = pre.xe;
    } else {
      xo.x = __shfl_down_sync(0xffffffffu, v0.x, 1, W);
      xo.y = __shfl_down_sync(0xffffffffu, v0.y, 1, W);
      if (sl == W - 1) xo = pre.xe;
    }
    if (hc) {
      cx<T> off = cmul<T>(C ? axm1 : axm0, C ? v0 : xo);
      off = cfma<T>(C ? axp1 : axp0, C ? xo : v0, off);
      off = cfma<T>(aym, pre.ym, off);
      off = cfma<T>(ayp, pre.yp, off);
      off = cfma<T>(op.am[2][p], vm, off);
      off = cfma<T>(op.ap[2][p], vp, off);
      if (RESID) {
        r[pc] = mkc<T>(-off.x, -off.y);
      } else {
        const cx<T> v = cmul<T>(csub<T>(f0, off), d0);
        u[pc] = v;
        if (WIDE) wide[rowoff + 2 * t + C + o] = cconv<double, T>(v);
      }
    }
    if (ho) {
      if (RESID) r[po] = zero;
      else if (WIDE) wide[rowoff + 2 * t + 1 - C + o] = cconv<double, T>(v0);
    }
    vm = v0;
    v0 = vp;
    vp = vpp;
    vpp = v3;
    f0 = f1;
    d0 = d1;
    f1 = f2;
    d1 = d2;
    pre = nx;
  };
  for (int p = l0; p < l1; ++p) {
    if (cur) step(std::integral_constant<int, 1>(), p);
    else step(std::integral_constant<int, 0>(), p);
    cur ^= 1;
    o += P;
  }
}

// Two consecutive complex64 values, moved as one 16-byte access.
struct c64x2 {
  float2 a, b;
};
__device__ __forceinline__ c64x2 ld_x2(const float2* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return c64x2{make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
__device__ __forceinline__ void st_x2(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}

// k_rbgs3z with two pairs of columns per thread (FP32 x-split levels with n0 a multiple of 4):
// thread tt of a row owns columns 4tt .. 4tt + 3, so the colour's two points of a plane, the two
// window values and their y neighbours sit at two consecutive x-split positions and each of them
// is one 16-byte access; per point, the loads, their address arithmetic and the loop overhead are
// half those of k_rbgs3z.  With n0 a multiple of 4 a thread has all four columns or none, and every
// 16-byte access is aligned when the arrays are.  The per-point arithmetic is k_rbgs3z's, operation
// for operation.  A row is a segment of W lanes (4, 8 or 16); the rows of a warp are blockDim.y
// apart (even), so the colour's column is uniform over the warp.
template <bool RESID, bool WIDE, int W, typename IDX>
__global__ void __launch_bounds__(128) k_rbgs3z2(OpView<float> op, float2* __restrict__ u,
                                                 const float2* __restrict__ f, float2* __restrict__ r,
                                                 int colour, int lz, double2* __restrict__ wide,
                                                 const int* skip) {
  using T = float;
  pdl_entry();
  if (skip && *skip) return;
  constexpr int SEGS = 32 / W;  // rows per warp
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2];
  const int h = n0 >> 1;
  const int sl = threadIdx.x % W, seg = threadIdx.x / W;
  const int tt = blockIdx.x * W + sl;
  const int x0 = 4 * tt;
  const int by = blockDim.y;
  const int j = blockIdx.y * (by * SEGS) + seg * by + threadIdx.y;
  const int l0 = blockIdx.z * lz, l1 = min(l0 + lz, n2);
  const float2 zero = make_float2(0.f, 0.f);
  const c64x2 zz{zero, zero};
  const bool row_ok = j < n1;
  const bool hp = row_ok && x0 < n0;  // all four columns
  const bool ylo = j > 0, yhi = j < n1 - 1;
  const bool xlo = hp && tt > 0 && sl == 0, xhi = hp && x0 + 4 < n0 && sl == W - 1;
  // x coefficients of the four columns
  float2 axm[4], axp[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    axm[c] = hp ? op.am[0][x0 + c] : zero;
    axp[c] = hp ? op.ap[0][x0 + c] : zero;
  }
  const float2 aym = row_ok ? op.am[1][j] : zero, ayp = row_ok ? op.ap[1][j] : zero;
  const IDX P = (IDX)n0 * n1;
  const IDX rowoff = (IDX)n0 * (row_ok ? j : 0);
  // the thread's positions in this row: even columns at ce, ce + 1, odd ones at co, co + 1
  const IDX ce = rowoff + 2 * tt, co = rowoff + h + 2 * tt;
  const float2* const dv = op.dinv;
  auto vload = [&](int q) -> c64x2 {  // V(q): the other colour's columns of plane q
    if (q < 0 || q >= n2 || !hp) return zz;
    const bool odd = ((j + q + colour) & 1) == 0;
    return ld_x2(u + (odd ? co : ce) + (IDX)q * P);
  };
  auto fd = [&](auto cc, IDX oo, c64x2& fv, c64x2& dvv) {
    constexpr int C = decltype(cc)::value;
    if (!RESID && hp) {
      const IDX pc = (C ? co : ce) + oo;
      fv = ld_x2(f + pc);
      dvv = ld_x2(dv + pc);
    }
  };
  struct Nb {
    c64x2 ym, yp;
    float2 xe;
  };
  auto nb = [&](auto cc, IDX oo) -> Nb {
    constexpr int C = decltype(cc)::value;
    const IDX pc = (C ? co : ce) + oo;
    Nb q;
    q.ym = hp && ylo ? ld_x2(u + pc - n0) : zz;
    q.yp = hp && yhi ? ld_x2(u + pc + n0) : zz;
    if (C == 0) q.xe = xlo ? u[co + oo - 1] : zero;  // column x0 - 1
    else q.xe = xhi ? u[ce + oo + 2] : zero;         // column x0 + 4
    return q;
  };
  int cur = (j + l0 + colour) & 1;
  IDX o = (IDX)l0 * P;
  c64x2 vm = vload(l0 - 1), v0 = vload(l0), vp = vload(l0 + 1), vpp = vload(l0 + 2);
  c64x2 f0, d0, f1, d1;
  Nb pre;
  if (cur) {
    fd(std::integral_constant<int, 1>(), o, f0, d0);
    if (l0 + 1 < l1) fd(std::integral_constant<int, 0>(), o + P, f1, d1);
    pre = nb(std::integral_constant<int, 1>(), o);
  } else {
    fd(std::integral_constant<int, 0>(), o, f0, d0);
    if (l0 + 1 < l1) fd(std::integral_constant<int, 1>(), o + P, f1, d1);
    pre = nb(std::integral_constant<int, 0>(), o);
  }
  // one point: k_rbgs3z's operation order
  auto point = [&](float2 am_x, float2 ap_x, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm, float2 zp,
                   float2 azm, float2 azp) {
    float2 off = cmul<T>(am_x, xm);
    off = cfma<T>(ap_x, xp, off);
    off = cfma<T>(aym, ym, off);
    off = cfma<T>(ayp, yp, off);
    off = cfma<T>(azm, zm, off);
    return cfma<T>(azp, zp, off);
  };
  auto step = [&](auto cc, int p) {
    constexpr int C = decltype(cc)::value;
    const IDX pc = (C ? co : ce) + o;  // the colour's points
    c64x2 f2, d2, v3 = zz;
    if (p + 2 < l1) fd(cc, o + 2 * P, f2, d2);
    if (p + 3 < n2 && p + 1 < l1 && hp) v3 = ld_x2(u + pc + 3 * P);
    Nb nx = pre;
    if (p + 1 < l1) nx = nb(std::integral_constant<int, 1 - C>(), o + P);
    float2 xo;  // the x neighbour outside the thread's columns
    if (C == 0) {
      xo.x = __shfl_up_sync(0xffffffffu, v0.b.x, 1, W);
      xo.y = __shfl_up_sync(0xffffffffu, v0.b.y, 1, W);
      if (sl == 0) xo = pre.xe;
    } else {
      xo.x = __shfl_down_sync(0xffffffffu, v0.a.x, 1, W);
      xo.y = __shfl_down_sync(0xffffffffu, v0.a.y, 1, W);
      if (sl == W - 1) xo = pre.xe;
    }
    if (hp) {
      const float2 azm = op.am[2][p], azp = op.ap[2][p];
      // colour columns x0 + C and x0 + 2 + C
      const float2 oa = C ? point(axm[1], axp[1], v0.a, v0.b, pre.ym.a, pre.yp.a, vm.a, vp.a, azm, azp)
                          : point(axm[0], axp[0], xo, v0.a, pre.ym.a, pre.yp.a, vm.a, vp.a, azm, azp);
      const float2 ob = C ? point(axm[3], axp[3], v0.b, xo, pre.ym.b, pre.yp.b, vm.b, vp.b, azm, azp)
                          : point(axm[2], axp[2], v0.a, v0.b, pre.ym.b, pre.yp.b, vm.b, vp.b, azm, azp);
      if (RESID) {
        st_x2(r + pc, make_float2(-oa.x, -oa.y), make_float2(-ob.x, -ob.y));
        st_x2(r + (C ? ce : co) + o, zero, zero);  // the other colour's points
      } else {
        const float2 va = cmul<T>(csub<T>(f0.a, oa), d0.a), vb = cmul<T>(csub<T>(f0.b, ob), d0.b);
        st_x2(u + pc, va, vb);
        if (WIDE) {
          double2* w = wide + rowoff + x0 + o;
          w[C] = cconv<double, T>(va);
          w[1 - C] = cconv<double, T>(v0.a);
          w[2 + C] = cconv<double, T>(vb);
          w[3 - C] = cconv<double, T>(v0.b);
        }
      }
    }
    vm = v0;
    v0 = vp;
    vp = vpp;
    vpp = v3;
    f0 = f1;
    d0 = d1;
    f1 = f2;
    d1 = d2;
    pre = nx;
  };
  for (int p = l0; p < l1; ++p) {
    if (cur) step(std::integral_constant<int, 1>(), p);
    else step(std::integral_constant<int, 0>(), p);
    cur ^= 1;
    o += P;
  }
}

// Residual right after the single pre-smoothing sweep from the zero guess, without the diagonal:
// damped Jacobi left D u = omega f, so r = (1 - omega) f - offdiag(u); red-black Gauss-Seidel
// left r = 0 on the black points and r = -offdiag(u) on the red ones (their neighbours are all
// black and were updated last).  RB: one thread per red/black pair of a row.
// (x-split 3D levels take the RESID form of k_rbgs3z2 / k_rbgs3z instead)
template <typename T, int DIM, bool RB>
__global__ void k_resid0(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                         cx<T>* __restrict__ r, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int t, j;
  if (RB) rb_pair_index<DIM>(t, j);
  else {
    t = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
  }
  int l = blockIdx.z;
  if (j >= op.n[1]) return;
  const long row = (long)op.n[0] * (j + (long)op.n[1] * l);
  if (RB) {
    int par = (j + l) & 1;
    int ir = 2 * t + par, ib = 2 * t + 1 - par;
    if (ib < op.n[0]) r[row + ib] = mkc<T>(T(0), T(0));
    if (ir < op.n[0]) {
      cx<T> acc = op_offdiag<T, T, DIM>(op, u, ir, j, l, row + ir);
      r[row + ir] = mkc<T>(-acc.x, -acc.y);
    }
  } else {
    if (t >= op.n[0]) return;
    long p = row + t;
    cx<T> acc = op_offdiag<T, T, DIM>(op, u, t, j, l, p);
    cx<T> fv = f[p];
    const T om1 = T(1) - omega;
    r[p] = mkc<T>(fma(om1, fv.x, -acc.x), fma(om1, fv.y, -acc.y));
  }
}

// ---- Galerkin (9-point) levels, 2D ---------------------------------------------------------

// Off-diagonal part of a 9-point row: the eight neighbours' weights times their values.
template <typename T>
__device__ __forceinline__ cx<T> off9(const OpView<T>& op, const cx<T>* __restrict__ x, int i, int j, long p) {
  cx<T> acc = mkc<T>(T(0), T(0));
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      if (di == 0 && dj == 0) continue;
      const int ii = i + di, jj = j + dj;
      if (ii < 0 || ii >= op.n[0] || jj < 0 || jj >= op.n[1]) continue;
      acc = cfma<T>(op.stg[(long)(3 * (dj + 1) + (di + 1)) * op.ntot + p], x[p + di + (long)dj * op.n[0]], acc);
    }
  return acc;
}

// y = M x, or y = f - M x when f is given, on a 9-point level.
template <typename T>
__global__ void k_apply9(OpView<T> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ f,
                         cx<T>* __restrict__ y, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  (void)l;
  cx<T> v = cfma<T>(op.stg[4 * op.ntot + p], x[p], off9<T>(op, x, i, j, p));
  y[p] = f ? csub<T>(f[p], v) : v;
}

// Damped-Jacobi sweep on a 9-point level (same form as k_jacobi; u == nullptr: zero guess).
template <typename T>
__global__ void k_jacobi9(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                          cx<T>* __restrict__ un, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  (void)l;
  cx<T> di = op.dinv[p];  // omega / D
  if (!u) {
    un[p] = cmul<T>(f[p], di);
    return;
  }
  cx<T> g = cmul<T>(csub<T>(f[p], off9<T>(op, u, i, j, p)), di);
  cx<T> u0 = u[p];
  const T om1 = T(1) - omega;
  un[p] = mkc<T>(fma(om1, u0.x, g.x), fma(om1, u0.y, g.y));
}

// Residual after the single Jacobi sweep from zero on a 9-point level: (1 - omega) f - offdiag(u).
template <typename T>
__global__ void k_resid0_9(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                           cx<T>* __restrict__ r, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  (void)l;
  cx<T> acc = off9<T>(op, u, i, j, p);
  cx<T> fv = f[p];
  const T om1 = T(1) - omega;
  r[p] = mkc<T>(fma(om1, fv.x, -acc.x), fma(om1, fv.y, -acc.y));
}

// ---- Galerkin (27-point) levels, 3D ---------------------------------------------------------

// Off-diagonal part of a 27-point row: the 26 neighbours' weights times their values.
template <typename T>
__device__ __forceinline__ cx<T> off27(const OpView<T>& op, const cx<T>* __restrict__ x, int i, int j, int l,
                                       long p) {
  cx<T> acc = mkc<T>(T(0), T(0));
  const long sy = op.n[0], sz = (long)op.n[0] * op.n[1];
#pragma unroll
  for (int dl = -1; dl <= 1; ++dl) {
    const int ll = l + dl;
    if (ll < 0 || ll >= op.n[2]) continue;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= op.n[1]) continue;
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        if (di == 0 && dj == 0 && dl == 0) continue;
        const int ii = i + di;
        if (ii < 0 || ii >= op.n[0]) continue;
        acc = cfma<T>(op.stg[(long)(9 * (dl + 1) + 3 * (dj + 1) + (di + 1)) * op.ntot + p],
                      x[p + di + dj * sy + dl * sz], acc);
      }
    }
  }
  return acc;
}

// y = M x, or y = f - M x when f is given, on a 27-point level.
template <typename T>
__global__ void k_apply27(OpView<T> op, const cx<T>* __restrict__ x, const cx<T>* __restrict__ f,
                          cx<T>* __restrict__ y, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> v = cfma<T>(op.stg[13 * op.ntot + p], x[p], off27<T>(op, x, i, j, l, p));
  y[p] = f ? csub<T>(f[p], v) : v;
}

// Damped-Jacobi sweep on a 27-point level (u == nullptr: zero guess); `wide` also receives the
// result in complex128 (the last sweep of an FP32 V-cycle).
template <typename T>
__global__ void k_jacobi27(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                           cx<T>* __restrict__ un, T omega, double2* wide, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> di = op.dinv[p];  // omega / D
  cx<T> r;
  if (!u) {
    r = cmul<T>(f[p], di);
  } else {
    cx<T> g = cmul<T>(csub<T>(f[p], off27<T>(op, u, i, j, l, p)), di);
    cx<T> u0 = u[p];
    const T om1 = T(1) - omega;
    r = mkc<T>(fma(om1, u0.x, g.x), fma(om1, u0.y, g.y));
  }
  un[p] = r;
  if (wide) wide[p] = cconv<double, T>(r);
}

// Residual after the single Jacobi sweep from zero on a 27-point level: (1 - omega) f - offdiag(u).
template <typename T>
__global__ void k_resid0_27(OpView<T> op, const cx<T>* __restrict__ u, const cx<T>* __restrict__ f,
                            cx<T>* __restrict__ r, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  POINT_INDEX(op);
  cx<T> acc = off27<T>(op, u, i, j, l, p);
  cx<T> fv = f[p];
  const T om1 = T(1) - omega;
  r[p] = mkc<T>(fma(om1, fv.x, -acc.x), fma(om1, fv.y, -acc.y));
}

// fine and coarse unknowns per axis, and the coarsening offsets (coarse c is fine 2c + o[a]:
// o = 1, or 0 on an axis with a Sommerfeld low side); fh / ch: the fine / coarse level is stored
// x-split with that many even x indices per row (0: natural order)
struct Dims { int f[3]; int c[3]; int o[3]; int fh = 0, ch = 0; };
__device__ __forceinline__ int xpos(int i, int h) { return h ? xs_pos(i, h) : i; }

// Full weighting in index space: coarse unknown c gathers fine unknowns 2c+o-1, 2c+o, 2c+o+1 per
// axis with weights 1/4, 1/2, 1/4 (tensor product); indices outside the grid are Dirichlet.  The
// weights are applied one axis at a time, (a + c) + 2 b, and the factor 4^-DIM once at the end.
template <typename T, int DIM>
__global__ void k_restrict(Dims d, const cx<T>* __restrict__ r, cx<T>* __restrict__ fc, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  int L = blockIdx.z;
  if (I >= d.c[0] || J >= d.c[1]) return;
  const cx<T> zero = mkc<T>(T(0), T(0));
  auto w3 = [](cx<T> a, cx<T> b, cx<T> c) {
    return mkc<T>(fma(T(2), b.x, a.x + c.x), fma(T(2), b.y, a.y + c.y));
  };
  // fine fi .. fi+2 along x: fi = -1 (offset 0, first coarse node) and fi + 2 past a ragged edge
  // are outside the grid
  const int fi = 2 * I + d.o[0] - 1;
  auto row_sum = [&](int fj, int fl) -> cx<T> {
    if ((DIM > 1 && (fj < 0 || fj >= d.f[1])) || (DIM > 2 && (fl < 0 || fl >= d.f[2]))) return zero;
    const cx<T>* row = r + (long)d.f[0] * (fj + (long)d.f[1] * fl);
    return w3(fi >= 0 ? row[xpos(fi, d.fh)] : zero, row[xpos(fi + 1, d.fh)],
              fi + 2 < d.f[0] ? row[xpos(fi + 2, d.fh)] : zero);
  };
  auto plane_sum = [&](int fl) -> cx<T> {
    if (DIM == 1) return row_sum(0, 0);
    const int fj = 2 * J + d.o[1] - 1;
    return w3(row_sum(fj, fl), row_sum(fj + 1, fl), row_sum(fj + 2, fl));
  };
  cx<T> acc;
  if (DIM < 3) acc = plane_sum(0);
  else {
    const int fl = 2 * L + d.o[2] - 1;
    acc = w3(plane_sum(fl), plane_sum(fl + 1), plane_sum(fl + 2));
  }
  const T sc = DIM == 1 ? T(0.25) : (DIM == 2 ? T(0.0625) : T(0.015625));
  fc[xpos(I, d.ch) + (long)d.c[0] * (J + (long)d.c[1] * L)] = cscale<T>(sc, acc);
}

// Linear interpolation along one axis: fine index i = 2c + o is coarse node c (weight 1); one
// between two coarse nodes takes both with weight 1/2 (nodes outside the coarse grid are
// Dirichlet zeros).  Returns the count of coarse nodes and their indices.
__device__ __forceinline__ int interp1(int i, int nc, int o, int* ci) {
  const int r = i - o;
  if (r >= 0 && !(r & 1)) { ci[0] = r >> 1; return 1; }
  int k = 0;
  const int left = (r - 1) >> 1, right = (r + 1) >> 1;  // r odd or -1
  if (left >= 0 && left < nc) ci[k++] = left;
  if (right >= 0 && right < nc) ci[k++] = right;
  return k;
}

// u += P ec (or u = P ec when overwrite), bilinear / trilinear interpolation.  All terms of a fine
// point carry the same weight (1/2 per even axis), so they are summed first and scaled once.
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
  int ni = interp1(i, d.c[0], d.o[0], ci);
  int nj = DIM > 1 ? interp1(j, d.c[1], d.o[1], cj) : 1;
  int nl = DIM > 2 ? interp1(l, d.c[2], d.o[2], cl) : 1;
  auto on_coarse = [](int x, int o) { return x - o >= 0 && !((x - o) & 1); };
  T w = on_coarse(i, d.o[0]) ? T(1) : T(0.5);
  if (DIM > 1 && !on_coarse(j, d.o[1])) w *= T(0.5);
  if (DIM > 2 && !on_coarse(l, d.o[2])) w *= T(0.5);
  cx<T> acc = mkc<T>(T(0), T(0));
  for (int c3 = 0; c3 < nl; ++c3)
    for (int c2 = 0; c2 < nj; ++c2) {
      const cx<T>* row = ec + (long)d.c[0] * (cj[c2] + (long)d.c[1] * cl[c3]);
      for (int c1 = 0; c1 < ni; ++c1) acc = cadd<T>(acc, row[xpos(ci[c1], d.ch)]);
    }
  long p = xpos(i, d.fh) + (long)d.f[0] * (j + (long)d.f[1] * l);
  if (overwrite) u[p] = cscale<T>(w, acc);
  else {
    cx<T> uo = u[p];
    u[p] = mkc<T>(fma(w, acc.x, uo.x), fma(w, acc.y, uo.y));
  }
}

// The 3D transfers onto / from an x-split fine level, marching along z (one thread per coarse
// point or fine pair, consecutive planes in registers).  Both keep the exact arithmetic of
// k_restrict / k_prolong, so either kernel gives bitwise the same result.
//
// Full weighting: thread (I, J) walks the coarse planes [L0, L1); the plane sum PS(fl) (rows and
// columns weighted first) of fine plane fl = 2L + o - 1 is the last one of coarse plane L - 1, so
// two new plane sums per coarse plane.
template <typename T, typename IDX>
__global__ void __launch_bounds__(128) k_restrict3z(Dims d, const cx<T>* __restrict__ r, cx<T>* __restrict__ fc,
                                                    int lz, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int L0 = blockIdx.z * lz, L1 = min(L0 + lz, d.c[2]);
  if (I >= d.c[0] || J >= d.c[1]) return;
  const cx<T> zero = mkc<T>(T(0), T(0));
  auto w3 = [](cx<T> a, cx<T> b, cx<T> c) {
    return mkc<T>(fma(T(2), b.x, a.x + c.x), fma(T(2), b.y, a.y + c.y));
  };
  const int fi = 2 * I + d.o[0] - 1, fj = 2 * J + d.o[1] - 1;
  const bool xl = fi >= 0, xh = fi + 2 < d.f[0];
  const IDX qa = xl ? xpos(fi, d.fh) : 0, qb = xpos(fi + 1, d.fh), qc = xh ? xpos(fi + 2, d.fh) : 0;
  const IDX P = (IDX)d.f[0] * d.f[1];
  auto plane_sum = [&](int fl) -> cx<T> {
    if (fl < 0 || fl >= d.f[2]) return zero;
    cx<T> rs[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int y = fj + k;
      if (y < 0 || y >= d.f[1]) {
        rs[k] = zero;
        continue;
      }
      const cx<T>* row = r + (IDX)fl * P + (IDX)d.f[0] * y;
      rs[k] = w3(xl ? row[qa] : zero, row[qb], xh ? row[qc] : zero);
    }
    return w3(rs[0], rs[1], rs[2]);
  };
  cx<T> prev = plane_sum(2 * L0 + d.o[2] - 1);
  const IDX cq = (IDX)xpos(I, d.ch) + (IDX)d.c[0] * J;
  const IDX CP = (IDX)d.c[0] * d.c[1];
  for (int L = L0; L < L1; ++L) {
    const int fl = 2 * L + d.o[2] - 1;
    const cx<T> mid = plane_sum(fl + 1), last = plane_sum(fl + 2);
    fc[cq + CP * L] = cscale<T>(T(0.015625), w3(prev, mid, last));
    prev = last;
  }
}

// Trilinear prolongation onto an x-split fine level: thread (t, j) owns the fine pair (2t, 2t + 1)
// of row j and walks fine planes [l0, l1).  The pair reads coarse columns a = t - o and a + 1, the
// row coarse rows jA (and jB); the coarse values of the two coarse planes a fine plane can need
// stay in registers.  Every fine point sums its coarse values in k_prolong's order (lower plane,
// row, column first) and scales once.
template <typename T, typename IDX>
__global__ void __launch_bounds__(128) k_prolong3z(Dims d, const cx<T>* __restrict__ ec, cx<T>* __restrict__ u,
                                                   int overwrite, int lz, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int l0 = blockIdx.z * lz, l1 = min(l0 + lz, d.f[2]);
  if (j >= d.f[1] || 2 * t >= d.f[0]) return;
  const cx<T> zero = mkc<T>(T(0), T(0));
  const bool has1 = 2 * t + 1 < d.f[0];
  // x: coarse columns a, a + 1; with o = 1 the even fine column lies between them and the odd one
  // on a + 1, with o = 0 the even one on a and the odd one between them
  const int o0 = d.o[0], a = t - o0;
  const bool va = a >= 0 && a < d.c[0], vb = a + 1 < d.c[0];
  const IDX pa = va ? xpos(a, d.ch) : 0, pb = vb ? xpos(a + 1, d.ch) : 0;
  // y: coarse rows
  const int ry = j - d.o[1];
  const bool yon = ry >= 0 && !(ry & 1);
  const int jA = yon ? ry >> 1 : (ry - 1) >> 1, jB = jA + 1;
  const bool vjA = jA >= 0 && jA < d.c[1], vjB = !yon && jB < d.c[1];
  const IDX CP = (IDX)d.c[0] * d.c[1];
  // coarse values of plane L: [row A / B][column a / a + 1]
  struct Cp { cx<T> e[2][2]; bool v; };
  auto load_plane = [&](int L) -> Cp {
    Cp q;
    q.v = L >= 0 && L < d.c[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const bool vr = q.v && (rr ? vjB : vjA);
      const IDX rb = (IDX)L * CP + (IDX)d.c[0] * (rr ? jB : jA);
      q.e[rr][0] = vr && va ? ec[rb + pa] : zero;
      q.e[rr][1] = vr && vb ? ec[rb + pb] : zero;
    }
    return q;
  };
  const T wy = yon ? T(1) : T(0.5);
  const T wxe = o0 ? T(0.5) : T(1), wxo = o0 ? T(1) : T(0.5);
  // the coarse values of one fine point in k_prolong's order: planes, rows, columns ascending
  auto point = [&](const Cp& A, const Cp& B, bool two, bool odd) -> cx<T> {
    cx<T> acc = zero;
    // the even column uses {a, a + 1} when o = 1, {a} when o = 0; the odd one {a + 1} / {a, a + 1}
    const bool ca = odd ? (o0 == 0) : true, cb = odd ? true : (o0 == 1);
#pragma unroll
    for (int z = 0; z < 2; ++z) {
      const Cp& Q = z ? B : A;
      if ((z && !two) || !Q.v) continue;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        if (!(rr ? vjB : vjA)) continue;
        if (ca && va) acc = cadd<T>(acc, Q.e[rr][0]);
        if (cb && vb) acc = cadd<T>(acc, Q.e[rr][1]);
      }
    }
    return acc;
  };
  const IDX P = (IDX)d.f[0] * d.f[1];
  const IDX ce = (IDX)d.f[0] * j + t, co = (IDX)d.f[0] * j + d.fh + t;
  int rz = l0 - d.o[2];
  int Lc = rz >> 1;  // floor
  Cp A = load_plane(Lc), B = load_plane(Lc + 1);
  for (int l = l0; l < l1; ++l, ++rz) {
    if ((rz >> 1) != Lc) {  // the next coarse plane pair
      ++Lc;
      A = B;
      B = load_plane(Lc + 1);
    }
    const bool zon = !(rz & 1);  // on coarse plane Lc; otherwise between Lc and Lc + 1
    const T wz = zon ? T(1) : T(0.5);
    const IDX oe = ce + (IDX)l * P, oo = co + (IDX)l * P;
    const cx<T> se = point(A, B, !zon, false);
    const T we = wxe * wy * wz;
    if (overwrite) u[oe] = cscale<T>(we, se);
    else {
      const cx<T> uo = u[oe];
      u[oe] = mkc<T>(fma(we, se.x, uo.x), fma(we, se.y, uo.y));
    }
    if (has1) {
      const cx<T> so = point(A, B, !zon, true);
      const T wo = wxo * wy * wz;
      if (overwrite) u[oo] = cscale<T>(wo, so);
      else {
        const cx<T> uo = u[oo];
        u[oo] = mkc<T>(fma(wo, so.x, uo.x), fma(wo, so.y, uo.y));
      }
    }
  }
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

// Between natural and x-split order (h even x indices per row of n0), converting the element type
// on the way: TO_XS reads natural and writes x-split, otherwise the reverse.  One thread per point
// of a row, so both sides are coalesced.
template <typename TI, typename TO, bool TO_XS>
__global__ void k_xs_convert(const cx<TI>* __restrict__ a, cx<TO>* __restrict__ b, int n0, long rows,
                             const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long r = blockIdx.y + (long)gridDim.y * blockIdx.z;
  if (i >= n0 || r >= rows) return;
  const long row = r * n0;
  const long q = row + xs_pos(i, (n0 + 1) >> 1);
  if (TO_XS) b[q] = cconv<TO, TI>(a[row + i]);
  else b[row + i] = cconv<TO, TI>(a[q]);
}

// ---- host side -------------------------------------------------------------------------

static void widen_c64(const helm_ctx*, const float2* a, double2* b, long n, const int* skip, cudaStream_t st) {
  launch_pdl(k_widen, dim3((int)((n + 255) / 256)), dim3(256), 0, st, a, b, n, skip);
}

// a (level L, natural order when to_xs, else x-split) -> b in the other order, element type TO
template <typename TI, typename TO>
static void xs_convert(const LevelHost& L, const cx<TI>* a, cx<TO>* b, bool to_xs, const int* skip, cudaStream_t st) {
  const long rows = L.ntot / L.n[0];
  const int gy = (int)std::min<long>(rows, 65535);
  const int gz = (int)((rows + gy - 1) / gy);
  const int thr = std::min(256, (L.n[0] + 31) / 32 * 32);
  dim3 g((L.n[0] + thr - 1) / thr, gy, gz);
  if (to_xs) launch_pdl(k_xs_convert<TI, TO, true>, g, dim3(thr), 0, st, a, b, L.n[0], rows, skip);
  else launch_pdl(k_xs_convert<TI, TO, false>, g, dim3(thr), 0, st, a, b, L.n[0], rows, skip);
}

template <typename T>
static void vcycle_unfused(helm_ctx* c, int l, const cx<T>* f, cx<T>* out, const int* skip, cudaStream_t st,
                           double2* wide = nullptr);

// a Galerkin level: 9-point in 2D, 27-point in 3D
template <typename T> static bool is9(const LevelHost& L) { return L.stg64 != nullptr; }

// planes per thread of a z-marching kernel whose x-y grid has `warps` warps: the most (up to 32)
// that still leave about 24 warps per SM (fewer planes per thread re-read more window values at
// the chunk ends)
static int plane_chunk(long warps, int nz) {
  int lz = 32;
  while (lz > 2 && warps * ((nz + lz - 1) / lz) < 152L * 24) lz /= 2;
  return lz;
}

// the z-marching sweep: row segments of 32 or 16 pairs (whichever idles fewer lanes), 4 warps a
// block
template <typename T, bool RESID, bool WIDE, int W, typename IDX>
static void launch_rbgs3z_g(const LevelHost& L, cx<T>* u, const cx<T>* f, cx<T>* r, int colour, double2* wide,
                            const int* skip, cudaStream_t st);
template <typename T, bool RESID, int W, typename IDX>
static void launch_rbgs3z_w(const LevelHost& L, cx<T>* u, const cx<T>* f, cx<T>* r, int colour, double2* wide,
                            const int* skip, cudaStream_t st) {
  if (wide) {
    launch_rbgs3z_g<T, RESID, true, W, IDX>(L, u, f, r, colour, wide, skip, st);
    return;
  }
  launch_rbgs3z_g<T, RESID, false, W, IDX>(L, u, f, r, colour, wide, skip, st);
}
template <typename T, bool RESID, bool WIDE, int W, typename IDX>
static void launch_rbgs3z_g(const LevelHost& L, cx<T>* u, const cx<T>* f, cx<T>* r, int colour, double2* wide,
                            const int* skip, cudaStream_t st) {
  const int h = (L.n[0] + 1) / 2;
  const int rows_per_block = 4 * (32 / W);
  const long gx = (h + W - 1) / W, gy = (L.n[1] + rows_per_block - 1) / rows_per_block;
  const int lz = plane_chunk(gx * gy * 4, L.n[2]);
  dim3 g((unsigned)gx, (unsigned)gy, (unsigned)((L.n[2] + lz - 1) / lz));
  launch_pdl(k_rbgs3z<T, RESID, WIDE, W, IDX>, g, dim3(32, 4), 0, st, L.view<T>(), u, f, r, colour, lz, wide, skip);
}
// k_rbgs3z2: W lanes (two pairs each) per row segment, whichever of 16, 8, 4 idles the fewest
// lanes; blockDim.y = 4 or 2 rows, whichever idles fewer; planes per thread: the fewest that still
// fit the grid in one wave of resident blocks (a thread's planes run one after another, so the
// kernel lasts about one chain of planes)
template <bool RESID, bool WIDE, int W, typename IDX>
static void launch_rbgs3z2_g(const LevelHost& L, float2* u, const float2* f, float2* r, int colour, double2* wide,
                             const int* skip, cudaStream_t st) {
  auto kern = k_rbgs3z2<RESID, WIDE, W, IDX>;
  const int h = L.n[0] / 2;
  const int segs = 32 / W;
  const int by4 = (L.n[1] + 4 * segs - 1) / (4 * segs) * 4 * segs, by2 = (L.n[1] + 2 * segs - 1) / (2 * segs) * 2 * segs;
  const int by = by2 < by4 ? 2 : 4;
  const long gx = (h + 2 * W - 1) / (2 * W), gy = (L.n[1] + by * segs - 1) / (by * segs);
  auto resident = [&](int rows) {  // blocks resident on the whole device
    int dev = 0, b = 0, s = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * rows, 0);
    return (long)(b > 0 ? b : 1) * (s > 0 ? s : 1);
  };
  static const long cap2 = resident(2), cap4 = resident(4);
  const long cap = by == 2 ? cap2 : cap4;
  int lz = 2;
  while (lz < L.n[2] && gx * gy * ((L.n[2] + lz - 1) / lz) > cap) ++lz;
  dim3 g((unsigned)gx, (unsigned)gy, (unsigned)((L.n[2] + lz - 1) / lz));
  launch_pdl(kern, g, dim3(32, by), 0, st, L.view<float>(), u, f, r, colour, lz, wide, skip);
}
template <bool RESID, int W, typename IDX>
static void launch_rbgs3z2_w(const LevelHost& L, float2* u, const float2* f, float2* r, int colour, double2* wide,
                             const int* skip, cudaStream_t st) {
  if (wide) launch_rbgs3z2_g<RESID, true, W, IDX>(L, u, f, r, colour, wide, skip, st);
  else launch_rbgs3z2_g<RESID, false, W, IDX>(L, u, f, r, colour, wide, skip, st);
}
template <bool RESID, typename IDX>
static void launch_rbgs3z2(const LevelHost& L, float2* u, const float2* f, float2* r, int colour, double2* wide,
                           const int* skip, cudaStream_t st) {
  const int h = L.n[0] / 2;
  const int p16 = (h + 31) / 32 * 32, p8 = (h + 15) / 16 * 16, p4 = (h + 7) / 8 * 8;
  if (p16 <= p8 && p16 <= p4) launch_rbgs3z2_w<RESID, 16, IDX>(L, u, f, r, colour, wide, skip, st);
  else if (p8 <= p4) launch_rbgs3z2_w<RESID, 8, IDX>(L, u, f, r, colour, wide, skip, st);
  else launch_rbgs3z2_w<RESID, 4, IDX>(L, u, f, r, colour, wide, skip, st);
}
// the two-pair kernel's conditions: n0 a multiple of 4 and 16-byte aligned arrays
static bool rbgs3z2_fits(const LevelHost& L, const void* u, const void* f, const void* r) {
  const uintptr_t a = (uintptr_t)u | (uintptr_t)f | (uintptr_t)r | (uintptr_t)L.dinv32;
  return L.n[0] % 4 == 0 && (a & 15) == 0;
}

// x-split half-sweep or zero-guess residual: two pairs a thread where the row length and the
// arrays allow, else one
template <typename T, bool RESID>
static void launch_rbgs3z(const LevelHost& L, cx<T>* u, const cx<T>* f, cx<T>* r, int colour, double2* wide,
                          const int* skip, cudaStream_t st) {
  if constexpr (sizeof(cx<T>) == 8) {
    if (rbgs3z2_fits(L, u, f, r)) {
      if (L.ntot < 0x7fffffffL) launch_rbgs3z2<RESID, int>(L, (float2*)u, (const float2*)f, (float2*)r, colour, wide, skip, st);
      else launch_rbgs3z2<RESID, long>(L, (float2*)u, (const float2*)f, (float2*)r, colour, wide, skip, st);
      return;
    }
  }
  const int h = (L.n[0] + 1) / 2;
  const bool w16 = (h + 15) / 16 * 16 < (h + 31) / 32 * 32;
  const bool i64 = L.ntot >= 0x7fffffffL;
  if (w16 && !i64) launch_rbgs3z_w<T, RESID, 16, int>(L, u, f, r, colour, wide, skip, st);
  else if (!i64) launch_rbgs3z_w<T, RESID, 32, int>(L, u, f, r, colour, wide, skip, st);
  else if (w16) launch_rbgs3z_w<T, RESID, 16, long>(L, u, f, r, colour, wide, skip, st);
  else launch_rbgs3z_w<T, RESID, 32, long>(L, u, f, r, colour, wide, skip, st);
}

template <typename T, int DIM> struct Launch {
  static void apply(const LevelHost& L, const cx<T>* x, const cx<T>* f, cx<T>* y, const int* skip, cudaStream_t st) {
    dim3 g, b; cfg<DIM>(L.n, g, b);
    if (DIM == 2 && is9<T>(L)) launch_pdl(k_apply9<T>, dim3(g), dim3(b), 0, st, L.view<T>(), x, f, y, skip);
    else if (DIM == 3 && is9<T>(L)) launch_pdl(k_apply27<T>, dim3(g), dim3(b), 0, st, L.view<T>(), x, f, y, skip);
    else if (DIM == 3 && L.xs) launch_pdl(k_mg_apply<T, DIM, true>, dim3(g), dim3(b), 0, st, L.view<T>(), x, f, y, skip);
    else launch_pdl(k_mg_apply<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), x, f, y, skip);
  }
  static void jacobi(const LevelHost& L, const cx<T>* u, const cx<T>* f, cx<T>* un, T omega, double2* wide,
                     const int* skip, cudaStream_t st) {
    dim3 g, b; cfg<DIM>(L.n, g, b);
    if (DIM == 2 && is9<T>(L)) launch_pdl(k_jacobi9<T>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, un, omega, skip);
    else if (DIM == 3 && is9<T>(L))
      launch_pdl(k_jacobi27<T>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, un, omega, wide, skip);
    else launch_pdl(k_jacobi<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, un, omega, wide, skip);
  }
  static void rbgs(const LevelHost& L, cx<T>* u, const cx<T>* f, int colour, int zero, double2* wide,
                   const int* skip, cudaStream_t st) {
    int half[3] = {(L.n[0] + 1) / 2, L.n[1], L.n[2]};
    dim3 g, b; rb_cfg<DIM>(half, g, b);
    if (DIM == 3 && L.xs && !zero) launch_rbgs3z<T, false>(L, u, f, nullptr, colour, wide, skip, st);
    else if (DIM == 3 && L.xs) launch_pdl(k_rbgs<T, DIM, true>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, colour, zero, wide, skip);
    else launch_pdl(k_rbgs<T, DIM>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, colour, zero, wide, skip);
  }
  static void resid0(const LevelHost& L, const cx<T>* u, const cx<T>* f, cx<T>* r, T omega, bool rb, const int* skip,
                     cudaStream_t st) {
    int half[3] = {(L.n[0] + 1) / 2, L.n[1], L.n[2]};
    dim3 g, b;
    if (rb) {
      rb_cfg<DIM>(half, g, b);
      if (DIM == 3 && L.xs) launch_rbgs3z<T, true>(L, const_cast<cx<T>*>(u), nullptr, r, 0, nullptr, skip, st);
      else launch_pdl(k_resid0<T, DIM, true>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, r, omega, skip);
    } else {
      cfg<DIM>(L.n, g, b);
      if (DIM == 2 && is9<T>(L)) launch_pdl(k_resid0_9<T>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, r, omega, skip);
      else if (DIM == 3 && is9<T>(L))
        launch_pdl(k_resid0_27<T>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, r, omega, skip);
      else launch_pdl(k_resid0<T, DIM, false>, dim3(g), dim3(b), 0, st, L.view<T>(), u, f, r, omega, skip);
    }
  }
  static void restrict_(const LevelHost& F, const LevelHost& C, const cx<T>* r, cx<T>* fc, const int* skip, cudaStream_t st) {
    Dims d; for (int a = 0; a < 3; ++a) { d.f[a] = F.n[a]; d.c[a] = C.n[a]; d.o[a] = F.offset(a); }
    d.fh = F.xs_half(); d.ch = C.xs_half();
    if (DIM == 3 && F.xs) {  // marching along z over the coarse planes
      const long gx = (C.n[0] + 31) / 32, gy = (C.n[1] + 3) / 4;
      const int lz = plane_chunk(gx * gy * 4, C.n[2]);
      dim3 g((unsigned)gx, (unsigned)gy, (unsigned)((C.n[2] + lz - 1) / lz));
      if (F.ntot < 0x7fffffffL) launch_pdl(k_restrict3z<T, int>, g, dim3(32, 4), 0, st, d, r, fc, lz, skip);
      else launch_pdl(k_restrict3z<T, long>, g, dim3(32, 4), 0, st, d, r, fc, lz, skip);
      return;
    }
    dim3 g, b; cfg<DIM>(C.n, g, b);
    launch_pdl(k_restrict<T, DIM>, dim3(g), dim3(b), 0, st, d, r, fc, skip);
  }
  static void prolong(const LevelHost& F, const LevelHost& C, const cx<T>* ec, cx<T>* u, int overwrite, const int* skip, cudaStream_t st) {
    Dims d; for (int a = 0; a < 3; ++a) { d.f[a] = F.n[a]; d.c[a] = C.n[a]; d.o[a] = F.offset(a); }
    d.fh = F.xs_half(); d.ch = C.xs_half();
    if (DIM == 3 && F.xs) {  // marching along z over the fine planes, one thread per fine pair
      const long gx = (d.fh + 31) / 32, gy = (F.n[1] + 3) / 4;
      const int lz = plane_chunk(gx * gy * 4, F.n[2]);
      dim3 g((unsigned)gx, (unsigned)gy, (unsigned)((F.n[2] + lz - 1) / lz));
      if (F.ntot < 0x7fffffffL) launch_pdl(k_prolong3z<T, int>, g, dim3(32, 4), 0, st, d, ec, u, overwrite, lz, skip);
      else launch_pdl(k_prolong3z<T, long>, g, dim3(32, 4), 0, st, d, ec, u, overwrite, lz, skip);
      return;
    }
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
  void jacobi(const cx<T>* u, const cx<T>* f, cx<T>* un, T om, const int* skip, cudaStream_t st,
              double2* wide = nullptr) const {
    if (dim == 1) Launch<T, 1>::jacobi(L, u, f, un, om, wide, skip, st);
    else if (dim == 2) Launch<T, 2>::jacobi(L, u, f, un, om, wide, skip, st);
    else Launch<T, 3>::jacobi(L, u, f, un, om, wide, skip, st);
  }
  void rbgs(cx<T>* u, const cx<T>* f, int colour, int zero, const int* skip, cudaStream_t st,
            double2* wide = nullptr) const {
    if (dim == 1) Launch<T, 1>::rbgs(L, u, f, colour, zero, wide, skip, st);
    else if (dim == 2) Launch<T, 2>::rbgs(L, u, f, colour, zero, wide, skip, st);
    else Launch<T, 3>::rbgs(L, u, f, colour, zero, wide, skip, st);
  }
  void resid0(const cx<T>* u, const cx<T>* f, cx<T>* r, T om, bool rb, const int* skip, cudaStream_t st) const {
    if (dim == 1) Launch<T, 1>::resid0(L, u, f, r, om, rb, skip, st);
    else if (dim == 2) Launch<T, 2>::resid0(L, u, f, r, om, rb, skip, st);
    else Launch<T, 3>::resid0(L, u, f, r, om, rb, skip, st);
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
  if (c->fdm.on) {
    fdm_apply<T>(c, f, z, skip, st);
    return;
  }
  int n = c->nco;
  int thr = 256;
  int blocks = (n * 32 + thr - 1) / thr;
  launch_pdl(k_coarse<T>, dim3(blocks), dim3(thr), 0, st, (const cx<T>*)c->coarse_inv, n, f, z, skip);
}

// Smoothing sweeps on level L; buffers b[2] with *cur the index holding u.  zero: start from u = 0.
// wide (optional): the last sweep also writes the result widened to complex128.
template <typename T>
static void smooth(helm_ctx* c, const LevelHost& L, cx<T>* b[2], int* cur, const cx<T>* f, int sweeps,
                   bool zero, const int* skip, cudaStream_t st, double2* wide = nullptr) {
  Ops<T> op{L, L.dim};
  for (int k = 0; k < sweeps; ++k) {
    bool z0 = zero && k == 0;
    double2* w = k == sweeps - 1 ? wide : nullptr;
    if (c->pc.smoother == HELM_SM_JACOBI) {
      op.jacobi(z0 ? nullptr : b[*cur], f, b[1 - *cur], (T)c->pc.omega, skip, st, w);
      *cur = 1 - *cur;
    } else if (c->pc.smoother == HELM_SM_ILU) {
      // u += (L U)^{-1} (f - M u), the residual in the spare buffer; from u = 0 the residual is f
      cx<T>* u = b[*cur];
      cx<T>* r = b[1 - *cur];
      if (z0) {
        ilu_solve<T>(L, f, r, u, true, skip, st);
      } else {
        op.apply(u, f, r, skip, st);
        ilu_solve<T>(L, r, r, u, false, skip, st);
      }
      if constexpr (sizeof(cx<T>) == 8) {
        if (w) widen_c64(c, (const float2*)u, w, L.ntot, skip, st);
      }
    } else {
      op.rbgs(b[*cur], f, 0, z0 ? 1 : 0, skip, st);
      op.rbgs(b[*cur], f, 1, 0, skip, st, w);
    }
  }
}

template <typename T>
static bool fused_applies(const helm_ctx* c, int l) {
  const helm_precond& pcf = c->pc;
  if (pcf.flags & HELM_PF_UNFUSED) return false;
  if (pcf.smoother == HELM_SM_ILU) return false;  // ILU(0) runs as its own kernels
  if (c->lv[l].stg64) return false;  // 9-point Galerkin levels run the per-component kernels
  if (c->lv[l].any_offset0()) return false;  // the fused tiles assume coarse c = fine 2c + 1
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
    // one-kernel-per-component path in the multigrid precision; the last sweep writes the
    // complex128 result (or, without one, a separate widening pass)
    vcycle_unfused<T>(c, l, f, (cx<T>*)c->scratch, skip, st, (double2*)out);
    return;
  }
  vcycle_unfused<T>(c, l, f, (cx<T>*)out, skip, st);
}

// the one-kernel-per-component V-cycle on level l (below it, fused levels may take over); with
// `wide` the result goes there as complex128 instead of to `out` (which is then scratch)
template <typename T>
static void vcycle_unfused(helm_ctx* c, int l, const cx<T>* f, cx<T>* out, const int* skip, cudaStream_t st,
                           double2* wide) {
  const LevelHost& L = c->lv[l];
  int nl = (int)c->lv.size();
  if (l == nl - 1) {
    coarse_solve<T>(c, f, out, skip, st);
    if (wide) widen_c64(c, (const float2*)out, wide, L.ntot, skip, st);
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
    // residual into the spare buffer; after a single sweep from zero without the diagonal
    if (pc.nu1 == 1 && pc.smoother != HELM_SM_ILU) op.resid0(b[cur], f, b[1 - cur], (T)pc.omega, !jac, skip, st);
    else op.apply(b[cur], f, b[1 - cur], skip, st);
    restrict_any<T>(L, C, b[1 - cur], fc, skip, st);
  } else {
    restrict_any<T>(L, C, f, fc, skip, st);
  }
  vcycle_level<T>(c, l + 1, fc, C.u, false, skip, st);
  prolong_any<T>(L, C, (const cx<T>*)C.u, b[cur], pc.nu1 > 0 ? 0 : 1, skip, st);
  smooth<T>(c, L, b, &cur, f, pc.nu2, false, skip, st, wide);
  if (wide && pc.nu2 == 0) {
    if (L.xs) xs_convert<float, double>(L, (const float2*)b[cur], wide, false, skip, st);
    else widen_c64(c, (const float2*)b[cur], wide, L.ntot, skip, st);
  }
}

template <typename T>
helm_status mg_vcycle(helm_ctx* c, const cx<T>* f0, void* u0, bool u0_f64, const int* skip, cudaStream_t st) {
  const bool wide = u0_f64 && !std::is_same<T, double>::value;
  vcycle_level<T>(c, 0, f0, u0, wide, skip, st);
  const LevelHost& L = c->lv[0];
  if (L.xs && !wide) {  // an x-split result in the multigrid precision: back to natural order
    HELM_CUDA(cudaMemcpyAsync(L.w, u0, sizeof(cx<T>) * L.ntot, cudaMemcpyDeviceToDevice, st));
    xs_convert<T, T>(L, (const cx<T>*)L.w, (cx<T>*)u0, false, skip, st);
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status xs_permute_c64(const LevelHost& L, const float2* in, float2* out, cudaStream_t st) {
  xs_convert<float, float>(L, in, out, true, nullptr, st);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

// the V-cycle input on level 0 from a complex128 vector: converted to the multigrid precision, in
// the level's storage order
helm_status mg_input_from_c128(helm_ctx* c, const double2* in, void* out, cudaStream_t st) {
  const LevelHost& L = c->lv[0];
  if (!L.xs) return convert_c128_to_mg(c, in, out, st);
  xs_convert<double, float>(L, in, (float2*)out, true, nullptr, st);
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
  const bool stored = (op & HELM_OP_STORED) != 0;
  op &= ~HELM_OP_STORED;
  const LevelHost& L = c->lv[lvl];
  // vectors in natural order: the index-only kernels run on a natural view of the levels (the
  // tables they read, phi and the stored diagonal, are natural on every level)
  LevelHost Ln = L, Cn = lvl + 1 < nl ? c->lv[lvl + 1] : L;
  if (!stored) Ln.xs = Cn.xs = 0;
  Ops<T> o{Ln, Ln.dim};
  cx<T>* A = (cx<T>*)a;
  const cx<T>* B = (const cx<T>*)bb;
  cx<T>* O = (cx<T>*)out;
  switch (op) {
    case HELM_OP_APPLY: if (!A || !O) return HELM_ERR_ARG; o.apply(A, nullptr, O, nullptr, st); break;
    case HELM_OP_RESIDUAL: if (!A || !B || !O) return HELM_ERR_ARG; o.apply(A, B, O, nullptr, st); break;
    case HELM_OP_SMOOTH:
    case HELM_OP_SMOOTH0: {
      if (!A || !B || count < 0) return HELM_ERR_ARG;
      if (c->pc.smoother == HELM_SM_ILU && !L.ilu64) {
        set_error("the coarsest level is solved directly and has no ILU(0) factors");
        return HELM_ERR_ARG;
      }
      // the sweeps read the level's reciprocal diagonal in its storage order: natural vectors of
      // an x-split level go through two x-split copies
      const bool conv = L.xs && !stored;
      std::vector<DevBlock> tmp(2);
      cx<T>* ua = A;
      const cx<T>* fb = B;
      if (conv) {
        void *t0 = nullptr, *t1 = nullptr;
        helm_status as = dev_alloc(&t0, sizeof(cx<T>) * L.ntot, st, &tmp[0]);
        if (as == HELM_OK) as = dev_alloc(&t1, sizeof(cx<T>) * L.ntot, st, &tmp[1]);
        if (as != HELM_OK) { dev_free_all(tmp, st); return as; }
        ua = (cx<T>*)t0;
        fb = (const cx<T>*)t1;
        xs_convert<T, T>(L, A, ua, true, nullptr, st);
        xs_convert<T, T>(L, B, (cx<T>*)t1, true, nullptr, st);
      }
      cx<T>* b2[2] = {ua, (cx<T>*)L.w};
      int cur = 0;
      smooth<T>(c, L, b2, &cur, fb, count, op == HELM_OP_SMOOTH0, nullptr, st);
      if (cur == 1) HELM_CUDA(cudaMemcpyAsync(ua, L.w, sizeof(cx<T>) * L.ntot, cudaMemcpyDeviceToDevice, st));
      if (conv) {
        xs_convert<T, T>(L, ua, A, false, nullptr, st);
        HELM_CUDA(cudaGetLastError());
        dev_free_all(tmp, st);
      }
      break;
    }
    case HELM_OP_RESTRICT: if (lvl >= nl - 1 || !A || !O) return HELM_ERR_ARG; restrict_any<T>(Ln, Cn, A, O, nullptr, st); break;
    case HELM_OP_PROLONG: if (lvl >= nl - 1 || !A || !B) return HELM_ERR_ARG; prolong_any<T>(Ln, Cn, B, A, 0, nullptr, st); break;
    case HELM_OP_COARSE: if (lvl != nl - 1 || !A || !O) return HELM_ERR_ARG; coarse_solve<T>(c, A, O, nullptr, st); break;
    case HELM_OP_TO_STORED:
    case HELM_OP_FROM_STORED:
      if (!A || !O || A == O) return HELM_ERR_ARG;
      if (!L.xs) HELM_CUDA(cudaMemcpyAsync(O, A, sizeof(cx<T>) * L.ntot, cudaMemcpyDeviceToDevice, st));
      else xs_convert<T, T>(L, A, O, op == HELM_OP_TO_STORED, nullptr, st);
      break;
    case HELM_OP_DOWN:
      if (lvl >= nl - 1 || L.dim != 2 || c->pc.nu1 != 1 || L.stg64 || L.any_offset0() || !A || !B || !O)
        return HELM_ERR_ARG;
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
