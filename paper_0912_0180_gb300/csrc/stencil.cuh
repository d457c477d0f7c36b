// stencil.cuh -- the Shortley-Weller row of a level operator evaluated at one grid point.
//   (A x)_P = sum_axes (am x_{P-e} + a0 x_P + ap x_{P+e}) - s * phi_P * x_P
// Section 3, eq. "shortwell", summed over axes; sigma = s * phi with s = 1 for H and CSG
// (eqs. "helmctu0", "lapctucsg") and s = beta^2 for CSL (eq. "helmctucsl").  Neighbours
// outside the grid are Dirichlet nodes and contribute nothing.
#pragma once
#include "helm_internal.cuh"

namespace helm {

// Along x the uniform-interior shortcut is decided for the aligned chunk of 32 points holding i:
// the chunk must lie inside the uniform run, else all its points take the per-axis tables.  The
// warps of the stencil kernels cover 32 consecutive x points from a multiple of 32, so a warp takes
// one formula along x instead of running both where the run begins or ends inside it; y and z are
// decided per point (a warp's points share them in the row-wise kernels).  The choice depends on a
// point's indices alone, so every kernel computes the same value at a point.
template <typename T>
__device__ __forceinline__ bool op_uniform_x(const OpView<T>& op, int i) {
  const int c0 = i & ~31;
  return c0 >= op.ulo[0] && c0 + 31 <= op.uhi[0];
}
template <int DIM, typename T>
__device__ __forceinline__ bool op_uniform(const OpView<T>& op, int i, int j, int l) {
  bool u = op_uniform_x(op, i);
  if (DIM > 1) u = u && j >= op.ulo[1] && j <= op.uhi[1];
  if (DIM > 2) u = u && l >= op.ulo[2] && l <= op.uhi[2];
  return u;
}

// Position of x index i in a row stored x-split (the red-black levels of 3D FP32 hierarchies):
// the even indices first, then the odd ones, h = (n0 + 1) / 2 of them even, so that the points of
// one colour in a row are contiguous.
__device__ __forceinline__ int xs_pos(int i, int h) { return (i & 1) ? h + (i >> 1) : (i >> 1); }

// Off-diagonal sum in the uniform interior; the x neighbours sit at pxm / pxp (p - 1 / p + 1 in
// natural order), the y and z neighbours one row or plane away.
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag_uniform(const OpView<T>& op, const cx<TX>* __restrict__ x, long p,
                                                    long pxm, long pxp) {
  cx<T> sx = cadd<T>(cconv<T, TX>(x[pxm]), cconv<T, TX>(x[pxp]));
  cx<T> sy, sz;
  if (DIM > 1) {
    long st = op.n[0];
    sy = cadd<T>(cconv<T, TX>(x[p - st]), cconv<T, TX>(x[p + st]));
  }
  if (DIM > 2) {
    long st = (long)op.n[0] * op.n[1];
    sz = cadd<T>(cconv<T, TX>(x[p - st]), cconv<T, TX>(x[p + st]));
  }
  if (DIM > 1 && op.uniform_iso) {  // one coefficient for all neighbours
    cx<T> sum = cadd<T>(sx, sy);
    if (DIM > 2) sum = cadd<T>(sum, sz);
    return op.uniform_real ? cscale<T>(op.ua[0].x, sum) : cmul<T>(op.ua[0], sum);
  }
  if (op.uniform_real) {
    cx<T> acc = cscale<T>(op.ua[0].x, sx);
    if (DIM > 1) acc = mkc<T>(fma(op.ua[1].x, sy.x, acc.x), fma(op.ua[1].x, sy.y, acc.y));
    if (DIM > 2) acc = mkc<T>(fma(op.ua[2].x, sz.x, acc.x), fma(op.ua[2].x, sz.y, acc.y));
    return acc;
  }
  cx<T> acc = cmul<T>(op.ua[0], sx);
  if (DIM > 1) acc = cfma<T>(op.ua[1], sy, acc);
  if (DIM > 2) acc = cfma<T>(op.ua[2], sz, acc);
  return acc;
}
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag_uniform(const OpView<T>& op, const cx<TX>* __restrict__ x, long p) {
  return op_offdiag_uniform<T, TX, DIM>(op, x, p, p - 1, p + 1);
}

// Off-diagonal sum of a point outside the uniform interior.  Axes along which the point still
// lies in the uniform run take the shared coefficient on the neighbour pair (one product instead
// of two); the others read their Shortley-Weller row, skipping Dirichlet neighbours.
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag_general(const OpView<T>& op, const cx<TX>* __restrict__ x,
                                                    int i, int j, int l, long p, long pxm, long pxp) {
  cx<T> acc = mkc<T>(T(0), T(0));
  const int idx[3] = {i, j, l};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const long st = a == 0 ? 1 : (a == 1 ? (long)op.n[0] : (long)op.n[0] * op.n[1]);
    const long qm = a == 0 ? pxm : p - st, qp = a == 0 ? pxp : p + st;
    const int q = idx[a];
    if (a == 0 ? op_uniform_x(op, q) : (q >= op.ulo[a] && q <= op.uhi[a])) {
      cx<T> pr = cadd<T>(cconv<T, TX>(x[qm]), cconv<T, TX>(x[qp]));
      acc = op.uniform_real ? mkc<T>(fma(op.ua[a].x, pr.x, acc.x), fma(op.ua[a].x, pr.y, acc.y))
                            : cfma<T>(op.ua[a], pr, acc);
    } else {
      if (q > 0) acc = cfma<T>(op.am[a][q], cconv<T, TX>(x[qm]), acc);
      if (q < op.n[a] - 1) acc = cfma<T>(op.ap[a][q], cconv<T, TX>(x[qp]), acc);
    }
  }
  return acc;
}
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag_general(const OpView<T>& op, const cx<TX>* __restrict__ x,
                                                    int i, int j, int l, long p) {
  return op_offdiag_general<T, TX, DIM>(op, x, i, j, l, p, p - 1, p + 1);
}

template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag(const OpView<T>& op, const cx<TX>* __restrict__ x,
                                            int i, int j, int l, long p) {
  if (op_uniform<DIM>(op, i, j, l)) return op_offdiag_uniform<T, TX, DIM>(op, x, p);
  return op_offdiag_general<T, TX, DIM>(op, x, i, j, l, p);
}

// (A x)_P.  In the uniform interior of an operator with real coefficients (H) the diagonal
// ud - s phi_P is real and multiplies x_P with two FMAs; elsewhere the stored diagonal is read
// when the operator has one.
// x is read at p (its x neighbours at pxm / pxp), the level's per-point tables (phi, the stored
// diagonal) at pn: p = pn in natural order.
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_row_at(const OpView<T>& op, const cx<TX>* __restrict__ x, int i, int j,
                                           int l, long p, long pn, long pxm, long pxp) {
  const cx<T> xp = cconv<T, TX>(x[p]);
  const T ph = op.phi ? op.phi[pn] : op.phi0;
  if (op_uniform<DIM>(op, i, j, l)) {
    const cx<T> off = op_offdiag_uniform<T, TX, DIM>(op, x, p, pxm, pxp);
    if (op.uniform_real) {
      const T d = fma(-ph, op.s.x, op.ud.x);
      return mkc<T>(fma(d, xp.x, off.x), fma(d, xp.y, off.y));
    }
    return cfma<T>(csub<T>(op.ud, cscale<T>(ph, op.s)), xp, off);
  }
  cx<T> d;
  if (op.dg) {
    d = op.dg[pn];  // the stored diagonal
  } else {
    d = op.a0[0][i];
    if (DIM > 1) d = cadd<T>(d, op.a0[1][j]);
    if (DIM > 2) d = cadd<T>(d, op.a0[2][l]);
    d = cadd<T>(d, cconv<T, double>(somm_diag(op, i, j, l, (double)ph)));
    d = op.phim ? csub<T>(d, cmul<T>(op.s, mkc<T>(ph, (T)op.phim[pn]))) : csub<T>(d, cscale<T>(ph, op.s));
  }
  return cfma<T>(d, xp, op_offdiag_general<T, TX, DIM>(op, x, i, j, l, p, pxm, pxp));
}
template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_row(const OpView<T>& op, const cx<TX>* __restrict__ x, int i,
                                        int j, int l, long p) {
  return op_row_at<T, TX, DIM>(op, x, i, j, l, p, p, p - 1, p + 1);
}

// 2D off-diagonal part from the four neighbour values (staged in shared memory by the fused
// kernels; zero outside the grid).
template <typename T>
__device__ __forceinline__ cx<T> off2d(const OpView<T>& op, int i, int j, cx<T> xw, cx<T> xe, cx<T> xs, cx<T> xn) {
  if (op_uniform<2>(op, i, j, 0)) {
    cx<T> sx = cadd<T>(xw, xe), sy = cadd<T>(xs, xn);
    if (op.uniform_iso) {
      cx<T> sum = cadd<T>(sx, sy);
      return op.uniform_real ? cscale<T>(op.ua[0].x, sum) : cmul<T>(op.ua[0], sum);
    }
    if (op.uniform_real) {
      cx<T> acc = cscale<T>(op.ua[0].x, sx);
      return mkc<T>(fma(op.ua[1].x, sy.x, acc.x), fma(op.ua[1].x, sy.y, acc.y));
    }
    return cfma<T>(op.ua[1], sy, cmul<T>(op.ua[0], sx));
  }
  // per axis: the shared coefficient on the pair where the axis is still uniform
  cx<T> acc;
  if (op_uniform_x(op, i)) {
    cx<T> pr = cadd<T>(xw, xe);
    acc = op.uniform_real ? cscale<T>(op.ua[0].x, pr) : cmul<T>(op.ua[0], pr);
  } else {
    acc = cfma<T>(op.ap[0][i], xe, cmul<T>(op.am[0][i], xw));
  }
  if (j >= op.ulo[1] && j <= op.uhi[1]) {
    cx<T> pr = cadd<T>(xs, xn);
    return op.uniform_real ? mkc<T>(fma(op.ua[1].x, pr.x, acc.x), fma(op.ua[1].x, pr.y, acc.y))
                           : cfma<T>(op.ua[1], pr, acc);
  }
  return cfma<T>(op.ap[1][j], xn, cfma<T>(op.am[1][j], xs, acc));
}

// point coordinates from a linear index
__device__ __forceinline__ void unflatten(long p, const int n[3], int& i, int& j, int& l) {
  i = (int)(p % n[0]);
  long q = p / n[0];
  j = (int)(q % n[1]);
  l = (int)(q / n[1]);
}

}  // namespace helm
