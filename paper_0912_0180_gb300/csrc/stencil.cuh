// stencil.cuh -- the Shortley-Weller row of a level operator evaluated at one grid point.
//   (A x)_P = sum_axes (am x_{P-e} + a0 x_P + ap x_{P+e}) - s * phi_P * x_P
// Section 3, eq. "shortwell", summed over axes; sigma = s * phi with s = 1 for H and CSG
// (eqs. "helmctu0", "lapctucsg") and s = beta^2 for CSL (eq. "helmctucsl").  Neighbours
// outside the grid are Dirichlet nodes and contribute nothing.
#pragma once
#include "helm_internal.cuh"

namespace helm {

template <int DIM, typename T>
__device__ __forceinline__ bool op_uniform(const OpView<T>& op, int i, int j, int l) {
  bool u = i >= op.ulo[0] && i <= op.uhi[0];
  if (DIM > 1) u = u && j >= op.ulo[1] && j <= op.uhi[1];
  if (DIM > 2) u = u && l >= op.ulo[2] && l <= op.uhi[2];
  return u;
}

template <typename T, int DIM>
__device__ __forceinline__ cx<T> op_diag(const OpView<T>& op, int i, int j, int l, long p) {
  if (op_uniform<DIM>(op, i, j, l)) {
    T ph = op.phi ? op.phi[p] : op.phi0;
    if (op.uniform_real) return mkc<T>(op.ud.x - ph * op.s.x, op.ud.y);
    return csub<T>(op.ud, cscale<T>(ph, op.s));
  }
  cx<T> d = op.a0[0][i];
  if (DIM > 1) d = cadd<T>(d, op.a0[1][j]);
  if (DIM > 2) d = cadd<T>(d, op.a0[2][l]);
  T ph = op.phi ? op.phi[p] : op.phi0;
  return csub<T>(d, cscale<T>(ph, op.s));
}

template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_offdiag_uniform(const OpView<T>& op, const cx<TX>* __restrict__ x, long p) {
  cx<T> sx = cadd<T>(cconv<T, TX>(x[p - 1]), cconv<T, TX>(x[p + 1]));
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
__device__ __forceinline__ cx<T> op_offdiag(const OpView<T>& op, const cx<TX>* __restrict__ x,
                                            int i, int j, int l, long p) {
  if (op_uniform<DIM>(op, i, j, l)) return op_offdiag_uniform<T, TX, DIM>(op, x, p);
  cx<T> acc = mkc<T>(T(0), T(0));
  if (i > 0) acc = cfma<T>(op.am[0][i], cconv<T, TX>(x[p - 1]), acc);
  if (i < op.n[0] - 1) acc = cfma<T>(op.ap[0][i], cconv<T, TX>(x[p + 1]), acc);
  if (DIM > 1) {
    long st = op.n[0];
    if (j > 0) acc = cfma<T>(op.am[1][j], cconv<T, TX>(x[p - st]), acc);
    if (j < op.n[1] - 1) acc = cfma<T>(op.ap[1][j], cconv<T, TX>(x[p + st]), acc);
  }
  if (DIM > 2) {
    long st = (long)op.n[0] * op.n[1];
    if (l > 0) acc = cfma<T>(op.am[2][l], cconv<T, TX>(x[p - st]), acc);
    if (l < op.n[2] - 1) acc = cfma<T>(op.ap[2][l], cconv<T, TX>(x[p + st]), acc);
  }
  return acc;
}

template <typename T, typename TX, int DIM>
__device__ __forceinline__ cx<T> op_row(const OpView<T>& op, const cx<TX>* __restrict__ x, int i,
                                        int j, int l, long p) {
  cx<T> d = op_diag<T, DIM>(op, i, j, l, p);
  return cfma<T>(d, cconv<T, TX>(x[p]), op_offdiag<T, TX, DIM>(op, x, i, j, l, p));
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
  cx<T> acc = cmul<T>(op.am[0][i], xw);
  acc = cfma<T>(op.ap[0][i], xe, acc);
  acc = cfma<T>(op.am[1][j], xs, acc);
  return cfma<T>(op.ap[1][j], xn, acc);
}

// point coordinates from a linear index
__device__ __forceinline__ void unflatten(long p, const int n[3], int& i, int& j, int& l) {
  i = (int)(p % n[0]);
  long q = p / n[0];
  j = (int)(q % n[1]);
  l = (int)(q / n[1]);
}

}  // namespace helm
