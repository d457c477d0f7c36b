// mg_fused.cu -- the V(1,1) cycle restructured for the GPU: the arithmetic of the per-component
// kernels of mg.cu (Section 5.1 / 6.1 components), fused so that a cycle costs few launches and
// little HBM traffic, and free of divisions (every level stores 1/D).
//
//  k_down2d  pre-smoothing sweep from the zero guess + residual + full-weighting restriction.
//            One block per 16 x 8 tile of coarse points; f of the fine tile plus a halo is
//            staged in shared memory, u is computed there and written once, and the residual
//            never leaves shared memory.  After a sweep from the zero guess the residual needs
//            no diagonal: D u = omega f for Jacobi, so r = (1 - omega) f - offdiag(u); for
//            red-black Gauss-Seidel r = -offdiag(u) on red points and r = 0 on black points.
//  k_up2d    bilinear prolongation of the coarse correction + the post-smoothing sweep, out of
//            place (reads u, writes the next iterate), halo staged in shared memory; the
//            finest level may write its result widened to complex128 (the precision boundary
//            into the FP64 Krylov vectors).
//  k_tail    the coarsest levels (a few hundred unknowns in FP32, a few dozen in FP64) in
//            ONE block: smoothing, residual, restriction, the dense coarsest solve,
//            prolongation and post-smoothing, with __syncthreads() between phases instead of
//            kernel launches.
//
// Outside the grid every value is a Dirichlet zero, as in the unfused kernels.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "stencil.cuh"

namespace helm {

// Tiles: the large ones (coarse 16 x 8 for k_down2d, fine 32 x 8 for k_up2d, 256 threads) on
// levels with at least two blocks per SM; otherwise quarter / half tiles of 128 threads, so
// that a small level still spreads over most SMs (in FP64 one block's arithmetic on one SM
// otherwise sets the level's time).  The autotuner chooses among these and a one-warp tile.
constexpr int DN_CX = 16, DN_CY = 8, DN_SCX = 8, DN_SCY = 4, DN_TCX = 4, DN_TCY = 2, DN_QCX = 8, DN_QCY = 8;
constexpr int UP_FX = 32, UP_FY = 8, UP_SFX = 16, UP_SFY = 8, UP_TFX = 8, UP_TFY = 4, UP_QFX = 16, UP_QFY = 16;
constexpr int FUSED_THREADS = 256, FUSED_SMALL_THREADS = 128, FUSED_TINY_THREADS = 32;
// tile choices (LevelHost::tile_down / tile_up): the autotuner also tries a tiny tile of one warp,
// which spreads a small FP64 level over many more SMs, and a square tile of 128 threads (8 x 8
// coarse / 16 x 16 fine), whose halo is smaller than the small tile's and whose block count falls
// between the small and the large tile's (for an even spread over the SMs)
// and a wide tile of 256 threads (16 x 12 coarse / 32 x 24 fine), whose halo is the smallest (the
// recomputed sweep and residual cost most in FP64, where the fine levels are bound by the FP64 pipe)
enum { TILE_SMALL = 0, TILE_BIG = 1, TILE_TINY = 2, TILE_SQUARE = 3, TILE_WIDE = 4 };
constexpr int NUM_TILES = 5;
constexpr int DN_WCX = 16, DN_WCY = 12, UP_WFX = 32, UP_WFY = 24;

// ---- down: smooth from zero + residual + restriction (2D, nu1 = 1) ---------------------------
// HF: halo of the staged region beyond the residual region (1 for Jacobi, 2 for RB-GS).
// The k-th point of colour c ((i + j) & 1 == c) of a W x H block whose corner is the grid point
// (gi0, gj0): row y = k / P, and in it the (k % P)-th point of that colour, P = ceil(W / 2) slots a
// row.  False when the slot lies past the end of a row with fewer points of that colour.  A loop
// over k < H P gives every lane of a warp a point of the colour, where a loop over all points
// leaves half of them idle on the colour's arithmetic.
__device__ __forceinline__ bool colour_item(int k, int W, int gi0, int gj0, int c, int& x, int& y) {
  const int P = (W + 1) >> 1;
  y = k / P;
  x = 2 * (k - y * P) + ((gi0 + gj0 + y + c) & 1);
  return x < W;
}

template <typename T, bool RBGS, int CX, int CY, int NT>
__device__ __forceinline__ void down2d_body(int bx_, int by_, const OpView<T>& op, int nc0, int nc1, const cx<T>* __restrict__ f, cx<T>* __restrict__ u_out,
         cx<T>* __restrict__ fc, T omega) {
  constexpr int HF = RBGS ? 2 : 1;
  constexpr int RX = 2 * CX + 1, RY = 2 * CY + 1;  // residual region
  constexpr int FX = RX + 2 * HF, FY = RY + 2 * HF;      // staged f / u region
  __shared__ cx<T> sf[FY][FX];
  __shared__ cx<T> su[FY][FX];
  __shared__ cx<T> sr[RY][RX];
  const int n0 = op.n[0], n1 = op.n[1];
  const int I0 = bx_ * CX, J0 = by_ * CY;
  const int fx0 = 2 * I0 - HF, fy0 = 2 * J0 - HF;  // origin of the staged region
  const int tid = threadIdx.x;
  // stage f; Jacobi: u = omega D^-1 f; RB-GS: red u = D^-1 f, black 0.  All loads of a
  // thread are issued before any is used.
  {
    constexpr int NS = (FX * FY + NT - 1) / NT;
    cx<T> fv[NS], dv[NS];
#pragma unroll
    for (int it = 0; it < NS; ++it) {
      int e = tid + it * NT;
      int x = e % FX, y = e / FX;
      int i = fx0 + x, j = fy0 + y;
      fv[it] = mkc<T>(T(0), T(0));
      dv[it] = mkc<T>(T(0), T(0));
      if (e < FX * FY && i >= 0 && i < n0 && j >= 0 && j < n1) {
        int p = i + n0 * j;
        fv[it] = f[p];
        dv[it] = op.dinv[p];
      }
    }
#pragma unroll
    for (int it = 0; it < NS; ++it) {
      int e = tid + it * NT;
      if (e >= FX * FY) break;
      int x = e % FX, y = e / FX;
      int i = fx0 + x, j = fy0 + y;
      cx<T> uv = mkc<T>(T(0), T(0));
      if (!RBGS || ((i + j) & 1) == 0) uv = cmul<T>(fv[it], dv[it]);  // dinv holds omega/D (Jacobi)
      sf[y][x] = fv[it];
      su[y][x] = uv;
    }
  }
  __syncthreads();
  if (RBGS) {  // black points of the inner region from the red values just computed
    constexpr int BW = FX - 2, BH = FY - 2;
    for (int e = tid; e < BH * ((BW + 1) / 2); e += NT) {
      int x, y;
      if (!colour_item(e, BW, fx0 + 1, fy0 + 1, 1, x, y)) continue;
      x += 1;
      y += 1;
      int i = fx0 + x, j = fy0 + y;
      if (i < 0 || i >= n0 || j < 0 || j >= n1) continue;
      cx<T> acc = off2d<T>(op, i, j, su[y][x - 1], su[y][x + 1], su[y - 1][x], su[y + 1][x]);
      su[y][x] = cmul<T>(csub<T>(sf[y][x], acc), op.dinv[i + n0 * j]);
    }
    __syncthreads();
  }
  // write the smoothed iterate of the points this tile owns (the last tile also owns the
  // fine point past the last coarse node when n is odd)
  {
    const int oi1 = (I0 + CX >= nc0) ? n0 : 2 * (I0 + CX);
    const int oj1 = (J0 + CY >= nc1) ? n1 : 2 * (J0 + CY);
    const int wx = oi1 - 2 * I0, wy = oj1 - 2 * J0;
    for (int e = tid; e < wx * wy; e += NT) {
      int x = e % wx, y = e / wx;
      int i = 2 * I0 + x, j = 2 * J0 + y;
      u_out[i + n0 * j] = su[y + HF][x + HF];
    }
  }
  // residual on the restriction region (fine 2I0 .. 2I0 + 2CX), zero outside the grid; with
  // red-black Gauss-Seidel only the red points have one, so the red points are one loop and the
  // black ones (zero) another (colour_item)
  if (!RBGS) {
    for (int e = tid; e < RX * RY; e += NT) {
      int x = e % RX, y = e / RX;
      int i = 2 * I0 + x, j = 2 * J0 + y;
      cx<T> rv = mkc<T>(T(0), T(0));
      if (i < n0 && j < n1) {
        int sx = x + HF, sy = y + HF;
        cx<T> acc = off2d<T>(op, i, j, su[sy][sx - 1], su[sy][sx + 1], su[sy - 1][sx], su[sy + 1][sx]);
        const T om1 = T(1) - omega;  // (1 - omega) f - acc in two fused multiply-adds, as k_resid0
        rv = mkc<T>(fma(om1, sf[sy][sx].x, -acc.x), fma(om1, sf[sy][sx].y, -acc.y));
      }
      sr[y][x] = rv;
    }
  } else {
    constexpr int RQ = RY * ((RX + 1) / 2);
    for (int e = tid; e < 2 * RQ; e += NT) {
      const int c = e < RQ ? 0 : 1;
      int x, y;
      if (!colour_item(e - c * RQ, RX, 2 * I0, 2 * J0, c, x, y)) continue;
      int i = 2 * I0 + x, j = 2 * J0 + y;
      cx<T> rv = mkc<T>(T(0), T(0));
      if (c == 0 && i < n0 && j < n1) {
        int sx = x + HF, sy = y + HF;
        cx<T> acc = off2d<T>(op, i, j, su[sy][sx - 1], su[sy][sx + 1], su[sy - 1][sx], su[sy + 1][sx]);
        rv = mkc<T>(-acc.x, -acc.y);
      }
      sr[y][x] = rv;
    }
  }
  __syncthreads();
  // full weighting (1/4, 1/2, 1/4 per axis)
  for (int e = tid; e < CX * CY; e += NT) {
    int cx_ = e % CX, cy = e / CX;
    int I = I0 + cx_, J = J0 + cy;
    if (I >= nc0 || J >= nc1) continue;
    // separable weights: each row (a + c) + 2 b, then the rows the same way, then / 16
    cx<T> rw[3];
#pragma unroll
    for (int dj = 0; dj < 3; ++dj) {
      cx<T> a = sr[2 * cy + dj][2 * cx_], b = sr[2 * cy + dj][2 * cx_ + 1], c = sr[2 * cy + dj][2 * cx_ + 2];
      rw[dj] = mkc<T>(fma(T(2), b.x, a.x + c.x), fma(T(2), b.y, a.y + c.y));
    }
    cx<T> acc = mkc<T>(fma(T(2), rw[1].x, rw[0].x + rw[2].x), fma(T(2), rw[1].y, rw[0].y + rw[2].y));
    fc[I + nc0 * J] = cscale<T>(T(0.0625), acc);
  }
}
template <typename T, bool RBGS, int CX, int CY, int NT>
__global__ void __launch_bounds__(NT)
k_down2d(OpView<T> op, int nc0, int nc1, const cx<T>* __restrict__ f, cx<T>* __restrict__ u_out,
         cx<T>* __restrict__ fc, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  down2d_body<T, RBGS, CX, CY, NT>(blockIdx.x, blockIdx.y, op, nc0, nc1, f, u_out, fc, omega);
}

// ---- up: prolongation + correction + post-smoothing (2D, nu2 = 1), out of place --------------
template <typename T, bool RBGS, typename TO, int FX, int FY, int NT>
__device__ __forceinline__ void up2d_body(int bx_, int by_, const OpView<T>& op, int nc0, int nc1, const cx<T>* __restrict__ u_in, const cx<T>* __restrict__ ec,
       const cx<T>* __restrict__ f, cx<TO>* __restrict__ u_out, T omega) {
  constexpr int HU = RBGS ? 2 : 1;                 // halo of the corrected iterate
  constexpr int UX = FX + 2 * HU, UY = FY + 2 * HU;
  constexpr int CXN = UX / 2 + 3, CYN = UY / 2 + 3;  // coarse values covering the region
  __shared__ cx<T> su[UY][UX];
  __shared__ cx<T> se[CYN][CXN];
  const int n0 = op.n[0], n1 = op.n[1];
  const int i0 = bx_ * FX, j0 = by_ * FY;
  const int ux0 = i0 - HU, uy0 = j0 - HU;
  const int cx0 = (ux0 >> 1) - 1, cy0 = (uy0 >> 1) - 1;  // floor division for negatives
  const int tid = threadIdx.x;
  for (int e = tid; e < CXN * CYN; e += NT) {
    int x = e % CXN, y = e / CXN;
    int I = cx0 + x, J = cy0 + y;
    se[y][x] = (I >= 0 && I < nc0 && J >= 0 && J < nc1) ? ec[I + nc0 * J] : mkc<T>(T(0), T(0));
  }
  __syncthreads();
  // corrected iterate u + P e on the tile and its halo (u loads issued up front).  The region's
  // points are taken parity class by parity class (local offsets (c & 1, c >> 1) on a 2 x 2
  // lattice; UX and UY are even, so every class has the same number of points and its own fine
  // (i, j) parities): a warp then takes one or two classes, not all four, and a class sums only the
  // one, two or four coarse values it needs.
  static_assert(UX % 2 == 0 && UY % 2 == 0, "parity classes of equal size");
  constexpr int HX = UX / 2, QC = HX * (UY / 2);
  auto item = [&](int e, int& x, int& y) {
    const int c = e / QC, k = e - c * QC;
    x = 2 * (k % HX) + (c & 1);
    y = 2 * (k / HX) + (c >> 1);
  };
  constexpr int NU = (UX * UY + NT - 1) / NT;
  cx<T> uold[NU];
#pragma unroll
  for (int it = 0; it < NU; ++it) {
    int e = tid + it * NT, x, y;
    item(e, x, y);
    int i = ux0 + x, j = uy0 + y;
    uold[it] = (e < UX * UY && i >= 0 && i < n0 && j >= 0 && j < n1) ? u_in[i + n0 * j] : mkc<T>(T(0), T(0));
  }
#pragma unroll
  for (int it = 0; it < NU; ++it) {
    int e = tid + it * NT, x, y;
    if (e >= UX * UY) break;
    item(e, x, y);
    int i = ux0 + x, j = uy0 + y;
    cx<T> v = mkc<T>(T(0), T(0));
    if (i >= 0 && i < n0 && j >= 0 && j < n1) {
      // per axis: odd fine index -> one coarse node, even -> the two around it (coarse index k
      // is se[.][k - c0]; indices outside the coarse grid read zero)
      int ia = (i & 1) ? (i - 1) >> 1 : (i >> 1) - 1, ib = (i & 1) ? ia : (i >> 1);
      int ja = (j & 1) ? (j - 1) >> 1 : (j >> 1) - 1, jb = (j & 1) ? ja : (j >> 1);
      T w = ((i & 1) ? T(1) : T(0.5)) * ((j & 1) ? T(1) : T(0.5));
      cx<T> acc = se[ja - cy0][ia - cx0];
      if (ib != ia) acc = cadd<T>(acc, se[ja - cy0][ib - cx0]);
      if (jb != ja) {
        acc = cadd<T>(acc, se[jb - cy0][ia - cx0]);
        if (ib != ia) acc = cadd<T>(acc, se[jb - cy0][ib - cx0]);
      }
      // the weight is a power of two, so w acc is exact and one FMA gives u + w acc as before
      const cx<T> uo = uold[it];
      v = mkc<T>(fma(w, acc.x, uo.x), fma(w, acc.y, uo.y));
    }
    su[y][x] = v;
  }
  __syncthreads();
  if (!RBGS) {
    for (int e = tid; e < FX * FY; e += NT) {
      int x = e % FX, y = e / FX;
      int i = i0 + x, j = j0 + y;
      if (i >= n0 || j >= n1) continue;
      int p = i + n0 * j;
      int sx = x + HU, sy = y + HU;
      cx<T> acc = off2d<T>(op, i, j, su[sy][sx - 1], su[sy][sx + 1], su[sy - 1][sx], su[sy + 1][sx]);
      cx<T> g = cmul<T>(csub<T>(f[p], acc), op.dinv[p]);  // dinv holds omega / D
      cx<T> uc = su[sy][sx];
      const T om1 = T(1) - omega;
      u_out[p] = cconv<TO, T>(mkc<T>(fma(om1, uc.x, g.x), fma(om1, uc.y, g.y)));
    }
  } else {
    // red points of the tile and one ring around it, from the corrected black values; the black
    // ones are copied.  Each colour is its own loop (colour_item), so no lane idles on the update.
    __shared__ cx<T> sred[FY + 2][FX + 2];
    constexpr int RW = FX + 2, RH = FY + 2, RQ = RH * ((RW + 1) / 2);
    for (int e = tid; e < 2 * RQ; e += NT) {
      const int c = e < RQ ? 0 : 1;  // red (updated), then black (copied)
      int x, y;
      if (!colour_item(e - c * RQ, RW, i0 - 1, j0 - 1, c, x, y)) continue;
      int i = i0 - 1 + x, j = j0 - 1 + y;
      int sx = x + 1, sy = y + 1;  // position in su (HU = 2)
      cx<T> v = su[sy][sx];
      if (c == 0 && i >= 0 && i < n0 && j >= 0 && j < n1) {
        int p = i + n0 * j;
        cx<T> acc = off2d<T>(op, i, j, su[sy][sx - 1], su[sy][sx + 1], su[sy - 1][sx], su[sy + 1][sx]);
        v = cmul<T>(csub<T>(f[p], acc), op.dinv[p]);
      }
      sred[y][x] = v;
    }
    __syncthreads();
    constexpr int BQ = FY * ((FX + 1) / 2);
    for (int e = tid; e < 2 * BQ; e += NT) {
      const int c = e < BQ ? 1 : 0;  // black (updated), then red (written as they are)
      int x, y;
      if (!colour_item(e - (1 - c) * BQ, FX, i0, j0, c, x, y)) continue;
      int i = i0 + x, j = j0 + y;
      if (i >= n0 || j >= n1) continue;
      int p = i + n0 * j;
      int sx = x + 1, sy = y + 1;  // position in sred
      cx<T> v = sred[sy][sx];
      if (c == 1) {
        cx<T> acc = off2d<T>(op, i, j, sred[sy][sx - 1], sred[sy][sx + 1], sred[sy - 1][sx], sred[sy + 1][sx]);
        v = cmul<T>(csub<T>(f[p], acc), op.dinv[p]);
      }
      u_out[p] = cconv<TO, T>(v);
    }
  }
}
template <typename T, bool RBGS, typename TO, int FX, int FY, int NT>
__global__ void __launch_bounds__(NT)
k_up2d(OpView<T> op, int nc0, int nc1, const cx<T>* __restrict__ u_in, const cx<T>* __restrict__ ec,
       const cx<T>* __restrict__ f, cx<TO>* __restrict__ u_out, T omega, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  up2d_body<T, RBGS, TO, FX, FY, NT>(blockIdx.x, blockIdx.y, op, nc0, nc1, u_in, ec, f, u_out, omega);
}

// ---- tail: the coarsest levels in one block ------------------------------------------------
constexpr int TAIL_MAX_LEVELS = 12;
constexpr int TAIL_THREADS = 1024;

template <typename T> struct TailArgs {
  int count;                        // levels in the tail (the last is the coarsest)
  OpView<T> op[TAIL_MAX_LEVELS];
  int n[TAIL_MAX_LEVELS];
  int off[TAIL_MAX_LEVELS];         // offset (elements) of each level's vectors in shared memory
  int toff[TAIL_MAX_LEVELS];        // offset of its coefficient tables (am, a0, ap per axis)
  int aoff;                         // offset of the staged coarsest inverse, -1: read from global
  const cx<T>* ainv;
  int nco;
  int nu1, nu2, smoother;
  T omega;
};

// Level k keeps five vectors in shared memory at base + off[k]: two iterate buffers (which one
// holds u is bit k of `swap`; a Jacobi sweep writes the other and flips it), f, 1/D and D
// (the last two copied in once, so that no phase waits on a global load).
constexpr int TAIL_VECS = 5;
template <typename T> struct TailMem {
  cx<T>* base;
  const TailArgs<T>* a;
  unsigned swap;
  __device__ cx<T>* U(int k) const { return base + a->off[k] + (((swap >> k) & 1u) ? a->n[k] : 0); }
  __device__ cx<T>* W(int k) const { return base + a->off[k] + (((swap >> k) & 1u) ? 0 : a->n[k]); }
  __device__ cx<T>* F(int k) const { return base + a->off[k] + 2 * a->n[k]; }
  __device__ cx<T>* DI(int k) const { return base + a->off[k] + 3 * a->n[k]; }
  __device__ cx<T>* DG(int k) const { return base + a->off[k] + 4 * a->n[k]; }
};

// Calls body(i, j, l, p) for every point of a level: each warp takes whole rows (fixed j, l) and
// its lanes walk along x, so no point needs an index division.
template <typename F>
__device__ __forceinline__ void tail_for_each(const int n[3], F&& body) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = n[1] * n[2];
  for (int row = warp; row < rows; row += TAIL_THREADS / 32) {
    const int j = row % n[1], l = row / n[1];
    const int base = row * n[0];
    for (int i = lane; i < n[0]; i += 32) body(i, j, l, base + i);
  }
}

template <typename T, int DIM>
__device__ void tail_smooth(const TailArgs<T>& a, const OpView<T>& op, TailMem<T>& m, int k, bool zero) {
  cx<T>* u = m.U(k);
  const cx<T>* f = m.F(k);
  const cx<T>* sdinv = m.DI(k);  // omega / D (Jacobi) or 1 / D (Gauss-Seidel)
  const T om1 = T(1) - a.omega;
  if (a.smoother == HELM_SM_JACOBI) {
    cx<T>* w = m.W(k);
    tail_for_each(op.n, [&](int i, int j, int l, int p) {
      if (zero) {
        w[p] = cmul<T>(f[p], sdinv[p]);
      } else {
        cx<T> g = cmul<T>(csub<T>(f[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)), sdinv[p]);
        cx<T> u0 = u[p];
        w[p] = mkc<T>(fma(om1, u0.x, g.x), fma(om1, u0.y, g.y));
      }
    });
    __syncthreads();
    m.swap ^= 1u << k;
  } else {
    for (int colour = 0; colour < 2; ++colour) {
      tail_for_each(op.n, [&](int i, int j, int l, int p) {
        int c = (i + j + l) & 1;
        if (zero && colour == 0) {
          u[p] = c == 0 ? cmul<T>(f[p], sdinv[p]) : mkc<T>(T(0), T(0));
        } else if (c == colour) {
          u[p] = cmul<T>(csub<T>(f[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)), sdinv[p]);
        }
      });
      __syncthreads();
    }
  }
}

// linear interpolation weights of fine index x from coarse indices (at most 2)
template <typename T>
__device__ __forceinline__ int tail_lin(int x, int nc, int* c, T* w) {
  if (x & 1) { c[0] = (x - 1) >> 1; w[0] = T(1); return 1; }
  int m = 0;
  if ((x >> 1) - 1 >= 0) { c[m] = (x >> 1) - 1; w[m] = T(0.5); ++m; }
  if ((x >> 1) < nc) { c[m] = x >> 1; w[m] = T(0.5); ++m; }
  return m;
}

template <typename T, int DIM, typename TO>
__device__ __forceinline__ void tail_body(const TailArgs<T>& a, const cx<T>* __restrict__ f_in,
                                          cx<TO>* __restrict__ u_outg) {
  extern __shared__ unsigned char tail_smem[];
  // every level's operator with its coefficient tables redirected to shared-memory copies, so
  // that no phase waits on a global load
  __shared__ OpView<T> sop[TAIL_MAX_LEVELS];
  TailMem<T> m{reinterpret_cast<cx<T>*>(tail_smem), &a, 0u};
  {
    cx<T>* F0 = m.F(0);
    for (int p = threadIdx.x; p < a.n[0]; p += TAIL_THREADS) F0[p] = f_in[p];
    for (int k = 0; k < a.count; ++k) {
      cx<T>* di = m.DI(k);
      cx<T>* dg = m.DG(k);
      for (int p = threadIdx.x; p < a.n[k]; p += TAIL_THREADS) {
        di[p] = a.op[k].dinv[p];
        dg[p] = a.op[k].dg[p];
      }
      cx<T>* tb = m.base + a.toff[k];
      for (int ax = 0; ax < DIM; ++ax) {
        const int na = a.op[k].n[ax];
        for (int q = threadIdx.x; q < 3 * na; q += TAIL_THREADS) {
          const int which = q / na, idx = q - which * na;
          const cx<T>* src = which == 0 ? a.op[k].am[ax] : (which == 1 ? a.op[k].a0[ax] : a.op[k].ap[ax]);
          tb[q] = src[idx];
        }
        tb += 3 * na;
      }
    }
    if (a.aoff >= 0) {
      cx<T>* ai = m.base + a.aoff;
      for (int q = threadIdx.x; q < a.nco * a.nco; q += TAIL_THREADS) ai[q] = a.ainv[q];
    }
    if (threadIdx.x < a.count) {
      const int k = threadIdx.x;
      OpView<T> v = a.op[k];
      cx<T>* tb = m.base + a.toff[k];
      for (int ax = 0; ax < DIM; ++ax) {
        const int na = v.n[ax];
        v.am[ax] = tb;
        v.a0[ax] = tb + na;
        v.ap[ax] = tb + 2 * na;
        tb += 3 * na;
      }
      sop[k] = v;
    }
  }
  __syncthreads();
  const int last = a.count - 1;
  // down: smooth, residual, full weighting into the next level's f
  for (int k = 0; k < last; ++k) {
    const OpView<T>& op = sop[k];
    const int n = a.n[k];
    if (a.nu1 > 0) {
      for (int s = 0; s < a.nu1; ++s) tail_smooth<T, DIM>(a, op, m, k, s == 0);
      cx<T>* u = m.U(k);
      cx<T>* w = m.W(k);
      const cx<T>* f = m.F(k);
      const cx<T>* dg = m.DG(k);
      tail_for_each(op.n, [&](int i, int j, int l, int p) {
        w[p] = csub<T>(f[p], cfma<T>(dg[p], u[p], op_offdiag<T, T, DIM>(op, u, i, j, l, p)));
      });
    } else {
      cx<T>* u = m.U(k);
      cx<T>* w = m.W(k);
      const cx<T>* f = m.F(k);
      for (int p = threadIdx.x; p < n; p += TAIL_THREADS) { w[p] = f[p]; u[p] = mkc<T>(T(0), T(0)); }
    }
    __syncthreads();
    const OpView<T>& oc = sop[k + 1];
    const cx<T>* r = m.W(k);
    cx<T>* fc = m.F(k + 1);
    const T wts[3] = {T(0.25), T(0.5), T(0.25)};
    tail_for_each(oc.n, [&](int I, int J, int Lz, int q) {
      cx<T> acc = mkc<T>(T(0), T(0));
      for (int dl = (DIM > 2 ? -1 : 0); dl <= (DIM > 2 ? 1 : 0); ++dl) {
        int fl = DIM > 2 ? 2 * Lz + 1 + dl : 0;
        if (fl >= op.n[2]) continue;
        for (int dj = (DIM > 1 ? -1 : 0); dj <= (DIM > 1 ? 1 : 0); ++dj) {
          int fj = DIM > 1 ? 2 * J + 1 + dj : 0;
          if (fj >= op.n[1]) continue;
          for (int di = -1; di <= 1; ++di) {
            int fi = 2 * I + 1 + di;
            if (fi >= op.n[0]) continue;
            T wt = wts[di + 1] * (DIM > 1 ? wts[dj + 1] : T(1)) * (DIM > 2 ? wts[dl + 1] : T(1));
            acc = cadd<T>(acc, cscale<T>(wt, r[fi + op.n[0] * (fj + op.n[1] * fl)]));
          }
        }
      }
      fc[q] = acc;
    });
    __syncthreads();
  }
  // coarsest: dense inverse, one warp per row
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const cx<T>* fl = m.F(last);
    cx<T>* ul = m.U(last);
    const cx<T>* ainv = a.aoff >= 0 ? m.base + a.aoff : a.ainv;
    for (int row = warp; row < a.nco; row += TAIL_THREADS / 32) {
      cx<T> acc = mkc<T>(T(0), T(0));
      for (int c = lane; c < a.nco; c += 32) acc = cfma<T>(ainv[row * a.nco + c], fl[c], acc);
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) ul[row] = acc;
    }
    __syncthreads();
  }
  // up: prolongation + correction, post-smoothing
  for (int k = last - 1; k >= 0; --k) {
    const OpView<T>& op = sop[k];
    const OpView<T>& oc = sop[k + 1];
    cx<T>* u = m.U(k);
    const cx<T>* e = m.U(k + 1);
    tail_for_each(op.n, [&](int i, int j, int l, int p) {
      int ci[2], cj[2] = {0, 0}, cl[2] = {0, 0};
      T wi[2], wj[2] = {T(1), T(1)}, wl[2] = {T(1), T(1)};
      int ni = tail_lin<T>(i, oc.n[0], ci, wi);
      int nj = DIM > 1 ? tail_lin<T>(j, oc.n[1], cj, wj) : 1;
      int nl = DIM > 2 ? tail_lin<T>(l, oc.n[2], cl, wl) : 1;
      cx<T> acc = mkc<T>(T(0), T(0));
      for (int c3 = 0; c3 < nl; ++c3)
        for (int c2 = 0; c2 < nj; ++c2)
          for (int c1 = 0; c1 < ni; ++c1)
            acc = cadd<T>(acc, cscale<T>(wi[c1] * wj[c2] * wl[c3], e[ci[c1] + oc.n[0] * (cj[c2] + oc.n[1] * cl[c3])]));
      u[p] = cadd<T>(u[p], acc);
    });
    __syncthreads();
    for (int s = 0; s < a.nu2; ++s) tail_smooth<T, DIM>(a, op, m, k, false);
  }
  {
    const cx<T>* u0 = m.U(0);
    for (int p = threadIdx.x; p < a.n[0]; p += TAIL_THREADS) u_outg[p] = cconv<TO, T>(u0[p]);
  }
}

template <typename T, int DIM, typename TO>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail(const __grid_constant__ TailArgs<T> a,
                                                       const cx<T>* __restrict__ f_in,
                                                       cx<TO>* __restrict__ u_outg, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  tail_body<T, DIM, TO>(a, f_in, u_outg);
}

// ---- host side ----------------------------------------------------------------------------

// Points handled by the single block: its phases cost a fraction of a microsecond each only while
// the block's threads have a few points each; FP64 runs at about a sixtieth of the FP32 rate, so
// its tail stays tiny.
template <typename T> static long tail_point_budget() { return std::is_same<T, double>::value ? 40 : 700; }
constexpr size_t TAIL_SMEM_BUDGET = 200 * 1024;
constexpr size_t TAIL_INVERSE_BYTES = 1 << 20;

template <typename T> int tail_first_level(const helm_ctx* c, long point_budget) {
  int nl = (int)c->lv.size();
  if (c->fdm.on) return nl;  // the one-block tail needs the dense coarsest inverse
  if (c->lv[0].any_offset0()) return nl;  // ... and coarsens with offset 1
  if (c->lv[nl - 1].stg64) return nl;  // ... and runs 5-point rows only
  long pts = c->lv[nl - 1].ntot;
  size_t bytes = TAIL_VECS * sizeof(cx<T>) * c->lv[nl - 1].ntot;
  if (bytes > TAIL_SMEM_BUDGET) return nl;  // the coarsest level alone is too big: no tail
  // one block streaming the dense coarsest inverse is slower than the whole-GPU product
  if ((size_t)pts * pts * sizeof(cx<T>) > TAIL_INVERSE_BYTES) return nl;
  int first = nl - 1;
  while (first > 0 && nl - (first - 1) <= TAIL_MAX_LEVELS) {
    long np = pts + c->lv[first - 1].ntot;
    size_t nb = bytes + TAIL_VECS * sizeof(cx<T>) * c->lv[first - 1].ntot;
    if (np > point_budget || nb > TAIL_SMEM_BUDGET) break;
    pts = np;
    bytes = nb;
    --first;
  }
  return first;
}

template <typename T, typename TO>
static helm_status tail_launch(const TailArgs<T>& a, int dim, size_t smem, const cx<T>* f, cx<TO>* out,
                               const int* skip, cudaStream_t st) {
  switch (dim) {
    case 1:
      HELM_CUDA(cudaFuncSetAttribute(k_tail<T, 1, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      launch_pdl(k_tail<T, 1, TO>, dim3(1), dim3(TAIL_THREADS), smem, st, a, f, out, skip);
      break;
    case 2:
      HELM_CUDA(cudaFuncSetAttribute(k_tail<T, 2, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      launch_pdl(k_tail<T, 2, TO>, dim3(1), dim3(TAIL_THREADS), smem, st, a, f, out, skip);
      break;
    default:
      HELM_CUDA(cudaFuncSetAttribute(k_tail<T, 3, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      launch_pdl(k_tail<T, 3, TO>, dim3(1), dim3(TAIL_THREADS), smem, st, a, f, out, skip);
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

// The tail's arguments for levels first.. of c, and the dynamic shared memory it needs.
template <typename T>
static size_t tail_args(const helm_ctx* c, int first, TailArgs<T>& a) {
  a = TailArgs<T>{};
  int nl = (int)c->lv.size();
  a.count = nl - first;
  int off = 0;
  for (int k = 0; k < a.count; ++k) {
    const LevelHost& L = c->lv[first + k];
    a.op[k] = L.view<T>();
    a.n[k] = (int)L.ntot;
    a.off[k] = off;
    off += TAIL_VECS * (int)L.ntot;
  }
  for (int k = 0; k < a.count; ++k) {
    const LevelHost& L = c->lv[first + k];
    a.toff[k] = off;
    for (int ax = 0; ax < L.dim; ++ax) off += 3 * L.n[ax];
  }
  a.ainv = (const cx<T>*)c->coarse_inv;
  a.nco = c->nco;
  a.aoff = -1;
  if ((size_t)(off + c->nco * c->nco) * sizeof(cx<T>) <= TAIL_SMEM_BUDGET) {
    a.aoff = off;
    off += c->nco * c->nco;
  }
  a.nu1 = c->pc.nu1;
  a.nu2 = c->pc.nu2;
  a.smoother = c->pc.smoother;
  a.omega = (T)c->pc.omega;
  return (size_t)off * sizeof(cx<T>);
}

template <typename T>
helm_status tail_vcycle(helm_ctx* c, int first, const cx<T>* f, void* out, bool out_f64, const int* skip,
                        cudaStream_t st) {
  TailArgs<T> a;
  const size_t smem = tail_args<T>(c, first, a);
  if (out_f64) return tail_launch<T, double>(a, c->grid.dim, smem, f, (double2*)out, skip, st);
  return tail_launch<T, T>(a, c->grid.dim, smem, f, (cx<T>*)out, skip, st);
}

static bool big_tiles(const helm_ctx* c, long blocks) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  return blocks >= 2L * sms;
}

template <typename T, bool RB, int CX, int CY, int NT>
static void down_launch(const LevelHost& F, const LevelHost& C, const cx<T>* f, cx<T>* u_out, cx<T>* fc, T om,
                        const int* skip, cudaStream_t st) {
  dim3 g((C.n[0] + CX - 1) / CX, (C.n[1] + CY - 1) / CY);
  launch_pdl(k_down2d<T, RB, CX, CY, NT>, dim3(g), dim3(NT), 0, st, F.view<T>(), C.n[0], C.n[1], f, u_out, fc, om, skip);
}

template <typename T, bool RB>
static void down_tile(int tile, const LevelHost& F, const LevelHost& C, const cx<T>* f, cx<T>* u_out, cx<T>* fc, T om,
                      const int* skip, cudaStream_t st) {
  if (tile == TILE_BIG) down_launch<T, RB, DN_CX, DN_CY, FUSED_THREADS>(F, C, f, u_out, fc, om, skip, st);
  else if (tile == TILE_TINY) down_launch<T, RB, DN_TCX, DN_TCY, FUSED_TINY_THREADS>(F, C, f, u_out, fc, om, skip, st);
  else if (tile == TILE_SQUARE) down_launch<T, RB, DN_QCX, DN_QCY, FUSED_SMALL_THREADS>(F, C, f, u_out, fc, om, skip, st);
  else if (tile == TILE_WIDE) down_launch<T, RB, DN_WCX, DN_WCY, FUSED_THREADS>(F, C, f, u_out, fc, om, skip, st);
  else down_launch<T, RB, DN_SCX, DN_SCY, FUSED_SMALL_THREADS>(F, C, f, u_out, fc, om, skip, st);
}

// The tile a level's fused kernels use (the autotuner's choice, else the block-count rule) and its
// coarse (down) or fine (up) extent.
static int down_tile_of(const helm_ctx* c, int l, int* tx, int* ty) {
  const LevelHost& F = c->lv[l];
  const LevelHost& C = c->lv[l + 1];
  long nb = (long)((C.n[0] + DN_CX - 1) / DN_CX) * ((C.n[1] + DN_CY - 1) / DN_CY);
  int tile = F.tile_down >= 0 ? F.tile_down : (big_tiles(c, nb) ? TILE_BIG : TILE_SMALL);
  *tx = tile == TILE_BIG ? DN_CX : tile == TILE_TINY ? DN_TCX : tile == TILE_SQUARE ? DN_QCX
      : tile == TILE_WIDE ? DN_WCX : DN_SCX;
  *ty = tile == TILE_BIG ? DN_CY : tile == TILE_TINY ? DN_TCY : tile == TILE_SQUARE ? DN_QCY
      : tile == TILE_WIDE ? DN_WCY : DN_SCY;
  return tile;
}
static int up_tile_of(const helm_ctx* c, int l, int* tx, int* ty) {
  const LevelHost& F = c->lv[l];
  long nb = (long)((F.n[0] + UP_FX - 1) / UP_FX) * ((F.n[1] + UP_FY - 1) / UP_FY);
  int tile = F.tile_up >= 0 ? F.tile_up : (big_tiles(c, nb) ? TILE_BIG : TILE_SMALL);
  *tx = tile == TILE_BIG ? UP_FX : tile == TILE_TINY ? UP_TFX : tile == TILE_SQUARE ? UP_QFX
      : tile == TILE_WIDE ? UP_WFX : UP_SFX;
  *ty = tile == TILE_BIG ? UP_FY : tile == TILE_TINY ? UP_TFY : tile == TILE_SQUARE ? UP_QFY
      : tile == TILE_WIDE ? UP_WFY : UP_SFY;
  return tile;
}

template <typename T>
void fused_down2d(const helm_ctx* c, int l, const cx<T>* f, cx<T>* u_out, cx<T>* fc, const int* skip, cudaStream_t st) {
  const LevelHost& F = c->lv[l];
  const LevelHost& C = c->lv[l + 1];
  long nb = (long)((C.n[0] + DN_CX - 1) / DN_CX) * ((C.n[1] + DN_CY - 1) / DN_CY);
  int tile = F.tile_down >= 0 ? F.tile_down : (big_tiles(c, nb) ? TILE_BIG : TILE_SMALL);
  T om = (T)c->pc.omega;
  if (c->pc.smoother == HELM_SM_RBGS) down_tile<T, true>(tile, F, C, f, u_out, fc, om, skip, st);
  else down_tile<T, false>(tile, F, C, f, u_out, fc, om, skip, st);
}

template <typename T, bool RB, typename TO, int FX, int FY, int NT>
static void up_launch(const LevelHost& F, const LevelHost& C, const cx<T>* u_in, const cx<T>* ec, const cx<T>* f,
                      TO* out, T om, const int* skip, cudaStream_t st) {
  dim3 g((F.n[0] + FX - 1) / FX, (F.n[1] + FY - 1) / FY);
  launch_pdl(k_up2d<T, RB, TO, FX, FY, NT>, dim3(g), dim3(NT), 0, st, F.view<T>(), C.n[0], C.n[1], u_in, ec, f,
             (cx<TO>*)out, om, skip);
}

template <typename T, bool RB, typename TO>
static void up_tile(int tile, const LevelHost& F, const LevelHost& C, const cx<T>* u_in, const cx<T>* ec,
                    const cx<T>* f, TO* o, T om, const int* skip, cudaStream_t st) {
  if (tile == TILE_BIG) up_launch<T, RB, TO, UP_FX, UP_FY, FUSED_THREADS>(F, C, u_in, ec, f, o, om, skip, st);
  else if (tile == TILE_TINY) up_launch<T, RB, TO, UP_TFX, UP_TFY, FUSED_TINY_THREADS>(F, C, u_in, ec, f, o, om, skip, st);
  else if (tile == TILE_SQUARE) up_launch<T, RB, TO, UP_QFX, UP_QFY, FUSED_SMALL_THREADS>(F, C, u_in, ec, f, o, om, skip, st);
  else if (tile == TILE_WIDE) up_launch<T, RB, TO, UP_WFX, UP_WFY, FUSED_THREADS>(F, C, u_in, ec, f, o, om, skip, st);
  else up_launch<T, RB, TO, UP_SFX, UP_SFY, FUSED_SMALL_THREADS>(F, C, u_in, ec, f, o, om, skip, st);
}

template <typename T, typename TO>
static void up_dispatch(const helm_ctx* c, const LevelHost& F, const LevelHost& C, const cx<T>* u_in, const cx<T>* ec,
                        const cx<T>* f, void* out, const int* skip, cudaStream_t st) {
  long nb = (long)((F.n[0] + UP_FX - 1) / UP_FX) * ((F.n[1] + UP_FY - 1) / UP_FY);
  int tile = F.tile_up >= 0 ? F.tile_up : (big_tiles(c, nb) ? TILE_BIG : TILE_SMALL);
  T om = (T)c->pc.omega;
  TO* o = (TO*)out;
  if (c->pc.smoother == HELM_SM_RBGS) up_tile<T, true, TO>(tile, F, C, u_in, ec, f, o, om, skip, st);
  else up_tile<T, false, TO>(tile, F, C, u_in, ec, f, o, om, skip, st);
}

template <typename T>
void fused_up2d(const helm_ctx* c, int l, const cx<T>* u_in, const cx<T>* ec, const cx<T>* f, void* out,
                bool out_f64, const int* skip, cudaStream_t st) {
  const LevelHost& F = c->lv[l];
  const LevelHost& C = c->lv[l + 1];
  if (out_f64) up_dispatch<T, double>(c, F, C, u_in, ec, f, out, skip, st);
  else up_dispatch<T, T>(c, F, C, u_in, ec, f, out, skip, st);
}

// ---- grouped V-cycle: one launch per level for many instances --------------------------------
// The instances of a group (2D, fused V(1,1) levels) run their V-cycles together: level l of every
// instance that still has a fused level there goes out in one k_down2d launch per tile shape (and
// one k_up2d launch on the way up), the one-block tails in one launch, and the coarsest dense
// solves of the others in one launch.  Each launch walks a work list (group_visit) whose virtual
// blocks are the instances' own tiles (or rows, or tail blocks), so each instance's arithmetic is
// exactly that of its own V-cycle and the results are bitwise those of the instance alone.

template <typename T> struct GDown {
  OpView<T> op;
  int nc0, nc1;
  const cx<T>* f;
  cx<T>* u_out;
  cx<T>* fc;
  T omega;
  const int* skip;
  int tiles_x;
};
template <typename T> struct GUp {
  OpView<T> op;
  int nc0, nc1;
  const cx<T>* u_in;
  const cx<T>* ec;
  const cx<T>* f;
  void* u_out;  // cx<T>, or complex128 on the finest level
  T omega;
  const int* skip;
  int tiles_x;
};
template <typename T> struct GCoarse {
  const cx<T>* ainv;
  int n;
  const cx<T>* f;
  cx<T>* z;
  const int* skip;
};
template <typename T> struct GTail {  // one virtual block per instance
  TailArgs<T> a;
  const cx<T>* f;
  void* out;
  const int* skip;
};

template <typename T, bool RBGS, int CX, int CY, int NT>
__global__ void __launch_bounds__(NT) kg_down2d(const GDown<T>* __restrict__ A, const GroupList* __restrict__ LT,
                                                int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GDown<T>& g = A[d];
    if (g.skip && *g.skip) return;
    down2d_body<T, RBGS, CX, CY, NT>(vb % g.tiles_x, vb / g.tiles_x, g.op, g.nc0, g.nc1, g.f, g.u_out, g.fc,
                                     g.omega);
  });
}

template <typename T, bool RBGS, typename TO, int FX, int FY, int NT>
__global__ void __launch_bounds__(NT) kg_up2d(const GUp<T>* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GUp<T>& g = A[d];
    if (g.skip && *g.skip) return;
    up2d_body<T, RBGS, TO, FX, FY, NT>(vb % g.tiles_x, vb / g.tiles_x, g.op, g.nc0, g.nc1, g.u_in, g.ec, g.f,
                                       (cx<TO>*)g.u_out, g.omega);
  });
}

// z = A^{-1} f with the dense coarsest inverse, one warp per row (as k_coarse, 256-thread blocks)
template <typename T>
__global__ void kg_coarse(const GCoarse<T>* __restrict__ A, const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int vb) {
    const GCoarse<T>& g = A[d];
    if (g.skip && *g.skip) return;
    const int warp = (vb * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.n) return;
    const cx<T>* row = g.ainv + (long)warp * g.n;
    cx<T> acc = mkc<T>(T(0), T(0));
    for (int c = lane; c < g.n; c += 32) acc = cfma<T>(row[c], g.f[c], acc);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) g.z[warp] = acc;
  });
}

template <typename T, typename TO>
__global__ void __launch_bounds__(TAIL_THREADS) kg_tail(const GTail<T>* __restrict__ A,
                                                        const GroupList* __restrict__ LT, int li) {
  pdl_entry();
  group_visit(LT[li], [&](int d, int) {
    const GTail<T>& g = A[d];
    if (g.skip && *g.skip) return;
    tail_body<T, 2, TO>(g.a, g.f, (cx<TO>*)g.out);
  });
}

struct GroupVcycle {
  bool rb = false;
  struct Launch {
    void* args = nullptr;  // device array of descriptors
    int li = -1;           // its work list
    int grid = 0;          // persistent blocks
    size_t smem = 0;
    int tile = 0;          // fused levels: the tile shape of every instance in this launch
  };
  // per level, one launch per tile shape in use there (each instance keeps the tile its own
  // V-cycle uses); up[0] writes the complex128 result
  std::vector<std::vector<Launch>> down, up;
  Launch tail0, tailk, coarse;  // tails from the finest level / from a coarser one; dense coarsest solves
  const GroupList* lists = nullptr;
  std::vector<DevBlock> mem;
};

template <typename D>
static helm_status group_upload(GroupVcycle* P, GroupLists* lists, const std::vector<D>& v,
                                const std::vector<int>& inst, const std::vector<int>& nb, GroupVcycle::Launch* L,
                                cudaStream_t st) {
  if (v.empty()) return HELM_OK;
  L->li = lists->add(inst, nb);
  DevBlock b;
  helm_status s = dev_alloc(&L->args, sizeof(D) * v.size(), st, &b);
  if (s != HELM_OK) return s;
  P->mem.push_back(b);
  HELM_CUDA(cudaMemcpyAsync(L->args, v.data(), sizeof(D) * v.size(), cudaMemcpyHostToDevice, st));
  return HELM_OK;
}

template <typename T>
helm_status group_vcycle_build(helm_ctx* const* cs, int ni, const void* const* in, double2* const* out,
                               const int* const* skip, GroupLists* lists, cudaStream_t st, GroupVcycle** plan) {
  *plan = nullptr;
  auto* P = new GroupVcycle();
  P->rb = cs[0]->pc.smoother == HELM_SM_RBGS;
  std::vector<int> tf(ni), stop(ni);
  int lmax = 0;
  for (int i = 0; i < ni; ++i) {
    const int nl = (int)cs[i]->lv.size();
    tf[i] = std::min(cs[i]->tail_first, nl);
    stop[i] = std::min(tf[i], nl - 1);  // fused levels above the tail or the coarsest
    lmax = std::max(lmax, stop[i]);
  }
  helm_status s = HELM_OK;
  P->down.resize(lmax);
  P->up.resize(lmax);
  for (int l = 0; l < lmax && s == HELM_OK; ++l) {
    for (int tile = 0; tile < NUM_TILES && s == HELM_OK; ++tile) {
      std::vector<GDown<T>> dv;
      std::vector<GUp<T>> uv;
      std::vector<int> di, dn, ui, un;
      for (int i = 0; i < ni; ++i) {
        if (l >= stop[i]) continue;
        const helm_ctx* c = cs[i];
        const LevelHost& F = c->lv[l];
        const LevelHost& C = c->lv[l + 1];
        const cx<T>* f = l == 0 ? (const cx<T>*)in[i] : (const cx<T>*)F.f;
        int tx, ty;
        if (down_tile_of(c, l, &tx, &ty) == tile) {
          GDown<T> d{F.view<T>(), C.n[0], C.n[1], f, (cx<T>*)F.w, (cx<T>*)C.f, (T)c->pc.omega, skip[i],
                     (C.n[0] + tx - 1) / tx};
          dv.push_back(d);
          di.push_back(i);
          dn.push_back(d.tiles_x * ((C.n[1] + ty - 1) / ty));
        }
        if (up_tile_of(c, l, &tx, &ty) == tile) {
          GUp<T> u{F.view<T>(), C.n[0], C.n[1], (const cx<T>*)F.w, (const cx<T>*)C.u, f,
                   l == 0 ? (void*)out[i] : F.u, (T)c->pc.omega, skip[i], (F.n[0] + tx - 1) / tx};
          uv.push_back(u);
          ui.push_back(i);
          un.push_back(u.tiles_x * ((F.n[1] + ty - 1) / ty));
        }
      }
      GroupVcycle::Launch ld, lu;
      ld.tile = lu.tile = tile;
      s = group_upload(P, lists, dv, di, dn, &ld, st);
      if (s == HELM_OK) s = group_upload(P, lists, uv, ui, un, &lu, st);
      if (ld.li >= 0) P->down[l].push_back(ld);
      if (lu.li >= 0) P->up[l].push_back(lu);
    }
  }
  std::vector<GTail<T>> t0, tk;
  std::vector<GCoarse<T>> co;
  std::vector<int> t0i, tki, coi, t0n, tkn, con;
  size_t smem0 = 0, smemk = 0;
  for (int i = 0; i < ni && s == HELM_OK; ++i) {
    helm_ctx* c = cs[i];
    const int nl = (int)c->lv.size();
    if (tf[i] < nl) {
      GTail<T> g;
      const size_t sm = tail_args<T>(c, tf[i], g.a);
      g.skip = skip[i];
      if (tf[i] == 0) {
        g.f = (const cx<T>*)in[i];
        g.out = out[i];
        t0.push_back(g);
        t0i.push_back(i);
        t0n.push_back(1);
        smem0 = std::max(smem0, sm);
      } else {
        g.f = (const cx<T>*)c->lv[tf[i]].f;
        g.out = c->lv[tf[i]].u;
        tk.push_back(g);
        tki.push_back(i);
        tkn.push_back(1);
        smemk = std::max(smemk, sm);
      }
    } else {
      const LevelHost& Lc = c->lv[nl - 1];
      co.push_back(GCoarse<T>{(const cx<T>*)c->coarse_inv, c->nco, (const cx<T>*)Lc.f, (cx<T>*)Lc.u, skip[i]});
      coi.push_back(i);
      con.push_back((c->nco * 32 + 255) / 256);
    }
  }
  if (s == HELM_OK) s = group_upload(P, lists, t0, t0i, t0n, &P->tail0, st);
  if (s == HELM_OK) s = group_upload(P, lists, tk, tki, tkn, &P->tailk, st);
  if (s == HELM_OK) s = group_upload(P, lists, co, coi, con, &P->coarse, st);
  P->tail0.smem = smem0;
  P->tailk.smem = smemk;
  if (s == HELM_OK && smem0)
    s = cuda_err(cudaFuncSetAttribute(kg_tail<T, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0));
  if (s == HELM_OK && smemk)
    s = cuda_err(cudaFuncSetAttribute(kg_tail<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemk));
  if (s != HELM_OK) {
    group_vcycle_free(P, st);
    return s;
  }
  *plan = P;
  return HELM_OK;
}

// Grid of a grouped launch: one block per virtual block of the full list.  The blocks past the
// running instances' total return after one load, and the hardware spreads the live ones over the
// SMs as they free up (a persistent grid with a fixed assignment was measured slower: the virtual
// blocks of a group differ too much in cost).
static int group_grid(int cap) { return std::max(cap, 1); }

template <typename T, bool RB>
static void group_grids_t(GroupVcycle* P, const GroupLists* lists) {
  for (auto& v : P->down)
    for (auto& L : v) L.grid = group_grid(lists->capacity(L.li));
  for (auto& v : P->up)
    for (auto& L : v) L.grid = group_grid(lists->capacity(L.li));
  for (GroupVcycle::Launch* L : {&P->tail0, &P->tailk, &P->coarse})
    if (L->li >= 0) L->grid = group_grid(lists->capacity(L->li));
}

template <typename T>
helm_status group_vcycle_finalize(GroupVcycle* P, const GroupLists* lists) {
  P->lists = lists->dev;
  if (P->rb) group_grids_t<T, true>(P, lists);
  else group_grids_t<T, false>(P, lists);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

template <typename T, bool RB>
static void group_down_launch(const GroupVcycle::Launch& L, const GroupList* LT, cudaStream_t st) {
  const GDown<T>* a = (const GDown<T>*)L.args;
  if (L.tile == TILE_BIG)
    launch_pdl(kg_down2d<T, RB, DN_CX, DN_CY, FUSED_THREADS>, dim3(L.grid), dim3(FUSED_THREADS), 0, st, a, LT, L.li);
  else if (L.tile == TILE_TINY)
    launch_pdl(kg_down2d<T, RB, DN_TCX, DN_TCY, FUSED_TINY_THREADS>, dim3(L.grid), dim3(FUSED_TINY_THREADS), 0, st, a,
               LT, L.li);
  else if (L.tile == TILE_SQUARE)
    launch_pdl(kg_down2d<T, RB, DN_QCX, DN_QCY, FUSED_SMALL_THREADS>, dim3(L.grid), dim3(FUSED_SMALL_THREADS), 0, st,
               a, LT, L.li);
  else if (L.tile == TILE_WIDE)
    launch_pdl(kg_down2d<T, RB, DN_WCX, DN_WCY, FUSED_THREADS>, dim3(L.grid), dim3(FUSED_THREADS), 0, st, a, LT, L.li);
  else
    launch_pdl(kg_down2d<T, RB, DN_SCX, DN_SCY, FUSED_SMALL_THREADS>, dim3(L.grid), dim3(FUSED_SMALL_THREADS), 0, st,
               a, LT, L.li);
}

template <typename T, bool RB, typename TO>
static void group_up_launch(const GroupVcycle::Launch& L, const GroupList* LT, cudaStream_t st) {
  const GUp<T>* a = (const GUp<T>*)L.args;
  if (L.tile == TILE_BIG)
    launch_pdl(kg_up2d<T, RB, TO, UP_FX, UP_FY, FUSED_THREADS>, dim3(L.grid), dim3(FUSED_THREADS), 0, st, a, LT, L.li);
  else if (L.tile == TILE_TINY)
    launch_pdl(kg_up2d<T, RB, TO, UP_TFX, UP_TFY, FUSED_TINY_THREADS>, dim3(L.grid), dim3(FUSED_TINY_THREADS), 0, st,
               a, LT, L.li);
  else if (L.tile == TILE_SQUARE)
    launch_pdl(kg_up2d<T, RB, TO, UP_QFX, UP_QFY, FUSED_SMALL_THREADS>, dim3(L.grid), dim3(FUSED_SMALL_THREADS), 0,
               st, a, LT, L.li);
  else if (L.tile == TILE_WIDE)
    launch_pdl(kg_up2d<T, RB, TO, UP_WFX, UP_WFY, FUSED_THREADS>, dim3(L.grid), dim3(FUSED_THREADS), 0, st, a, LT,
               L.li);
  else
    launch_pdl(kg_up2d<T, RB, TO, UP_SFX, UP_SFY, FUSED_SMALL_THREADS>, dim3(L.grid), dim3(FUSED_SMALL_THREADS), 0,
               st, a, LT, L.li);
}

template <typename T, bool RB>
static void group_vcycle_enqueue_t(const GroupVcycle* P, cudaStream_t st) {
  const GroupList* LT = P->lists;
  for (size_t l = 0; l < P->down.size(); ++l)
    for (const auto& L : P->down[l]) group_down_launch<T, RB>(L, LT, st);
  if (P->tail0.li >= 0)
    launch_pdl(kg_tail<T, double>, dim3(P->tail0.grid), dim3(TAIL_THREADS), P->tail0.smem, st,
               (const GTail<T>*)P->tail0.args, LT, P->tail0.li);
  if (P->tailk.li >= 0)
    launch_pdl(kg_tail<T, T>, dim3(P->tailk.grid), dim3(TAIL_THREADS), P->tailk.smem, st,
               (const GTail<T>*)P->tailk.args, LT, P->tailk.li);
  if (P->coarse.li >= 0)
    launch_pdl(kg_coarse<T>, dim3(P->coarse.grid), dim3(256), 0, st, (const GCoarse<T>*)P->coarse.args, LT,
               P->coarse.li);
  for (size_t l = P->up.size(); l-- > 0;)
    for (const auto& L : P->up[l]) {
      if (l == 0) group_up_launch<T, RB, double>(L, LT, st);
      else group_up_launch<T, RB, T>(L, LT, st);
    }
}

template <typename T>
void group_vcycle_enqueue(const GroupVcycle* P, cudaStream_t st) {
  if (P->rb) group_vcycle_enqueue_t<T, true>(P, st);
  else group_vcycle_enqueue_t<T, false>(P, st);
}

long group_vcycle_launches(const GroupVcycle* P) {
  long k = (P->tail0.li >= 0) + (P->tailk.li >= 0) + (P->coarse.li >= 0);
  for (const auto& v : P->down) k += (long)v.size();
  for (const auto& v : P->up) k += (long)v.size();
  return k;
}

void group_vcycle_free(GroupVcycle* P, cudaStream_t st) {
  if (!P) return;
  dev_free_all(P->mem, st);
  delete P;
}

template helm_status group_vcycle_build<float>(helm_ctx* const*, int, const void* const*, double2* const*,
                                               const int* const*, GroupLists*, cudaStream_t, GroupVcycle**);
template helm_status group_vcycle_build<double>(helm_ctx* const*, int, const void* const*, double2* const*,
                                                const int* const*, GroupLists*, cudaStream_t, GroupVcycle**);
template helm_status group_vcycle_finalize<float>(GroupVcycle*, const GroupLists*);
template helm_status group_vcycle_finalize<double>(GroupVcycle*, const GroupLists*);
template void group_vcycle_enqueue<float>(const GroupVcycle*, cudaStream_t);
template void group_vcycle_enqueue<double>(const GroupVcycle*, cudaStream_t);

// ---- autotuner ------------------------------------------------------------------------------
// On every fused 2D level the large, small, square, wide and one-warp tiles of k_down2d and k_up2d are timed
// with CUDA events (the fastest of three rounds of three launches, after one warm-up) on zeroed buffers of
// the level's shape,
// and the fastest is kept; then whole V-cycles are timed for every admissible depth of the
// one-block tail (from the deepest that fits its budgets to none) and the fastest depth is kept.
// Choices are cached for the process (tiles by precision, smoother and level shape; depth by
// precision, smoother and hierarchy), so contexts of shapes seen before skip the timing.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune;       // tiles per level shape
std::map<std::tuple<int, int, int, int, int, int, int>, int> g_depth;       // tail depth per hierarchy
}
// the tail depths the autotuner tries are bounded by this many points (and by shared memory)
constexpr long TAIL_TUNE_POINTS = 700;

// Decisions persist across processes when HELM_TUNE_CACHE names a file: it is read once (lines
// "tile <bytes> <rbgs> <n0> <n1> <down> <up>" and "depth <bytes> <rbgs> <dim> <n0> <n1> <n2> <levels>
// <first>") and every new decision is appended, so that a later process -- one under a profiler,
// whose serialised launches would distort the timings -- makes the same choices.
static const char* tune_cache_path() {
  const char* p = std::getenv("HELM_TUNE_CACHE");
  return p && *p ? p : nullptr;
}
static void tune_cache_load_locked() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return;
  char kind[16];
  while (std::fscanf(fp, "%15s", kind) == 1) {
    if (!std::strcmp(kind, "tile")) {
      int b, rb, n0, n1, d, u;
      if (std::fscanf(fp, "%d %d %d %d %d %d", &b, &rb, &n0, &n1, &d, &u) != 6) break;
      g_tune[std::make_tuple(b, rb, n0, n1)] = {d, u};
    } else if (!std::strcmp(kind, "depth")) {
      int b, rb, dim, n0, n1, n2, nl, first;
      if (std::fscanf(fp, "%d %d %d %d %d %d %d %d", &b, &rb, &dim, &n0, &n1, &n2, &nl, &first) != 8) break;
      g_depth[std::make_tuple(b, rb, dim, n0, n1, n2, nl)] = first;
    } else {
      break;
    }
  }
  std::fclose(fp);
}
static void tune_cache_append(const char* line) {
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* fp = std::fopen(path, "a");
  if (!fp) return;
  std::fputs(line, fp);
  std::fclose(fp);
}

template <typename F_>
static float time_variant(F_ launch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  launch();
  float best = 1e30f;
  for (int round = 0; round < 3; ++round) {  // the fastest of three rounds: tiles often differ by
    cudaEventRecord(e0, st);                 // less than one round's noise
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  return best;
}

template <typename T, bool RB>
static helm_status autotune_t(helm_ctx* c, cudaStream_t st) {
  int nl = (int)c->lv.size();
  if (nl < 2) return HELM_OK;
  // levels coarsened with offset 0 (a Sommerfeld low side) run the per-component kernels only
  const bool fused2d = c->lv[0].dim == 2 && c->pc.nu1 == 1 && c->pc.nu2 == 1 && !c->lv[0].any_offset0();
  // 1. tiles of every level that can run the fused 2D kernels
  std::vector<int> todo;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load_locked();
  }
  if (fused2d) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int l = 0; l < nl - 1; ++l) {
      if (c->lv[l].stg64) continue;  // Galerkin levels do not run the fused kernels
      auto it = g_tune.find(std::make_tuple((int)sizeof(T), (int)RB, c->lv[l].n[0], c->lv[l].n[1]));
      auto valid = [](int t) { return t >= 0 && t < NUM_TILES; };
      if (it != g_tune.end() && valid(it->second.first) && valid(it->second.second)) {
        c->lv[l].tile_down = it->second.first;
        c->lv[l].tile_up = it->second.second;
      } else {
        todo.push_back(l);
      }
    }
  }
  // 2. depth of the one-block tail: from the deepest the shared-memory and point budgets admit to none
  const int deepest = tail_first_level<T>(c, TAIL_TUNE_POINTS);
  auto dkey = std::make_tuple((int)sizeof(T), (int)RB, c->lv[0].dim, c->lv[0].n[0], c->lv[0].n[1], c->lv[0].n[2], nl);
  bool tune_depth = deepest < nl;
  if (tune_depth) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_depth.find(dkey);
    if (it != g_depth.end() && it->second >= deepest && it->second <= nl) {  // a cached depth must fit
      c->tail_first = it->second;
      tune_depth = false;
    }
  }
  if (todo.empty() && !tune_depth) return HELM_OK;
  size_t nf = (size_t)c->lv[0].ntot, ncs = (size_t)c->lv[1].ntot;
  void* buf = nullptr;
  size_t bytes = sizeof(cx<T>) * (4 * nf + ncs);
  DevBlock blk;
  helm_status as = dev_alloc(&buf, bytes, st, &blk);
  if (as != HELM_OK) return as;
  HELM_CUDA(cudaMemsetAsync(buf, 0, bytes, st));
  cx<T>* f = (cx<T>*)buf;
  cx<T>* u = f + nf;
  cx<T>* o = u + nf;
  cx<T>* w = o + nf;
  cx<T>* fc = w + nf;
  (void)w;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  T om = (T)c->pc.omega;
  for (int l : todo) {
    const LevelHost& F = c->lv[l];
    const LevelHost& C = c->lv[l + 1];
    int best_d = TILE_BIG, best_u = TILE_BIG;
    float td = 1e30f, tu = 1e30f;
    for (int tile : {TILE_BIG, TILE_SMALL, TILE_TINY, TILE_SQUARE, TILE_WIDE}) {
      float a = time_variant([&] { down_tile<T, RB>(tile, F, C, f, u, fc, om, nullptr, st); }, st, e0, e1);
      float b = time_variant([&] { up_tile<T, RB, T>(tile, F, C, u, fc, f, (T*)o, om, nullptr, st); }, st, e0, e1);
      if (a < td) { td = a; best_d = tile; }
      if (b < tu) { tu = b; best_u = tile; }
    }
    c->lv[l].tile_down = best_d;
    c->lv[l].tile_up = best_u;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple((int)sizeof(T), (int)RB, F.n[0], F.n[1])] = {c->lv[l].tile_down, c->lv[l].tile_up};
    char line[128];
    std::snprintf(line, sizeof line, "tile %d %d %d %d %d %d\n", (int)sizeof(T), (int)RB, F.n[0], F.n[1],
                  c->lv[l].tile_down, c->lv[l].tile_up);
    tune_cache_append(line);
  }
  if (tune_depth) {
    int best = c->tail_first;
    float tb = 1e30f;
    for (int first = deepest; first <= nl; ++first) {
      c->tail_first = first;
      float t = time_variant([&] { mg_vcycle<T>(c, f, (void*)u, false, nullptr, st); }, st, e0, e1);
      if (t < tb) { tb = t; best = first; }
    }
    c->tail_first = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_depth[dkey] = best;
    char line[160];
    std::snprintf(line, sizeof line, "depth %d %d %d %d %d %d %d %d\n", (int)sizeof(T), (int)RB, c->lv[0].dim,
                  c->lv[0].n[0], c->lv[0].n[1], c->lv[0].n[2], nl, best);
    tune_cache_append(line);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(blk, st);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

helm_status autotune_tiles(helm_ctx* c, cudaStream_t st) {
  if ((c->pc.flags & (HELM_PF_NO_AUTOTUNE | HELM_PF_UNFUSED)) || c->pc.kind == HELM_PC_NONE || c->lv.empty() ||
      c->pc.smoother == HELM_SM_ILU)  // ILU(0) hierarchies run no fused kernel
    return HELM_OK;
  bool f32 = c->pc.mg_dtype == HELM_C64, rb = c->pc.smoother == HELM_SM_RBGS;
  if (f32) return rb ? autotune_t<float, true>(c, st) : autotune_t<float, false>(c, st);
  return rb ? autotune_t<double, true>(c, st) : autotune_t<double, false>(c, st);
}

template <typename T> int tail_first_level(const helm_ctx* c) { return tail_first_level<T>(c, tail_point_budget<T>()); }
template int tail_first_level<float>(const helm_ctx*);
template int tail_first_level<double>(const helm_ctx*);
template helm_status tail_vcycle<float>(helm_ctx*, int, const float2*, void*, bool, const int*, cudaStream_t);
template helm_status tail_vcycle<double>(helm_ctx*, int, const double2*, void*, bool, const int*, cudaStream_t);
template void fused_down2d<float>(const helm_ctx*, int, const float2*, float2*, float2*, const int*, cudaStream_t);
template void fused_down2d<double>(const helm_ctx*, int, const double2*, double2*, double2*, const int*, cudaStream_t);
template void fused_up2d<float>(const helm_ctx*, int, const float2*, const float2*, const float2*, void*, bool, const int*, cudaStream_t);
template void fused_up2d<double>(const helm_ctx*, int, const double2*, const double2*, const double2*, void*, bool, const int*, cudaStream_t);

}  // namespace helm
