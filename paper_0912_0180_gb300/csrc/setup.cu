// setup.cu -- grid, coefficient and hierarchy setup kernels (run once per context).
//
// Grid: Section 3, eq. "ecsgrid" (vertex-centred, turning points are nodes) with the ECS
// layer width h e^{i theta_gamma} of Section 2; CSG scales widths by beta = e^{i theta_beta}
// (Section 5.3, eqs. "CSL-CSG", "lapctucsg").  Coefficients: Shortley-Weller, Section 3,
// eq. "shortwell".  Hierarchy: coarse unknown c <-> fine unknown 2c+1 (0-based), coarse widths
// are sums of fine widths, phi is injected; the coarsest operator is inverted densely in FP64
// (Gauss-Jordan with partial pivoting) and stored in the multigrid precision.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "helm_internal.cuh"

namespace helm {

// One thread per width: interior widths are h * scale_in; layer widths (the first nlo and the
// last ones) are h e^{i theta_gamma} * scale_ly, except, with a ramp of R > 1 widths, the m-th
// layer width from the turning point for m < R, which turns by only theta_gamma * m / R.
// somm: bit 0 a Sommerfeld high side, bit 1 a Sommerfeld low side (its ghost width is width 0).
__global__ void k_axis_gaps(double2* gap, int ngap, int nlo, int nin, double2 w_layer,
                            double2 w_int, int ramp, double h, double theta_g, double2 scale_ly,
                            int somm) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ngap) return;
  if ((j >= nlo && j < nlo + nin) || ((somm & 1) && j == ngap - 1) || ((somm & 2) && j == 0)) {
    // interior widths; a Sommerfeld ghost mirrors h
    gap[j] = w_int;
    return;
  }
  int m = j < nlo ? nlo - j : j - (nlo + nin) + 1;  // 1 = the width next to the turning point
  if (ramp > 1 && m < ramp) {
    double th = theta_g * m / ramp;
    gap[j] = cmul<double>(mkc<double>(h * cos(th), h * sin(th)), scale_ly);
  } else {
    gap[j] = w_layer;
  }
}

// Coarse unknown c is fine unknown 2c + o (o = 1; o = 0 on an axis with a Sommerfeld low side, so
// that its boundary node 0 stays a node).  Coarse width c (c >= 1, or c = 0 with o = 1) spans the
// fine widths 2c+o-1 and 2c+o; with o = 0 width 0 leads to the low ghost and mirrors width 1.  The
// last coarse width reaches the fine Dirichlet node and gathers the remaining fine widths, or, on
// a Sommerfeld high side (whose boundary node n-1 is then a coarse node), mirrors the last coarse
// width.  somm: bit 0 high side, bit 1 low side.  The hierarchy coarsens only axes of >= 3
// unknowns, so nc >= 2 when o = 0.
__global__ void k_axis_coarsen(const double2* __restrict__ gf, int nf, double2* __restrict__ gc,
                               int nc, int somm) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > nc) return;
  const int o = (somm & 2) ? 0 : 1;
  if (c < nc) {
    const int ci = (o == 0 && c == 0) ? 1 : c;
    gc[c] = cadd<double>(gf[2 * ci + o - 1], gf[2 * ci + o]);
  } else if (somm & 1) {
    gc[c] = cadd<double>(gf[2 * (nc - 1) + o - 1], gf[2 * (nc - 1) + o]);
  } else {
    double2 acc = mkc<double>(0.0, 0.0);
    for (int j = 2 * (nc - 1) + o + 1; j <= nf; ++j) acc = cadd<double>(acc, gf[j]);
    gc[c] = acc;
  }
}

// Shortley-Weller row of -d^2/dz^2 at unknown j with left width hl, right width hr:
//   am = -2 / (hl (hl + hr)),  a0 = 2 / (hl hr),  ap = -2 / (hr (hl + hr)).
// A Sommerfeld boundary node (somm, last row): the mirrored ghost u_g = u_{N-1} - 2 i k h_l u_N
// folds into the row, doubling the left weight and removing the right one (its diagonal part
// 2 i k / h_l is added where the diagonal is formed).
__global__ void k_axis_coeffs(const double2* __restrict__ gap, int n, double2* am, double2* a0,
                              double2* ap, float2* am32, float2* a032, float2* ap32, int somm) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double2 hl = gap[j], hr = gap[j + 1];
  double2 sum = cadd<double>(hl, hr);
  double2 two = mkc<double>(2.0, 0.0);
  double2 m = cdiv<double>(two, cmul<double>(hl, sum));
  double2 p = cdiv<double>(two, cmul<double>(hr, sum));
  double2 c = cdiv<double>(two, cmul<double>(hl, hr));
  am[j] = mkc<double>(-m.x, -m.y);
  a0[j] = c;
  ap[j] = mkc<double>(-p.x, -p.y);
  if ((somm & 1) && j == n - 1) {
    am[j] = mkc<double>(-2.0 * m.x, -2.0 * m.y);
    ap[j] = mkc<double>(0.0, 0.0);
  }
  if ((somm & 2) && j == 0) {  // low side: the ghost u_g = u_1 - 2 i k h_r u_0 mirrors the other way
    ap[j] = mkc<double>(-2.0 * p.x, -2.0 * p.y);
    am[j] = mkc<double>(0.0, 0.0);
  }
  if (am32) {
    am32[j] = cconv<float, double>(am[j]);
    a032[j] = cconv<float, double>(c);
    ap32[j] = cconv<float, double>(ap[j]);
  }
}

// phi on the coarse level: value of the fine node that coincides with the coarse node (fine
// index 2c + o per axis, o = offs bit clear ? 1 : 0 -- bit a set: offset 0 on axis a).
__global__ void k_phi_inject(const double* __restrict__ pf, int f0, int f1, int dim,
                             double* __restrict__ pc, float* __restrict__ pc32, int c0, int c1,
                             int c2, int offs) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long nc = (long)c0 * c1 * c2;
  if (p >= nc) return;
  int i = (int)(p % c0);
  long q = p / c0;
  int j = (int)(q % c1);
  int l = (int)(q / c1);
  const int o0 = (offs & 1) ? 0 : 1, o1 = (offs & 2) ? 0 : 1, o2 = (offs & 4) ? 0 : 1;
  int fi = 2 * i + o0, fj = dim > 1 ? 2 * j + o1 : 0, fl = dim > 2 ? 2 * l + o2 : 0;
  double v = pf[fi + (long)f0 * (fj + (long)f1 * fl)];
  pc[p] = v;
  if (pc32) pc32[p] = (float)v;
}

// omega_s / D at every point of a level (omega_s = omega for damped Jacobi, 1 for Gauss-Seidel),
// D = sum_axes a0 - s * phi, computed in FP64 and stored in the multigrid precision together with
// D itself (the smoothers multiply instead of dividing).
template <int DIM>
__global__ void k_dinv(OpView<double> op, double omega_s, double2* d64, float2* d32, double2* g64, float2* g32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y;
  int l = blockIdx.z;
  if (i >= op.n[0]) return;
  long p = i + (long)op.n[0] * (j + (long)op.n[1] * l);
  double2 d = op.a0[0][i];
  if (DIM > 1) d = cadd<double>(d, op.a0[1][j]);
  if (DIM > 2) d = cadd<double>(d, op.a0[2][l]);
  double ph = op.phi ? op.phi[p] : op.phi0;
  d = cadd<double>(d, somm_diag(op, i, j, l, ph));
  d = csub<double>(d, sigma64(op, p, ph));
  double2 r = cscale<double>(omega_s, crecip<double>(d));
  if (d64) d64[p] = r;
  if (g64) g64[p] = d;
  if (d32) d32[p] = cconv<float, double>(r);
  if (g32) g32[p] = cconv<float, double>(d);
}

// phi = k(x)^2 for the Gaussian bump k = k0 (1 + amp exp(-|x - c|^2 / width2)) (the variable wave
// number of Section 4, eq. "Helgen", in the form of the benchmark configurations), at the real node
// positions: along each axis x = (u - off) h, with off the index of the interior node at x = 0 (the
// ECS layers continue the real coordinate linearly, h per node).
struct BumpAxes {
  int n[3];
  int off[3];
  double h[3];
  double c[3];
};
__global__ void k_phi_bump(BumpAxes ax, int dim, double k0, double amp, double width2, double* __restrict__ phi) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long ntot = (long)ax.n[0] * ax.n[1] * ax.n[2];
  if (p >= ntot) return;
  long q = p;
  double r2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    const int u = (int)(q % ax.n[a]);
    q /= ax.n[a];
    const double d = (double)(u - ax.off[a]) * ax.h[a] - ax.c[a];
    r2 += d * d;
  }
  const double k = k0 * (1.0 + amp * exp(-r2 / width2));
  phi[p] = k * k;
}

// phi = k^2 from a caller's device field of k values; *bad is set when an entry is not finite.
__global__ void k_phi_field(const double* __restrict__ kf, double* __restrict__ phi, long n, int* bad) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double k = kf[p];
  if (!isfinite(k)) *bad = 1;
  phi[p] = k * k;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, long n) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p < n) b[p] = (float)a[p];
}

__global__ void k_c128_to_c64(const double2* __restrict__ a, float2* __restrict__ b, long n) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p < n) b[p] = cconv<float, double>(a[p]);
}

// Dense matrix of the coarsest operator (row-major, FP64), one thread per row.
__global__ void k_dense_assemble(OpView<double> op, int dim, double2* A, int n) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i = p % op.n[0];
  int j = (p / op.n[0]) % op.n[1];
  int l = p / (op.n[0] * op.n[1]);
  double2* row = A + (long)p * n;
  for (int c = 0; c < n; ++c) row[c] = mkc<double>(0.0, 0.0);
  double ph = op.phi ? op.phi[p] : op.phi0;
  double2 d = op.a0[0][i];
  if (dim > 1) d = cadd<double>(d, op.a0[1][j]);
  if (dim > 2) d = cadd<double>(d, op.a0[2][l]);
  d = cadd<double>(d, somm_diag(op, i, j, l, ph));
  d = csub<double>(d, sigma64(op, p, ph));
  row[p] = d;
  if (i > 0) row[p - 1] = op.am[0][i];
  if (i < op.n[0] - 1) row[p + 1] = op.ap[0][i];
  if (dim > 1) {
    if (j > 0) row[p - op.n[0]] = op.am[1][j];
    if (j < op.n[1] - 1) row[p + op.n[0]] = op.ap[1][j];
  }
  if (dim > 2) {
    int st = op.n[0] * op.n[1];
    if (l > 0) row[p - st] = op.am[2][l];
    if (l < op.n[2] - 1) row[p + st] = op.ap[2][l];
  }
}

// Gauss-Jordan inversion with partial pivoting, one block.  A (n x n) is destroyed; X = A^{-1}.
// status[0] = 1 if a pivot is exactly zero.
__global__ void k_gauss_jordan(double2* A, double2* X, int n, int* status) {
  extern __shared__ unsigned char smem_raw[];
  double* best = reinterpret_cast<double*>(smem_raw);
  int* bidx = reinterpret_cast<int*>(best + blockDim.x);
  __shared__ int piv;
  __shared__ double2 inv_p;
  int tid = threadIdx.x, nt = blockDim.x;
  for (long e = tid; e < (long)n * n; e += nt) X[e] = mkc<double>((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double b = -1.0;
    int bi = k;
    for (int r = k + tid; r < n; r += nt) {
      double v = cabs2<double>(A[(long)r * n + k]);
      if (v > b) { b = v; bi = r; }
    }
    best[tid] = b;
    bidx[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        if (best[tid + s] > best[tid] || (best[tid + s] == best[tid] && bidx[tid + s] < bidx[tid])) {
          best[tid] = best[tid + s];
          bidx[tid] = bidx[tid + s];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      piv = bidx[0];
      if (best[0] <= 0.0) status[0] = 1;
    }
    __syncthreads();
    int p = piv;
    if (p != k) {
      for (int c = tid; c < n; c += nt) {
        double2 t = A[(long)k * n + c]; A[(long)k * n + c] = A[(long)p * n + c]; A[(long)p * n + c] = t;
        t = X[(long)k * n + c]; X[(long)k * n + c] = X[(long)p * n + c]; X[(long)p * n + c] = t;
      }
    }
    __syncthreads();
    if (tid == 0) inv_p = crecip<double>(A[(long)k * n + k]);
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
      A[(long)k * n + c] = cmul<double>(A[(long)k * n + c], inv_p);
      X[(long)k * n + c] = cmul<double>(X[(long)k * n + c], inv_p);
    }
    __syncthreads();
    for (long e = tid; e < (long)n * n; e += nt) {
      int r = (int)(e / n), c = (int)(e % n);
      if (r == k) continue;
      double2 f = A[(long)r * n + k];
      if (c != k) A[e] = csub<double>(A[e], cmul<double>(f, A[(long)k * n + c]));
      X[e] = csub<double>(X[e], cmul<double>(f, X[(long)k * n + c]));
    }
    __syncthreads();
    for (int r = tid; r < n; r += nt)
      if (r != k) A[(long)r * n + k] = mkc<double>(0.0, 0.0);
    __syncthreads();
  }
}

static int ceil_div(long a, int b) { return (int)((a + b - 1) / b); }

// ---- Galerkin coarse operators (2D) ---------------------------------------------------------
// Entry of the finer operator between fine unknowns (i, j) and (ii, jj): its 9-point stencil when
// it is a Galerkin level, else its Shortley-Weller row (centre: axis centre weights - s phi).
__device__ double2 fine_entry(const OpView<double>& F, int i, int j, int ii, int jj) {
  if (ii < 0 || ii >= F.n[0] || jj < 0 || jj >= F.n[1]) return mkc<double>(0.0, 0.0);
  const int di = ii - i, dj = jj - j;
  const long p = i + (long)F.n[0] * j;
  if (F.stg) return F.stg[(long)(3 * (dj + 1) + (di + 1)) * F.ntot + p];
  if (di == 0 && dj == 0) {
    double ph = F.phi ? F.phi[p] : F.phi0;
    double2 d = cadd<double>(cadd<double>(F.a0[0][i], F.a0[1][j]), somm_diag(F, i, j, 0, ph));
    return csub<double>(d, sigma64(F, p, ph));
  }
  if (di != 0 && dj != 0) return mkc<double>(0.0, 0.0);  // a 5-point row has no corner weights
  if (dj == 0) return di < 0 ? F.am[0][i] : F.ap[0][i];
  return dj < 0 ? F.am[1][j] : F.ap[1][j];
}

// C = R F P for one coarse unknown per thread: R gathers fine 2I+{0,1,2} x 2J+{0,1,2} with the
// full-weighting weights, P spreads coarse (K, M) over fine 2K+{0,1,2} x 2M+{0,1,2} with the
// linear-interpolation weights; only |K - I|, |M - J| <= 1 survive.
__global__ void k_galerkin2d(OpView<double> F, int nc0, int nc1, double2* __restrict__ c64, float2* __restrict__ c32) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  if (I >= nc0) return;
  const long ncs = (long)nc0 * nc1;
  const long q = I + (long)nc0 * J;
  const double wr[3] = {0.25, 0.5, 0.25};
  double2 acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = mkc<double>(0.0, 0.0);
  for (int b = 0; b < 3; ++b) {
    const int fj = 2 * J + b;
    if (fj >= F.n[1]) continue;
    for (int a = 0; a < 3; ++a) {
      const int fi = 2 * I + a;
      if (fi >= F.n[0]) continue;
      const double r = wr[a] * wr[b];
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const double2 e = fine_entry(F, fi, fj, fi + di, fj + dj);
          if (e.x == 0.0 && e.y == 0.0) continue;
          const int gi = fi + di, gj = fj + dj;  // the fine unknown the entry reaches
          // coarse (K, M) with |gi - (2K+1)| <= 1 and |gj - (2M+1)| <= 1
          for (int dM = -1; dM <= 1; ++dM) {
            const int M = J + dM;
            const int ty = gj - (2 * M + 1);
            if (M < 0 || M >= nc1 || ty < -1 || ty > 1) continue;
            const double py = ty == 0 ? 1.0 : 0.5;
            for (int dK = -1; dK <= 1; ++dK) {
              const int K = I + dK;
              const int tx = gi - (2 * K + 1);
              if (K < 0 || K >= nc0 || tx < -1 || tx > 1) continue;
              const double w = r * py * (tx == 0 ? 1.0 : 0.5);
              double2& o = acc[3 * (dM + 1) + (dK + 1)];
              o = mkc<double>(fma(w, e.x, o.x), fma(w, e.y, o.y));
            }
          }
        }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    c64[k * ncs + q] = acc[k];
    if (c32) c32[k * ncs + q] = cconv<float, double>(acc[k]);
  }
}

// ---- Galerkin coarse operators (3D) ---------------------------------------------------------
// Entry of a finer 3D operator between fine unknowns (i, j, l) and (ii, jj, ll): its 27-point
// stencil when it is a Galerkin level, else its Shortley-Weller row.
__device__ double2 fine_entry3(const OpView<double>& F, int i, int j, int l, int ii, int jj, int ll) {
  if (ii < 0 || ii >= F.n[0] || jj < 0 || jj >= F.n[1] || ll < 0 || ll >= F.n[2]) return mkc<double>(0.0, 0.0);
  const int di = ii - i, dj = jj - j, dl = ll - l;
  const long p = i + (long)F.n[0] * (j + (long)F.n[1] * l);
  if (F.stg) return F.stg[(long)(9 * (dl + 1) + 3 * (dj + 1) + (di + 1)) * F.ntot + p];
  const int nz = (di != 0) + (dj != 0) + (dl != 0);
  if (nz == 0) {
    double ph = F.phi ? F.phi[p] : F.phi0;
    double2 d = cadd<double>(cadd<double>(F.a0[0][i], F.a0[1][j]), F.a0[2][l]);
    d = cadd<double>(d, somm_diag(F, i, j, l, ph));
    return csub<double>(d, sigma64(F, p, ph));
  }
  if (nz > 1) return mkc<double>(0.0, 0.0);  // a 7-point row has only axis neighbours
  if (di) return di < 0 ? F.am[0][i] : F.ap[0][i];
  if (dj) return dj < 0 ? F.am[1][j] : F.ap[1][j];
  return dl < 0 ? F.am[2][l] : F.ap[2][l];
}

// C = R F P in 3D for one coarse unknown (I, J, L) per thread: R gathers the 27 fine unknowns
// 2I+{0,1,2} x 2J+{0,1,2} x 2L+{0,1,2} with the full-weighting weights; each entry of F reaches a
// fine unknown g, which the trilinear interpolation takes from the coarse unknowns K with
// |g - (2K+1)| <= 1 on every axis (weight 1 or 1/2 per axis); only |K - I| <= 1 per axis survive.
__global__ void k_galerkin3d(OpView<double> F, int nc0, int nc1, int nc2, double2* __restrict__ c64,
                             float2* __restrict__ c32) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y, L = blockIdx.z;
  if (I >= nc0) return;
  const long ncs = (long)nc0 * nc1 * nc2;
  const long q = I + (long)nc0 * (J + (long)nc1 * L);
  const double wr[3] = {0.25, 0.5, 0.25};
  double2 acc[27];
  for (int k = 0; k < 27; ++k) acc[k] = mkc<double>(0.0, 0.0);
  for (int c = 0; c < 3; ++c) {
    const int fl = 2 * L + c;
    if (fl >= F.n[2]) continue;
    for (int b = 0; b < 3; ++b) {
      const int fj = 2 * J + b;
      if (fj >= F.n[1]) continue;
      for (int a = 0; a < 3; ++a) {
        const int fi = 2 * I + a;
        if (fi >= F.n[0]) continue;
        const double r = wr[a] * wr[b] * wr[c];
        for (int dl = -1; dl <= 1; ++dl)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              const double2 e = fine_entry3(F, fi, fj, fl, fi + di, fj + dj, fl + dl);
              if (e.x == 0.0 && e.y == 0.0) continue;
              const int gi = fi + di, gj = fj + dj, gl = fl + dl;
              for (int dN = -1; dN <= 1; ++dN) {
                const int N = L + dN, tz = gl - (2 * N + 1);
                if (N < 0 || N >= nc2 || tz < -1 || tz > 1) continue;
                const double pz = tz == 0 ? 1.0 : 0.5;
                for (int dM = -1; dM <= 1; ++dM) {
                  const int M = J + dM, ty = gj - (2 * M + 1);
                  if (M < 0 || M >= nc1 || ty < -1 || ty > 1) continue;
                  const double py = ty == 0 ? 1.0 : 0.5;
                  for (int dK = -1; dK <= 1; ++dK) {
                    const int K = I + dK, tx = gi - (2 * K + 1);
                    if (K < 0 || K >= nc0 || tx < -1 || tx > 1) continue;
                    const double w = r * pz * py * (tx == 0 ? 1.0 : 0.5);
                    double2& o = acc[9 * (dN + 1) + 3 * (dM + 1) + (dK + 1)];
                    o = mkc<double>(fma(w, e.x, o.x), fma(w, e.y, o.y));
                  }
                }
              }
            }
      }
    }
  }
  for (int k = 0; k < 27; ++k) {
    c64[k * ncs + q] = acc[k];
    if (c32) c32[k * ncs + q] = cconv<float, double>(acc[k]);
  }
}

// omega / D and D of a Galerkin level (D = the stencil's centre weight, index `centre`).
__global__ void k_dinvg(const double2* __restrict__ stg, long n, int centre, double omega_s, double2* d64,
                        float2* d32, double2* g64, float2* g32) {
  long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  double2 d = stg[(long)centre * n + p];
  double2 r = cscale<double>(omega_s, crecip<double>(d));
  if (d64) d64[p] = r;
  if (g64) g64[p] = d;
  if (d32) d32[p] = cconv<float, double>(r);
  if (g32) g32[p] = cconv<float, double>(d);
}

// Dense matrix of a Galerkin coarsest level (row-major, FP64), one thread per row; n2 = 1 in 2D
// (9 weights), > 1 in 3D (27 weights).
__global__ void k_dense_assembleg(const double2* __restrict__ stg, int n0, int n1, int n2, int dim, double2* A,
                                  int n) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int i = p % n0, j = (p / n0) % n1, l = p / (n0 * n1);
  double2* row = A + (long)p * n;
  for (int c = 0; c < n; ++c) row[c] = mkc<double>(0.0, 0.0);
  const int lr = dim == 3 ? 1 : 0;
  for (int dl = -lr; dl <= lr; ++dl)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        int ii = i + di, jj = j + dj, ll = l + dl;
        if (ii < 0 || ii >= n0 || jj < 0 || jj >= n1 || ll < 0 || ll >= n2) continue;
        const int k = dim == 3 ? 9 * (dl + 1) + 3 * (dj + 1) + (di + 1) : 3 * (dj + 1) + (di + 1);
        row[ii + n0 * (jj + n1 * ll)] = stg[(long)k * n + p];
      }
}


// In-place Gauss-Jordan with partial pivoting over the whole GPU, for coarsest levels too
// large for one block: A (n x n, row-major) is overwritten with A^{-1}.  Step k: one block picks
// the pivot row p >= k of column k; rows k and p are exchanged while the pivot row is scaled
// into `prow` (prow[k] = 1 / a_pk) and column k is saved into `fcol`; every other row r then
// becomes A[r, :] - fcol[r] prow, column k being replaced by -fcol[r] / a_pk.  The row exchanges
// are undone on the columns at the end, last step first.
constexpr int GJ_ONE_BLOCK_MAX = 512;
// coarsest levels above this size with a constant phi use the separable solve of coarse_fdm.cu
constexpr long FDM_MIN_UNKNOWNS = 512;

struct GjPivot {
  double2 apk, akk;
  int p;
};

__global__ void k_gj_pivot(const double2* __restrict__ A, int n, int k, GjPivot* pv, int* perm, int* status) {
  __shared__ double best[1024];
  __shared__ int bidx[1024];
  int tid = threadIdx.x, nt = blockDim.x;
  double b = -1.0;
  int bi = k;
  for (int r = k + tid; r < n; r += nt) {
    double v = cabs2<double>(A[(long)r * n + k]);
    if (v > b) { b = v; bi = r; }
  }
  best[tid] = b;
  bidx[tid] = bi;
  __syncthreads();
  for (int s = nt / 2; s > 0; s >>= 1) {
    if (tid < s && (best[tid + s] > best[tid] || (best[tid + s] == best[tid] && bidx[tid + s] < bidx[tid]))) {
      best[tid] = best[tid + s];
      bidx[tid] = bidx[tid + s];
    }
    __syncthreads();
  }
  if (tid == 0) {
    int p = bidx[0];
    if (best[0] <= 0.0) status[0] = 1;
    pv->p = p;
    pv->apk = A[(long)p * n + k];
    pv->akk = A[(long)k * n + k];
    perm[k] = p;
  }
}

// thread t owns column t of rows k and p, and row t of column k
__global__ void k_gj_swap(double2* __restrict__ A, int n, int k, const GjPivot* pv, double2* __restrict__ prow,
                          double2* __restrict__ fcol) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int p = pv->p;
  double2 ip = crecip<double>(pv->apk);
  double2 ak = A[(long)k * n + t], ap = A[(long)p * n + t];
  double2 pr = t == k ? ip : cmul<double>(ap, ip);
  prow[t] = pr;
  A[(long)k * n + t] = pr;
  if (p != k) A[(long)p * n + t] = ak;
  fcol[t] = t == k ? mkc<double>(0.0, 0.0) : (t == p ? pv->akk : A[(long)t * n + k]);
}

__global__ void k_gj_update(double2* __restrict__ A, int n, int k, const double2* __restrict__ prow,
                            const double2* __restrict__ fcol) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (c >= n || r == k) return;
  double2 f = fcol[r];
  if (f.x == 0.0 && f.y == 0.0) return;  // the row does not change
  long e = (long)r * n + c;
  double2 a = c == k ? mkc<double>(0.0, 0.0) : A[e];
  A[e] = csub<double>(a, cmul<double>(f, prow[c]));
}

__global__ void k_gj_unpermute(double2* __restrict__ A, int n, const int* __restrict__ perm) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double2* row = A + (long)r * n;
  for (int k = n - 1; k >= 0; --k) {
    int p = perm[k];
    if (p != k) {
      double2 t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
}


static helm_status build_axes(helm_ctx* c, LevelHost& L, double2 scale_in, double2 scale_ly,
                              bool want32, cudaStream_t st) {
  const helm_grid& g = c->grid;
  L.dim = g.dim;
  L.ntot = 1;
  for (int a = 0; a < 3; ++a) L.n[a] = 1;
  for (int a = 0; a < g.dim; ++a) {
    int lo = g.n_layer[a][0], hi = g.n_layer[a][1];
    // Sommerfeld sides (bit 0 high, bit 1 low): one mirrored width each, to the ghost node
    const int somm = (hi < 0 ? 1 : 0) | (lo < 0 ? 2 : 0);
    int nlo = lo > 0 ? lo + 1 : (lo < 0 ? 1 : 0), nhi = hi > 0 ? hi + 1 : (hi < 0 ? 1 : 0);
    int nin = g.n_int[a] - 1;
    int ngap = nlo + nin + nhi;
    int n = ngap - 1;
    double h = g.extent[a] / (g.n_int[a] - 1);
    double2 hg = mkc<double>(h * cos(g.theta_gamma), h * sin(g.theta_gamma));
    double2 wl = cmul<double>(hg, scale_ly);
    double2 wi = cscale<double>(h, scale_in);
    helm_status s;
    if ((s = ctx_alloc(c, (void**)&L.gap[a], sizeof(double2) * ngap)) != HELM_OK) return s;
    for (int k = 0; k < 3; ++k) {
      if ((s = ctx_alloc(c, (void**)&L.coef64[a][k], sizeof(double2) * n)) != HELM_OK) return s;
      if (want32 && (s = ctx_alloc(c, (void**)&L.coef32[a][k], sizeof(float2) * n)) != HELM_OK) return s;
    }
    k_axis_gaps<<<ceil_div(ngap, 256), 256, 0, st>>>(L.gap[a], ngap, nlo, nin, wl, wi, g.ecs_ramp, h,
                                                     g.theta_gamma, scale_ly, somm);
    k_axis_coeffs<<<ceil_div(n, 256), 256, 0, st>>>(L.gap[a], n, L.coef64[a][0], L.coef64[a][1],
                                                    L.coef64[a][2], L.coef32[a][0], L.coef32[a][1],
                                                    L.coef32[a][2], somm);
    if (somm & 1) {  // boundary weight 2i / h_l, h_l = the last (interior) width
      L.somm |= 1 << a;
      L.bt[a] = cdiv<double>(mkc<double>(0.0, 2.0), wi);
    }
    if (somm & 2) {  // boundary weight 2i / h_r, h_r = the first (interior) width
      L.somm |= 8 << a;
      L.btl[a] = cdiv<double>(mkc<double>(0.0, 2.0), wi);
    }
    HELM_CUDA(cudaGetLastError());
    L.n[a] = n;
    L.ntot *= n;
  }
  return HELM_OK;
}

// Finds, per axis, the longest run of unknowns around the middle whose Shortley-Weller rows are
// bitwise identical with am == ap (the uniform interior); rows are copied from the device once.
static helm_status find_uniform(LevelHost& L, cudaStream_t st) {
  L.ud = mkc<double>(0.0, 0.0);
  for (int a = 0; a < 3; ++a) { L.ulo[a] = 1; L.uhi[a] = 0; L.ua[a] = mkc<double>(0.0, 0.0); }
  bool all = true;
  double2 ud = mkc<double>(0.0, 0.0);
  for (int a = 0; a < L.dim; ++a) {
    int n = L.n[a];
    std::vector<double2> am(n), a0(n), ap(n);
    HELM_CUDA(cudaMemcpyAsync(am.data(), L.coef64[a][0], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaMemcpyAsync(a0.data(), L.coef64[a][1], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaMemcpyAsync(ap.data(), L.coef64[a][2], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaStreamSynchronize(st));
    auto same = [&](int j, int m) {
      return std::memcmp(&am[j], &am[m], sizeof(double2)) == 0 && std::memcmp(&a0[j], &a0[m], sizeof(double2)) == 0 &&
             std::memcmp(&ap[j], &ap[m], sizeof(double2)) == 0 && std::memcmp(&am[j], &ap[j], sizeof(double2)) == 0;
    };
    int mid = n / 2;
    if (n < 3 || !same(mid, mid)) { all = false; break; }
    int lo = mid, hi = mid;
    while (lo - 1 >= 0 && same(lo - 1, mid)) --lo;
    while (hi + 1 < n && same(hi + 1, mid)) ++hi;
    // the row must also read both neighbours inside the grid to use the uniform formula
    if (lo < 1) lo = 1;
    if (hi > n - 2) hi = n - 2;
    if (hi < lo) { all = false; break; }
    L.ulo[a] = lo;
    L.uhi[a] = hi;
    L.ua[a] = am[mid];
    ud = cadd<double>(ud, a0[mid]);
  }
  if (!all)
    for (int a = 0; a < 3; ++a) { L.ulo[a] = 1; L.uhi[a] = 0; }
  L.ud = ud;
  return HELM_OK;
}

// The uniform-interior rows take a real phi (the diagonal ud - s phi without an imaginary part).
// With a complex phi -- k read at complex node positions, which are real in the interior -- the
// shortcut stays only if the imaginary part vanishes on the whole uniform box; else it is dropped
// for this level and every row reads its stored diagonal.
static helm_status uniform_needs_real_phi(LevelHost& L, cudaStream_t st) {
  if (!L.phim64 || L.uhi[0] < L.ulo[0]) return HELM_OK;
  std::vector<double> im(L.ntot);
  HELM_CUDA(cudaMemcpyAsync(im.data(), L.phim64, sizeof(double) * L.ntot, cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaStreamSynchronize(st));
  const int lo1 = L.dim > 1 ? L.ulo[1] : 0, hi1 = L.dim > 1 ? L.uhi[1] : 0;
  const int lo2 = L.dim > 2 ? L.ulo[2] : 0, hi2 = L.dim > 2 ? L.uhi[2] : 0;
  for (int l = lo2; l <= hi2; ++l)
    for (int j = lo1; j <= hi1; ++j)
      for (int i = L.ulo[0]; i <= L.uhi[0]; ++i)
        if (im[i + (long)L.n[0] * (j + (long)L.n[1] * l)] != 0.0) {
          for (int a = 0; a < 3; ++a) { L.ulo[a] = 1; L.uhi[a] = 0; }
          return HELM_OK;
        }
  return HELM_OK;
}

template <typename T> OpView<T> LevelHost::view() const {
  OpView<T> v{};
  for (int a = 0; a < 3; ++a) {
    v.n[a] = n[a];
    for (int k = 0; k < 3; ++k) {
      const void* src = nullptr;
      if (a < dim) src = std::is_same<T, double>::value ? (const void*)coef64[a][k] : (const void*)coef32[a][k];
      const cx<T>* p = reinterpret_cast<const cx<T>*>(src);
      if (k == 0) v.am[a] = p;
      if (k == 1) v.a0[a] = p;
      if (k == 2) v.ap[a] = p;
    }
  }
  v.phi = std::is_same<T, double>::value ? (const T*)(const void*)phi64 : (const T*)(const void*)phi32;
  v.phi0 = (T)phi0;
  v.s = mkc<T>((T)s.x, (T)s.y);
  bool real = s.y == 0.0;
  for (int a = 0; a < 3; ++a) {
    v.ulo[a] = a < dim ? ulo[a] : 0;
    v.uhi[a] = a < dim ? uhi[a] : 0;
    v.ua[a] = mkc<T>((T)ua[a].x, (T)ua[a].y);
    if (a < dim && ua[a].y != 0.0) real = false;
  }
  v.ud = mkc<T>((T)ud.x, (T)ud.y);
  if (ud.y != 0.0) real = false;
  v.uniform_real = real ? 1 : 0;
  bool iso = dim > 1;
  for (int a = 1; a < dim; ++a)
    if (std::memcmp(&ua[a], &ua[0], sizeof(double2)) != 0) iso = false;
  v.uniform_iso = iso ? 1 : 0;
  v.dinv = std::is_same<T, double>::value ? (const cx<T>*)(const void*)dinv64 : (const cx<T>*)(const void*)dinv32;
  v.dg = std::is_same<T, double>::value ? (const cx<T>*)(const void*)dg64 : (const cx<T>*)(const void*)dg32;
  v.stg = std::is_same<T, double>::value ? (const cx<T>*)(const void*)stg64 : (const cx<T>*)(const void*)stg32;
  v.ntot = ntot;
  v.somm = somm;
  for (int a = 0; a < 3; ++a) {
    v.bt[a] = bt[a];
    v.btl[a] = btl[a];
  }
  v.phim = phim64;
  return v;
}
template OpView<double> LevelHost::view<double>() const;
template OpView<float> LevelHost::view<float>() const;

helm_status build_operator(helm_ctx* c, const helm_kspec* k, cudaStream_t st) {
  LevelHost& H = c->H;
  helm_status s = build_axes(c, H, mkc<double>(1, 0), mkc<double>(1, 0), false, st);
  if (s != HELM_OK) return s;
  if ((s = find_uniform(H, st)) != HELM_OK) return s;
  c->n = H.ntot;
  H.s = mkc<double>(1.0, 0.0);
  H.phi0 = k->k0 * k->k0;
  if (k->phi) {
    if ((s = ctx_alloc(c, (void**)&H.phi64, sizeof(double) * H.ntot)) != HELM_OK) return s;
    HELM_CUDA(cudaMemcpyAsync(H.phi64, k->phi, sizeof(double) * H.ntot, cudaMemcpyHostToDevice, st));
  } else if (k->kind == HELM_K_GAUSS_BUMP) {
    if ((s = ctx_alloc(c, (void**)&H.phi64, sizeof(double) * H.ntot)) != HELM_OK) return s;
    BumpAxes ax{};
    for (int a = 0; a < 3; ++a) {
      ax.n[a] = H.n[a];
      const int lo = c->grid.n_layer[a][0];
      ax.off[a] = lo > 0 ? lo : (lo < 0 ? 0 : -1);  // index of the unknown at x = 0
      ax.h[a] = c->grid.extent[a] / (c->grid.n_int[a] - 1);
      ax.c[a] = k->centre[a];
    }
    k_phi_bump<<<ceil_div(H.ntot, 256), 256, 0, st>>>(ax, H.dim, k->k0, k->amp, k->width2, H.phi64);
    HELM_CUDA(cudaGetLastError());
  } else if (k->kind == HELM_K_FIELD) {
    if ((s = ctx_alloc(c, (void**)&H.phi64, sizeof(double) * H.ntot)) != HELM_OK) return s;
    if ((s = ctx_alloc(c, (void**)&c->field_bad, sizeof(int))) != HELM_OK) return s;
    HELM_CUDA(cudaMemsetAsync(c->field_bad, 0, sizeof(int), st));
    k_phi_field<<<ceil_div(H.ntot, 256), 256, 0, st>>>(k->field, H.phi64, H.ntot, c->field_bad);
    HELM_CUDA(cudaGetLastError());
  }
  if (k->phi_im) {
    if ((s = ctx_alloc(c, (void**)&H.phim64, sizeof(double) * H.ntot)) != HELM_OK) return s;
    HELM_CUDA(cudaMemcpyAsync(H.phim64, k->phi_im, sizeof(double) * H.ntot, cudaMemcpyHostToDevice, st));
    if ((s = uniform_needs_real_phi(H, st)) != HELM_OK) return s;
  }
  // the diagonal of H at every point: outside the uniform interior the stencil kernels read it
  // instead of summing the axes' centre coefficients and subtracting phi (FP64 operations are
  // what bound them; the 16 B per point are cheap)
  if ((s = ctx_alloc(c, (void**)&H.dg64, sizeof(double2) * H.ntot)) != HELM_OK) return s;
  {
    OpView<double> v = H.view<double>();
    dim3 g((H.n[0] + 127) / 128, H.n[1], H.n[2]);
    if (H.dim == 1) k_dinv<1><<<g, 128, 0, st>>>(v, 1.0, nullptr, nullptr, H.dg64, nullptr);
    else if (H.dim == 2) k_dinv<2><<<g, 128, 0, st>>>(v, 1.0, nullptr, nullptr, H.dg64, nullptr);
    else k_dinv<3><<<g, 128, 0, st>>>(v, 1.0, nullptr, nullptr, H.dg64, nullptr);
    HELM_CUDA(cudaGetLastError());
  }
  return HELM_OK;
}

static helm_status tune_and_lay_out(helm_ctx* c, cudaStream_t st);

helm_status build_hierarchy(helm_ctx* c, cudaStream_t st) {
  const helm_precond& pc = c->pc;
  if (pc.kind == HELM_PC_NONE) return HELM_OK;
  bool f32 = pc.mg_dtype == HELM_C64;
  size_t esz = f32 ? sizeof(float2) : sizeof(double2);
  double2 beta = mkc<double>(cos(pc.theta_beta), sin(pc.theta_beta));
  double2 one = mkc<double>(1.0, 0.0);
  double2 sc_in = one, sc_ly = one, s = one;
  if (pc.kind == HELM_PC_CSL) s = mkc<double>(pc.shift_re, pc.shift_im);
  if (pc.kind == HELM_PC_CSG_UNIFORM) { sc_in = beta; sc_ly = beta; }
  if (pc.kind == HELM_PC_CSG_INTERIOR) sc_in = beta;
  helm_status rc;
  c->lv.clear();
  c->lv.reserve(pc.max_levels);
  const bool galerkin = (pc.flags & HELM_PF_GALERKIN) != 0;
  c->lv.emplace_back();
  {
    LevelHost& L0 = c->lv[0];
    if ((rc = build_axes(c, L0, sc_in, sc_ly, f32, st)) != HELM_OK) return rc;
    if ((rc = find_uniform(L0, st)) != HELM_OK) return rc;
    L0.s = s;
    L0.phi0 = c->H.phi0;
    L0.phi64 = c->H.phi64;  // same field, shared
    L0.phim64 = c->H.phim64;
    if (L0.phim64 && (rc = uniform_needs_real_phi(L0, st)) != HELM_OK) return rc;
    if (L0.phi64 && f32) {
      if ((rc = ctx_alloc(c, (void**)&L0.phi32, sizeof(float) * L0.ntot)) != HELM_OK) return rc;
      k_to_f32<<<ceil_div(L0.ntot, 256), 256, 0, st>>>(L0.phi64, L0.phi32, L0.ntot);
    }
  }
  while ((int)c->lv.size() < pc.max_levels) {
    const LevelHost& F = c->lv.back();
    bool all_small = true;
    int min_n = 1 << 30;
    for (int a = 0; a < F.dim; ++a) {
      if (F.n[a] > pc.coarse_max) all_small = false;
      if (F.n[a] < min_n) min_n = F.n[a];
    }
    // a Sommerfeld high side keeps its boundary node (fine 2c+o = n-1) only when n-1-o is even
    bool odd_somm = false;
    for (int a = 0; a < F.dim; ++a)
      if (((F.somm >> a) & 1) && ((F.n[a] - 1 - F.offset(a)) & 1)) odd_somm = true;
    if (all_small || min_n < 3 || odd_somm) break;
    LevelHost C;
    C.dim = F.dim;
    C.ntot = 1;
    C.somm = F.somm;
    for (int a = 0; a < F.dim; ++a) {
      const int o = F.offset(a);
      int nf = F.n[a], nc = o ? nf / 2 : (nf + 1) / 2;
      const int somm = ((F.somm >> a) & 1) | (((F.somm >> (a + 3)) & 1) << 1);
      if ((rc = ctx_alloc(c, (void**)&C.gap[a], sizeof(double2) * (nc + 1))) != HELM_OK) return rc;
      for (int k = 0; k < 3; ++k) {
        if ((rc = ctx_alloc(c, (void**)&C.coef64[a][k], sizeof(double2) * nc)) != HELM_OK) return rc;
        if (f32 && (rc = ctx_alloc(c, (void**)&C.coef32[a][k], sizeof(float2) * nc)) != HELM_OK) return rc;
      }
      k_axis_coarsen<<<ceil_div(nc + 1, 256), 256, 0, st>>>(F.gap[a], nf, C.gap[a], nc, somm);
      k_axis_coeffs<<<ceil_div(nc, 256), 256, 0, st>>>(C.gap[a], nc, C.coef64[a][0], C.coef64[a][1],
                                                       C.coef64[a][2], C.coef32[a][0],
                                                       C.coef32[a][1], C.coef32[a][2], somm);
      // the last coarse width is the sum of the two last fine ones, both h_l: 2i / (2 h_l)
      C.bt[a] = (somm & 1) ? mkc<double>(0.5 * F.bt[a].x, 0.5 * F.bt[a].y) : mkc<double>(0.0, 0.0);
      C.btl[a] = (somm & 2) ? mkc<double>(0.5 * F.btl[a].x, 0.5 * F.btl[a].y) : mkc<double>(0.0, 0.0);
      C.n[a] = nc;
      C.ntot *= nc;
    }
    C.s = F.s;
    C.phi0 = F.phi0;
    if (F.phi64) {
      if ((rc = ctx_alloc(c, (void**)&C.phi64, sizeof(double) * C.ntot)) != HELM_OK) return rc;
      if (f32 && (rc = ctx_alloc(c, (void**)&C.phi32, sizeof(float) * C.ntot)) != HELM_OK) return rc;
      k_phi_inject<<<ceil_div(C.ntot, 256), 256, 0, st>>>(F.phi64, F.n[0], F.n[1], F.dim, C.phi64,
                                                          C.phi32, C.n[0], C.n[1], C.n[2], F.somm >> 3);
    }
    if (F.phim64) {  // the imaginary part is injected like the real part
      if ((rc = ctx_alloc(c, (void**)&C.phim64, sizeof(double) * C.ntot)) != HELM_OK) return rc;
      k_phi_inject<<<ceil_div(C.ntot, 256), 256, 0, st>>>(F.phim64, F.n[0], F.n[1], F.dim, C.phim64,
                                                          nullptr, C.n[0], C.n[1], C.n[2], F.somm >> 3);
    }
    HELM_CUDA(cudaGetLastError());
    if ((rc = find_uniform(C, st)) != HELM_OK) return rc;
    if (C.phim64 && (rc = uniform_needs_real_phi(C, st)) != HELM_OK) return rc;
    if (galerkin) {
      // R F P replaces the rediscretised row; its uniform-interior shortcut does not apply
      for (int a = 0; a < 3; ++a) { C.ulo[a] = 1; C.uhi[a] = 0; }
      const int nw = C.dim == 3 ? 27 : 9;
      if ((rc = ctx_alloc(c, (void**)&C.stg64, sizeof(double2) * nw * C.ntot)) != HELM_OK) return rc;
      if (f32 && (rc = ctx_alloc(c, (void**)&C.stg32, sizeof(float2) * nw * C.ntot)) != HELM_OK) return rc;
      if (C.dim == 3) {
        dim3 gg(ceil_div(C.n[0], 64), C.n[1], C.n[2]);
        k_galerkin3d<<<gg, 64, 0, st>>>(F.view<double>(), C.n[0], C.n[1], C.n[2], C.stg64, C.stg32);
      } else {
        dim3 gg(ceil_div(C.n[0], 128), C.n[1]);
        k_galerkin2d<<<gg, 128, 0, st>>>(F.view<double>(), C.n[0], C.n[1], C.stg64, C.stg32);
      }
      HELM_CUDA(cudaGetLastError());
    }
    c->lv.push_back(C);
  }
  // work vectors: level 0 needs one spare buffer (its f and u are the caller's); coarser
  // levels need u, f and a spare.  Every level gets its reciprocal diagonal.
  for (size_t l = 0; l < c->lv.size(); ++l) {
    LevelHost& L = c->lv[l];
    if (f32) {
      if ((rc = ctx_alloc(c, (void**)&L.dinv32, sizeof(float2) * L.ntot)) != HELM_OK) return rc;
      if ((rc = ctx_alloc(c, (void**)&L.dg32, sizeof(float2) * L.ntot)) != HELM_OK) return rc;
    } else {
      if ((rc = ctx_alloc(c, (void**)&L.dinv64, sizeof(double2) * L.ntot)) != HELM_OK) return rc;
      if ((rc = ctx_alloc(c, (void**)&L.dg64, sizeof(double2) * L.ntot)) != HELM_OK) return rc;
    }
    {
      OpView<double> v = L.view<double>();
      dim3 g((L.n[0] + 127) / 128, L.n[1], L.n[2]);
      double om = pc.smoother == HELM_SM_JACOBI ? pc.omega : 1.0;
      if (L.stg64)
        k_dinvg<<<ceil_div(L.ntot, 256), 256, 0, st>>>(L.stg64, L.ntot, L.dim == 3 ? 13 : 4, om, L.dinv64, L.dinv32,
                                                       L.dg64, L.dg32);
      else if (L.dim == 1) k_dinv<1><<<g, 128, 0, st>>>(v, om, L.dinv64, L.dinv32, L.dg64, L.dg32);
      else if (L.dim == 2) k_dinv<2><<<g, 128, 0, st>>>(v, om, L.dinv64, L.dinv32, L.dg64, L.dg32);
      else k_dinv<3><<<g, 128, 0, st>>>(v, om, L.dinv64, L.dinv32, L.dg64, L.dg32);
      HELM_CUDA(cudaGetLastError());
    }
    if ((rc = ctx_alloc(c, &L.w, esz * L.ntot)) != HELM_OK) return rc;
    if (l > 0) {
      if ((rc = ctx_alloc(c, &L.u, esz * L.ntot)) != HELM_OK) return rc;
      if ((rc = ctx_alloc(c, &L.f, esz * L.ntot)) != HELM_OK) return rc;
    }
  }
  // ILU(0) factors of every level above the coarsest (solved directly)
  if (pc.smoother == HELM_SM_ILU) {
    for (size_t l = 0; l + 1 < c->lv.size(); ++l) {
      if ((rc = ilu_check(c->lv[l].dim, c->lv[l].n, f32)) != HELM_OK) return rc;
      if ((rc = ilu_build(c, c->lv[l], f32, st)) != HELM_OK) return rc;
    }
  }
  // dense inverse of the coarsest operator, computed in FP64: one block for small levels,
  // the whole GPU (one launch sequence per pivot) above GJ_ONE_BLOCK_MAX unknowns
  LevelHost& Cst = c->lv.back();
  // constant phi on a large coarsest level: the separable exact solve, no dense inverse
  if (Cst.ntot > FDM_MIN_UNKNOWNS && !Cst.phi64 && !Cst.stg64 && !Cst.somm) {  // (somm: either side)
    if ((rc = fdm_build(c, Cst, f32, st)) != HELM_OK) return rc;
    if (c->fdm.on) {
      c->nco = 0;
      c->tail_first = (int)c->lv.size();  // the one-block tail needs the dense inverse
      return tune_and_lay_out(c, st);
    }
  }
  if (Cst.ntot > HELM_COARSE_MAX_UNKNOWNS) {
    set_error("coarsest level too large for the dense direct solve (> 16384 unknowns); raise max_levels");
    return HELM_ERR_ARG;
  }
  int n = (int)Cst.ntot;
  c->nco = n;
  const bool one_block = n <= GJ_ONE_BLOCK_MAX;
  double2 *A = nullptr, *X = nullptr, *prow = nullptr, *fcol = nullptr;
  int *flag = nullptr, *perm = nullptr;
  GjPivot* pv = nullptr;
  std::vector<DevBlock> tmp(3);
  auto free_all = [&]() { dev_free_all(tmp, st); };
  // X holds the inverse (one block) or the pivot row, saved column, pivots and pivot order
  size_t xbytes = one_block ? sizeof(double2) * (size_t)n * n
                            : sizeof(double2) * 2 * (size_t)n + sizeof(GjPivot) + sizeof(int) * (size_t)n + 256;
  helm_status ae = dev_alloc((void**)&A, sizeof(double2) * (size_t)n * n, st, &tmp[0]);
  if (ae == HELM_OK) ae = dev_alloc((void**)&X, xbytes, st, &tmp[1]);
  if (ae == HELM_OK) ae = dev_alloc((void**)&flag, sizeof(int), st, &tmp[2]);
  if (ae != HELM_OK) {
    free_all();
    return ae;
  }
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (Cst.stg64)
    k_dense_assembleg<<<ceil_div(n, 128), 128, 0, st>>>(Cst.stg64, Cst.n[0], Cst.n[1], Cst.n[2], Cst.dim, A, n);
  else k_dense_assemble<<<ceil_div(n, 128), 128, 0, st>>>(Cst.view<double>(), Cst.dim, A, n);
  const double2* inv = X;
  if (one_block) {
    int thr = 1024;
    k_gauss_jordan<<<1, thr, thr * (sizeof(double) + sizeof(int)), st>>>(A, X, n, flag);
  } else {
    prow = X;
    fcol = X + n;
    pv = reinterpret_cast<GjPivot*>(X + 2 * (size_t)n);
    perm = reinterpret_cast<int*>(reinterpret_cast<char*>(pv) + 256);
    dim3 ug(ceil_div(n, 256), n);
    for (int k = 0; k < n; ++k) {
      k_gj_pivot<<<1, 1024, 0, st>>>(A, n, k, pv, perm, flag);
      k_gj_swap<<<ceil_div(n, 256), 256, 0, st>>>(A, n, k, pv, prow, fcol);
      k_gj_update<<<ug, 256, 0, st>>>(A, n, k, prow, fcol);
    }
    k_gj_unpermute<<<ceil_div(n, 128), 128, 0, st>>>(A, n, perm);
    inv = A;
  }
  HELM_CUDA(cudaGetLastError());
  if ((rc = ctx_alloc(c, &c->coarse_inv, esz * (size_t)n * n)) != HELM_OK) {
    free_all();
    return rc;
  }
  if (f32) k_c128_to_c64<<<ceil_div((long)n * n, 256), 256, 0, st>>>(inv, (float2*)c->coarse_inv, (long)n * n);
  else cudaMemcpyAsync(c->coarse_inv, inv, sizeof(double2) * (size_t)n * n, cudaMemcpyDeviceToDevice, st);
  int hflag = 0;
  cudaError_t e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  free_all();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  HELM_CUDA(e);
  if (hflag) {
    set_error("coarsest operator is singular");
    return HELM_ERR_ARG;
  }
  c->tail_first = f32 ? tail_first_level<float>(c) : tail_first_level<double>(c);
  if (galerkin) c->tail_first = (int)c->lv.size();  // the one-block tail runs 5-point rows only
  if (pc.smoother == HELM_SM_ILU) c->tail_first = (int)c->lv.size();  // nor does it smooth with ILU(0)
  return tune_and_lay_out(c, st);
}

// Storage order of the levels, fixed once the tail depth is known: on a 3D FP32 hierarchy with
// red-black Gauss-Seidel, every 7-point level above the coarsest one and the one-block tail stores
// its rows x-split (even x indices first), its reciprocal diagonal permuted to match.
static helm_status assign_layouts(helm_ctx* c, cudaStream_t st) {
  const helm_precond& pc = c->pc;
  if (pc.kind == HELM_PC_NONE || pc.mg_dtype != HELM_C64 || pc.smoother != HELM_SM_RBGS) return HELM_OK;
  const int nl = (int)c->lv.size();
  const int tail = (pc.flags & HELM_PF_UNFUSED) ? nl : c->tail_first;  // unfused: no level runs in the tail
  for (int l = 0; l < nl - 1 && l < tail; ++l) {
    LevelHost& L = c->lv[l];
    if (L.dim != 3 || L.stg64 || L.xs) continue;
    void* tmp = nullptr;
    DevBlock blk;
    helm_status s = dev_alloc(&tmp, sizeof(float2) * L.ntot, st, &blk);
    if (s != HELM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(tmp, L.dinv32, sizeof(float2) * L.ntot, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) s = xs_permute_c64(L, (const float2*)tmp, L.dinv32, st);
    dev_free(blk, st);
    HELM_CUDA(e);
    if (s != HELM_OK) return s;
    L.xs = 1;
  }
  return HELM_OK;
}

static helm_status tune_and_lay_out(helm_ctx* c, cudaStream_t st) {
  helm_status s = autotune_tiles(c, st);
  return s == HELM_OK ? assign_layouts(c, st) : s;
}

helm_status convert_c128_to_mg(helm_ctx* c, const double2* in, void* out, cudaStream_t st) {
  k_c128_to_c64<<<ceil_div(c->n, 256), 256, 0, st>>>(in, (float2*)out, c->n);
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}

}  // namespace helm
