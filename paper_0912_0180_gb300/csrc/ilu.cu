// ilu.cu -- ILU(0) smoothing on 1D and 2D multigrid levels (Section 6.1: the smoother of the
// paper's experiments).
//
// The factors: L (unit lower) and U (upper) keep the sparsity pattern of the level matrix M
// (unknowns in lexicographic order, x fastest) and L U agrees with M on that pattern -- the
// row-wise form of Gaussian elimination with every fill entry outside the pattern dropped.  The
// pattern is the level's stencil: the Shortley-Weller cross (3 points in 1D, 5 in 2D) or the
// 9-point box of a Galerkin coarse operator.  One smoothing step is the defect correction
// u <- u + (L U)^{-1} (f - M u).
//
// Both the factorisation and the two triangular solves are recurrences over the rows: the row of
// (i, j) needs rows (i-1, j-1), (i, j-1), (i+1, j-1) and (i-1, j) first (the solve with U the
// mirror image).  Along the wavefronts t = i + 2j those rows lie on t-3, t-2, t-1 and t-1, so
// every point of one wavefront is independent of the others: one block walks the wavefronts, a
// thread per row (one point of each row lies on a wavefront), with a barrier between wavefronts.
// The values of the last three wavefronts stay in a shared-memory ring indexed by row, so a point
// reads its neighbours from shared memory.  The factors are computed once, in FP64, at create and
// stored in the multigrid precision; a level's 9 factor entries of point p sit at [9p + s], slot
// s = 3 (dj + 1) + (di + 1) of the neighbour (i + di, j + dj): L at the lower slots 0..3, U at 5..8,
// and at slot 4 the reciprocal of U's pivot (both the elimination and the solve multiply by it).
#include <algorithm>
#include <type_traits>

#include "helm_internal.cuh"

namespace helm {

constexpr int ILU_THREADS = 1024;        // the solve: a thread per row, up to 1024
constexpr int ILU_FACTOR_THREADS = 512;  // the factorisation (more registers a thread)

// whether (i + di, j + dj) is in row (i, j)'s pattern: inside the grid and the 3 x 3 box (the
// elimination also produces offsets of 2, fill outside every pattern), on the cross unless box
__device__ __forceinline__ bool ilu_in_pattern(int n0, int n1, bool box, int i, int j, int di, int dj) {
  const int ii = i + di, jj = j + dj;
  if (ii < 0 || ii >= n0 || jj < 0 || jj >= n1) return false;
  if (di < -1 || di > 1 || dj < -1 || dj > 1) return false;
  return box || di == 0 || dj == 0;
}

// The factors of one level, FP64.  stg: the Galerkin weights [9][ntot] (box pattern), else the
// Shortley-Weller rows of op.  f64 / f32: where the factors go (either may be null).
__global__ void __launch_bounds__(ILU_FACTOR_THREADS) k_ilu_factor(OpView<double> op, const double2* __restrict__ stg,
                                                            double2* __restrict__ f64, float2* __restrict__ f32) {
  const int n0 = op.n[0], n1 = op.n[1];
  const long ntot = (long)n0 * n1;
  const bool box = stg != nullptr;
  const int lo[4][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}};  // lower neighbours, columns increasing
  const int up[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};      // upper neighbours
  const int waves = n0 + 2 * (n1 - 1);
  for (int t = 0; t < waves; ++t) {
    for (int j = threadIdx.x; j < n1; j += blockDim.x) {
      const int i = t - 2 * j;
      if (i < 0 || i >= n0) continue;
      const long p = i + (long)n0 * j;
      double2 a[9];
#pragma unroll
      for (int s = 0; s < 9; ++s) a[s] = make_double2(0.0, 0.0);
      if (box) {
#pragma unroll
        for (int s = 0; s < 9; ++s)
          if (ilu_in_pattern(n0, n1, true, i, j, s % 3 - 1, s / 3 - 1)) a[s] = stg[(long)s * ntot + p];
      } else {
        double2 d = op.a0[0][i];
        if (n1 > 1) d = cadd<double>(d, op.a0[1][j]);
        const double ph = op.phi ? op.phi[p] : op.phi0;
        d = cadd<double>(d, somm_diag(op, i, j, 0, ph));
        a[4] = csub<double>(d, sigma64(op, p, ph));
        if (i > 0) a[3] = op.am[0][i];
        if (i < n0 - 1) a[5] = op.ap[0][i];
        if (j > 0) a[1] = op.am[1][j];
        if (j < n1 - 1) a[7] = op.ap[1][j];
      }
      // eliminate with the rows above, in increasing column order; fill outside the pattern is
      // dropped
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int di = lo[k][0], dj = lo[k][1];
        if (!ilu_in_pattern(n0, n1, box, i, j, di, dj)) continue;
        const double2* uk = f64 + 9 * (p + di + (long)n0 * dj);  // row k, factored on an earlier wavefront
        const int sk = 3 * (dj + 1) + (di + 1);
        const double2 l = cmul<double>(a[sk], uk[4]);  // uk[4]: 1 / row k's pivot
        a[sk] = l;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int ei = up[v][0], ej = up[v][1];
          if (!ilu_in_pattern(n0, n1, box, i + di, j + dj, ei, ej)) continue;
          const int ti = di + ei, tj = dj + ej;
          if (!ilu_in_pattern(n0, n1, box, i, j, ti, tj)) continue;
          const int st = 3 * (tj + 1) + (ti + 1);
          a[st] = csub<double>(a[st], cmul<double>(l, uk[3 * (ej + 1) + (ei + 1)]));
        }
      }
      a[4] = crecip<double>(a[4]);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        f64[9 * p + s] = a[s];
        if (f32) f32[9 * p + s] = cconv<float, double>(a[s]);
      }
    }
    __syncthreads();
  }
}

// One ILU(0) step's solves: y = L^{-1} in (y may be in itself), then z = U^{-1} y and u += z
// (u = z when zero: the step from u = 0, whose residual is f).  ring: [4][n1] values of the last
// wavefronts, dynamic shared memory.
template <typename T>
__global__ void __launch_bounds__(ILU_THREADS) k_ilu_solve(int n0, int n1, const cx<T>* __restrict__ fac,
                                                           const cx<T>* in, cx<T>* y, cx<T>* __restrict__ u,
                                                           int zero, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char ilu_ring[];
  cx<T>* ring = reinterpret_cast<cx<T>*>(ilu_ring);
  const int waves = n0 + 2 * (n1 - 1);
  for (int t = 0; t < waves; ++t) {
    for (int j = threadIdx.x; j < n1; j += blockDim.x) {
      const int i = t - 2 * j;
      if (i < 0 || i >= n0) continue;
      const long p = i + (long)n0 * j;
      const cx<T>* w = fac + 9 * p;
      cx<T> v = in[p];
      if (j > 0) {
        if (i > 0) v = csub<T>(v, cmul<T>(w[0], ring[((t - 3) & 3) * n1 + j - 1]));
        v = csub<T>(v, cmul<T>(w[1], ring[((t - 2) & 3) * n1 + j - 1]));
        if (i < n0 - 1) v = csub<T>(v, cmul<T>(w[2], ring[((t - 1) & 3) * n1 + j - 1]));
      }
      if (i > 0) v = csub<T>(v, cmul<T>(w[3], ring[((t - 1) & 3) * n1 + j]));
      ring[(t & 3) * n1 + j] = v;
      y[p] = v;
    }
    __syncthreads();
  }
  for (int t = waves - 1; t >= 0; --t) {
    for (int j = threadIdx.x; j < n1; j += blockDim.x) {
      const int i = t - 2 * j;
      if (i < 0 || i >= n0) continue;
      const long p = i + (long)n0 * j;
      const cx<T>* w = fac + 9 * p;
      cx<T> v = y[p];
      if (i < n0 - 1) v = csub<T>(v, cmul<T>(w[5], ring[((t + 1) & 3) * n1 + j]));
      if (j < n1 - 1) {
        if (i > 0) v = csub<T>(v, cmul<T>(w[6], ring[((t + 1) & 3) * n1 + j + 1]));
        v = csub<T>(v, cmul<T>(w[7], ring[((t + 2) & 3) * n1 + j + 1]));
        if (i < n0 - 1) v = csub<T>(v, cmul<T>(w[8], ring[((t + 3) & 3) * n1 + j + 1]));
      }
      v = cmul<T>(v, w[4]);  // w[4]: 1 / the pivot
      ring[(t & 3) * n1 + j] = v;
      u[p] = zero ? v : cadd<T>(u[p], v);
    }
    __syncthreads();
  }
}

static int ilu_threads(int n1) { return std::min(ILU_THREADS, (n1 + 31) / 32 * 32); }

template <typename T>
static size_t ilu_smem(int n1) {
  return sizeof(cx<T>) * 4 * (size_t)n1;
}

helm_status ilu_check(int dim, const int n[3], bool f32) {
  if (dim > 2) {
    set_error("ILU(0) smoothing runs on 1D and 2D levels");
    return HELM_ERR_ARG;
  }
  const size_t smem = f32 ? ilu_smem<float>(n[1]) : ilu_smem<double>(n[1]);
  if (smem > ILU_SMEM_MAX) {
    set_error("ILU(0) smoothing keeps 4 values per row in shared memory: at most " +
              std::to_string(ILU_SMEM_MAX / (4 * (f32 ? 8 : 16))) + " rows in this precision");
    return HELM_ERR_ARG;
  }
  return HELM_OK;
}

helm_status ilu_build(helm_ctx* c, LevelHost& L, bool f32, cudaStream_t st) {
  helm_status rc;
  if ((rc = ctx_alloc(c, (void**)&L.ilu64, sizeof(double2) * 9 * L.ntot)) != HELM_OK) return rc;
  if (f32 && (rc = ctx_alloc(c, (void**)&L.ilu32, sizeof(float2) * 9 * L.ntot)) != HELM_OK) return rc;
  k_ilu_factor<<<1, std::min(ILU_FACTOR_THREADS, ilu_threads(L.n[1])), 0, st>>>(L.view<double>(), L.stg64, L.ilu64, f32 ? L.ilu32 : nullptr);
  HELM_CUDA(cudaGetLastError());
  // the solve's ring may exceed the default 48 KB: raise the block's limit here, outside any
  // stream capture
  if (f32) HELM_CUDA(cudaFuncSetAttribute(k_ilu_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ILU_SMEM_MAX));
  else HELM_CUDA(cudaFuncSetAttribute(k_ilu_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ILU_SMEM_MAX));
  return HELM_OK;
}

template <typename T>
void ilu_solve(const LevelHost& L, const cx<T>* in, cx<T>* y, cx<T>* u, bool zero, const int* skip, cudaStream_t st) {
  const cx<T>* fac = std::is_same<T, double>::value ? (const cx<T>*)(const void*)L.ilu64 : (const cx<T>*)(const void*)L.ilu32;
  const int n1 = L.n[1];
  launch_pdl(k_ilu_solve<T>, dim3(1), dim3(ilu_threads(n1)), ilu_smem<T>(n1), st, L.n[0], n1, fac, in, y, u,
             zero ? 1 : 0, skip);
}

template void ilu_solve<float>(const LevelHost&, const float2*, float2*, float2*, bool, const int*, cudaStream_t);
template void ilu_solve<double>(const LevelHost&, const double2*, double2*, double2*, bool, const int*, cudaStream_t);

}  // namespace helm
