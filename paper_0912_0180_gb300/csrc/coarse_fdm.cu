// coarse_fdm.cu -- exact coarsest-level solve by separation of variables.
//
// When k (so phi) is constant on the coarsest level, its operator is a Kronecker sum of the
// per-axis Shortley-Weller matrices minus a constant: M = T_x (+) T_y (+) T_z - s phi0 I (Section 3,
// eq. "shortwell", summed over axes).  With T_a = V_a diag(lambda_a) V_a^{-1},
//   M^{-1} = (V_x (x) V_y (x) V_z) diag(1 / (lambda_x,i + lambda_y,j + lambda_z,l - s phi0)) (V_x^{-1} (x) ...),
// applied as one dense n_a x n_a transform along each axis, the scaling, and the transforms back:
// about 2 d n^(d+1) complex multiply-adds instead of the n^(2d) of a dense inverse.  This is the
// direct coarse solve of the V-cycle, exact up to rounding (like the dense inverse, which serves
// levels with variable k).
//
// The eigendecompositions are computed once on the host in FP64: complex Schur form by the
// single-shift QR algorithm (Wilkinson shifts, Givens bulge chasing, on the tridiagonal matrix,
// which is already Hessenberg), eigenvectors by back substitution on the triangular factor, V^{-1}
// by Gauss-Jordan with partial pivoting.  The decomposition is used only if it reproduces T_a
// (||T V - V Lambda|| and ||V V^{-1} - I|| below 1e-11 relative); otherwise the dense inverse is built.
#include <cmath>
#include <complex>
#include <vector>

#include "helm_internal.cuh"

namespace helm {

using zc = std::complex<double>;

namespace {

struct Dense {
  int n;
  std::vector<zc> a;  // row-major
  explicit Dense(int n_) : n(n_), a((size_t)n_ * n_) {}
  zc& operator()(int i, int j) { return a[(size_t)i * n + j]; }
};

double max_abs(const Dense& m) {
  double r = 0.0;
  for (const zc& v : m.a) r = std::max(r, std::abs(v));
  return r;
}

// Rotation [c s; -conj(s) c] (c real) that maps (x, y) to (r, 0).
void givens(zc x, zc y, double& c, zc& s) {
  double ax = std::abs(x), ay = std::abs(y);
  if (ay == 0.0) { c = 1.0; s = 0.0; return; }
  if (ax == 0.0) { c = 0.0; s = std::conj(y) / ay; return; }
  double r = std::hypot(ax, ay);
  c = ax / r;
  s = (x / ax) * std::conj(y) / r;
}

// H <- G H G^H on rows / columns k, k+1; Z <- Z G^H.
void rotate(Dense& H, Dense& Z, int k, double c, zc s) {
  const int n = H.n;
  for (int j = 0; j < n; ++j) {
    zc a = H(k, j), b = H(k + 1, j);
    H(k, j) = c * a + s * b;
    H(k + 1, j) = -std::conj(s) * a + c * b;
  }
  for (int i = 0; i < n; ++i) {
    zc a = H(i, k), b = H(i, k + 1);
    H(i, k) = a * c + b * std::conj(s);
    H(i, k + 1) = -a * s + b * c;
    zc za = Z(i, k), zb = Z(i, k + 1);
    Z(i, k) = za * c + zb * std::conj(s);
    Z(i, k + 1) = -za * s + zb * c;
  }
}

// Complex Schur form of an upper Hessenberg H: H <- R (upper triangular), Z accumulates the
// unitary factor (A = Z R Z^H).  Returns false if an eigenvalue does not converge.
bool schur(Dense& H, Dense& Z) {
  const int n = H.n;
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      double tiny = eps * (std::abs(H(l - 1, l - 1)) + std::abs(H(l, l)));
      if (std::abs(H(l, l - 1)) <= tiny) { H(l, l - 1) = 0.0; break; }
      --l;
    }
    if (l == hi) { --hi; iter = 0; continue; }
    if (++iter > 60 * n) return false;
    // Wilkinson shift from the trailing 2 x 2 block, or an exceptional one now and then
    zc a = H(hi - 1, hi - 1), b = H(hi - 1, hi), cc = H(hi, hi - 1), d = H(hi, hi);
    zc mu;
    if (iter % 11 == 10) {
      mu = d + std::abs(H(hi, hi - 1));
    } else {
      zc tr2 = 0.5 * (a + d);
      zc disc = std::sqrt(0.25 * (a - d) * (a - d) + b * cc);
      zc m1 = tr2 + disc, m2 = tr2 - disc;
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    // one implicit QR sweep on rows / columns l..hi
    zc x = H(l, l) - mu, y = H(l + 1, l);
    for (int k = l; k < hi; ++k) {
      double c;
      zc s;
      givens(x, y, c, s);
      rotate(H, Z, k, c, s);
      if (k < hi - 1) { x = H(k + 1, k); y = H(k + 2, k); }
    }
  }
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < i; ++j) H(i, j) = 0.0;
  return true;
}

// Inverse by Gauss-Jordan with partial pivoting; false if singular.
bool invert(const Dense& A, Dense& X) {
  const int n = A.n;
  Dense W = A;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) X(i, j) = i == j ? 1.0 : 0.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::abs(W(r, k)) > std::abs(W(p, k))) p = r;
    if (std::abs(W(p, k)) == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) { std::swap(W(k, j), W(p, j)); std::swap(X(k, j), X(p, j)); }
    zc ip = 1.0 / W(k, k);
    for (int j = 0; j < n; ++j) { W(k, j) *= ip; X(k, j) *= ip; }
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      zc f = W(r, k);
      if (f == zc(0.0)) continue;
      for (int j = 0; j < n; ++j) { W(r, j) -= f * W(k, j); X(r, j) -= f * X(k, j); }
    }
  }
  return true;
}

}  // namespace

// Eigendecomposition of the tridiagonal T (rows am, a0, ap; am[0] and ap[n-1] unused):
// T = V diag(lam) V^{-1}.  Returns false when the decomposition does not reproduce T.
bool fdm_axis(int n, const double2* am, const double2* a0, const double2* ap, std::vector<zc>& V,
              std::vector<zc>& Vi, std::vector<zc>& lam) {
  Dense T(n), H(n), Z(n);
  for (int i = 0; i < n; ++i) {
    T(i, i) = zc(a0[i].x, a0[i].y);
    if (i > 0) T(i, i - 1) = zc(am[i].x, am[i].y);
    if (i < n - 1) T(i, i + 1) = zc(ap[i].x, ap[i].y);
    Z(i, i) = 1.0;
  }
  H = T;
  if (!schur(H, Z)) return false;
  const double rn = max_abs(H);
  // eigenvectors of the triangular factor by back substitution
  Dense Y(n);
  for (int k = 0; k < n; ++k) {
    zc lk = H(k, k);
    Y(k, k) = 1.0;
    for (int j = k - 1; j >= 0; --j) {
      zc acc = 0.0;
      for (int m = j + 1; m <= k; ++m) acc += H(j, m) * Y(m, k);
      zc den = H(j, j) - lk;
      if (std::abs(den) < 1e-14 * rn) den = 1e-14 * rn;
      Y(j, k) = -acc / den;
    }
  }
  Dense Vm(n), Vim(n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      zc acc = 0.0;
      for (int m = 0; m <= k; ++m) acc += Z(i, m) * Y(m, k);
      Vm(i, k) = acc;
    }
  for (int k = 0; k < n; ++k) {  // unit columns
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::norm(Vm(i, k));
    s = 1.0 / std::sqrt(s);
    for (int i = 0; i < n; ++i) Vm(i, k) *= s;
  }
  if (!invert(Vm, Vim)) return false;
  // checks: T V = V Lambda and V V^{-1} = I
  const double tn = max_abs(T);
  double e1 = 0.0, e2 = 0.0;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      zc tv = 0.0, vv = 0.0;
      for (int m = 0; m < n; ++m) { tv += T(i, m) * Vm(m, k); vv += Vm(i, m) * Vim(m, k); }
      e1 = std::max(e1, std::abs(tv - Vm(i, k) * H(k, k)));
      e2 = std::max(e2, std::abs(vv - (i == k ? 1.0 : 0.0)));
    }
  if (!(e1 <= 1e-11 * tn) || !(e2 <= 1e-11)) return false;
  V = Vm.a;
  Vi = Vim.a;
  lam.resize(n);
  for (int k = 0; k < n; ++k) lam[k] = H(k, k);
  return true;
}

// ---- device side ----------------------------------------------------------------------------

// out = A along `axis` applied to in (one dense n_a x n_a product per grid line); with dsc, each
// result is then multiplied by dsc at its point (the 1 / (eigenvalue sum) scaling).
template <typename T>
__global__ void k_fdm_axis(const cx<T>* __restrict__ in, cx<T>* __restrict__ out, const cx<T>* __restrict__ A,
                           int axis, int n0, int n1, int n2, const cx<T>* __restrict__ dsc, const int* skip) {
  pdl_entry();
  if (skip && *skip) return;
  const long ntot = (long)n0 * n1 * n2;
  const long p = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (p >= ntot) return;
  const int i = (int)(p % n0), j = (int)((p / n0) % n1), l = (int)(p / ((long)n0 * n1));
  const int na = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
  const int q = axis == 0 ? i : (axis == 1 ? j : l);
  const long st = axis == 0 ? 1 : (axis == 1 ? (long)n0 : (long)n0 * n1);
  const long base = p - (long)q * st;
  const cx<T>* row = A + (long)q * na;
  cx<T> acc = mkc<T>(T(0), T(0));
  for (int m = 0; m < na; ++m) acc = cfma<T>(row[m], in[base + m * st], acc);
  if (dsc) acc = cmul<T>(acc, dsc[p]);
  out[p] = acc;
}

// z = M^{-1} f on the coarsest level: forward transforms (V_a^{-1}) along every axis, the scaling,
// and the transforms back (V_a), ping-ponging through two scratch vectors.
template <typename T>
void fdm_apply(const helm_ctx* c, const cx<T>* f, cx<T>* z, const int* skip, cudaStream_t st) {
  const FdmCoarse& F = c->fdm;
  const int d = F.dim;
  const long ntot = (long)F.n[0] * F.n[1] * F.n[2];
  const int thr = 256, blocks = (int)((ntot + thr - 1) / thr);
  cx<T>* s[2] = {(cx<T>*)F.scr, (cx<T>*)F.scr + ntot};
  const cx<T>* src = f;
  int k = 0;
  for (int a = 0; a < d; ++a) {  // forward
    const cx<T>* dsc = a == d - 1 ? (const cx<T>*)F.dinv : nullptr;
    launch_pdl(k_fdm_axis<T>, dim3(blocks), dim3(thr), 0, st, src, s[k], (const cx<T>*)F.Vi[a], a, F.n[0], F.n[1],
               F.n[2], dsc, skip);
    src = s[k];
    k ^= 1;
  }
  for (int a = d - 1; a >= 0; --a) {  // back
    cx<T>* dst = a == 0 ? z : s[k];
    launch_pdl(k_fdm_axis<T>, dim3(blocks), dim3(thr), 0, st, src, dst, (const cx<T>*)F.V[a], a, F.n[0], F.n[1],
               F.n[2], (const cx<T>*)nullptr, skip);
    src = dst;
    k ^= 1;
  }
}
template void fdm_apply<float>(const helm_ctx*, const float2*, float2*, const int*, cudaStream_t);
template void fdm_apply<double>(const helm_ctx*, const double2*, double2*, const int*, cudaStream_t);

// Builds the separable coarsest solve when the coarsest level has a constant phi; c->fdm.on stays
// false (and the dense inverse is built instead) when a decomposition does not pass its checks or
// an eigenvalue sum vanishes.
helm_status fdm_build(helm_ctx* c, const LevelHost& L, bool f32, cudaStream_t st) {
  FdmCoarse& F = c->fdm;
  F = FdmCoarse{};
  if (L.phi64 || L.dim < 1) return HELM_OK;
  std::vector<zc> V[3], Vi[3], lam[3];
  for (int a = 0; a < L.dim; ++a) {
    const int n = L.n[a];
    std::vector<double2> am(n), a0(n), ap(n);
    HELM_CUDA(cudaMemcpyAsync(am.data(), L.coef64[a][0], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaMemcpyAsync(a0.data(), L.coef64[a][1], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaMemcpyAsync(ap.data(), L.coef64[a][2], sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaStreamSynchronize(st));
    if (!fdm_axis(n, am.data(), a0.data(), ap.data(), V[a], Vi[a], lam[a])) return HELM_OK;
  }
  const int n0 = L.n[0], n1 = L.dim > 1 ? L.n[1] : 1, n2 = L.dim > 2 ? L.n[2] : 1;
  const long ntot = (long)n0 * n1 * n2;
  const zc shift = zc(L.s.x, L.s.y) * L.phi0;
  std::vector<zc> dinv(ntot);
  double dmax = 0.0, dmin = 1e300;
  for (int l = 0; l < n2; ++l)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        zc dv = lam[0][i] + (L.dim > 1 ? lam[1][j] : zc(0.0)) + (L.dim > 2 ? lam[2][l] : zc(0.0)) - shift;
        dmax = std::max(dmax, std::abs(dv));
        dmin = std::min(dmin, std::abs(dv));
        dinv[i + (long)n0 * (j + (long)n1 * l)] = 1.0 / dv;
      }
  if (!(dmin > 1e-12 * dmax)) return HELM_OK;
  const size_t esz = f32 ? sizeof(float2) : sizeof(double2);
  auto upload = [&](const std::vector<zc>& h, void** dst) -> helm_status {
    helm_status s = ctx_alloc(c, dst, esz * h.size());
    if (s != HELM_OK) return s;
    std::vector<unsigned char> buf(esz * h.size());
    for (size_t q = 0; q < h.size(); ++q) {
      if (f32) reinterpret_cast<float2*>(buf.data())[q] = make_float2((float)h[q].real(), (float)h[q].imag());
      else reinterpret_cast<double2*>(buf.data())[q] = make_double2(h[q].real(), h[q].imag());
    }
    HELM_CUDA(cudaMemcpyAsync(*dst, buf.data(), buf.size(), cudaMemcpyHostToDevice, st));
    return cudaStreamSynchronize(st) == cudaSuccess ? HELM_OK : HELM_ERR_CUDA;
  };
  helm_status s;
  for (int a = 0; a < L.dim; ++a) {
    if ((s = upload(V[a], &F.V[a])) != HELM_OK) return s;
    if ((s = upload(Vi[a], &F.Vi[a])) != HELM_OK) return s;
  }
  if ((s = upload(dinv, &F.dinv)) != HELM_OK) return s;
  if ((s = ctx_alloc(c, &F.scr, esz * 2 * ntot)) != HELM_OK) return s;
  F.dim = L.dim;
  F.n[0] = n0;
  F.n[1] = n1;
  F.n[2] = n2;
  F.on = true;
  return HELM_OK;
}

}  // namespace helm
