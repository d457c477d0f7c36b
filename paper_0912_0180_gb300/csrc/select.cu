// Choosing the CSL shift or the CSG angle automatically (Section 7, remark on choosing the CSL and
// CSG parameters): multigrid is run as a stationary solver of the preconditioner's own equation
// M u = f, and the parameter is reduced for as long as that iteration still converges within a
// given number of cycles.  The iteration runs on FP64 hierarchies; one norm per cycle is read back
// to the host (this is set-up work, done once before the Krylov solves).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int NORM_BLOCKS = 304;  // 2 x 152 SMs
constexpr int NORM_THREADS = 256;

// partial[b] = sum of |r_i|^2 over the grid-stride slice of block b (fixed order per block)
__global__ void __launch_bounds__(NORM_THREADS) k_sumsq(const double2* __restrict__ r, long n,
                                                        double* __restrict__ partial) {
  __shared__ double sh[NORM_THREADS / 32];
  double s = 0.0;
  for (long i = blockIdx.x * (long)NORM_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * NORM_THREADS) {
    double2 v = r[i];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NORM_THREADS / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// out = sqrt(sum of the partial sums), one block
__global__ void __launch_bounds__(NORM_THREADS) k_sumsq_final(const double* __restrict__ partial, int nb,
                                                              double* __restrict__ out) {
  __shared__ double sh[NORM_THREADS / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += NORM_THREADS) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NORM_THREADS / 32; ++w) t += sh[w];
    *out = sqrt(t);
  }
}

__global__ void k_accumulate(double2* __restrict__ u, const double2* __restrict__ z, long n) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) {
    double2 a = u[i], b = z[i];
    u[i] = make_double2(a.x + b.x, a.y + b.y);
  }
}

__global__ void k_sub_from(const double2* __restrict__ f, double2* __restrict__ r, long n) {  // r = f - r
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) {
    double2 a = f[i], b = r[i];
    r[i] = make_double2(a.x - b.x, a.y - b.y);
  }
}

struct Scratch {
  void* buf = nullptr;
  DevBlock blk;
  double* host = nullptr;
  cudaStream_t st = nullptr;
  ~Scratch() {
    dev_free(blk, st);
    if (host) pinned_slot_put(host);
  }
};

helm_status device_norm(const double2* r, long n, double* partial, double* dnorm, double* host, cudaStream_t st,
                        double* out) {
  k_sumsq<<<NORM_BLOCKS, NORM_THREADS, 0, st>>>(r, n, partial);
  k_sumsq_final<<<1, NORM_THREADS, 0, st>>>(partial, NORM_BLOCKS, dnorm);
  HELM_CUDA(cudaGetLastError());
  HELM_CUDA(cudaMemcpyAsync(host, dnorm, sizeof(double), cudaMemcpyDeviceToHost, st));
  HELM_CUDA(cudaStreamSynchronize(st));
  *out = *host;
  return HELM_OK;
}

}  // namespace

helm_status mg_iterate(helm_ctx* c, const double2* f, double2* u, int max_cycles, double reduction, int* cycles,
                       double* hist, cudaStream_t st) {
  *cycles = -1;
  long n = c->n;
  Scratch s;
  s.st = st;
  size_t bytes = sizeof(double2) * 2 * (size_t)n + sizeof(double) * (NORM_BLOCKS + 2);
  helm_status as = dev_alloc(&s.buf, bytes, st, &s.blk);
  if (as != HELM_OK) return as;
  s.host = (double*)pinned_slot_get(sizeof(double));
  if (!s.host) { set_error("pinned host slot"); return HELM_ERR_OOM; }
  double2* r = (double2*)s.buf;
  double2* z = r + n;
  double* partial = (double*)(z + n);
  double* dnorm = partial + NORM_BLOCKS;
  HELM_CUDA(cudaMemsetAsync(u, 0, sizeof(double2) * n, st));
  double fn = 0.0;
  helm_status e = device_norm(f, n, partial, dnorm, s.host, st, &fn);
  if (e != HELM_OK) return e;
  if (fn == 0.0) { *cycles = 0; return HELM_OK; }
  HELM_CUDA(cudaMemcpyAsync(r, f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
  int blocks = (int)((n + 255) / 256);
  for (int k = 1; k <= max_cycles; ++k) {
    if ((e = mg_vcycle<double>(c, r, z, false, nullptr, st)) != HELM_OK) return e;  // z = V r
    k_accumulate<<<blocks, 256, 0, st>>>(u, z, n);                                 // u += z
    if ((e = mg_level_op(c, HELM_OP_APPLY, 0, u, nullptr, r, 0, st)) != HELM_OK) return e;  // r = M u
    k_sub_from<<<blocks, 256, 0, st>>>(f, r, n);                                   // r = f - M u
    HELM_CUDA(cudaGetLastError());
    double rn = 0.0;
    if ((e = device_norm(r, n, partial, dnorm, s.host, st, &rn)) != HELM_OK) return e;
    double rel = rn / fn;
    if (hist) hist[k - 1] = rel;
    if (rel <= reduction) { *cycles = k; break; }
    if (!(rel <= 1e6)) break;  // diverging or not finite
  }
  return HELM_OK;
}

}  // namespace helm

using namespace helm;

extern "C" {

helm_status helm_mg_iterate(helm_ctx* c, const void* f, void* u, int max_cycles, double reduction, int* cycles,
                            double* hist, void* stream) {
  if (!c || !f || !u || !cycles || f == u) { set_error("helm_mg_iterate: NULL or aliased arguments"); return HELM_ERR_ARG; }
  *cycles = -1;
  if (c->pc.kind == HELM_PC_NONE || c->pc.mg_dtype != HELM_C128) {
    set_error("helm_mg_iterate needs a multigrid preconditioner with an FP64 hierarchy");
    return HELM_ERR_ARG;
  }
  if (max_cycles < 1 || max_cycles > 100000 || !(reduction > 0.0 && reduction < 1.0)) {
    set_error("helm_mg_iterate: max_cycles in [1, 100000], reduction in (0, 1)");
    return HELM_ERR_ARG;
  }
  if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) { set_error("helm_mg_iterate: misaligned"); return HELM_ERR_ARG; }
  return mg_iterate(c, (const double2*)f, (double2*)u, max_cycles, reduction, cycles, hist, (cudaStream_t)stream);
}

helm_status helm_select_precond(const helm_grid* grid, const helm_kspec* k, const helm_precond* start,
                                const void* f, int max_cycles, double reduction, double factor, int max_trials,
                                helm_precond* out, double* params, int* cycles, int* trials, void* stream) {
  if (!grid || !k || !start || !f || !out || !trials) { set_error("helm_select_precond: NULL argument"); return HELM_ERR_ARG; }
  *trials = 0;
  if (start->kind == HELM_PC_NONE) { set_error("helm_select_precond: needs a CSL or CSG preconditioner"); return HELM_ERR_ARG; }
  if (!(factor > 0.0 && factor < 1.0) || max_trials < 1 || max_trials > 64) {
    set_error("helm_select_precond: factor in (0, 1), max_trials in [1, 64]");
    return HELM_ERR_ARG;
  }
  if (max_cycles < 1 || max_cycles > 100000 || !(reduction > 0.0 && reduction < 1.0)) {
    set_error("helm_select_precond: max_cycles in [1, 100000], reduction in (0, 1)");
    return HELM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  *out = *start;
  helm_precond pc = *start;
  pc.mg_dtype = HELM_C128;            // the decision is taken on FP64 hierarchies
  pc.flags |= HELM_PF_NO_AUTOTUNE;    // each trial's hierarchy runs a few cycles only
  double p = start->kind == HELM_PC_CSL ? start->shift_im : start->theta_beta;
  bool any = false;
  void* u = nullptr;
  DevBlock ublk;
  helm_status result = HELM_OK;
  for (int t = 0; t < max_trials; ++t) {
    if (t > 0) p *= factor;
    if (pc.kind == HELM_PC_CSL) pc.shift_im = p; else pc.theta_beta = p;
    helm_ctx* c = nullptr;
    helm_status e = helm_create(grid, k, &pc, stream, &c);
    if (e != HELM_OK) { result = e; break; }
    if (!u) {
      helm_status ae = dev_alloc(&u, sizeof(double2) * c->n, st, &ublk);
      if (ae != HELM_OK) { helm_destroy(c); result = ae; break; }
    }
    int kc = -1;
    e = helm_mg_iterate(c, f, u, max_cycles, reduction, &kc, nullptr, stream);
    helm_destroy(c);
    if (e != HELM_OK) { result = e; break; }
    if (params) params[t] = p;
    if (cycles) cycles[t] = kc;
    *trials = t + 1;
    if (kc < 0) break;
    any = true;
    *out = *start;
    if (out->kind == HELM_PC_CSL) out->shift_im = p; else out->theta_beta = p;
  }
  dev_free(ublk, st);
  cudaStreamSynchronize(st);
  if (result != HELM_OK) return result;
  if (!any) { set_error("helm_select_precond: multigrid does not converge at the starting parameter"); return HELM_ERR_MAXIT; }
  return HELM_OK;
}

}  // extern "C"
