// noalloc.cu -- helm_residual_noalloc: r = b - H x and ||r|| / ||b|| without any device
// allocation.  It is the true-residual kernel that helm_solve runs after its Krylov loop, with
// the per-block partial sums and the completion ticket kept in a file-scope static device array
// instead of the context's Krylov workspace.
//
// The array lives in the module: every device that loads libhelm.so holds
// sizeof(g_noalloc_scratch) bytes until the process exits.  Host code cannot use the array's
// name as a device address, so the entry point looks the address up with cudaGetSymbolAddress
// (with the context's device current) and every launch gets that pointer.
#include <mutex>

#include "stencil.cuh"

namespace helm {

constexpr int NA_THREADS = 256;
constexpr long NA_POINTS_PER_BLOCK = 1024;  // each block reduces a fixed slice of the grid
constexpr int NA_MAX_BLOCKS = 4096;         // -> at most 4,194,304 unknowns
constexpr int NA_PARTIALS = 2 * NA_MAX_BLOCKS;  // ||r||^2 and ||b||^2 per block
constexpr int NA_TICKET = NA_PARTIALS;          // one slot used as the completion counter
constexpr int NA_DOUBLES = NA_PARTIALS + 32;    // partials, ticket, padding to 256 B

// 64 KiB + 256 B, shared by every call on a device.
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

template <int DIM>
__global__ void __launch_bounds__(NA_THREADS)
k_residual_noalloc(OpView<double> H, const double2* __restrict__ b, const double2* __restrict__ x,
                   double2* __restrict__ r, long n, double* scratch, double* rel_out) {
  __shared__ double s_rr[NA_THREADS / 32], s_bb[NA_THREADS / 32];
  __shared__ bool last;
  long lo = blockIdx.x * NA_POINTS_PER_BLOCK;
  long hi = lo + NA_POINTS_PER_BLOCK < n ? lo + NA_POINTS_PER_BLOCK : n;
  double rr = 0.0, bb = 0.0;
  for (long p = lo + threadIdx.x; p < hi; p += NA_THREADS) {
    int i, j, l;
    unflatten(p, H.n, i, j, l);
    double2 bp = b[p];
    double2 ri = csub<double>(bp, op_row<double, double, DIM>(H, x, i, j, l, p));
    r[p] = ri;
    rr = fma(ri.x, ri.x, fma(ri.y, ri.y, rr));
    bb = fma(bp.x, bp.x, fma(bp.y, bp.y, bb));
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { s_rr[w] = rr; s_bb[w] = bb; }
  __syncthreads();
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + NA_TICKET);
  if (threadIdx.x == 0) {
    double tr = 0.0, tb = 0.0;
    for (int k = 0; k < NA_THREADS / 32; ++k) { tr += s_rr[k]; tb += s_bb[k]; }
    scratch[2 * blockIdx.x] = tr;
    scratch[2 * blockIdx.x + 1] = tb;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block sums the partials in a fixed order
  rr = 0.0; bb = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += NA_THREADS) {
    rr += __ldcg(&scratch[2 * k]);
    bb += __ldcg(&scratch[2 * k + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    bb += __shfl_down_sync(0xffffffffu, bb, o);
  }
  __syncthreads();
  if (lane == 0) { s_rr[w] = rr; s_bb[w] = bb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tb = 0.0;
    for (int k = 0; k < NA_THREADS / 32; ++k) { tr += s_rr[k]; tb += s_bb[k]; }
    *rel_out = tb > 0.0 ? sqrt(tr) / sqrt(tb) : 0.0;
    *ticket = 0u;
  }
}

// Device address of g_noalloc_scratch on the current device, which must be the context's.  It is
// looked up with that device current on every call made outside a stream capture (cheap, and
// correct again after a device reset reloads the module) and cached per device for calls made
// while `st` is being captured, where the cached value from an earlier call is used.
static std::mutex g_na_mutex;
static double* g_na_ptr[64] = {};

static helm_status scratch_for_context_device(const helm_ctx* c, cudaStream_t st, double** out) {
  int dev = 0;
  HELM_CUDA(cudaGetDevice(&dev));
  if (dev != c->dev) {
    set_error("helm_residual_noalloc: the current device is not the context's device");
    return HELM_ERR_ARG;
  }
  if (dev < 0 || dev >= 64) { set_error("helm_residual_noalloc: device ordinal >= 64"); return HELM_ERR_ARG; }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  HELM_CUDA(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (cs == cudaStreamCaptureStatusNone || !g_na_ptr[dev]) {
    if (cs != cudaStreamCaptureStatusNone) {
      set_error("helm_residual_noalloc: the first call on a device must come before any stream capture");
      return HELM_ERR_ARG;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return HELM_OK;
}

}  // namespace helm

using namespace helm;

extern "C" helm_status helm_residual_noalloc(helm_ctx* c, const void* b, const void* x, void* r,
                                             double* rel_out, void* stream) {
  if (!c || !b || !x || !r || !rel_out || b == r || x == r) {
    set_error("helm_residual_noalloc: NULL or aliased arguments");
    return HELM_ERR_ARG;
  }
  if (c->n < 1) {
    set_error("helm_residual_noalloc: the context has no unknowns");
    return HELM_ERR_ARG;
  }
  if (c->n > (long)NA_MAX_BLOCKS * NA_POINTS_PER_BLOCK) {
    set_error("helm_residual_noalloc: more than 4194304 unknowns (the size of its static scratch)");
    return HELM_ERR_ARG;
  }
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!al16(b) || !al16(x) || !al16(r) || (reinterpret_cast<uintptr_t>(rel_out) & 7u)) {
    set_error("helm_residual_noalloc: misaligned pointer");
    return HELM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  helm_status s = scratch_for_context_device(c, st, &scratch);
  if (s != HELM_OK) return s;
  // the completion counter must start at zero
  HELM_CUDA(cudaMemsetAsync(scratch + NA_TICKET, 0, sizeof(unsigned int), st));
  int blocks = (int)((c->n + NA_POINTS_PER_BLOCK - 1) / NA_POINTS_PER_BLOCK);
  OpView<double> H = c->H.view<double>();
  const double2* bb = (const double2*)b;
  const double2* xx = (const double2*)x;
  double2* rr = (double2*)r;
  switch (c->grid.dim) {
    case 1: k_residual_noalloc<1><<<blocks, NA_THREADS, 0, st>>>(H, bb, xx, rr, c->n, scratch, rel_out); break;
    case 2: k_residual_noalloc<2><<<blocks, NA_THREADS, 0, st>>>(H, bb, xx, rr, c->n, scratch, rel_out); break;
    default: k_residual_noalloc<3><<<blocks, NA_THREADS, 0, st>>>(H, bb, xx, rr, c->n, scratch, rel_out);
  }
  HELM_CUDA(cudaGetLastError());
  return HELM_OK;
}
