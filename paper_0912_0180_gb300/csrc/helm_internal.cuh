// helm_internal.cuh -- types shared by the translation units of libhelm (device views of
// the operators, the multigrid hierarchy, the Krylov state, complex helpers).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/helm.h"

namespace helm {

// ---- complex arithmetic on float2 / double2 ------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using cx = typename cvec<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mkc(T re, T im) {
  cx<T> z; z.x = re; z.y = im; return z;
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * b + c
template <typename T> __host__ __device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c) {
  return mkc<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) * b
// c - a b, four FMAs
template <typename T> __host__ __device__ __forceinline__ cx<T> cfms(cx<T> a, cx<T> b, cx<T> c) {
  return mkc<T>(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + conj(a) b, four FMAs (the accumulation step of a complex inner product a^H b)
template <typename T> __host__ __device__ __forceinline__ cx<T> cfmac(cx<T> a, cx<T> b, cx<T> c) {
  return mkc<T>(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mkc<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> cscale(T s, cx<T> a) { return mkc<T>(s * a.x, s * a.y); }
template <typename T> __host__ __device__ __forceinline__ T cabs2(cx<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __host__ __device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
  T d = b.x * b.x + b.y * b.y;
  return mkc<T>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <typename T> __host__ __device__ __forceinline__ cx<T> crecip(cx<T> b) {
  T d = b.x * b.x + b.y * b.y;
  return mkc<T>(b.x / d, -b.y / d);
}
template <typename TO, typename TI> __host__ __device__ __forceinline__ cx<TO> cconv(cx<TI> a) {
  return mkc<TO>((TO)a.x, (TO)a.y);
}

// ---- operator view ---------------------------------------------------------------------
// A level operator: per-axis Shortley-Weller rows (am, a0, ap) and sigma = s * phi.
// Uniform interior: on axis a, unknowns ulo[a]..uhi[a] share one row (am = ap = ua[a], a0 equal);
// a point inside all the ranges has the row ud x_P + sum_a ua[a] (x_{P-e_a} + x_{P+e_a}) - s phi x_P,
// evaluated with fewer operations (uniform_real: ua and s real, as for H).
template <typename T> struct OpView {
  int n[3];
  const cx<T>* am[3];
  const cx<T>* a0[3];
  const cx<T>* ap[3];
  const T* phi;   // nullptr -> phi0 everywhere
  T phi0;
  cx<T> s;
  int ulo[3], uhi[3];
  cx<T> ua[3];
  cx<T> ud;
  int uniform_real;
  int uniform_iso;    // every axis has the same uniform coefficient (square interior cells)
  const cx<T>* dinv;  // omega/D (damped Jacobi) or 1/D (Gauss-Seidel) at every point of a
                      // multigrid level; nullptr otherwise
  const cx<T>* dg;    // the diagonal itself (multigrid levels; nullptr otherwise)
  const cx<T>* stg;   // Galerkin level: weight k of unknown p at stg[k * ntot + p], with
                      // k = 3 (dj + 1) + (di + 1) in 2D (9 weights) and k = 9 (dl + 1) + 3 (dj + 1)
                      // + (di + 1) in 3D (27); nullptr for a Shortley-Weller level
  long ntot;
  int somm;           // bit a: the last unknown of axis a is a Sommerfeld boundary node; bit a + 3:
                      // the first one is (a low side)
  double2 bt[3];      // the last node's boundary weight 2i / h_l (the diagonal gains bt * sqrt(phi))
  double2 btl[3];     // the first node's, 2i / h_r
  const double* phim; // imaginary part of phi (k at complex node positions; zero in the uniform
                      // interior) or nullptr
};

// The potential term s * phi of the diagonal at p in FP64, phi complex when phim is given.
inline __host__ __device__ double2 sigma64(const OpView<double>& op, long p, double ph) {
  if (op.phim) return cmul<double>(op.s, mkc<double>(ph, op.phim[p]));
  return cscale<double>(ph, op.s);
}

// Sommerfeld boundary part of the diagonal at (i, j, l) (Section 2, eq. "sommerfeld1", by a
// mirrored ghost node): sum over the axes whose last (or, on a low side, first) unknown this is of
// 2 i k / h, with k = sqrt(phi) the unshifted wave number.  FP64; zero away from such nodes.
template <typename T>
__host__ __device__ inline double2 somm_diag(const OpView<T>& op, int i, int j, int l, double ph) {
  double2 d = {0.0, 0.0};
  if (!op.somm) return d;
  const int idx[3] = {i, j, l};
  for (int a = 0; a < 3; ++a) {
    if (((op.somm >> a) & 1) && idx[a] == op.n[a] - 1) {
      const double k = sqrt(ph);
      d.x += op.bt[a].x * k;
      d.y += op.bt[a].y * k;
    }
    if (((op.somm >> (a + 3)) & 1) && idx[a] == 0) {
      const double k = sqrt(ph);
      d.x += op.btl[a].x * k;
      d.y += op.btl[a].y * k;
    }
  }
  return d;
}

// Unknowns along one axis: interior nodes minus Dirichlet walls, plus m + 1 per ECS layer of m
// nodes, plus the boundary node of each Sommerfeld side (-1).
inline long axis_unknowns(int n_int, int lo, int hi) {
  return (long)n_int - 2 + (lo > 0 ? lo + 1 : (lo < 0 ? 1 : 0)) + (hi > 0 ? hi + 1 : (hi < 0 ? 1 : 0));
}

// ---- owned device storage of one level ---------------------------------------------------
struct LevelHost {
  int dim = 0;
  int n[3] = {1, 1, 1};
  long ntot = 0;
  // FP64 tables (always), FP32 copies (MG in FP32)
  double2* gap[3] = {nullptr, nullptr, nullptr};   // n+1 widths
  double* pos[3] = {nullptr, nullptr, nullptr};    // n real positions
  double2* coef64[3][3] = {};                      // [axis][am,a0,ap]
  float2* coef32[3][3] = {};
  double* phi64 = nullptr;   // nullptr when constant
  float* phi32 = nullptr;
  double phi0 = 0.0;
  double2 s = {1.0, 0.0};
  // uniform interior (see OpView), found at setup from the FP64 tables
  int ulo[3] = {1, 1, 1}, uhi[3] = {0, 0, 0};
  double2 ua[3] = {};
  double2 ud = {0.0, 0.0};
  // reciprocal of the diagonal, multigrid precision (multigrid levels only)
  double2* dinv64 = nullptr;
  float2* dinv32 = nullptr;
  double2* dg64 = nullptr;   // the diagonal itself, same precision
  float2* dg32 = nullptr;
  // Galerkin coarse operator (9-point in 2D, 27-point in 3D), [9 or 27][ntot]; FP64 always, FP32
  // copy for FP32 multigrid
  double2* stg64 = nullptr;
  float2* stg32 = nullptr;
  // ILU(0) factors (ILU smoothing, 1D / 2D levels above the coarsest), [ntot][9]: L at the slots
  // of the lower neighbours, U at the upper neighbours and the reciprocal of U's pivot at the
  // point's own slot; FP64 always, FP32 copy for FP32 multigrid
  double2* ilu64 = nullptr;
  float2* ilu32 = nullptr;
  // Sommerfeld sides: bit a set when the last unknown of axis a is the boundary node, bit a + 3 when
  // the first one is (a low side: that axis coarsens with offset 0, keeping node 0)
  int somm = 0;
  double2 bt[3] = {};
  double2 btl[3] = {};
  // coarsening offset of axis a: coarse unknown c is fine unknown 2c + offset(a)
  int offset(int a) const { return ((somm >> (a + 3)) & 1) ? 0 : 1; }
  bool any_offset0() const { return (somm >> 3) != 0; }
  double* phim64 = nullptr;  // imaginary part of phi (FP64), nullptr when phi is real
  // fused 2D kernel tiles picked by the autotuner: 1 large, 0 small, 2 one warp, 3 square, -1 by the
  // block-count rule
  int tile_down = -1, tile_up = -1;
  // x-split storage (FP32 red-black levels of a 3D hierarchy above the coarsest and the one-block
  // tail): u, f, the spare vector and dinv32 store each row's even x indices first, then the odd
  // ones, so that a half-sweep reads only its own colour's sectors.  phi32 and dg32 stay natural.
  int xs = 0;
  int xs_half() const { return xs ? (n[0] + 1) / 2 : 0; }
  // work vectors (MG type), allocated for multigrid levels
  void* u = nullptr;
  void* f = nullptr;
  void* w = nullptr;

  template <typename T> OpView<T> view() const;
};

struct KrylovState;  // device-side scalars, defined in krylov.cu

// One device allocation and the release function of the allocator that made it (free == nullptr:
// cudaMallocAsync, released by cudaFreeAsync; otherwise the allocator registered with
// helm_set_allocator when the block was allocated).
struct DevBlock {
  void* p = nullptr;
  void (*free)(void*, void*, void*) = nullptr;
  void* user = nullptr;
};

struct Workspace;    // Krylov vectors, defined in krylov.cu

}  // namespace helm

// Separable exact solve of the coarsest level (see coarse_fdm.cu): per axis the eigenvector
// matrices V_a and V_a^{-1} (n_a x n_a, row-major) and the pointwise 1 / (eigenvalue sums), in the
// V-cycle precision, and two scratch vectors of the level's size.
struct FdmCoarse {
  bool on = false;
  int dim = 0;
  int n[3] = {1, 1, 1};
  void* V[3] = {nullptr, nullptr, nullptr};
  void* Vi[3] = {nullptr, nullptr, nullptr};
  void* dinv = nullptr;
  void* scr = nullptr;
};

struct helm_ctx {
  helm_grid grid{};
  helm_precond pc{};
  int dev = 0;
  long n = 0;
  helm::LevelHost H;                 // the FP64 Helmholtz operator
  std::vector<helm::LevelHost> lv;   // preconditioner hierarchy
  void* coarse_inv = nullptr;        // dense inverse of the coarsest M (mg dtype)
  int nco = 0;
  size_t bytes = 0;                  // device bytes held
  std::vector<helm::DevBlock> allocs;  // everything to free
  helm::Workspace* ws = nullptr;     // Krylov workspace (lazily created)
  void* scratch = nullptr;           // FP32 hierarchies: 2N complex64, the unfused V-cycle's level-0
                                     // output before widening, then helm_vcycle's converted input
  cudaStream_t alloc_stream = nullptr;  // stream of the stream-ordered allocations of helm_create
  int tail_first = 1 << 30;          // first level run by the single-block tail kernel
  FdmCoarse fdm;                     // separable coarsest solve (constant phi there), or off
  int* field_bad = nullptr;          // set by helm_create when a device k field has a non-finite entry
};

namespace helm {

// error bookkeeping (per thread)
void set_error(const std::string& msg);
helm_status cuda_check(cudaError_t e, const char* what);
inline helm_status cuda_err(cudaError_t e) { return e == cudaSuccess ? HELM_OK : cuda_check(e, "CUDA call"); }
#define HELM_CUDA(call)                                            \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess) return ::helm::cuda_check(_e, #call);   \
  } while (0)

// Device memory through the allocator registered with helm_set_allocator (default: stream-ordered
// cudaMallocAsync on `st`).  HELM_ERR_OOM (and *p = nullptr) when it fails.  dev_free releases one
// block; dev_free_all a list, after `st` has finished its queued work when any block came from a
// registered allocator (whose release is immediate), else stream-ordered.
helm_status dev_alloc(void** p, size_t bytes, cudaStream_t st, DevBlock* rec);
void dev_free(const DevBlock& b, cudaStream_t st);
void dev_free_all(std::vector<DevBlock>& v, cudaStream_t st);
// device allocation owned by the context (on the context's creation stream)
helm_status ctx_alloc(helm_ctx* c, void** p, size_t bytes);

// ILU(0) smoothing (ilu.cu).  ilu_check: whether a level of this shape can take it (1D / 2D, the
// row ring within one block's shared memory); ilu_build: the factors of level L, at create;
// ilu_solve: u += (L U)^{-1} in (u = (L U)^{-1} in when zero), y a level-sized buffer (may be in).
constexpr size_t ILU_SMEM_MAX = 227 * 1024;
helm_status ilu_check(int dim, const int n[3], bool f32);
helm_status ilu_build(helm_ctx* c, LevelHost& L, bool f32, cudaStream_t st);
template <typename T>
void ilu_solve(const LevelHost& L, const cx<T>* in, cx<T>* y, cx<T>* u, bool zero, const int* skip, cudaStream_t st);
// releases a context: every buffer is freed in order on `st` after the work already queued there
// (no device-wide synchronisation); the caller guarantees all its work was queued on `st`
void ctx_release_on(helm_ctx* c, cudaStream_t st);
// pinned host buffers for the per-solve statistics, recycled (freeing pinned memory may
// synchronise the device)
void* pinned_slot_get(size_t bytes);
void pinned_slot_put(void* p);

// setup.cu
helm_status build_operator(helm_ctx* c, const helm_kspec* k, cudaStream_t st);
helm_status build_hierarchy(helm_ctx* c, cudaStream_t st);

// mg.cu
// z = V-cycle(f0); u0 is cx<T> or, with u0_f64, complex128 (the multigrid result widened in the
// kernel that writes it -- the precision boundary into the FP64 Krylov vectors)
template <typename T>
helm_status mg_vcycle(helm_ctx* c, const cx<T>* f0, void* u0, bool u0_f64, const int* skip, cudaStream_t st);
helm_status mg_level_op(helm_ctx* c, int op, int lvl, void* a, const void* b, void* out, int count,
                        cudaStream_t st);
// y = H x (FP64 arithmetic); x of type TX; optional fused partial inner products handled in krylov.cu
helm_status h_apply(helm_ctx* c, bool x_is_f32, const void* x, double2* y, cudaStream_t st);
helm_status convert_c128_to_mg(helm_ctx* c, const double2* in, void* out, cudaStream_t st);
// the same in level 0's storage order (the V-cycle's input)
helm_status mg_input_from_c128(helm_ctx* c, const double2* in, void* out, cudaStream_t st);
// out = in (natural order, complex64) with level L's rows x-split
helm_status xs_permute_c64(const LevelHost& L, const float2* in, float2* out, cudaStream_t st);

// mg_fused.cu
helm_status autotune_tiles(helm_ctx* c, cudaStream_t st);
// ---- grouped launches: compacted work lists ------------------------------------------------------
// A grouped launch runs one block per virtual block of its work list (blocks past the running
// instances' total return at once; group_visit also serves smaller grids that stride): while
// instance inst[d] is running, descriptor d of the launch owns the virtual blocks
// [first[d], first[d] + nb[d]) and map[w] = d for each of them; once it has finished its range is
// empty.  Each virtual block does exactly what one block of the instance's own launch does.
struct GroupList {
  int nd;            // descriptors
  const int* inst;   // instance of each descriptor
  const int* nb;     // virtual blocks of each descriptor
  int* first;        // nd + 1 entries; first[nd] = the running total
  int* map;          // virtual block -> descriptor (capacity: sum of nb)
};

// The visiting loop of a grouped kernel: fn(d, vb) for every virtual block w = blockIdx.x,
// blockIdx.x + gridDim.x, ... of the list, vb being w's index within descriptor d.
template <typename F>
__device__ __forceinline__ void group_visit(const GroupList& L, F&& fn) {
  const int total = L.first[L.nd];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int d = L.map[w];
    fn(d, w - L.first[d]);
    __syncthreads();  // the next virtual block reuses the shared memory
  }
}

// Host registry of a grouped solve's work lists (group.cu).  add() records a list's descriptors
// (their instances and block counts) and returns its index; upload() puts every list into one
// device table, compacted over all instances (the device re-compacts them when instances finish).
struct GroupLists {
  std::vector<std::vector<int>> inst, nb;
  std::vector<GroupList> host;
  GroupList* dev = nullptr;
  int* listed = nullptr;   // per instance: 1 while the lists include it
  int* changed = nullptr;  // set when an instance's state differs from `listed`
  std::vector<DevBlock> mem;
  int add(const std::vector<int>& in, const std::vector<int>& nbl) {
    inst.push_back(in);
    nb.push_back(nbl);
    return (int)inst.size() - 1;
  }
  int capacity(int li) const {
    int t = 0;
    for (int v : nb[li]) t += v;
    return t;
  }
  helm_status upload(int ninst, cudaStream_t st);
};

// Grouped V-cycles (mg_fused.cu): the V-cycles of ni contexts (2D, fused V(1,1) levels, dense
// coarsest inverse, one smoother kind, multigrid precision T) enqueued as one launch per level and
// kernel kind.  in[i] (cx<T>) is instance i's right-hand side, out[i] its complex128 result,
// skip[i] its skip flag; the plan keeps device descriptors until group_vcycle_free.
struct GroupVcycle;
template <typename T>
helm_status group_vcycle_build(helm_ctx* const* cs, int ni, const void* const* in, double2* const* out,
                               const int* const* skip, GroupLists* lists, cudaStream_t st, GroupVcycle** plan);
// after lists->upload(): the persistent grid of every launch and the device table of the lists
template <typename T> helm_status group_vcycle_finalize(GroupVcycle* plan, const GroupLists* lists);
template <typename T> void group_vcycle_enqueue(const GroupVcycle* plan, cudaStream_t st);
long group_vcycle_launches(const GroupVcycle* plan);
void group_vcycle_free(GroupVcycle* plan, cudaStream_t st);
// coarse_fdm.cu
helm_status fdm_build(helm_ctx* c, const LevelHost& L, bool f32, cudaStream_t st);
template <typename T>
void fdm_apply(const helm_ctx* c, const cx<T>* f, cx<T>* z, const int* skip, cudaStream_t st);
template <typename T> int tail_first_level(const helm_ctx* c);
template <typename T>
helm_status tail_vcycle(helm_ctx* c, int first, const cx<T>* f, void* out, bool out_f64, const int* skip,
                        cudaStream_t st);
template <typename T>
void fused_down2d(const helm_ctx* c, int l, const cx<T>* f, cx<T>* u_out, cx<T>* fc, const int* skip, cudaStream_t st);
template <typename T>
void fused_up2d(const helm_ctx* c, int l, const cx<T>* u_in, const cx<T>* ec, const cx<T>* f, void* out,
                bool out_f64, const int* skip, cudaStream_t st);

// krylov.cu
helm_status krylov_solve(helm_ctx* c, const double2* b, double2* x, const helm_solve_opts* o,
                         helm_solve_info* info, cudaStream_t st);
helm_status krylov_solve_batch(helm_ctx* const* cs, const double2* const* b, double2* const* x, int n,
                               const helm_solve_opts* o, helm_solve_info* infos, cudaStream_t user);
// grouped Bi-CGSTAB (group.cu): arguments already checked per instance
helm_status krylov_solve_group(helm_ctx* const* cs, const double2* const* b, double2* const* x, int n,
                               const helm_solve_opts* o, helm_solve_info* infos, cudaStream_t st);
// resumable solves (used by the batch and the server)
struct SolveJob;
void krylov_free(helm_ctx* c, cudaStream_t st);

// Programmatic dependent launch: kernels on the solve path are launched so that the next kernel's
// blocks may be scheduled as the previous one's blocks exit; every such kernel starts with
// pdl_entry(), which waits for the previous kernel's completion and memory (griddepcontrol.wait)
// before anything is read.  No kernel triggers its dependents earlier (launch_dependents): the
// next grid's blocks would then sit resident at their wait while this kernel runs, and the
// resources they hold cost more than the launch latency they hide (measured: every workload
// slower, the 3D FP32 path by a third).  A kernel launched without the attribute passes the wait
// at once.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// process-wide switch read by launch_pdl (set per call chain by the entry points)
extern thread_local bool g_use_pdl;

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  if (!g_use_pdl) {
    kernel<<<grid, block, smem, st>>>(static_cast<KArgs>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline int grid_blocks(long work, int threads, int cap) {
  long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace helm
