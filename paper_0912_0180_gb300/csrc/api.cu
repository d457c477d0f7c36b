// api.cu -- the extern "C" entry points declared in include/helm.h: argument validation on
// the host, context lifetime, and dispatch to the setup, multigrid and Krylov code.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "helm_internal.cuh"

namespace helm {

static thread_local std::string g_last_error;
thread_local bool g_use_pdl = true;

// Sets the launch mode of the solve-path kernels for the calls made on this context.
struct PdlScope {
  bool saved;
  explicit PdlScope(const helm_ctx* c) : saved(g_use_pdl) { g_use_pdl = !(c->pc.flags & HELM_PF_NO_PDL); }
  ~PdlScope() { g_use_pdl = saved; }
};

void set_error(const std::string& msg) { g_last_error = msg; }

helm_status cuda_check(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA;
}

// The allocator registered with helm_set_allocator (alloc == nullptr: the CUDA stream-ordered one).
struct Allocator {
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free)(void*, void*, void*) = nullptr;
  void* user = nullptr;
};
static std::mutex g_alloc_mu;
static Allocator g_alloc;

helm_status dev_alloc(void** p, size_t bytes, cudaStream_t st, DevBlock* rec) {
  *p = nullptr;
  *rec = DevBlock{};
  Allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.alloc) {
    void* q = a.alloc(bytes, (void*)st, a.user);
    if (!q) {
      set_error("the registered allocator returned NULL for " + std::to_string(bytes) + " bytes");
      return HELM_ERR_OOM;
    }
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {  // every kernel assumes aligned vectors
      a.free(q, (void*)st, a.user);
      set_error("the registered allocator returned a block that is not 256-byte aligned");
      return HELM_ERR_OOM;
    }
    *p = q;
    *rec = DevBlock{q, a.free, a.user};
    return HELM_OK;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    return HELM_ERR_OOM;
  }
  rec->p = *p;
  return HELM_OK;
}

void dev_free(const DevBlock& b, cudaStream_t st) {
  if (!b.p) return;
  if (b.free) {
    cudaStreamSynchronize(st);
    b.free(b.p, (void*)st, b.user);
  } else {
    cudaFreeAsync(b.p, st);
  }
}

void dev_free_all(std::vector<DevBlock>& v, cudaStream_t st) {
  bool custom = false;
  for (const DevBlock& b : v) custom = custom || (b.p && b.free);
  if (custom) cudaStreamSynchronize(st);
  for (const DevBlock& b : v) {
    if (!b.p) continue;
    if (b.free) b.free(b.p, (void*)st, b.user);
    else cudaFreeAsync(b.p, st);
  }
  v.clear();
}

helm_status ctx_alloc(helm_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HELM_OK;
  DevBlock b;
  helm_status s = dev_alloc(p, bytes, c->alloc_stream, &b);
  if (s != HELM_OK) return s;
  c->allocs.push_back(b);
  c->bytes += bytes;
  return HELM_OK;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static helm_status check_grid(const helm_grid* g) {
  if (!g || g->dim < 1 || g->dim > 3) { set_error("grid.dim must be 1, 2 or 3"); return HELM_ERR_ARG; }
  if (!(g->theta_gamma >= 0.0 && g->theta_gamma < M_PI / 2)) { set_error("theta_gamma out of [0, pi/2)"); return HELM_ERR_ARG; }
  if (g->ecs_ramp < 0 || g->ecs_ramp > (1 << 20)) { set_error("ecs_ramp out of [0, 2^20]"); return HELM_ERR_ARG; }
  long total = 1;
  for (int a = 0; a < g->dim; ++a) {
    int lo = g->n_layer[a][0], hi = g->n_layer[a][1];
    if (lo < -1 || hi < -1 || g->n_int[a] < 2 || !(g->extent[a] > 0.0) || !std::isfinite(g->extent[a])) {
      set_error("invalid n_int / n_layer / extent (every side >= -1)");
      return HELM_ERR_ARG;
    }
    long n = axis_unknowns(g->n_int[a], lo, hi);
    if (n < 1 || n > 65535) { set_error("an axis has no unknowns or more than 65535"); return HELM_ERR_ARG; }
    total *= n;
    if (total > (1L << 34)) { set_error("grid too large"); return HELM_ERR_ARG; }
  }
  return HELM_OK;
}

static helm_status check_precond(const helm_precond* p) {
  if (!p) { set_error("precond is NULL"); return HELM_ERR_ARG; }
  if (p->kind < HELM_PC_NONE || p->kind > HELM_PC_CSG_INTERIOR) { set_error("precond.kind"); return HELM_ERR_ARG; }
  if (p->kind == HELM_PC_NONE) return HELM_OK;
  if (p->nu1 < 0 || p->nu1 > 8 || p->nu2 < 0 || p->nu2 > 8) { set_error("nu1/nu2 must be in 0..8"); return HELM_ERR_ARG; }
  if (p->smoother != HELM_SM_JACOBI && p->smoother != HELM_SM_RBGS && p->smoother != HELM_SM_ILU) { set_error("smoother"); return HELM_ERR_ARG; }
  if (p->smoother == HELM_SM_JACOBI && !(p->omega > 0.0 && p->omega <= 1.0)) { set_error("omega must be in (0, 1]"); return HELM_ERR_ARG; }
  if (p->max_levels < 1 || p->max_levels > 32) { set_error("max_levels must be in 1..32"); return HELM_ERR_ARG; }
  if (p->coarse_max < 1) { set_error("coarse_max must be >= 1"); return HELM_ERR_ARG; }
  if (p->mg_dtype != HELM_C64 && p->mg_dtype != HELM_C128) { set_error("mg_dtype"); return HELM_ERR_ARG; }
  if (p->flags & ~(HELM_PF_UNFUSED | HELM_PF_NO_PDL | HELM_PF_NO_AUTOTUNE | HELM_PF_GALERKIN)) { set_error("unknown precond.flags bits"); return HELM_ERR_ARG; }
  if ((p->flags & HELM_PF_GALERKIN) && p->smoother == HELM_SM_RBGS) {
    set_error("Galerkin coarse operators need the damped-Jacobi or the ILU(0) smoother");
    return HELM_ERR_ARG;
  }
  if (!std::isfinite(p->theta_beta) || !std::isfinite(p->shift_re) || !std::isfinite(p->shift_im)) {
    set_error("non-finite preconditioner parameter");
    return HELM_ERR_ARG;
  }
  return HELM_OK;
}

void ctx_release_on(helm_ctx* c, cudaStream_t st) {
  if (!c) return;
  krylov_free(c, st);
  dev_free_all(c->allocs, st);
  delete c;
}

// helm_destroy: the context may have been used on any stream, so wait for the device first.
static void ctx_release(helm_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  ctx_release_on(c, (cudaStream_t)0);
  cudaStreamSynchronize((cudaStream_t)0);
}

static std::mutex g_pinned_mu;
static std::vector<void*> g_pinned_free;

void* pinned_slot_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    if (!g_pinned_free.empty()) {
      void* p = g_pinned_free.back();
      g_pinned_free.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes < 4096 ? 4096 : bytes) != cudaSuccess) return nullptr;
  return p;
}

void pinned_slot_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.push_back(p);
}

}  // namespace helm

using namespace helm;

extern "C" {

helm_status helm_create(const helm_grid* grid, const helm_kspec* k, const helm_precond* pc, void* stream,
                        helm_ctx** out) {
  if (!out) { set_error("out is NULL"); return HELM_ERR_ARG; }
  *out = nullptr;
  helm_status s;
  if ((s = check_grid(grid)) != HELM_OK) return s;
  if ((s = check_precond(pc)) != HELM_OK) return s;
  if ((pc->flags & HELM_PF_GALERKIN) && pc->kind != HELM_PC_NONE && grid->dim < 2) {
    set_error("Galerkin coarse operators need a 2D or 3D grid");
    return HELM_ERR_ARG;
  }
  if (pc->smoother == HELM_SM_ILU && pc->kind != HELM_PC_NONE && grid->dim > 2) {
    set_error("ILU(0) smoothing runs on 1D and 2D levels");
    return HELM_ERR_ARG;
  }
  if (!k || !std::isfinite(k->k0)) { set_error("kspec missing or k0 not finite"); return HELM_ERR_ARG; }
  helm_ctx* c = new helm_ctx();
  c->grid = *grid;
  c->pc = *pc;
  for (int a = grid->dim; a < 3; ++a) {
    c->grid.n_int[a] = 3;
    c->grid.n_layer[a][0] = c->grid.n_layer[a][1] = 0;
    c->grid.extent[a] = 1.0;
  }
  cudaGetDevice(&c->dev);
  cudaStream_t st = (cudaStream_t)stream;
  c->alloc_stream = st;
  bool somm = false;
  bool somm_lo = false;
  for (int a = 0; a < grid->dim; ++a) {
    somm = somm || grid->n_layer[a][1] < 0 || grid->n_layer[a][0] < 0;
    somm_lo = somm_lo || grid->n_layer[a][0] < 0;
  }
  if (somm_lo && (pc->flags & HELM_PF_GALERKIN) && pc->kind != HELM_PC_NONE) {
    delete c;
    set_error("Galerkin coarse operators are not built for a grid with a Sommerfeld low side");
    return HELM_ERR_ARG;
  }
  if (k->phi_im && !k->phi) { delete c; set_error("phi_im needs phi"); return HELM_ERR_ARG; }
  if (!k->phi) {
    bool ok = k->kind == HELM_K_CONST ||
              (k->kind == HELM_K_GAUSS_BUMP && k->width2 > 0.0 && std::isfinite(k->width2) &&
               std::isfinite(k->amp) && std::isfinite(k->centre[0]) && std::isfinite(k->centre[1]) &&
               std::isfinite(k->centre[2])) ||
              (k->kind == HELM_K_FIELD && k->field && aligned(k->field, 8));
    if (!ok) {
      delete c;
      set_error("kspec: kind must be HELM_K_CONST, HELM_K_GAUSS_BUMP (finite amp and centre, width2 > 0) or "
                "HELM_K_FIELD (an 8-byte aligned device field)");
      return HELM_ERR_ARG;
    }
  }
  if (k->phi) {
    long n = 1;
    for (int a = 0; a < grid->dim; ++a) n *= axis_unknowns(grid->n_int[a], grid->n_layer[a][0], grid->n_layer[a][1]);
    for (long i = 0; i < n; ++i) {
      if (k->phi_im && !std::isfinite(k->phi_im[i])) { delete c; set_error("phi_im has a non-finite entry"); return HELM_ERR_ARG; }
      if (!std::isfinite(k->phi[i])) { delete c; set_error("phi has a non-finite entry"); return HELM_ERR_ARG; }
      // a Sommerfeld boundary needs the real wave number k = sqrt(phi)
      if (somm && k->phi[i] < 0.0) { delete c; set_error("phi < 0 with a Sommerfeld side"); return HELM_ERR_ARG; }
    }
  }
  if ((s = build_operator(c, k, st)) != HELM_OK) { ctx_release(c); return s; }
  if ((s = build_hierarchy(c, st)) != HELM_OK) { ctx_release(c); return s; }
  if (pc->kind != HELM_PC_NONE && pc->mg_dtype == HELM_C64) {
    // two vectors: the V-cycle's level-0 output before widening, and helm_vcycle's converted input
    if ((s = ctx_alloc(c, &c->scratch, 2 * sizeof(float2) * c->n)) != HELM_OK) { ctx_release(c); return s; }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { ctx_release(c); return cuda_check(e, "helm_create"); }
  if (c->field_bad) {
    int bad = 0;
    e = cudaMemcpy(&bad, c->field_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { ctx_release(c); return cuda_check(e, "helm_create"); }
    if (bad) { ctx_release(c); set_error("kspec.field has a non-finite entry"); return HELM_ERR_ARG; }
  }
  *out = c;
  return HELM_OK;
}

long helm_size(const helm_ctx* c) { return c ? c->n : 0; }

size_t helm_workspace_bytes(const helm_ctx* c) { return c ? c->bytes : 0; }

int helm_num_levels(const helm_ctx* c) { return c ? (int)c->lv.size() : 0; }

helm_status helm_level_shape(const helm_ctx* c, int lvl, int* n) {
  if (!c || !n || lvl < 0 || lvl >= (int)c->lv.size()) { set_error("bad level"); return HELM_ERR_ARG; }
  for (int a = 0; a < 3; ++a) n[a] = c->lv[lvl].n[a];
  return HELM_OK;
}

helm_status helm_apply(helm_ctx* c, helm_dtype dtype, const void* x, void* y, void* stream) {
  if (!c || !x || !y || x == y) { set_error("helm_apply: NULL or aliased arguments"); return HELM_ERR_ARG; }
  if (dtype != HELM_C64 && dtype != HELM_C128) { set_error("helm_apply: dtype"); return HELM_ERR_ARG; }
  if (!aligned(x, dtype == HELM_C64 ? 8 : 16) || !aligned(y, 16)) { set_error("helm_apply: misaligned"); return HELM_ERR_ARG; }
  PdlScope pdl(c);
  return h_apply(c, dtype == HELM_C64, x, (double2*)y, (cudaStream_t)stream);
}

// The preconditioner a hierarchy was built for: everything that changes M or the cycle.
static bool same_precond(const helm_precond& a, const helm_precond& b) {
  if (a.kind != b.kind) return false;
  if (a.kind == HELM_PC_NONE) return true;
  if ((a.kind == HELM_PC_CSG_UNIFORM || a.kind == HELM_PC_CSG_INTERIOR) && a.theta_beta != b.theta_beta) return false;
  if (a.kind == HELM_PC_CSL && (a.shift_re != b.shift_re || a.shift_im != b.shift_im)) return false;
  if (a.smoother == HELM_SM_JACOBI && b.smoother == HELM_SM_JACOBI && a.omega != b.omega) return false;
  return a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.smoother == b.smoother && a.max_levels == b.max_levels &&
         a.coarse_max == b.coarse_max && a.mg_dtype == b.mg_dtype &&
         (a.flags & HELM_PF_GALERKIN) == (b.flags & HELM_PF_GALERKIN);
}

helm_status helm_vcycle(helm_ctx* c, const helm_precond* pc, helm_dtype dtype, const void* r, void* z,
                        void* stream) {
  if (!c || !r || !z || r == z) { set_error("helm_vcycle: NULL or aliased arguments"); return HELM_ERR_ARG; }
  if (pc && !same_precond(*pc, c->pc)) {
    set_error("helm_vcycle: the context's hierarchy was built for another preconditioner");
    return HELM_ERR_ARG;
  }
  if (dtype != HELM_C64 && dtype != HELM_C128) { set_error("helm_vcycle: dtype"); return HELM_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  PdlScope pdl(c);
  bool f32 = c->pc.mg_dtype == HELM_C64;
  bool z64 = dtype == HELM_C128;
  if (!aligned(r, 16) || !aligned(z, z64 ? 16 : 8)) { set_error("helm_vcycle: misaligned"); return HELM_ERR_ARG; }
  if (c->pc.kind == HELM_PC_NONE) {
    if (!z64) {
      if (!f32) { set_error("helm_vcycle: complex64 output needs an FP32 context"); return HELM_ERR_ARG; }
      return convert_c128_to_mg(c, (const double2*)r, z, st);
    }
    cudaError_t e = cudaMemcpyAsync(z, r, sizeof(double2) * c->n, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HELM_OK : cuda_check(e, "helm_vcycle copy");
  }
  if (f32) {
    float2* in = (float2*)c->scratch + c->n;  // not the first half: the unfused cycle's output goes there
    helm_status s = mg_input_from_c128(c, (const double2*)r, in, st);
    if (s != HELM_OK) return s;
    return mg_vcycle<float>(c, in, z, z64, nullptr, st);
  }
  if (!z64) { set_error("helm_vcycle: an FP64 hierarchy gives complex128 output"); return HELM_ERR_ARG; }
  return mg_vcycle<double>(c, (const double2*)r, z, false, nullptr, st);
}

helm_status helm_level_op(helm_ctx* c, int op, int lvl, void* a, const void* b, void* out, int count,
                          void* stream) {
  if (!c) { set_error("ctx is NULL"); return HELM_ERR_ARG; }
  PdlScope pdl(c);
  return mg_level_op(c, op, lvl, a, b, out, count, (cudaStream_t)stream);
}

static helm_status check_solve_args(const helm_ctx* c, const void* b, const void* x, const helm_solve_opts* o) {
  if (!c || !b || !x || !o || b == x) { set_error("helm_solve: NULL or aliased arguments"); return HELM_ERR_ARG; }
  if (!aligned(b, 16) || !aligned(x, 16)) { set_error("helm_solve: misaligned"); return HELM_ERR_ARG; }
  if (o->method != HELM_BICGSTAB && o->method != HELM_IDR && o->method != HELM_GMRES) { set_error("method"); return HELM_ERR_ARG; }
  if (o->method == HELM_IDR && (o->s < 1 || o->s > 8 || !o->shadow)) { set_error("IDR needs 1 <= s <= 8 and a shadow array"); return HELM_ERR_ARG; }
  if (o->method == HELM_GMRES && (o->s < 1 || o->s > HELM_GMRES_MAX_M)) { set_error("GMRES needs 1 <= m <= HELM_GMRES_MAX_M"); return HELM_ERR_ARG; }
  if (!(o->tol > 0.0) || o->maxmv < 1 || o->max_restarts < 0) { set_error("tol / maxmv / max_restarts"); return HELM_ERR_ARG; }
  return HELM_OK;
}

helm_status helm_solve_batch(helm_ctx* const* cs, const void* const* b, void* const* x, int n,
                             const helm_solve_opts* o, helm_solve_info* infos, void* stream) {
  if (infos && n > 0) std::memset(infos, 0, sizeof(*infos) * n);
  if (n < 0 || (n > 0 && (!cs || !b || !x || !o))) { set_error("helm_solve_batch: bad arrays"); return HELM_ERR_ARG; }
  for (int i = 0; i < n; ++i) {
    helm_status s = check_solve_args(cs[i], b[i], x[i], &o[i]);
    if (s != HELM_OK) return s;
    for (int j = 0; j < i; ++j)
      if (cs[j] == cs[i]) { set_error("helm_solve_batch: a context appears twice"); return HELM_ERR_ARG; }
  }
  if (n == 0) return HELM_OK;
  PdlScope pdl(cs[0]);
  helm_status s = krylov_solve_batch(cs, (const double2* const*)b, (double2* const*)x, n, o, infos,
                                     (cudaStream_t)stream);
  return s;
}

helm_status helm_solve_group(helm_ctx* const* cs, const void* const* b, void* const* x, int n,
                             const helm_solve_opts* o, helm_solve_info* infos, void* stream) {
  if (infos && n > 0) std::memset(infos, 0, sizeof(*infos) * n);
  if (n < 1 || !cs || !b || !x || !o) { set_error("helm_solve_group: bad arrays"); return HELM_ERR_ARG; }
  for (int i = 0; i < n; ++i) {
    helm_status s = check_solve_args(cs[i], b[i], x[i], o);
    if (s != HELM_OK) return s;
    for (int j = 0; j < i; ++j)
      if (cs[j] == cs[i]) { set_error("helm_solve_group: a context appears twice"); return HELM_ERR_ARG; }
  }
  PdlScope pdl(cs[0]);
  return krylov_solve_group(cs, (const double2* const*)b, (double2* const*)x, n, o, infos, (cudaStream_t)stream);
}

helm_status helm_solve(helm_ctx* c, const void* b, void* x, const helm_solve_opts* o, helm_solve_info* info,
                       void* stream) {
  if (info) std::memset(info, 0, sizeof(*info));
  helm_status cs = check_solve_args(c, b, x, o);
  if (cs != HELM_OK) return cs;
  PdlScope pdl(c);
  helm_status s = krylov_solve(c, (const double2*)b, (double2*)x, o, info, (cudaStream_t)stream);
  if (info) info->status = s;
  return s;
}

void helm_destroy(helm_ctx* c) { ctx_release(c); }

void helm_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_fn)(void*, void*, void*), void* user) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (alloc && free_fn) g_alloc = Allocator{alloc, free_fn, user};
  else g_alloc = Allocator{};
}

const char* helm_status_str(helm_status s) {
  switch (s) {
    case HELM_OK: return "ok";
    case HELM_ERR_ARG: return "invalid argument";
    case HELM_ERR_OOM: return "out of device memory";
    case HELM_ERR_CUDA: return "CUDA error";
    case HELM_ERR_BREAKDOWN: return "Krylov breakdown";
    case HELM_ERR_MAXIT: return "matvec cap reached";
    case HELM_ERR_NAN: return "non-finite value";
    case HELM_ERR_TIMEOUT: return "device wait timed out";
    case HELM_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

const char* helm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
