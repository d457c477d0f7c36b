// server.cu -- a solve server with continuous batching.
//
// Requests (grid, k(x), preconditioner, solve options, right-hand side on the host) are queued by
// helm_server_submit and admitted, in arrival order, as soon as both an execution slot and the
// device-memory budget allow; every admitted request gets its own stream, context and
// device-resident solve, so requests admitted while others run overlap with them on the GPU.  A
// worker thread admits, starts and polls; nothing in its loop synchronises the device (allocations
// and frees are stream-ordered), so a request's completion is noticed as soon as its own stream
// reaches it.  Latency is measured from submission to the moment the solution is in host memory.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <complex>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "helm_internal.cuh"

namespace helm {

struct SolveJob;
helm_status job_begin(SolveJob& j);
helm_status job_poll(SolveJob& j, bool block);
void job_release(SolveJob& j);
SolveJob* job_new();
void job_delete(SolveJob* j);
void job_setup(SolveJob* j, helm_ctx* c, const double2* b, double2* x, const helm_solve_opts* o,
               helm_solve_info* info, cudaStream_t st);
bool job_finished(const SolveJob* j);
helm_status job_status(const SolveJob* j);

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static long axis_n(const helm_grid& g, int a) {
  return axis_unknowns(g.n_int[a], g.n_layer[a][0], g.n_layer[a][1]);
}

}  // namespace helm

using namespace helm;

// Device bytes one request holds while it runs (operator, hierarchy, coarse inverse, Krylov
// workspace, right-hand side and solution), mirroring the allocations of helm_create and of the
// first helm_solve; an upper bound up to the few kilobytes of per-axis tables.
extern "C" size_t helm_estimate_bytes(const helm_grid* g, const helm_precond* pc, const helm_solve_opts* o) {
  if (!g || !pc || !o || g->dim < 1 || g->dim > 3) return 0;
  long n[3] = {1, 1, 1};
  long N = 1;
  for (int a = 0; a < g->dim; ++a) { n[a] = axis_n(*g, a); N *= n[a]; }
  size_t bytes = 0;
  for (int a = 0; a < g->dim; ++a) bytes += (size_t)(n[a] + 1) * 16 * 4;  // H tables
  bytes += (size_t)N * 8 * 2;                                             // phi and its imaginary part
  bytes += (size_t)N * 16;                                                // diagonal of H
  bool pcon = pc->kind != HELM_PC_NONE;
  size_t esz = pcon && pc->mg_dtype == HELM_C64 ? 8 : 16;
  if (pcon) {
    long m[3] = {n[0], n[1], n[2]};
    long Nl = N;
    int levels = 0;
    long last = N;
    for (;;) {
      ++levels;
      for (int a = 0; a < g->dim; ++a) bytes += (size_t)(m[a] + 1) * (16 * 4 + 8 * 3);
      bytes += (size_t)Nl * (8 + 4 + 2 * esz + (levels == 1 ? 1 : 3) * esz);
      if (levels > 1 && (pc->flags & HELM_PF_GALERKIN))  // the stencil, FP64 and the V-cycle precision
        bytes += (size_t)Nl * (g->dim == 3 ? 27 : 9) * (16 + (esz == 8 ? 8 : 0)) + (size_t)Nl * 8;
      if (pc->smoother == HELM_SM_ILU)  // ILU(0) factors, FP64 and the V-cycle precision
        bytes += (size_t)Nl * 9 * (16 + (esz == 8 ? 8 : 0));
      last = Nl;
      bool all_small = true;
      long min_n = 1L << 40;
      for (int a = 0; a < g->dim; ++a) {
        if (m[a] > pc->coarse_max) all_small = false;
        if (m[a] < min_n) min_n = m[a];
      }
      if (levels >= pc->max_levels || all_small || min_n < 3) break;
      Nl = 1;
      for (int a = 0; a < g->dim; ++a) { m[a] /= 2; Nl *= m[a]; }
    }
    bytes += (size_t)last * last * esz;     // coarse inverse
    bytes += (size_t)last * last * 32 + 4;  // its FP64 factorisation (transient)
    if (esz == 8) bytes += (size_t)N * 16;  // the two-vector scratch of an FP32 hierarchy
  }
  // Krylov workspace
  if (o->method == HELM_IDR) bytes += (size_t)N * ((5 + 3 * (size_t)o->s) * 16 + esz);
  else if (o->method == HELM_GMRES) bytes += (size_t)N * ((5 + 1 + (size_t)o->s) * 16 + esz) + (size_t)(o->s + 2) * o->s * 16;
  else bytes += (size_t)N * (9 * 16 + 2 * esz);
  bytes += (size_t)N * 32;  // the request's own b and x on the device
  bytes += 64 * 1024;       // state and partial sums
  return bytes;
}

struct helm_server {
  struct Req {
    uint64_t id = 0;
    helm_grid grid{};
    helm_precond pc{};
    helm_solve_opts opts{};
    double k0 = 0.0;
    std::vector<double> phi, phi_im;
    helm_kspec kform{};  // kind and bump parameters when phi is not given
    std::vector<std::complex<double>> b, shadow;
    void* x_host = nullptr;
    long n = 0;
    size_t bytes = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    int nrhs = 1, cur = 0;      // right-hand sides, the one being solved
    int bypassed = 0;           // times a later request was admitted before this one
    helm_solve_info info{};     // summed over the right-hand sides solved so far
    helm_solve_info one{};      // the current right-hand side
    helm_status status = HELM_OK;
    // running
    helm_ctx* ctx = nullptr;
    void* bd = nullptr;
    void* xd = nullptr;
    std::vector<DevBlock> vecs;  // bd and xd
    SolveJob* job = nullptr;
    int slot = -1;
    cudaStream_t stream = nullptr;  // the slot's stream at this request's priority
    // 0: admitted, waiting for the setup thread; 1: set up (setup_status says how); 2: solving
    std::atomic<int> phase{0};
    helm_status setup_status = HELM_OK;
  };
  size_t budget = 0, used = 0;
  int max_active = 1;
  int policy = HELM_SERVE_FIFO;
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::unordered_map<uint64_t, Req*> reqs;
  // per slot, one stream per priority level (greatest .. least): requests run smallest work first
  std::vector<cudaStream_t> streams;
  int prio_levels = 1, prio_greatest = 0;
  std::vector<bool> slot_busy;
  std::thread worker;
  // helm_create of admitted requests (operator, hierarchy, autotuning) runs on its own thread, so
  // that the worker keeps polling and advancing the running solves meanwhile
  std::thread setup_worker;
  std::deque<Req*> setup_queue;
  std::condition_variable cv_setup;
  bool setup_stop = false;
  bool stop = false;
  uint64_t next_id = 1;
  std::string last_error;

  // Statistics of the right-hand side just finished, folded into the request's: counts add up,
  // residuals take the worst, the status the first failure.
  static void accumulate(Req* r) {
    helm_solve_info& a = r->info;
    const helm_solve_info& o = r->one;
    if (r->cur == 0) a = o;
    else {
      a.iters += o.iters; a.matvecs += o.matvecs; a.restarts += o.restarts; a.kernels += o.kernels;
      a.vcycles += o.vcycles; a.seconds += o.seconds;
      a.history_len = 0;
      if (o.rel_res_recur > a.rel_res_recur) a.rel_res_recur = o.rel_res_recur;
      if (o.rel_res_true > a.rel_res_true) a.rel_res_true = o.rel_res_true;
      if (a.status == HELM_OK) a.status = o.status;
    }
  }

  // Copies the finished right-hand side's solution (or last iterate) to the host and folds its
  // statistics in.
  void collect(Req* r) {
    cudaStream_t s = r->stream;
    cudaMemcpyAsync((double2*)r->x_host + (size_t)r->cur * r->n, r->xd, sizeof(double2) * r->n,
                    cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    accumulate(r);
  }

  // Starts the solve of right-hand side r->cur on the request's context (its hierarchy and
  // Krylov workspace stay resident between right-hand sides).
  helm_status begin_rhs(Req* r) {
    cudaStream_t s = r->stream;
    if (r->job) { job_release(*r->job); job_delete(r->job); r->job = nullptr; }
    size_t vb = sizeof(double2) * r->n;
    if (cudaMemcpyAsync(r->bd, r->b.data() + (size_t)r->cur * r->n, vb, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return HELM_ERR_CUDA;
    r->one = helm_solve_info{};
    r->job = job_new();
    job_setup(r->job, r->ctx, (const double2*)r->bd, (double2*)r->xd, &r->opts, &r->one, s);
    return job_begin(*r->job);
  }

  void finish(Req* r, helm_status st) {
    cudaStream_t s = r->stream;
    if (r->ctx && r->xd && r->job && job_finished(r->job)) collect(r);  // the solution, or the last iterate
    if (r->job) { job_release(*r->job); job_delete(r->job); r->job = nullptr; }
    dev_free_all(r->vecs, s);
    if (r->ctx) ctx_release_on(r->ctx, s);
    r->bd = r->xd = nullptr;
    r->ctx = nullptr;
    r->t_done = now_s();
    std::lock_guard<std::mutex> lk(mu);
    if (r->status == HELM_OK) r->status = st;
    r->info.status = r->status;
    r->state = 2;
    used -= r->bytes;
    if (r->slot >= 0) slot_busy[r->slot] = false;
    active.erase(std::find(active.begin(), active.end(), r));
    cv_done.notify_all();
  }

  // Index in the queue of the request to admit next, or queue.size() if none fits the free
  // budget.  FIFO: the head (a request that does not fit blocks the ones behind it, so admission
  // order is submission order).  SMALLEST_FIRST: a request bypassed 2 x max_active times goes
  // first (no starvation); otherwise the one with the least work (unknowns x right-hand sides)
  // among those that fit, the earliest on ties.
  size_t next_admission() const {
    const size_t none = queue.size();
    if (policy == HELM_SERVE_FIFO) return used + queue.front()->bytes <= budget ? 0 : none;
    for (size_t q = 0; q < queue.size(); ++q)
      if (queue[q]->bypassed >= 2 * max_active) return used + queue[q]->bytes <= budget ? q : none;
    size_t best = none;
    double bw = 0.0;
    for (size_t q = 0; q < queue.size(); ++q) {
      if (used + queue[q]->bytes > budget) continue;
      double w = (double)queue[q]->n * queue[q]->nrhs;
      if (best == none || w < bw) { best = q; bw = w; }
    }
    return best;
  }

  // Priority bucket of a request: one level per decade of unknowns x right-hand sides above 1e4,
  // the smallest work at the greatest priority, so that short requests overtake long ones on the
  // GPU while admission stays first come, first served.
  int prio_level(const Req* r) const {
    double work = (double)r->n * r->nrhs;
    int b = (int)std::floor(std::log10(work > 1.0 ? work : 1.0)) - 4;
    if (b < 0) b = 0;
    if (b > prio_levels - 1) b = prio_levels - 1;
    return b;
  }

  // On the setup thread: the request's context (operator, hierarchy, autotuned tiles) and its b and
  // x vectors, on the request's stream.
  helm_status setup(Req* r) {
    cudaStream_t s = r->stream;
    helm_kspec k = r->kform;
    k.k0 = r->k0;
    k.phi = r->phi.empty() ? nullptr : r->phi.data();
    k.phi_im = r->phi_im.empty() ? nullptr : r->phi_im.data();
    k.field = nullptr;
    helm_status st = helm_create(&r->grid, &k, &r->pc, (void*)s, &r->ctx);
    if (st != HELM_OK) return st;
    size_t vb = sizeof(double2) * r->n;
    r->vecs.assign(2, DevBlock{});
    helm_status ae = dev_alloc(&r->bd, vb, s, &r->vecs[0]);
    if (ae == HELM_OK) ae = dev_alloc(&r->xd, vb, s, &r->vecs[1]);
    if (ae != HELM_OK) return ae;
    if (!r->shadow.empty()) r->opts.shadow = r->shadow.data();
    r->opts.history = nullptr;
    r->opts.host_loop = 0;
    return HELM_OK;
  }

  void setup_run() {
    cudaSetDevice(dev);
    for (;;) {
      Req* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_setup.wait(lk, [this] { return setup_stop || !setup_queue.empty(); });
        if (setup_queue.empty()) return;  // stop requested and nothing left
        r = setup_queue.front();
        setup_queue.pop_front();
      }
      r->setup_status = setup(r);
      r->phase.store(1, std::memory_order_release);
    }
  }

  // On the worker thread, once the setup thread has finished with r: its first right-hand side.
  helm_status start(Req* r) {
    r->t_start = now_s();
    r->cur = 0;
    return begin_rhs(r);
  }

  void run() {
    cudaSetDevice(dev);
    for (;;) {
      std::vector<Req*> to_start;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop && queue.empty() && active.empty()) return;
        while (!queue.empty() && (int)active.size() < max_active) {
          const size_t k = next_admission();
          if (k >= queue.size()) break;  // nothing fits the free budget yet
          Req* r = queue[k];
          for (size_t q = 0; q < k; ++q) queue[q]->bypassed += 1;
          queue.erase(queue.begin() + (long)k);
          for (int i = 0; i < (int)slot_busy.size(); ++i)
            if (!slot_busy[i]) { slot_busy[i] = true; r->slot = i; break; }
          used += r->bytes;
          r->state = 1;
          r->stream = streams[(size_t)r->slot * prio_levels + prio_level(r)];
          active.push_back(r);
          setup_queue.push_back(r);
          to_start.push_back(r);
        }
        if (!to_start.empty()) cv_setup.notify_one();
        if (to_start.empty() && active.empty()) {
          cv_work.wait_for(lk, std::chrono::milliseconds(5));
          continue;
        }
      }
      bool progressed = !to_start.empty();
      std::vector<Req*> snapshot;
      {
        std::lock_guard<std::mutex> lk(mu);
        snapshot = active;
      }
      for (Req* r : snapshot) {
        if (r->phase.load(std::memory_order_acquire) == 1) {  // set up: start its first right-hand side
          r->phase.store(2, std::memory_order_relaxed);
          progressed = true;
          helm_status st = r->setup_status == HELM_OK ? start(r) : r->setup_status;
          if (st != HELM_OK) { finish(r, st); continue; }
        }
        if (!r->job) continue;
        helm_status st = job_poll(*r->job, false);
        if (st == HELM_ERR_BUSY) continue;
        progressed = true;
        if (st != HELM_OK) { finish(r, st); continue; }
        if (!job_finished(r->job)) continue;
        helm_status js = job_status(r->job);
        if (js != HELM_OK || r->cur + 1 >= r->nrhs) { finish(r, js); continue; }
        collect(r);
        r->cur += 1;
        if ((st = begin_rhs(r)) != HELM_OK) finish(r, st);
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
};

extern "C" {

helm_status helm_server_create(size_t budget_bytes, int max_active, helm_server** out) {
  if (!out || max_active < 1 || max_active > 256 || budget_bytes == 0) {
    set_error("helm_server_create: bad arguments");
    return HELM_ERR_ARG;
  }
  helm_server* s = new helm_server();
  s->budget = budget_bytes;
  s->max_active = max_active;
  cudaGetDevice(&s->dev);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  s->prio_levels = least - greatest + 1;
  s->prio_greatest = greatest;
  const int ns = max_active * s->prio_levels;
  s->streams.assign(ns, nullptr);
  s->slot_busy.assign(max_active, false);
  for (int i = 0; i < ns; ++i) {
    int level = i % s->prio_levels;
    cudaError_t e = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, greatest + level);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
      delete s;
      return cuda_check(e, "helm_server_create: stream");
    }
  }
  s->worker = std::thread([s] { s->run(); });
  s->setup_worker = std::thread([s] { s->setup_run(); });
  *out = s;
  return HELM_OK;
}

helm_status helm_server_set_policy(helm_server* s, int policy) {
  if (!s || (policy != HELM_SERVE_FIFO && policy != HELM_SERVE_SMALLEST_FIRST)) {
    set_error("helm_server_set_policy: bad arguments");
    return HELM_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->policy = policy;
  return HELM_OK;
}

helm_status helm_server_submit(helm_server* s, const helm_request* rq, uint64_t* ticket) {
  if (!s || !rq || !ticket || !rq->b || !rq->x) { set_error("helm_server_submit: NULL argument"); return HELM_ERR_ARG; }
  if (rq->grid.dim < 1 || rq->grid.dim > 3) { set_error("helm_server_submit: grid.dim"); return HELM_ERR_ARG; }
  auto* r = new helm_server::Req();
  r->grid = rq->grid;
  r->pc = rq->pc;
  r->opts = rq->opts;
  r->k0 = rq->k.k0;
  if (!rq->k.phi && rq->k.kind == HELM_K_FIELD) {
    delete r;
    set_error("helm_server_submit: a device k field is not accepted (pass phi)");
    return HELM_ERR_ARG;
  }
  r->kform = rq->k;
  r->n = 1;
  for (int a = 0; a < rq->grid.dim; ++a) r->n *= axis_n(rq->grid, a);
  if (r->n < 1) { delete r; set_error("helm_server_submit: empty grid"); return HELM_ERR_ARG; }
  if (rq->k.phi) r->phi.assign(rq->k.phi, rq->k.phi + r->n);
  if (rq->k.phi_im) r->phi_im.assign(rq->k.phi_im, rq->k.phi_im + r->n);
  r->nrhs = rq->nrhs < 1 ? 1 : rq->nrhs;
  if (r->nrhs > HELM_MAX_RHS) { delete r; set_error("helm_server_submit: nrhs"); return HELM_ERR_ARG; }
  const std::complex<double>* b = (const std::complex<double>*)rq->b;
  r->b.assign(b, b + (size_t)r->nrhs * r->n);
  if (rq->opts.method == HELM_IDR) {
    if (!rq->opts.shadow || rq->opts.s < 1 || rq->opts.s > 8) { delete r; set_error("helm_server_submit: IDR shadow"); return HELM_ERR_ARG; }
    const std::complex<double>* sh = (const std::complex<double>*)rq->opts.shadow;
    r->shadow.assign(sh, sh + (size_t)rq->opts.s * r->n);
  }
  r->x_host = rq->x;
  r->bytes = helm_estimate_bytes(&rq->grid, &rq->pc, &rq->opts);
  if (r->bytes > s->budget) {
    delete r;
    set_error("helm_server_submit: the request needs more device memory than the whole budget");
    return HELM_ERR_OOM;
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->id;
  return HELM_OK;
}

helm_status helm_server_poll(helm_server* s, uint64_t ticket, helm_solve_info* info, double* latency_s) {
  if (!s) { set_error("helm_server_poll: NULL server"); return HELM_ERR_ARG; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) { set_error("helm_server_poll: unknown ticket"); return HELM_ERR_ARG; }
  helm_server::Req* r = it->second;
  if (r->state != 2) return HELM_ERR_BUSY;
  if (info) *info = r->info;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  return r->status;
}

helm_status helm_server_wait(helm_server* s, uint64_t ticket, helm_solve_info* info, double* latency_s) {
  if (!s) { set_error("helm_server_wait: NULL server"); return HELM_ERR_ARG; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) { set_error("helm_server_wait: unknown ticket"); return HELM_ERR_ARG; }
  helm_server::Req* r = it->second;
  s->cv_done.wait(lk, [r] { return r->state == 2; });
  if (info) *info = r->info;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  return r->status;
}

helm_status helm_server_stats(helm_server* s, int* queued, int* active, size_t* used_bytes) {
  if (!s) return HELM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->queue.size();
  if (active) *active = (int)s->active.size();
  if (used_bytes) *used_bytes = s->used;
  return HELM_OK;
}

void helm_server_destroy(helm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();  // every admitted request is set up and finished
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->setup_stop = true;
  }
  s->cv_setup.notify_all();
  if (s->setup_worker.joinable()) s->setup_worker.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
