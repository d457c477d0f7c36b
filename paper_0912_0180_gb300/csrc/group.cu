// group.cu -- helm_solve_group: right-preconditioned Bi-CGSTAB (Section 6.2) on many independent
// instances at once, with every kernel of an iteration issued as ONE launch over all instances'
// blocks (the grouped kernels of krylov.cu and mg_fused.cu).  The instances run in lockstep inside
// one captured loop graph whose WHILE node runs while any of them is still iterating; an instance
// that has finished skips each later launch with one flag read per block.  Each instance keeps
// its own operator, hierarchy, workspace, scalars and block decomposition, so its iterates,
// statistics and solution are bitwise those it gets from helm_solve alone.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "krylov_state.cuh"

namespace helm {

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct GroupRun {
  std::vector<DevBlock> mem;
  GroupVcycle* vp = nullptr;  // V-cycle on p (or its FP32 copy) -> p^
  GroupVcycle* vs = nullptr;  // V-cycle on s (or its FP32 copy) -> s^
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t body_nodes = 0;
  cudaStream_t st = nullptr;
  ~GroupRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    group_vcycle_free(vp, st);
    group_vcycle_free(vs, st);
    dev_free_all(mem, st);
  }
};

// Whether a context can join a group, and the reason when not.
const char* group_refusal(const helm_ctx* c, const helm_ctx* c0, int dev) {
  if (c->dev != dev) return "a context belongs to another device";
  if (c->grid.dim != 2) return "grouped solves take 2D grids";
  if (c->pc.kind == HELM_PC_NONE) return "grouped solves need a multigrid preconditioner";
  if (c->pc.nu1 != 1 || c->pc.nu2 != 1) return "grouped solves run V(1,1) cycles";
  if (c->pc.flags & (HELM_PF_UNFUSED | HELM_PF_GALERKIN)) return "grouped solves need the fused rediscretised levels";
  if (c->fdm.on) return "grouped solves need a dense coarsest inverse";
  if (!c->lv.empty() && c->lv[0].any_offset0()) return "grouped solves do not take Sommerfeld low sides";
  if ((int)c->lv.size() < 2 && c->tail_first > 0) return "grouped solves need at least two levels";
  if (c->pc.smoother != c0->pc.smoother) return "the instances of a group share one smoother kind";
  if (c->pc.mg_dtype != c0->pc.mg_dtype) return "the instances of a group share one multigrid precision";
  return nullptr;
}

template <typename TM>
helm_status group_solve_t(helm_ctx* const* cs, const double2* const* b, double2* const* x, int ni,
                          const helm_solve_opts* o, helm_solve_info* infos, cudaStream_t st) {
  const double t0 = now_s();
  GroupRun R;
  R.st = st;
  helm_status s;
  for (int i = 0; i < ni; ++i)
    if ((s = group_member_begin(cs[i], o, st)) != HELM_OK) return s;
  const bool f32 = std::is_same<TM, float>::value;
  std::vector<GroupBicg> A(ni);
  std::vector<const void*> inp(ni), ins(ni);
  std::vector<double2*> outp(ni), outs(ni);
  std::vector<const int*> skip(ni);
  int blocks = 0;
  for (int i = 0; i < ni; ++i) {
    const helm_ctx* c = cs[i];
    Workspace* w = c->ws;
    A[i] = GroupBicg{w->st, c->H.view<double>(), w->x, w->r, w->rh, w->p, w->v, w->sv, w->t, w->ph, w->sh,
                     f32 ? w->pmg : nullptr, f32 ? w->smg : nullptr, c->n, w->partials, w->G, blocks};
    blocks += w->G;
    inp[i] = f32 ? (const void*)w->pmg : (const void*)w->p;
    ins[i] = f32 ? (const void*)w->smg : (const void*)w->sv;
    outp[i] = w->ph;
    outs[i] = w->sh;
    skip[i] = &w->st->done;
  }
  GroupBicg* dA = nullptr;
  int* loops = nullptr;
  {
    DevBlock b1, b2;
    if ((s = dev_alloc((void**)&dA, sizeof(GroupBicg) * ni, st, &b1)) != HELM_OK) return s;
    R.mem.push_back(b1);
    if ((s = dev_alloc((void**)&loops, sizeof(int), st, &b2)) != HELM_OK) return s;
    R.mem.push_back(b2);
  }
  HELM_CUDA(cudaMemcpyAsync(dA, A.data(), sizeof(GroupBicg) * ni, cudaMemcpyHostToDevice, st));
  if ((s = group_vcycle_build<TM>(cs, ni, inp.data(), outp.data(), skip.data(), st, &R.vp)) != HELM_OK) return s;
  if ((s = group_vcycle_build<TM>(cs, ni, ins.data(), outs.data(), skip.data(), st, &R.vs)) != HELM_OK) return s;

  // the loop graph: [condition from the instances' states] -> WHILE(any running) { one iteration }
  const int cap = o->maxmv + 16;
  HELM_CUDA(cudaGraphCreate(&R.graph, 0));
  cudaGraphConditionalHandle h;
  HELM_CUDA(cudaGraphConditionalHandleCreate(&h, R.graph, 0, 0));
  cudaStream_t cs0;
  HELM_CUDA(cudaStreamCreateWithFlags(&cs0, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs0, R.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaStreamBeginCaptureToGraph(group)"); }
  group_cond_launch(h, dA, ni, loops, cap, 0, cs0);
  cudaGraph_t dummy = nullptr;
  e = cudaStreamEndCapture(cs0, &dummy);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaStreamEndCapture(group head)"); }
  size_t nh = 0;
  cudaGraphGetNodes(R.graph, nullptr, &nh);
  std::vector<cudaGraphNode_t> heads(nh);
  cudaGraphGetNodes(R.graph, heads.data(), &nh);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t cn;
  e = cudaGraphAddNode(&cn, R.graph, heads.data(), nullptr, nh, &np);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaGraphAddNode(group WHILE)"); }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cs0, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaStreamBeginCaptureToGraph(group body)"); }
  group_krylov_launch<TM>(GK_P, dA, ni, blocks, cs0);
  group_vcycle_enqueue<TM>(R.vp, cs0);
  group_krylov_launch<TM>(GK_V, dA, ni, blocks, cs0);
  group_krylov_launch<TM>(GK_S, dA, ni, blocks, cs0);
  group_krylov_launch<TM>(GK_XHALF, dA, ni, blocks, cs0);
  group_vcycle_enqueue<TM>(R.vs, cs0);
  group_krylov_launch<TM>(GK_T, dA, ni, blocks, cs0);
  group_krylov_launch<TM>(GK_XR, dA, ni, blocks, cs0);
  group_cond_launch(h, dA, ni, loops, cap, 1, cs0);
  cudaGraph_t bout = nullptr;
  e = cudaStreamEndCapture(cs0, &bout);
  cudaStreamDestroy(cs0);
  if (e != cudaSuccess) return cuda_check(e, "cudaStreamEndCapture(group body)");
  cudaGraphGetNodes(body, nullptr, &R.body_nodes);
  HELM_CUDA(cudaGraphInstantiate(&R.exec, R.graph, 0));

  // passes: start (or restart) the instances that need it, run the loop, certify by the FP64 true
  // residual; an instance whose recurrence met tol while its true residual did not restarts
  std::vector<int> restarts(ni, 0);
  std::vector<char> run(ni, 1);
  long kernels = 0;
  bool first = true;
  for (;;) {
    for (int i = 0; i < ni; ++i)
      if (run[i]) group_member_start(cs[i], b[i], first, st);
    HELM_CUDA(cudaMemsetAsync(loops, 0, sizeof(int), st));
    HELM_CUDA(cudaGraphLaunch(R.exec, st));
    for (int i = 0; i < ni; ++i)
      if (run[i]) group_member_true_res(cs[i], b[i], st);
    int hl = 0;
    HELM_CUDA(cudaMemcpyAsync(&hl, loops, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CUDA(cudaStreamSynchronize(st));
    int nrun = 0;
    for (int i = 0; i < ni; ++i) nrun += run[i];
    kernels += 1 + (long)hl * (long)R.body_nodes + 2L * nrun;
    first = false;
    bool more = false;
    for (int i = 0; i < ni; ++i) {
      const KrylovState& hs = *cs[i]->ws->hst;
      run[i] = 0;
      if (hs.status == HELM_OK && !(hs.rel_true < o->tol) && restarts[i] < o->max_restarts) {
        ++restarts[i];
        run[i] = 1;
        more = true;
      }
    }
    if (!more) break;
  }
  helm_status result = HELM_OK;
  const double secs = now_s() - t0;
  for (int i = 0; i < ni; ++i) {
    Workspace* w = cs[i]->ws;
    HELM_CUDA(cudaMemcpyAsync(x[i], w->x, sizeof(double2) * cs[i]->n, cudaMemcpyDeviceToDevice, st));
    const KrylovState& hs = *w->hst;
    helm_status fs = (helm_status)hs.status;
    if (fs == HELM_OK && !(hs.rel_true < o->tol)) fs = HELM_ERR_MAXIT;
    if (infos) {
      helm_solve_info& in = infos[i];
      in.status = fs;
      in.iters = hs.iters;
      in.matvecs = hs.matvecs;
      in.restarts = restarts[i];
      in.rel_res_recur = hs.rel_recur;
      in.rel_res_true = hs.rel_true;
      in.kernels = kernels;
      in.vcycles = hs.matvecs;
      in.seconds = secs;
      in.history_len = 0;
    }
    if (result == HELM_OK && fs != HELM_OK) result = fs;
  }
  HELM_CUDA(cudaStreamSynchronize(st));
  return result;
}

}  // namespace

helm_status krylov_solve_group(helm_ctx* const* cs, const double2* const* b, double2* const* x, int ni,
                               const helm_solve_opts* o, helm_solve_info* infos, cudaStream_t st) {
  int dev = 0;
  HELM_CUDA(cudaGetDevice(&dev));
  if (o->method != HELM_BICGSTAB) { set_error("helm_solve_group: the grouped solve runs Bi-CGSTAB"); return HELM_ERR_ARG; }
  if (o->history) { set_error("helm_solve_group: no residual history in a grouped solve"); return HELM_ERR_ARG; }
  for (int i = 0; i < ni; ++i) {
    const char* why = group_refusal(cs[i], cs[0], dev);
    if (why) { set_error(std::string("helm_solve_group: ") + why); return HELM_ERR_ARG; }
  }
  const bool f32 = cs[0]->pc.mg_dtype == HELM_C64;
  return f32 ? group_solve_t<float>(cs, b, x, ni, o, infos, st) : group_solve_t<double>(cs, b, x, ni, o, infos, st);
}

}  // namespace helm
