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

// ---- work-list compaction --------------------------------------------------------------------

// The WHILE condition of the grouped loop (any instance running), the instances the work lists
// should hold (`listed`) and whether that changed (`changed`).  At the end of the body it also
// counts the group's bodies and, like the single-instance loop, ends a loop that ran more bodies
// than the matvec cap allows (HELM_ERR_TIMEOUT for the instances still running); an instance that
// ended on a half step had x += alpha p^ applied in this body, and no later body applies it again.
__global__ void kg_cond(cudaGraphConditionalHandle h, const GroupBicg* __restrict__ A, int ni, int* loops,
                        int cap, int in_body, int* listed, int* changed) {
  pdl_entry();
  __shared__ int any, chg;
  if (threadIdx.x == 0) {
    any = 0;
    chg = 0;
    if (in_body) *loops += 1;
  }
  __syncthreads();
  const bool over = in_body && *loops > cap;
  for (int i = threadIdx.x; i < ni; i += blockDim.x) {
    KrylovState* S = A[i].S;
    if (in_body && S->half == 1) S->half = 2;
    if (!S->done && over) {
      S->status = HELM_ERR_TIMEOUT;
      S->done = 1;
    }
    const int run = S->done ? 0 : 1;
    if (run) any = 1;
    if (listed[i] != run) {
      listed[i] = run;
      chg = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *changed = chg;
    cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// first[] of every list from the listed instances (one warp per list, an exclusive scan of the
// descriptors' block counts); nothing to do unless the listed set changed.
__global__ void kg_prefix(GroupList* __restrict__ LT, int nl, const int* __restrict__ listed,
                          const int* __restrict__ changed) {
  pdl_entry();
  if (!*changed) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nl) return;
  const GroupList& L = LT[warp];
  int carry = 0;
  for (int base = 0; base < L.nd; base += 32) {
    const int d = base + lane;
    const int v = (d < L.nd && listed[L.inst[d]]) ? L.nb[d] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (d < L.nd) L.first[d] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) L.first[L.nd] = carry;
}

// map[] of every list: each listed descriptor marks its virtual blocks (blockIdx.y = list).
__global__ void kg_fill(GroupList* __restrict__ LT, int nl, const int* __restrict__ listed,
                        const int* __restrict__ changed) {
  pdl_entry();
  if (!*changed || (int)blockIdx.y >= nl) return;
  const GroupList& L = LT[blockIdx.y];
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < L.nd; d += gridDim.x * blockDim.x) {
    if (!listed[L.inst[d]]) continue;
    const int f = L.first[d], n = L.nb[d];
    for (int k = 0; k < n; ++k) L.map[f + k] = d;
  }
}

helm_status GroupLists::upload(int ninst, cudaStream_t st) {
  const int nl = (int)inst.size();
  host.resize(nl);
  auto alloc = [&](void** p, size_t bytes) {
    DevBlock b;
    helm_status s = dev_alloc(p, bytes, st, &b);
    if (s == HELM_OK) mem.push_back(b);
    return s;
  };
  helm_status s;
  for (int li = 0; li < nl; ++li) {
    GroupList& L = host[li];
    L.nd = (int)inst[li].size();
    int *di = nullptr, *dn = nullptr;
    if ((s = alloc((void**)&di, sizeof(int) * L.nd)) != HELM_OK) return s;
    if ((s = alloc((void**)&dn, sizeof(int) * L.nd)) != HELM_OK) return s;
    if ((s = alloc((void**)&L.first, sizeof(int) * (L.nd + 1))) != HELM_OK) return s;
    if ((s = alloc((void**)&L.map, sizeof(int) * std::max(capacity(li), 1))) != HELM_OK) return s;
    HELM_CUDA(cudaMemcpyAsync(di, inst[li].data(), sizeof(int) * L.nd, cudaMemcpyHostToDevice, st));
    HELM_CUDA(cudaMemcpyAsync(dn, nb[li].data(), sizeof(int) * L.nd, cudaMemcpyHostToDevice, st));
    HELM_CUDA(cudaMemsetAsync(L.first, 0, sizeof(int) * (L.nd + 1), st));  // empty until compacted
    L.inst = di;
    L.nb = dn;
  }
  if ((s = alloc((void**)&dev, sizeof(GroupList) * std::max(nl, 1))) != HELM_OK) return s;
  if (nl) HELM_CUDA(cudaMemcpyAsync(dev, host.data(), sizeof(GroupList) * nl, cudaMemcpyHostToDevice, st));
  if ((s = alloc((void**)&listed, sizeof(int) * ninst)) != HELM_OK) return s;
  if ((s = alloc((void**)&changed, sizeof(int))) != HELM_OK) return s;
  HELM_CUDA(cudaMemsetAsync(listed, 0, sizeof(int) * ninst, st));
  HELM_CUDA(cudaMemsetAsync(changed, 0, sizeof(int), st));
  HELM_CUDA(cudaStreamSynchronize(st));  // the host vectors are pageable copies' sources
  return HELM_OK;
}

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct GroupRun {
  GroupLists lists;
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
    dev_free_all(lists.mem, st);
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
  if (c->pc.smoother == HELM_SM_ILU) return "grouped solves smooth with damped Jacobi or red-black Gauss-Seidel";
  if (c->pc.smoother != c0->pc.smoother) return "the instances of a group share one smoother kind";
  if (c->pc.mg_dtype != c0->pc.mg_dtype) return "the instances of a group share one multigrid precision";
  return nullptr;
}

// the condition and compaction launches (head and end of the body)
void enqueue_control(cudaGraphConditionalHandle h, const GroupBicg* dA, int ni, int* loops, int cap, int in_body,
                     GroupLists& Ls, cudaStream_t cs) {
  const int nl = (int)Ls.inst.size();
  launch_pdl(kg_cond, dim3(1), dim3(256), 0, cs, h, dA, ni, loops, cap, in_body, Ls.listed, Ls.changed);
  launch_pdl(kg_prefix, dim3((nl + 7) / 8), dim3(256), 0, cs, Ls.dev, nl, (const int*)Ls.listed,
             (const int*)Ls.changed);
  launch_pdl(kg_fill, dim3(1, nl), dim3(256), 0, cs, Ls.dev, nl, (const int*)Ls.listed, (const int*)Ls.changed);
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
  std::vector<int> kinst, knb;
  int blocks = 0;
  for (int i = 0; i < ni; ++i) {
    const helm_ctx* c = cs[i];
    Workspace* w = c->ws;
    A[i] = GroupBicg{w->st, c->H.view<double>(), w->x, w->r, w->rh, w->p, w->v, w->sv, w->t, w->ph, w->sh,
                     f32 ? w->pmg : nullptr, f32 ? w->smg : nullptr, c->n, w->partials, w->G};
    kinst.push_back(i);
    knb.push_back(w->G);
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
  const int kli = R.lists.add(kinst, knb);  // the work list of the Krylov kernels
  if ((s = group_vcycle_build<TM>(cs, ni, inp.data(), outp.data(), skip.data(), &R.lists, st, &R.vp)) != HELM_OK)
    return s;
  if ((s = group_vcycle_build<TM>(cs, ni, ins.data(), outs.data(), skip.data(), &R.lists, st, &R.vs)) != HELM_OK)
    return s;
  if ((s = R.lists.upload(ni, st)) != HELM_OK) return s;
  if ((s = group_vcycle_finalize<TM>(R.vp, &R.lists)) != HELM_OK) return s;
  if ((s = group_vcycle_finalize<TM>(R.vs, &R.lists)) != HELM_OK) return s;
  const GroupList* LT = R.lists.dev;
  const int kgrid = std::max(1, blocks);  // one block per virtual block (see group_grid in mg_fused.cu)

  // the loop graph: [condition from the instances' states] -> WHILE(any running) { one iteration }
  const int cap = o->maxmv + 16;
  HELM_CUDA(cudaGraphCreate(&R.graph, 0));
  cudaGraphConditionalHandle h;
  HELM_CUDA(cudaGraphConditionalHandleCreate(&h, R.graph, 0, 0));
  cudaStream_t cs0;
  HELM_CUDA(cudaStreamCreateWithFlags(&cs0, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs0, R.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaStreamBeginCaptureToGraph(group)"); }
  enqueue_control(h, dA, ni, loops, cap, 0, R.lists, cs0);
  cudaGraph_t dummy = nullptr;
  e = cudaStreamEndCapture(cs0, &dummy);
  if (e != cudaSuccess) { cudaStreamDestroy(cs0); return cuda_check(e, "cudaStreamEndCapture(group head)"); }
  // the WHILE node follows the head's last node (the compaction kernels run after the condition)
  size_t nh = 0;
  cudaGraphGetNodes(R.graph, nullptr, &nh);
  std::vector<cudaGraphNode_t> all(nh);
  cudaGraphGetNodes(R.graph, all.data(), &nh);
  std::vector<cudaGraphNode_t> heads;
  for (cudaGraphNode_t nd : all) {
    size_t nout = 0;
    cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout);
    if (nout == 0) heads.push_back(nd);
  }
  nh = heads.size();
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
  group_krylov_launch<TM>(GK_P, dA, LT, kli, kgrid, cs0);
  group_vcycle_enqueue<TM>(R.vp, cs0);
  group_krylov_launch<TM>(GK_V, dA, LT, kli, kgrid, cs0);
  group_krylov_launch<TM>(GK_S, dA, LT, kli, kgrid, cs0);
  group_krylov_launch<TM>(GK_XHALF, dA, LT, kli, kgrid, cs0);
  group_vcycle_enqueue<TM>(R.vs, cs0);
  group_krylov_launch<TM>(GK_T, dA, LT, kli, kgrid, cs0);
  group_krylov_launch<TM>(GK_XR, dA, LT, kli, kgrid, cs0);
  enqueue_control(h, dA, ni, loops, cap, 1, R.lists, cs0);
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
    kernels += 3 + (long)hl * (long)R.body_nodes + 2L * nrun;
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
