// krylov_state.cuh -- the device-side state and workspace of a Krylov solve, shared by the
// single-instance solver (krylov.cu) and the grouped solver that runs many instances' iterations
// as one launch per kernel (group.cu).
#pragma once

#include <vector>

#include "helm_internal.cuh"

namespace helm {

constexpr int KT = 256;      // threads per block of the vector kernels
#ifndef KRYLOV_BLOCKS_PER_SM
#define KRYLOV_BLOCKS_PER_SM 2
#endif
constexpr int SMAX = 8;      // largest IDR shadow dimension
constexpr int NRED = SMAX + 2;
constexpr int GMRES_MMAX = HELM_GMRES_MAX_M;  // largest GMRES restart length

struct KrylovState {
  double2 rho, rho_old, alpha, omega, beta;
  double bnorm, tol, rel_recur, rel_true;
  int done, status, half, matvecs, iters, maxmv;
  int k, oldest, s, loops;  // loops: body executions of the WHILE node in this solve
  double2 M[SMAX * SMAX];  // IDR: P^H dR, column-major M[i + s*j]
  double2 m[SMAX];         // IDR: P^H r
  double2 c[SMAX];         // IDR: M^{-1} m
  unsigned int ticket[8];  // last-block counters, one per reduction site
  double* hist;            // optional residual history (device), capacity maxmv
  double hn;               // GMRES: norm of the last orthogonalised vector, h_{j+1,j}
  int gmm;                 // GMRES: restart length m
  double2* gm;             // GMRES: Hessenberg matrix, rotations, g, y and the two h passes
  int xs_n0, xs_h;         // level 0 of an FP32 hierarchy stored x-split: row length and even
                           // x indices per row (xs_n0 = 0: natural order)
};

struct Workspace {
  int method = -1, s = 0;
  int G = 0;                   // blocks of the vector kernels (fixed -> fixed reduction order)
  KrylovState* st = nullptr;   // device
  KrylovState* hst = nullptr;  // pinned host copy
  double2* partials = nullptr; // [NRED][G]
  double2 *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *sv = nullptr, *t = nullptr, *q = nullptr;
  void *pmg = nullptr, *smg = nullptr;  // V-cycle inputs in the multigrid precision
  double2 *ph = nullptr, *sh = nullptr; // V-cycle outputs, widened to complex128
  double2 *P = nullptr, *dR = nullptr, *dX = nullptr;                  // IDR, s vectors each
  double2 *V = nullptr, *gm = nullptr;  // GMRES: m + 1 basis vectors; its small dense arrays
  int nred = NRED;                      // partial-sum slots per block
  const void* shadow_key = nullptr;
  cudaGraphExec_t loop = nullptr;
  cudaGraphExec_t body = nullptr;       // host-driven loop: one iteration per launch
  cudaGraphExec_t idr_init = nullptr;
  cudaGraph_t loop_graph = nullptr, init_graph = nullptr, body_graph = nullptr;
  size_t body_nodes = 0, init_nodes = 0;  // kernels per loop body / IDR start graph
  std::vector<DevBlock> mem;
  size_t bytes = 0;  // device bytes of mem (counted in the context's total while it lives)
};


// One instance of a grouped Bi-CGSTAB launch: its scalars, operator and workspace vectors, and
// its block count G (as in its single-instance launches, so that every reduction sums in the same
// order as when it runs alone).
struct GroupBicg {
  KrylovState* S;
  OpView<double> H;
  double2 *x, *r, *rh, *p, *v, *sv, *t, *ph, *sh;
  void *pmg, *smg;  // V-cycle inputs in FP32 (FP32 multigrid), else nullptr
  long n;
  double2* partials;
  int G;
};

// The grouped Bi-CGSTAB kernels (2D operators; krylov.cu): each is one launch of `grid` blocks (the
// list's capacity) over the work list LT[li] of the instances in A (device array).
enum { GK_P = 0, GK_V, GK_S, GK_XHALF, GK_T, GK_XR };
template <typename TM>
void group_krylov_launch(int which, const GroupBicg* A, const GroupList* LT, int li, int grid, cudaStream_t st);

// One instance's steps outside the grouped loop (krylov.cu): its Bi-CGSTAB workspace and per-solve
// scalars with x = 0; its start kernel (first: r = b, else a restart from the true residual); its
// FP64 true residual followed by the copy of its scalars to the pinned host struct.
helm_status group_member_begin(helm_ctx* c, const helm_solve_opts* o, cudaStream_t st);
void group_member_start(helm_ctx* c, const double2* b, bool first, cudaStream_t st);
void group_member_true_res(helm_ctx* c, const double2* b, cudaStream_t st);

}  // namespace helm
