/*
 * helm_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the preconditioned
 * Krylov solve of the ECS-discretised indefinite Helmholtz equation of
 * Reps, Vanroose & bin Zubair, "On the indefinite Helmholtz equation: complex stretched
 * absorbing boundary layers, iterative analysis, and preconditioning" (arXiv 0912.0180).
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA path; only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is written as loops over the definitions, in the paper's order:
 *   - grid and complex mesh widths: Section 2 (ECS map z = (x - r) e^{i theta} + r, mesh width
 *     h_gamma = h e^{i theta}) and Section 3 (vertex-centred ECS grid, eq. "ecsgrid");
 *   - Shortley-Weller second difference on non-uniform (complex) widths: Section 3, eq.
 *     "shortwell"; H = -(Laplacian + phi) with phi = k(x)^2: eq. "helmctu0" / "Helgen";
 *   - preconditioners: CSL M = -(L + beta^2 k^2), eq. "helmctucsl" (Section 5.2); CSG, every
 *     (or only the interior) mesh width multiplied by beta = e^{i theta_beta}, eq. "CSL-CSG"
 *     and eq. "lapctucsg" (Section 5.3);
 *   - geometric multigrid on the preconditioner (Section 5.1, Section 6.1 components: full
 *     weighting restriction, bilinear prolongation, rediscretised ("direct") coarse operators
 *     or (2D) Galerkin coarse operators R A P, omega-Jacobi; red-black Gauss-Seidel as a
 *     second smoother; ILU(0), the paper's smoother, on 1D and 2D levels; direct coarsest
 *     solve);
 *   - right-preconditioned Bi-CGSTAB (van der Vorst 1992) and IDR(s) (Sonneveld & van Gijzen
 *     2008), the Krylov methods of Section 6.2, stopped on ||d_m|| / ||d_0|| < tol (the
 *     stopping rule of Section 6.2), followed by a true-residual check.
 *
 * Readings where the paper is silent (documented in the design notes): hierarchy by
 * index-even coarsening with summed complex gaps; phi injected at the coarse nodes; FW and
 * linear interpolation weights in index space; red = even (i + j + l), red first; Hermitian
 * inner products conjugating the first argument; zero initial guess.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Point-wise loops (stencil, smoothers, transfers, vector updates) may run on several threads:
 * every element is computed by the same expression in the same order whatever the thread count,
 * and every inner product and norm is a single-threaded sum in index order, so results are
 * bitwise the same on one thread and on many.  PAR_FOR2 splits the two outer loops of a grid
 * sweep, PAR_FOR a flat loop over unknowns; both stay serial up to 4096 unknowns. */
#define PAR_PRAGMA(x) _Pragma(#x)
#ifdef _OPENMP
#define PAR_FOR2(n) PAR_PRAGMA(omp parallel for collapse(2) schedule(static) if ((n) > 4096))
#define PAR_FOR(n) PAR_PRAGMA(omp parallel for schedule(static) if ((n) > 4096))
#else
#define PAR_FOR2(n)
#define PAR_FOR(n)
#endif

/* Threads used by the point-wise loops (1 = serial); returns the previous value. */
int orc_set_threads(int t) {
#ifdef _OPENMP
  int old = omp_get_max_threads();
  if (t >= 1) omp_set_num_threads(t);
  return old;
#else
  (void)t;
  return 1;
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- public structs (mirrored by the ctypes wrapper in oracle.py) -------------------- */
typedef struct {
  int dim;              /* 1, 2 or 3 */
  int n_int[3];         /* interior grid nodes per axis, both ends (turning points) included */
  int n_layer[3][2];    /* ECS layer nodes on the low / high side; 0 = Dirichlet wall; -1 on a
                           high side = first-order Sommerfeld condition there (Section 2,
                           eq. "sommerfeld1"): the boundary node is an unknown */
  double extent[3];     /* length of the real interior along each axis */
  double theta_gamma;   /* ECS angle */
  int ecs_ramp;         /* R > 1: the m-th layer width from the turning point has angle
                           theta_gamma * min(m, R) / R (smooth ECS transition, Section 7);
                           0 or 1: the sharp contour */
} orc_grid;

typedef struct {
  int kind;             /* 0 identity, 1 CSL, 2 CSG on every width, 3 CSG on interior widths */
  double theta_beta;    /* CSG angle */
  double shift_re, shift_im; /* CSL: beta^2 */
  int nu1, nu2;         /* pre / post smoothing sweeps */
  int smoother;         /* 0 damped Jacobi, 1 red-black Gauss-Seidel, 2 ILU(0) (1D / 2D) */
  double omega;         /* Jacobi damping */
  int max_levels;       /* cap on the number of levels (>= 1) */
  int coarse_max;       /* stop coarsening once every axis has <= coarse_max unknowns */
  int galerkin;         /* 1: coarse operators R A P (2D, 9-point) instead of rediscretised */
} orc_precond;

typedef struct {
  int method;           /* 0 Bi-CGSTAB, 1 IDR(s), 2 GMRES(m) */
  int s;                /* IDR shadow dimension; GMRES restart length m */
  double tol;           /* stop on ||r|| / ||b|| < tol */
  int maxmv;            /* cap on preconditioned matvecs */
  int max_restarts;     /* true-residual restarts allowed */
} orc_solve_opts;

typedef struct {
  int status;           /* 0 ok, 4 breakdown, 5 max matvecs, 6 not finite */
  int iters;            /* Bi-CGSTAB iterations, or IDR steps */
  int matvecs;          /* preconditioned matvecs (one V-cycle + one H apply each) */
  int restarts;
  double rel_res_recur; /* last recurrence residual / ||b|| */
  double rel_res_true;  /* ||b - H x|| / ||b|| of the returned x */
} orc_info;

/* ---- grid ---------------------------------------------------------------------------- */
typedef struct {
  int n;          /* unknowns on this axis */
  cplx* gap;      /* n + 1 widths: gap[j] = z(node j+1) - z(node j), nodes 0 and n+1 Dirichlet;
                     with a Sommerfeld high side, gap[n] is the mirror width to the ghost node */
  double* pos;    /* n real positions of the unknowns (only used to sample phi) */
  cplx *am, *a0, *ap; /* Shortley-Weller row of -d^2/dz^2 at each unknown */
  int somm;       /* 1: the last unknown is a Sommerfeld boundary node */
  cplx bt;        /* its boundary weight 2i / h_l: the diagonal gains bt * k */
  int somm_lo;    /* 1: the first unknown is a Sommerfeld boundary node (low side) */
  cplx bt_lo;     /* its boundary weight 2i / h_r */
  int off;        /* coarsening offset: coarse unknown c is fine unknown 2c + off (0 with a
                     Sommerfeld low side, whose boundary node 0 every level keeps; else 1) */
} axis_t;

typedef struct {
  int dim;
  int n[3];
  long ntot;
  axis_t ax[3];
  double* phi;    /* k(x)^2 at every unknown */
  double* phi_im; /* imaginary part of phi (k evaluated at complex node positions); NULL = real */
  cplx s;         /* sigma = s * phi; 1 for H and CSG, beta^2 for CSL */
  cplx* st9;      /* Galerkin levels (2D): row p is st9[9p + 3(dj+1) + (di+1)], the weight of the
                     unknown (i+di, j+dj); NULL for a Shortley-Weller level */
  cplx* st27;     /* Galerkin levels (3D): row p is st27[27p + 9(dl+1) + 3(dj+1) + (di+1)] */
  cplx* ilu;      /* ILU(0) factors (1D / 2D), laid out as st9: at the lower neighbours of row p
                     the entries of L (unit diagonal implied), at p and its upper neighbours U */
} level_t;

typedef struct orc_ctx {
  orc_grid grid;
  orc_precond pc;
  level_t H;      /* the Helmholtz operator itself */
  int nlev;
  level_t* M;     /* preconditioner hierarchy, M[0] on the finest grid */
  cplx* lu;       /* dense LU (partial pivoting) of the coarsest M */
  int* piv;
  long nco;
} orc_ctx;

static long imax(long a, long b) { return a > b ? a : b; }

/* Complex mesh widths of one axis (Section 2: h_gamma = h e^{i theta_gamma} on the layers;
 * Section 5.3: CSG multiplies widths by beta).  scale_in multiplies the interior widths,
 * scale_ly the layer widths. */
/* Width of the m-th layer gap counted outwards from the turning point (m >= 1): h e^{i theta},
 * theta = theta_gamma for the sharp contour, theta_gamma * min(m, R) / R for a ramp of R widths. */
static cplx layer_width(double h, double theta_g, int ramp, int m) {
  double th = theta_g;
  if (ramp > 1 && m < ramp) th = theta_g * m / ramp;
  return h * cexp(I * th);
}

static void axis_build(axis_t* a, int n_int, const int nl[2], double extent, double theta_g,
                       int ramp, cplx scale_in, cplx scale_ly) {
  double h = extent / (n_int - 1);
  int lo = nl[0], hi = nl[1];
  /* a Sommerfeld side adds one width: the mirror of the adjacent interior one, to the ghost node */
  int ngap = (n_int - 1) + (lo > 0 ? lo + 1 : (lo < 0 ? 1 : 0)) + (hi > 0 ? hi + 1 : (hi < 0 ? 1 : 0));
  a->n = ngap - 1;
  a->somm = hi < 0;
  a->somm_lo = lo < 0;
  a->off = lo < 0 ? 0 : 1;
  a->gap = malloc(sizeof(cplx) * ngap);
  a->pos = malloc(sizeof(double) * imax(a->n, 1));
  int g = 0;
  if (lo > 0)  /* outermost first: gap m = lo + 1 down to 1 */
    for (int m = lo + 1; m >= 1; --m) a->gap[g++] = layer_width(h, theta_g, ramp, m) * scale_ly;
  if (lo < 0) a->gap[g++] = h * scale_in;
  for (int m = 0; m < n_int - 1; ++m) a->gap[g++] = h * scale_in;
  if (hi > 0)
    for (int m = 1; m <= hi + 1; ++m) a->gap[g++] = layer_width(h, theta_g, ramp, m) * scale_ly;
  if (hi < 0) a->gap[g++] = h * scale_in;
  /* real positions: the layers continue the real coordinate */
  int u = 0;
  for (int m = lo; m >= 1; --m) a->pos[u++] = -m * h;
  int first = lo != 0 ? 0 : 1, last = hi != 0 ? n_int - 1 : n_int - 2;
  for (int j = first; j <= last; ++j) a->pos[u++] = j * h;
  for (int m = 1; m <= hi; ++m) a->pos[u++] = extent + m * h;
}

/* Shortley-Weller (Section 3, eq. "shortwell"): with left width hl = gap[j], right width
 * hr = gap[j+1],  -u'' ~ -2/(hl+hr) (u_{j-1}/hl - (1/hl + 1/hr) u_j + u_{j+1}/hr). */
static void axis_coeffs(axis_t* a) {
  a->am = malloc(sizeof(cplx) * imax(a->n, 1));
  a->a0 = malloc(sizeof(cplx) * imax(a->n, 1));
  a->ap = malloc(sizeof(cplx) * imax(a->n, 1));
  for (int j = 0; j < a->n; ++j) {
    cplx hl = a->gap[j], hr = a->gap[j + 1];
    cplx f = 2.0 / (hl + hr);
    a->am[j] = -f / hl;
    a->a0[j] = f * (1.0 / hl + 1.0 / hr);
    a->ap[j] = -f / hr;
  }
  a->bt = 0;
  if (a->somm && a->n > 0) {
    /* Sommerfeld node N (Section 2, eq. "sommerfeld1", du/dn = -i k u): the centred difference
     * (u_g - u_{N-1}) / (2 h_l) = -i k u_N puts the ghost value u_g = u_{N-1} - 2 i k h_l u_N into
     * the row: the left weight doubles, the right one vanishes, and the diagonal gains
     * -2 i k h_l ap = 2 i k / h_l (the gap to the ghost mirrors h_l). */
    int N = a->n - 1;
    cplx hl = a->gap[N];
    a->bt = -2.0 * I * hl * a->ap[N];
    a->am[N] *= 2.0;
    a->ap[N] = 0;
  }
  a->bt_lo = 0;
  if (a->somm_lo && a->n > 0) {
    /* Sommerfeld node 0 on the low side (outward normal -x, so du/dx = i k u there): the centred
     * difference (u_1 - u_g) / (2 h_r) = i k u_0 gives the ghost u_g = u_1 - 2 i k h_r u_0, so the
     * right weight doubles, the left one vanishes and the diagonal gains -2 i k h_r am = 2 i k / h_r
     * (the gap to the ghost mirrors h_r) */
    cplx hr = a->gap[0];
    a->bt_lo = -2.0 * I * hr * a->am[0];
    a->ap[0] *= 2.0;
    a->am[0] = 0;
  }
}

/* Index-even coarsening: coarse unknown c is fine unknown 2c+1 (0-based), i.e. coarse node
 * c+1 is fine node 2(c+1); coarse widths are the sums of the fine widths between coarse
 * nodes; the last one reaches the fine Dirichlet node and spans one or two fine widths.
 * With a Sommerfeld low side the offset is 0 instead (coarse c is fine 2c), so that the boundary
 * node 0 stays a node of every level; its ghost width mirrors the first coarse width. */
static void axis_coarsen(const axis_t* f, axis_t* c) {
  const int o = f->off;
  c->n = o ? f->n / 2 : (f->n + 1) / 2;
  c->somm = f->somm;
  c->somm_lo = f->somm_lo;
  c->off = f->off;
  c->gap = malloc(sizeof(cplx) * (c->n + 1));
  c->pos = malloc(sizeof(double) * imax(c->n, 1));
  for (int ci = 0; ci < c->n; ++ci) {
    /* the widths between fine nodes 2(ci-1)+o and 2ci+o; before the first coarse node, those
     * from the low end (its Dirichlet node, or the ghost) */
    c->gap[ci] = (2 * ci + o - 1 >= 0 ? f->gap[2 * ci + o - 1] : 0) + f->gap[2 * ci + o];
    c->pos[ci] = f->pos[2 * ci + o];
  }
  if (c->somm_lo && c->n > 1) c->gap[0] = c->gap[1];
  cplx last = 0;
  for (int j = 2 * (c->n - 1) + o + 1; j <= f->n; ++j) last += f->gap[j];
  /* a Sommerfeld high side is coarsened only when its boundary node n-1 is a coarse node; its
   * ghost width mirrors the last coarse width */
  c->gap[c->n] = c->somm ? c->gap[c->n - 1] : last;
  axis_coeffs(c);
}

static void axis_free(axis_t* a) {
  free(a->gap); free(a->pos); free(a->am); free(a->a0); free(a->ap);
}

static void level_free(level_t* L) {
  free(L->st9);
  free(L->st27);
  free(L->ilu);
  for (int d = 0; d < L->dim; ++d) axis_free(&L->ax[d]);
  free(L->phi);
  free(L->phi_im);
}

static long lidx(const level_t* L, int i, int j, int l) {
  return i + (long)L->n[0] * (j + (long)L->n[1] * l);
}

/* Fine level: gaps for the requested operator, phi sampled (or constant). */
static void level_fine(level_t* L, const orc_grid* g, const double* phi, const double* phi_im, double k0,
                       cplx scale_in, cplx scale_ly, cplx s) {
  memset(L, 0, sizeof(*L));
  L->dim = g->dim;
  L->ntot = 1;
  for (int d = 0; d < 3; ++d) L->n[d] = 1;
  for (int d = 0; d < g->dim; ++d) {
    axis_build(&L->ax[d], g->n_int[d], g->n_layer[d], g->extent[d], g->theta_gamma, g->ecs_ramp,
               scale_in, scale_ly);
    axis_coeffs(&L->ax[d]);
    L->n[d] = L->ax[d].n;
    L->ntot *= L->n[d];
  }
  L->phi = malloc(sizeof(double) * imax(L->ntot, 1));
  for (long p = 0; p < L->ntot; ++p) L->phi[p] = phi ? phi[p] : k0 * k0;
  if (phi_im) {
    L->phi_im = malloc(sizeof(double) * imax(L->ntot, 1));
    memcpy(L->phi_im, phi_im, sizeof(double) * L->ntot);
  }
  L->s = s;
}

/* Coarse level: coarsened axes, phi injected at the coarse nodes. */
static void level_coarse(const level_t* F, level_t* C) {
  memset(C, 0, sizeof(*C));
  C->dim = F->dim;
  C->ntot = 1;
  for (int d = 0; d < 3; ++d) C->n[d] = 1;
  for (int d = 0; d < F->dim; ++d) {
    axis_coarsen(&F->ax[d], &C->ax[d]);
    C->n[d] = C->ax[d].n;
    C->ntot *= C->n[d];
  }
  C->phi = malloc(sizeof(double) * imax(C->ntot, 1));
  for (int l = 0; l < C->n[2]; ++l)
    for (int j = 0; j < C->n[1]; ++j)
      for (int i = 0; i < C->n[0]; ++i) {
        int fi = 2 * i + F->ax[0].off, fj = F->dim > 1 ? 2 * j + F->ax[1].off : 0;
        int fl = F->dim > 2 ? 2 * l + F->ax[2].off : 0;
        C->phi[lidx(C, i, j, l)] = F->phi[lidx(F, fi, fj, fl)];
      }
  if (F->phi_im) {  /* injected like the real part */
    C->phi_im = malloc(sizeof(double) * imax(C->ntot, 1));
    for (int l = 0; l < C->n[2]; ++l)
      for (int j = 0; j < C->n[1]; ++j)
        for (int i = 0; i < C->n[0]; ++i) {
          int fi = 2 * i + F->ax[0].off, fj = F->dim > 1 ? 2 * j + F->ax[1].off : 0;
          int fl = F->dim > 2 ? 2 * l + F->ax[2].off : 0;
          C->phi_im[lidx(C, i, j, l)] = F->phi_im[lidx(F, fi, fj, fl)];
        }
  }
  C->s = F->s;
}

/* Diagonal of the operator at point (i,j,l): sum of the per-axis centre weights - s*phi
 * (a Galerkin level: its stencil's centre weight). */
static cplx diag_at(const level_t* L, int i, int j, int l) {
  if (L->st9) return L->st9[9 * lidx(L, i, j, l) + 4];
  if (L->st27) return L->st27[27 * lidx(L, i, j, l) + 13];
  int ix[3] = {i, j, l};
  cplx d = 0;
  double ph = L->phi[lidx(L, i, j, l)];
  for (int a = 0; a < L->dim; ++a) {
    d += L->ax[a].a0[ix[a]];
    /* Sommerfeld boundary node: + 2 i k / h_l with k = sqrt(phi), the unshifted wave number */
    if (L->ax[a].somm && ix[a] == L->ax[a].n - 1) d += L->ax[a].bt * sqrt(ph);
    if (L->ax[a].somm_lo && ix[a] == 0) d += L->ax[a].bt_lo * sqrt(ph);
  }
  cplx phc = ph + I * (L->phi_im ? L->phi_im[lidx(L, i, j, l)] : 0.0);
  return d - L->s * phc;
}

/* Off-diagonal part of row (i,j,l) applied to x (Dirichlet neighbours contribute 0). */
static cplx offdiag_at(const level_t* L, const cplx* x, int i, int j, int l) {
  if (L->st9) {  /* the eight neighbours of a Galerkin stencil */
    cplx acc = 0;
    const cplx* w = L->st9 + 9 * lidx(L, i, j, l);
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        if (di == 0 && dj == 0) continue;
        int ii = i + di, jj = j + dj;
        if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1]) continue;
        acc += w[3 * (dj + 1) + (di + 1)] * x[lidx(L, ii, jj, 0)];
      }
    return acc;
  }
  if (L->st27) {  /* the 26 neighbours of a 3D Galerkin stencil */
    cplx acc = 0;
    const cplx* w = L->st27 + 27 * lidx(L, i, j, l);
    for (int dl = -1; dl <= 1; ++dl)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (di == 0 && dj == 0 && dl == 0) continue;
          int ii = i + di, jj = j + dj, ll = l + dl;
          if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1] || ll < 0 || ll >= L->n[2]) continue;
          acc += w[9 * (dl + 1) + 3 * (dj + 1) + (di + 1)] * x[lidx(L, ii, jj, ll)];
        }
    return acc;
  }
  int ix[3] = {i, j, l};
  cplx acc = 0;
  for (int a = 0; a < L->dim; ++a) {
    int k = ix[a];
    int lo[3] = {i, j, l}, hi[3] = {i, j, l};
    lo[a] = k - 1;
    hi[a] = k + 1;
    if (k > 0) acc += L->ax[a].am[k] * x[lidx(L, lo[0], lo[1], lo[2])];
    if (k < L->n[a] - 1) acc += L->ax[a].ap[k] * x[lidx(L, hi[0], hi[1], hi[2])];
  }
  return acc;
}

/* y = A x for the operator of a level: the d-fold sum of Shortley-Weller rows minus
 * sigma = s * phi (eq. "helmctu0" / "Helgen"; CSL eq. "helmctucsl"). */
static void level_apply(const level_t* L, const cplx* x, cplx* y) {
  PAR_FOR2(L->ntot)
  for (int l = 0; l < L->n[2]; ++l)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        long p = lidx(L, i, j, l);
        y[p] = diag_at(L, i, j, l) * x[p] + offdiag_at(L, x, i, j, l);
      }
}

/* ---- dense LU with partial pivoting (the "direct" coarsest solve) ---------------------- */
static int lu_factor(cplx* A, int* piv, long n) {
  for (long k = 0; k < n; ++k) {
    long p = k;
    double best = cabs(A[k * n + k]);
    for (long r = k + 1; r < n; ++r)
      if (cabs(A[r * n + k]) > best) { best = cabs(A[r * n + k]); p = r; }
    piv[k] = (int)p;
    if (best == 0.0) return -1;
    if (p != k)
      for (long c = 0; c < n; ++c) { cplx t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t; }
    PAR_FOR((n - k) * (n - k))
    for (long r = k + 1; r < n; ++r) {
      cplx m = A[r * n + k] / A[k * n + k];
      A[r * n + k] = m;
      for (long c = k + 1; c < n; ++c) A[r * n + c] -= m * A[k * n + c];
    }
  }
  return 0;
}

static void lu_solve(const cplx* A, const int* piv, long n, const cplx* b, cplx* x) {
  if (x != b) memcpy(x, b, sizeof(cplx) * n);
  for (long k = 0; k < n; ++k)
    if (piv[k] != k) { cplx t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (long r = 0; r < n; ++r)
    for (long c = 0; c < r; ++c) x[r] -= A[r * n + c] * x[c];
  for (long r = n - 1; r >= 0; --r) {
    for (long c = r + 1; c < n; ++c) x[r] -= A[r * n + c] * x[c];
    x[r] /= A[r * n + r];
  }
}

/* Dense matrix of a level's operator, row-major, assembled entry by entry. */
static void level_dense(const level_t* L, cplx* A) {
  long n = L->ntot;
  memset(A, 0, sizeof(cplx) * n * n);
  if (L->st9) {
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i)
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            int ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1]) continue;
            A[lidx(L, i, j, 0) * n + lidx(L, ii, jj, 0)] = L->st9[9 * lidx(L, i, j, 0) + 3 * (dj + 1) + (di + 1)];
          }
    return;
  }
  if (L->st27) {
    for (int l = 0; l < L->n[2]; ++l)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i)
          for (int dl = -1; dl <= 1; ++dl)
            for (int dj = -1; dj <= 1; ++dj)
              for (int di = -1; di <= 1; ++di) {
                int ii = i + di, jj = j + dj, ll = l + dl;
                if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1] || ll < 0 || ll >= L->n[2]) continue;
                A[lidx(L, i, j, l) * n + lidx(L, ii, jj, ll)] =
                    L->st27[27 * lidx(L, i, j, l) + 9 * (dl + 1) + 3 * (dj + 1) + (di + 1)];
              }
    return;
  }
  for (int l = 0; l < L->n[2]; ++l)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        long p = lidx(L, i, j, l);
        A[p * n + p] = diag_at(L, i, j, l);
        int ix[3] = {i, j, l};
        for (int a = 0; a < L->dim; ++a) {
          int k = ix[a];
          long stride = a == 0 ? 1 : (a == 1 ? L->n[0] : (long)L->n[0] * L->n[1]);
          if (k > 0) A[p * n + p - stride] = L->ax[a].am[k];
          if (k < L->n[a] - 1) A[p * n + p + stride] = L->ax[a].ap[k];
        }
      }
}

/* Weight of fine unknown `fine` in the full-weighting row of coarse unknown `coarse` along one
 * axis: the row gathers fine 2c, 2c+1, 2c+2 with 1/4, 1/2, 1/4. */
static double fw_weight(int fine, int coarse) {
  int d = fine - (2 * coarse + 1);
  return d == 0 ? 0.5 : (d == 1 || d == -1 ? 0.25 : 0.0);
}

/* Weight of coarse unknown `coarse` in the linear interpolation of fine unknown `fine` along
 * one axis: 1 at fine 2c+1, 1/2 at fine 2c and 2c+2. */
static double lin_weight(int fine, int coarse) {
  int d = fine - (2 * coarse + 1);
  return d == 0 ? 1.0 : (d == 1 || d == -1 ? 0.5 : 0.0);
}

/* Entry (row p, column q) of a 2D level's operator, by its definition. */
static cplx entry2d(const level_t* L, int i, int j, int ii, int jj) {
  if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1]) return 0;
  if (L->st9) {
    int di = ii - i, dj = jj - j;
    if (di < -1 || di > 1 || dj < -1 || dj > 1) return 0;
    return L->st9[9 * lidx(L, i, j, 0) + 3 * (dj + 1) + (di + 1)];
  }
  if (ii == i && jj == j) return diag_at(L, i, j, 0);
  if (jj == j && ii == i - 1) return L->ax[0].am[i];
  if (jj == j && ii == i + 1) return L->ax[0].ap[i];
  if (ii == i && jj == j - 1) return L->ax[1].am[j];
  if (ii == i && jj == j + 1) return L->ax[1].ap[j];
  return 0;
}

/* Galerkin coarse operator (2D): C = R F P with R the full weighting and P the linear
 * interpolation of the V-cycle, entry by entry:
 *   C[(I,J), (K,M)] = sum_{fine a,b} R[(I,J),(a,b)] sum_{fine c,d} F[(a,b),(c,d)] P[(c,d),(K,M)],
 * where only |K - I| <= 1, |M - J| <= 1 can be non-zero (the 9-point result); in the loops
 * (I, J) is (ci, cj) and (K, M) is (ck, cm). */
static void level_galerkin(const level_t* F, level_t* C) {
  C->st9 = calloc(9 * (size_t)imax(C->ntot, 1), sizeof(cplx));
  for (int cj = 0; cj < C->n[1]; ++cj)
    for (int ci = 0; ci < C->n[0]; ++ci)
      for (int dm = -1; dm <= 1; ++dm)
        for (int dk = -1; dk <= 1; ++dk) {
          int ck = ci + dk, cm = cj + dm;
          if (ck < 0 || ck >= C->n[0] || cm < 0 || cm >= C->n[1]) continue;
          cplx acc = 0;
          for (int b = 2 * cj; b <= 2 * cj + 2; ++b)
            for (int a = 2 * ci; a <= 2 * ci + 2; ++a) {
              if (a >= F->n[0] || b >= F->n[1]) continue;
              double r = fw_weight(a, ci) * fw_weight(b, cj);
              for (int d = b - 1; d <= b + 1; ++d)
                for (int c2 = a - 1; c2 <= a + 1; ++c2) {
                  double pw = lin_weight(c2, ck) * lin_weight(d, cm);
                  if (pw == 0.0) continue;
                  acc += r * entry2d(F, a, b, c2, d) * pw;
                }
            }
          C->st9[9 * lidx(C, ci, cj, 0) + 3 * (dm + 1) + (dk + 1)] = acc;
        }
}

/* Entry (row p, column q) of a 3D level's operator, by its definition. */
static cplx entry3d(const level_t* L, int i, int j, int l, int ii, int jj, int ll) {
  if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1] || ll < 0 || ll >= L->n[2]) return 0;
  int di = ii - i, dj = jj - j, dl = ll - l;
  if (L->st27) {
    if (di < -1 || di > 1 || dj < -1 || dj > 1 || dl < -1 || dl > 1) return 0;
    return L->st27[27 * lidx(L, i, j, l) + 9 * (dl + 1) + 3 * (dj + 1) + (di + 1)];
  }
  if (di == 0 && dj == 0 && dl == 0) return diag_at(L, i, j, l);
  if (dj == 0 && dl == 0 && di == -1) return L->ax[0].am[i];
  if (dj == 0 && dl == 0 && di == 1) return L->ax[0].ap[i];
  if (di == 0 && dl == 0 && dj == -1) return L->ax[1].am[j];
  if (di == 0 && dl == 0 && dj == 1) return L->ax[1].ap[j];
  if (di == 0 && dj == 0 && dl == -1) return L->ax[2].am[l];
  if (di == 0 && dj == 0 && dl == 1) return L->ax[2].ap[l];
  return 0;
}

/* Galerkin coarse operator (3D): C = R F P as in 2D, with the full weighting and the trilinear
 * interpolation tensorised over three axes; only coarse neighbours within one index on every
 * axis can be non-zero (the 27-point result).  (I,J,L) = (ci,cj,cl), (K,M,N) = (ck,cm,cn). */
static void level_galerkin3d(const level_t* F, level_t* C) {
  C->st27 = calloc(27 * (size_t)imax(C->ntot, 1), sizeof(cplx));
  for (int cl = 0; cl < C->n[2]; ++cl)
    for (int cj = 0; cj < C->n[1]; ++cj)
      for (int ci = 0; ci < C->n[0]; ++ci)
        for (int dn = -1; dn <= 1; ++dn)
          for (int dm = -1; dm <= 1; ++dm)
            for (int dk = -1; dk <= 1; ++dk) {
              int ck = ci + dk, cm = cj + dm, cn = cl + dn;
              if (ck < 0 || ck >= C->n[0] || cm < 0 || cm >= C->n[1] || cn < 0 || cn >= C->n[2]) continue;
              cplx acc = 0;
              for (int e = 2 * cl; e <= 2 * cl + 2; ++e)
                for (int b = 2 * cj; b <= 2 * cj + 2; ++b)
                  for (int a = 2 * ci; a <= 2 * ci + 2; ++a) {
                    if (a >= F->n[0] || b >= F->n[1] || e >= F->n[2]) continue;
                    double r = fw_weight(a, ci) * fw_weight(b, cj) * fw_weight(e, cl);
                    for (int g = e - 1; g <= e + 1; ++g)
                      for (int d = b - 1; d <= b + 1; ++d)
                        for (int c2 = a - 1; c2 <= a + 1; ++c2) {
                          double pw = lin_weight(c2, ck) * lin_weight(d, cm) * lin_weight(g, cn);
                          if (pw == 0.0) continue;
                          acc += r * entry3d(F, a, b, e, c2, d, g) * pw;
                        }
                  }
              C->st27[27 * lidx(C, ci, cj, cl) + 9 * (dn + 1) + 3 * (dm + 1) + (dk + 1)] = acc;
            }
}

/* ---- context ------------------------------------------------------------------------- */
/* phi_im (optional): the imaginary part of phi at every unknown, for k evaluated at the complex
 * node positions of the layers (the alternative to reading k at real positions); the Sommerfeld
 * boundary term keeps sqrt of the real part (its nodes are real). */
void orc_destroy(orc_ctx* c);
static void level_ilu(level_t* L);

/* Returns NULL when the coarsest preconditioner level is singular (its dense LU meets a zero
 * pivot), or for Galerkin coarse operators on a grid with a Sommerfeld low side. */
orc_ctx* orc_create(const orc_grid* g, const double* phi, const double* phi_im, double k0,
                    const orc_precond* pc) {
  orc_ctx* c = calloc(1, sizeof(orc_ctx));
  c->grid = *g;
  c->pc = *pc;
  level_fine(&c->H, g, phi, phi_im, k0, 1.0, 1.0, 1.0);
  if (pc->kind == 0) return c; /* identity preconditioner: no hierarchy */
  if (pc->smoother == 2 && g->dim > 2) { orc_destroy(c); return NULL; }  /* ILU(0): 1D / 2D */
  if (pc->galerkin)  /* the Galerkin products are written for the offset-1 coarsening only */
    for (int d = 0; d < g->dim; ++d)
      if (g->n_layer[d][0] < 0) { orc_destroy(c); return NULL; }
  cplx beta = cexp(I * pc->theta_beta);
  cplx scale_in = 1.0, scale_ly = 1.0, s = 1.0;
  if (pc->kind == 1) s = pc->shift_re + I * pc->shift_im;           /* CSL: sigma = beta^2 phi */
  else if (pc->kind == 2) { scale_in = beta; scale_ly = beta; }      /* CSG, every width */
  else if (pc->kind == 3) { scale_in = beta; }                       /* CSG, interior widths */
  int maxl = pc->max_levels < 1 ? 1 : pc->max_levels;
  c->M = calloc(maxl, sizeof(level_t));
  level_fine(&c->M[0], g, phi, phi_im, k0, scale_in, scale_ly, s);
  c->nlev = 1;
  while (c->nlev < maxl) {
    const level_t* F = &c->M[c->nlev - 1];
    int all_small = 1, min_n = 1 << 30;
    for (int d = 0; d < F->dim; ++d) {
      if (F->n[d] > pc->coarse_max) all_small = 0;
      if (F->n[d] < min_n) min_n = F->n[d];
    }
    /* a Sommerfeld high side keeps its boundary node n-1 only when n-1-o is even (o the axis's
     * coarsening offset: an even n with o = 1, an odd n with o = 0) */
    int odd_somm = 0;
    for (int d = 0; d < F->dim; ++d)
      if (F->ax[d].somm && ((F->n[d] - 1 - F->ax[d].off) & 1)) odd_somm = 1;
    if (all_small || min_n < 3 || odd_somm) break;
    level_coarse(F, &c->M[c->nlev]);
    if (pc->galerkin && g->dim == 2) level_galerkin(F, &c->M[c->nlev]);
    if (pc->galerkin && g->dim == 3) level_galerkin3d(F, &c->M[c->nlev]);
    c->nlev++;
  }
  if (pc->smoother == 2)
    for (int k = 0; k < c->nlev - 1; ++k) level_ilu(&c->M[k]);
  level_t* C = &c->M[c->nlev - 1];
  c->nco = C->ntot;
  c->lu = malloc(sizeof(cplx) * c->nco * c->nco);
  c->piv = malloc(sizeof(int) * c->nco);
  level_dense(C, c->lu);
  if (lu_factor(c->lu, c->piv, c->nco) != 0) {
    /* singular coarsest operator (a coarse grid at a resonance of M, Section 5.1): no
     * preconditioner can be built, so the caller gets no context rather than NaNs later */
    orc_destroy(c);
    return NULL;
  }
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  level_free(&c->H);
  for (int k = 0; k < c->nlev; ++k) level_free(&c->M[k]);
  free(c->M); free(c->lu); free(c->piv); free(c);
}

int orc_num_levels(const orc_ctx* c) { return c->nlev; }

static const level_t* pick(const orc_ctx* c, int which, int lvl) {
  return which == 0 ? &c->H : &c->M[lvl];
}

void orc_level_shape(const orc_ctx* c, int which, int lvl, int* n_out) {
  const level_t* L = pick(c, which, lvl);
  for (int d = 0; d < 3; ++d) n_out[d] = L->n[d];
}

/* Per-axis tables of a level: gaps (n+1), am, a0, ap (n each), real positions (n). */
void orc_axis_tables(const orc_ctx* c, int which, int lvl, int axis, cplx* gap, cplx* am,
                     cplx* a0, cplx* ap, double* pos) {
  const axis_t* a = &pick(c, which, lvl)->ax[axis];
  memcpy(gap, a->gap, sizeof(cplx) * (a->n + 1));
  memcpy(am, a->am, sizeof(cplx) * a->n);
  memcpy(a0, a->a0, sizeof(cplx) * a->n);
  memcpy(ap, a->ap, sizeof(cplx) * a->n);
  memcpy(pos, a->pos, sizeof(double) * a->n);
}

void orc_level_phi(const orc_ctx* c, int which, int lvl, double* phi, cplx* s) {
  const level_t* L = pick(c, which, lvl);
  memcpy(phi, L->phi, sizeof(double) * L->ntot);
  *s = L->s;
}

/* y = H x (which = 0) or y = M_lvl x (which = 1). */
void orc_level_st9(const orc_ctx* c, int lvl, cplx* out) {
  const level_t* L = pick(c, 1, lvl);
  if (L->st9) memcpy(out, L->st9, sizeof(cplx) * 9 * L->ntot);
  else memset(out, 0, sizeof(cplx) * 9 * L->ntot);
}
void orc_level_st27(const orc_ctx* c, int lvl, cplx* out) {
  const level_t* L = pick(c, 1, lvl);
  if (L->st27) memcpy(out, L->st27, sizeof(cplx) * 27 * L->ntot);
  else memset(out, 0, sizeof(cplx) * 27 * L->ntot);
}

void orc_apply(const orc_ctx* c, int which, int lvl, const cplx* x, cplx* y) {
  level_apply(pick(c, which, lvl), x, y);
}

void orc_dense(const orc_ctx* c, int which, int lvl, cplx* A) { level_dense(pick(c, which, lvl), A); }

/* The ILU(0) factors of preconditioner level lvl (9 entries per unknown, laid out as a Galerkin
 * stencil); 0 when the hierarchy has none there (another smoother, or the coarsest level). */
int orc_ilu_factors(const orc_ctx* c, int lvl, cplx* out) {
  if (lvl < 0 || lvl >= c->nlev || !c->M[lvl].ilu) return 0;
  memcpy(out, c->M[lvl].ilu, sizeof(cplx) * 9 * c->M[lvl].ntot);
  return 1;
}

/* ---- multigrid components (Section 5.1 / 6.1) ----------------------------------------- */

/* One damped-Jacobi sweep: u <- u + omega D^{-1} (f - A u). */
static void jacobi_sweep(const level_t* L, double omega, cplx* u, const cplx* f, cplx* tmp) {
  level_apply(L, u, tmp);
  PAR_FOR2(L->ntot)
  for (int l = 0; l < L->n[2]; ++l)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        long p = lidx(L, i, j, l);
        tmp[p] = u[p] + omega * (f[p] - tmp[p]) / diag_at(L, i, j, l);
      }
  memcpy(u, tmp, sizeof(cplx) * L->ntot);
}

/* One red-black Gauss-Seidel sweep: red points ((i+j+l) even) then black points, each
 * solving its own row with the current neighbour values. */
static void rbgs_sweep(const level_t* L, cplx* u, const cplx* f) {
  for (int colour = 0; colour < 2; ++colour) {
    /* the points of one colour read only the other colour: any order gives the same values */
    PAR_FOR2(L->ntot)
    for (int l = 0; l < L->n[2]; ++l)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i) {
          if (((i + j + l) & 1) != colour) continue;
          long p = lidx(L, i, j, l);
          u[p] = (f[p] - offdiag_at(L, u, i, j, l)) / diag_at(L, i, j, l);
        }
  }
}

/* ---- ILU(0) smoothing (Section 6.1: the smoother of the paper's experiments) --------------
 * Incomplete LU factorisation without fill: L (unit lower) and U (upper) keep the sparsity
 * pattern of the level's matrix A, unknowns in lexicographic order (x fastest), and LU agrees
 * with A at every position of that pattern.  The factors follow the row-wise ("IKJ") form of
 * Gaussian elimination restricted to the pattern (Saad, Iterative Methods for Sparse Linear
 * Systems, ILU(0)): for each row p, for each lower entry k of p in increasing column order,
 * a_pk /= u_kk, then a_pq -= a_pk u_kq for every upper entry q of row k that lies in row p's
 * pattern.  The pattern is the level's stencil: the 5-point Shortley-Weller cross (3 points in
 * 1D), or the 9-point box of a Galerkin level.  One smoothing step is the defect correction
 * u <- u + (LU)^{-1} (f - A u): a forward solve with L, then a backward solve with U. */
static int ilu_in_pattern(const level_t* L, int i, int j, int di, int dj) {
  int ii = i + di, jj = j + dj;
  if (ii < 0 || ii >= L->n[0] || jj < 0 || jj >= L->n[1]) return 0;
  if (di < -1 || di > 1 || dj < -1 || dj > 1) return 0;
  return L->st9 ? 1 : (di == 0 || dj == 0);
}

static int ilu_slot(int di, int dj) { return 3 * (dj + 1) + (di + 1); }

static void level_ilu(level_t* L) {
  L->ilu = calloc(9 * (size_t)imax(L->ntot, 1), sizeof(cplx));
  /* lower neighbours of a row in increasing column order, upper ones of a row */
  static const int lo[4][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}};
  static const int up[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};
  for (int j = 0; j < L->n[1]; ++j)
    for (int i = 0; i < L->n[0]; ++i) {
      cplx a[9] = {0};
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di)
          if (ilu_in_pattern(L, i, j, di, dj)) a[ilu_slot(di, dj)] = entry2d(L, i, j, i + di, j + dj);
      for (int t = 0; t < 4; ++t) {
        int di = lo[t][0], dj = lo[t][1];
        if (!ilu_in_pattern(L, i, j, di, dj)) continue;
        const cplx* uk = L->ilu + 9 * lidx(L, i + di, j + dj, 0);  /* row k, already factored */
        cplx lk = a[ilu_slot(di, dj)] / uk[4];
        a[ilu_slot(di, dj)] = lk;
        for (int v = 0; v < 4; ++v) {
          int ei = up[v][0], ej = up[v][1];
          if (!ilu_in_pattern(L, i + di, j + dj, ei, ej)) continue;   /* not in row k */
          int ti = di + ei, tj = dj + ej;                             /* the column, seen from p */
          if (!ilu_in_pattern(L, i, j, ti, tj)) continue;             /* not in row p: dropped */
          a[ilu_slot(ti, tj)] -= lk * uk[ilu_slot(ei, ej)];
        }
      }
      memcpy(L->ilu + 9 * lidx(L, i, j, 0), a, sizeof(a));
    }
}

static void ilu_sweep(const level_t* L, cplx* u, const cplx* f, cplx* tmp) {
  static const int lo[4][2] = {{-1, -1}, {0, -1}, {1, -1}, {-1, 0}};
  static const int up[4][2] = {{1, 0}, {-1, 1}, {0, 1}, {1, 1}};
  level_apply(L, u, tmp);
  for (long p = 0; p < L->ntot; ++p) tmp[p] = f[p] - tmp[p];
  for (int j = 0; j < L->n[1]; ++j)       /* L y = r, rows in increasing order */
    for (int i = 0; i < L->n[0]; ++i) {
      const cplx* w = L->ilu + 9 * lidx(L, i, j, 0);
      cplx y = tmp[lidx(L, i, j, 0)];
      for (int t = 0; t < 4; ++t)
        if (ilu_in_pattern(L, i, j, lo[t][0], lo[t][1]))
          y -= w[ilu_slot(lo[t][0], lo[t][1])] * tmp[lidx(L, i + lo[t][0], j + lo[t][1], 0)];
      tmp[lidx(L, i, j, 0)] = y;
    }
  for (int j = L->n[1] - 1; j >= 0; --j)  /* U z = y, rows in decreasing order */
    for (int i = L->n[0] - 1; i >= 0; --i) {
      const cplx* w = L->ilu + 9 * lidx(L, i, j, 0);
      cplx z = tmp[lidx(L, i, j, 0)];
      for (int v = 0; v < 4; ++v)
        if (ilu_in_pattern(L, i, j, up[v][0], up[v][1]))
          z -= w[ilu_slot(up[v][0], up[v][1])] * tmp[lidx(L, i + up[v][0], j + up[v][1], 0)];
      tmp[lidx(L, i, j, 0)] = z / w[4];
    }
  for (long p = 0; p < L->ntot; ++p) u[p] += tmp[p];
}

static void smooth(const orc_ctx* c, int lvl, cplx* u, const cplx* f, int sweeps, cplx* tmp) {
  const level_t* L = &c->M[lvl];
  for (int k = 0; k < sweeps; ++k) {
    if (c->pc.smoother == 0) jacobi_sweep(L, c->pc.omega, u, f, tmp);
    else if (c->pc.smoother == 2) ilu_sweep(L, u, f, tmp);
    else rbgs_sweep(L, u, f);
  }
}

/* Full weighting in index space: coarse unknown c gathers fine unknowns 2c+o-1, 2c+o, 2c+o+1
 * (o the axis's coarsening offset, 1 unless a Sommerfeld low side makes it 0) with weights
 * 1/4, 1/2, 1/4 per axis (tensor product); missing neighbours are Dirichlet. */
static void restrict_fw(const level_t* F, const level_t* C, const cplx* r, cplx* fc) {
  static const double w[3] = {0.25, 0.5, 0.25};
  PAR_FOR2(C->ntot)
  for (int cl = 0; cl < C->n[2]; ++cl)
    for (int cj = 0; cj < C->n[1]; ++cj)
      for (int Ii = 0; Ii < C->n[0]; ++Ii) {
        cplx acc = 0;
        for (int dl = (F->dim > 2 ? -1 : 0); dl <= (F->dim > 2 ? 1 : 0); ++dl)
          for (int dj = (F->dim > 1 ? -1 : 0); dj <= (F->dim > 1 ? 1 : 0); ++dj)
            for (int di = -1; di <= 1; ++di) {
              int fi = 2 * Ii + F->ax[0].off + di;
              int fj = F->dim > 1 ? 2 * cj + F->ax[1].off + dj : 0;
              int fl = F->dim > 2 ? 2 * cl + F->ax[2].off + dl : 0;
              if (fi < 0 || fi >= F->n[0] || fj < 0 || fj >= F->n[1] || fl < 0 || fl >= F->n[2]) continue;
              double wt = w[di + 1] * (F->dim > 1 ? w[dj + 1] : 1.0) * (F->dim > 2 ? w[dl + 1] : 1.0);
              acc += wt * r[lidx(F, fi, fj, fl)];
            }
        fc[lidx(C, Ii, cj, cl)] = acc;
      }
}

/* Linear interpolation weights of fine index i from coarse indices (per axis): fine 2c + o is
 * coarse c itself, a fine index between two coarse ones takes half of each (o the coarsening
 * offset; a coarse index outside 0..nc-1 is a Dirichlet zero). */
static int interp1(int i, int nc, int o, int* ci, double* w) {
  int r = i - o;
  if (r >= 0 && !(r & 1)) { ci[0] = r / 2; w[0] = 1.0; return 1; }
  int k = 0;
  int left = (r - 1) / 2, right = (r + 1) / 2;  /* r odd (or -1): its coarse neighbours */
  if (r < 0) { left = -1; right = 0; }
  if (left >= 0 && left < nc) { ci[k] = left; w[k] = 0.5; ++k; }
  if (right >= 0 && right < nc) { ci[k] = right; w[k] = 0.5; ++k; }
  return k;
}

/* u_f += P e_c, bilinear / trilinear interpolation (tensor product of 1D linear). */
static void prolong_add(const level_t* F, const level_t* C, const cplx* ec, cplx* u) {
  PAR_FOR2(F->ntot)
  for (int l = 0; l < F->n[2]; ++l)
    for (int j = 0; j < F->n[1]; ++j)
      for (int i = 0; i < F->n[0]; ++i) {
        int ci[2], cj[2] = {0}, cl[2] = {0};
        double wi[2], wj[2] = {1.0}, wl[2] = {1.0};
        int ni = interp1(i, C->n[0], F->ax[0].off, ci, wi);
        int nj = F->dim > 1 ? interp1(j, C->n[1], F->ax[1].off, cj, wj) : 1;
        int nl = F->dim > 2 ? interp1(l, C->n[2], F->ax[2].off, cl, wl) : 1;
        cplx acc = 0;
        for (int c3 = 0; c3 < nl; ++c3)
          for (int c2 = 0; c2 < nj; ++c2)
            for (int c1 = 0; c1 < ni; ++c1)
              acc += wi[c1] * wj[c2] * wl[c3] * ec[lidx(C, ci[c1], cj[c2], cl[c3])];
        u[lidx(F, i, j, l)] += acc;
      }
}

/* V(nu1, nu2) cycle for M_lvl u = f from a zero initial guess (recursive). */
static void vcycle_rec(const orc_ctx* c, int lvl, const cplx* f, cplx* u) {
  const level_t* L = &c->M[lvl];
  if (lvl == c->nlev - 1) { lu_solve(c->lu, c->piv, c->nco, f, u); return; }
  const level_t* C = &c->M[lvl + 1];
  long n = L->ntot;
  cplx* tmp = malloc(sizeof(cplx) * n);
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* fc = malloc(sizeof(cplx) * C->ntot);
  cplx* ec = malloc(sizeof(cplx) * C->ntot);
  memset(u, 0, sizeof(cplx) * n);
  smooth(c, lvl, u, f, c->pc.nu1, tmp);
  level_apply(L, u, tmp);
  PAR_FOR(n)
  for (long p = 0; p < n; ++p) r[p] = f[p] - tmp[p];
  restrict_fw(L, C, r, fc);
  vcycle_rec(c, lvl + 1, fc, ec);
  prolong_add(L, C, ec, u);
  smooth(c, lvl, u, f, c->pc.nu2, tmp);
  free(tmp); free(r); free(fc); free(ec);
}

/* z ~ M^{-1} r: one V-cycle (identity when there is no preconditioner). */
void orc_vcycle(const orc_ctx* c, const cplx* r, cplx* z) {
  if (c->pc.kind == 0) { memcpy(z, r, sizeof(cplx) * c->H.ntot); return; }
  vcycle_rec(c, 0, r, z);
}

/* Component entry points for tests. */
void orc_smooth(const orc_ctx* c, int lvl, cplx* u, const cplx* f, int sweeps) {
  cplx* tmp = malloc(sizeof(cplx) * c->M[lvl].ntot);
  smooth(c, lvl, u, f, sweeps, tmp);
  free(tmp);
}
void orc_restrict(const orc_ctx* c, int lvl, const cplx* r, cplx* fc) {
  restrict_fw(&c->M[lvl], &c->M[lvl + 1], r, fc);
}
void orc_prolong_add(const orc_ctx* c, int lvl, const cplx* ec, cplx* u) {
  prolong_add(&c->M[lvl], &c->M[lvl + 1], ec, u);
}
void orc_coarse_solve(const orc_ctx* c, const cplx* f, cplx* z) { lu_solve(c->lu, c->piv, c->nco, f, z); }

/* Direct solve of H x = b by dense LU (plain definition of the discrete solution). */
int orc_dense_solve(const orc_ctx* c, const cplx* b, cplx* x) {
  long n = c->H.ntot;
  cplx* A = malloc(sizeof(cplx) * n * n);
  int* piv = malloc(sizeof(int) * n);
  level_dense(&c->H, A);
  int rc = lu_factor(A, piv, n);
  if (rc == 0) lu_solve(A, piv, n, b, x);
  free(A); free(piv);
  return rc;
}

/* ---- Krylov ---------------------------------------------------------------------------- */
static cplx dotc(const cplx* x, const cplx* y, long n) { /* x^H y */
  cplx s = 0;
  for (long i = 0; i < n; ++i) s += conj(x[i]) * y[i];
  return s;
}
static double nrm2(const cplx* x, long n) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
  return sqrt(s);
}
static int finite_c(cplx z) { return isfinite(creal(z)) && isfinite(cimag(z)); }

enum { ST_OK = 0, ST_BREAKDOWN = 4, ST_MAXMV = 5, ST_NAN = 6 };

/* Right-preconditioned Bi-CGSTAB (van der Vorst 1992) from the current x with residual r.
 * Returns ST_OK when the recurrence residual meets tol.  2 preconditioned matvecs per
 * iteration; the half-step exit after s counts one. */
static int bicgstab_run(const orc_ctx* c, const cplx* b, cplx* x, cplx* r, double bn,
                        const orc_solve_opts* o, orc_info* info, double* hist, int hist_cap) {
  long n = c->H.ntot;
  cplx *rh = malloc(sizeof(cplx) * n), *p = calloc(n, sizeof(cplx)), *v = calloc(n, sizeof(cplx));
  cplx *ph = malloc(sizeof(cplx) * n), *sv = malloc(sizeof(cplx) * n), *sh = malloc(sizeof(cplx) * n);
  cplx *t = malloc(sizeof(cplx) * n);
  memcpy(rh, r, sizeof(cplx) * n);
  cplx rho_old = 1, alpha = 1, omega = 1;
  int st = ST_MAXMV;
  for (;;) {
    if (info->matvecs >= o->maxmv) { st = ST_MAXMV; break; }
    cplx rho = dotc(rh, r, n);
    if (!finite_c(rho)) { st = ST_NAN; break; }
    if (rho == 0) { st = ST_BREAKDOWN; break; }
    cplx beta = (rho / rho_old) * (alpha / omega);
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    orc_vcycle(c, p, ph);
    level_apply(&c->H, ph, v);
    info->matvecs++;
    info->iters++;
    cplx rv = dotc(rh, v, n);
    if (!finite_c(rv)) { st = ST_NAN; break; }
    if (rv == 0) { st = ST_BREAKDOWN; break; }
    alpha = rho / rv;
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) sv[i] = r[i] - alpha * v[i];
    double sn = nrm2(sv, n) / bn;
    if (hist && info->matvecs - 1 < hist_cap) hist[info->matvecs - 1] = sn;
    info->rel_res_recur = sn;
    if (!isfinite(sn)) { st = ST_NAN; break; }
    if (sn < o->tol) {
      PAR_FOR(n)
      for (long i = 0; i < n; ++i) x[i] += alpha * ph[i];
      memcpy(r, sv, sizeof(cplx) * n);
      st = ST_OK;
      break;
    }
    if (info->matvecs >= o->maxmv) {
      PAR_FOR(n)
      for (long i = 0; i < n; ++i) x[i] += alpha * ph[i];
      memcpy(r, sv, sizeof(cplx) * n);
      st = ST_MAXMV;
      break;
    }
    orc_vcycle(c, sv, sh);
    level_apply(&c->H, sh, t);
    info->matvecs++;
    cplx ts = dotc(t, sv, n);
    double tt = creal(dotc(t, t, n));
    if (!isfinite(tt) || !finite_c(ts)) { st = ST_NAN; break; }
    if (tt == 0) { st = ST_BREAKDOWN; break; }
    omega = ts / tt;
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * ph[i] + omega * sh[i];
      r[i] = sv[i] - omega * t[i];
    }
    double rn = nrm2(r, n) / bn;
    if (hist && info->matvecs - 1 < hist_cap) hist[info->matvecs - 1] = rn;
    info->rel_res_recur = rn;
    if (!isfinite(rn)) { st = ST_NAN; break; }
    if (rn < o->tol) { st = ST_OK; break; }
    if (omega == 0) { st = ST_BREAKDOWN; break; }
    rho_old = rho;
  }
  free(rh); free(p); free(v); free(ph); free(sv); free(sh); free(t);
  return st;
}

/* Solve the s x s system Mk c = m (column-major Mk[row + s*col]) by Gaussian elimination
 * with partial pivoting; returns -1 when singular. */
static int small_solve(const cplx* Mk, const cplx* m, cplx* out, int s) {
  cplx A[64 * 64], rhs[64];
  for (int i = 0; i < s; ++i) {
    rhs[i] = m[i];
    for (int j = 0; j < s; ++j) A[i * s + j] = Mk[i + s * j];
  }
  for (int k = 0; k < s; ++k) {
    int p = k;
    for (int r = k + 1; r < s; ++r) if (cabs(A[r * s + k]) > cabs(A[p * s + k])) p = r;
    if (A[p * s + k] == 0) return -1;
    if (p != k) {
      for (int j = 0; j < s; ++j) { cplx tt = A[k * s + j]; A[k * s + j] = A[p * s + j]; A[p * s + j] = tt; }
      cplx tt = rhs[k]; rhs[k] = rhs[p]; rhs[p] = tt;
    }
    for (int r = k + 1; r < s; ++r) {
      cplx f = A[r * s + k] / A[k * s + k];
      for (int j = k; j < s; ++j) A[r * s + j] -= f * A[k * s + j];
      rhs[r] -= f * rhs[k];
    }
  }
  for (int r = s - 1; r >= 0; --r) {
    cplx acc = rhs[r];
    for (int j = r + 1; j < s; ++j) acc -= A[r * s + j] * out[j];
    out[r] = acc / A[r * s + r];
  }
  return 0;
}

/* Right-preconditioned IDR(s) (Sonneveld & van Gijzen 2008): the residual is pushed through
 * nested spaces G_j; s differences dR (with their x-space twins dX) are kept, the next
 * residual is made orthogonal to the shadow space P by an s x s solve, and each step costs
 * one preconditioned matvec.  P holds s orthonormal columns (row-major P[j*n + i]). */
static int idr_run(const orc_ctx* c, const cplx* b, cplx* x, cplx* r, double bn, const cplx* P,
                   const orc_solve_opts* o, orc_info* info, double* hist, int hist_cap) {
  long n = c->H.ntot;
  int s = o->s;
  cplx* dR = calloc((size_t)s * n, sizeof(cplx));
  cplx* dX = calloc((size_t)s * n, sizeof(cplx));
  cplx *v = malloc(sizeof(cplx) * n), *z = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
  cplx *q = malloc(sizeof(cplx) * n), *xs = malloc(sizeof(cplx) * n);
  cplx Mk[64 * 64], m[64], cc[64], dm[64];
  cplx omega = 1;
  int st = ST_MAXMV;
  double rn = nrm2(r, n) / bn;
  /* s minimal-residual steps build the first difference vectors */
  for (int k = 0; k < s; ++k) {
    if (info->matvecs >= o->maxmv) { st = ST_MAXMV; goto done; }
    orc_vcycle(c, r, z);
    level_apply(&c->H, z, t);
    info->matvecs++;
    info->iters++;
    double tt = creal(dotc(t, t, n));
    if (!isfinite(tt)) { st = ST_NAN; goto done; }
    if (tt == 0) { st = ST_BREAKDOWN; goto done; }
    omega = dotc(t, r, n) / tt;
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) {
      dX[k * n + i] = omega * z[i];
      dR[k * n + i] = -omega * t[i];
      x[i] += dX[k * n + i];
      r[i] += dR[k * n + i];
    }
    rn = nrm2(r, n) / bn;
    if (hist && info->matvecs - 1 < hist_cap) hist[info->matvecs - 1] = rn;
    info->rel_res_recur = rn;
    if (!isfinite(rn)) { st = ST_NAN; goto done; }
    if (rn < o->tol) { st = ST_OK; goto done; }
  }
  for (int j = 0; j < s; ++j) {
    for (int i = 0; i < s; ++i) Mk[i + s * j] = dotc(&P[(long)i * n], &dR[(long)j * n], n);
    m[j] = dotc(&P[(long)j * n], r, n);
  }
  int oldest = 0;
  for (;;) {
    for (int k = 0; k <= s; ++k) {
      if (info->matvecs >= o->maxmv) { st = ST_MAXMV; goto done; }
      if (small_solve(Mk, m, cc, s) != 0) { st = ST_BREAKDOWN; goto done; }
      PAR_FOR(n)
      for (long i = 0; i < n; ++i) {
        cplx acc = 0;
        for (int j = 0; j < s; ++j) acc -= dR[(long)j * n + i] * cc[j];
        q[i] = acc;
        v[i] = r[i] + acc;
      }
      orc_vcycle(c, v, z);
      /* new x-space difference: -dX c + omega z */
      PAR_FOR(n)
      for (long i = 0; i < n; ++i) {
        cplx acc = 0;
        for (int j = 0; j < s; ++j) acc -= dX[(long)j * n + i] * cc[j];
        xs[i] = acc; /* -dX c, combined below */
      }
      cplx* dRo = &dR[(long)oldest * n];
      cplx* dXo = &dX[(long)oldest * n];
      if (k == 0) {
        level_apply(&c->H, z, t);
        double tt = creal(dotc(t, t, n));
        if (!isfinite(tt)) { st = ST_NAN; goto done; }
        if (tt == 0) { st = ST_BREAKDOWN; goto done; }
        omega = dotc(t, v, n) / tt;
        PAR_FOR(n)
        for (long i = 0; i < n; ++i) {
          dRo[i] = q[i] - omega * t[i];
          dXo[i] = xs[i] + omega * z[i];
        }
      } else {
        PAR_FOR(n)
        for (long i = 0; i < n; ++i) dXo[i] = xs[i] + omega * z[i];
        level_apply(&c->H, dXo, t);
        PAR_FOR(n)
        for (long i = 0; i < n; ++i) dRo[i] = -t[i];
      }
      info->matvecs++;
      info->iters++;
      PAR_FOR(n)
      for (long i = 0; i < n; ++i) { r[i] += dRo[i]; x[i] += dXo[i]; }
      rn = nrm2(r, n) / bn;
      if (hist && info->matvecs - 1 < hist_cap) hist[info->matvecs - 1] = rn;
      info->rel_res_recur = rn;
      if (!isfinite(rn)) { st = ST_NAN; goto done; }
      if (rn < o->tol) { st = ST_OK; goto done; }
      for (int i = 0; i < s; ++i) dm[i] = dotc(&P[(long)i * n], dRo, n);
      for (int i = 0; i < s; ++i) { Mk[i + s * oldest] = dm[i]; m[i] += dm[i]; }
      oldest = (oldest + 1) % s;
    }
  }
done:
  free(dR); free(dX); free(v); free(z); free(t); free(q); free(xs);
  return st;
}

/* Modified Gram-Schmidt on the s rows of P (in place). */
static void orthonormalise(cplx* P, int s, long n) {
  for (int j = 0; j < s; ++j) {
    cplx* pj = &P[(long)j * n];
    for (int i = 0; i < j; ++i) {
      cplx* pi = &P[(long)i * n];
      cplx h = dotc(pi, pj, n);
      PAR_FOR(n)
      for (long k = 0; k < n; ++k) pj[k] -= h * pi[k];
    }
    double nn = nrm2(pj, n);
    PAR_FOR(n)
    for (long k = 0; k < n; ++k) pj[k] /= nn;
  }
}

/* Right-preconditioned restarted GMRES(m) (Saad & Schultz; the paper's remark on testing GMRES
 * in Section 7), from the current x with residual r = b - H x.  Each cycle builds an Arnoldi
 * basis v_0 = r / ||r||, ..., orthogonalising w = H M^{-1} v_j against it by classical
 * Gram-Schmidt applied twice (all inner products of a pass first, then one update), reduces the
 * Hessenberg matrix by complex Givens rotations (the rotated right-hand side gives the residual
 * norm |g_{j+1}| of the least-squares problem), and after m steps -- or when |g_{j+1}| / ||b||
 * < tol -- sets x += M^{-1} (V y) with R y = g and recomputes r = b - H x.  One preconditioned
 * matvec per Arnoldi step. */
static int gmres_run(const orc_ctx* c, const cplx* b, cplx* x, cplx* r, double bn,
                     const orc_solve_opts* o, orc_info* info, double* hist, int hist_cap) {
  long n = c->H.ntot;
  int m = o->s;
  cplx* V = malloc(sizeof(cplx) * (size_t)(m + 1) * n);
  cplx* Hs = calloc((size_t)(m + 1) * m, sizeof(cplx)); /* Hs[i + (m+1) j] */
  double* cs = malloc(sizeof(double) * m);
  cplx* sn = malloc(sizeof(cplx) * m);
  cplx* g = malloc(sizeof(cplx) * (m + 1));
  cplx* h = malloc(sizeof(cplx) * (m + 1));
  cplx* y = malloc(sizeof(cplx) * m);
  cplx *z = malloc(sizeof(cplx) * n), *w = malloc(sizeof(cplx) * n);
  int st = ST_MAXMV;
  for (;;) {
    double beta = nrm2(r, n);
    if (!isfinite(beta)) { st = ST_NAN; break; }
    if (beta / bn < o->tol) { st = ST_OK; break; }
    if (info->matvecs >= o->maxmv) { st = ST_MAXMV; break; }
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= m; ++i) g[i] = 0;
    g[0] = beta;
    int k = 0, done = 0;
    st = ST_MAXMV;
    for (int j = 0; j < m; ++j) {
      if (info->matvecs >= o->maxmv) { st = ST_MAXMV; done = 1; break; }
      cplx* vj = V + (size_t)j * n;
      orc_vcycle(c, vj, z);
      level_apply(&c->H, z, w);
      info->matvecs++;
      info->iters++;
      cplx* col = Hs + (size_t)(m + 1) * j;
      for (int i = 0; i <= j; ++i) col[i] = 0;
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i <= j; ++i) h[i] = dotc(V + (size_t)i * n, w, n);
        PAR_FOR(n)
        for (long q = 0; q < n; ++q) {
          cplx acc = 0;
          for (int i = 0; i <= j; ++i) acc += h[i] * V[(size_t)i * n + q];
          w[q] -= acc;
        }
        for (int i = 0; i <= j; ++i) col[i] += h[i];
      }
      double hn = nrm2(w, n);
      /* earlier rotations on the new column, then the one that annihilates hn */
      for (int i = 0; i < j; ++i) {
        cplx a = col[i], bb = col[i + 1];
        col[i] = cs[i] * a + sn[i] * bb;
        col[i + 1] = -conj(sn[i]) * a + cs[i] * bb;
      }
      cplx a = col[j];
      double aa = cabs(a);
      if (hn == 0) { cs[j] = 1; sn[j] = 0; }
      else if (aa == 0) { cs[j] = 0; sn[j] = 1; col[j] = hn; }
      else {
        double t = hypot(aa, hn);
        cs[j] = aa / t;
        sn[j] = (a / aa) * (hn / t);
        col[j] = (a / aa) * t;
      }
      col[j + 1] = 0;
      g[j + 1] = -conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      double est = cabs(g[j + 1]) / bn;
      if (hist && info->matvecs - 1 < hist_cap) hist[info->matvecs - 1] = est;
      info->rel_res_recur = est;
      if (!isfinite(est) || !isfinite(hn)) { st = ST_NAN; done = 1; break; }
      if (est < o->tol || hn == 0) { st = ST_OK; done = 1; break; }
      PAR_FOR(n)
      for (long q = 0; q < n; ++q) V[(size_t)(j + 1) * n + q] = w[q] / hn;
    }
    /* x += M^{-1} V y, R y = g (upper triangular k x k) */
    for (int i = k - 1; i >= 0; --i) {
      cplx acc = g[i];
      for (int l = i + 1; l < k; ++l) acc -= Hs[i + (size_t)(m + 1) * l] * y[l];
      y[i] = acc / Hs[i + (size_t)(m + 1) * i];
    }
    if (k > 0) {
      PAR_FOR(n)
      for (long q = 0; q < n; ++q) {
        cplx acc = 0;
        for (int i = 0; i < k; ++i) acc += y[i] * V[(size_t)i * n + q];
        w[q] = acc;
      }
      orc_vcycle(c, w, z);
      PAR_FOR(n)
      for (long q = 0; q < n; ++q) x[q] += z[q];
    }
    level_apply(&c->H, x, r);
    PAR_FOR(n)
    for (long q = 0; q < n; ++q) r[q] = b[q] - r[q];
    if (done) break;
  }
  free(V); free(Hs); free(cs); free(sn); free(g); free(h); free(y); free(z); free(w);
  return st;
}

/* Full solve H x = b from x = 0 (the stopping rule of Section 6.2 is relative to d_0 = b),
 * then the true residual b - H x is recomputed; if it misses tol the method restarts from
 * the current x (at most max_restarts times).  shadow: s x n raw random vectors for IDR. */
int orc_solve(const orc_ctx* c, const cplx* b, cplx* x, const orc_solve_opts* o,
              const cplx* shadow, orc_info* info, double* hist, int hist_cap) {
  long n = c->H.ntot;
  memset(info, 0, sizeof(*info));
  memset(x, 0, sizeof(cplx) * n);
  double bn = nrm2(b, n);
  if (!isfinite(bn)) { info->status = ST_NAN; return ST_NAN; }
  if (bn == 0) { info->status = ST_OK; return ST_OK; }
  if (o->method == 1 && (o->s < 1 || o->s > 64 || !shadow)) { info->status = 1; return 1; }
  if (o->method == 2 && (o->s < 1 || o->s > 128)) { info->status = 1; return 1; }
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* P = NULL;
  if (o->method == 1) {
    P = malloc(sizeof(cplx) * (size_t)o->s * n);
    memcpy(P, shadow, sizeof(cplx) * (size_t)o->s * n);
    orthonormalise(P, o->s, n);
  }
  memcpy(r, b, sizeof(cplx) * n);
  int st;
  for (;;) {
    st = o->method == 0 ? bicgstab_run(c, b, x, r, bn, o, info, hist, hist_cap)
       : o->method == 1 ? idr_run(c, b, x, r, bn, P, o, info, hist, hist_cap)
                        : gmres_run(c, b, x, r, bn, o, info, hist, hist_cap);
    /* true residual */
    level_apply(&c->H, x, r);
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    info->rel_res_true = nrm2(r, n) / bn;
    if (st != ST_OK) break;
    if (info->rel_res_true < o->tol) break;
    if (info->restarts >= o->max_restarts) { st = ST_MAXMV; break; }
    info->restarts++;
  }
  info->status = st;
  free(r); free(P);
  return st;
}

/* ---- choosing the CSL shift / CSG angle (Section 7, remark on choosing the parameters) --- */

/* Multigrid as a stationary solver of M u = f (M = the preconditioner's finest operator) from
 * u = 0: each cycle u <- u + V(f - M u).  Returns the number of cycles after which
 * ||f - M u|| <= reduction ||f|| (0 when f = 0), or -1 when that does not happen within
 * max_cycles, or the residual grows past 1e6 ||f|| or stops being finite.  hist[k-1] (if
 * given) receives ||f - M u|| / ||f|| after cycle k, for the cycles run. */
int orc_mg_iterate(const orc_ctx* c, const cplx* f, int max_cycles, double reduction, cplx* u,
                   double* hist) {
  long n = c->H.ntot;
  memset(u, 0, sizeof(cplx) * n);
  if (c->pc.kind == 0) return -1;
  double fn = nrm2(f, n);
  if (fn == 0) return 0;
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* z = malloc(sizeof(cplx) * n);
  memcpy(r, f, sizeof(cplx) * n);
  int result = -1;
  for (int k = 1; k <= max_cycles; ++k) {
    vcycle_rec(c, 0, r, z);
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) u[i] += z[i];
    level_apply(&c->M[0], u, r);
    PAR_FOR(n)
    for (long i = 0; i < n; ++i) r[i] = f[i] - r[i];
    double rel = nrm2(r, n) / fn;
    if (hist) hist[k - 1] = rel;
    if (rel <= reduction) { result = k; break; }
    if (!(rel <= 1e6)) break; /* diverging or not finite */
  }
  free(r); free(z);
  return result;
}

/* From the starting preconditioner (CSL: its imaginary shift is the parameter; CSG: its angle
 * theta_beta), the parameter is multiplied by `factor` (0 < factor < 1) from one trial to the
 * next for as long as multigrid on the resulting M converges within max_cycles (orc_mg_iterate
 * with right-hand side f); *out receives the last preconditioner that converged.  params[t] and
 * cycles[t] record each trial (cycles -1 = did not converge).  Returns the number of trials run;
 * *status = 0 when the start converged, else 5 and *out = the start. */
int orc_select_precond(const orc_grid* g, const double* phi, const double* phi_im, double k0,
                       const orc_precond* start,
                       const cplx* f, int max_cycles, double reduction, double factor,
                       int max_trials, orc_precond* out, double* params, int* cycles, int* status) {
  *out = *start;
  *status = 5;
  long n = 1;
  for (int d = 0; d < g->dim; ++d) {
    int lo = g->n_layer[d][0], hi = g->n_layer[d][1];
    n *= g->n_int[d] - 2 + (lo > 0 ? lo + 1 : lo < 0 ? 1 : 0) + (hi > 0 ? hi + 1 : hi < 0 ? 1 : 0);
  }
  cplx* u = malloc(sizeof(cplx) * n);
  orc_precond pc = *start;
  double p = start->kind == 1 ? start->shift_im : start->theta_beta;
  int t = 0;
  for (; t < max_trials; ++t) {
    if (t > 0) p *= factor;
    if (pc.kind == 1) pc.shift_im = p; else pc.theta_beta = p;
    orc_ctx* c = orc_create(g, phi, phi_im, k0, &pc);
    int k = c ? orc_mg_iterate(c, f, max_cycles, reduction, u, NULL) : -1; /* singular: no M */
    orc_destroy(c);
    params[t] = p;
    cycles[t] = k;
    if (k < 0) { ++t; break; }
    *out = pc;
    *status = 0;
  }
  free(u);
  return t;
}
