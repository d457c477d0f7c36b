"""Seeded synthetic inputs for the ECS Helmholtz solver and its oracle.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's tests.
It holds no arithmetic of the method itself: it only describes problems (grid sizes,
layer widths, angles, wave-number fields phi = k(x)^2 sampled at the real node
positions, right-hand sides, Krylov shadow vectors) and draws the random numbers
those descriptions need, from numpy's seeded PCG64 generator.

Node positions follow the problem statement of the paper (Section 2, the ECS map
z(x) = (x - r) e^{i theta} + r on the layers, and Section 3's vertex-centred grid):
interior nodes sit at x = 0, h, ..., L (h = L / (n_int - 1)); a layer of n_l nodes
continues past each end with real positions -m h and L + m h (m = 1..n_l); a side with
n_l = 0 is a Dirichlet wall, whose end node is not an unknown.  The wave number is
evaluated at these real positions (the layers continue the coordinate, not the
potential; Section 1 on ECS and non-analytic potentials).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20091201

# Preconditioner kinds and solver codes, mirrored by both the C-ABI and the oracle.
PC_NONE, PC_CSL, PC_CSG_UNIFORM, PC_CSG_INTERIOR = 0, 1, 2, 3
SM_JACOBI, SM_RBGS, SM_ILU = 0, 1, 2
BICGSTAB, IDR, GMRES = 0, 1, 2  # GMRES: SolveOpts.s is the restart length m


@dataclasses.dataclass
class Problem:
    """One ECS Helmholtz instance: grid, layers, wave-number field and RHS."""

    dim: int
    n_int: Tuple[int, int, int]
    n_layer: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]]
    extent: Tuple[float, float, float]
    theta_gamma: float
    phi: Optional[np.ndarray]  # k(x)^2 at the unknowns (float64, x fastest) or None for constant
    k0: float                  # constant wave number when phi is None
    b: np.ndarray              # right-hand side (complex128, x fastest)
    name: str = ""
    ecs_ramp: int = 0          # > 1: the layer contour turns over this many widths (smooth ECS)
    phi_im: Optional[np.ndarray] = None  # imaginary part of phi (k at complex node positions)

    @property
    def shape(self) -> Tuple[int, ...]:
        """Unknowns per axis, x first."""
        return tuple(axis_unknowns(self.n_int[a], self.n_layer[a]) for a in range(self.dim))

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def h(self, axis: int = 0) -> float:
        return self.extent[axis] / (self.n_int[axis] - 1)


def axis_unknowns(n_int: int, nl: Tuple[int, int]) -> int:
    """Number of unknowns along one axis (interior nodes, minus Dirichlet walls, plus layers; a
    side of -1 is a Sommerfeld boundary whose node is an unknown)."""
    lo, hi = nl
    return n_int - 2 + (lo + 1 if lo > 0 else (1 if lo < 0 else 0)) + (hi + 1 if hi > 0 else (1 if hi < 0 else 0))


def axis_positions(n_int: int, nl: Tuple[int, int], extent: float) -> np.ndarray:
    """Real coordinates of the unknowns along one axis (layers continue the real axis)."""
    h = extent / (n_int - 1)
    lo, hi = nl
    xs: List[float] = []
    xs += [-m * h for m in range(lo, 0, -1)]
    first = 0 if lo != 0 else 1
    last = n_int - 1 if hi != 0 else n_int - 2
    xs += [j * h for j in range(first, last + 1)]
    xs += [extent + m * h for m in range(1, hi + 1)]
    return np.asarray(xs, dtype=np.float64)


def axis_positions_complex(n_int: int, nl: Tuple[int, int], extent: float, theta: float,
                           ramp: int = 0) -> np.ndarray:
    """Complex coordinates of the unknowns along one axis: real in the interior, and in a layer of
    m nodes the turning point plus the sum of the layer widths h e^{i theta min(q, R) / R} (R the
    ramp, sharp contour for R <= 1) up to the node -- the ECS map of Section 2."""
    h = extent / (n_int - 1)
    lo, hi = nl

    def depth(m):
        if ramp > 1:
            return sum(h * np.exp(1j * theta * min(q, ramp) / ramp) for q in range(1, m + 1))
        return m * h * np.exp(1j * theta)

    zs: List[complex] = [-depth(m) for m in range(lo, 0, -1)]
    first = 0 if lo != 0 else 1
    last = n_int - 1 if hi != 0 else n_int - 2
    zs += [complex(j * h) for j in range(first, last + 1)]
    zs += [extent + depth(m) for m in range(1, hi + 1)] if hi > 0 else []
    return np.asarray(zs, dtype=np.complex128)


def mesh_complex(p: Problem) -> List[np.ndarray]:
    """Like mesh(), with the complex node coordinates of the layers."""
    axes = [axis_positions_complex(p.n_int[a], p.n_layer[a], p.extent[a], p.theta_gamma, p.ecs_ramp)
            for a in range(p.dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]


def mesh(p: Problem) -> List[np.ndarray]:
    """Broadcastable real coordinate arrays, ordered so that arr.ravel() is x-fastest."""
    axes = [axis_positions(p.n_int[a], p.n_layer[a], p.extent[a]) for a in range(p.dim)]
    # index order (z, y, x) so that C-order ravel is x-fastest
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]


def interior_node_index(p: Problem, axis: int, j: int) -> int:
    """0-based unknown index along `axis` of interior grid node j (0..n_int-1)."""
    lo = p.n_layer[axis][0]
    return j + lo if lo > 0 else (j if lo < 0 else j - 1)


def _dims3(dim, v):
    v = list(v) + [v[-1]] * (3 - len(v))
    return tuple(v[:3])


def make_problem(dim: int, n_int: int | Sequence[int], n_l: int | Sequence, *, extent=1.0,
                 theta_gamma=0.5, k0: float = 0.0, phi_kind: str = "const", bump_amp=0.3,
                 bump_width2=0.02, bump_centre=(0.5, 0.5, 0.5), rhs: str = "point",
                 rhs_width_h: float = 2.0, seed: int = BASE_SEED, name: str = "",
                 phi_fn=None, rhs_fn=None, ecs_ramp: int = 0, complex_z: bool = False) -> Problem:
    """Build a seeded synthetic instance shaped like the paper's model problems.

    n_l: int (all sides), one (lo, hi) pair for every axis, or per-axis (lo, hi) pairs.
    phi_kind: "const" (k = k0), "bump" (k = k0 (1 + amp exp(-|x - c|^2 / width2))), or "field"
         (phi = phi_fn(x, y[, z]) at the real node positions).
    ecs_ramp: 0 = sharp ECS contour; R > 1 = the contour turns by theta_gamma / R per layer width
         over the first R widths (the smooth transition of the paper's Section 7 remark).
    complex_z: evaluate the "bump" / "field" phi at the complex node coordinates of the layers (the
         analytic continuation of k; |x - c|^2 becomes sum (z - c)^2), giving phi_im; False reads k
         at the real positions.
    rhs: "point" (value 1 at the interior node floor((n_int-1)/2) per axis, as in MP1),
         "gauss" (exp(-|x - x_s|^2 / (2 sigma^2)), sigma = rhs_width_h * h, x_s uniform in
         [0.1, 0.9]^d from the seed), "random" (complex normal entries), "zero", "field"
         (rhs_fn(x, y[, z]) at the real node positions).
    """
    rng = np.random.default_rng(seed)
    ni = _dims3(dim, [n_int] if np.isscalar(n_int) else list(n_int))
    if np.isscalar(n_l):
        nl = tuple((int(n_l), int(n_l)) for _ in range(3))
    elif len(n_l) == 2 and all(np.isscalar(v) for v in n_l):
        nl = tuple((int(n_l[0]), int(n_l[1])) for _ in range(3))
    else:
        nl_list = [tuple(x) for x in n_l]
        nl = _dims3(dim, nl_list)
    ext = _dims3(dim, [extent] if np.isscalar(extent) else list(extent))
    p = Problem(dim=dim, n_int=tuple(int(x) for x in ni), n_layer=nl,
                extent=tuple(float(x) for x in ext), theta_gamma=float(theta_gamma),
                phi=None, k0=float(k0), b=np.zeros(0, np.complex128), name=name,
                ecs_ramp=int(ecs_ramp))
    shape = p.shape
    X = mesh(p)
    Z = mesh_complex(p) if complex_z else X
    if phi_kind == "bump":
        r2 = sum((Z[a] - bump_centre[a] * ext[a]) ** 2 for a in range(dim))
        k = k0 * (1.0 + bump_amp * np.exp(-r2 / bump_width2))
        ph = (k * k).ravel()
    elif phi_kind == "field":
        ph = np.broadcast_to(phi_fn(*Z[:dim]), shape[::-1]).ravel()
    elif phi_kind != "const":
        raise ValueError(phi_kind)
    if phi_kind != "const":
        p.phi = np.ascontiguousarray(np.real(ph), dtype=np.float64)
        if complex_z:
            p.phi_im = np.ascontiguousarray(np.imag(ph), dtype=np.float64)
    n = int(np.prod(shape))
    if rhs == "point":
        b = np.zeros(shape[::-1], np.complex128)
        idx = tuple(interior_node_index(p, a, (ni[a] - 1) // 2) for a in range(dim))
        b[idx[::-1]] = 1.0
        p.b = b.ravel()
    elif rhs == "gauss":
        xs = rng.uniform(0.1, 0.9, size=dim) * np.asarray(ext[:dim])
        sig = rhs_width_h * p.h(0)
        r2 = sum((X[a] - xs[a]) ** 2 for a in range(dim))
        p.b = np.ascontiguousarray(np.exp(-r2 / (2 * sig * sig)).ravel().astype(np.complex128))
    elif rhs == "random":
        p.b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    elif rhs == "zero":
        p.b = np.zeros(n, np.complex128)
    elif rhs == "field":
        p.b = np.ascontiguousarray(np.broadcast_to(rhs_fn(*X[:dim]), shape[::-1]).ravel().astype(np.complex128))
    else:
        raise ValueError(rhs)
    return p


def shadow_space(n: int, s: int, seed: int = BASE_SEED + 17) -> np.ndarray:
    """Raw random shadow vectors for IDR(s): an (s, n) complex128 array, row j = vector j.

    Entries are independent with real and imaginary parts uniform in [-1, 1).  The solver
    orthonormalises them itself; only the random draw lives here.
    """
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1, 1, (s, n)) + 1j * rng.uniform(-1, 1, (s, n))).astype(np.complex128)


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ---- the workloads the solver is measured on -------------------------------------------

def workload_small_2d(seed: int = BASE_SEED) -> Problem:
    """64^2 interior + 16-point ECS layer per side (theta_gamma 0.5), k = 20, centre point source."""
    return make_problem(2, 64, 16, theta_gamma=0.5, k0=20.0, rhs="point", seed=seed,
                        name="2d-64sq-L16-k20-point")


def workload_2d_512(seed: int = BASE_SEED) -> Problem:
    """512^2 interior + 64-point ECS layers, kh = 0.5, Gaussian-bump k(x), Gaussian source (sigma 2h)."""
    h = 1.0 / 511.0
    k0 = 0.5 / h
    return make_problem(2, 512, 64, theta_gamma=0.5, k0=k0, phi_kind="bump", bump_amp=0.3,
                        bump_width2=0.02, bump_centre=(0.5, 0.5), rhs="gauss", rhs_width_h=2.0,
                        seed=seed, name="2d-512sq-L64-kh0.5-bump-gauss")


def workload_3d_128(seed: int = BASE_SEED) -> Problem:
    """128^3 interior + 16-point ECS layers, k = 40, centre point source."""
    return make_problem(3, 128, 16, theta_gamma=0.5, k0=40.0, rhs="point", seed=seed,
                        name="3d-128cube-L16-k40-point")


def workload_mp1(k: float = 160.0, n_int: int = 257, n_l: int = 64, theta_gamma: float = np.pi / 6) -> Problem:
    """The paper's model problem 1 (Section 4, eq. "MP1"): constant k on the unit square with a unit
    point source at the centre node, absorbing on all four edges -- ECS layers of n_l nodes per side
    (theta_gamma = pi/6), or, with n_l = -1, the first-order Sommerfeld condition on every edge (the
    boundary nodes are unknowns).  Defaults: k = 160 on 257 nodes per axis (h = 1/256, kh = 0.625,
    the accuracy limit; the paper's 256 cell-centred points, its Table MP1)."""
    tag = "-sommerfeld" if n_l < 0 else f"-L{n_l}"
    return make_problem(2, n_int, n_l, theta_gamma=theta_gamma, k0=k, rhs="point",
                        name=f"mp1-k{k:g}-{n_int - 1}sq{tag}")


def workload_mp2(nu: float = 7.0, k: float = 2.0, n_int: int = 385, n_l: int = 128, r: float = 50.0,
                 theta_gamma: float = np.pi / 6, ecs_ramp: int = 0) -> Problem:
    """The paper's model problem 2 (Section 4, eq. "MP2"): phi = nu (e^{-x^2} + e^{-y^2}) + k^2,
    source chi = e^{-(x^2 + y^2)} on [0, r]^2, Dirichlet on the south / west edges (x = 0, y = 0) and
    ECS layers of n_l nodes on the east / north edges (n_l = -1: the first-order Sommerfeld
    condition there instead, eq. "BC").  Defaults: the paper's 384^2 interior grid with 128 layer
    nodes (512^2 unknowns; 384^2 with Sommerfeld edges).  ecs_ramp > 1 turns the contour gradually
    (Section 7's smooth ECS transition)."""
    tag = f"-ramp{ecs_ramp}" if ecs_ramp > 1 else ""
    if n_l < 0:
        tag += "-sommerfeld"
    return make_problem(2, n_int, ((0, n_l), (0, n_l)), extent=r, theta_gamma=theta_gamma, k0=k,
                        ecs_ramp=ecs_ramp,
                        phi_kind="field", rhs="field", name=f"mp2-nu{nu:g}-k{k:g}-{n_int - 1}sq-L{n_l}{tag}",
                        phi_fn=lambda x, y: nu * (np.exp(-x * x) + np.exp(-y * y)) + k * k,
                        rhs_fn=lambda x, y: np.exp(-(x * x + y * y)))


def workload_mp3(r: float = 90.0, k: float = 2.0, n_int: int = 1025, n_l: int = 256,
                 theta_gamma: float = np.pi / 6) -> Problem:
    """The paper's model problem 3 (Section 4, eq. "MP3"): phi = 1/x + 1/y + k^2 (singular at the
    origin, which is a Dirichlet node here, so no unknown sits on it), chi = e^{-(x^2 + y^2)} on
    [0, r]^2, Dirichlet south / west, ECS layers east / north (n_l = -1: Sommerfeld edges).
    Defaults: r = 90 with the paper's 1024^2 interior grid and 256 layer nodes (1280^2 unknowns)."""
    tag = "-sommerfeld" if n_l < 0 else ""
    return make_problem(2, n_int, ((0, n_l), (0, n_l)), extent=r, theta_gamma=theta_gamma, k0=k,
                        phi_kind="field", rhs="field", name=f"mp3-r{r:g}-k{k:g}-{n_int - 1}sq-L{n_l}{tag}",
                        phi_fn=lambda x, y: 1.0 / x + 1.0 / y + k * k,
                        rhs_fn=lambda x, y: np.exp(-(x * x + y * y)))


def workload_batch_2d(count: int = 256, seed: int = BASE_SEED) -> List[Problem]:
    """Uneven batch: n_int in {63,127,255,511}, layers 16..32, kh in [0.3,0.6], const or bump k."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n_int = int(rng.choice([63, 127, 255, 511]))
        n_l = int(rng.integers(16, 33))
        kh = float(rng.uniform(0.3, 0.6))
        k0 = kh * (n_int - 1)
        bump = bool(rng.integers(0, 2))
        amp = float(rng.uniform(0.0, 0.4)) if bump else 0.0
        cen = tuple(rng.uniform(0.2, 0.8, 2))
        p = make_problem(2, n_int, n_l, theta_gamma=0.5, k0=k0,
                         phi_kind="bump" if bump else "const", bump_amp=amp,
                         bump_centre=(cen[0], cen[1]), rhs="point", seed=seed + 1 + i,
                         name=f"batch{i}")
        # point source at a random interior node instead of the centre
        b = np.zeros(p.shape[::-1], np.complex128)
        idx = tuple(interior_node_index(p, a, int(rng.integers(1, n_int - 1))) for a in range(2))
        b[idx[::-1]] = 1.0
        p.b = b.ravel()
        out.append(p)
    return out


@dataclasses.dataclass
class ServeRequest:
    arrival_s: float          # offset from the start of the stream
    problem: Problem
    rhs: np.ndarray           # nrhs x N complex128 point sources


def workload_serve(count: int = 32, rate_hz: float = 200.0, frac_3d: float = 0.5,
                   seed: int = BASE_SEED + 5) -> List[ServeRequest]:
    """Poisson-arrival request stream: exponential gaps of mean 1/rate_hz; 2D requests with
    n_int in {127, 255, 511, 1023}, 3D requests with n_int in {64, 96, 128, 160} (3D with
    probability frac_3d); layers of 16..32 nodes per side; kh uniform in [0.3, 0.6]; k constant
    or (probability 1/2) a Gaussian bump of amplitude 0..0.4 at a seeded centre; 1..8 right-hand
    sides per request, each a unit point source at a seeded interior node."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        dim = 3 if rng.uniform() < frac_3d else 2
        n_int = int(rng.choice([127, 255, 511, 1023] if dim == 2 else [64, 96, 128, 160]))
        n_l = int(rng.integers(16, 33))
        kh = float(rng.uniform(0.3, 0.6))
        bump = bool(rng.integers(0, 2))
        amp = float(rng.uniform(0.0, 0.4)) if bump else 0.0
        cen = tuple(rng.uniform(0.2, 0.8, 3))
        p = make_problem(dim, n_int, n_l, theta_gamma=0.5, k0=kh * (n_int - 1),
                         phi_kind="bump" if bump else "const", bump_amp=amp, bump_centre=cen[:dim],
                         rhs="point", seed=seed + 1 + i, name=f"serve{i}-{dim}d-{n_int}")
        nrhs = int(rng.integers(1, 9))
        rhs = np.zeros((nrhs,) + p.shape[::-1], np.complex128)
        for k in range(nrhs):
            idx = tuple(interior_node_index(p, a, int(rng.integers(1, n_int - 1))) for a in range(dim))
            rhs[(k,) + idx[::-1]] = 1.0
        out.append(ServeRequest(t, p, rhs.reshape(nrhs, -1)))
    return out


@dataclasses.dataclass
class Precond:
    """Description of the preconditioner (plain parameters, no arithmetic).

    kind: PC_NONE (identity), PC_CSL (M = -(L + beta^2 k^2), beta^2 = shift),
    PC_CSG_UNIFORM (every mesh width times e^{i theta_beta}), PC_CSG_INTERIOR (interior
    widths only).  V(nu1, nu2) cycles with damped Jacobi (omega), red-black Gauss-Seidel or
    ILU(0) (1D / 2D).
    """

    kind: int = PC_CSG_UNIFORM
    theta_beta: float = 0.3
    shift: complex = 1.0 + 0.5j
    nu1: int = 1
    nu2: int = 1
    smoother: int = SM_RBGS
    omega: float = 0.5
    max_levels: int = 32
    coarse_max: int = 8
    galerkin: bool = False   # 2D, omega-Jacobi or ILU(0): coarse operators R A P instead of rediscretised


@dataclasses.dataclass
class SolveOpts:
    method: int = BICGSTAB
    s: int = 4
    tol: float = 1e-6
    maxmv: int = 2000
    max_restarts: int = 3
