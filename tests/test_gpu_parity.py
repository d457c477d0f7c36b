"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element.

Tolerances, derived from the arithmetic:
  - FP64 kernels: the same formulas summed in a different order differ by a few ulps of the
    largest term; relative 1e-12 of the vector norm (stencil terms cancel up to ~1/h^2 * |x|
    against |H x|, so the bound is taken against |coefficients| * |x|).
  - FP32 multigrid: one sweep rounds every term to 2^-24 ~ 6e-8 relative; a V-cycle chains a
    few dozen such operations through the levels, so 2e-5 relative.
  - Krylov: two FP64 runs with different rounding follow the same residual history for the
    first steps and then drift; the solutions both satisfy ||b - Hx|| <= tol ||b||, so they
    agree to about cond * tol; at tol 1e-10 the bar is 1e-9 relative, matvec counts within 2.
"""
import os

import numpy as np
import pytest
import torch

import helm_inputs as hi
from oracle import Oracle

pytestmark = pytest.mark.gpu

from paper_0912_0180_gb300 import _lib as L  # noqa: E402
from paper_0912_0180_gb300.helm import Helm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def cu(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def relmax(a, b):
    """Element-wise: max_i |a_i - b_i| / max_i |b_i|."""
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300) if len(b) else 0.0


def check(a, ref, tol, rows=None):
    """a matches ref within tol both as a relative 2-norm and element by element
    (max |a_i - ref_i| / max |ref_i|); with `rows` (boolean mask) also on those rows alone,
    against their own largest reference entry, so that a wrong boundary or turning-point row
    cannot hide among the many interior rows."""
    a = np.asarray(a).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    assert rel(a, ref) < tol, ("2-norm", rel(a, ref), tol)
    assert relmax(a, ref) < tol, ("max-norm", relmax(a, ref), tol)
    if rows is not None and rows.any():
        assert relmax(a[rows], ref[rows]) < tol, ("edge rows", relmax(a[rows], ref[rows]), tol)


def edge_rows(o, lvl, which=1):
    """Rows of level `lvl` whose Shortley-Weller row is not the uniform interior one on some axis:
    the ECS layer rows, the turning points, the rows next to a coarse width that sums an uneven
    number of fine widths, and the Sommerfeld boundary rows (from the oracle's own tables)."""
    shape = o.level_shape(which, lvl)
    masks = []
    for a, n in enumerate(shape):
        t = o.axis_tables(which, lvl, a)
        mid = n // 2
        uni = (np.isclose(t["am"], t["am"][mid], rtol=1e-12, atol=0) &
               np.isclose(t["ap"], t["ap"][mid], rtol=1e-12, atol=0) &
               np.isclose(t["a0"], t["a0"][mid], rtol=1e-12, atol=0))
        masks.append(~uni)
    m = np.zeros(shape[::-1], bool)  # indexed [l][j][i], x fastest when flattened
    for a, ma in enumerate(masks):
        sh = [1] * len(shape)
        sh[len(shape) - 1 - a] = len(ma)
        m |= ma.reshape(sh)
    return m.reshape(-1)


# Cases whose GPU matvec count differs from the oracle's by more than 2 and is checked against
# the oracle's own count range under rounding-level perturbations of b (printed with -s).
SPREAD_CASES = []


def counts_match(o, b, opts, gpu, ref, shadow=None, eps=(1e-16,) * 15 + (1e-15,) * 15 + (1e-14,) * 15, seed=99):
    """Matvec-count bar of a solve at a tight tolerance: within 2 of the oracle's count, or else
    within 2 of the range of counts the oracle itself reaches when b changes by 1e-16 .. 1e-14
    relative (1 to 100 units of its rounding; 15 runs each).  Near the stopping tolerance two FP64
    runs that round differently (another summation order, fused multiply-adds) follow different
    Krylov histories, and the step at which the recurrence first crosses tol moves; the perturbed
    oracle runs measure how far it moves for this problem (on the most sensitive case, a
    Sommerfeld Bi-CGSTAB solve, by +-25 around 230 already at 1e-16)."""
    if abs(gpu - ref) <= 2:
        return
    rng = np.random.default_rng(seed)
    counts = [ref]
    for e in eps:
        bp = b * (1 + e * rng.standard_normal(len(b)))
        counts.append(o.solve(bp, opts, shadow=shadow)[1]["matvecs"])
    where = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    SPREAD_CASES.append((where, gpu, ref, min(counts), max(counts)))
    print(f"\ncount bar by the oracle's spread: {where}: GPU {gpu}, oracle {ref}, "
          f"perturbed {min(counts)}..{max(counts)} ({len(counts) - 1} runs)")
    assert min(counts) - 2 <= gpu <= max(counts) + 2, (gpu, counts)


CASES = [
    # dim, n_int, layers, theta, k0, phi kind
    (1, 50, (7, 5), 0.5, 9.0, "const"),
    (2, 33, 6, 0.5, 15.0, "const"),
    (2, (40, 29), ((5, 0), (3, 8)), 0.4, 12.0, "bump"),
    (2, 64, 16, 0.5, 20.0, "const"),
    (3, 13, 3, 0.5, 6.0, "const"),
    (3, (12, 9, 10), ((2, 3), (0, 2), (3, 0)), 0.5, 5.0, "bump"),
]


def _problem(case, rhs="random", seed=11):
    dim, n_int, nl, th, k0, kind = case
    return hi.make_problem(dim, n_int, nl, theta_gamma=th, k0=k0, phi_kind=kind, rhs=rhs, seed=seed,
                           bump_centre=(0.4, 0.6, 0.5))


@pytest.mark.parametrize("case", CASES)
def test_helmholtz_apply_fp64(case):
    p = _problem(case)
    o = Oracle(p)
    h = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    x = hi.random_vector(p.n, 3)
    y = h.apply(cu(x)).cpu().numpy()
    ref = o.apply(x)
    check(y, ref, 1e-12, edge_rows(o, 0, which=0))
    # complex64 input: exact upcast, then FP64 arithmetic
    x32 = x.astype(np.complex64)
    y32 = h.apply(cu(x32, torch.complex64)).cpu().numpy()
    check(y32, o.apply(x32.astype(np.complex128)), 1e-12)
    h.close()


PCS = [
    hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS),
    hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5, nu1=2, nu2=1),
    hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.8),
    hi.Precond(kind=hi.PC_CSG_INTERIOR, theta_beta=0.25, smoother=hi.SM_RBGS, nu1=0, nu2=2),
]


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("pci", range(len(PCS)))
@pytest.mark.parametrize("case", CASES)
def test_multigrid_components(case, pci, mg):
    """Every level: operator, residual, smoothing (from zero and from a guess), restriction,
    prolongation and the coarsest direct solve."""
    p = _problem(case)
    pc = PCS[pci]
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    assert h.nlev == o.nlev
    dt = torch.complex128 if mg == "c128" else torch.complex64
    tol = 1e-11 if mg == "c128" else 2e-5
    rng = np.random.default_rng(5)
    for lvl in range(o.nlev):
        assert h.level_shape(lvl) == o.level_shape(1, lvl)
        n = o.level_size(1, lvl)
        a = (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        b = (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        if mg == "c64":
            a = a.astype(np.complex64).astype(np.complex128)
            b = b.astype(np.complex64).astype(np.complex128)
        if lvl == o.nlev - 1:
            out = torch.empty(n, dtype=dt, device="cuda")
            h.level_op(L.HELM_OP_COARSE, lvl, cu(a, dt), None, out)
            check(out.cpu().numpy(), o.coarse_solve(a), (1e-10 if mg == "c128" else 1e-4))
            continue
        edge = edge_rows(o, lvl)
        out = torch.empty(n, dtype=dt, device="cuda")
        h.level_op(L.HELM_OP_APPLY, lvl, cu(a, dt), None, out)
        check(out.cpu().numpy(), o.apply(a, 1, lvl), tol, edge)
        h.level_op(L.HELM_OP_RESIDUAL, lvl, cu(a, dt), cu(b, dt), out)
        check(out.cpu().numpy(), b - o.apply(a, 1, lvl), tol, edge)
        u = cu(a, dt)
        h.level_op(L.HELM_OP_SMOOTH, lvl, u, cu(b, dt), None, count=2)
        check(u.cpu().numpy(), o.smooth(lvl, a, b, 2), tol, edge)
        u = cu(a, dt)
        h.level_op(L.HELM_OP_SMOOTH0, lvl, u, cu(b, dt), None, count=2)
        check(u.cpu().numpy(), o.smooth(lvl, np.zeros(n), b, 2), tol, edge)
        nc = o.level_size(1, lvl + 1)
        fc = torch.empty(nc, dtype=dt, device="cuda")
        h.level_op(L.HELM_OP_RESTRICT, lvl, cu(a, dt), None, fc)
        check(fc.cpu().numpy(), o.restrict(lvl, a), tol)
        ec = rng.standard_normal(nc) + 1j * rng.standard_normal(nc)
        if mg == "c64":
            ec = ec.astype(np.complex64).astype(np.complex128)
        u = cu(a, dt)
        h.level_op(L.HELM_OP_PROLONG, lvl, u, cu(ec, dt))
        check(u.cpu().numpy(), o.prolong_add(lvl, ec, a), tol, edge)
    h.close()


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("pci", [0, 2])
@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[3]])
def test_fused_down_kernel(case, pci, mg):
    """HELM_OP_DOWN (one kernel): smoothing from the zero guess, residual and full weighting,
    against the oracle's three separate steps on every non-coarsest level."""
    p = _problem(case)
    pc = PCS[pci]
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    dt = torch.complex128 if mg == "c128" else torch.complex64
    tol = 1e-11 if mg == "c128" else 2e-5
    rng = np.random.default_rng(7)
    for lvl in range(o.nlev - 1):
        n, nc = o.level_size(1, lvl), o.level_size(1, lvl + 1)
        f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        if mg == "c64":
            f = f.astype(np.complex64).astype(np.complex128)
        u = torch.empty(n, dtype=dt, device="cuda")
        fc = torch.empty(nc, dtype=dt, device="cuda")
        h.level_op(L.HELM_OP_DOWN, lvl, u, cu(f, dt), fc)
        u_ref = o.smooth(lvl, np.zeros(n), f, 1)
        fc_ref = o.restrict(lvl, f - o.apply(u_ref, 1, lvl))
        check(u.cpu().numpy(), u_ref, tol)
        check(fc.cpu().numpy(), fc_ref, (10 * tol))
    h.close()


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("pci", range(len(PCS)))
@pytest.mark.parametrize("case", CASES)
def test_vcycle(case, pci, mg, fused):
    """The whole V-cycle: the fused path (single-block tail for the small levels; fused
    smooth+residual+restriction and prolongation+smooth kernels on 2D V(1,1) levels) and the
    one-kernel-per-component path."""
    p = _problem(case)
    pc = PCS[pci]
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg, fused=fused)
    r = hi.random_vector(p.n, 21)
    z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
    ref = o.vcycle(r)
    check(z, ref, (1e-10 if mg == "c128" else 5e-5))
    h.close()


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("sm", [hi.SM_JACOBI, hi.SM_RBGS])
@pytest.mark.parametrize("shape", [(300, 8), (97, 3), (161, 0), ((130, 70), ((0, 9), (5, 5))),
                                   ((561, 300), ((8, 7), (4, 4)))])
def test_vcycle_fused_levels_large(shape, sm, mg):
    """Grids large enough that several levels run the fused 2D kernels with many tiles and
    ragged edges (odd and even sizes, one-sided layers) before the tail takes over; the last
    shape is big enough for the large tiles on its finest level and the small ones below."""
    n_int, nl = shape
    p = hi.make_problem(2, n_int, nl, theta_gamma=0.5, k0=0.3 * (np.max(n_int) - 1), phi_kind="bump",
                        rhs="random", seed=8, bump_centre=(0.3, 0.6))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=sm)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    r = hi.random_vector(p.n, 2)
    z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
    check(z, o.vcycle(r), (1e-10 if mg == "c128" else 5e-5))
    h.close()


SOLVE_CASES = [
    (2, 33, 6, 0.5, 15.0, "const"),
    (2, (40, 29), ((5, 0), (3, 8)), 0.4, 12.0, "bump"),
    (2, 64, 16, 0.5, 20.0, "const"),
    (3, (12, 9, 10), ((2, 3), (0, 2), (3, 0)), 0.5, 5.0, "bump"),
]


@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR])
@pytest.mark.parametrize("pci", [0, 2])
@pytest.mark.parametrize("case", SOLVE_CASES)
def test_fp64_solve_matches_oracle(case, pci, method):
    """FP64 path vs the oracle at tol 1e-10: the same residual history until rounding drift
    (first 8 matvecs to 1e-9 relative), relative solution difference <= 1e-9, and a matvec
    count within 2 of the oracle's (or of its spread under rounding-level changes of b)."""
    p = _problem(case, rhs="point")
    pc = PCS[pci]
    o = Oracle(p, pc)
    sh = hi.shadow_space(p.n, 4)
    opts = hi.SolveOpts(method=method, s=4, tol=1e-10, maxmv=1500)
    x_ref, info_ref = o.solve(p.b, opts, shadow=sh, history=True)
    h = Helm(p, pc, mg_dtype="c128")
    x, info = h.solve(cu(p.b), method=method, s=4, tol=1e-10, maxmv=1500, shadow=sh, history=True)
    assert info.status == 0 and info_ref["status"] == 0
    assert info.rel_res_true < 1e-10
    m = min(8, info.matvecs, info_ref["matvecs"])
    assert np.allclose(info.history[:m], info_ref["history"][:m], rtol=1e-9, atol=0)
    check(x.cpu().numpy(), x_ref, 1e-9)
    counts_match(o, p.b, opts, info.matvecs, info_ref["matvecs"], shadow=sh)
    h.close()


@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR])
@pytest.mark.parametrize("case", SOLVE_CASES)
def test_mixed_precision_solve_error(case, method):
    """FP32 V-cycle, FP64 Krylov: true residual below tol and the error against the oracle's
    solution at 1e-12 within 1e-5 at the operating tolerance 1e-6 (and within 1e-6 at 1e-7)."""
    p = _problem(case, rhs="point")
    pc = PCS[0]
    o = Oracle(p, pc)
    sh = hi.shadow_space(p.n, 4)
    x_ref, _ = o.solve(p.b, hi.SolveOpts(method=hi.BICGSTAB, tol=1e-12, maxmv=3000))
    h = Helm(p, pc, mg_dtype="c64")
    for tol, bar in ((1e-6, 1e-5), (1e-7, 1e-6)):
        x, info = h.solve(cu(p.b), method=method, s=4, tol=tol, maxmv=1500, shadow=sh)
        assert info.status == 0 and info.rel_res_true < tol
        assert rel(x.cpu().numpy(), x_ref) < bar, (tol, rel(x.cpu().numpy(), x_ref))
    h.close()


@pytest.mark.parametrize("s", [1, 2, 8])
def test_idr_other_shadow_dimensions(s):
    p = _problem(SOLVE_CASES[0], rhs="point")
    pc = PCS[0]
    o = Oracle(p, pc)
    sh = hi.shadow_space(p.n, s, seed=77)
    opts = hi.SolveOpts(method=hi.IDR, s=s, tol=1e-10, maxmv=1500)
    x_ref, info_ref = o.solve(p.b, opts, shadow=sh)
    h = Helm(p, pc, mg_dtype="c128")
    x, info = h.solve(cu(p.b), method=hi.IDR, s=s, tol=1e-10, maxmv=1500, shadow=sh)
    assert info.status == 0
    counts_match(o, p.b, opts, info.matvecs, info_ref["matvecs"], shadow=sh)
    check(x.cpu().numpy(), x_ref, 1e-9)
    h.close()


def test_unpreconditioned_and_edge_cases():
    p = _problem((2, 12, 3, 0.5, 6.0, "const"), rhs="point")
    o = Oracle(p)
    x_ref = o.dense_solve(p.b)
    h = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    for method in (hi.BICGSTAB, hi.IDR):
        x, info = h.solve(cu(p.b), method=method, tol=1e-12, maxmv=5000, shadow=hi.shadow_space(p.n, 4))
        assert info.status == 0
        check(x.cpu().numpy(), x_ref, 1e-9)
    # zero right-hand side: x = 0 without a matvec
    x, info = h.solve(torch.zeros(p.n, dtype=torch.complex128, device="cuda"))
    assert info.status == 0 and info.matvecs == 0 and not torch.any(x)
    # non-finite right-hand side
    b = cu(p.b)
    b[3] = float("nan")
    x, info = h.solve(b)
    assert info.status == L.HELM_ERR_NAN
    # matvec cap: status MAXIT, x holds the last iterate (matches the oracle's iterate)
    x, info = h.solve(cu(p.b), tol=1e-14, maxmv=7)
    assert info.status == L.HELM_ERR_MAXIT and info.matvecs == 7
    xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-14, maxmv=7, max_restarts=0))
    assert io["status"] == 5
    check(x.cpu().numpy(), xo, 1e-10)
    h.close()


def test_single_unknown_and_single_level():
    # one unknown per axis: the hierarchy is one level, the V-cycle is the direct solve
    p = hi.make_problem(2, 3, 0, theta_gamma=0.0, k0=1.0, rhs="random", seed=2)
    assert p.n == 1
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype="c128")
    assert h.nlev == 1
    check(h.vcycle(cu(p.b)).cpu().numpy(), o.vcycle(p.b), 1e-13)
    x, info = h.solve(cu(p.b), tol=1e-12)
    assert info.status == 0 and info.matvecs <= 2
    h.close()


def test_bad_arguments_are_rejected_on_the_host():
    p = _problem(CASES[1])
    h = Helm(p, PCS[0], mg_dtype="c64")
    b = cu(p.b)
    from paper_0912_0180_gb300.helm import HelmError
    with pytest.raises(HelmError):
        h.solve(b, x=b)  # aliasing
    with pytest.raises(HelmError):
        h.solve(b, method=hi.IDR, s=9, shadow=hi.shadow_space(p.n, 9))
    with pytest.raises(HelmError):
        h.level_op(L.HELM_OP_COARSE, 0, b, None, b)  # level 0 is not the coarsest
    h.close()


def test_large_2d_workload_sampled():
    """The 512^2 + 64-layer workload (kh = 0.5, bump k, Gaussian source) at full size: the
    matvec and one V-cycle element by element, and the full mixed-precision solves through the
    same entry point the benchmark times, certified by the oracle's own true residual."""
    p = hi.workload_2d_512()
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype="c64")
    x = hi.random_vector(p.n, 4)
    check(h.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
    z = h.vcycle(cu(x)).cpu().numpy().astype(np.complex128)
    check(z, o.vcycle(x), 5e-5)
    for method in (hi.BICGSTAB, hi.IDR):
        xs, info = h.solve(cu(p.b), method=method, s=4, tol=1e-6, maxmv=3000,
                           shadow=hi.shadow_space(p.n, 4))
        assert info.status == 0
        r = p.b - o.apply(xs.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(p.b) < 1e-6
    h.close()


def test_full_size_2d_solves_match_oracle():
    """The benchmark's 640^2 problem (512^2 interior + 64-node ECS layers, kh = 0.5, bump k,
    Gaussian source) at full size.  (1) Bi-CGSTAB with the CSG omega-Jacobi V(1,1) preconditioner,
    FP64 path at tol 1e-10, against the oracle's own solve at 1e-10: relative solution difference
    <= 1e-9 (2-norm and element-wise) and the matvec count within 2 of the oracle's, or of the
    counts the oracle gives for b perturbed by 1e-15 and 1e-14 relative.  (2) The benchmark's four solves
    ({Bi-CGSTAB, IDR(4)} x {CSG, CSL}) at its tolerance 1e-6 in both precisions, against the
    oracle's solution at 1e-12 (the discrete solution does not depend on the preconditioner):
    every error below 1e-5."""
    p = hi.workload_2d_512()
    csg = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    csl = hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5)
    o = Oracle(p, csg)
    x10, i10 = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=6000))
    x12, i12 = o.solve(p.b, hi.SolveOpts(tol=1e-12, maxmv=8000))
    assert i10["status"] == 0 and i12["status"] == 0 and i12["rel_res_true"] < 1e-12
    h = Helm(p, csg, mg_dtype="c128")
    x, info = h.solve(cu(p.b), tol=1e-10, maxmv=6000)
    assert info.status == 0 and info.rel_res_true < 1e-10
    check(x.cpu().numpy(), x10, 1e-9)
    # over ~800 matvecs: four perturbed oracle runs at most (each takes seconds at this size)
    counts_match(o, p.b, hi.SolveOpts(tol=1e-10, maxmv=6000), info.matvecs, i10["matvecs"],
                 eps=(1e-15, 1e-15, 1e-14, 1e-14))
    h.close()
    sh = hi.shadow_space(p.n, 4)
    for mg in ("c128", "c64"):
        for pc in (csg, csl):
            h = Helm(p, pc, mg_dtype=mg)
            for method in (hi.BICGSTAB, hi.IDR):
                xs, inf = h.solve(cu(p.b), method=method, s=4, tol=1e-6, maxmv=4000, shadow=sh)
                assert inf.status == 0 and inf.rel_res_true < 1e-6
                assert rel(xs.cpu().numpy(), x12) < 1e-5, (mg, pc.kind, method, rel(xs.cpu().numpy(), x12))
            h.close()


@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR])
def test_device_loop_is_deterministic_and_matches_host_loop(method):
    """The reductions sum in a fixed order, so repeated solves, and the host-driven loop over
    the same captured iteration, give bitwise the same iterate and the same statistics."""
    p = _problem(SOLVE_CASES[1], rhs="point")
    h = Helm(p, PCS[0], mg_dtype="c64")
    sh = hi.shadow_space(p.n, 4)
    b = cu(p.b)
    x1, i1 = h.solve(b, method=method, tol=1e-8, shadow=sh)
    x1 = x1.clone()
    x2, i2 = h.solve(b, method=method, tol=1e-8, shadow=sh)
    x2 = x2.clone()
    x3, i3 = h.solve(b, method=method, tol=1e-8, shadow=sh, host_loop=True)
    assert torch.equal(x1, x2) and torch.equal(x1, x3)
    assert i1.matvecs == i2.matvecs == i3.matvecs and i1.rel_res_true == i3.rel_res_true
    # the device loop adds its head node and one condition-setting node per loop body; the loop
    # runs one body per Bi-CGSTAB iteration, or per IDR step after the s starting steps
    bodies = i1.iters if method == hi.BICGSTAB else i1.iters - 4
    assert i1.kernels == i3.kernels + 1 + bodies
    h.close()


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["bump", "const"])
@pytest.mark.parametrize("shape", [(2, (44, 50), ((4, 3), (5, 0)), 1), (3, 17, 2, 1), (3, (30, 34, 32), 2, 2)])
def test_vcycle_large_coarsest(shape, kind, mg):
    """Coarsest levels above 512 unknowns: with a variable k their dense inverse comes from the
    whole-GPU Gauss-Jordan (one pivot step per launch sequence) instead of the one-block kernel;
    with a constant k they are solved by separation of variables (per-axis eigendecompositions)."""
    dim, n_int, nl, levels = shape
    p = hi.make_problem(dim, n_int, nl, theta_gamma=0.5, k0=0.4 * (np.max(n_int) - 1), phi_kind=kind,
                        rhs="random", seed=5, bump_centre=(0.3, 0.6, 0.5))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS, max_levels=levels + 1)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    shp = h.level_shape(h.nlev - 1)
    assert int(np.prod(shp[:dim])) > 512
    r = hi.random_vector(p.n, 4)
    z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
    check(z, o.vcycle(r), (1e-10 if mg == "c128" else 5e-5))
    h.close()


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("sm", [hi.SM_JACOBI, hi.SM_RBGS])
def test_autotuned_tiles_give_the_same_vcycle(sm, mg):
    """The autotuner changes speed, not the method: its tiles regroup identical per-point formulas
    and its tail depth moves levels between kernels that sum in different orders, so the V-cycle
    equals the rule-chosen one to rounding, and both match the oracle."""
    p = hi.make_problem(2, (561, 300), ((8, 7), (4, 4)), theta_gamma=0.5, k0=168.0, phi_kind="bump",
                        rhs="random", seed=9, bump_centre=(0.3, 0.6))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=sm)
    r = cu(hi.random_vector(p.n, 6))
    ha = Helm(p, pc, mg_dtype=mg, autotune=True)
    hb = Helm(p, pc, mg_dtype=mg, autotune=False)
    za, zb = ha.vcycle(r), hb.vcycle(r)
    check(za.cpu().numpy(), zb.cpu().numpy(), (1e-13 if mg == "c128" else 2e-6))
    ref = Oracle(p, pc).vcycle(r.cpu().numpy())
    check(za.cpu().numpy().astype(np.complex128), ref, (1e-10 if mg == "c128" else 5e-5))
    ha.close()
    hb.close()


def test_large_3d_workload_sampled():
    """The 128^3 + 16-layer, k = 40 workload at full size in the benchmark's configuration (CSG,
    red-black Gauss-Seidel V(1,1) on 4 levels, coarsest 20^3 inverted densely): the matvec element
    by element against the oracle; the V-cycle by properties that hold at any size (linearity, and
    the FP32 cycle against the FP64 one); both solves certified by the oracle's own residual."""
    p = hi.workload_3d_128()
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS, max_levels=4)
    o = Oracle(p, hi.Precond(kind=hi.PC_NONE))
    h64 = Helm(p, pc, mg_dtype="c128")
    h32 = Helm(p, pc, mg_dtype="c64")
    assert h64.nlev == 4 and tuple(h64.level_shape(3)[:3]) == (20, 20, 20)
    x = hi.random_vector(p.n, 4)
    y = hi.random_vector(p.n, 5)
    check(h64.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    vx, vy = h64.vcycle(cu(x)), h64.vcycle(cu(y))
    vxy = h64.vcycle(cu(a * x + b * y))
    check(vxy.cpu().numpy(), (a * vx + b * vy).cpu().numpy(), 1e-12)
    check(h32.vcycle(cu(x)).cpu().numpy().astype(np.complex128), vx.cpu().numpy(), 5e-5)
    for h in (h64, h32):
        xs, info = h.solve(cu(p.b), tol=1e-6, maxmv=3000)
        assert info.status == 0 and info.rel_res_true < 1e-6
        r = p.b - o.apply(xs.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(p.b) < 1e-6
    h64.close()
    h32.close()


XS_CASES = [
    ((41, 30, 27), ((3, 4), (2, 0), (5, 1)), "bump"),   # 48 x 32 x 33 unknowns: even row length
    ((26, 19, 22), ((2, 3), (1, 2), (0, 3)), "const"),  # 31 x 22 x 25: odd row length
    # Sommerfeld low sides on x and y (those axes coarsen with offset 0), a high one on z
    ((26, 21, 22), ((-1, 3), (-1, 0), (2, -1)), "bump"),  # 29 x 20 x 24 unknowns, 3 levels
    # rows of 128 and 64 points: the two-pair sweep with 16-lane row segments
    ((120, 10, 12), ((4, 4), (2, 2), (2, 2)), "bump"),    # 128 x 14 x 16 unknowns
]


def _xsplit(v, shape):
    """Rows of shape[0] points with their even x indices first, then the odd ones."""
    a = np.asarray(v).reshape(-1, shape[0])
    return np.concatenate([a[:, 0::2], a[:, 1::2]], axis=1).reshape(-1)


@pytest.mark.parametrize("shape", XS_CASES)
def test_xsplit_levels_3d_fp32(shape):
    """The FP32 red-black levels of a 3D hierarchy above the coarsest store their rows x-split:
    the storage order is exactly that permutation on each such level (the coarsest stays natural),
    the level kernels on stored vectors give bitwise the natural results permuted, and the
    V-cycle (complex64 and widened output) and mixed-precision solves match the oracle."""
    n_int, nl, kind = shape
    p = hi.make_problem(3, n_int, nl, theta_gamma=0.5, k0=5.0, phi_kind=kind, rhs="point", seed=4,
                        bump_centre=(0.4, 0.6, 0.5))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype="c64", fused=False)
    assert h.nlev >= 3
    dt = torch.complex64
    rng = np.random.default_rng(9)
    rnd = lambda n: (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    S = L.HELM_OP_STORED
    for lvl in range(h.nlev):
        shp = h.level_shape(lvl)
        n = int(np.prod(shp))
        split = lvl < h.nlev - 1
        perm = (lambda v, s=shp: _xsplit(v, s)) if split else (lambda v: np.asarray(v))
        a, b = rnd(n), rnd(n)
        st = torch.empty(n, dtype=dt, device="cuda")
        h.level_op(L.HELM_OP_TO_STORED, lvl, cu(a, dt), None, st)
        assert np.array_equal(st.cpu().numpy(), perm(a)), lvl
        back = torch.empty_like(st)
        h.level_op(L.HELM_OP_FROM_STORED, lvl, st, None, back)
        assert np.array_equal(back.cpu().numpy(), a)
        if not split:
            continue
        for op in (L.HELM_OP_SMOOTH, L.HELM_OP_SMOOTH0):
            un, us = cu(a, dt), cu(perm(a), dt)
            h.level_op(op, lvl, un, cu(b, dt), None, count=2)
            h.level_op(op | S, lvl, us, cu(perm(b), dt), None, count=2)
            assert np.array_equal(us.cpu().numpy(), perm(un.cpu().numpy())), (lvl, op)
        for op, bb in ((L.HELM_OP_APPLY, None), (L.HELM_OP_RESIDUAL, b)):
            on, os_ = torch.empty(n, dtype=dt, device="cuda"), torch.empty(n, dtype=dt, device="cuda")
            h.level_op(op, lvl, cu(a, dt), None if bb is None else cu(bb, dt), on)
            h.level_op(op | S, lvl, cu(perm(a), dt), None if bb is None else cu(perm(bb), dt), os_)
            assert np.array_equal(os_.cpu().numpy(), perm(on.cpu().numpy())), (lvl, op)
        shc = h.level_shape(lvl + 1)
        nc = int(np.prod(shc))
        permc = (lambda v, s=shc: _xsplit(v, s)) if lvl + 1 < h.nlev - 1 else (lambda v: np.asarray(v))
        fn, fs = torch.empty(nc, dtype=dt, device="cuda"), torch.empty(nc, dtype=dt, device="cuda")
        h.level_op(L.HELM_OP_RESTRICT, lvl, cu(a, dt), None, fn)
        h.level_op(L.HELM_OP_RESTRICT | S, lvl, cu(perm(a), dt), None, fs)
        assert np.array_equal(fs.cpu().numpy(), permc(fn.cpu().numpy())), lvl
        check(fn.cpu().numpy(), o.restrict(lvl, a.astype(np.complex128)), 2e-5)
        ec = rnd(nc)
        un, us = cu(a, dt), cu(perm(a), dt)
        h.level_op(L.HELM_OP_PROLONG, lvl, un, cu(ec, dt))
        h.level_op(L.HELM_OP_PROLONG | S, lvl, us, cu(permc(ec), dt))
        assert np.array_equal(us.cpu().numpy(), perm(un.cpu().numpy())), lvl
        check(un.cpu().numpy(), o.prolong_add(lvl, ec.astype(np.complex128), a.astype(np.complex128)), 2e-5)
    r = hi.random_vector(p.n, 21)
    ref = o.vcycle(r)
    check(h.vcycle(cu(r)).cpu().numpy().astype(np.complex128), ref, 5e-5)
    check(h.vcycle(cu(r), dtype=torch.complex128).cpu().numpy(), ref, 5e-5)
    # every Krylov method feeds the cycle through its x-split input: the solution matches the
    # oracle's, and the matvec count is that of the natural-order FP64 hierarchy up to rounding
    x_ref, _ = o.solve(p.b, hi.SolveOpts(method=hi.BICGSTAB, tol=1e-12, maxmv=3000))
    sh = hi.shadow_space(p.n, 4)
    h64 = Helm(p, pc, mg_dtype="c128", fused=False)
    for method in (hi.BICGSTAB, hi.IDR, hi.GMRES):
        kw = dict(method=method, s=(4 if method == hi.IDR else 30), tol=1e-8, maxmv=1500,
                  shadow=sh if method == hi.IDR else None)
        x, info = h.solve(cu(p.b), **kw)
        _, info64 = h64.solve(cu(p.b), **kw)
        assert info.status == 0 and info.rel_res_true < 1e-8
        assert rel(x.cpu().numpy(), x_ref) < 1e-6, (method, rel(x.cpu().numpy(), x_ref))
        # a broken input or output order would ruin the preconditioner and multiply the count; GMRES
        # with an FP32 preconditioner may need one certification restart more at 1e-8 (its residual
        # estimate assumes an exact preconditioner), which costs up to one more cycle
        slack = max(3, info64.matvecs // 10)
        if method == hi.GMRES and info.restarts != info64.restarts:
            slack += kw["s"]
        assert abs(info.matvecs - info64.matvecs) <= slack, (method, info.matvecs, info64.matvecs, info.restarts)
    h64.close()
    h.close()


def test_batch256_workload_sampled():
    """All 256 instances of the uneven batch in one helm_solve_batch call (FP32 multigrid, the
    benchmark's configuration); a seeded sample of them certified by the oracle's own residual."""
    from paper_0912_0180_gb300.helm import solve_batch
    inst = hi.workload_batch_2d(256)
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    hs = [Helm(p, pc, mg_dtype="c64") for p in inst]
    xs, infos = solve_batch(hs, [cu(p.b) for p in inst], tol=1e-6, maxmv=4000)
    assert all(i.status == 0 and i.rel_res_true < 1e-6 for i in infos)
    rng = np.random.default_rng(7)
    for k in rng.choice(len(inst), 8, replace=False):
        p = inst[k]
        r = p.b - Oracle(p, hi.Precond(kind=hi.PC_NONE)).apply(xs[k].cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(p.b) < 1e-6
    for h in hs:
        h.close()


@pytest.mark.parametrize("which", ["mp2", "mp3"])
def test_model_problems_small(which):
    """The paper's model problems 2 and 3 (analytic phi and source, Dirichlet south / west, ECS
    north / east) on small grids with the paper's mesh width: V-cycle and FP64 solve against the
    oracle, and the FP32-multigrid solve certified by the oracle's own residual."""
    if which == "mp2":
        p = hi.workload_mp2(n_int=49, n_l=16, r=50.0 * 48 / 384)
        pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=np.pi / 20, smoother=hi.SM_JACOBI, omega=0.5)
    else:
        p = hi.workload_mp3(n_int=65, n_l=16, r=90.0 * 64 / 1024)
        pc = hi.Precond(kind=hi.PC_CSL, shift=1 + 0.38j, smoother=hi.SM_JACOBI, omega=0.5)
    o = Oracle(p, pc)
    r = hi.random_vector(p.n, 3)
    h64 = Helm(p, pc, mg_dtype="c128")
    check(h64.apply(cu(r)).cpu().numpy(), o.apply(r), 1e-12)
    check(h64.vcycle(cu(r)).cpu().numpy(), o.vcycle(r), 1e-10)
    x, info = h64.solve(cu(p.b), tol=1e-10, maxmv=4000)
    xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=4000))
    assert info.status == 0 and io["status"] == 0
    check(x.cpu().numpy(), xo, 1e-9)
    h32 = Helm(p, pc, mg_dtype="c64")
    x32, i32 = h32.solve(cu(p.b), tol=1e-7, maxmv=4000)
    assert i32.status == 0
    assert np.linalg.norm(p.b - o.apply(x32.cpu().numpy())) / np.linalg.norm(p.b) < 1e-7
    h64.close()
    h32.close()


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("shape", [((29, 22), ((3, 0), (2, 4)), "bump"), (64, 16, "const"), ((161, 130), ((0, 9), (5, 5)), "bump")])
def test_galerkin_vcycle(shape, mg):
    """Galerkin coarse operators (R A P, 9-point): every level's operator against the oracle's
    (itself pinned to dense R A P), and the whole V-cycle element by element."""
    n_int, nl, kind = shape
    p = hi.make_problem(2, n_int, nl, theta_gamma=0.5, k0=0.3 * (np.max(n_int) - 1), phi_kind=kind,
                        rhs="random", seed=12, bump_centre=(0.3, 0.6))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, galerkin=True)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    assert h.nlev == o.nlev
    dt = torch.complex128 if mg == "c128" else torch.complex64
    for lvl in range(h.nlev):
        x = hi.random_vector(o.level_size(1, lvl), 30 + lvl)
        y = h.level_op(L.HELM_OP_APPLY, lvl, cu(x, dt), None, torch.empty(len(x), dtype=dt, device="cuda"))
        check(y.cpu().numpy().astype(np.complex128), o.apply(x, 1, lvl), (1e-12 if mg == "c128" else 2e-5))
    r = hi.random_vector(p.n, 2)
    z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
    check(z, o.vcycle(r), (1e-10 if mg == "c128" else 5e-5))
    h.close()


def test_galerkin_solve_matches_oracle():
    """An FP64 Bi-CGSTAB solve preconditioned by the Galerkin V-cycle against the oracle's."""
    p = _problem(CASES[2])
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, galerkin=True)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype="c128")
    x, info = h.solve(cu(p.b), tol=1e-10, maxmv=3000)
    xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=3000))
    assert info.status == 0 and io["status"] == 0
    check(x.cpu().numpy(), xo, 1e-9)
    with pytest.raises(Exception):  # Galerkin levels need the Jacobi smoother
        Helm(p, hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_RBGS, galerkin=True))
    h.close()


RAMP_CASES = [
    # dim, n_int, layers, ramp, k0, phi kind
    (2, (45, 38), ((12, 9), (0, 10)), 6, 14.0, "bump"),
    (2, 64, 16, 16, 20.0, "const"),
    (3, (14, 11, 12), ((4, 3), (0, 5), (3, 4)), 3, 6.0, "bump"),
]


@pytest.mark.parametrize("case", RAMP_CASES)
def test_smooth_contour_parity(case):
    """The smooth ECS contour (layer widths turning over `ramp` widths): the FP64 operator, every
    level's operator and the V-cycle in both precisions, and an FP64 solve, against the oracle."""
    dim, n_int, nl, ramp, k0, kind = case
    p = hi.make_problem(dim, n_int, nl, theta_gamma=0.5, k0=k0, phi_kind=kind, rhs="gauss", seed=17,
                        bump_centre=(0.4, 0.6, 0.5), ecs_ramp=ramp)
    x = hi.random_vector(p.n, 8)
    for mg in ("c128", "c64"):
        pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3,
                        smoother=hi.SM_RBGS if dim == 3 else hi.SM_JACOBI)
        o = Oracle(p, pc)
        h = Helm(p, pc, mg_dtype=mg)
        assert h.nlev == o.nlev
        if mg == "c128":
            check(h.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
        dt = torch.complex128 if mg == "c128" else torch.complex64
        for lvl in range(o.nlev - 1):
            n = o.level_size(1, lvl)
            a = hi.random_vector(n, 9 + lvl).astype(np.complex64).astype(np.complex128)
            out = torch.empty(n, dtype=dt, device="cuda")
            h.level_op(L.HELM_OP_APPLY, lvl, cu(a, dt), None, out)
            check(out.cpu().numpy(), o.apply(a, 1, lvl), (1e-12 if mg == "c128" else 2e-5))
        z = h.vcycle(cu(x)).cpu().numpy().astype(np.complex128)
        check(z, o.vcycle(x), (1e-11 if mg == "c128" else 2e-5))
        if mg == "c128":
            xs, info = h.solve(cu(p.b), tol=1e-10, maxmv=2000)
            xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=2000))
            assert info.status == 0 and io["status"] == 0
            counts_match(o, p.b, hi.SolveOpts(tol=1e-10, maxmv=2000), info.matvecs, io["matvecs"])
            check(xs.cpu().numpy(), xo, 1e-9)
        h.close()


GMRES_CASES = [
    # case index into CASES, preconditioner, restart length m
    (2, hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5), 10),
    (3, hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5), 40),
    (5, hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_RBGS), 7),
    (0, hi.Precond(kind=hi.PC_NONE), 64),
]


@pytest.mark.parametrize("gi", range(len(GMRES_CASES)))
def test_gmres_solve_matches_oracle(gi):
    """Restarted right-preconditioned GMRES(m): the FP64 solve against the oracle's (matvecs within
    2, same solution to 1e-9 at tol 1e-10, the same residual estimates step by step while they are
    far above rounding), the host-driven loop bitwise equal to the device loop, and the FP32
    V-cycle path certified by its FP64 true residual."""
    ci, pc, m = GMRES_CASES[gi]
    p = _problem(CASES[ci], rhs="gauss", seed=23)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype="c128")
    maxmv = 4000
    xo, io = o.solve(p.b, hi.SolveOpts(method=hi.GMRES, s=m, tol=1e-10, maxmv=maxmv), history=True)
    x, info = h.solve(cu(p.b), method=hi.GMRES, s=m, tol=1e-10, maxmv=maxmv, history=True)
    assert info.status == 0 and io["status"] == 0, (info, io)
    assert info.rel_res_true < 1e-10
    counts_match(o, p.b, hi.SolveOpts(method=hi.GMRES, s=m, tol=1e-10, maxmv=maxmv), info.matvecs, io["matvecs"])
    check(x.cpu().numpy(), xo, 1e-9)
    hg = info.history[: min(info.matvecs, io["matvecs"])]
    ho = io["history"][: len(hg)]
    far = ho > 1e-6
    assert np.allclose(hg[far], ho[far], rtol=1e-6)
    x2, info2 = h.solve(cu(p.b), method=hi.GMRES, s=m, tol=1e-10, maxmv=maxmv, host_loop=True)
    assert info2.matvecs == info.matvecs and torch.equal(x2, x)
    h.close()
    if pc.kind != hi.PC_NONE:
        h32 = Helm(p, pc, mg_dtype="c64")
        x3, info3 = h32.solve(cu(p.b), method=hi.GMRES, s=m, tol=1e-8, maxmv=maxmv)
        assert info3.status == 0 and info3.rel_res_true < 1e-8
        xo8, io8 = o.solve(p.b, hi.SolveOpts(method=hi.GMRES, s=m, tol=1e-8, maxmv=maxmv))
        assert abs(info3.matvecs - io8["matvecs"]) <= max(3, io8["matvecs"] // 10)
        h32.close()


def test_gmres_full_and_batch():
    """GMRES with m above the step count (no restart) equals the oracle; a batch mixing GMRES,
    Bi-CGSTAB and IDR gives every instance its lone result bitwise."""
    p = _problem(CASES[1], rhs="gauss", seed=24)
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    o = Oracle(p, pc)
    xo, io = o.solve(p.b, hi.SolveOpts(method=hi.GMRES, s=128, tol=1e-10, maxmv=128))
    hs = [Helm(p, pc, mg_dtype="c128") for _ in range(3)]
    x, info = hs[0].solve(cu(p.b), method=hi.GMRES, s=128, tol=1e-10, maxmv=128)
    assert io["status"] == 0 and info.status == 0 and info.restarts == 0
    assert abs(info.matvecs - io["matvecs"]) <= 1
    check(x.cpu().numpy(), xo, 1e-9)
    from paper_0912_0180_gb300.helm import solve_batch
    shadow = hi.shadow_space(p.n, 4)
    lone = [hs[0].solve(cu(p.b), method=hi.GMRES, s=20, tol=1e-8)[0],
            hs[1].solve(cu(p.b), method=hi.BICGSTAB, tol=1e-8)[0],
            hs[2].solve(cu(p.b), method=hi.IDR, s=4, tol=1e-8, shadow=shadow)[0]]
    xs, infos = solve_batch(hs, [cu(p.b)] * 3, method=[hi.GMRES, hi.BICGSTAB, hi.IDR], s=[20, 4, 4],
                            tol=1e-8, shadows=[None, None, shadow])
    for a, b_, inf in zip(xs, lone, infos):
        assert inf.status == 0 and torch.equal(a, b_)
    with pytest.raises(Exception):
        hs[0].solve(cu(p.b), method=hi.GMRES, s=129)
    for h in hs:
        h.close()


# First-order Sommerfeld condition on high sides (n_layer = -1): unknown counts even over
# several levels so that coarsening keeps the boundary node (fine 2c+1 = n-1), ragged shapes,
# ECS layers on some low sides, a bump k.
SOMM_CASES = [
    # dim, n_int, layers, theta, k0, phi kind
    (1, 48, (6, -1), 0.5, 9.0, "bump"),                                   # 54 unknowns
    (2, (44, 49), ((4, -1), (0, -1)), 0.5, 12.0, "bump"),                 # 48 x 48
    (2, (65, 33), ((0, -1), (7, 0)), 0.4, 14.0, "const"),                 # 64 x 39
    (3, (13, 14, 12), ((0, -1), (2, -1), (0, 0)), 0.5, 5.0, "bump"),      # 12 x 16 x 10
]
# Sommerfeld low sides (n_layer = -1 on a low side; MP1's edges): the axis coarsens with offset 0,
# keeping node 0; both sides on one axis (odd counts), low side with layers on the high side, 3D
SOMM_LO_CASES = [
    (1, 49, (-1, 6), 0.5, 9.0, "bump"),                                    # 55 unknowns
    (2, (45, 49), ((-1, -1), (-1, 0)), 0.5, 12.0, "bump"),                 # 45 x 48
    (2, (33, 40), ((-1, 4), (6, -1)), 0.4, 11.0, "const"),                 # 37 x 46
    (3, (13, 13, 12), ((-1, -1), (2, 0), (-1, 2)), 0.5, 5.0, "bump"),      # 13 x 14 x 14
]
SOMM_PCS = [
    hi.Precond(kind=hi.PC_CSL, shift=1 - 0.5j, smoother=hi.SM_JACOBI, omega=0.5),
    hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=-0.3, smoother=hi.SM_RBGS),
]


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("pci", range(len(SOMM_PCS)))
@pytest.mark.parametrize("case", SOMM_CASES + SOMM_LO_CASES)
def test_sommerfeld_operator_levels_and_vcycle(case, pci, mg):
    """The Sommerfeld boundary rows: H itself, every level's operator (the ghost-node row with its
    2 i k / h_l diagonal on each coarse grid), the smoother, and the whole V-cycle, fused and
    one kernel per component, against the oracle."""
    p = _problem(case)
    pc = SOMM_PCS[pci]
    o = Oracle(p, pc)
    if mg == "c128":
        h0 = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
        x = hi.random_vector(p.n, 3)
        check(h0.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
        h0.close()
    h = Helm(p, pc, mg_dtype=mg)
    assert h.nlev == o.nlev and o.nlev >= 2
    dt = torch.complex128 if mg == "c128" else torch.complex64
    tol = 1e-11 if mg == "c128" else 2e-5
    for lvl in range(o.nlev - 1):
        n = o.level_size(1, lvl)
        a = hi.random_vector(n, 9 + lvl).astype(np.complex64).astype(np.complex128)
        b = hi.random_vector(n, 19 + lvl).astype(np.complex64).astype(np.complex128)
        out = torch.empty(n, dtype=dt, device="cuda")
        edge = edge_rows(o, lvl)
        h.level_op(L.HELM_OP_APPLY, lvl, cu(a, dt), None, out)
        check(out.cpu().numpy(), o.apply(a, 1, lvl), tol, edge)
        u = cu(a, dt)
        h.level_op(L.HELM_OP_SMOOTH, lvl, u, cu(b, dt), None, count=2)
        check(u.cpu().numpy(), o.smooth(lvl, a, b, 2), tol, edge)
    nco = o.level_size(1, o.nlev - 1)
    a = hi.random_vector(nco, 5)
    out = torch.empty(nco, dtype=dt, device="cuda")
    h.level_op(L.HELM_OP_COARSE, o.nlev - 1, cu(a, dt), None, out)
    check(out.cpu().numpy(), o.coarse_solve(a), (1e-10 if mg == "c128" else 1e-4))
    r = hi.random_vector(p.n, 21)
    for fused in (True, False):
        hf = h if fused else Helm(p, pc, mg_dtype=mg, fused=False)
        z = hf.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
        check(z, o.vcycle(r), (1e-10 if mg == "c128" else 5e-5))
        if not fused:
            hf.close()
    h.close()


@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR, hi.GMRES])
@pytest.mark.parametrize("case", SOMM_CASES[1:3] + SOMM_LO_CASES[1:3])
def test_sommerfeld_solve_matches_oracle(case, method):
    """FP64 solves of Sommerfeld problems against the oracle (matvecs within 2, solution to 1e-9),
    the FP32-multigrid path certified by its FP64 true residual, and Galerkin coarse operators
    built from the Sommerfeld rows (2D)."""
    p = _problem(case, rhs="gauss", seed=29)
    pc = SOMM_PCS[0]
    o = Oracle(p, pc)
    sh = hi.shadow_space(p.n, 4) if method == hi.IDR else None
    s = 60 if method == hi.GMRES else 4  # few GMRES cycles, so that the matvec counts stay close
    xo, io = o.solve(p.b, hi.SolveOpts(method=method, s=s, tol=1e-10, maxmv=3000), shadow=sh)
    h = Helm(p, pc, mg_dtype="c128")
    x, info = h.solve(cu(p.b), method=method, s=s, tol=1e-10, maxmv=3000, shadow=sh)
    assert info.status == 0 and io["status"] == 0
    counts_match(o, p.b, hi.SolveOpts(method=method, s=s, tol=1e-10, maxmv=3000), info.matvecs, io["matvecs"], shadow=sh)
    check(x.cpu().numpy(), xo, 1e-9)
    h.close()
    h32 = Helm(p, pc, mg_dtype="c64")
    x3, i3 = h32.solve(cu(p.b), method=method, s=s, tol=1e-7, maxmv=3000, shadow=sh)
    assert i3.status == 0 and i3.rel_res_true < 1e-7
    h32.close()
    if method == hi.BICGSTAB and min(lo for lo, _ in p.n_layer[: p.dim]) >= 0:  # Galerkin: no low sides
        pg = hi.Precond(kind=hi.PC_CSL, shift=1 - 0.5j, smoother=hi.SM_JACOBI, omega=0.5, galerkin=True)
        og = Oracle(p, pg)
        hg = Helm(p, pg, mg_dtype="c128")
        for lvl in range(og.nlev):
            xx = hi.random_vector(og.level_size(1, lvl), 40 + lvl)
            y = hg.level_op(L.HELM_OP_APPLY, lvl, cu(xx), None, torch.empty(len(xx), dtype=torch.complex128, device="cuda"))
            check(y.cpu().numpy(), og.apply(xx, 1, lvl), 1e-12)
        xg, ig = hg.solve(cu(p.b), tol=1e-10, maxmv=3000)
        xgo, igo = og.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=3000))
        assert ig.status == 0 and igo["status"] == 0
        check(xg.cpu().numpy(), xgo, 1e-9)
        hg.close()


def test_sommerfeld_arguments():
    """A side below -1, Galerkin operators with a Sommerfeld low side, and a negative phi at a
    Sommerfeld grid are refused."""
    from paper_0912_0180_gb300.helm import HelmError
    p = hi.make_problem(2, 17, ((-1, 0), (0, 0)), k0=3.0, rhs="zero")
    Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128").close()
    with pytest.raises(HelmError):
        Helm(p, hi.Precond(kind=hi.PC_CSL, smoother=hi.SM_JACOBI, galerkin=True), mg_dtype="c128")
    q = hi.make_problem(2, 17, ((0, -1), (0, 0)), k0=3.0, rhs="zero")
    q.phi = np.full(q.n, -1.0)
    with pytest.raises(HelmError):
        Helm(q, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("shape", [((14, 12, 13), ((2, 0), (0, 3), (0, 0)), "bump"),
                                   ((13, 11, 13), ((2, 0), (0, 3), (0, -1)), "bump"),
                                   (22, 4, "const")])
def test_galerkin3d_levels_vcycle_and_solve(shape, mg):
    """3D Galerkin coarse operators (27-point R A P): every level's operator and the whole
    V-cycle against the oracle's (pinned to dense R A P), and an FP64 Bi-CGSTAB solve."""
    n_int, nl, kind = shape
    p = hi.make_problem(3, n_int, nl, theta_gamma=0.5, k0=0.3 * (np.max(n_int) - 1), phi_kind=kind,
                        rhs="gauss", seed=13, bump_centre=(0.3, 0.6, 0.5))
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, galerkin=True, coarse_max=3)
    o = Oracle(p, pc)
    h = Helm(p, pc, mg_dtype=mg)
    assert h.nlev == o.nlev and o.nlev >= 3
    dt = torch.complex128 if mg == "c128" else torch.complex64
    for lvl in range(h.nlev):
        x = hi.random_vector(o.level_size(1, lvl), 30 + lvl).astype(np.complex64).astype(np.complex128)
        y = h.level_op(L.HELM_OP_APPLY, lvl, cu(x, dt), None, torch.empty(len(x), dtype=dt, device="cuda"))
        check(y.cpu().numpy().astype(np.complex128), o.apply(x, 1, lvl), (1e-12 if mg == "c128" else 2e-5))
    r = hi.random_vector(p.n, 2)
    z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
    check(z, o.vcycle(r), (1e-10 if mg == "c128" else 5e-5))
    if mg == "c128":
        x, info = h.solve(cu(p.b), tol=1e-10, maxmv=3000)
        xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=3000))
        assert info.status == 0 and io["status"] == 0
        counts_match(o, p.b, hi.SolveOpts(tol=1e-10, maxmv=3000), info.matvecs, io["matvecs"])
        check(x.cpu().numpy(), xo, 1e-9)
    h.close()


CZ_CASES = [
    # dim, n_int, layers, ramp, k0, preconditioner index into PCS
    (2, (40, 29), ((5, 0), (3, 8)), 0, 12.0, 0),
    (2, 64, 16, 6, 20.0, 2),
    (3, (12, 9, 10), ((2, 3), (0, 2), (3, 0)), 0, 5.0, 0),
]


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("ci", range(len(CZ_CASES)))
def test_complex_z_potential_parity(ci, mg):
    """k read at the complex node positions of the layers (phi complex there): H, every level's
    operator, the V-cycle fused and unfused, and an FP64 solve against the oracle."""
    dim, n_int, nl, ramp, k0, pci = CZ_CASES[ci]
    p = hi.make_problem(dim, n_int, nl, theta_gamma=0.5, k0=k0, phi_kind="bump", rhs="gauss", seed=41,
                        bump_centre=(0.15, 0.8, 0.5), bump_width2=0.05, ecs_ramp=ramp, complex_z=True)
    assert np.abs(p.phi_im).max() > 1e-3
    pc = PCS[pci]
    o = Oracle(p, pc)
    x = hi.random_vector(p.n, 4)
    if mg == "c128":
        h0 = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
        check(h0.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
        h0.close()
    dt = torch.complex128 if mg == "c128" else torch.complex64
    tol = 1e-11 if mg == "c128" else 2e-5
    for fused in (True, False):
        h = Helm(p, pc, mg_dtype=mg, fused=fused)
        assert h.nlev == o.nlev
        if fused:
            for lvl in range(o.nlev - 1):
                a = hi.random_vector(o.level_size(1, lvl), 9 + lvl).astype(np.complex64).astype(np.complex128)
                out = torch.empty(len(a), dtype=dt, device="cuda")
                h.level_op(L.HELM_OP_APPLY, lvl, cu(a, dt), None, out)
                check(out.cpu().numpy(), o.apply(a, 1, lvl), tol)
        z = h.vcycle(cu(x)).cpu().numpy().astype(np.complex128)
        check(z, o.vcycle(x), (1e-10 if mg == "c128" else 5e-5))
        if mg == "c128" and fused:
            xs, info = h.solve(cu(p.b), tol=1e-10, maxmv=3000)
            xo, io = o.solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=3000))
            assert info.status == 0 and io["status"] == 0
            counts_match(o, p.b, hi.SolveOpts(tol=1e-10, maxmv=3000), info.matvecs, io["matvecs"])
            check(xs.cpu().numpy(), xo, 1e-9)
        h.close()


def test_complex_phi_inside_the_uniform_interior():
    """An imaginary part of phi inside the interior (not what complex node positions give, but
    allowed) drops the uniform-interior shortcut rather than being ignored there."""
    p = _problem(CASES[3])
    p.phi = np.full(p.n, 20.0 ** 2)
    p.phi_im = 0.3 * np.random.default_rng(3).standard_normal(p.n)
    o = Oracle(p, PCS[0])
    x = hi.random_vector(p.n, 5)
    h0 = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    check(h0.apply(cu(x)).cpu().numpy(), o.apply(x), 1e-12)
    h0.close()
    for mg in ("c128", "c64"):
        h = Helm(p, PCS[0], mg_dtype=mg)
        z = h.vcycle(cu(x)).cpu().numpy().astype(np.complex128)
        check(z, o.vcycle(x), (1e-10 if mg == "c128" else 5e-5))
        h.close()


ILU_CASES = [
    (1, 60, ((5, 6),)),                  # tridiagonal levels: ILU(0) is their exact LU
    (2, (29, 23), ((4, 5), (3, 4))),     # odd sizes, uneven layers
    (2, (40, 31), ((6, 0), (2, 7))),     # one-sided layers, an even row length
]


@pytest.mark.parametrize("mg", ["c128", "c64"])
@pytest.mark.parametrize("galerkin", [False, True])
@pytest.mark.parametrize("case", ILU_CASES)
def test_ilu0_levels_vcycle_and_solve(case, galerkin, mg):
    """ILU(0) smoothing (Section 6.1) on the GPU against the oracle: every non-coarsest level's
    smoothing steps from a guess and from zero (Shortley-Weller cross levels and 9-point Galerkin
    levels), the V(0,1) and V(1,1) cycles, and a right-preconditioned Bi-CGSTAB solve with the
    paper's multigrid (Galerkin coarse operators, V(0,1), ILU(0))."""
    dim, n_int, nl = case
    if galerkin and dim == 1:
        pytest.skip("Galerkin coarse operators are built in 2D and 3D")
    p = hi.make_problem(dim, n_int, nl, theta_gamma=0.5, k0=6.0, phi_kind="bump", rhs="point", seed=7,
                        bump_centre=(0.4, 0.6, 0.5))
    dt = torch.complex128 if mg == "c128" else torch.complex64
    tol = 1e-10 if mg == "c128" else 5e-5
    rng = np.random.default_rng(17)
    for nu1, nu2 in ((0, 1), (1, 1)):
        pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.4, smoother=hi.SM_ILU, galerkin=galerkin, nu1=nu1,
                        nu2=nu2)
        o = Oracle(p, pc)
        h = Helm(p, pc, mg_dtype=mg)
        assert h.nlev == o.nlev >= 3
        if nu1 == 0:
            for lvl in range(o.nlev - 1):
                n = o.level_size(1, lvl)
                a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
                b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
                if mg == "c64":
                    a = a.astype(np.complex64).astype(np.complex128)
                    b = b.astype(np.complex64).astype(np.complex128)
                u = cu(a, dt)
                h.level_op(L.HELM_OP_SMOOTH, lvl, u, cu(b, dt), None, count=2)
                check(u.cpu().numpy(), o.smooth(lvl, a, b, 2), tol)
                u = cu(a, dt)
                h.level_op(L.HELM_OP_SMOOTH0, lvl, u, cu(b, dt), None, count=1)
                check(u.cpu().numpy(), o.smooth(lvl, np.zeros(n), b, 1), tol)
        r = hi.random_vector(p.n, 23)
        z = h.vcycle(cu(r)).cpu().numpy().astype(np.complex128)
        check(z, o.vcycle(r), tol)
        h.close()
    if not galerkin or mg == "c64":
        return
    # the paper's multigrid in a solve: FP64 path against the oracle at a tight tolerance
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.4, smoother=hi.SM_ILU, galerkin=True, nu1=0, nu2=1)
    o = Oracle(p, pc)
    opts = hi.SolveOpts(method=hi.BICGSTAB, tol=1e-10, maxmv=1500)
    x_ref, info_ref = o.solve(p.b, opts)
    h = Helm(p, pc, mg_dtype="c128")
    x, info = h.solve(cu(p.b), method=hi.BICGSTAB, tol=1e-10, maxmv=1500)
    assert info.status == 0 and info_ref["status"] == 0 and info.rel_res_true < 1e-10
    check(x.cpu().numpy(), x_ref, 1e-9)
    counts_match(o, p.b, opts, info.matvecs, info_ref["matvecs"])
    h.close()


def test_ilu0_is_refused_where_it_does_not_run():
    """ILU(0) smoothing is built for 1D and 2D levels: a 3D hierarchy is refused at create, and
    the coarsest level (solved directly) has no factors to smooth with."""
    p3 = hi.make_problem(3, (9, 9, 9), ((2, 2), (2, 2), (2, 2)), theta_gamma=0.5, k0=3.0)
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_ILU)
    with pytest.raises(Exception, match="ILU"):
        Helm(p3, pc, mg_dtype="c128")
    p2 = hi.make_problem(2, (21, 17), ((3, 3), (3, 3)), theta_gamma=0.5, k0=4.0)
    h = Helm(p2, pc, mg_dtype="c128")
    lvl = h.nlev - 1
    n = int(np.prod(h.level_shape(lvl)))
    u = torch.zeros(n, dtype=torch.complex128, device="cuda")
    with pytest.raises(Exception, match="ILU"):
        h.level_op(L.HELM_OP_SMOOTH, lvl, u, u.clone(), None, count=1)
    h.close()
