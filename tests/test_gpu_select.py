"""The automatic CSL shift / CSG angle choice (Section 7, remark on choosing the parameters) and
its inner loop -- multigrid as a stationary solver of M u = f -- against the oracle.

Both sides take every decision (a cycle count against the reduction, a trial converging or not)
in FP64 from norms that differ only in summation order; the parameters of the trials are the same
floating-point products on both sides, so they must agree bit for bit.
"""
import numpy as np
import pytest
import torch

import helm_inputs as hi
from oracle import Oracle, select_precond as oracle_select

pytestmark = pytest.mark.gpu

from paper_0912_0180_gb300 import _lib as L  # noqa: E402
from paper_0912_0180_gb300.helm import Helm, HelmError, select_precond  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


ITER_CASES = [
    # problem, preconditioner, max cycles, reduction
    (dict(dim=2, n_int=12, n_l=3, k0=4.0, phi_kind="const"),
     hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_JACOBI, omega=0.5), 80, 1e-10),
    (dict(dim=2, n_int=(90, 71), n_l=((12, 9), (0, 10)), k0=25.0, phi_kind="bump"),
     hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.6, smoother=hi.SM_RBGS), 40, 1e-8),
    (dict(dim=3, n_int=(14, 11, 12), n_l=((3, 2), (0, 3), (2, 2)), k0=6.0, phi_kind="bump"),
     hi.Precond(kind=hi.PC_CSL, shift=1 + 0.8j, smoother=hi.SM_RBGS), 40, 1e-8),
]


@pytest.mark.parametrize("ci", range(len(ITER_CASES)))
def test_mg_iterate_matches_oracle(ci):
    spec, pc, max_cycles, red = ITER_CASES[ci]
    p = hi.make_problem(spec["dim"], spec["n_int"], spec["n_l"], theta_gamma=0.5, k0=spec["k0"],
                        phi_kind=spec["phi_kind"], rhs="zero", seed=31, bump_centre=(0.4, 0.6, 0.5))
    f = hi.random_vector(p.n, 32)
    o = Oracle(p, pc)
    ko, uo, ho = o.mg_iterate(f, max_cycles, red)
    h = Helm(p, pc, mg_dtype="c128")
    k, u, hist = h.mg_iterate(cu(f), max_cycles, red)
    assert ko > 0 and k == ko
    # ||f - M u|| / ||f|| is a difference of nearly equal vectors once small: its rounding floor is
    # about eps ||M|| ||u|| / ||f|| (~1e-13 here), below which the two summation orders differ
    assert np.allclose(hist, ho, rtol=1e-9, atol=1e-13)
    assert rel(u.cpu().numpy(), uo) < 1e-9
    h.close()


@pytest.mark.parametrize("kind", [hi.PC_CSL, hi.PC_CSG_UNIFORM])
def test_select_precond_matches_oracle(kind):
    p = hi.make_problem(2, 20, 4, theta_gamma=0.5, k0=8.0, rhs="zero", seed=1)
    f = hi.random_vector(p.n, 22)
    if kind == hi.PC_CSL:
        start = hi.Precond(kind=kind, shift=1 + 1.2j, smoother=hi.SM_RBGS)
    else:
        start = hi.Precond(kind=kind, theta_beta=0.9, smoother=hi.SM_RBGS)
    co, so, po, ko = oracle_select(p, start, f, 12, 1e-6, 0.7, 12)
    chosen, st, params, cycles = select_precond(p, start, cu(f), 12, 1e-6, 0.7, 12)
    assert st == so == 0
    assert np.array_equal(params, po) and np.array_equal(cycles, ko)
    got = chosen.shift.imag if kind == hi.PC_CSL else chosen.theta_beta
    assert got == co
    assert ko[-1] == -1 and len(ko) >= 3


def test_select_precond_larger_grid_and_errors():
    """A grid of several tiles with a variable k (the C2 shape at a quarter of the size): the GPU's
    sequence equals the oracle's; bad arguments are rejected before any launch."""
    p = hi.make_problem(2, 128, 16, theta_gamma=0.5, k0=0.5 * 127, phi_kind="bump", bump_amp=0.3,
                        rhs="zero", seed=3)
    f = hi.random_vector(p.n, 33)
    start = hi.Precond(kind=hi.PC_CSL, shift=1 + 1.0j, smoother=hi.SM_JACOBI, omega=0.5)
    co, so, po, ko = oracle_select(p, start, f, 30, 1e-6, 0.75, 10)
    chosen, st, params, cycles = select_precond(p, start, cu(f), 30, 1e-6, 0.75, 10)
    assert st == so
    assert np.array_equal(params, po) and np.array_equal(cycles, ko)
    assert chosen.shift.imag == co
    with pytest.raises(HelmError):
        select_precond(p, start, cu(f), 30, 1e-6, 1.0, 10)
    with pytest.raises(HelmError):
        select_precond(p, hi.Precond(kind=hi.PC_NONE), cu(f))
    h32 = Helm(p, start, mg_dtype="c64")
    with pytest.raises(HelmError):
        h32.mg_iterate(cu(f))
    h32.close()
