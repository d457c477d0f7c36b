"""The C ABI's boundary on the GPU: the registered allocator (helm_set_allocator), the ways of giving
k(x) (helm_kspec kinds), helm_vcycle's preconditioner and output-type arguments, the statistics of
helm_solve_info, and the failure statuses (breakdown, out of memory) produced from host-chosen
inputs -- each through the same ctypes calls the package makes."""
import ctypes

import numpy as np
import pytest
import torch

import helm_inputs as hi
from oracle import Oracle

pytestmark = pytest.mark.gpu

from paper_0912_0180_gb300 import _lib as L  # noqa: E402
from paper_0912_0180_gb300 import helm as H  # noqa: E402
from paper_0912_0180_gb300.helm import Helm, HelmError  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def cu(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


class Counting:
    """An allocator over torch's caching allocator that records every block, and refuses (returns
    NULL) from its `fail_at`-th request on."""

    def __init__(self, fail_at=None):
        self.live = {}
        self.calls = 0
        self.frees = 0
        self.fail_at = fail_at

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.fail_at is not None and self.calls >= self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(max(nbytes, 1), torch.cuda.current_device(), stream)
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "freed a block it did not allocate"
        del self.live[ptr]
        self.frees += 1
        torch.cuda.caching_allocator_delete(ptr)


@pytest.fixture
def counting():
    yield Counting
    H.use_torch_allocator(force=True)


def _problem():
    return hi.make_problem(2, 40, 8, theta_gamma=0.5, k0=15.0, phi_kind="bump", rhs="gauss", seed=5)


PC = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)


def test_registered_allocator_serves_every_device_allocation(counting):
    """helm_create, the Krylov workspace and the solve all allocate through the registered
    callbacks; helm_destroy returns every block; the solution equals the library allocator's."""
    p = _problem()
    b = cu(p.b)
    H.set_allocator()  # the library's own cudaMallocAsync, for the reference solution
    h0 = Helm(p, PC, mg_dtype="c64", autotune=False)
    ref, _ = h0.solve(b, tol=1e-8)
    ref = ref.clone()
    h0.close()
    alloc = counting()
    H.set_allocator(alloc.alloc, alloc.free)
    h = Helm(p, PC, mg_dtype="c64", autotune=False)
    after_create = alloc.calls
    assert after_create > 10 and alloc.live
    # every byte the context holds came from the callbacks
    assert sum(alloc.live.values()) == h.workspace_bytes
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0 and alloc.calls > after_create  # the Krylov workspace
    assert torch.equal(x, ref)
    h.close()
    assert alloc.live == {} and alloc.frees == alloc.calls


@pytest.mark.parametrize("fail_at", [1, 2, 7, 25])
def test_allocator_refusal_is_out_of_memory_with_nothing_leaked(counting, fail_at):
    """An allocator that returns NULL makes helm_create return HELM_ERR_OOM; every block it had
    handed out before is returned."""
    alloc = counting(fail_at=fail_at)
    H.set_allocator(alloc.alloc, alloc.free)
    with pytest.raises(HelmError) as e:
        Helm(_problem(), PC, mg_dtype="c64", autotune=False)
    assert e.value.status == L.HELM_ERR_OOM
    assert alloc.live == {} and alloc.frees == alloc.calls - 1


def test_allocator_refusal_in_the_solve_workspace(counting):
    """A refusal while the first solve allocates its Krylov workspace: helm_solve returns
    HELM_ERR_OOM, the context stays usable once memory is available, and destroy frees all."""
    alloc = counting()
    H.set_allocator(alloc.alloc, alloc.free)
    p = _problem()
    h = Helm(p, PC, mg_dtype="c64", autotune=False)
    alloc.fail_at = alloc.calls + 3
    with pytest.raises(HelmError) as e:
        h.solve(cu(p.b), tol=1e-8)
    assert e.value.status == L.HELM_ERR_OOM
    alloc.fail_at = None
    x, info = h.solve(cu(p.b), tol=1e-8)
    assert info.status == 0 and info.rel_res_true < 1e-8
    h.close()
    assert alloc.live == {}


def test_k_kinds_formed_on_the_device():
    """HELM_K_GAUSS_BUMP (k formed on the device at the real node positions) and HELM_K_FIELD (a
    device field of k values) give the operator the host phi array gives: the same H x to rounding
    (the bump's exp) and bit for bit (the field's k^2); a non-finite field entry is refused."""
    p = hi.make_problem(2, (45, 38), ((6, 3), (0, 5)), theta_gamma=0.5, k0=14.0, phi_kind="bump", bump_amp=0.3,
                        bump_width2=0.02, bump_centre=(0.4, 0.6), rhs="random", seed=8)
    x = cu(hi.random_vector(p.n, 2))
    none = hi.Precond(kind=hi.PC_NONE)
    h_host = Helm(p, none, mg_dtype="c128")
    y_host = h_host.apply(x)
    h_bump = Helm(p, none, mg_dtype="c128", k_bump={"amp": 0.3, "width2": 0.02, "centre": (0.4, 0.6, 0.0)})
    y_bump = h_bump.apply(x)
    assert (torch.linalg.vector_norm(y_bump - y_host) / torch.linalg.vector_norm(y_host)).item() < 1e-14
    kf = torch.from_numpy(np.sqrt(p.phi)).cuda()
    h_field = Helm(p, none, mg_dtype="c128", k_field=kf)
    y_field = h_field.apply(x)
    o = Oracle(p)
    ref = o.apply(x.cpu().numpy())
    # the oracle reads phi; the field path squares sqrt(phi), exact to an ulp of phi
    assert np.linalg.norm(y_field.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-13
    kf2 = kf.clone()
    kf2[7] = float("nan")
    with pytest.raises(HelmError) as e:
        Helm(p, none, mg_dtype="c128", k_field=kf2)
    assert e.value.status == L.HELM_ERR_ARG
    # a whole solve with the device-formed bump against the oracle's on the host phi
    pc = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    hb = Helm(p, pc, mg_dtype="c128", k_bump={"amp": 0.3, "width2": 0.02, "centre": (0.4, 0.6, 0.0)})
    xs, info = hb.solve(cu(p.b), tol=1e-10, maxmv=2000)
    xo, io = Oracle(p, pc).solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=2000))
    assert info.status == 0 and io["status"] == 0
    assert np.linalg.norm(xs.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-9
    for h in (h_host, h_bump, h_field, hb):
        h.close()


def test_vcycle_precond_and_output_type():
    """helm_vcycle: complex128 output from an FP32 hierarchy is its complex64 output widened (the
    precision boundary, bit for bit); the context's own preconditioner is accepted, another one or
    a narrowing output type is refused on the host."""
    p = _problem()
    r = cu(hi.random_vector(p.n, 3))
    h32 = Helm(p, PC, mg_dtype="c64")
    z32 = h32.vcycle(r)
    z64 = h32.vcycle(r, dtype=torch.complex128)
    assert z64.dtype == torch.complex128 and torch.equal(z64, z32.to(torch.complex128))
    assert torch.equal(h32.vcycle(r, precond=PC), z32)
    import dataclasses
    with pytest.raises(HelmError):
        h32.vcycle(r, precond=dataclasses.replace(PC, theta_beta=0.25))
    with pytest.raises(HelmError):
        h32.vcycle(r, precond=dataclasses.replace(PC, nu2=2))
    h64 = Helm(p, PC, mg_dtype="c128")
    with pytest.raises(HelmError):
        h64.vcycle(r, dtype=torch.complex64)
    ref = Oracle(p, PC).vcycle(r.cpu().numpy())
    assert np.linalg.norm(h64.vcycle(r).cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10
    h32.close()
    h64.close()


def test_solve_info_statistics():
    """vcycles = one per preconditioned matvec (plus one per GMRES cycle for its update), seconds
    measured, history_len = the entries written."""
    p = _problem()
    b = cu(p.b)
    h = Helm(p, PC, mg_dtype="c64")
    x, info = h.solve(b, tol=1e-8, history=True)
    assert info.vcycles == info.matvecs and info.history_len == info.matvecs == len(info.history)
    assert info.seconds > 0
    x, info = h.solve(b, method=hi.GMRES, s=10, tol=1e-8)
    cycles = -(-info.matvecs // 10)  # each cycle of at most 10 Arnoldi steps ends with one update
    assert info.vcycles >= info.matvecs + cycles and info.history_len == 0
    h.close()
    h0 = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    x, info = h0.solve(b, tol=1e-6, maxmv=4000)
    assert info.vcycles == 0
    h0.close()


def _breakdown_problem():
    """Three unknowns with h = 1 and phi = 2: the Shortley-Weller diagonal 2 / h^2 - phi is exactly
    zero, so H = -[[0, 1, 0], [1, 0, 1], [0, 1, 0]] and b = e_0 gives b^H H b = 0 exactly."""
    p = hi.make_problem(1, 5, 0, theta_gamma=0.0, extent=4.0, k0=0.0, rhs="zero")
    p.phi = np.full(p.n, 2.0)
    b = np.zeros(p.n, np.complex128)
    b[0] = 1.0
    p.b = b
    return p


@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR])
def test_breakdown_status(method):
    """Bi-CGSTAB: (r^, H p) = b^H H b = 0 at the first step.  IDR(1): its first minimal-residual
    step has t^H r = 0, so omega = 0, the first difference vectors vanish and the 1 x 1 system
    P^H dR is singular.  Both end with HELM_ERR_BREAKDOWN, as the oracle's do."""
    p = _breakdown_problem()
    sh = hi.shadow_space(p.n, 1)
    o = Oracle(p)
    xo, io = o.solve(p.b, hi.SolveOpts(method=method, s=1, tol=1e-10, maxmv=50), shadow=sh)
    assert io["status"] == L.HELM_ERR_BREAKDOWN
    h = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    x, info = h.solve(cu(p.b), method=method, s=1, tol=1e-10, maxmv=50, shadow=sh)
    assert info.status == L.HELM_ERR_BREAKDOWN
    h.close()


def test_server_refuses_a_request_above_its_budget():
    """A request whose own memory exceeds the server's whole budget is refused at submission with
    HELM_ERR_OOM; a request that fits is then served."""
    p = _problem()
    need = H.estimate_bytes(p, PC, "c64")
    srv = H.Server(budget_bytes=need // 2, max_active=2)
    with pytest.raises(HelmError) as e:
        srv.submit(p, PC)
    assert e.value.status == L.HELM_ERR_OOM
    srv.close()
    srv = H.Server(budget_bytes=2 * need, max_active=2)
    t = srv.submit(p, PC, tol=1e-8)
    x, info, lat = srv.wait(t)
    assert info.status == 0 and info.vcycles == info.matvecs and info.seconds > 0
    srv.close()
