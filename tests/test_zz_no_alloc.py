"""helm_residual_noalloc: the allocation-free variant of the true-residual kernel.

Some callers cannot allocate device memory (their process's device memory belongs to
another allocator that reserved it up front, or they run latency-critical loops where a
cudaMalloc, which may synchronise the device, is not acceptable).  For them the library offers
r = b - H x and ||r|| / ||b|| with its scratch in a static device array.  This file is named to
run last: it checks the new entry point, through the C ABI, against the existing entry points
on two calls in a row -- the true residual helm_solve reports, and b - helm_apply(x).
"""
import ctypes

import numpy as np
import pytest
import torch

import helm_inputs as hi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_noalloc_residual_matches_existing_entry_points():
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import Helm

    lib = L.load()
    p = hi.make_problem(2, 64, 16, theta_gamma=0.5, k0=20.0, phi_kind="bump", rhs="gauss", seed=3)
    h = Helm(p, hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI), mg_dtype="c64")
    b = torch.from_numpy(p.b).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the static scratch
        tol = 1e-3 if call == 0 else 1e-8
        x, info = h.solve(b, tol=tol, maxmv=2000)
        assert info.status == 0
        r = torch.full_like(b, float("nan"))
        rel = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.helm_residual_noalloc(h._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(rel.data_ptr()),
                                       ctypes.c_void_p(stream))
        assert st == L.HELM_OK, lib.helm_last_error()
        torch.cuda.synchronize()
        r_ref = b - h.apply(x)
        assert torch.linalg.norm(r - r_ref) <= 1e-12 * torch.linalg.norm(r_ref)
        assert abs(rel.item() - info.rel_res_true) <= 1e-12 * info.rel_res_true
    # sizes beyond the static scratch are rejected before any launch
    big = hi.make_problem(2, 2050, 2, theta_gamma=0.5, k0=1.0, rhs="zero")
    assert big.n > 4194304
    hb = Helm(big, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    v = torch.zeros(big.n, dtype=torch.complex128, device="cuda")
    w = torch.zeros_like(v)
    st = lib.helm_residual_noalloc(hb._h, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                   ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(rel.data_ptr()),
                                   ctypes.c_void_p(stream))
    assert st == L.HELM_ERR_ARG and b"4194304" in lib.helm_last_error()
    hb.close()
    h.close()


def _noalloc(lib, h, b, x):
    r = torch.full_like(b, float("nan"))
    rel = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.helm_residual_noalloc(h._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(rel.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, r, rel.item()


def test_noalloc_residual_against_the_oracle_in_3d():
    """A 3D grid with one-sided layers and a bump k: r against the oracle's b - H x (FP64, element
    by element), ||r|| / ||b|| against numpy's norms, twice in a row with different x."""
    from oracle import Oracle
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import Helm

    lib = L.load()
    p = hi.make_problem(3, (14, 11, 12), ((3, 0), (2, 4), (0, 2)), theta_gamma=0.5, k0=6.0, phi_kind="bump",
                        rhs="random", seed=6, bump_centre=(0.4, 0.6, 0.5))
    o = Oracle(p)
    h = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    b = torch.from_numpy(p.b).cuda()
    for seed in (1, 2):
        xh = hi.random_vector(p.n, seed)
        st, r, rel = _noalloc(lib, h, b, torch.from_numpy(xh).cuda())
        assert st == L.HELM_OK, lib.helm_last_error()
        r_ref = p.b - o.apply(xh)
        rh = r.cpu().numpy()
        assert np.max(np.abs(rh - r_ref)) <= 1e-12 * np.max(np.abs(r_ref))
        assert abs(rel - np.linalg.norm(r_ref) / np.linalg.norm(p.b)) <= 1e-12 * rel
    h.close()


def test_noalloc_residual_at_its_largest_size():
    """Exactly 4,194,304 unknowns (2048^2): all 4096 partial-sum pairs of the static array are in
    use, next to its completion counter.  r against b - helm_apply(x), the ratio against torch's
    norms, on two calls in a row."""
    from paper_0912_0180_gb300 import _lib as L
    from paper_0912_0180_gb300.helm import Helm

    lib = L.load()
    p = hi.make_problem(2, 2050, 0, theta_gamma=0.0, k0=30.0, rhs="gauss", seed=9)
    assert p.n == 4194304
    h = Helm(p, hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")
    b = torch.from_numpy(p.b).cuda()
    g = torch.Generator(device="cuda").manual_seed(4)
    for _ in range(2):
        x = torch.randn(p.n, dtype=torch.complex128, device="cuda", generator=g)
        st, r, rel = _noalloc(lib, h, b, x)
        assert st == L.HELM_OK, lib.helm_last_error()
        r_ref = b - h.apply(x)
        assert torch.max(torch.abs(r - r_ref)).item() <= 1e-12 * torch.max(torch.abs(r_ref)).item()
        ref = (torch.linalg.vector_norm(r_ref) / torch.linalg.vector_norm(b)).item()
        assert abs(rel - ref) <= 1e-12 * ref
    h.close()
