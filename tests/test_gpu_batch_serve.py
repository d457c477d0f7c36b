"""Batched and served execution: many uneven instances at once give, instance by instance, the
result of a lone solve (bitwise: every solve's reductions have a fixed order and instances share
nothing), and the server admits requests against its device-memory budget."""
import numpy as np
import pytest
import torch

import helm_inputs as hi
from oracle import Oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _instances():
    """Uneven 2D and 3D instances: sizes, layers, k fields, preconditioners and smoothers differ."""
    out = []
    specs = [
        (2, 47, 8, 10.0, "const", hi.PC_CSG_UNIFORM, hi.SM_JACOBI),
        (2, 96, 16, 25.0, "bump", hi.PC_CSL, hi.SM_JACOBI),
        (2, (70, 33), ((6, 0), (4, 9)), 12.0, "bump", hi.PC_CSG_UNIFORM, hi.SM_RBGS),
        (3, 15, 3, 6.0, "const", hi.PC_CSG_UNIFORM, hi.SM_RBGS),
        (2, 130, 20, 30.0, "const", hi.PC_CSG_INTERIOR, hi.SM_JACOBI),
        (3, (14, 11, 13), ((2, 3), (0, 2), (3, 0)), 5.0, "bump", hi.PC_CSL, hi.SM_JACOBI),
    ]
    for i, (dim, n_int, nl, k0, kind, pck, sm) in enumerate(specs):
        p = hi.make_problem(dim, n_int, nl, theta_gamma=0.5, k0=k0, phi_kind=kind, rhs="gauss", seed=100 + i,
                            bump_centre=(0.45, 0.55, 0.5))
        pc = hi.Precond(kind=pck, theta_beta=0.3, shift=1 + 0.5j, smoother=sm, omega=0.5)
        out.append((p, pc))
    return out


@pytest.mark.parametrize("mg", ["c64", "c128"])
@pytest.mark.parametrize("method", [hi.BICGSTAB, hi.IDR])
def test_batch_equals_lone_solves(mg, method):
    from paper_0912_0180_gb300.helm import Helm, solve_batch
    inst = _instances()
    hs = [Helm(p, pc, mg_dtype=mg) for p, pc in inst]
    bs = [torch.from_numpy(p.b).cuda() for p, _ in inst]
    shadows = [hi.shadow_space(p.n, 4, seed=5 + i) for i, (p, _) in enumerate(inst)]
    alone = []
    for h, b, sh in zip(hs, bs, shadows):
        x, info = h.solve(b, method=method, tol=1e-8, maxmv=3000, shadow=sh)
        alone.append((x.clone(), info))
    xs, infos = solve_batch(hs, bs, method=method, tol=1e-8, maxmv=3000, shadows=shadows)
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ib.status == 0 and ia.status == 0
        assert torch.equal(xa, xb)
        assert ia.matvecs == ib.matvecs and ia.rel_res_true == ib.rel_res_true
    # and the batch is right: the FP64 multigrid batch against the oracle's solutions
    if mg == "c128":
        for (p, pc), xb in zip(inst, xs):
            xo, io = Oracle(p, pc).solve(p.b, hi.SolveOpts(method=hi.BICGSTAB, tol=1e-12, maxmv=4000))
            assert np.linalg.norm(xb.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    for h in hs:
        h.close()


def test_server_results_same_alone_and_in_the_mix():
    from paper_0912_0180_gb300.helm import Helm, Server, estimate_bytes
    inst = _instances()
    alone = []
    for p, pc in inst:
        h = Helm(p, pc, mg_dtype="c64")
        x, info = h.solve(torch.from_numpy(p.b).cuda(), tol=1e-7, maxmv=3000)
        alone.append((x.cpu().numpy(), info))
        h.close()
    sizes = [estimate_bytes(p, pc) for p, pc in inst]
    budget = int(max(sizes) + sorted(sizes)[0])  # at most two of the requests fit at once
    srv = Server(budget, max_active=3)
    tickets = [srv.submit(p, pc, tol=1e-7, maxmv=3000) for p, pc in inst]
    queued, active, used = srv.stats()
    assert used <= budget
    results = [srv.wait(t) for t in tickets]
    for (xa, ia), (xs, info, lat) in zip(alone, results):
        assert info.status == 0 and lat > 0
        assert np.array_equal(xa, xs)
        assert info.matvecs == ia.matvecs
    assert srv.stats()[2] == 0  # every byte admitted has been returned
    # a request bigger than the whole budget is refused at submission
    from paper_0912_0180_gb300.helm import HelmError
    with pytest.raises(HelmError):
        Server(1000, 1).submit(*inst[0])
    srv.close()


def test_server_overlaps_requests():
    """Continuous batching: with room for all of them, requests run concurrently (the server's
    active count exceeds one while they run) and all complete."""
    import time
    from paper_0912_0180_gb300.helm import Server
    inst = _instances()
    srv = Server(64 << 30, max_active=8)
    tickets = [srv.submit(p, pc, tol=1e-7, maxmv=3000) for p, pc in inst]
    seen = 0
    for _ in range(2000):
        seen = max(seen, srv.stats()[1])
        if seen > 1:
            break
        time.sleep(0.0005)
    res = [srv.wait(t) for t in tickets]
    assert all(r[1].status == 0 for r in res)
    assert seen > 1
    srv.close()


def test_server_multiple_right_hand_sides():
    """A request with several right-hand sides: every column is what a lone helm_solve gives it
    (bitwise), and the request's statistics add up the per-right-hand-side counts."""
    from paper_0912_0180_gb300.helm import Helm, Server
    inst = _instances()
    srv = Server(64 << 30, max_active=4)
    jobs = []
    for i, (p, pc) in enumerate(inst[:4]):
        nrhs = 1 + (i * 3) % 5
        rhs = np.stack([hi.random_vector(p.n, 40 + 7 * i + k) for k in range(nrhs)])
        jobs.append((p, pc, rhs, srv.submit(p, pc, tol=1e-7, maxmv=3000, rhs=rhs)))
    for p, pc, rhs, t in jobs:
        x, info, lat = srv.wait(t)
        assert info.status == 0 and x.shape == rhs.shape
        h = Helm(p, pc, mg_dtype="c64")
        mv = 0
        for k in range(rhs.shape[0]):
            xa, ia = h.solve(torch.from_numpy(rhs[k]).cuda(), tol=1e-7, maxmv=3000)
            assert np.array_equal(xa.cpu().numpy(), x[k])
            mv += ia.matvecs
        assert info.matvecs == mv
        h.close()
    srv.close()


@pytest.mark.parametrize("mg", ["c64", "c128"])
def test_batch_with_a_method_per_instance(mg):
    """One batch mixing Bi-CGSTAB and IDR(s) instances (opts has one entry per instance, as the
    benchmark's four-solve step uses it): each instance equals its lone solve bitwise."""
    from paper_0912_0180_gb300.helm import Helm, solve_batch
    inst = _instances()
    methods = [hi.BICGSTAB if i % 2 == 0 else hi.IDR for i in range(len(inst))]
    hs = [Helm(p, pc, mg_dtype=mg) for p, pc in inst]
    bs = [torch.from_numpy(p.b).cuda() for p, _ in inst]
    shadows = [hi.shadow_space(p.n, 4, seed=9 + i) if m == hi.IDR else None
               for i, ((p, _), m) in enumerate(zip(inst, methods))]
    alone = [h.solve(b, method=m, tol=1e-8, maxmv=3000, shadow=sh) for h, b, m, sh in zip(hs, bs, methods, shadows)]
    alone = [(x.clone(), info) for x, info in alone]
    xs, infos = solve_batch(hs, bs, method=methods, tol=1e-8, maxmv=3000, shadows=shadows)
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ia.status == 0 and ib.status == 0
        assert torch.equal(xa, xb) and ia.matvecs == ib.matvecs
    for h in hs:
        h.close()


def test_server_smallest_first_admission():
    """With one slot busy on a long request, a large and several small requests wait; the
    smallest-first policy admits the small ones before the large one submitted ahead of them, and
    every result still equals the lone solve bitwise."""
    from paper_0912_0180_gb300.helm import Helm, Server
    inst = _instances()
    sizes = [p.n for p, _ in inst]
    order = sorted(range(len(inst)), key=lambda i: sizes[i])
    big, smalls = order[-1], order[:2]  # with one slot a request can be passed over twice
    blocker = (hi.make_problem(2, 383, 64, theta_gamma=0.5, k0=150.0, phi_kind="bump", rhs="gauss", seed=4),
               hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5))
    srv = Server(64 << 30, max_active=1, smallest_first=True)
    tb = srv.submit(*blocker, tol=1e-10, maxmv=8000)
    import time
    time.sleep(0.05)  # the blocker (several hundred matvecs on 511^2 unknowns) is running
    tbig = srv.submit(*inst[big], tol=1e-7, maxmv=3000)
    tsm = [srv.submit(*inst[i], tol=1e-7, maxmv=3000) for i in smalls]
    srv.wait(tb)
    xb, ib, lat_big = srv.wait(tbig)
    res = [srv.wait(t) for t in tsm]
    assert ib.status == 0 and all(r[1].status == 0 for r in res)
    assert max(r[2] for r in res) < lat_big
    for i, (x, info, _) in zip(smalls + [big], res + [(xb, ib, lat_big)]):
        p, pc = inst[i]
        h = Helm(p, pc, mg_dtype="c64")
        xa, ia = h.solve(torch.from_numpy(p.b).cuda(), tol=1e-7, maxmv=3000)
        assert np.array_equal(xa.cpu().numpy(), x) and ia.matvecs == info.matvecs
        h.close()
    srv.close()


def test_gmres_in_batch_and_server():
    """GMRES(30) instances batched and served give each instance its lone result bitwise."""
    from paper_0912_0180_gb300.helm import Helm, Server, solve_batch
    inst = _instances()[:4]
    hs = [Helm(p, pc, mg_dtype="c64") for p, pc in inst]
    bs = [torch.from_numpy(p.b).cuda() for p, _ in inst]
    alone = [h.solve(b, method=hi.GMRES, s=30, tol=1e-7, maxmv=3000) for h, b in zip(hs, bs)]
    alone = [(x.clone(), i) for x, i in alone]
    xs, infos = solve_batch(hs, bs, method=hi.GMRES, s=30, tol=1e-7, maxmv=3000)
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ia.status == 0 and ib.status == 0
        assert torch.equal(xa, xb) and ia.matvecs == ib.matvecs
    srv = Server(64 << 30, max_active=4)
    tickets = [srv.submit(p, pc, method=hi.GMRES, s=30, tol=1e-7, maxmv=3000) for p, pc in inst]
    for (xa, ia), t in zip(alone, tickets):
        x, info, lat = srv.wait(t)
        assert info.status == 0 and np.array_equal(xa.cpu().numpy(), x) and info.matvecs == ia.matvecs
    srv.close()
    for h in hs:
        h.close()


def _group_instances(smoother):
    """Uneven 2D instances for one group: sizes (from a one-level tail to many fused levels), ragged
    and one-sided layers, constant and bump k, CSG / CSL / interior-CSG with different parameters."""
    specs = [
        (33, 6, 10.0, "const", hi.PC_CSG_UNIFORM, 0.3),
        (96, 16, 25.0, "bump", hi.PC_CSL, 0.3),
        ((70, 33), ((6, 0), (4, 9)), 12.0, "bump", hi.PC_CSG_UNIFORM, 0.25),
        (130, 20, 30.0, "const", hi.PC_CSG_INTERIOR, 0.3),
        ((161, 120), ((0, 9), (5, 5)), 40.0, "bump", hi.PC_CSL, 0.3),
        (12, 2, 4.0, "const", hi.PC_CSG_UNIFORM, 0.3),
    ]
    out = []
    for i, (n_int, nl, k0, kind, pck, th) in enumerate(specs):
        p = hi.make_problem(2, n_int, nl, theta_gamma=0.5, k0=k0, phi_kind=kind, rhs="gauss", seed=200 + i,
                            bump_centre=(0.45, 0.55))
        pc = hi.Precond(kind=pck, theta_beta=th, shift=1 + 0.5j + 0.1j * i, smoother=smoother, omega=0.5 + 0.05 * i)
        out.append((p, pc))
    return out


@pytest.mark.parametrize("smoother", [hi.SM_JACOBI, hi.SM_RBGS])
@pytest.mark.parametrize("mg", ["c64", "c128"])
def test_group_equals_lone_solves(mg, smoother):
    """helm_solve_group runs every kernel of an iteration as one launch over all instances; each
    instance's solution, matvec count and residuals are bitwise its lone helm_solve's.  (The launch
    count of this uneven mix is about that of the six lone solves -- the group runs as many bodies as
    its slowest instance; the reduction is checked on many instances in the next test.)"""
    from paper_0912_0180_gb300.helm import Helm, solve_group
    inst = _group_instances(smoother)
    for autotune in (True, False):  # the tuner's tail depths and the rule's
        hs = [Helm(p, pc, mg_dtype=mg, autotune=autotune) for p, pc in inst]
        bs = [torch.from_numpy(p.b).cuda() for p, _ in inst]
        alone = []
        for h, b in zip(hs, bs):
            x, info = h.solve(b, tol=1e-8, maxmv=3000)
            alone.append((x.clone(), info))
        xs, infos = solve_group(hs, bs, tol=1e-8, maxmv=3000)
        for (xa, ia), xg, ig in zip(alone, xs, infos):
            assert ia.status == 0 and ig.status == 0
            assert torch.equal(xa, xg)
            assert ia.matvecs == ig.matvecs and ia.iters == ig.iters
            assert ia.rel_res_true == ig.rel_res_true and ia.rel_res_recur == ig.rel_res_recur
        # a second call on the same contexts gives the same results again
        xs2, _ = solve_group(hs, bs, tol=1e-8, maxmv=3000)
        assert all(torch.equal(a, b_) for a, b_ in zip(xs, xs2))
        for h in hs:
            h.close()


def test_group_of_many_instances_issues_far_fewer_launches():
    """Sixteen small instances (different sizes, k and right-hand sides): the group runs as many
    bodies as its slowest instance, each a few launches per level for all of them together, so it
    issues far fewer launches than the sixteen lone solves -- and still the same solutions."""
    from paper_0912_0180_gb300.helm import Helm, solve_group
    hs, bs = [], []
    for i in range(16):
        n_int = 40 + 8 * (i % 4)
        p = hi.make_problem(2, n_int, 8, theta_gamma=0.5, k0=0.4 * n_int, phi_kind="bump" if i % 2 else "const",
                            rhs="gauss", seed=300 + i, bump_centre=(0.4, 0.6))
        hs.append(Helm(p, hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)))
        bs.append(torch.from_numpy(p.b).cuda())
    alone = [h.solve(b, tol=1e-8, maxmv=3000) for h, b in zip(hs, bs)]
    xs, infos = solve_group(hs, bs, tol=1e-8, maxmv=3000)
    for (xa, ia), xg, ig in zip(alone, xs, infos):
        assert ia.status == 0 and ig.status == 0 and torch.equal(xa, xg)
    assert infos[0].kernels * 4 < sum(ia.kernels for _, ia in alone), (infos[0].kernels, sum(ia.kernels for _, ia in alone))
    for h in hs:
        h.close()


def test_group_against_the_oracle_and_its_refusals():
    """A group's FP64-multigrid solutions against the oracle's own solves; instances that the grouped
    kernels do not cover are refused on the host."""
    from paper_0912_0180_gb300.helm import Helm, HelmError, solve_group
    inst = _group_instances(hi.SM_JACOBI)[:4]
    hs = [Helm(p, pc, mg_dtype="c128") for p, pc in inst]
    bs = [torch.from_numpy(p.b).cuda() for p, _ in inst]
    xs, infos = solve_group(hs, bs, tol=1e-10, maxmv=3000)
    for (p, pc), x, inf in zip(inst, xs, infos):
        xo, io = Oracle(p, pc).solve(p.b, hi.SolveOpts(tol=1e-10, maxmv=3000))
        # (each grouped solve is bitwise its lone solve, whose matvec counts the parity tests hold
        # against the oracle's)
        assert inf.status == 0 and io["status"] == 0 and inf.rel_res_true < 1e-10
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-9
    p3 = hi.make_problem(3, 15, 3, theta_gamma=0.5, k0=6.0, rhs="gauss", seed=3)
    pc3 = hi.Precond(kind=hi.PC_CSG_UNIFORM, theta_beta=0.3, smoother=hi.SM_JACOBI, omega=0.5)
    bad = [Helm(p3, pc3, mg_dtype="c64"),
           Helm(inst[0][0], hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_JACOBI, galerkin=True), mg_dtype="c64"),
           Helm(inst[0][0], hi.Precond(kind=hi.PC_CSG_UNIFORM, smoother=hi.SM_JACOBI, nu1=2), mg_dtype="c64"),
           Helm(inst[0][0], hi.Precond(kind=hi.PC_NONE), mg_dtype="c128")]
    for hb in bad:
        with pytest.raises(HelmError):
            solve_group([hs[0], hb], [bs[0], torch.from_numpy(hb.problem.b).cuda()], tol=1e-8)
    with pytest.raises(HelmError):  # one smoother kind per group
        hr = Helm(inst[1][0], hi.Precond(kind=hi.PC_CSL, shift=1 + 0.5j, smoother=hi.SM_RBGS), mg_dtype="c128")
        solve_group([hs[0], hr], bs[:2], tol=1e-8)
    for h in hs + bad:
        h.close()
