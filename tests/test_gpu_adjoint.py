"""Adjoint gradient kernel and the differentiable solve vs the oracle and
central finite differences (the loss is 1/2 sum_l B_l (u_l - t_l)^2)."""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, ctx_for, dev, global_from_L, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N", [2, 5, 7, 11])
def test_grad_h1_kernel(N):
    dev()
    mesh = si.box_mesh((3, 2, 2), N, warp=0.1, perm_seed=N)
    ctx = ctx_for(mesh, prec_copies=0)
    lev = O.level_from_mesh(mesh)
    rng = np.random.default_rng(N)
    u = rng.standard_normal(mesh["x"].shape)
    lam = rng.standard_normal(mesh["x"].shape)
    g = H(ctx.grad_h1(T(u), T(lam)))
    ref = O.grad_h1_local(lev, u, lam).ravel()
    assert relmax(g, ref) < 1e-12
    gs = H(ctx.grad_h1(T(u), T(lam), sum_copies=True))
    assert relmax(gs, O.qqt(ref, lev.node, lev.n_G)) < 1e-12


def _problem(e=4, N=7):
    mesh = si.box_mesh(e, N, warp=0.1, perm_seed=0)
    h1 = np.exp(0.5 * si.smooth_random_field(mesh, 1))
    t = si.smooth_random_field(mesh, 2)
    f = si.smooth_random_field(mesh, 3)
    return mesh, h1, t, f


def test_autograd_matches_oracle_adjoint():
    dev()
    from paper_2104_05829_gb300.autograd import helmholtz_solve
    mesh, h1, t, f = _problem(e=2, N=5)
    ctx = ctx_for(mesh, prec_copies=0)
    lev = O.level_from_mesh(mesh)
    ft = T(f).requires_grad_(True)
    ht = T(h1).requires_grad_(True)
    tt = T(t)
    B = ctx.mass_local(torch.ones_like(tt))
    u = helmholtz_solve(ctx, ft, ht, h2=1.0, tol=1e-13)
    loss = 0.5 * torch.sum(B * (u - tt) ** 2)
    loss.backward()
    lo, uo, lam, dfo, dho = O.adjoint_loss_and_grads(lev, f, h1, 1.0, t)
    assert abs(loss.item() - lo) < 1e-10 * abs(lo)
    assert relmax(H(ft.grad), dfo.ravel()) < 1e-8
    assert relmax(H(ht.grad), dho.ravel()) < 1e-8


def test_autograd_finite_differences_4x4x4_N7():
    """Central differences of GPU solves along a continuous direction, E = 4^3, N = 7."""
    dev()
    from paper_2104_05829_gb300.autograd import helmholtz_solve
    mesh, h1, t, f = _problem(e=4, N=7)
    ctx = ctx_for(mesh, prec_copies=0)
    lev = O.level_from_mesh(mesh)
    tt = T(t)
    B = ctx.mass_local(torch.ones_like(tt))

    def loss_of(fv, hv):
        u = helmholtz_solve(ctx, fv, hv, h2=1.0, tol=1e-13)
        return 0.5 * torch.sum(B * (u - tt) ** 2)

    ft = T(f).requires_grad_(True)
    ht = T(h1).requires_grad_(True)
    loss_of(ft, ht).backward()
    rng = np.random.default_rng(0)
    v = T(O.q_gather(rng.standard_normal(lev.n_G), lev.node))
    with torch.no_grad():
        for grad, which in ((ht.grad, "h1"), (ft.grad, "f")):
            dd = torch.dot(grad, v).item()
            fd = []
            for eps in (1e-3, 1e-4):
                def at(s):
                    return (loss_of(T(f), T(h1) + s * v) if which == "h1" else loss_of(T(f) + s * v, T(h1))).item()
                fd.append((at(eps) - at(-eps)) / (2 * eps))
            assert abs(fd[-1] - dd) < 1e-6 * abs(dd), (which, fd, dd)
            if which == "h1":
                assert abs(fd[0] - dd) > 10 * abs(fd[1] - dd)


def test_grad_h1_kernel_full_size_sampled():
    """The gradient kernel on the 32^3, N=7 box the benchmark's differentiated solve uses:
    per-point values of sampled elements, and the copy-summed values at their nodes, against
    the oracle evaluated on the sample's element neighbourhood."""
    dev()
    import types
    mesh = si.box_mesh(32, 7, warp=0.1, perm_seed=0)
    ctx = ctx_for(mesh, prec_copies=0, mg_orders=[7])
    rng = np.random.default_rng(7)
    u = rng.standard_normal(mesh["x"].shape)
    lam = rng.standard_normal(mesh["x"].shape)
    ut, lt = T(u), T(lam)
    g = H(ctx.grad_h1(ut, lt)).reshape(mesh["E"], -1)
    gs = H(ctx.grad_h1(ut, lt, sum_copies=True)).reshape(mesh["E"], -1)
    sample = rng.choice(mesh["E"], 24, replace=False)
    gid = mesh["gid"].reshape(mesh["E"], -1)
    hood = np.flatnonzero(np.isin(gid, np.unique(gid[sample])).any(axis=1))
    G, B, _ = O.geometry(mesh["x"][hood], mesh["y"][hood], mesh["z"][hood], 7)
    lev = types.SimpleNamespace(G=G, D=O.deriv_matrix(7))
    ref = O.grad_h1_local(lev, u[hood], lam[hood]).reshape(hood.size, -1)
    pos = {e: i for i, e in enumerate(hood)}
    idx = [pos[e] for e in sample]
    assert relmax(g[sample], ref[idx]) < 1e-12
    sums = np.zeros(gid.max() + 1)
    np.add.at(sums, gid[hood].ravel(), ref.ravel())
    assert relmax(gs[sample], sums[gid[sample]]) < 1e-12


# ---- p-multigrid with the nodal h1 (the oracle's PMG with a nodal coefficient) ----------

def _nodal_problem(shape=(4, 3, 3), N=7, orders=(7, 3, 1)):
    mesh = si.box_mesh(shape, N, warp=0.1, perm_seed=2, dirichlet=("x0", "y1"))
    h1 = np.exp(0.5 * si.smooth_random_field(mesh, 1))
    levels = O.build_levels(mesh, list(orders))
    return mesh, h1, levels


def test_nodal_h1_vcycle_matches_oracle():
    """Eigenvalue estimates and one FP64 V-cycle (8 coarse iterations) with a nodal h1
    against the oracle's PMG with the same coefficient carried to its coarse levels."""
    dev()
    mesh, h1, levels = _nodal_problem()
    ctx = ctx_for(mesh, coarse_tol=0.0, coarse_maxit=8)
    ctx.precond_setup(h1_L=T(h1), h2=1.0, prec="fp64")
    lam = ctx.lmax()
    L0 = levels[0]
    ref_est = O.PMG(levels, h1.reshape(L0.x.shape), 1.0, O.MGParams(coarse_tol=0.0, coarse_maxit=8))
    for a, b in zip(lam, ref_est.lmax):
        assert abs(a - b) < 1e-10 * b
    mg = O.PMG(levels, h1.reshape(L0.x.shape), 1.0, O.MGParams(coarse_tol=0.0, coarse_maxit=8, lmax=lam))
    r = L0.mask(np.random.default_rng(4).standard_normal(L0.n_G))
    z = H(ctx.vcycle(T(O.q_gather(r, L0.node))))
    assert relmax(z, O.q_gather(mg(r), L0.node)) < 1e-10


def test_nodal_h1_pmg_solve_matches_oracle():
    """FCG + p-MG with a nodal h1 at the default settings (pipelined coarse solve with
    h1-scaled factors, early stop at 1e-1) against the oracle: equal outer and coarse
    iteration counts, x to 1e-10; far fewer iterations than Jacobi-PCG."""
    dev()
    mesh, h1, levels = _nodal_problem((5, 4, 4))
    L0 = levels[0]
    ctx = ctx_for(mesh)
    f = si.smooth_random_field(mesh, 3)
    ht = T(h1)
    x, info = ctx.solve(T(f), h1_L=ht, h2=1.0, tol=1e-10, maxit=200, precond="pmg", prec="fp64")
    xj, ij = ctx.solve(T(f), h1_L=ht, h2=1.0, tol=1e-10, maxit=5000, precond="jacobi")
    b = L0.rhs_from_nodal(f.reshape(L0.x.shape))
    mg = O.PMG(levels, h1.reshape(L0.x.shape), 1.0, O.MGParams(lmax=info["lmax"]))
    ref = O.pcg(lambda v: L0.apply(v, h1.reshape(L0.x.shape), 1.0), b, mg, 1e-10, 200, flexible=True)
    print(f"nodal h1: p-MG {info['iters']} (oracle {ref.iters}), coarse {info['coarse_iters']} "
          f"(oracle {sum(mg.coarse_iters)}); Jacobi-PCG {ij['iters']}")
    assert info["iters"] == ref.iters and info["coarse_iters"] == sum(mg.coarse_iters)
    assert relmax(H(x), O.q_gather(ref.x, L0.node)) < 1e-10
    assert relmax(H(x), H(xj)) < 1e-8
    assert info["iters"] * 5 < ij["iters"]
    # the FP32-pair outer operator with the nodal h1: same iterations, solution to the pairs' accuracy
    xp, ip = ctx.solve(T(f), h1_L=ht, h2=1.0, tol=1e-10, maxit=200, precond="pmg", prec="fp64", outer_pairs=True)
    assert abs(ip["iters"] - info["iters"]) <= 1 and relmax(H(xp), H(x)) < 1e-9
    # the FP32 V-cycle reaches the same residual, by the oracle's measure
    x32, i32 = ctx.solve(T(f), h1_L=ht, h2=1.0, tol=1e-10, maxit=200, precond="pmg", prec="fp32")
    xg = global_from_L(L0, H(x32))
    assert np.linalg.norm(b - L0.apply(xg, h1.reshape(L0.x.shape), 1.0)) / np.linalg.norm(b) < 2e-10


def test_autograd_with_pmg_matches_oracle_adjoint():
    dev()
    from paper_2104_05829_gb300.autograd import helmholtz_solve
    mesh, h1, t, f = _problem(e=3, N=5)
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    ft = T(f).requires_grad_(True)
    ht = T(h1).requires_grad_(True)
    tt = T(t)
    B = ctx.mass_local(torch.ones_like(tt))
    u = helmholtz_solve(ctx, ft, ht, h2=1.0, tol=1e-13, precond="pmg")
    loss = 0.5 * torch.sum(B * (u - tt) ** 2)
    loss.backward()
    lo, uo, lam, dfo, dho = O.adjoint_loss_and_grads(lev, f, h1, 1.0, t)
    assert abs(loss.item() - lo) < 1e-10 * abs(lo)
    assert relmax(H(ft.grad), dfo.ravel()) < 1e-8
    assert relmax(H(ht.grad), dho.ravel()) < 1e-8


def test_autograd_pmg_with_pair_outer_operator_matches_oracle_adjoint():
    dev()
    from paper_2104_05829_gb300.autograd import helmholtz_solve
    mesh, h1, t, f = _problem(e=3, N=5)
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    ft = T(f).requires_grad_(True)
    ht = T(h1).requires_grad_(True)
    tt = T(t)
    B = ctx.mass_local(torch.ones_like(tt))
    u = helmholtz_solve(ctx, ft, ht, h2=1.0, tol=1e-12, precond="pmg", prec="fp32", outer_pairs=True)
    loss = 0.5 * torch.sum(B * (u - tt) ** 2)
    loss.backward()
    lo, uo, lam, dfo, dho = O.adjoint_loss_and_grads(lev, f, h1, 1.0, t)
    assert abs(loss.item() - lo) < 1e-10 * abs(lo)
    assert relmax(H(ft.grad), dfo.ravel()) < 1e-8
    assert relmax(H(ht.grad), dho.ravel()) < 1e-8
