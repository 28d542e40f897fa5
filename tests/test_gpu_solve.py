"""GPU solvers, smoother and multigrid transfers vs the oracle.

Krylov parity follows one rule: both sides run the same algorithm with the same
parameters, so they take the same number of iterations; the solutions then
agree to 1e-10 (relative, max-norm) and both residuals meet the tolerance.
Mixed-precision solves are checked by the oracle's own residual of the GPU
solution and by their error against a tightly converged oracle solve.
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, ctx_for, dev, global_from_L, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gL(level, xg):
    return O.q_gather(xg, level.node)


def test_dinv_matches_oracle_diagonal():
    dev()
    mesh = si.box_mesh((3, 4, 2), 5, warp=0.1, perm_seed=2, dirichlet=("x0", "y1"))
    ctx = ctx_for(mesh, mg_orders=[5, 2, 1])
    levels = O.build_levels(mesh, [5, 2, 1])
    for l, Lo in enumerate(levels):
        d = H(ctx.level_dinv(l, 1.0, 0.3))
        ref = np.where(Lo.free, 1.0 / Lo.diag(1.0, 0.3), 0.0)[Lo.node]
        assert relmax(d, ref) < 1e-13


def test_transfers_match_oracle():
    dev()
    mesh = si.box_mesh((3, 2, 3), 7, warp=0.1, perm_seed=4, dirichlet=("z0",))
    ctx = ctx_for(mesh)
    levels = O.build_levels(mesh, [7, 3, 1])
    rng = np.random.default_rng(1)
    for l in (0, 1):
        F, Cl = levels[l], levels[l + 1]
        ec = Cl.mask(rng.standard_normal(Cl.n_G))
        xf = F.mask(rng.standard_normal(F.n_G))
        got = H(ctx.prolong_add(l, T(_gL(Cl, ec)), T(_gL(F, xf))))
        ref = _gL(F, xf + O.prolong(F, Cl, ec))
        assert relmax(got, ref) < 1e-13
        rf = F.mask(rng.standard_normal(F.n_G))
        got = H(ctx.restrict(l, T(_gL(F, rf))))
        ref = _gL(Cl, O.restrict(F, Cl, rf))
        assert relmax(got, ref) < 1e-13


def test_jacobi_pcg_manufactured_4x4x4_N7():
    """Config: 4^3 affine box, N=7, f = 3 pi^2 sin sin sin, Dirichlet, Jacobi-PCG to 1e-10."""
    dev()
    mesh = si.box_mesh(4, 7, warp=0.0, perm_seed=0)
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    uex, f = si.manufactured(mesh)
    x, info = ctx.solve(T(f), tol=1e-10, maxit=2000)
    ref = O.solve(lev, lev.rhs_from_nodal(f), tol=1e-10, maxit=2000)
    assert abs(info["iters"] - ref.iters) <= 1
    assert info["relres"] <= 1e-10 and ref.relres <= 1e-10
    assert relmax(H(x), _gL(lev, ref.x)) < 1e-10
    # both reach the same discretisation error against the exact solution
    e_gpu = np.max(np.abs(H(x) - uex.ravel()))
    e_ref = np.max(np.abs(_gL(lev, ref.x) - uex.ravel()))
    assert abs(e_gpu - e_ref) < 1e-9 and e_gpu < 1e-5


def test_jacobi_pcg_helmholtz_nodal_h1():
    dev()
    mesh = si.box_mesh((3, 3, 2), 5, warp=0.1, perm_seed=1)
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    h1 = np.exp(0.5 * si.smooth_random_field(mesh, 1))
    f = si.smooth_random_field(mesh, 3)
    x, info = ctx.solve(T(f), h1_L=T(h1), h2=1.0, tol=1e-12, maxit=2000)
    ref = O.solve(lev, lev.rhs_from_nodal(f), h1, 1.0, tol=1e-12, maxit=2000)
    assert abs(info["iters"] - ref.iters) <= 1
    assert relmax(H(x), _gL(lev, ref.x)) < 1e-10


def _mg_pair(shape=(3, 3, 3), N=5, orders=(5, 2, 1), coarse_maxit=8):
    mesh = si.box_mesh(shape, N, warp=0.1, perm_seed=6, dirichlet=("x0",))
    opts = dict(mg_orders=list(orders), coarse_tol=0.0, coarse_maxit=coarse_maxit)
    ctx = ctx_for(mesh, **opts)
    levels = O.build_levels(mesh, list(orders))
    return mesh, ctx, levels


def test_lanczos_estimates_match_oracle():
    dev()
    mesh, ctx, levels = _mg_pair()
    ctx.precond_setup(1.0, 0.0, "fp64")
    lam = ctx.lmax()
    mg = O.PMG(levels, params=O.MGParams())
    for a, b in zip(lam, mg.lmax):
        assert abs(a - b) < 1e-10 * b


def test_chebyshev_and_vcycle_match_oracle():
    dev()
    mesh, ctx, levels = _mg_pair()
    ctx.precond_setup(1.0, 0.0, "fp64")
    params = O.MGParams(coarse_tol=0.0, coarse_maxit=8, lmax=ctx.lmax())
    mg = O.PMG(levels, params=params)
    L0 = levels[0]
    r = L0.mask(np.random.default_rng(3).standard_normal(L0.n_G))
    # smoother from zero and from a nonzero guess
    x = torch.zeros(L0.x.size, dtype=torch.float64, device=dev())
    ctx.cheb_smooth(0, T(_gL(L0, r)), x, x_is_zero=True)
    ref = mg.smooth(0, r, None)
    assert relmax(H(x), _gL(L0, ref)) < 1e-12
    ctx.cheb_smooth(0, T(_gL(L0, r)), x, x_is_zero=False)
    ref = mg.smooth(0, r, ref)
    assert relmax(H(x), _gL(L0, ref)) < 1e-12
    # one full V-cycle (fixed coarse iteration count on both sides)
    z = H(ctx.vcycle(T(_gL(L0, r))))
    assert relmax(z, _gL(L0, mg(r))) < 1e-10


def test_pmg_fcg_fixed_iterations_match_oracle():
    dev()
    mesh, ctx, levels = _mg_pair()
    L0 = levels[0]
    b = si.gaussian_assembled_rhs(mesh, 0)
    bg = L0.mask(global_from_L(L0, b))
    K = 6
    x, info = ctx.solve(T(b), tol=0.0, maxit=K, precond="pmg", rhs="assembled", raise_on_error=False)
    assert info["iters"] == K
    params = O.MGParams(coarse_tol=0.0, coarse_maxit=8, lmax=info["lmax"])
    mg = O.PMG(levels, params=params)
    ref = O.pcg(lambda v: L0.apply(v), bg, mg, 0.0, K, flexible=True)
    assert relmax(H(x), _gL(L0, ref.x)) < 1e-10
    assert abs(info["relres"] - ref.relres) < 1e-8 * ref.relres + 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16g"])
def test_pmg_solve_to_1e8_residual_checked_by_oracle(prec):
    dev()
    mesh = si.box_mesh((4, 4, 4), 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    b = si.gaussian_assembled_rhs(mesh, 0)
    x, info = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec=prec, rhs="assembled")
    assert info["relres"] <= 1e-8
    bg = lev.mask(global_from_L(lev, b))
    xg = global_from_L(lev, H(x))
    true_res = np.linalg.norm(bg - lev.apply(xg)) / np.linalg.norm(bg)
    assert true_res < 2e-8
    ref = O.solve(lev, bg, tol=1e-13, maxit=5000)
    err = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    assert err < 1e-5, err    # kappa * 1e-8 at most


def test_solve_helmholtz_x0_and_nodal_rhs():
    dev()
    mesh = si.box_mesh((3, 2, 2), 6, warp=0.1, perm_seed=2)
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    f = si.smooth_random_field(mesh, 5)
    x0 = si.uniform_field(mesh, 1) * (1 - mesh["dirichlet"])
    x, info = ctx.solve(T(f), h1=0.7, h2=2.0, tol=1e-13, maxit=2000, x0=T(x0))
    ref = O.solve(lev, lev.rhs_from_nodal(f), 0.7, 2.0, tol=1e-14, maxit=2000)
    assert relmax(H(x), _gL(lev, ref.x)) < 1e-9


@pytest.mark.parametrize("smoother", ["jacobi", "asm"])
def test_pmg_solve_graph_replay_matches_direct_launches(smoother):
    """From its second iteration the flexible-CG solve replays the preconditioner step
    (V-cycle, beta, direction) from a CUDA graph. Repeated solves on one context give
    identical bits, and match a context whose coarse execution waits on the host (the
    batched kernels: its capture fails, so it launches directly) to the rounding of the
    different coarse summation orders."""
    dev()
    mesh = si.box_mesh((4, 4, 4), 7, warp=0.1, perm_seed=1, dirichlet=("x0",))
    b = T(si.gaussian_assembled_rhs(mesh, 3))
    ctx = ctx_for(mesh, smoother=smoother, coarse_mode="pipe", coarse_tol=0.0, coarse_maxit=20)
    x1, i1 = ctx.solve(b, tol=1e-9, maxit=200, precond="pmg", prec="fp64", rhs="assembled")
    x2, i2 = ctx.solve(b, tol=1e-9, maxit=200, precond="pmg", prec="fp64", rhs="assembled")
    assert i1["iters"] == i2["iters"] > 2
    # every preconditioner step after the first V-cycle of a solve comes from the graph
    assert i1["graph_steps"] == i2["graph_steps"] == i1["iters"] - 1
    assert np.array_equal(H(x1), H(x2))
    ref = ctx_for(mesh, smoother=smoother, coarse_mode="kernels", coarse_tol=0.0, coarse_maxit=20)
    x3, i3 = ref.solve(b, tol=1e-9, maxit=200, precond="pmg", prec="fp64", rhs="assembled")
    assert i3["iters"] == i1["iters"] and i3["graph_steps"] == 0
    assert relmax(H(x1), H(x3)) < 1e-9


def test_pmg_solve_with_pair_arithmetic_outer_operator():
    dev()
    mesh = si.box_mesh((4, 4, 4), 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    ctx = ctx_for(mesh)
    lev = O.level_from_mesh(mesh)
    b = si.gaussian_assembled_rhs(mesh, 0)
    x, info = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec="fp32", rhs="assembled", outer_pairs=True)
    bg = lev.mask(global_from_L(lev, b))
    xg = global_from_L(lev, H(x))
    true_res = np.linalg.norm(bg - lev.apply(xg)) / np.linalg.norm(bg)
    assert info["relres"] <= 1e-8 and true_res < 2e-8


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-4), ("bf16g", 5e-2)])
def test_low_precision_vcycle_matches_oracle(prec, tol):
    """FP32 / BF16-factor V-cycle (pipelined order-1 coarse solve) against
    the FP64 oracle V-cycle with the same eigenvalue bounds and 8 coarse iterations.
    Tolerance: FP32 rounding (6e-8) amplified by the V-cycle's operator norm, and the
    BF16 factor rounding (4e-3) for the BF16 variant."""
    dev()
    mesh, ctx, levels = _mg_pair(shape=(4, 3, 3), N=7, orders=(7, 3, 1))
    ctx.precond_setup(1.0, 0.0, prec)
    params = O.MGParams(coarse_tol=0.0, coarse_maxit=8, lmax=ctx.lmax())
    mg = O.PMG(levels, params=params)
    L0 = levels[0]
    r = L0.mask(np.random.default_rng(5).standard_normal(L0.n_G))
    z = H(ctx.vcycle(T(_gL(L0, r))))
    err = relmax(z, _gL(L0, mg(r)))
    print(f"{prec} V-cycle relmax {err:.3e}")
    assert err < tol


def test_pmg_solve_48cube_all_precisions_residual_by_oracle():
    """The 48^3-element N=7 pressure problem (56.6M local points): FP64, FP32, BF16-factor and
    FP32 + pair-arithmetic outer operator each reach ||r||/||b|| <= 1e-8, and the oracle's own
    residual of every GPU solution is <= 2e-8; the solutions agree with each other to the
    accuracy 1e-8 residuals allow."""
    dev()
    mesh = si.box_mesh(48, 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    ctx = ctx_for(mesh)
    b = si.gaussian_assembled_rhs(mesh, 0)
    bt = T(b)
    sols = {}
    for name, prec, op in (("fp64", "fp64", False), ("fp32", "fp32", False), ("bf16g", "bf16g", False),
                           ("fp32_pairs", "fp32", True)):
        x, info = ctx.solve(bt, tol=1e-8, maxit=300, precond="pmg", prec=prec, rhs="assembled", outer_pairs=op)
        assert info["relres"] <= 1e-8, (name, info)
        sols[name] = H(x)
        print(name, info["iters"], info["relres"])
    del ctx, bt
    lev = O.level_from_mesh(mesh)
    bg = lev.mask(global_from_L(lev, b))
    nb = np.linalg.norm(bg)
    ref = global_from_L(lev, sols["fp64"])
    for name, xs in sols.items():
        xg = global_from_L(lev, xs)
        res = np.linalg.norm(bg - lev.apply(xg)) / nb
        diff = np.linalg.norm(xg - ref) / np.linalg.norm(ref)
        print(f"{name}: oracle residual {res:.3e}, difference from the FP64 solve {diff:.3e}")
        assert res < 2e-8, (name, res)
        assert diff < 1e-5, (name, diff)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4), ("bf16g", 1e-4)])
def test_coarse_solve_executions_agree(prec, tol):
    """The two executions of the coarse Jacobi-PCG (pipelined PCG on sub-domains in one
    cooperative launch, and batched kernels) run the same iterates in exact arithmetic: one
    V-cycle with 8 coarse iterations gives the same result up to the rounding of their
    different summation orders."""
    dev()
    mesh = si.box_mesh((4, 3, 3), 7, warp=0.1, perm_seed=6, dirichlet=("x0",))
    L0 = O.level_from_mesh(mesh)
    r = L0.mask(np.random.default_rng(5).standard_normal(L0.n_G))
    zs = {}
    for mode in ("auto", "pipe", "kernels"):
        ctx = ctx_for(mesh, mg_orders=[7, 3, 1], coarse_tol=0.0, coarse_maxit=8, coarse_mode=mode)
        ctx.precond_setup(1.0, 0.0, prec)
        zs[mode] = H(ctx.vcycle(T(_gL(L0, r))))
        ctx.close()
    assert np.array_equal(zs["auto"], zs["pipe"])
    assert relmax(zs["pipe"], zs["kernels"]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pipelined_coarse_solve_is_deterministic(prec):
    """Every block of the pipelined coarse solve adds the same copies and the same block
    partials in the same order, so repeated V-cycles (each a fresh cooperative launch whose
    blocks run in a different interleaving) return identical bits; a torn or stale read of
    the exchanged words would show up as a difference."""
    dev()
    mesh = si.box_mesh((6, 5, 4), 7, warp=0.1, perm_seed=2, dirichlet=("x0",))
    L0 = O.level_from_mesh(mesh)
    r = T(_gL(L0, L0.mask(np.random.default_rng(11).standard_normal(L0.n_G))))
    ctx = ctx_for(mesh, mg_orders=[7, 3, 1], coarse_tol=1e-6, coarse_maxit=200, coarse_mode="pipe")
    ctx.precond_setup(1.0, 0.0, prec)
    z0 = H(ctx.vcycle(r))
    for _ in range(5):
        assert np.array_equal(H(ctx.vcycle(r)), z0)
    ctx.close()


def test_pipelined_coarse_solve_on_the_48cube_coarse_level():
    """At 48^3 elements the coarse level (110,592 order-1 elements) splits into sub-domains
    of about 730 elements in the pipelined solve; one FP32 V-cycle agrees with the
    batched-kernel solve to FP32 rounding."""
    dev()
    mesh = si.box_mesh(48, 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    b = T(si.gaussian_assembled_rhs(mesh, 0))
    zs = {}
    for mode in ("pipe", "kernels"):
        ctx = ctx_for(mesh, coarse_tol=0.0, coarse_maxit=6, coarse_mode=mode, prec_copies=1)
        ctx.precond_setup(1.0, 0.0, "fp32")
        zs[mode] = H(ctx.vcycle(b))
        ctx.close()
    assert relmax(zs["pipe"], zs["kernels"]) < 1e-4
