"""GPU overlapping Schwarz smoother with fast-diagonalisation local solves and
CHEBY-ASM p-multigrid (Section 3.4) vs the oracle.

The Schwarz application is compared element by element (FP64 to round-off,
FP32 to single-precision accuracy); the Arnoldi eigenvalue bounds, the
Chebyshev-Schwarz smoother, one V-cycle and a fixed number of FCG iterations
are compared with the oracle run on the same parameters; full solves are
judged by the oracle's own residual of the GPU solution.
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


def _mg_pair(shape=(3, 3, 3), N=5, orders=(5, 2, 1), coarse_maxit=8, dirichlet=("x0",)):
    mesh = si.box_mesh(shape, N, warp=0.1, perm_seed=6, dirichlet=dirichlet)
    opts = dict(mg_orders=list(orders), coarse_tol=0.0, coarse_maxit=coarse_maxit, smoother="asm")
    ctx = ctx_for(mesh, **opts)
    levels = O.build_levels(mesh, list(orders))
    return mesh, ctx, levels


@pytest.mark.parametrize("N,orders", [(5, (5, 2, 1)), (7, (7, 3, 1))])
def test_asm_apply_matches_oracle_on_every_smoothed_level(N, orders):
    dev()
    mesh, ctx, levels = _mg_pair(shape=(3, 2, 3), N=N, orders=orders, dirichlet=("x0", "z1"))
    rng = np.random.default_rng(N)
    for l, Lo in enumerate(levels[:-1]):
        sch = O.schwarz_setup(Lo)
        assert set(np.unique(sch.btype)) == {O.SCH_NB, O.SCH_DIR, O.SCH_NEU}
        r = Lo.mask(rng.standard_normal(Lo.n_G))
        for h1, h2 in ((1.0, 0.0), (0.7, 2.5)):
            ref = O.asm_apply(Lo, sch, r, h1, h2)
            z = H(ctx.asm_apply(l, T(_gL(Lo, r)), h1=h1, h2=h2))
            assert relmax(z, _gL(Lo, ref)) < 1e-12, (l, h1, h2)
            z32 = H(ctx.asm_apply(l, T(_gL(Lo, r), torch.float32), h1=h1, h2=h2, prec="fp32"))
            assert relmax(z32, _gL(Lo, ref)) < 2e-5, (l, h1, h2)


@pytest.mark.parametrize("N,orders", [(5, (5, 2, 1)), (7, (7, 3, 1))])
def test_asm_apply_tf32_tensor_cores_match_oracle(N, orders):
    """The BF16-G V-cycle's Schwarz application: the FDM local solves as TF32 tensor-core
    products (operands rounded to 11 significant bits, FP32 accumulation), on levels with an
    even box edge (N = 7, 3: paired stores) and an odd one (N = 5, 2), all side types and 18
    elements (not a multiple of the four elements of a block)."""
    dev()
    mesh, ctx, levels = _mg_pair(shape=(3, 2, 3), N=N, orders=orders, dirichlet=("x0", "z1"))
    rng = np.random.default_rng(10 + N)
    for l, Lo in enumerate(levels[:-1]):
        sch = O.schwarz_setup(Lo)
        r = Lo.mask(rng.standard_normal(Lo.n_G))
        for h1, h2 in ((1.0, 0.0), (0.7, 2.5)):
            ref = _gL(Lo, O.asm_apply(Lo, sch, r, h1, h2))
            z = H(ctx.asm_apply(l, T(_gL(Lo, r), torch.float32), h1=h1, h2=h2, prec="bf16g"))
            err_max = relmax(z, ref)
            err_2 = np.linalg.norm(z - ref) / np.linalg.norm(ref)
            print(f"N={Lo.N} h1={h1} h2={h2}: TF32 Schwarz error {err_max:.2e} (max) {err_2:.2e} (2-norm)")
            assert err_max < 2e-2 and err_2 < 5e-3, (l, h1, h2, err_max, err_2)


@pytest.mark.parametrize("N", [8, 9, 10, 11])
def test_asm_apply_high_orders_every_precision_match_oracle(N):
    """Box edges M = N + 3 = 11..14: the tensor-core tile plans with padded rows (M = 11, 13, 14)
    and with grouped remainder lines (M = 12), one and two k-steps, and the largest shared-memory
    blocks; FP64, FP32 (three TF32 products) and TF32 (BF16-G) against the oracle on a 3x2x2 box
    (12 elements) with Dirichlet and Neumann sides."""
    dev()
    mesh = si.box_mesh((3, 2, 2), N, warp=0.1, perm_seed=4, dirichlet=("x0",))
    ctx = ctx_for(mesh, mg_orders=[N], smoother="asm")
    Lo = O.level_from_mesh(mesh)
    sch = O.schwarz_setup(Lo)
    r = Lo.mask(np.random.default_rng(N).standard_normal(Lo.n_G))
    ref = _gL(Lo, O.asm_apply(Lo, sch, r, 0.8, 1.5))
    z = H(ctx.asm_apply(0, T(_gL(Lo, r)), h1=0.8, h2=1.5))
    assert relmax(z, ref) < 1e-12
    z32 = H(ctx.asm_apply(0, T(_gL(Lo, r), torch.float32), h1=0.8, h2=1.5, prec="fp32"))
    assert relmax(z32, ref) < 2e-5
    zt = H(ctx.asm_apply(0, T(_gL(Lo, r), torch.float32), h1=0.8, h2=1.5, prec="bf16g"))
    err_max, err_2 = relmax(zt, ref), np.linalg.norm(zt - ref) / np.linalg.norm(ref)
    print(f"N={N}: FP32 {relmax(z32, ref):.2e}, TF32 {err_max:.2e} (max) {err_2:.2e} (2-norm)")
    assert err_max < 2e-2 and err_2 < 5e-3


def test_asm_apply_full_neumann_box_and_single_element():
    dev()
    for mesh in (si.box_mesh(2, 4, warp=0.1, perm_seed=1, dirichlet=()), si.box_mesh(1, 6, warp=0.0)):
        ctx = ctx_for(mesh)
        Lo = O.level_from_mesh(mesh)
        sch = O.schwarz_setup(Lo)
        r = Lo.mask(np.random.default_rng(2).standard_normal(Lo.n_G))
        ref = _gL(Lo, O.asm_apply(Lo, sch, r, 1.0, 0.5))
        z = H(ctx.asm_apply(0, T(_gL(Lo, r)), h1=1.0, h2=0.5))
        assert relmax(z, ref) < 1e-12
        r32 = T(_gL(Lo, r), torch.float32)
        assert relmax(H(ctx.asm_apply(0, r32, h1=1.0, h2=0.5, prec="fp32")), ref) < 2e-5
        zt = H(ctx.asm_apply(0, r32, h1=1.0, h2=0.5, prec="bf16g"))
        assert relmax(zt, ref) < 2e-2 and np.linalg.norm(zt - ref) < 5e-3 * np.linalg.norm(ref)


def test_arnoldi_bounds_match_oracle():
    dev()
    mesh, ctx, levels = _mg_pair()
    ctx.precond_setup(1.0, 0.0, "fp64")
    lam = ctx.lmax()
    mg = O.PMG(levels, params=O.MGParams(smoother="asm"))
    for a, b in zip(lam, mg.lmax):
        assert abs(a - b) < 1e-10 * b


def test_cheby_asm_smoother_vcycle_and_fcg_match_oracle():
    dev()
    mesh, ctx, levels = _mg_pair()
    ctx.precond_setup(1.0, 0.0, "fp64")
    params = O.MGParams(coarse_tol=0.0, coarse_maxit=8, lmax=ctx.lmax(), smoother="asm")
    mg = O.PMG(levels, params=params)
    L0 = levels[0]
    r = L0.mask(np.random.default_rng(3).standard_normal(L0.n_G))
    x = torch.zeros(L0.x.size, dtype=torch.float64, device=dev())
    ctx.cheb_smooth(0, T(_gL(L0, r)), x, x_is_zero=True)
    ref = mg.smooth(0, r, None)
    assert relmax(H(x), _gL(L0, ref)) < 1e-12
    ctx.cheb_smooth(0, T(_gL(L0, r)), x, x_is_zero=False)
    ref = mg.smooth(0, r, ref)
    assert relmax(H(x), _gL(L0, ref)) < 1e-12
    z = H(ctx.vcycle(T(_gL(L0, r))))
    assert relmax(z, _gL(L0, mg(r))) < 1e-10
    # a fixed number of flexible-PCG iterations
    b = si.gaussian_assembled_rhs(mesh, 0)
    bg = L0.mask(global_from_L(L0, b))
    K = 5
    x, info = ctx.solve(T(b), tol=0.0, maxit=K, precond="pmg", rhs="assembled", raise_on_error=False)
    assert info["iters"] == K
    ref = O.pcg(lambda v: L0.apply(v), bg, O.PMG(levels, params=params), 0.0, K, flexible=True)
    assert relmax(H(x), _gL(L0, ref.x)) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16g"])
def test_cheby_asm_solve_to_1e8_and_fewer_iterations_than_cheby_jacobi(prec):
    dev()
    mesh = si.box_mesh((4, 4, 4), 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    lev = O.level_from_mesh(mesh)
    b = si.gaussian_assembled_rhs(mesh, 0)
    its = {}
    for sm in ("jacobi", "asm"):
        ctx = ctx_for(mesh, smoother=sm)
        x, info = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec=prec, rhs="assembled")
        bg = lev.mask(global_from_L(lev, b))
        xg = global_from_L(lev, H(x))
        true_res = np.linalg.norm(bg - lev.apply(xg)) / np.linalg.norm(bg)
        assert info["relres"] <= 1e-8 and true_res < 2e-8
        its[sm] = info["iters"]
    print(prec, its)
    assert its["asm"] < its["jacobi"], its
