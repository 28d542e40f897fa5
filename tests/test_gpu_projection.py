"""GPU projection of successive right-hand sides (sem_proj_*, sem_solve_proj) vs the oracle.

Step parity: the oracle's project and update steps, run on the basis the GPU
holds, give the GPU's projected guess, residual and new basis vector. Sequence
parity: GPU and oracle projected solves of the same right-hand sides take the
same iteration counts, start from the same projected residual, and both meet
the tolerance on the oracle's own residual of the GPU solution.
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, ctx_for, dev, global_from_L, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mesh():
    return si.box_mesh((3, 2, 3), 5, warp=0.1, perm_seed=3, dirichlet=("x0", "z1"))


def _rhs(lev, seed):
    return lev.mask(np.random.default_rng(seed).standard_normal(lev.n_G))


def _gpu_basis(proj, lev):
    X, AX = [], []
    for i in range(len(proj)):
        x, a = proj.vectors(i)
        X.append(global_from_L(lev, H(x)))
        AX.append(global_from_L(lev, H(a)))
    return X, AX


def test_projection_steps_match_oracle_on_the_gpu_basis():
    from paper_2104_05829_gb300 import Projection
    dev()
    mesh = _mesh()
    lev = O.level_from_mesh(mesh)
    ctx = ctx_for(mesh)
    proj = Projection(ctx, 6)
    h2 = 0.3
    for s in range(3):
        b = _rhs(lev, s)
        ctx.solve(T(b[lev.node]), 1.0, h2, tol=1e-12, maxit=2000, rhs="assembled", proj=proj)
    assert len(proj) == 3
    X, AX = _gpu_basis(proj, lev)
    op = lambda v: lev.apply(v, 1.0, h2)
    # the stored basis is A-orthonormal and carries A x_i, by the oracle's operator
    G = np.array([[xi @ op(xj) for xj in X] for xi in X])
    assert np.max(np.abs(G - np.eye(3))) < 1e-12
    for xi, ai in zip(X, AX):
        assert relmax(ai, op(xi)) < 1e-12
    # project: same xbar and r0 as the oracle on that basis
    ref = O.Projection(op, 6)
    ref.X, ref.AX = [x.copy() for x in X], [a.copy() for a in AX]
    b = _rhs(lev, 9)
    xbar, r0 = proj.project(T(b[lev.node]))
    xr, rr = ref.project(b)
    assert relmax(H(xbar), xr[lev.node]) < 1e-13
    assert relmax(H(r0), rr[lev.node]) < 1e-13
    # update: the same new direction
    dx = lev.mask(np.random.default_rng(11).standard_normal(lev.n_G))
    assert proj.update(T(dx[lev.node]), h1=1.0, h2=h2)
    assert ref.update(None, dx)
    assert len(proj) == 4
    x4, a4 = proj.vectors(3)
    assert relmax(global_from_L(lev, H(x4)), ref.X[3]) < 1e-11
    assert relmax(global_from_L(lev, H(a4)), ref.AX[3]) < 1e-11


@pytest.mark.parametrize("precond", ["jacobi", "pmg"])
def test_projected_sequence_matches_oracle(precond):
    from paper_2104_05829_gb300 import Projection
    dev()
    mesh = si.box_mesh(3, 5, warp=0.1, perm_seed=1)
    lev = O.level_from_mesh(mesh)
    ctx = ctx_for(mesh, mg_orders=[5, 2, 1])
    proj = Projection(ctx, 4)
    op = lambda v: lev.apply(v)
    ref = O.Projection(op, 4)
    mg = None
    if precond == "pmg":
        levels = O.build_levels(mesh, [5, 2, 1])
        ctx.precond_setup(1.0, 0.0, "fp64")
        mg = O.PMG(levels, 1.0, 0.0, O.MGParams(lmax=ctx.lmax()))
    tol = 1e-10
    for k in range(7):
        f = si.travelling_field(mesh, 5, 0.02 * k)
        b = lev.rhs_from_nodal(f)
        u, info = ctx.solve(T(f), tol=tol, maxit=2000, precond=precond, proj=proj)
        res = O.solve_projected(lev, ref, b, tol=tol, maxit=2000, precond=precond, mg=mg)
        ug = global_from_L(lev, H(u))
        # the oracle's residual of the GPU solution meets the tolerance
        assert np.linalg.norm(b - op(ug)) <= 1.05 * tol * np.linalg.norm(b)
        assert abs(info["iters"] - res.iters) <= 1, (k, info["iters"], res.iters)
        assert abs(info["relres0"] - res.relres0) <= 1e-3 * res.relres0 + 1e-9, (k, info["relres0"], res.relres0)
        assert info["proj_count"] == len(ref.X)
        assert relmax(ug, res.x) < 1e-5
    # the restart happened (4 vectors, 7 solves) and the later solves were cheaper than the first
    assert info["proj_count"] <= 4


def test_rhs_in_span_and_operator_change():
    from paper_2104_05829_gb300 import Projection
    dev()
    mesh = _mesh()
    lev = O.level_from_mesh(mesh)
    ctx = ctx_for(mesh)
    proj = Projection(ctx, 8)
    b1, b2 = _rhs(lev, 1), _rhs(lev, 2)
    for b in (b1, b2):
        ctx.solve(T(b[lev.node]), 1.0, 0.2, tol=1e-13, maxit=3000, rhs="assembled", proj=proj)
    u, info = ctx.solve(T((2.0 * b1 - 0.5 * b2)[lev.node]), 1.0, 0.2, tol=1e-9, maxit=3000, rhs="assembled",
                        proj=proj)
    assert info["iters"] == 0 and info["relres0"] < 1e-11
    assert info["proj_count"] == 2          # nothing new to keep
    # a new operator (h2 changed) empties the space before the solve
    u, info = ctx.solve(T(b1[lev.node]), 1.0, 0.5, tol=1e-9, maxit=3000, rhs="assembled", proj=proj)
    assert info["relres0"] == pytest.approx(1.0, abs=1e-14) and info["proj_count"] == 1
    ref = O.solve(lev, b1, 1.0, 0.5, tol=1e-13, maxit=5000).x
    assert relmax(global_from_L(lev, H(u)), ref) < 1e-6


def test_projection_argument_errors():
    from paper_2104_05829_gb300 import Projection, SemError
    dev()
    mesh = _mesh()
    lev = O.level_from_mesh(mesh)
    ctx = ctx_for(mesh)
    for bad in (0, 17):
        with pytest.raises(SemError):
            Projection(ctx, bad)
    proj = Projection(ctx, 2)
    with pytest.raises(SemError):
        proj.vectors(0)
    b = T(_rhs(lev, 1)[lev.node])
    with pytest.raises(SemError):
        ctx.solve(b, rhs="assembled", x0=torch.zeros_like(b), proj=proj)
    other = ctx_for(mesh)
    with pytest.raises(SemError):
        other.solve(b, rhs="assembled", proj=proj)
    proj.reset()
    assert len(proj) == 0
