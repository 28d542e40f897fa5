"""p-multigrid flexible-CG solves at the library's production settings vs the oracle.

The pressure solve of Section 3.4 runs with every default: orders 7 -> 3 -> 1,
degree-2 Chebyshev smoothing (Jacobi or overlapping Schwarz), the pipelined
sub-domain coarse Jacobi-PCG with its early stop at ||r_c|| <= 1e-1 ||b_c||
(at most 100 iterations), the preconditioner steps replayed from a CUDA graph.
The oracle runs the same algorithm with the same parameters (its coarse PCG
stops by the same rule; only the eigenvalue estimates are read from the GPU,
whose Lanczos/Arnoldi runs are pinned separately), so both take the same outer
and coarse iteration counts and their iterates agree to 1e-10.

The mixed-precision variants (FP32 and BF16-factor V-cycles, FP64 or FP32-pair
outer operator) are judged by the oracle's own residual of every GPU solution
and by their FP64 error against a reference solution whose oracle residual is
at round-off level.
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


@pytest.mark.parametrize("smoother", ["jacobi", "asm"])
def test_fp64_pmg_fcg_default_settings_match_oracle(smoother):
    """FP64 FCG + p-MG 7-3-1 on a warped 9x8x7 box (504 elements: the coarse level spans
    63 sub-domains of the pipelined solve) with x=0 Dirichlet and the Gaussian assembled
    right-hand side, to ||r||/||b|| <= 1e-8 with default options."""
    dev()
    mesh = si.box_mesh((9, 8, 7), 7, warp=0.1, perm_seed=3, dirichlet=("x0",))
    ctx = ctx_for(mesh, smoother=smoother)           # every other option at its default
    d = O.MGParams()
    assert (d.coarse_tol, d.coarse_maxit, d.degree) == (1e-1, 100, 2)
    levels = O.build_levels(mesh, [7, 3, 1])
    L0 = levels[0]
    b = si.gaussian_assembled_rhs(mesh, 0)
    x, info = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec="fp64", rhs="assembled")
    assert info["graph_steps"] == info["iters"] - 1     # the captured (pipelined) coarse execution ran
    mg = O.PMG(levels, params=O.MGParams(smoother=smoother, lmax=info["lmax"]))
    bg = L0.mask(global_from_L(L0, b))
    ref = O.pcg(lambda v: L0.apply(v), bg, mg, 1e-8, 200, flexible=True)
    print(f"{smoother}: outer {info['iters']} (oracle {ref.iters}), coarse {info['coarse_iters']} "
          f"(oracle {sum(mg.coarse_iters)} over {len(mg.coarse_iters)} cycles: {mg.coarse_iters})")
    assert info["iters"] == ref.iters
    # the early-stopped coarse solves took the same number of iterations in every cycle
    # (the totals agree and each cycle stops by the same rule)
    assert info["coarse_iters"] == sum(mg.coarse_iters)
    assert max(mg.coarse_iters) < 100 and min(mg.coarse_iters) > 1
    assert info["relres"] <= 1e-8 and ref.relres <= 1e-8
    assert relmax(H(x), _gL(L0, ref.x)) < 1e-10
    assert abs(info["relres"] - ref.relres) < 1e-6 * ref.relres


# the nine solve variants the benchmark times: (name, V-cycle precision, pair outer operator, smoother)
VARIANTS = (("fp64", "fp64", False, "jacobi"), ("fp32", "fp32", False, "jacobi"),
            ("bf16g", "bf16g", False, "jacobi"), ("fp32_outer_pairs", "fp32", True, "jacobi"),
            ("bf16g_outer_pairs", "bf16g", True, "jacobi"),
            ("asm_fp64", "fp64", False, "asm"), ("asm_fp32", "fp32", False, "asm"),
            ("asm_fp32_outer_pairs", "fp32", True, "asm"), ("asm_bf16g_outer_pairs", "bf16g", True, "asm"))


def test_24cube_every_solve_variant_by_the_oracle():
    """The 24^3-element N=7 pressure problem (7.08M local points) in every variant the
    benchmark times. The reference is the FP64 solve to 1e-13, whose oracle residual must
    be at round-off level; every variant reaches 1e-8 by its own residual and by the
    oracle's, and its FP64 error against the reference is reported."""
    dev()
    mesh = si.box_mesh(24, 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    b = si.gaussian_assembled_rhs(mesh, 0)
    bt = T(b)
    ctxs = {sm: ctx_for(mesh, smoother=sm) for sm in ("jacobi", "asm")}
    xref, iref = ctxs["jacobi"].solve(bt, tol=1e-13, maxit=400, precond="pmg", prec="fp64", rhs="assembled")
    sols, infos = {}, {}
    for name, prec, op, sm in VARIANTS:
        x, info = ctxs[sm].solve(bt, tol=1e-8, maxit=300, precond="pmg", prec=prec, rhs="assembled", outer_pairs=op)
        assert info["relres"] <= 1e-8, (name, info)
        sols[name], infos[name] = H(x), info
    xref = H(xref)
    for c in ctxs.values():
        c.close()
    del bt
    lev = O.level_from_mesh(mesh)
    bg = lev.mask(global_from_L(lev, b))
    nb = np.linalg.norm(bg)
    xr = global_from_L(lev, xref)
    res_ref = np.linalg.norm(bg - lev.apply(xr)) / nb
    print(f"reference: FP64 FCG to 1e-13 in {iref['iters']} iterations, oracle residual {res_ref:.3e}")
    assert res_ref < 1e-11
    for name, _, _, _ in VARIANTS:
        xg = global_from_L(lev, sols[name])
        res = np.linalg.norm(bg - lev.apply(xg)) / nb
        err = np.linalg.norm(xg - xr) / np.linalg.norm(xr)
        errmax = np.max(np.abs(xg - xr)) / np.max(np.abs(xr))
        print(f"{name}: {infos[name]['iters']} it, own residual {infos[name]['relres']:.3e}, oracle residual "
              f"{res:.3e}, FP64 error vs reference {err:.3e} (2-norm) {errmax:.3e} (max-norm)")
        assert res < 2e-8, (name, res)
        assert err < 1e-5, (name, err)


def _zero_mean(level, xL):
    """Unique-node vector of a continuous L-vector with its unique-node mean removed."""
    xg = global_from_L(level, xL)
    return xg - xg.mean()


@pytest.mark.parametrize("smoother", ["jacobi", "asm"])
def test_all_neumann_pressure_problem_matches_oracle(smoother):
    """The singular case: no Dirichlet face, h2 = 0, so A 1 = 0 and the pressure is fixed up to a
    constant. The Gaussian right-hand side has zero mean over the unique nodes, so it lies in the
    range of A and every restricted residual does too (P interpolates constants exactly). The GPU
    and the oracle run the same FCG + p-MG with default settings to 1e-8 in the same number of
    iterations and agree, up to a constant, to 1e-10; the FP32 V-cycle reaches the same residual
    by the oracle's own measure."""
    dev()
    mesh = si.box_mesh((5, 4, 3), 7, warp=0.1, perm_seed=5, dirichlet=())
    ctx = ctx_for(mesh, smoother=smoother)
    levels = O.build_levels(mesh, [7, 3, 1])
    L0 = levels[0]
    assert L0.mask(np.ones(L0.n_G)).min() == 1.0            # no Dirichlet node anywhere
    b = si.gaussian_assembled_rhs(mesh, 2)
    bg = global_from_L(L0, b)
    assert abs(bg.sum()) < 1e-9 * np.abs(bg).sum()
    x, info = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec="fp64", rhs="assembled")
    mg = O.PMG(levels, params=O.MGParams(smoother=smoother, lmax=info["lmax"]))
    ref = O.pcg(lambda v: L0.apply(v), bg, mg, 1e-8, 200, flexible=True)
    print(f"{smoother}: outer {info['iters']} (oracle {ref.iters}), coarse {info['coarse_iters']} "
          f"(oracle {sum(mg.coarse_iters)})")
    assert info["iters"] == ref.iters and info["relres"] <= 1e-8
    xr = ref.x - ref.x.mean()
    assert relmax(_zero_mean(L0, H(x)), xr) < 1e-10
    x32, i32 = ctx.solve(T(b), tol=1e-8, maxit=200, precond="pmg", prec="fp32", rhs="assembled")
    xg = global_from_L(L0, H(x32))
    res = np.linalg.norm(bg - L0.apply(xg)) / np.linalg.norm(bg)
    assert i32["relres"] <= 1e-8 and res < 2e-8
    assert relmax(_zero_mean(L0, H(x32)), xr) < 1e-5
