"""GPU dealiased advection operator (sem_advect) vs the oracle (Sections 2.1 and 3.3).

Element-local and assembled results are compared point by point with the
oracle's advect_local / advect_assembled (FP64 to 1e-12, FP32 pairs to 3e-11,
32 times the FP64 bar for the pair format's 2^-48 against 2^-53, FP32 to single
precision), for every compiled order on small warped meshes, and on a sample
of elements of the 32^3-element N = 7 box (the oracle evaluates the sampled
elements alone: the local operator is element by element).
"""
import types

import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, ctx_for, dev, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fields(mesh, seed):
    c = np.stack([si.smooth_random_field(mesh, seed + q, modes=16, kmax=3) for q in range(3)])
    u = np.stack([si.smooth_random_field(mesh, seed + 10 + q, modes=16, kmax=3) for q in range(3)])
    return c, u


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7, 8])
def test_advect_local_and_assembled_match_oracle(N):
    dev()
    mesh = si.box_mesh((3, 2, 2), N, warp=0.1, perm_seed=N, dirichlet=("x0",))
    lev = O.level_from_mesh(mesh)
    cub = O.cubature_setup(lev)
    ctx = ctx_for(mesh, prec_copies=0)
    c, u = _fields(mesh, 3 * N)
    ct, ut = T(c.reshape(3, -1)).reshape(3, -1), T(u.reshape(3, -1)).reshape(3, -1)
    w = H(ctx.advect(ct, ut))
    for q in range(3):
        ref = O.advect_local(lev, cub, c, u[q])
        assert relmax(w[q], ref.ravel()) < 1e-12, (N, q)
    wa = H(ctx.advect(ct, ut, assemble=True))
    for q in range(3):
        ref = O.q_scatter(O.advect_local(lev, cub, c, u[q]), lev.node, lev.n_G)[lev.node]
        assert relmax(wa[q], ref) < 1e-12, (N, q)
    w32 = H(ctx.advect(ct.float(), ut.float(), prec="fp32"))
    for q in range(3):
        ref = O.advect_local(lev, cub, c, u[q])
        assert relmax(w32[q], ref.ravel()) < 5e-5, (N, q)
    wp = H(ctx.advect(ct, ut, prec="fp64p"))
    wpa = H(ctx.advect(ct, ut, assemble=True, prec="fp64p"))
    for q in range(3):
        ref = O.advect_local(lev, cub, c, u[q])
        refa = O.q_scatter(ref, lev.node, lev.n_G)[lev.node]
        print(f"N={N} q={q}: FP32-pair error {relmax(wp[q], ref.ravel()):.2e} (local), {relmax(wpa[q], refa):.2e} (assembled)")
        assert relmax(wp[q], ref.ravel()) < 3e-11, (N, q)
        assert relmax(wpa[q], refa) < 3e-11, (N, q)


def test_advect_sample_of_the_32cube_box():
    dev()
    N = 7
    mesh = si.box_mesh(32, N, warp=0.1, perm_seed=0)
    ctx = ctx_for(mesh, prec_copies=0, mg_orders=[7])
    rng = np.random.default_rng(5)
    c = rng.standard_normal((3,) + mesh["x"].shape)
    u = rng.standard_normal((3,) + mesh["x"].shape)
    w = H(ctx.advect(T(c.reshape(3, -1)).reshape(3, -1), T(u.reshape(3, -1)).reshape(3, -1)))
    w = w.reshape(3, *mesh["x"].shape)
    pick = np.random.default_rng(0).choice(mesh["E"], 48, replace=False)
    xi, _ = O.gll(N)
    sub = types.SimpleNamespace(N=N, xi=xi, x=mesh["x"][pick], y=mesh["y"][pick], z=mesh["z"][pick])
    cub = O.cubature_setup(sub)
    wp = H(ctx.advect(T(c.reshape(3, -1)).reshape(3, -1), T(u.reshape(3, -1)).reshape(3, -1), prec="fp64p"))
    wp = wp.reshape(3, *mesh["x"].shape)
    for q in range(3):
        ref = O.advect_local(sub, cub, c[:, pick], u[q][pick])
        assert relmax(w[q][pick], ref) < 1e-12
        assert relmax(wp[q][pick], ref) < 3e-11


def test_advect_argument_errors():
    from paper_2104_05829_gb300 import SemError
    dev()
    mesh = si.box_mesh(2, 3, warp=0.0)
    ctx = ctx_for(mesh, prec_copies=0)
    n = ctx.nL
    c = torch.zeros(3 * n, dtype=torch.float64, device=dev())
    u = torch.zeros(n, dtype=torch.float64, device=dev())
    with pytest.raises(SemError):
        ctx.advect(c, u, w=u)                      # output aliases the input
    hi = ctx_for(si.box_mesh(1, 9, warp=0.0), prec_copies=0, mg_orders=[9])
    with pytest.raises(SemError):
        hi.advect(torch.zeros(3 * hi.nL, dtype=torch.float64, device=dev()),
                  torch.zeros(hi.nL, dtype=torch.float64, device=dev()))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp64p", 3e-10), ("fp32", 1e-3)])
def test_char_advance_matches_oracle(prec, tol):
    """RK4 substeps of the characteristics subproblem with a wind linear in time. FP32:
    twelve stage evaluations, each within 5e-5 of the operator's scale, summed into w with
    the inverse mass; the advected change over the interval is several times |w| here."""
    dev()
    mesh = si.box_mesh((3, 2, 2), 5, warp=0.1, perm_seed=9, dirichlet=())
    lev = O.level_from_mesh(mesh)
    cub = O.cubature_setup(lev)
    ctx = ctx_for(mesh, prec_copies=0)
    c0 = np.stack([si.smooth_random_field(mesh, 40 + q, modes=8, kmax=2) for q in range(3)])
    c1 = np.stack([si.smooth_random_field(mesh, 50 + q, modes=8, kmax=2) for q in range(3)])
    wg = [O.q_scatter(si.smooth_random_field(mesh, 60 + q, modes=8, kmax=2), lev.node, lev.n_G)
          / np.bincount(lev.node, minlength=lev.n_G) for q in range(2)]
    ref = O.char_advance(lev, cub, c0, c1, wg, 0.1, 0.3, 3)
    dt = torch.float32 if prec == "fp32" else torch.float64
    w = torch.stack([T(g[lev.node]) for g in wg]).to(dt).contiguous()
    ctx.char_advance(T(c0.reshape(3, -1)).reshape(3, -1).to(dt).contiguous(), w, 0.1, 0.3, 3,
                     c1=T(c1.reshape(3, -1)).reshape(3, -1).to(dt).contiguous(), prec=prec)
    got = H(w)
    for q in range(2):
        assert relmax(got[q], ref[q][lev.node]) < tol, q


def test_char_advance_translates_a_linear_field():
    dev()
    mesh = si.box_mesh((2, 3, 2), 4, warp=0.0, perm_seed=2, dirichlet=())
    ctx = ctx_for(mesh, prec_copies=0)
    a = np.array([0.4, -0.3, 0.8])
    bvec = np.array([1.5, 2.0, -0.5])
    x, y, z = mesh["x"].ravel(), mesh["y"].ravel(), mesh["z"].ravel()
    w0 = bvec[0] * x + bvec[1] * y + bvec[2] * z
    c = T(np.stack([np.full_like(x, q) for q in a]).ravel()).reshape(3, -1)
    w = T(w0)
    ctx.char_advance(c, w, 0.0, 0.3, 4)
    assert relmax(H(w), w0 - (a @ bvec) * 0.3) < 1e-12
