"""GPU dealiased advection operator (sem_advect) vs the oracle (Sections 2.1 and 3.3).

Element-local and assembled results are compared point by point with the
oracle's advect_local / advect_assembled (FP64 to 1e-12, FP32 to single
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
    for q in range(3):
        ref = O.advect_local(sub, cub, c[:, pick], u[q][pick])
        assert relmax(w[q][pick], ref) < 1e-12


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
