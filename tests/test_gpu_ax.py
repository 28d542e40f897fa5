"""GPU operator kernels vs the oracle through the C ABI.

Tolerances (norm-wise, max|gpu - oracle| / max|oracle|):
* FP64 Ax and gather-scatter: 1e-12 (the paper's FP64 operator; the two
  sides differ only in summation order, a few ulp times the ~N terms per sum);
* FP32 Ax: 2e-6 (unit roundoff 6e-8 times the O(N) terms and the factor
  rounding);
* FP32 arithmetic with BF16 factors: 2e-2 (BF16 keeps 8 bits: 2^-9 = 2e-3 per
  factor, amplified by cancellation in the contraction sums).
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, ctx_for, dev, global_from_L, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(shape, N, warp=0.1, seed=0, **kw):
    mesh = si.box_mesh(shape, N, warp=warp, perm_seed=seed, **kw)
    return mesh, ctx_for(mesh), O.level_from_mesh(mesh)


@pytest.mark.parametrize("N", range(1, 12))
def test_ax_local_fp64_all_orders(N):
    dev()
    mesh, ctx, lev = _setup((3, 2, 5), N, seed=N)   # 30 elements: ragged for every block size
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, mesh["x"].shape)
    for h1, h2 in ((1.0, 0.0), (0.8, 0.5)):
        w = H(ctx.ax(T(u), h1=h1, h2=h2, assemble=False))
        ref = O.ax_local(u, lev.G, lev.B, lev.D, h1, h2).ravel()
        assert relmax(w, ref) < 1e-12, (N, h1, h2)


def test_ax_local_fp64_nodal_h1():
    dev()
    mesh, ctx, lev = _setup((4, 3, 2), 7)
    g = si.smooth_random_field(mesh, seed=1)
    h1 = np.exp(0.5 * g)
    u = si.uniform_field(mesh, 0)
    w = H(ctx.ax(T(u), h1_L=T(h1), h2=1.0, assemble=False))
    assert relmax(w, O.ax_local(u, lev.G, lev.B, lev.D, h1, 1.0).ravel()) < 1e-12


@pytest.mark.parametrize("N,dirichlet", [(7, si.FACES), (3, ("x0",)), (5, ())])
def test_ax_assembled_fp64(N, dirichlet):
    dev()
    mesh, ctx, lev = _setup((4, 4, 3), N, dirichlet=dirichlet)
    u = si.uniform_field(mesh, 0)          # continuous field, Dirichlet entries nonzero
    w = H(ctx.ax(T(u), h1=1.0, h2=0.5, assemble=True))
    # R QQ^T A_L u: the input is used as given, the output is masked
    wl = O.ax_local(u, lev.G, lev.B, lev.D, 1.0, 0.5)
    ref = O.q_gather(lev.mask(O.q_scatter(wl, lev.node, lev.n_G)), lev.node)
    assert relmax(w, ref) < 1e-12
    # with a masked input this is the SPD operator R Q^T A_L Q R^T
    um = np.where(lev.dir_g[lev.node], 0.0, u.ravel())
    w2 = H(ctx.ax(T(um), h1=1.0, h2=0.5, assemble=True))
    assert relmax(w2, O.q_gather(lev.apply(global_from_L(lev, um), 1.0, 0.5), lev.node)) < 1e-12


def test_gs_matches_oracle_qqt():
    dev()
    mesh, ctx, lev = _setup((5, 3, 4), 4, dirichlet=("y0", "z1"))
    v = np.random.default_rng(0).standard_normal(mesh["x"].size)
    got = H(ctx.gs(T(v)))
    ref = O.qqt(v, lev.node, lev.n_G)
    assert relmax(got, ref) < 1e-15
    got = H(ctx.gs(T(v), mask=True))
    refm = np.where(lev.dir_g[lev.node], 0.0, ref)
    assert relmax(got, refm) < 1e-15
    ones = H(ctx.gs(T(np.ones(mesh["x"].size))))
    np.testing.assert_array_equal(ones, lev.maps["mult"])


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("bf16g", 2e-2)])
def test_ax_low_precision(prec, tol):
    dev()
    mesh, ctx, lev = _setup((4, 3, 3), 7)
    u = si.uniform_field(mesh, 0)
    w = H(ctx.level_ax(0, T(u, torch.float32), h1=1.0, h2=0.5, prec=prec, assemble=False))
    ref = O.ax_local(u, lev.G, lev.B, lev.D, 1.0, 0.5).ravel()
    assert relmax(w, ref) < tol


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("bf16g", 2e-2)])
def test_ax_low_precision_on_an_offset_view(prec, tol):
    """A caller's FP32 vector that does not start on a 16-byte boundary (a view at offset 1
    of a larger tensor) cannot be staged by the bulk copy; the operator then reads it with
    plain loads and gives the same result."""
    dev()
    mesh, ctx, lev = _setup((4, 3, 3), 7)
    u = si.uniform_field(mesh, 0)
    n = u.size
    big = torch.zeros(n + 4, dtype=torch.float32, device=dev())
    big[1:n + 1] = T(u, torch.float32)
    uv = big[1:n + 1]
    assert uv.data_ptr() % 16 == 4
    w = H(ctx.level_ax(0, uv, h1=1.0, h2=0.5, prec=prec, assemble=False))
    ref = O.ax_local(u, lev.G, lev.B, lev.D, 1.0, 0.5).ravel()
    assert relmax(w, ref) < tol
    wa = H(ctx.level_ax(0, T(u, torch.float32), h1=1.0, h2=0.5, prec=prec, assemble=False))
    assert relmax(w, wa) < 1e-6


def test_level_ax_on_coarse_levels():
    dev()
    mesh = si.box_mesh((3, 3, 2), 7, warp=0.1, perm_seed=1, dirichlet=("x0",))
    ctx = ctx_for(mesh)
    levels = O.build_levels(mesh, [7, 3, 1])
    for l in (1, 2):
        Lo = levels[l]
        u = np.random.default_rng(l).standard_normal(Lo.x.size)
        w = H(ctx.level_ax(l, T(u), h1=1.0, h2=0.0, assemble=False))
        ref = O.ax_local(u.reshape(Lo.x.shape), Lo.G, Lo.B, Lo.D).ravel()
        assert relmax(w, ref) < 1e-12


def test_ax_full_size_sampled():
    """The 32^3, N=7 warped Helmholtz workload: local Ax on sampled elements and the
    assembled result at their nodes, against the oracle evaluated on the sample's
    element neighbourhood only."""
    dev()
    mesh = si.box_mesh(32, 7, warp=0.1, perm_seed=0)
    ctx = ctx_for(mesh, prec_copies=0, mg_orders=[7])
    u = si.uniform_field(mesh, 0)
    ut = T(u)
    wl = H(ctx.ax(ut, h1=1.0, h2=0.5, assemble=False)).reshape(mesh["E"], -1)
    wa = H(ctx.ax(ut, h1=1.0, h2=0.5, assemble=True)).reshape(mesh["E"], -1)
    rng = np.random.default_rng(0)
    sample = rng.choice(mesh["E"], 24, replace=False)
    # neighbourhood: every element sharing a node with the sample
    gid = mesh["gid"].reshape(mesh["E"], -1)
    sgids = np.unique(gid[sample])
    hood = np.flatnonzero(np.isin(gid, sgids).any(axis=1))
    sub = {k: mesh[k][hood] for k in ("x", "y", "z")}
    G, B, _ = O.geometry(sub["x"], sub["y"], sub["z"], 7)
    D = O.deriv_matrix(7)
    wref = O.ax_local(u[hood], G, B, D, 1.0, 0.5).reshape(hood.size, -1)
    pos = {e: i for i, e in enumerate(hood)}
    idx = [pos[e] for e in sample]
    assert relmax(wl[sample], wref[idx]) < 1e-12
    # assembled: sum the oracle's local results over all copies inside the neighbourhood
    flat_g = gid[hood].ravel()
    sums_arr = np.zeros(flat_g.max() + 1)
    np.add.at(sums_arr, flat_g, wref.ravel())
    dm = mesh["dirichlet"].reshape(mesh["E"], -1)
    ref = np.where(dm[sample], 0.0, sums_arr[gid[sample]])
    assert relmax(wa[sample], ref) < 1e-12


# ---- FP64-accurate operator in FP32-pair arithmetic (SEM_AX_PAIRS / SEM_FP64P) ----
# Tolerance: the pair format carries ~48 significant bits (2^-48 vs 2^-53 for FP64),
# so its rounding errors are up to 32x those of the FP64 kernel, which stays below
# 1.5e-13 here; 32 * 1.5e-13 = 4.8e-12 -> PAIRS_TOL = 5e-12.
PAIRS_TOL = 5e-12
@pytest.mark.parametrize("N", range(1, 12))
def test_ax_pairs_all_orders(N):
    dev()
    mesh, ctx, lev = _setup((3, 2, 5), N, seed=N)
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, mesh["x"].shape)
    for h1, h2 in ((1.0, 0.0), (0.8, 0.5)):
        w = H(ctx.ax(T(u), h1=h1, h2=h2, assemble=False, pairs=True))
        ref = O.ax_local(u, lev.G, lev.B, lev.D, h1, h2).ravel()
        err = relmax(w, ref)
        print(f"pairs N={N} h1={h1} h2={h2} relmax={err:.3e}")
        assert err < PAIRS_TOL, (N, err)


@pytest.mark.parametrize("N", [3, 7])
def test_ax_pairs_nodal_h1(N):
    """The FP32-pair kernel with a nodal h1 (split into pairs as it is read) against the oracle."""
    dev()
    mesh, ctx, lev = _setup((3, 2, 5), N, seed=N + 20)
    rng = np.random.default_rng(N)
    u = rng.uniform(-1, 1, mesh["x"].shape)
    h1 = np.exp(0.5 * si.smooth_random_field(mesh, 1))
    w = H(ctx.ax(T(u), h1_L=T(h1), h2=0.5, assemble=False, pairs=True))
    ref = O.ax_local(u, lev.G, lev.B, lev.D, h1, 0.5).ravel()
    assert relmax(w, ref) < PAIRS_TOL


def test_ax_pairs_smooth_field_and_level_api():
    """A smooth input (strong cancellation in D u) through the level API."""
    dev()
    mesh, ctx, lev = _setup((4, 4, 4), 7)
    u = np.sin(np.pi * mesh["x"]) * np.cos(2 * np.pi * mesh["y"]) * np.exp(mesh["z"])
    w = H(ctx.level_ax(0, T(u), h1=1.0, h2=0.5, prec="fp64p", assemble=True))
    wl = O.ax_local(u, lev.G, lev.B, lev.D, 1.0, 0.5)
    ref = O.q_gather(lev.mask(O.q_scatter(wl, lev.node, lev.n_G)), lev.node)
    err = relmax(w, ref)
    print(f"pairs smooth assembled relmax={err:.3e}")
    assert err < PAIRS_TOL


def test_ax_pairs_full_size_sampled():
    dev()
    mesh = si.box_mesh(32, 7, warp=0.1, perm_seed=0)
    ctx = ctx_for(mesh, prec_copies=4, mg_orders=[7])
    u = si.uniform_field(mesh, 0)
    wl = H(ctx.ax(T(u), h1=1.0, h2=0.5, assemble=False, pairs=True)).reshape(mesh["E"], -1)
    sample = np.random.default_rng(1).choice(mesh["E"], 32, replace=False)
    G, B, _ = O.geometry(mesh["x"][sample], mesh["y"][sample], mesh["z"][sample], 7)
    ref = O.ax_local(u[sample], G, B, O.deriv_matrix(7), 1.0, 0.5).reshape(sample.size, -1)
    err = relmax(wl[sample], ref)
    print(f"pairs full-size sample relmax={err:.3e}")
    assert err < PAIRS_TOL
