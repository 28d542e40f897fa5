"""GPU setup products vs the oracle: gather-scatter maps (bit-exact), geometric
factors (FP64 to 1e-13, FP32/BF16 copies to the rounding of the oracle's
values), and the coarse p-multigrid levels (ids bit-exact, coordinates)."""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si
from gpu_common import H, T, bf16_rne, ctx_for, dev, relmax

pytestmark = pytest.mark.gpu


def _assert_maps_equal(got, ref):
    np.testing.assert_array_equal(got["ids"], ref["ids"])
    np.testing.assert_array_equal(got["off"], ref["off"])
    np.testing.assert_array_equal(got["idx"], ref["idx"])
    np.testing.assert_array_equal(got["mult"], ref["mult"])
    np.testing.assert_array_equal(got["node"], ref["node"])
    np.testing.assert_array_equal(got["label"], ref["label"])
    assert got["n_G"] == ref["n_G"]


@pytest.mark.parametrize("shape,N,kw", [
    ((4, 4, 4), 7, {}),                                   # 64 elements, N=7
    ((3, 5, 2), 3, {}),                                   # ragged element counts
    ((2, 2, 2), 4, {"interior_zero": True}),              # gslib 0 = singleton
    ((1, 1, 1), 1, {}),
    ((5, 3, 4), 2, {"dirichlet": ("x0",)}),
])
def test_gs_maps_bit_exact(shape, N, kw):
    dev()
    mesh = si.box_mesh(shape, N, warp=0.1, perm_seed=3, **kw)
    ctx = ctx_for(mesh)
    got = ctx.maps(0)
    ref = O.gs_maps(mesh["gid"])
    _assert_maps_equal(got, ref)
    lev = O.level_from_mesh(mesh)
    np.testing.assert_array_equal(got["dmask"], lev.dir_g[lev.node].astype(np.uint8))


def test_gs_maps_arbitrary_ids():
    """Sparse 64-bit ids with singletons: the sort needs every digit pass."""
    dev()
    rng = np.random.default_rng(9)
    mesh = si.box_mesh((3, 3, 2), 2, perm_seed=1)
    base = rng.integers(1, 2 ** 52, size=mesh["gid"].max() + 1)
    gid = np.where(mesh["gid"] > 0, base[mesh["gid"]], 0)
    gid.ravel()[rng.choice(gid.size, 40, replace=False)] = 0
    m2 = dict(mesh, gid=gid)
    ctx = ctx_for(m2)
    _assert_maps_equal(ctx.maps(0), O.gs_maps(gid))


def test_gs_maps_bit_exact_full_size():
    """The 32^3-element N=7 box (16.8M local points) of the throughput workload."""
    dev()
    mesh = si.box_mesh(32, 7, warp=0.1, perm_seed=0)
    ctx = ctx_for(mesh, prec_copies=0, mg_orders=[7])
    _assert_maps_equal(ctx.maps(0), O.gs_maps(mesh["gid"]))
    assert ctx.levels[0]["nG"] == (32 * 7 + 1) ** 3


@pytest.mark.parametrize("N", range(1, 12))
def test_geometry_fp64(N):
    dev()
    mesh = si.box_mesh((2, 3, 2), N, warp=0.1, perm_seed=5)
    ctx = ctx_for(mesh)
    G = ctx.geom(0)
    Go, Bo, _ = O.geometry(mesh["x"], mesh["y"], mesh["z"], N)
    ref = np.concatenate([Go, Bo[None]]).reshape(7, mesh["E"], -1).transpose(1, 0, 2)
    # norm-wise per component, scaled by the largest diagonal factor (the
    # off-diagonal factors can be rounding-level where the warp is nearly affine)
    scale = np.max(np.abs(ref[:, [0, 3, 5]]))
    for c in range(7):
        sc = scale if c < 6 else np.max(np.abs(ref[:, 6]))
        assert np.max(np.abs(G[:, c] - ref[:, c])) < 1e-13 * sc, (N, c)


def test_geometry_lowp_copies_round_the_fp64_values():
    dev()
    mesh = si.box_mesh((2, 2, 3), 7, warp=0.1, perm_seed=2)
    ctx = ctx_for(mesh)
    G = ctx.geom(0)
    Go, Bo, _ = O.geometry(mesh["x"], mesh["y"], mesh["z"], 7)
    ref = np.concatenate([Go, Bo[None]]).reshape(7, mesh["E"], -1).transpose(1, 0, 2)
    # FP32: round-to-nearest of the FP64 factors
    g32 = ctx.geom_lowp(0, "fp32").view(np.float32)
    np.testing.assert_array_equal(g32, G.astype(np.float32))
    assert relmax(g32.astype(np.float64), ref) < 1e-7
    # BF16: round-to-nearest-even of the FP64 factors, direct from double
    g16 = ctx.geom_lowp(0, "bf16g")
    codes, q = bf16_rne(ref)
    diff = g16 != codes
    # a different code is only allowed where the oracle's value sits within
    # 1e-12 (relative) of a rounding tie, i.e. where last-bit FP64 differences decide
    # or where the value itself is rounding-level (|G| < 1e-13 of the component scale)
    if diff.any():
        ulp = np.abs(q) * 2.0 ** -8
        tie_dist = np.abs(np.abs(ref - q) - 0.5 * ulp)
        scale = np.max(np.abs(ref), axis=(0, 2), keepdims=True) * np.ones_like(ref)
        ok = (tie_dist < 1e-12 * np.abs(ref)) | (np.abs(ref) < 1e-13 * scale)
        assert np.all(ok[diff])
    big = np.abs(ref) >= 1e-13 * np.max(np.abs(ref), axis=(0, 2), keepdims=True)
    assert diff[big].mean() < 1e-6


@pytest.mark.parametrize("Nf,orders", [(7, [7, 3, 1]), (5, [5, 2, 1]), (4, [4, 2, 1])])
def test_coarse_levels_match_oracle(Nf, orders):
    dev()
    mesh = si.box_mesh((3, 2, 4), Nf, warp=0.1, perm_seed=7, dirichlet=("x0", "z1"))
    ctx = ctx_for(mesh, mg_orders=orders)
    levels = O.build_levels(mesh, orders)
    assert len(ctx.levels) == len(orders)
    for l in range(1, len(orders)):
        x, y, z, gid = ctx.coords(l)
        Lo = levels[l]
        np.testing.assert_array_equal(gid, Lo.gid.ravel())
        assert relmax(x, Lo.x.ravel()) < 1e-14
        assert relmax(z, Lo.z.ravel()) < 1e-14
        got = ctx.maps(l)
        _assert_maps_equal(got, Lo.maps)
        np.testing.assert_array_equal(got["dmask"], Lo.dir_g[Lo.node].astype(np.uint8))
        G = ctx.geom(l)
        ref = np.concatenate([Lo.G, Lo.B[None]]).reshape(7, mesh["E"], -1).transpose(1, 0, 2)
        assert relmax(G, ref) < 1e-13


def test_default_schedule_orders():
    dev()
    mesh = si.box_mesh(2, 7, warp=0.0)
    ctx = ctx_for(mesh)
    assert [l["N"] for l in ctx.levels] == [7, 3, 1]
    ctx1 = ctx_for(si.box_mesh(2, 1))
    assert [l["N"] for l in ctx1.levels] == [1]


def test_measured_peaks_are_plausible():
    """sem_measure_peaks: FP64 FMA and FP64 mma.sync near GB300's 1.25 TFLOP/s nominal FP64 rate,
    FP32 FMA tens of TFLOP/s (the arithmetic denominators of the roofline reports)."""
    dev()
    from paper_2104_05829_gb300 import measure_peaks
    p = measure_peaks()
    print(p)
    assert 0.3 < p["fp64_fma"] < 3.0 and 0.3 < p["fp64_mma"] < 3.0
    assert 20.0 < p["fp32_fma"] < 200.0
