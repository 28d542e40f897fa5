"""Pins for the oracle's geometry, gather-scatter maps and local operator.

Sources of truth: closed forms on affine boxes (eq. gij, eq. vBu), lattice
counts for box meshes, the Kronecker definition of eq. Ae assembled as
Q^T A_L Q, a brute-force stiffness matrix from independently built Lagrange
basis gradients, and the Neumann-operator properties of the footnote below
eq. dssum (symmetric, PSD, orthogonal to constants).
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
import sem_inputs as si


def _close(a, b, rtol):
    np.testing.assert_allclose(a, np.broadcast_to(b, np.shape(a)), rtol=rtol)


def _mesh(e1, N, warp=0.0, seed=0, **kw):
    return si.box_mesh(e1, N, warp=warp, perm_seed=seed, **kw)


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("N", [1, 2, 5, 7])
def test_affine_geometry_closed_form(N):
    m = _mesh(2, N)
    G, B, J = O.geometry(m["x"], m["y"], m["z"], N)
    h = 0.5
    _, rho = O.gll(N)
    w = O.weights3(rho)[None]
    _close(J, (h / 2) ** 3, 1e-12)
    _close(B, w * (h / 2) ** 3, 1e-12)
    for c in (0, 3, 5):
        _close(G[c], w * (h / 2) ** 3 * (2 / h) ** 2, 1e-12)
    for c in (1, 2, 4):
        assert np.max(np.abs(G[c])) < 1e-13
    assert abs(B.sum() - 1.0) < 1e-13


def test_anisotropic_affine_geometry():
    m = si.box_mesh((1, 2, 4), 3, perm_seed=None)
    G, B, _ = O.geometry(m["x"], m["y"], m["z"], 3)
    _, rho = O.gll(3)
    w = O.weights3(rho)[None]
    hx, hy, hz = 1.0, 0.5, 0.25
    vol = hx * hy * hz / 8
    _close(G[0], w * vol * (2 / hx) ** 2, 1e-12)
    _close(G[3], w * vol * (2 / hy) ** 2, 1e-12)
    _close(G[5], w * vol * (2 / hz) ** 2, 1e-12)


def test_warped_volume_converges_spectrally():
    errs = []
    for N in (3, 5, 7, 9, 11):
        m = _mesh(2, N, warp=0.1)
        _, B, J = O.geometry(m["x"], m["y"], m["z"], N)
        assert J.min() > 0
        errs.append(abs(B.sum() - 1.0))
    assert errs[-1] < 1e-9
    assert all(errs[i + 1] < 0.5 * errs[i] or errs[i + 1] < 1e-12 for i in range(len(errs) - 1))


def test_inverted_element_is_rejected():
    m = _mesh(2, 3)
    x = m["x"].copy()
    x[0] = x[0][:, :, ::-1]          # mirror element 0 in r
    with pytest.raises(ValueError):
        O.geometry(x, m["y"], m["z"], 3)


# ---------------------------------------------------------------- gather-scatter
@pytest.mark.parametrize("e1,N", [(1, 1), (2, 3), (3, 4), (4, 7)])
def test_gs_counts_on_box(e1, N):
    m = _mesh(e1, N)
    maps = O.gs_maps(m["gid"])
    assert maps["n_G"] == (e1 * N + 1) ** 3
    mult = maps["mult"]
    assert abs(np.sum(1.0 / mult) - maps["n_G"]) < 1e-9
    # multiplicity from lattice position: 2 per interior element-boundary plane crossed
    L = m["lattice"].ravel()
    LX = e1 * N + 1
    I, J, K = L % LX, (L // LX) % LX, L // (LX * LX)
    f = lambda a: np.where((a % N == 0) & (a > 0) & (a < e1 * N), 2, 1)
    np.testing.assert_array_equal(mult, f(I) * f(J) * f(K))
    ones = np.ones(m["x"].size)
    np.testing.assert_array_equal(O.qqt(ones, maps["node"], maps["n_G"]), mult)


def test_gs_maps_canonical_and_bruteforce():
    rng = np.random.default_rng(3)
    gid = rng.integers(0, 12, size=200)
    maps = O.gs_maps(gid)
    ids, off, idx = maps["ids"], maps["off"], maps["idx"]
    assert np.all(np.diff(ids) > 0) and ids.min() > 0
    for s in range(ids.size):
        seg = idx[off[s]:off[s + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(gid[seg] == ids[s])
        assert np.all(maps["label"][seg] == seg.min())
    w = rng.standard_normal(200)
    out = O.qqt(w, maps["node"], maps["n_G"])
    for l in range(200):
        ref = w[l] if gid[l] == 0 else w[gid == gid[l]].sum()
        assert abs(out[l] - ref) < 1e-13
    assert maps["n_G"] == ids.size + np.sum(gid == 0)


def test_interior_zero_ids_give_same_qqt():
    a = _mesh(2, 4)
    b = _mesh(2, 4, interior_zero=True)
    ma, mb = O.gs_maps(a["gid"]), O.gs_maps(b["gid"])
    w = np.random.default_rng(0).standard_normal(a["x"].size)
    np.testing.assert_allclose(O.qqt(w, ma["node"], ma["n_G"]), O.qqt(w, mb["node"], mb["n_G"]), rtol=0, atol=0)
    assert ma["n_G"] == mb["n_G"]


# ---------------------------------------------------------------- local operator
@pytest.mark.parametrize("e1,N,warp", [(1, 1, 0.0), (2, 2, 0.1), (2, 3, 0.1), (3, 2, 0.1), (2, 5, 0.1)])
def test_sumfact_equals_kronecker_assembly(e1, N, warp):
    m = _mesh(e1, N, warp=warp)
    L = O.level_from_mesh(m)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(m["x"].shape)
    h1 = 1.0 + 0.5 * rng.random(m["x"].shape)
    for h1v, h2v in ((1.0, 0.0), (0.7, 0.5), (h1, 0.3)):
        w = O.ax_local(u, L.G, L.B, L.D, h1v, h2v)
        Ae = O.element_matrices(L.G, L.B, L.D, h1v, h2v)
        w2 = np.einsum("eab,eb->ea", Ae, u.reshape(L.E, -1)).reshape(u.shape)
        assert np.max(np.abs(w - w2)) <= 1e-13 * np.max(np.abs(w))


def _lagrange_poly_derivs(xi):
    """Cardinal polynomials on xi via a Vandermonde solve (independent of D_hat)."""
    n = xi.size
    V = np.vander(xi, n, increasing=True)
    C = np.linalg.solve(V, np.eye(n))        # column b: monomial coefficients of h_b
    vals = V @ C
    dcoef = C[1:] * np.arange(1, n)[:, None]
    dV = np.vander(xi, n - 1, increasing=True)
    return vals, dV @ dcoef                    # h_b(xi_a), h_b'(xi_a)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_element_stiffness_bruteforce_quadrature(N):
    """A^e_ij = sum_q rho_q J_q grad(phi_i) . grad(phi_j) on an affine anisotropic element."""
    m = si.box_mesh((1, 1, 1), N, perm_seed=None)
    sx, sy, sz = 1.0, 0.5, 2.0
    x, y, z = m["x"] * sx, m["y"] * sy, m["z"] * sz
    L = O.Level(N, 1, x, y, z, m["gid"], m["dirichlet"])
    xi, rho = O.gll(N)
    H, dH = _lagrange_poly_derivs(xi)
    NP = N + 1
    pts = list(itertools.product(range(NP), repeat=3))  # (k, j, i)
    n = NP ** 3
    A = np.zeros((n, n))
    jac = sx * sy * sz / 8
    scale = np.array([2 / sx, 2 / sy, 2 / sz])
    def grad(b, q):
        bk, bj, bi = b
        qk, qj, qi = q
        return scale * np.array([dH[qi, bi] * H[qj, bj] * H[qk, bk],
                                 H[qi, bi] * dH[qj, bj] * H[qk, bk],
                                 H[qi, bi] * H[qj, bj] * dH[qk, bk]])
    flat = lambda p: p[2] + NP * (p[1] + NP * p[0])
    for q in pts:
        wq = rho[q[0]] * rho[q[1]] * rho[q[2]] * jac
        g = {flat(b): grad(b, q) for b in pts}
        for a in range(n):
            for b in range(n):
                A[a, b] += wq * g[a] @ g[b]
    Ae = O.element_matrices(L.G, L.B, L.D)[0]
    np.testing.assert_allclose(Ae, A, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("warp", [0.0, 0.1])
def test_neumann_operator_properties(warp):
    m = _mesh(2, 3, warp=warp)
    L = O.level_from_mesh(m)
    A = O.assemble(O.element_matrices(L.G, L.B, L.D), L.node, L.n_G)
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 * ev.max()
    assert np.max(np.abs(A @ np.ones(L.n_G))) < 1e-12 * np.abs(A).max()
    # with Dirichlet rows removed the operator is SPD
    free = L.free
    Ar = A[np.ix_(free, free)]
    assert np.linalg.eigvalsh(Ar).min() > 0
    # matrix-free masked apply equals the assembled, restricted matrix
    v = np.random.default_rng(2).standard_normal(L.n_G)
    ref = np.zeros(L.n_G)
    ref[free] = Ar @ v[free]
    np.testing.assert_allclose(L.apply(v), ref, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("N", [2, 3, 5])
def test_linear_and_quadratic_energy_on_affine_cube(N):
    m = _mesh(2, N)
    L = O.level_from_mesh(m)
    a = np.array([0.3, -1.2, 0.7])
    # global nodal values via the local coordinates (continuous)
    lin = a[0] * m["x"] + a[1] * m["y"] + a[2] * m["z"]
    w = O.ax_local(lin, L.G, L.B, L.D)
    # energy (grad u, grad u)_N = |a|^2 on the unit cube
    assert abs(np.sum(lin * w) - a @ a) < 1e-12
    # A u = 0 at nodes interior to the domain (integrand degree <= 2N-1: exact)
    wg = O.q_scatter(w, L.node, L.n_G)
    on_bd = np.bincount(L.node, weights=np.ravel(si.box_mesh(2, N, perm_seed=0)["dirichlet"]).astype(float),
                        minlength=L.n_G) > 0
    assert np.max(np.abs(wg[~on_bd])) < 1e-12
    # quadratic u = x^2: (grad u, grad u) = int 4x^2 = 4/3, exact for N >= 2
    q = m["x"] ** 2
    assert abs(np.sum(q * O.ax_local(q, L.G, L.B, L.D)) - 4.0 / 3.0) < 1e-12
    # mass term: 1^T B 1 = volume
    one = np.ones_like(lin)
    assert abs(np.sum(one * O.ax_local(one, L.G, L.B, L.D, 1.0, 1.0)) - 1.0) < 1e-12


def test_planted_wrong_metric_sign_fails_energy_pin():
    """A cross-term sign error in the pointwise G-combine must break the Kronecker pin."""
    m = _mesh(2, 3, warp=0.1)
    L = O.level_from_mesh(m)
    u = np.random.default_rng(0).standard_normal(m["x"].shape)
    Gbad = L.G.copy()
    Gbad[1] = -Gbad[1]
    w_bad = O.ax_local(u, Gbad, L.B, L.D)
    Ae = O.element_matrices(L.G, L.B, L.D)
    w_ref = np.einsum("eab,eb->ea", Ae, u.reshape(L.E, -1)).reshape(u.shape)
    assert np.max(np.abs(w_bad - w_ref)) > 1e-6 * np.max(np.abs(w_ref))


@pytest.mark.parametrize("warp", [0.0, 0.1])
def test_jacobi_diagonal_equals_assembled_diagonal(warp):
    m = _mesh(2, 3, warp=warp)
    L = O.level_from_mesh(m)
    rng = np.random.default_rng(5)
    h1 = 1.0 + rng.random(m["x"].shape)
    for h1v, h2v in ((1.0, 0.0), (h1, 0.4)):
        A = O.assemble(O.element_matrices(L.G, L.B, L.D, h1v, h2v), L.node, L.n_G)
        d = np.where(L.dir_g, 1.0, np.diag(A))
        np.testing.assert_allclose(L.diag(h1v, h2v), d, rtol=1e-13)


def test_paper_op_counts_golden():
    """The work formula used for the roofline is the paper's count (tests/golden/paper_counts.txt)."""
    rows = [l.split("|") for l in open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for name, N, val in rows:
        N, val, name = int(N), int(val), name.strip()
        NP = N + 1
        f = {"ax_ops": 12 * NP ** 4 + 15 * NP ** 3, "ax_refs": 7 * NP ** 3, "grad_ops": 6 * NP ** 4 + 15 * NP ** 3}[name]
        assert f == val
