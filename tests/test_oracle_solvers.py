"""Pins for the oracle's solvers, smoother, multigrid transfers and adjoint.

Sources of truth: dense linear algebra on tiny meshes (solves, eigenvalues,
adjoint gradients from the explicit derivative of the assembled matrix),
closed forms (the Chebyshev error polynomial T_k((theta-lambda)/delta)/T_k(sigma),
polynomial reproduction of interpolation), central finite differences, and
the spectral convergence the paper states for smooth solutions (Section 2.3).
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si


def _dense(L, h1=1.0, h2=0.0):
    A = O.assemble(O.element_matrices(L.G, L.B, L.D, h1, h2), L.node, L.n_G)
    f = L.free
    return A, f


def test_pcg_matches_dense_solve():
    m = si.box_mesh(2, 3, warp=0.1)
    L = O.level_from_mesh(m)
    A, f = _dense(L, 1.0, 0.3)
    b = L.mask(np.random.default_rng(0).standard_normal(L.n_G))
    ref = np.zeros(L.n_G)
    ref[f] = np.linalg.solve(A[np.ix_(f, f)], b[f])
    res = O.solve(L, b, 1.0, 0.3, tol=1e-14, maxit=500)
    assert res.relres <= 1e-14
    assert np.max(np.abs(res.x - ref)) < 1e-12 * np.max(np.abs(ref))


def test_flexible_cg_equals_cg_with_fixed_preconditioner():
    m = si.box_mesh(2, 4, warp=0.1)
    L = O.level_from_mesh(m)
    b = L.rhs_from_nodal(si.manufactured(m)[1])
    op = lambda v: L.apply(v)
    dinv = np.where(L.free, 1.0 / L.diag(), 0.0)
    a = O.pcg(op, b, lambda v: dinv * v, 0.0, 25)
    c = O.pcg(op, b, lambda v: dinv * v, 0.0, 25, flexible=True)
    assert np.max(np.abs(a.x - c.x)) < 1e-9 * np.max(np.abs(a.x))


def test_manufactured_solution_converges_spectrally():
    """Dirichlet Poisson with f = 3 pi^2 sin sin sin on a 4^3 box: max error falls geometrically in N."""
    errs = []
    for N in (2, 3, 4, 5, 6, 7, 8):
        m = si.box_mesh(4, N, warp=0.0)
        L = O.level_from_mesh(m)
        uex, f = si.manufactured(m)
        res = O.solve(L, L.rhs_from_nodal(f), tol=1e-12, maxit=2000)
        uL = O.q_gather(res.x, L.node).reshape(uex.shape)
        errs.append(np.max(np.abs(uL - uex)))
    for a, b in zip(errs, errs[1:]):
        assert b < 0.5 * a, errs
    assert errs[-1] < 1e-6


def test_lanczos_estimate_vs_dense_eigenvalue():
    m = si.box_mesh(2, 3, warp=0.1, dirichlet=("x0",))
    L = O.level_from_mesh(m)
    A, f = _dense(L)
    dvec = L.diag()
    Dm = np.diag(1.0 / np.sqrt(dvec[f]))
    lam_true = np.linalg.eigvalsh(Dm @ A[np.ix_(f, f)] @ Dm).max()
    dinv = np.where(L.free, 1.0 / dvec, 0.0)
    lam = O.lanczos_lmax(lambda v: L.apply(v), dinv, O.lanczos_start(L, 1), 10)
    assert lam <= lam_true * (1 + 1e-12)
    assert lam >= 0.9 * lam_true
    # with as many steps as unknowns Lanczos is exact
    lam_full = O.lanczos_lmax(lambda v: L.apply(v), dinv, O.lanczos_start(L, 1), int(f.sum()))
    assert abs(lam_full - lam_true) < 1e-8 * lam_true


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_chebyshev_error_polynomial(degree):
    """Error after the smoother from x0 = 0 is T_k((theta - lam)/delta) / T_k(sigma) times each eigenvector."""
    m = si.box_mesh(2, 2, warp=0.1)
    L = O.level_from_mesh(m)
    A, f = _dense(L)
    Af = A[np.ix_(f, f)]
    d = L.diag()[f]
    # generalized eigenproblem A v = lam D v
    s = 1.0 / np.sqrt(d)
    lam, W = np.linalg.eigh(s[:, None] * Af * s[None, :])
    V = s[:, None] * W
    lmax = lam.max()
    lo, hi = 0.1 * lmax, 1.1 * lmax
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = lambda k, x: np.cos(k * np.arccos(x)) if abs(x) <= 1 else np.cosh(k * np.arccosh(abs(x))) * np.sign(x) ** k
    dinv = np.where(L.free, 1.0 / L.diag(), 0.0)
    for c in (0, lam.size // 2, lam.size - 1):
        v = np.zeros(L.n_G)
        v[f] = V[:, c]
        x = O.cheb_smooth(lambda z: L.apply(z), dinv, L.apply(v), None, lo, hi, degree)
        e = v - x
        expect = T(degree, (theta - lam[c]) / delta) / T(degree, theta / delta)
        np.testing.assert_allclose(e[f], expect * V[:, c], atol=1e-10 * np.abs(V[:, c]).max())


def test_coarse_numbering_matches_direct_box_mesh():
    """The order-Nc level built from an order-Nf box has the node classes of an order-Nc box."""
    for (Nf, Nc) in ((7, 3), (3, 1), (6, 3), (4, 2)):
        mf = si.box_mesh(3, Nf, warp=0.0, perm_seed=4, dirichlet=("x0", "y1"))
        mc = si.box_mesh(3, Nc, warp=0.0, perm_seed=4, dirichlet=("x0", "y1"))
        Lf = O.level_from_mesh(mf)
        Lc = O.coarsen(Lf, Nc)
        ref = O.gs_maps(mc["gid"])
        np.testing.assert_array_equal(Lc.maps["label"], ref["label"])
        assert Lc.n_G == (3 * Nc + 1) ** 3
        np.testing.assert_array_equal(np.ravel(Lc.dirichlet), np.ravel(mc["dirichlet"]))
        np.testing.assert_allclose(Lc.x, mc["x"], atol=1e-14)


def test_transfers_adjoint_and_exact_on_coarse_polynomials():
    m = si.box_mesh(2, 5, warp=0.1, dirichlet=())
    levels = O.build_levels(m, [5, 2, 1])
    Lf, Lc = levels[0], levels[1]
    rng = np.random.default_rng(7)
    x, y = rng.standard_normal(Lc.n_G), rng.standard_normal(Lf.n_G)
    lhs = O.restrict(Lf, Lc, y) @ x
    rhs = y @ O.prolong(Lf, Lc, x)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # P reproduces polynomials of degree <= Nc of the reference coordinates: use
    # an affine mesh where coordinates are linear in r
    ma = si.box_mesh(2, 5, warp=0.0, dirichlet=())
    la = O.build_levels(ma, [5, 2])
    poly = lambda X, Y, Z: 1 + X - 2 * Y * Y + X * Z + 0.5 * Z * Z
    pc = np.zeros(la[1].n_G)
    pc[la[1].node] = poly(la[1].x, la[1].y, la[1].z).ravel()
    pf = O.prolong(la[0], la[1], pc)
    ref = np.zeros(la[0].n_G)
    ref[la[0].node] = poly(la[0].x, la[0].y, la[0].z).ravel()
    np.testing.assert_allclose(pf, ref, atol=1e-13)


def test_vcycle_symmetric_positive_with_exact_coarse_solve():
    m = si.box_mesh(2, 5, warp=0.1, dirichlet=("x0",))
    levels = O.build_levels(m, [5, 2, 1])
    mg = O.PMG(levels, params=O.MGParams(coarse_tol=1e-15, coarse_maxit=1000))
    rng = np.random.default_rng(11)
    L = levels[0]
    r1, r2 = L.mask(rng.standard_normal(L.n_G)), L.mask(rng.standard_normal(L.n_G))
    a, b = mg(r1) @ r2, r1 @ mg(r2)
    assert abs(a - b) < 1e-10 * abs(a)
    assert mg(r1) @ r1 > 0


def test_pmg_fcg_beats_jacobi_and_matches_dense():
    m = si.box_mesh(3, 5, warp=0.1, dirichlet=("x0",))
    levels = O.build_levels(m, [5, 2, 1])
    L = levels[0]
    b = L.mask(O.q_scatter(si.gaussian_assembled_rhs(m, 0) / L.maps["mult"].reshape(m["x"].shape), L.node, L.n_G))
    pm = O.solve(L, b, tol=1e-8, maxit=200, precond="pmg", levels=levels)
    jc = O.solve(L, b, tol=1e-8, maxit=2000)
    assert pm.relres <= 1e-8 and jc.relres <= 1e-8
    assert pm.iters < jc.iters / 3
    A, f = _dense(L)
    ref = np.zeros(L.n_G)
    ref[f] = np.linalg.solve(A[np.ix_(f, f)], b[f])
    cond_bound = 1e-8 * 1e4
    assert np.linalg.norm(pm.x - ref) < cond_bound * np.linalg.norm(ref)


def test_adjoint_gradients_vs_finite_differences():
    m = si.box_mesh(2, 3, warp=0.1)
    L = O.level_from_mesh(m)
    g = si.smooth_random_field(m, seed=1)
    h1 = np.exp(0.5 * g)
    t = si.smooth_random_field(m, seed=2)
    f = si.smooth_random_field(m, seed=3)
    loss, u, lam, dfL, dh1L = O.adjoint_loss_and_grads(L, f, h1, 1.0, t)
    rng = np.random.default_rng(0)
    for name, grad, base in (("h1", dh1L, h1), ("f", dfL, f)):
        v = O.q_gather(rng.standard_normal(L.n_G), L.node).reshape(h1.shape)   # continuous direction
        dd = float(np.sum(grad * v))
        fd = []
        for eps in (1e-3, 1e-4):
            def lossat(s):
                hh, ff = (base + s * v, f) if name == "h1" else (h1, base + s * v)
                return O.adjoint_loss_and_grads(L, ff, hh, 1.0, t)[0]
            fd.append((lossat(eps) - lossat(-eps)) / (2 * eps))
        assert abs(fd[-1] - dd) < 1e-6 * abs(dd), (name, fd, dd)
        if name == "h1":
            # Taylor remainder of the central difference falls like eps^2
            assert abs(fd[0] - dd) > 10 * abs(fd[1] - dd)
        else:
            # the loss is quadratic in f: central differences are exact up to rounding
            assert abs(fd[0] - dd) < 1e-8 * abs(dd)


def test_adjoint_gradient_vs_assembled_derivative():
    """-lam^T (dA/dh1_l) u from explicit element matrices with h1 = indicator of point l."""
    m = si.box_mesh(2, 2, warp=0.1)
    L = O.level_from_mesh(m)
    rng = np.random.default_rng(4)
    u = L.mask(rng.standard_normal(L.n_G))
    lam = L.mask(rng.standard_normal(L.n_G))
    uL = O.q_gather(u, L.node).reshape(m["x"].shape)
    lamL = O.q_gather(lam, L.node).reshape(m["x"].shape)
    g = O.grad_h1_local(L, uL, lamL).ravel()
    for l in rng.choice(uL.size, 12, replace=False):
        ind = np.zeros(uL.size)
        ind[l] = 1.0
        dA = O.assemble(O.element_matrices(L.G, L.B, L.D, ind.reshape(uL.shape), 0.0), L.node, L.n_G)
        assert abs(-(lam @ dA @ u) - g[l]) < 1e-12 * max(1.0, abs(g[l]))


def test_coarsen_field_evaluates_the_fine_interpolant_at_the_coarse_points():
    """coarsen_field evaluates each element's fine interpolant at the coarse GLL points. On an
    affine box a field of degree <= Nf in x, y, z is its own fine interpolant, so the coarse
    values equal the field at the coarse points whatever the coarse order; a field of higher
    degree is not, except at the element vertices, which are GLL points of every order."""
    mesh = si.box_mesh((3, 2, 2), 7, warp=0.0, perm_seed=1)
    levels = O.build_levels(mesh, [7, 3, 1])
    deg5 = lambda L: 1.0 + 0.3 * L.x ** 5 - 0.2 * L.y * L.z ** 2 + 0.1 * L.z
    f3 = O.coarsen_field(levels[0], levels[1], deg5(levels[0]))
    assert np.max(np.abs(f3 - deg5(levels[1]))) < 1e-13
    lin = lambda L: 1.0 + 0.3 * L.x - 0.2 * L.y + 0.1 * L.z
    f1 = O.coarsen_field(levels[1], levels[2], O.coarsen_field(levels[0], levels[1], lin(levels[0])))
    assert np.max(np.abs(f1 - lin(levels[2]))) < 1e-13
    deg9 = lambda L: L.x ** 9 * L.y
    assert np.max(np.abs(O.coarsen_field(levels[0], levels[1], deg9(levels[0])) - deg9(levels[1]))) > 1e-10
    chain = O.coarsen_field(levels[1], levels[2], O.coarsen_field(levels[0], levels[1], deg9(levels[0])))
    assert np.max(np.abs(chain - deg9(levels[2]))) < 1e-13


def test_pmg_with_a_constant_nodal_h1_is_the_scalar_pmg():
    mesh = si.box_mesh((3, 3, 2), 5, warp=0.1, perm_seed=4, dirichlet=("x0",))
    levels = O.build_levels(mesh, [5, 2, 1])
    params = O.MGParams(coarse_tol=0.0, coarse_maxit=8)
    r = levels[0].mask(np.random.default_rng(2).standard_normal(levels[0].n_G))
    a = O.PMG(levels, 0.7, 0.3, params)
    b = O.PMG(levels, np.full(levels[0].x.shape, 0.7), 0.3, params)
    assert np.allclose(a.lmax, b.lmax, rtol=1e-13)
    za, zb = a(r), b(r)
    assert np.max(np.abs(za - zb)) < 1e-12 * np.max(np.abs(za))


def test_pmg_with_nodal_h1_solves_the_variable_coefficient_helmholtz_problem():
    """FCG with the nodal-h1 p-MG and Jacobi-PCG converge to the same solution of
    A(h1, h2) u = b with h1 = exp(0.5 g) (a smooth random field), the multigrid in far fewer
    iterations."""
    mesh = si.box_mesh((3, 3, 3), 5, warp=0.1, perm_seed=0)
    levels = O.build_levels(mesh, [5, 2, 1])
    L0 = levels[0]
    h1 = np.exp(0.5 * si.smooth_random_field(mesh, 1)).reshape(L0.x.shape)
    b = L0.rhs_from_nodal(si.smooth_random_field(mesh, 3).reshape(L0.x.shape))
    jac = O.solve(L0, b, h1, 1.0, tol=1e-12, maxit=5000)
    mg = O.solve(L0, b, h1, 1.0, tol=1e-12, maxit=200, precond="pmg", levels=levels)
    assert jac.relres <= 1e-12 and mg.relres <= 1e-12
    assert mg.iters < jac.iters / 3, (mg.iters, jac.iters)
    assert np.max(np.abs(mg.x - jac.x)) < 1e-9 * np.max(np.abs(jac.x))
