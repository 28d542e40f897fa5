"""Pins for the oracle's dealiased advection operator (Sections 2.1 and 3.3).

Sources of truth: the Gauss rule's exactness; skew-symmetry of the assembled
operator for a divergence-free advecting field tangent to the boundary when
the quadrature integrates every product exactly (and its failure when it does
not: the aliasing the dealiased evaluation removes); a brute-force evaluation
of the weak form with explicitly evaluated Lagrange basis functions and
isoparametric map at many quadrature points; constants advected to zero; and
linear fields under a constant wind, whose weak form is a closed form in the
mass.
"""
import itertools

import numpy as np

import oracle as O
import sem_inputs as si


def _field(L, f):
    return f(L.x, L.y, L.z)


def _wind_tangent(L):
    """c = (x(1-x)(1-2y), -y(1-y)(1-2x), 0): divergence free, c.n = 0 on the unit cube."""
    x, y = L.x, L.y
    return np.stack([x * (1 - x) * (1 - 2 * y), -y * (1 - y) * (1 - 2 * x), np.zeros_like(x)])


def _wind_quartic(L):
    """c = (d psi/dy, -d psi/dx, 0) with psi = x^2 (1-x)^2 y^2 (1-y)^2: divergence free,
    c.n = 0 on the unit cube, degree 4 in each coordinate (held exactly at N >= 4)."""
    x, y = L.x, L.y
    return np.stack([x ** 2 * (1 - x) ** 2 * 2 * y * (1 - y) * (1 - 2 * y),
                     -2 * x * (1 - x) * (1 - 2 * x) * y ** 2 * (1 - y) ** 2, np.zeros_like(x)])


def test_cubature_rule_is_exact_to_degree_2nq_minus_1():
    for N in (2, 3, 5, 7):
        z, w = O.cubature_points(N)
        nq = len(z)
        assert nq == (3 * (N + 1) + 1) // 2
        for k in range(2 * nq):
            exact = (1 - (-1) ** (k + 1)) / (k + 1)
            assert abs(np.sum(w * z ** k) - exact) < 1e-14
        assert abs(np.sum(w * z ** (2 * nq)) - 2 / (2 * nq + 1)) > 1e-10   # degree 2 nq is not exact


def _assembled_matrix(L, cub, cL):
    n = L.n_G
    C = np.zeros((n, n))
    for g in range(n):
        e = np.zeros(n)
        e[g] = 1.0
        C[:, g] = O.advect_assembled(L, cub, cL, e)
    return C


def test_dealiased_operator_is_skew_symmetric_and_the_aliased_one_is_not():
    """Per direction the products phi_i c du/dx reach degree N + 4 + N - 1 = 11 at N = 4:
    exact with the dealiased 8 Gauss points (degree 15), not with N + 1 = 5 (degree 9)."""
    N = 4
    m = si.box_mesh(2, N, warp=0.0, perm_seed=3, dirichlet=())
    L = O.level_from_mesh(m)
    cL = _wind_quartic(L)
    C = _assembled_matrix(L, O.cubature_setup(L), cL)              # nq = 8
    scale = np.max(np.abs(C))
    assert np.max(np.abs(C + C.T)) < 1e-13 * scale
    Ca = _assembled_matrix(L, O.cubature_setup(L, nq=N + 1), cL)   # nq = N+1: aliased
    assert np.max(np.abs(Ca + Ca.T)) > 1e-4 * scale


def _lagrange(xi, x):
    """phi_b(x) for cardinal polynomials on nodes xi, at points x: (len(x), len(xi))."""
    out = np.ones((len(x), len(xi)))
    for b in range(len(xi)):
        for c in range(len(xi)):
            if c != b:
                out[:, b] *= (x - xi[c]) / (xi[b] - xi[c])
    return out


def _lagrange_d(xi, x):
    """phi_b'(x) by the product rule."""
    out = np.zeros((len(x), len(xi)))
    for b in range(len(xi)):
        for c in range(len(xi)):
            if c == b:
                continue
            term = np.ones(len(x)) / (xi[b] - xi[c])
            for e in range(len(xi)):
                if e not in (b, c):
                    term = term * (x - xi[e]) / (xi[b] - xi[e])
            out[:, b] += term
    return out


def test_matches_brute_force_weak_form_with_explicit_basis():
    """Element by element: sum over many Gauss points of w J phi_i (c . grad u), with the
    basis, the map and its Jacobian evaluated point by point from the Lagrange formulae."""
    N, nq = 3, 9
    m = si.box_mesh(2, N, warp=0.1, perm_seed=2, dirichlet=())
    L = O.level_from_mesh(m)
    rng = np.random.default_rng(4)
    cL = rng.standard_normal((3,) + L.x.shape)
    uL = rng.standard_normal(L.x.shape)
    got = O.advect_local(L, O.cubature_setup(L, nq=nq), cL, uL)
    z, w = np.polynomial.legendre.leggauss(nq)
    P, dP = _lagrange(L.xi, z), _lagrange_d(L.xi, z)
    for e in range(L.E):
        X = np.stack([L.x[e], L.y[e], L.z[e]])                 # (3, k, j, i)
        ref = np.zeros(L.x.shape[1:])
        for a, b, c in itertools.product(range(nq), repeat=3):  # point (z_a, z_b, z_c) in (r, s, t)
            phi = np.einsum("k,j,i->kji", P[c], P[b], P[a])
            dphi = [np.einsum("k,j,i->kji", P[c], P[b], dP[a]),
                    np.einsum("k,j,i->kji", P[c], dP[b], P[a]),
                    np.einsum("k,j,i->kji", dP[c], P[b], P[a])]
            Jm = np.array([[np.sum(X[mm] * dphi[q]) for q in range(3)] for mm in range(3)])
            rinv = np.linalg.inv(Jm)                          # dr_q / dx_m
            cvec = np.array([np.sum(cL[mm, e] * phi) for mm in range(3)])
            du_dr = np.array([np.sum(uL[e] * dphi[q]) for q in range(3)])
            conv = cvec @ (rinv.T @ du_dr)                     # c . grad u
            ref += w[a] * w[b] * w[c] * np.linalg.det(Jm) * conv * phi
        assert np.max(np.abs(got[e] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_constant_is_advected_to_zero_and_linear_field_gives_the_mass():
    m = si.box_mesh((2, 2, 1), 4, warp=0.0, perm_seed=1, dirichlet=())
    L = O.level_from_mesh(m)
    cub = O.cubature_setup(L)
    a = np.array([0.3, -1.2, 0.7])
    bvec = np.array([2.0, 0.5, -1.0])
    cL = np.stack([np.full_like(L.x, a[0]), np.full_like(L.x, a[1]), np.full_like(L.x, a[2])])
    w0 = O.advect_local(L, cub, cL, np.full_like(L.x, 3.0))
    assert np.max(np.abs(w0)) < 1e-14
    uL = bvec[0] * L.x + bvec[1] * L.y + bvec[2] * L.z
    w = O.q_scatter(O.advect_local(L, cub, cL, uL), L.node, L.n_G)
    # c . grad u = a . b everywhere, and int phi_i = sum of B over the copies (exact for degree N)
    assert np.max(np.abs(w - (a @ bvec) * L.mass())) < 1e-13 * np.max(np.abs(w))


def test_warped_tangent_wind_integrates_to_zero():
    """(1, C u) = int c . grad u = (boundary flux of u c) - int u div c = 0 for a divergence-free
    wind tangent to the boundary, up to the quadrature error of the warped map."""
    m = si.box_mesh(3, 5, warp=0.1, perm_seed=4, dirichlet=())
    L = O.level_from_mesh(m)
    cub = O.cubature_setup(L)
    cL = _wind_tangent(L)
    uL = np.sin(np.pi * L.x) * np.cos(2 * L.y) + L.z ** 2
    w = O.advect_local(L, cub, cL, uL)
    ref = O.advect_local(L, cub, cL, np.abs(uL))
    assert abs(w.sum()) < 1e-6 * np.abs(ref).sum()


def test_characteristics_translate_a_linear_field_exactly():
    """Constant wind a, linear w0 = b . x: c . grad w = a . b everywhere, M^-1 C w = a . b exactly
    (the GLL mass integrates phi_i exactly), so w(t) = w0 - (a . b) t at every node, and RK4 is
    exact for an integrand constant in time."""
    m = si.box_mesh((2, 2, 2), 4, warp=0.0, perm_seed=3, dirichlet=())
    L = O.level_from_mesh(m)
    cub = O.cubature_setup(L)
    a = np.array([0.4, -0.3, 0.8])
    bvec = np.array([1.5, 2.0, -0.5])
    cL = np.stack([np.full_like(L.x, q) for q in a])
    xg = np.zeros((L.n_G, 3))
    xg[L.node] = np.stack([L.x.ravel(), L.y.ravel(), L.z.ravel()], 1)
    w0 = xg @ bvec
    w = O.char_advance(L, cub, cL, None, [w0], 0.0, 0.3, 3)[0]
    assert np.max(np.abs(w - (w0 - (a @ bvec) * 0.3))) < 1e-12 * np.max(np.abs(w0))


def test_characteristics_rk4_converges_at_fourth_order_and_conserves_the_mass_norm():
    """Divergence-free wind tangent to the walls, held exactly (N = 4): the dealiased C is skew,
    so w^T M w is conserved by the semi-discrete system; RK4 errors against a fine-step
    reference fall by about 2^4 per halving of the step."""
    m = si.box_mesh(2, 4, warp=0.0, perm_seed=5, dirichlet=())
    L = O.level_from_mesh(m)
    cub = O.cubature_setup(L)
    cL = 3.0 * _wind_quartic(L)
    xg = np.zeros((L.n_G, 3))
    xg[L.node] = np.stack([L.x.ravel(), L.y.ravel(), L.z.ravel()], 1)
    w0 = np.sin(2 * xg[:, 0]) * np.cos(3 * xg[:, 1]) + xg[:, 2]
    M = L.mass()
    ref = O.char_advance(L, cub, cL, None, [w0], 0.0, 0.5, 64)[0]
    errs = [np.max(np.abs(O.char_advance(L, cub, cL, None, [w0], 0.0, 0.5, n)[0] - ref)) for n in (4, 8, 16)]
    for e1, e2 in zip(errs, errs[1:]):
        assert 12.0 < e1 / e2 < 20.0, errs
    e0 = w0 @ (M * w0)
    assert abs(ref @ (M * ref) - e0) < 1e-9 * e0
