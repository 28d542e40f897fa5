"""Direct pins for the oracle's helper functions (they are also exercised through
the public functions that call them).

Sources of truth: closed forms of the Legendre polynomials and their values at the
end points; exact differentiation and interpolation of polynomials within the
degree the GLL basis holds (Section 2.3); the transpose relations the operator
and the multigrid transfers rely on (eq. Ae and the R = P^T of Section 3.4); the
element lengths of an affine box.
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si


def test_legendre_pair_closed_forms_and_end_values():
    x = np.linspace(-1, 1, 23)
    closed = {0: np.ones_like(x), 1: x, 2: (3 * x**2 - 1) / 2, 3: (5 * x**3 - 3 * x) / 2,
              4: (35 * x**4 - 30 * x**2 + 3) / 8}
    for n in range(1, 5):
        p, pm = O.legendre_pair(n, x)
        np.testing.assert_allclose(p, closed[n], atol=1e-14)
        np.testing.assert_allclose(pm, closed[n - 1], atol=1e-14)
    for n in range(1, 15):
        p1, _ = O.legendre_pair(n, np.array([1.0, -1.0]))
        np.testing.assert_allclose(p1, [1.0, (-1.0) ** n], atol=1e-13)


def test_legendre_pair_orthogonality():
    z, w = np.polynomial.legendre.leggauss(20)
    for m in range(1, 9):
        for n in range(1, 9):
            pm, _ = O.legendre_pair(m, z)
            pn, _ = O.legendre_pair(n, z)
            ref = 2.0 / (2 * n + 1) if m == n else 0.0
            assert abs(np.sum(w * pm * pn) - ref) < 1e-13


def _reference_grid(N, E=2):
    xi, _ = O.gll(N)
    k, j, i = np.meshgrid(xi, xi, xi, indexing="ij")
    return xi, np.broadcast_to(i, (E,) + i.shape), np.broadcast_to(j, (E,) + j.shape), np.broadcast_to(k, (E,) + k.shape)


@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_grad_ref_differentiates_polynomials_exactly(N):
    xi, r, s, t = _reference_grid(N)
    D = O.deriv_matrix(N)
    a, b, c = N, max(N - 1, 0), min(1, N)
    u = r**a * s**b * t**c
    ur, us, ut = O.grad_ref(u, D)
    np.testing.assert_allclose(ur, a * r ** max(a - 1, 0) * s**b * t**c * (a > 0), atol=1e-11)
    np.testing.assert_allclose(us, b * r**a * s ** max(b - 1, 0) * t**c * (b > 0), atol=1e-11)
    np.testing.assert_allclose(ut, c * r**a * s**b * t ** max(c - 1, 0) * (c > 0), atol=1e-11)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_grad_ref_T_is_the_transpose(N):
    rng = np.random.default_rng(N)
    shape = (3, N + 1, N + 1, N + 1)
    u = rng.standard_normal(shape)
    wr, ws, wt = (rng.standard_normal(shape) for _ in range(3))
    D = O.deriv_matrix(N)
    ur, us, ut = O.grad_ref(u, D)
    lhs = np.sum(ur * wr) + np.sum(us * ws) + np.sum(ut * wt)
    rhs = np.sum(u * O.grad_ref_T(wr, ws, wt, D))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("Nc,Nf", [(1, 3), (3, 7), (2, 5)])
def test_interp_local_is_exact_on_coarse_polynomials_and_its_transpose(Nc, Nf):
    xc, _ = O.gll(Nc)
    xf, _ = O.gll(Nf)
    J = O.interp_matrix(xc, xf)
    kc, jc, ic = np.meshgrid(xc, xc, xc, indexing="ij")
    kf, jf, i_f = np.meshgrid(xf, xf, xf, indexing="ij")
    f = lambda x, y, z: x**Nc * y ** (Nc - 1 if Nc > 1 else 1) * z + 0.5 * z**Nc - y   # degree <= Nc per direction
    uc = f(ic, jc, kc)[None]
    np.testing.assert_allclose(O.interp_local(uc, J)[0], f(i_f, jf, kf), atol=1e-12)
    rng = np.random.default_rng(Nf)
    a = rng.standard_normal((2, Nc + 1, Nc + 1, Nc + 1))
    v = rng.standard_normal((2, Nf + 1, Nf + 1, Nf + 1))
    assert abs(np.sum(O.interp_local(a, J) * v) - np.sum(a * O.interp_local_T(v, J))) < 1e-12 * np.abs(v).sum()


def test_element_lengths_of_an_affine_box():
    mesh = si.box_mesh((4, 3, 2), 3, warp=0.0, perm_seed=5, dirichlet=())
    L = O.level_from_mesh(mesh)
    lengths = O.element_lengths(L)
    np.testing.assert_allclose(lengths, np.tile([1 / 4, 1 / 3, 1 / 2], (L.E, 1)), atol=1e-14)
