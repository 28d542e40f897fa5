"""Pins for the oracle's 1-D building blocks: GLL rule, D_hat, interpolation.

Each check comes from something the paper or the mathematics fixes, not from
the oracle itself: the closed-form rules in tests/golden, the quadrature
exactness of Section 2.3 (degree <= 2N-1), exact differentiation of P_N
(eq. dh), and the antisymmetry of D_hat on symmetric nodes.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_gll_golden():
    rows = {}
    for line in open(os.path.join(GOLDEN, "gll_closed_forms.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, nodes, wts = (s.strip() for s in line.split("|"))
        ev = lambda s: float(eval(s, {"sqrt": math.sqrt}))
        rows[int(n)] = (np.array([ev(t) for t in nodes.split(";")]), np.array([ev(t) for t in wts.split(";")]))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_gll_closed_forms(N):
    xi_ref, rho_ref = _read_gll_golden()[N]
    xi, rho = O.gll(N)
    np.testing.assert_allclose(xi, xi_ref, atol=1e-15)
    np.testing.assert_allclose(rho, rho_ref, rtol=1e-14)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_quadrature_exactness(N):
    xi, rho = O.gll(N)
    assert abs(rho.sum() - 2.0) < 1e-13
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(rho @ xi ** k - exact) < 1e-13, (N, k)
    # degree 2N is not integrated exactly (Section 2.3: exact only up to 2N-1)
    k = 2 * N
    assert abs(rho @ xi ** k - 2.0 / (k + 1)) > 1e-10


@pytest.mark.parametrize("N", range(2, 16))
def test_gll_nodes_are_roots_of_dP(N):
    xi, _ = O.gll(N)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()(xi[1:-1])
    assert np.max(np.abs(dP)) < 1e-11 * N * N


@pytest.mark.parametrize("N", range(1, 16))
def test_deriv_matrix_exact_on_PN(N):
    xi, _ = O.gll(N)
    D = O.deriv_matrix(N)
    scale = N * N
    for k in range(0, N + 1):
        ref = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        assert np.max(np.abs(D @ xi ** k - ref)) < 1e-12 * scale * max(1, k), (N, k)
    # row sums vanish (derivative of a constant) and centro-antisymmetry
    assert np.max(np.abs(D.sum(1))) < 1e-12 * scale
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-12 * scale)
    # not exact one degree higher
    k = N + 1
    assert np.max(np.abs(D @ xi ** k - k * xi ** (k - 1))) > 1e-6


@pytest.mark.parametrize("N", range(1, 13))
def test_deriv_matrix_matches_lagrange_product(N):
    xi, _ = O.gll(N)
    np.testing.assert_allclose(O.deriv_matrix(N), O.lagrange_deriv_matrix(xi), atol=2e-13 * N * N)


@pytest.mark.parametrize("Nf,Nc", [(7, 3), (3, 1), (5, 2), (11, 5)])
def test_interp_matrix_reproduces_polynomials(Nf, Nc):
    xf, _ = O.gll(Nf)
    xc, _ = O.gll(Nc)
    J = O.interp_matrix(xc, xf)
    np.testing.assert_allclose(J.sum(1), 1.0, atol=1e-14)
    for k in range(Nc + 1):
        np.testing.assert_allclose(J @ xc ** k, xf ** k, atol=1e-13)
    # interpolation at the nodes themselves is the identity
    np.testing.assert_allclose(O.interp_matrix(xc, xc), np.eye(Nc + 1), atol=1e-15)


def test_planted_transposed_D_fails_exactness():
    """A transposed D_hat (the index mix-up eq. dh invites) must fail the exactness pin."""
    N = 5
    xi, _ = O.gll(N)
    Dt = O.deriv_matrix(N).T
    assert np.max(np.abs(Dt @ xi ** 2 - 2 * xi)) > 1e-3


def test_splitmix64_reference_values():
    """SplitMix64 first outputs for seed 0 (published reference sequence of the generator)."""
    z = O.splitmix64(0, np.arange(3))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
