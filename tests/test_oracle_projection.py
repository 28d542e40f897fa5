"""Pins for the oracle's projection of successive right-hand sides (Section 3.4,
"projection-based initial guesses"; Fischer, CMAME 163, 1998).

Sources of truth: the definition of the projected guess as the A-norm-closest
element of the span of earlier solutions, checked by a brute-force weighted
least-squares problem on the Cholesky factor of the dense assembled matrix;
A-orthonormality of the stored basis against that dense matrix; exactness when
the right-hand side lies in the span of earlier ones; the restart rule; and the
iteration savings on a right-hand side that changes smoothly in time.
"""
import numpy as np

import oracle as O
import sem_inputs as si


def _setup(n_el=2, N=3, warp=0.1, h1=1.0, h2=0.2):
    m = si.box_mesh(n_el, N, warp=warp)
    L = O.level_from_mesh(m)
    A = O.assemble(O.element_matrices(L.G, L.B, L.D, h1, h2), L.node, L.n_G)
    f = L.free
    Aff = A[np.ix_(f, f)]
    return m, L, A, f, Aff


def _dense_solve(Aff, f, b):
    x = np.zeros_like(b)
    x[f] = np.linalg.solve(Aff, b[f])
    return x


def _rhs(L, seed):
    return L.mask(np.random.default_rng(seed).standard_normal(L.n_G))


def test_projected_guess_is_a_norm_best_approximation():
    m, L, A, f, Aff = _setup()
    proj = O.Projection(lambda v: L.apply(v, 1.0, 0.2), 6)
    sols = []
    for s in range(3):
        res = O.solve_projected(L, proj, _rhs(L, s), 1.0, 0.2, tol=1e-13, maxit=500)
        sols.append(res.x)
    b = _rhs(L, 10)
    xbar, r0 = proj.project(b)
    # brute force: min_c || x* - S c ||_A over the span S of the earlier solutions
    xs = _dense_solve(Aff, f, b)
    C = np.linalg.cholesky(Aff)
    S = np.stack([s[f] for s in sols], 1)
    c, *_ = np.linalg.lstsq(C.T @ S, C.T @ xs[f], rcond=None)
    best = np.zeros_like(b)
    best[f] = S @ c
    assert np.max(np.abs(xbar - best)) < 1e-10 * np.max(np.abs(best))
    # the residual comes without an operator application and equals b - A xbar
    assert np.max(np.abs(r0 - (b - A @ xbar) * f)) < 1e-11 * np.max(np.abs(b))
    # and the projection reduces the A-norm error of the zero guess
    err = lambda y: float((xs - y)[f] @ Aff @ (xs - y)[f])
    assert err(xbar) < err(np.zeros_like(b))


def test_basis_is_a_orthonormal_with_stored_products():
    m, L, A, f, Aff = _setup()
    proj = O.Projection(lambda v: L.apply(v, 1.0, 0.2), 8)
    for s in range(5):
        O.solve_projected(L, proj, _rhs(L, s), 1.0, 0.2, tol=1e-10, maxit=500)
    X = np.stack(proj.X, 1)
    AX = np.stack(proj.AX, 1)
    assert X.shape[1] == 5
    assert np.max(np.abs(X.T @ A @ X - np.eye(5))) < 1e-12
    assert np.max(np.abs(AX - (A @ X) * f[:, None])) < 1e-12 * np.max(np.abs(AX))
    # Dirichlet entries stay zero
    assert np.all(X[L.dir_g] == 0.0)


def test_rhs_in_span_of_earlier_ones_needs_no_iterations():
    m, L, A, f, Aff = _setup()
    proj = O.Projection(lambda v: L.apply(v, 1.0, 0.2), 8)
    b1, b2 = _rhs(L, 1), _rhs(L, 2)
    O.solve_projected(L, proj, b1, 1.0, 0.2, tol=1e-13, maxit=500)
    O.solve_projected(L, proj, b2, 1.0, 0.2, tol=1e-13, maxit=500)
    b3 = 2.0 * b1 - 0.5 * b2
    res = O.solve_projected(L, proj, b3, 1.0, 0.2, tol=1e-8, maxit=500)
    assert res.relres0 < 1e-11
    assert res.iters == 0
    xs = _dense_solve(Aff, f, b3)
    assert np.max(np.abs(res.x - xs)) < 1e-10 * np.max(np.abs(xs))
    assert not res.added and len(proj.X) == 2       # nothing new to add
    # a zero right-hand side adds nothing either
    res0 = O.solve_projected(L, proj, np.zeros(L.n_G), 1.0, 0.2, tol=1e-8, maxit=10)
    assert res0.iters == 0 and not res0.added and np.all(res0.x == 0.0)


def test_full_basis_restarts_from_the_last_solution():
    m, L, A, f, Aff = _setup()
    proj = O.Projection(lambda v: L.apply(v, 1.0, 0.2), 2)
    for s in range(2):
        O.solve_projected(L, proj, _rhs(L, s), 1.0, 0.2, tol=1e-10, maxit=500)
    assert len(proj.X) == 2
    res = O.solve_projected(L, proj, _rhs(L, 7), 1.0, 0.2, tol=1e-10, maxit=500)
    assert len(proj.X) == 1
    x = res.x
    xa = x / np.sqrt(float(x @ A @ x))
    assert np.max(np.abs(proj.X[0] - xa)) < 1e-12 * np.max(np.abs(xa))


def test_smoothly_varying_rhs_converges_in_fewer_iterations():
    m, L, A, f, Aff = _setup(n_el=3, N=4, warp=0.1, h1=1.0, h2=0.0)
    proj = O.Projection(lambda v: L.apply(v), 8)
    it_p, it_0 = [], []
    for k in range(8):
        b = L.rhs_from_nodal(si.travelling_field(m, 5, 0.02 * k))
        res = O.solve_projected(L, proj, b, tol=1e-8, maxit=1000)
        plain = O.solve(L, b, tol=1e-8, maxit=1000)
        # the projected solve meets the same tolerance on the true residual
        assert np.linalg.norm((b - A @ res.x) * f) <= 1.0001e-8 * np.linalg.norm(b)
        it_p.append(res.iters)
        it_0.append(plain.iters)
    assert it_p[0] == it_0[0]
    assert sum(it_p[3:]) < 0.5 * sum(it_0[3:]), (it_p, it_0)
