"""Pins for the oracle's overlapping Schwarz smoother with fast-diagonalisation
local solves and its Chebyshev acceleration (Section 3.4, CHEBY-ASM).

Sources of truth: the closed-form quadratic 1-D element matrices; the dense
assembled matrix, whose principal submatrix on an interior element's extended
box of a uniform affine mesh the fast-diagonalisation solve must invert
exactly; coordinates of the face-layer nodes on affine meshes; subdomain
counts derived by hand; exactness on a single Dirichlet element; symmetry of
the unweighted Schwarz sum; field-of-values bounds on the eigenvalue estimate.
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si


def _dense(L, h1=1.0, h2=0.0):
    return O.assemble(O.element_matrices(L.G, L.B, L.D, h1, h2), L.node, L.n_G)


def test_fdm_1d_matches_closed_form_quadratic_matrices():
    # quadratic element on [-1, 1]: stiffness (1/2) [[7/3, -8/3, 1/3], ...], GLL mass (1/3, 4/3, 1/3)
    K = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 6.0
    m = np.array([1, 4, 1]) / 3.0
    # three elements, 7 nodes; the extended segment is nodes 1..5 (left mid, self 0..2, right mid)
    A = np.zeros((7, 7))
    B = np.zeros(7)
    for el in range(3):
        A[2 * el:2 * el + 3, 2 * el:2 * el + 3] += K
        B[2 * el:2 * el + 3] += m
    cases = {(O.SCH_NB, O.SCH_NB): [1, 2, 3, 4, 5], (O.SCH_DIR, O.SCH_NEU): [3, 4],
             (O.SCH_NEU, O.SCH_NB): [2, 3, 4, 5], (O.SCH_NB, O.SCH_DIR): [1, 2, 3]}
    slot_of_node = {1: 0, 2: 1, 3: 2, 4: 3, 5: 4}
    for (lt, rt), nodes in cases.items():
        # a side without a neighbour element contributes no stiffness or mass from it
        Ae = np.zeros((7, 7))
        Be = np.zeros(7)
        for el, present in ((0, lt == O.SCH_NB), (1, True), (2, rt == O.SCH_NB)):
            if present:
                Ae[2 * el:2 * el + 3, 2 * el:2 * el + 3] += K
                Be[2 * el:2 * el + 3] += m
        As = Ae[np.ix_(nodes, nodes)]
        Bs = np.diag(Be[nodes])
        S, lam = O.fdm_1d(2, lt, rt)
        slots = [slot_of_node[n] for n in nodes]
        Sp = S[slots][:, : len(nodes)]
        assert np.allclose(Sp.T @ Bs @ Sp, np.eye(len(nodes)), atol=1e-13)
        assert np.allclose(Sp.T @ As @ Sp, np.diag(lam[: len(nodes)]), atol=1e-12)
        assert np.allclose(Sp @ np.diag(1 / lam[: len(nodes)]) @ Sp.T, np.linalg.inv(As), atol=1e-12)
        absent = [s for s in range(5) if s not in slots]
        assert np.all(S[absent] == 0.0)


def _box_nodes(L, e, N):
    """Unique nodes of the (N+3)^3 extended box of element e on a uniform affine box
    mesh, located by coordinates (slot order k, j, i)."""
    xi, _ = O.gll(N)
    X = np.stack([L.x[e], L.y[e], L.z[e]])                 # (3, k, j, i)
    lo = X[:, 0, 0, 0]
    h = X[:, -1, -1, -1] - lo
    ext = np.concatenate([[xi[N - 1] - 2.0], xi, [xi[1] + 2.0]])   # reference coords of slots -1..N+1
    coords = lo[:, None] + (ext[None, :] + 1.0) * h[:, None] / 2.0  # (3, N+3)
    allx = np.stack([L.x.ravel(), L.y.ravel(), L.z.ravel()], 1)
    nodes = np.empty((N + 3,) * 3, dtype=np.int64)
    for k in range(N + 3):
        for j in range(N + 3):
            for i in range(N + 3):
                p = np.array([coords[0, i], coords[1, j], coords[2, k]])
                hit = np.nonzero(np.all(np.abs(allx - p) < 1e-12, 1))[0]
                nodes[k, j, i] = L.node[hit[0]]
    return nodes


def test_fdm_inverts_the_assembled_matrix_on_an_interior_extended_box():
    N = 3
    m = si.box_mesh(3, N, warp=0.0, perm_seed=5, dirichlet=())
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    cen = np.stack([L.x.mean((1, 2, 3)), L.y.mean((1, 2, 3)), L.z.mean((1, 2, 3))], 1)
    e = int(np.argmin(((cen - 0.5) ** 2).sum(1)))
    assert np.all(sch.btype[e] == O.SCH_NB)
    box = _box_nodes(L, e, N).ravel()
    h1, h2 = 1.3, 0.4
    Abox = _dense(L, h1, h2)[np.ix_(box, box)]
    nb = (N + 3) ** 3
    F = np.zeros((nb, nb))
    for q in range(nb):
        u = np.zeros(nb)
        u[q] = 1.0
        F[:, q] = O.fdm_solve(sch, e, u.reshape((N + 3,) * 3), h1, h2).ravel()
    assert np.max(np.abs(F @ Abox - np.eye(nb))) < 1e-11


def test_face_layer_nodes_sit_one_gll_step_inside_the_neighbour():
    N = 4
    m = si.box_mesh((3, 2, 2), N, warp=0.0, perm_seed=7, dirichlet=("x0",))
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    xi, _ = O.gll(N)
    xg = np.zeros((L.n_G, 3))
    xg[L.node] = np.stack([L.x.ravel(), L.y.ravel(), L.z.ravel()], 1)
    NP = N + 1
    node = L.node.reshape(L.E, NP, NP, NP)
    nb = 0
    for e in range(L.E):
        X = np.stack([L.x[e], L.y[e], L.z[e]])
        h = X[:, -1, -1, -1] - X[:, 0, 0, 0]
        for f in range(6):
            d, side = divmod(f, 2)
            if sch.btype[e, f] != O.SCH_NB:
                continue
            nb += 1
            i, j, k = O.face_points(N, f)
            face = xg[node[e][k, j, i]]                       # (a, b, 3)
            lay = xg[sch.layer[e, f]]
            step = np.zeros(3)
            step[d] = (1.0 + xi[1]) * h[d] / 2.0 * (-1.0 if side == 0 else 1.0)
            assert np.allclose(lay - face, step, atol=1e-13)
    assert nb > 0
    # boundary types: x0 faces Dirichlet, every other outer face Neumann
    assert set(np.unique(sch.btype)) == {O.SCH_NB, O.SCH_DIR, O.SCH_NEU}


def test_subdomain_counts_by_hand():
    """Interior element of a 5^3 mesh, N = 5: a node is counted once per element
    copy, plus once per copy and per direction in which the copy sits one node off
    a face (1 or N-1): that is where the neighbour's face layer lies."""
    N = 5
    m = si.box_mesh(5, N, warp=0.0, perm_seed=3, dirichlet=())
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    cen = np.stack([L.x.mean((1, 2, 3)), L.y.mean((1, 2, 3)), L.z.mean((1, 2, 3))], 1)
    e = int(np.argmin(((cen - 0.5) ** 2).sum(1)))
    NP = N + 1
    node = L.node.reshape(L.E, NP, NP, NP)
    expect = {  # (i, j, k): count
        (3, 3, 3): 1,   # element interior, away from every face
        (1, 3, 3): 2,   # own + the r- neighbour's layer
        (1, 1, 3): 3,
        (1, 1, 1): 4,
        (4, 4, 4): 4,   # N-1 is the mirror of 1
        (0, 3, 3): 2,   # face node: two copies, no layers
        (0, 0, 3): 4,   # edge node: four copies
        (0, 0, 0): 8,   # vertex: eight copies
        (1, 0, 3): 4,   # two copies, each one node off an r-face
        (0, 1, 1): 6,   # two copies, each one node off an s-face and a t-face
    }
    for (i, j, k), c in expect.items():
        g = node[e][k, j, i]
        assert sch.W[g] == pytest.approx(1.0 / c), ((i, j, k), 1.0 / sch.W[g])


def test_asm_is_the_exact_inverse_on_one_dirichlet_element():
    m = si.box_mesh(1, 5, warp=0.0)
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    A = _dense(L, 1.0, 0.3)
    f = L.free
    r = L.mask(np.random.default_rng(0).standard_normal(L.n_G))
    z = O.asm_apply(L, sch, r, 1.0, 0.3)
    zx = np.zeros_like(r)
    zx[f] = np.linalg.solve(A[np.ix_(f, f)], r[f])
    assert np.max(np.abs(z - zx)) < 1e-13 * np.max(np.abs(zx))


def test_unweighted_schwarz_sum_is_symmetric_positive():
    m = si.box_mesh(2, 3, warp=0.1, perm_seed=2, dirichlet=("x0", "y1"))
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    f = np.nonzero(L.free)[0]
    S = np.zeros((len(f), len(f)))
    for q, g in enumerate(f):
        r = np.zeros(L.n_G)
        r[g] = 1.0
        z = L.mask(O.schwarz_sum(L, sch, lambda e, box: O.fdm_solve(sch, e, box, 1.0, 0.0), r))
        S[:, q] = z[f]
    assert np.max(np.abs(S - S.T)) < 1e-12 * np.max(np.abs(S))
    assert np.min(np.linalg.eigvalsh(0.5 * (S + S.T))) > 0.0


def test_arnoldi_estimate_within_field_of_values_bounds():
    m = si.box_mesh(2, 4, warp=0.1, perm_seed=1, dirichlet=("x0",))
    L = O.level_from_mesh(m)
    sch = O.schwarz_setup(L)
    op = lambda v: L.apply(v)
    minv = lambda r: O.asm_apply(L, sch, r)
    est = O.arnoldi_lmax(op, minv, O.lanczos_start(L, 1), 10)
    f = np.nonzero(L.free)[0]
    MA = np.zeros((len(f), len(f)))
    for q, g in enumerate(f):
        v = np.zeros(L.n_G)
        v[g] = 1.0
        MA[:, q] = minv(op(v))[f]
    re_max = np.max(np.linalg.eigvals(MA).real)
    sym_max = np.max(np.linalg.eigvalsh(0.5 * (MA + MA.T)))
    assert 0.9 * re_max <= est <= sym_max + 1e-12, (est, re_max, sym_max)


def test_cheby_asm_pmg_beats_cheby_jacobi_and_matches_dense():
    m = si.box_mesh(3, 5, warp=0.1, perm_seed=0, dirichlet=("x0",))
    levels = O.build_levels(m, [5, 2, 1])
    L = levels[0]
    A = _dense(L)
    f = L.free
    b = L.mask(np.random.default_rng(3).standard_normal(L.n_G))
    xs = np.zeros_like(b)
    xs[f] = np.linalg.solve(A[np.ix_(f, f)], b[f])
    its = {}
    for sm in ("jacobi", "asm"):
        mg = O.PMG(levels, params=O.MGParams(smoother=sm))
        res = O.pcg(lambda v: L.apply(v), b, mg, 1e-10, 200, flexible=True)
        assert res.relres <= 1e-10
        assert np.max(np.abs(res.x - xs)) < 1e-7 * np.max(np.abs(xs))
        its[sm] = res.iters
    assert its["asm"] < its["jacobi"], its
