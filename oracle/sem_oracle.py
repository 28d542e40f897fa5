"""Plain FP64 CPU oracle for the SEM elliptic path.

TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import this module. The CUDA library never
calls it, and it shares no code with the library: the only shared module is
the seeded input generator ``sem_inputs`` (meshes and fields, no method
arithmetic).

Everything here is written for readability against the paper
(Fischer et al., "NekRS, a GPU-accelerated spectral element Navier-Stokes
solver"), Section 2.3 ("Spectral Element Discretization"), Section 3.2
("Parallel Communication") and Section 3.4 ("Poisson Solve Preconditioning"), in float64:

* GLL rule and derivative matrix (eq. xijk, eq. dh),
* geometric factors (eq. grad, eq. vBu, eq. gij),
* local operator A^e = D^T G D (+ h2 B) by sum factorisation (eq. Ae) and, for
  tiny meshes, as explicit Kronecker-product element matrices assembled into
  Q^T A_L Q (the "assembled stiffness matrix" below eq. dssum),
* the gather-scatter QQ^T on global ids (the gs_op(+) interface, Section 3.2),
* Jacobi-PCG, flexible PCG, Chebyshev-Jacobi smoothing and the p-multigrid
  V-cycle with orders N, N/2 .. 1 (Section 3.4),
* projection of successive right-hand sides onto earlier solutions (Section 3.4),
* the dealiased advection operator on Gauss points (Sections 2.1 and 3.3),
* the adjoint gradient of a mass-weighted loss with respect to nodal h1.

Global (unique-node) vectors are used for every solver here; the library works
on replicated L-vectors. Arrays of local data are shaped (E, N+1, N+1, N+1)
with axes (e, k, j, i): point (i, j, k) of element e sits at flat index
i + (N+1)(j + (N+1)(k + (N+1)e)), eq. uijk.

Parity pins live in tests/test_oracle_*.py. Every function below is pinned
there; none is "parity unpinned".
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# 1-D building blocks: GLL rule, derivative and interpolation matrices
# ----------------------------------------------------------------------------


def legendre_pair(N: int, x):
    """Return (P_N(x), P_{N-1}(x)) by the recurrence (k+1)P_{k+1} = (2k+1)xP_k - kP_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    return p, p_prev


def gll(N: int):
    """Gauss-Lobatto-Legendre nodes xi_0 < ... < xi_N and weights rho_j (Section 2.3).

    The nodes are -1, +1 and the N-1 roots of P_N'. The roots are found by Newton's
    method on P_N' started from the Chebyshev-Gauss-Lobatto points, with
    P_N'(x) = N (x P_N - P_{N-1}) / (x^2 - 1) and, from Legendre's equation,
    P_N''(x) = (2 x P_N' - N (N+1) P_N) / (1 - x^2).
    The weights are rho_j = 2 / (N (N+1) P_N(xi_j)^2).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    xi = np.empty(N + 1)
    xi[0], xi[N] = -1.0, 1.0
    if N >= 2:
        x = -np.cos(np.pi * np.arange(1, N) / N)
        for _ in range(100):
            P, Pm1 = legendre_pair(N, x)
            dP = N * (x * P - Pm1) / (x * x - 1.0)
            d2P = (2.0 * x * dP - N * (N + 1) * P) / (1.0 - x * x)
            step = dP / d2P
            x = x - step
            if np.max(np.abs(step)) < 1e-16:
                break
        xi[1:N] = x
    xi = 0.5 * (xi - xi[::-1])
    P, _ = legendre_pair(N, xi)
    rho = 2.0 / (N * (N + 1) * P * P)
    return xi, rho


def deriv_matrix(N: int) -> np.ndarray:
    """D_hat[a, b] = h_b'(xi_a), eq. dh (first index: the point where the derivative is taken).

    Closed form for GLL cardinal polynomials:
    D[a, b] = P_N(xi_a) / (P_N(xi_b) (xi_a - xi_b)) for a != b,
    D[0, 0] = -N(N+1)/4, D[N, N] = +N(N+1)/4, other diagonal entries 0.
    """
    xi, _ = gll(N)
    P, _ = legendre_pair(N, xi)
    D = np.zeros((N + 1, N + 1))
    for a in range(N + 1):
        for b in range(N + 1):
            if a != b:
                D[a, b] = P[a] / (P[b] * (xi[a] - xi[b]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def lagrange_deriv_matrix(xi) -> np.ndarray:
    """h_b'(xi_a) by differentiating the cardinal product h_b(x) = prod_{c!=b} (x-xi_c)/(xi_b-xi_c).

    Independent cross-check of deriv_matrix (no Legendre closed form used).
    """
    xi = np.asarray(xi, dtype=np.float64)
    n = xi.size
    D = np.zeros((n, n))
    for b in range(n):
        denom = np.prod([xi[b] - xi[c] for c in range(n) if c != b])
        for a in range(n):
            if a == b:
                D[a, b] = sum(1.0 / (xi[b] - xi[c]) for c in range(n) if c != b)
            else:
                D[a, b] = np.prod([xi[a] - xi[c] for c in range(n) if c not in (a, b)]) / denom
    return D


def interp_matrix(xi_from, x_to) -> np.ndarray:
    """J[a, b] = h_b(x_a): the cardinal polynomials on nodes xi_from evaluated at points x_to."""
    xi_from = np.asarray(xi_from, dtype=np.float64)
    x_to = np.asarray(x_to, dtype=np.float64)
    n = xi_from.size
    J = np.ones((x_to.size, n))
    for b in range(n):
        for c in range(n):
            if c != b:
                J[:, b] *= (x_to - xi_from[c]) / (xi_from[b] - xi_from[c])
    return J


# ----------------------------------------------------------------------------
# Tensor-product derivatives and geometry (eq. gradr-gradt, grad, vBu, gij)
# ----------------------------------------------------------------------------


def grad_ref(u: np.ndarray, D: np.ndarray):
    """(u_r, u_s, u_t) = (D1 u, D2 u, D3 u) with D1 = I x I x D_hat acting on i, D2 on j, D3 on k."""
    ur = np.einsum("ab,ekjb->ekja", D, u)
    us = np.einsum("ab,ekbi->ekai", D, u)
    ut = np.einsum("ab,ebji->eaji", D, u)
    return ur, us, ut


def grad_ref_T(wr: np.ndarray, ws: np.ndarray, wt: np.ndarray, D: np.ndarray) -> np.ndarray:
    """D1^T wr + D2^T ws + D3^T wt (the transposed contractions of eq. Ae)."""
    return (np.einsum("ba,ekjb->ekja", D, wr)
            + np.einsum("ba,ekbi->ekai", D, ws)
            + np.einsum("ba,ebji->eaji", D, wt))


def weights3(rho: np.ndarray) -> np.ndarray:
    """rho_ijk = rho_i rho_j rho_k laid out as [k, j, i]."""
    return rho[:, None, None] * rho[None, :, None] * rho[None, None, :]


def geometry(x, y, z, N: int):
    """Geometric factors of Section 2.3.

    Returns (G, B, Jac) where G has shape (6, E, NP, NP, NP) holding
    G11, G12, G13, G22, G23, G33 of eq. gij, B = rho_ijk J_ijk (eq. vBu) and Jac
    the Jacobian determinant. The metric matrix dx_p/dr_q = D_q x_p is inverted
    pointwise by cofactors (eq. grad) to give dr_q/dx_p.

    The coordinates are differentiated relative to each element's first node:
    D_q (x_p - c) = D_q x_p because D_hat differentiates constants to zero
    (eq. dh). In floating point the rows of D_hat sum to ~1e-15 rather than 0,
    and on small elements far from the origin that rounding times the absolute
    coordinate would dominate the metrics; the shift removes it.
    """
    xi, rho = gll(N)
    D = deriv_matrix(N)
    d = [grad_ref(c - c[:, :1, :1, :1], D) for c in (x, y, z)]  # d[p][q] = dx_p / dr_q
    a, b, c = d[0]
    dd, e, f = d[1]
    g, h, i = d[2]
    jac = a * (e * i - f * h) - b * (dd * i - f * g) + c * (dd * h - e * g)
    if np.any(jac <= 0):
        raise ValueError("non-positive Jacobian")
    inv = [[(e * i - f * h), (c * h - b * i), (b * f - c * e)],
           [(f * g - dd * i), (a * i - c * g), (c * dd - a * f)],
           [(dd * h - e * g), (b * g - a * h), (a * e - b * dd)]]
    rx = [[inv[q][p] / jac for p in range(3)] for q in range(3)]  # rx[q][p] = dr_q/dx_p
    B = weights3(rho)[None] * jac
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    G = np.stack([(rx[m][0] * rx[n][0] + rx[m][1] * rx[n][1] + rx[m][2] * rx[n][2]) * B for m, n in pairs])
    return G, B, jac


def _g_full(G):
    """3x3 symmetric view [[G11,G12,G13],[G12,G22,G23],[G13,G23,G33]]."""
    return [[G[0], G[1], G[2]], [G[1], G[3], G[4]], [G[2], G[4], G[5]]]


def ax_local(u, G, B, D, h1=1.0, h2=0.0):
    """w_L = A_L u_L with A^e = D^T (h1 G) D + h2 B (eq. Ae; h2 B is the Helmholtz mass term of eq. ns_wrt2).

    h1 and h2 may be scalars or arrays shaped like u (nodal coefficients).
    """
    ur, us, ut = grad_ref(u, D)
    Gf = _g_full(G)
    grads = (ur, us, ut)
    wq = [h1 * (Gf[m][0] * grads[0] + Gf[m][1] * grads[1] + Gf[m][2] * grads[2]) for m in range(3)]
    w = grad_ref_T(wq[0], wq[1], wq[2], D)
    return w + h2 * B * u


# ----------------------------------------------------------------------------
# Global numbering, Q, Q^T and QQ^T (eq. dssum; gs_setup / gs_op semantics)
# ----------------------------------------------------------------------------


def gs_maps(gid) -> dict:
    """Canonical gather-scatter maps from per-point global ids (0 = singleton).

    ids   : distinct nonzero ids, ascending
    off   : CSR offsets of each id's local points in ``idx``
    idx   : local indices sorted by (id, local index)
    mult  : multiplicity of each local point's node (1 for a singleton)
    node  : unique-node number of each local point; nonzero ids take 0.. in
            ascending id order, singletons follow in local-index order
    label : smallest local index sharing the point's node
    n_G   : number of unique nodes
    """
    g = np.asarray(gid, dtype=np.int64).ravel()
    if np.any(g < 0):
        raise ValueError("negative global id")
    nL = g.size
    loc = np.arange(nL, dtype=np.int64)
    nz = g != 0
    lnz, gnz = loc[nz], g[nz]
    order = np.lexsort((lnz, gnz))
    idx, gs = lnz[order], gnz[order]
    start = np.ones(gs.size, dtype=bool)
    start[1:] = gs[1:] != gs[:-1]
    first = np.flatnonzero(start)
    ids = gs[first]
    off = np.append(first, gs.size).astype(np.int64)
    m_nz = np.diff(off)
    mult = np.ones(nL, dtype=np.int64)
    mult[idx] = np.repeat(m_nz, m_nz)
    node = np.empty(nL, dtype=np.int64)
    node[idx] = np.repeat(np.arange(ids.size), m_nz)
    zero = loc[~nz]
    node[zero] = ids.size + np.arange(zero.size)
    label = np.empty(nL, dtype=np.int64)
    label[idx] = np.repeat(idx[first], m_nz)
    label[zero] = zero
    return {"ids": ids, "off": off, "idx": idx, "mult": mult, "node": node,
            "label": label, "n_G": int(ids.size + zero.size)}


def q_gather(xg, node):
    """u_L = Q u (copy each unique value to its local points)."""
    return xg[node]


def q_scatter(wL, node, n_G):
    """w = Q^T w_L (sum the local copies of each unique node)."""
    return np.bincount(node, weights=np.ravel(wL), minlength=n_G)


def qqt(wL, node, n_G):
    """w_L <- QQ^T w_L (gs_op with +), eq. dssum."""
    return q_scatter(wL, node, n_G)[node].reshape(np.shape(wL))


# ----------------------------------------------------------------------------
# Brute-force assembled operator for tiny meshes
# ----------------------------------------------------------------------------


def element_matrices(G, B, D, h1=1.0, h2=0.0):
    """Dense A^e = sum_{m,m'} D_m^T (h1 G_mm') D_m' + h2 B from explicit Kronecker matrices (eq. Ae).

    D1 = I x I x D_hat, D2 = I x D_hat x I, D3 = D_hat x I x I with the
    i-fastest flat index i + NP j + NP^2 k.
    """
    NP = D.shape[0]
    I = np.eye(NP)
    Dm = [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]
    E = G.shape[1]
    n = NP ** 3
    Gf = _g_full(G)
    h1a = np.broadcast_to(np.asarray(h1, dtype=np.float64), G.shape[1:]).reshape(E, n)
    h2a = np.broadcast_to(np.asarray(h2, dtype=np.float64), G.shape[1:]).reshape(E, n)
    A = np.zeros((E, n, n))
    for e in range(E):
        for m in range(3):
            for mp in range(3):
                gdiag = h1a[e] * Gf[m][mp][e].ravel()
                A[e] += Dm[m].T @ (gdiag[:, None] * Dm[mp])
        A[e] += np.diag(h2a[e] * B[e].ravel())
    return A


def assemble(Ae, node, n_G):
    """Assembled (Neumann) matrix Q^T A_L Q as a dense array (tiny meshes only)."""
    E, n, _ = Ae.shape
    nd = np.asarray(node).reshape(E, n)
    A = np.zeros((n_G, n_G))
    for e in range(E):
        A[np.ix_(nd[e], nd[e])] += Ae[e]
    return A


# ----------------------------------------------------------------------------
# A discretisation level: geometry, numbering, Dirichlet mask, Jacobi diagonal
# ----------------------------------------------------------------------------


@dataclass
class Level:
    """One order-N discretisation of the mesh with its operator data."""
    N: int
    E: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    gid: np.ndarray
    dirichlet: np.ndarray
    xi: np.ndarray = field(init=False)
    rho: np.ndarray = field(init=False)
    D: np.ndarray = field(init=False)
    G: np.ndarray = field(init=False)
    B: np.ndarray = field(init=False)
    maps: dict = field(init=False)

    def __post_init__(self):
        self.xi, self.rho = gll(self.N)
        self.D = deriv_matrix(self.N)
        self.G, self.B, _ = geometry(self.x, self.y, self.z, self.N)
        self.maps = gs_maps(self.gid)
        self.node = self.maps["node"]
        self.n_G = self.maps["n_G"]
        dflag = np.bincount(self.node, weights=np.ravel(self.dirichlet).astype(np.float64), minlength=self.n_G)
        self.dir_g = dflag > 0          # Dirichlet unique nodes (rows removed by R)
        self.free = ~self.dir_g

    # -- operators on global vectors -------------------------------------------------
    def mask(self, v):
        """R^T R: zero the Dirichlet entries (the footnote below eq. dssum)."""
        return np.where(self.dir_g, 0.0, v)

    def apply(self, xg, h1=1.0, h2=0.0):
        """Masked assembled operator R Q^T A_L Q R^T on a global vector."""
        uL = q_gather(self.mask(xg), self.node).reshape(self.x.shape)
        wL = ax_local(uL, self.G, self.B, self.D, h1, h2)
        return self.mask(q_scatter(wL, self.node, self.n_G))

    def rhs_from_nodal(self, fL):
        """b = R Q^T B_L f_L, the GLL inner products b_i = (phi_i, f)_N (eq. qN-vBu)."""
        return self.mask(q_scatter(self.B * fL, self.node, self.n_G))

    def mass(self):
        """Assembled diagonal mass M = Q^T B_L Q (as a global vector)."""
        return q_scatter(self.B, self.node, self.n_G)

    def diag(self, h1=1.0, h2=0.0):
        """Exact diagonal of R Q^T A_L Q R^T (Dirichlet entries set to 1).

        Per element, diag(D_m^T G D_m) at point p sums D_hat[l, p_m]^2 G_mm over
        the line through p; the cross terms m != m' meet the diagonal only at
        q = p and give 2 D_hat[p_m, p_m] D_hat[p_m', p_m'] G_mm'(p).
        """
        D = self.D
        NP = D.shape[0]
        Gf = _g_full(self.G)
        h1a = np.broadcast_to(np.asarray(h1, dtype=np.float64), self.x.shape)
        h2a = np.broadcast_to(np.asarray(h2, dtype=np.float64), self.x.shape)
        D2 = D * D
        d = np.einsum("li,ekjl->ekji", D2, h1a * Gf[0][0])
        d += np.einsum("lj,ekli->ekji", D2, h1a * Gf[1][1])
        d += np.einsum("lk,elji->ekji", D2, h1a * Gf[2][2])
        dd = np.diag(D)
        di = dd[None, None, None, :] * np.ones((1, NP, NP, 1))
        dj = dd[None, None, :, None] * np.ones((1, NP, 1, NP))
        dk = dd[None, :, None, None] * np.ones((1, 1, NP, NP))
        d += 2.0 * h1a * (di * dj * Gf[0][1] + di * dk * Gf[0][2] + dj * dk * Gf[1][2])
        d += h2a * self.B
        dg = q_scatter(d, self.node, self.n_G)
        return np.where(self.dir_g, 1.0, dg)


def level_from_mesh(mesh: dict) -> Level:
    return Level(mesh["N"], mesh["E"], mesh["x"], mesh["y"], mesh["z"], mesh["gid"], mesh["dirichlet"])


# ----------------------------------------------------------------------------
# p-multigrid level construction (orders N, N/2, ..., 1; Section 3.4)
# ----------------------------------------------------------------------------


def interp_local(uL, Jm):
    """Tensor-product interpolation J x J x J applied to every element."""
    return np.einsum("ka,jb,ic,eabc->ekji", Jm, Jm, Jm, uL)


def interp_local_T(uL, Jm):
    """Transpose of interp_local."""
    return np.einsum("ak,bj,ci,eabc->ekji", Jm, Jm, Jm, uL)


def coarse_numbering(gid_f, dir_f, Nf: int, Nc: int):
    """Global ids and Dirichlet flags at the order-Nc points of every element.

    The paper builds coarse levels of the same elements at lower order but does
    not say how their points are numbered; this is the reading used here.
    A coarse point is classified by how many of its indices are interior to
    (0, Nc): none -> element vertex, one -> edge, two -> face, three -> element
    interior (a singleton, id 0).
    * vertex: key of the fine vertex id;
    * edge: the edge is named by the smallest nonzero fine id on its interior,
      the position t along it is counted from the endpoint with the smaller
      fine id;
    * face: the face is named by the smallest nonzero fine id on its interior;
      the in-face position (a, b) is taken in the frame whose origin is the
      face corner with the smallest fine id and whose first axis points to the
      origin's neighbour corner with the smaller fine id.
    key = (entity * 3 + type) * 256 + position, type 0/1/2 for vertex/edge/face.
    An entity whose fine interior ids are all 0 is unshared: its points get 0.
    The Dirichlet flag of a vertex is the fine vertex flag; of an edge or face
    point, whether any fine point on the entity's interior is flagged.
    """
    E = gid_f.shape[0]
    NPf, NPc = Nf + 1, Nc + 1
    gf = np.asarray(gid_f, dtype=np.int64).reshape(E, NPf, NPf, NPf)
    df = np.asarray(dir_f).reshape(E, NPf, NPf, NPf).astype(bool)
    gc = np.zeros((E, NPc, NPc, NPc), dtype=np.int64)
    dc = np.zeros((E, NPc, NPc, NPc), dtype=np.uint8)

    def fine_at(arr, ijk):   # ijk in (i, j, k) order, each an int or a slice/array
        i, j, k = ijk
        return arr[:, k, j, i]

    def end(c):              # coarse end index -> fine end index
        return 0 if c == 0 else Nf

    def min_nonzero(block):
        b = block.reshape(E, -1)
        big = np.iinfo(np.int64).max
        m = np.where(b > 0, b, big).min(axis=1)
        return np.where(m == big, 0, m)

    for k, j, i in itertools.product(range(NPc), repeat=3):
        c = (i, j, k)
        mids = [d for d in range(3) if 0 < c[d] < Nc]
        if len(mids) == 3:
            continue
        if len(mids) == 0:
            fi = tuple(end(v) for v in c)
            g = fine_at(gf, fi)
            gc[:, k, j, i] = np.where(g > 0, (g * 3 + 0) * 256, 0)
            dc[:, k, j, i] = fine_at(df, fi)
        elif len(mids) == 1:
            dd = mids[0]
            base = [end(v) for v in c]
            a_ijk, b_ijk = list(base), list(base)
            a_ijk[dd], b_ijk[dd] = 0, Nf
            gA, gB = fine_at(gf, a_ijk), fine_at(gf, b_ijk)
            inner = list(base)
            inner[dd] = slice(1, Nf)
            ent = min_nonzero(fine_at(gf, inner))
            t = np.where(gA < gB, c[dd], Nc - c[dd])
            gc[:, k, j, i] = np.where(ent > 0, (ent * 3 + 1) * 256 + t, 0)
            dc[:, k, j, i] = fine_at(df, inner).reshape(E, -1).any(axis=1)
        else:
            d1, d2 = mids
            base = [end(v) for v in c]

            def corner(s1, s2):
                p = list(base)
                p[d1], p[d2] = s1 * Nf, s2 * Nf
                return fine_at(gf, p)

            cg = np.stack([corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)], 1)  # (E,4): s1 + 2 s2
            o = np.argmin(cg, axis=1)
            o1, o2 = o % 2, o // 2
            n1 = cg[np.arange(E), (1 - o1) + 2 * o2]
            n2 = cg[np.arange(E), o1 + 2 * (1 - o2)]
            a_o = np.where(o1 == 0, c[d1], Nc - c[d1])
            b_o = np.where(o2 == 0, c[d2], Nc - c[d2])
            ap = np.where(n1 < n2, a_o, b_o)
            bp = np.where(n1 < n2, b_o, a_o)
            inner = list(base)
            inner[d1], inner[d2] = slice(1, Nf), slice(1, Nf)
            ent = min_nonzero(fine_at(gf, inner))
            gc[:, k, j, i] = np.where(ent > 0, (ent * 3 + 2) * 256 + ap * 16 + bp, 0)
            dc[:, k, j, i] = fine_at(df, inner).reshape(E, -1).any(axis=1)
    return gc, dc


def coarsen(fine: Level, Nc: int) -> Level:
    """Order-Nc level on the same elements: coordinates are the fine isoparametric
    map evaluated at the order-Nc GLL points (eq. xijk), the operator is
    rediscretised there, and the numbering comes from coarse_numbering."""
    xic, _ = gll(Nc)
    Jfc = interp_matrix(fine.xi, xic)          # (NPc, NPf): fine nodal values -> coarse points
    xc = interp_local(fine.x, Jfc)
    yc = interp_local(fine.y, Jfc)
    zc = interp_local(fine.z, Jfc)
    gc, dc = coarse_numbering(fine.gid, fine.dirichlet, fine.N, Nc)
    return Level(Nc, fine.E, xc, yc, zc, gc, dc)


def coarsen_field(fine: Level, coarse: Level, fL):
    """A nodal field of the fine level evaluated at the coarse level's GLL points, element by
    element, the way coarsen() evaluates the coordinates (the fine interpolant at the coarse
    points). Used for a nodal coefficient h1 on the multigrid levels."""
    Jfc = interp_matrix(fine.xi, coarse.xi)
    return interp_local(np.asarray(fL, dtype=np.float64).reshape(fine.x.shape), Jfc)


def prolong(fine: Level, coarse: Level, ec):
    """P e_c = R_f Q_f^T W_f J_L Q_c e_c: interpolate every element, average the copies."""
    Jcf = interp_matrix(coarse.xi, fine.xi)    # (NPf, NPc)
    uc = q_gather(coarse.mask(ec), coarse.node).reshape(coarse.x.shape)
    uf = interp_local(uc, Jcf)
    w = 1.0 / fine.maps["mult"].reshape(fine.x.shape)
    return fine.mask(q_scatter(w * uf, fine.node, fine.n_G))


def restrict(fine: Level, coarse: Level, rf):
    """R = P^T: r_c = R_c Q_c^T J_L^T W_f Q_f R_f^T r_f."""
    Jcf = interp_matrix(coarse.xi, fine.xi)
    w = 1.0 / fine.maps["mult"].reshape(fine.x.shape)
    uf = w * q_gather(fine.mask(rf), fine.node).reshape(fine.x.shape)
    uc = interp_local_T(uf, Jcf)
    return coarse.mask(q_scatter(uc, coarse.node, coarse.n_G))


def build_levels(mesh: dict, orders=None):
    """Levels for the multigrid schedule N, N/2, ..., 1 (default) or the given orders."""
    top = level_from_mesh(mesh)
    if orders is None:
        orders = [top.N]
        while orders[-1] > 1:
            orders.append(max(1, orders[-1] // 2))
    if orders[0] != top.N:
        raise ValueError("first order must be the mesh order")
    levels = [top]
    for Nc in orders[1:]:
        levels.append(coarsen(levels[-1], Nc))
    return levels


# ----------------------------------------------------------------------------
# Overlapping additive Schwarz smoother with fast-diagonalisation local solves
# (Section 3.4: ASM on extended elements of (N+3)^3 points, local solves by
# tensor-product fast diagonalisation in about 12 E (N+3)^4 operations; the
# method of Lynch, Rice and Thomas (1964) as used for spectral elements by
# Deville, Fischer and Mund (2002) and Lottes and Fischer (2005))
# ----------------------------------------------------------------------------

# face-side boundary types of the 1-D extended segment
SCH_NB, SCH_DIR, SCH_NEU = 0, 1, 2


def fdm_1d(N: int, left: int, right: int):
    """Reference (element length 2) 1-D data of the extended segment of an element.

    The segment is the element's N+1 GLL nodes plus one node on each side: the
    first interior node of the neighbouring element, taken as an element of the
    same length (SCH_NB). The 1-D stiffness K = D^T diag(rho) D and mass
    diag(rho) of the (up to) three elements are assembled and restricted to the
    segment's nodes, i.e. homogeneous Dirichlet conditions one node beyond the
    overlap. A side on a Dirichlet boundary (SCH_DIR) drops the boundary node
    and the extension node; a Neumann side (SCH_NEU) keeps the boundary node and
    has no extension node.

    Returns S (N+3, N+3) and lam (N+3): S^T B S = I and S^T A S = diag(lam) on
    the present slots (slot s = extended index + 1, extended index -1..N+1);
    rows of absent slots and the unused columns are zero (their lam is 1).
    """
    _, rho = gll(N)
    D = deriv_matrix(N)
    K = D.T @ np.diag(rho) @ D
    n = 3 * N + 1
    A = np.zeros((n, n))
    Bd = np.zeros(n)
    for el, present in ((0, left == SCH_NB), (1, True), (2, right == SCH_NB)):
        if present:
            sl = slice(el * N, el * N + N + 1)
            A[sl, sl] += K
            Bd[sl] += rho
    slots = []
    for ext in range(-1, N + 2):
        if ext == -1 and left != SCH_NB:
            continue
        if ext == 0 and left == SCH_DIR:
            continue
        if ext == N and right == SCH_DIR:
            continue
        if ext == N + 1 and right != SCH_NB:
            continue
        slots.append(ext)
    g = np.array([N + ext for ext in slots])
    As = A[np.ix_(g, g)]
    bs = Bd[g]
    # A s = lam B s with B diagonal: symmetric form B^-1/2 A B^-1/2 = Q diag(lam) Q^T, S = B^-1/2 Q
    isq = 1.0 / np.sqrt(bs)
    lam, Q = np.linalg.eigh(isq[:, None] * As * isq[None, :])
    S = np.zeros((N + 3, N + 3))
    lam_full = np.ones(N + 3)
    S[np.array(slots) + 1, : len(slots)] = isq[:, None] * Q
    lam_full[: len(slots)] = lam
    return S, lam_full


def element_lengths(level: "Level") -> np.ndarray:
    """(E, 3) lengths of each element along r, s, t: the mean, over the (N+1)^2
    grid lines in that direction, of the distance between the line's end nodes."""
    X = np.stack([level.x, level.y, level.z])          # (3, E, k, j, i)
    N = level.N
    Lr = np.sqrt(((X[..., N] - X[..., 0]) ** 2).sum(0)).mean(axis=(1, 2))
    Ls = np.sqrt(((X[..., N, :] - X[..., 0, :]) ** 2).sum(0)).mean(axis=(1, 2))
    Lt = np.sqrt(((X[:, :, N] - X[:, :, 0]) ** 2).sum(0)).mean(axis=(1, 2))
    return np.stack([Lr, Ls, Lt], 1)


def face_points(N: int, f: int):
    """Local (i, j, k) of face f (2d + side: d = 0 r, 1 s, 2 t; side 0 at index 0,
    side 1 at index N) as arrays indexed [a, b], with (a, b) the two other
    indices in r, s, t order."""
    d, side = divmod(f, 2)
    a, b = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    c = np.full_like(a, side * N)
    ijk = [None, None, None]
    ijk[d] = c
    others = [q for q in range(3) if q != d]
    ijk[others[0]] = a
    ijk[others[1]] = b
    return ijk


@dataclass
class Schwarz:
    """Per-level data of the Schwarz smoother.

    layer[e, f, a, b]: unique node of the face-layer slot of face f of element e
    at face position (a, b) -- the node one step inside the neighbouring element
    from the shared face node -- or -1 when the face has no neighbour.
    btype[e, f]: SCH_NB, SCH_DIR or SCH_NEU. L[e]: element lengths (r, s, t).
    W: 1 / (number of subdomain slots holding each unique node), 0 at Dirichlet nodes.
    """
    layer: np.ndarray
    btype: np.ndarray
    L: np.ndarray
    W: np.ndarray
    fdm: dict


def schwarz_setup(level: "Level") -> Schwarz:
    """Face-layer maps from the node numbering: the neighbour across face f is the
    other element holding the face's centre node; in that element the face is
    the one on which all of the face's nodes lie, and each layer node is one
    step from the face along that element's face-normal index."""
    N, E = level.N, level.E
    if N < 2:
        raise ValueError("the Schwarz smoother needs N >= 2")
    NP = N + 1
    node = level.node.reshape(E, NP, NP, NP)           # [e, k, j, i]
    holders = {}
    for e in range(E):
        for loc, g in enumerate(node[e].ravel()):
            holders.setdefault(int(g), []).append((e, loc))
    layer = -np.ones((E, 6, NP, NP), dtype=np.int64)
    btype = np.zeros((E, 6), dtype=np.int64)
    for e in range(E):
        for f in range(6):
            i, j, k = face_points(N, f)
            fn = node[e][k, j, i]                       # face nodes [a, b]
            centre = int(fn[1, 1])
            other = [h for h in holders[centre] if h[0] != e]
            if not other:
                btype[e, f] = SCH_DIR if level.dir_g[centre] else SCH_NEU
                continue
            btype[e, f] = SCH_NB
            e2 = other[0][0]
            loc2 = {int(g): l for l, g in enumerate(node[e2].ravel())}
            pos = np.array([[np.unravel_index(loc2[int(g)], (NP, NP, NP)) for g in row] for row in fn])  # (a, b, [k, j, i])
            # the coordinate that is constant (0 or N) over the face in e2, and the step inward
            for ax in range(3):
                v = pos[..., ax]
                if np.all(v == v.flat[0]) and v.flat[0] in (0, N):
                    break
            else:
                raise ValueError("non-conforming face")
            pos2 = pos.copy()
            pos2[..., ax] = 1 if pos[0, 0, ax] == 0 else N - 1
            layer[e, f] = node[e2][pos2[..., 0], pos2[..., 1], pos2[..., 2]]
    L = element_lengths(level)
    fdm = {}
    for e in range(E):
        for d in range(3):
            key = (int(btype[e, 2 * d]), int(btype[e, 2 * d + 1]))
            if key not in fdm:
                fdm[key] = fdm_1d(N, *key)
    sch = Schwarz(layer, btype, L, np.zeros(level.n_G), fdm)
    c = schwarz_sum(level, sch, lambda e, box: box, np.ones(level.n_G))
    sch.W = np.where(level.free & (c > 0), 1.0 / np.maximum(c, 1.0), 0.0)
    return sch


def box_face_slots(N: int, f: int, a=None):
    """Index tuple (k, j, i) into an (N+3)^3 box of the face-layer slots of face f."""
    d, side = divmod(f, 2)
    c = 0 if side == 0 else N + 2
    inner = slice(1, N + 2)
    ijk = [inner, inner, inner]
    ijk[d] = c
    return (ijk[2], ijk[1], ijk[0])


def schwarz_sum(level: "Level", sch: Schwarz, local, r):
    """sum_e P_e^T local(e, P_e r): P_e r is the (N+3)^3 box of element e holding r
    at its own nodes and at its face-layer nodes (zero elsewhere: absent layers
    and the box's edge and corner strips); P_e^T adds the own and face-layer
    slots of a box back to their nodes."""
    N, E = level.N, level.E
    NP = N + 1
    node = level.node.reshape(E, NP, NP, NP)
    z = np.zeros(level.n_G)
    for e in range(E):
        box = np.zeros((NP + 2,) * 3)
        box[1:-1, 1:-1, 1:-1] = r[node[e]]
        for f in range(6):
            if sch.btype[e, f] == SCH_NB:
                # face positions (a, b) run over the two other indices in r, s, t order; the box
                # slice of face f keeps its remaining axes in (k, j, i) order, i.e. (b, a)
                box[box_face_slots(N, f)] = r[sch.layer[e, f]].T
        out = local(e, box)
        np.add.at(z, node[e], out[1:-1, 1:-1, 1:-1])
        for f in range(6):
            if sch.btype[e, f] == SCH_NB:
                np.add.at(z, sch.layer[e, f].T, out[box_face_slots(N, f)])
    return z


def fdm_solve(sch: Schwarz, e: int, box, h1: float, h2: float):
    """Fast-diagonalisation solve on the extended box of element e:
    (S_t x S_s x S_r) diag(1 / (h1 (lam_r + lam_s + lam_t) + h2)) (S_t x S_s x S_r)^T box,
    for the separable operator h1 (B B A + B A B + A B B) + h2 (B B B) of a box
    with the element's lengths; S_d = sqrt(2/L_d) S_ref and lam_d = (2/L_d)^2 lam_ref
    scale the reference data of fdm_1d to length L_d."""
    Lr, Ls, Lt = sch.L[e]
    Sr, lr = sch.fdm[(int(sch.btype[e, 0]), int(sch.btype[e, 1]))]
    Ss, ls = sch.fdm[(int(sch.btype[e, 2]), int(sch.btype[e, 3]))]
    St, lt = sch.fdm[(int(sch.btype[e, 4]), int(sch.btype[e, 5]))]
    u = np.einsum("ma,kjm->kja", Sr, box)             # S_r^T along i
    u = np.einsum("mb,kma->kba", Ss, u)               # S_s^T along j
    u = np.einsum("mc,mba->cba", St, u)               # S_t^T along k
    lam = h1 * ((2.0 / Lt) ** 2 * lt[:, None, None] + (2.0 / Ls) ** 2 * ls[None, :, None]
                + (2.0 / Lr) ** 2 * lr[None, None, :]) + h2
    u = np.where(lam != 0.0, u / np.where(lam != 0.0, lam, 1.0), 0.0)
    u = u * ((2.0 / Lr) * (2.0 / Ls) * (2.0 / Lt))
    u = np.einsum("cm,mba->cba", St, u)
    u = np.einsum("bm,kma->kba", Ss, u)
    u = np.einsum("am,kjm->kja", Sr, u)
    return u


def asm_apply(level: "Level", sch: Schwarz, r, h1: float = 1.0, h2: float = 0.0):
    """Weighted additive Schwarz: z = W sum_e P_e^T F_e P_e r, F_e the local FDM solve,
    masked. The weight W makes the preconditioner slightly nonsymmetric (Section 3.4)."""
    z = schwarz_sum(level, sch, lambda e, box: fdm_solve(sch, e, box, h1, h2), r)
    return level.mask(sch.W * z)


def arnoldi_lmax(apply, minv, v0, steps: int = 10) -> float:
    """Estimate of the largest eigenvalue of M A by ``steps`` Arnoldi steps (modified
    Gram-Schmidt) from v0: the largest eigenvalue of the symmetric part (H + H^T)/2
    of the Hessenberg matrix H = V^T M A V, an upper bound on the real parts of
    its Ritz values."""
    V = [v0 / np.linalg.norm(v0)]
    H = np.zeros((steps + 1, steps))
    k = steps
    for j in range(steps):
        w = minv(apply(V[j]))
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            k = j + 1
            break
        V.append(w / H[j + 1, j])
    Hk = H[:k, :k]
    return float(np.max(np.linalg.eigvalsh(0.5 * (Hk + Hk.T))))


# ----------------------------------------------------------------------------
# Krylov solvers, smoother, eigenvalue estimate, V-cycle
# ----------------------------------------------------------------------------


def splitmix64(seed: int, counters) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood 2014), counter form mix(seed + (c+1)*0x9E3779B97F4A7C15)."""
    c = np.asarray(counters).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def lanczos_start(level: Level, seed: int = 1):
    """Seeded start vector: U[-1,1) per unique node, drawn at the node's smallest local index."""
    label = level.maps["label"]
    first = np.zeros(level.n_G, dtype=np.int64)
    first[level.node] = label
    u = (splitmix64(seed, first) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return level.mask(2.0 * u - 1.0)


def lanczos_lmax(apply, dinv, v0, steps: int = 10) -> float:
    """Largest Ritz value of ``steps`` Lanczos steps on S = D^{-1/2} A D^{-1/2} (same spectrum as D^{-1} A)."""
    s = np.sqrt(dinv)
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    beta = 0.0
    alphas, betas = [], []
    for j in range(steps):
        w = s * apply(s * v) - beta * v_prev
        alpha = float(w @ v)
        w = w - alpha * v
        alphas.append(alpha)
        beta = float(np.linalg.norm(w))
        if j == steps - 1 or beta == 0.0:
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
    return float(np.linalg.eigvalsh(T).max())


def cheb_smooth(apply, dinv, b, x, lmin: float, lmax: float, degree: int):
    """Chebyshev-accelerated Jacobi, ``degree`` steps on A x = b (Saad, Alg. 12.1 form).

    theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma = theta/delta, rho = 1/sigma;
    d = D^{-1} r / theta, x += d; then for each further step:
    r = b - A x, rho' = 1/(2 sigma - rho), d = rho' rho d + (2 rho'/delta) D^{-1} r, x += d.
    ``x`` None means a zero initial guess (r = b without a matvec). A callable
    ``dinv`` replaces D^{-1} r by dinv(r) (Chebyshev-accelerated Schwarz, CHEBY-ASM).
    """
    if not callable(dinv):
        dvec = dinv
        dinv = lambda v: dvec * v
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x is None:
        r = b
        x = np.zeros_like(b)
    else:
        r = b - apply(x)
    d = dinv(r) / theta
    x = x + d
    for _ in range(1, degree):
        r = b - apply(x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * dinv(r)
        x = x + d
        rho = rho_new
    return x


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    relres: float
    history: list


def pcg(apply, b, minv, tol: float, maxit: int, flexible: bool = False, bnorm: float | None = None) -> SolveResult:
    """Preconditioned CG from x0 = 0 (Saad, Alg. 9.1), stopping when ||r||/||b|| <= tol.

    With ``flexible`` the Polak-Ribiere form beta = (z_{k+1}, r_{k+1} - r_k) / (z_k, r_k)
    is used (flexible CG, Section 3.4); otherwise
    beta = (z_{k+1}, r_{k+1}) / (z_k, r_k). ``bnorm`` replaces ||b|| in the stopping
    test and the reported residuals (a projected solve measures its residual
    against the norm of the right-hand side before projection).
    """
    x = np.zeros_like(b)
    r = b.copy()
    if bnorm is None:
        bnorm = float(np.linalg.norm(b))
    hist = [float(np.linalg.norm(b)) / bnorm if bnorm > 0.0 else 0.0]
    if bnorm == 0.0 or hist[0] <= tol:
        return SolveResult(x, 0, hist[0], hist)
    z = minv(r)
    p = z.copy()
    rz = float(r @ z)
    k = 0
    relres = hist[0]
    while k < maxit:
        w = apply(p)
        alpha = rz / float(p @ w)
        x = x + alpha * p
        r_old = r
        r = r - alpha * w
        k += 1
        relres = float(np.linalg.norm(r)) / bnorm
        hist.append(relres)
        if relres <= tol:
            break
        z = minv(r)
        if flexible:
            beta = float(z @ (r - r_old)) / rz
        else:
            beta = float(z @ r) / rz
        rz = float(r @ z)
        p = z + beta * p
    return SolveResult(x, k, relres, hist)


@dataclass
class MGParams:
    degree: int = 2
    lmin_factor: float = 0.1
    lmax_factor: float = 1.1
    lanczos_steps: int = 10
    lanczos_seed: int = 1
    coarse_tol: float = 1e-1
    coarse_maxit: int = 100
    lmax: list | None = None     # per smoothed level; estimated by Lanczos/Arnoldi when None
    smoother: str = "jacobi"     # "jacobi" (CHEBY-JAC) or "asm" (CHEBY-ASM)


class PMG:
    """p-multigrid V-cycle with Chebyshev-accelerated smoothing (Jacobi or the
    overlapping Schwarz smoother) on every level but the coarsest and a
    Jacobi-PCG coarse solve (Section 3.4, "Poisson Solve Preconditioning")."""

    def __init__(self, levels, h1=1.0, h2=0.0, params: MGParams | None = None):
        """h1: a scalar, or a nodal coefficient on the fine level (an L-vector shaped like
        levels[0].x), carried to every coarser level by coarsen_field (level by level)."""
        self.levels = levels
        self.h1, self.h2 = h1, h2
        self.p = params or MGParams()
        if np.ndim(h1) == 0:
            h1s = [h1] * len(levels)
        else:
            h1s = [np.asarray(h1, dtype=np.float64).reshape(levels[0].x.shape)]
            for l in range(1, len(levels)):
                h1s.append(coarsen_field(levels[l - 1], levels[l], h1s[-1]))
            if self.p.smoother == "asm":
                raise ValueError("the Schwarz smoother takes a scalar h1")
        self.h1_levels = h1s
        self.dinv = [np.where(L.free, 1.0 / L.diag(h, h2), 0.0) for L, h in zip(levels, h1s)]
        self.ops = [(lambda v, L=L, h=h: L.apply(v, h, h2)) for L, h in zip(levels, h1s)]
        nsm = len(levels) - 1
        if self.p.smoother == "asm":
            self.sch = [schwarz_setup(levels[l]) for l in range(nsm)]
            self.minv = [(lambda r, L=levels[l], S=self.sch[l]: asm_apply(L, S, r, h1, h2)) for l in range(nsm)]
        elif self.p.smoother == "jacobi":
            self.minv = [self.dinv[l] for l in range(nsm)]
        else:
            raise ValueError(self.p.smoother)
        if self.p.lmax is None:
            if self.p.smoother == "asm":
                self.lmax = [arnoldi_lmax(self.ops[l], self.minv[l], lanczos_start(levels[l], self.p.lanczos_seed),
                                          self.p.lanczos_steps) for l in range(nsm)]
            else:
                self.lmax = [lanczos_lmax(self.ops[l], self.dinv[l], lanczos_start(levels[l], self.p.lanczos_seed),
                                          self.p.lanczos_steps) for l in range(nsm)]
        else:
            self.lmax = list(self.p.lmax)
        self.coarse_iters = []

    def smooth(self, l, b, x):
        lam = self.lmax[l]
        return cheb_smooth(self.ops[l], self.minv[l], b, x, self.p.lmin_factor * lam,
                           self.p.lmax_factor * lam, self.p.degree)

    def vcycle(self, l, r):
        if l == len(self.levels) - 1:
            res = pcg(self.ops[l], r, lambda v: self.dinv[l] * v, self.p.coarse_tol, self.p.coarse_maxit)
            self.coarse_iters.append(res.iters)
            return res.x
        x = self.smooth(l, r, None)
        res = r - self.ops[l](x)
        ec = self.vcycle(l + 1, restrict(self.levels[l], self.levels[l + 1], res))
        x = x + prolong(self.levels[l], self.levels[l + 1], ec)
        return self.smooth(l, r, x)

    def __call__(self, r):
        return self.vcycle(0, r)


def solve(level: Level, b, h1=1.0, h2=0.0, tol=1e-8, maxit=1000, precond="jacobi",
          levels=None, params: MGParams | None = None) -> SolveResult:
    """Solve R Q^T A_L Q R^T x = b: Jacobi-PCG, or flexible PCG with the p-MG V-cycle
    (h1 a scalar or a nodal L-vector on `level`, which must be levels[0] for p-MG)."""
    op = lambda v: level.apply(v, h1, h2)
    if precond == "jacobi":
        dinv = np.where(level.free, 1.0 / level.diag(h1, h2), 0.0)
        return pcg(op, b, lambda v: dinv * v, tol, maxit)
    if precond == "pmg":
        mg = PMG(levels, h1, h2, params)
        res = pcg(op, b, mg, tol, maxit, flexible=True)
        res.mg = mg
        return res
    raise ValueError(precond)


# ----------------------------------------------------------------------------
# Projection of successive right-hand sides (Section 3.4, "projection-based
# initial guesses"; Fischer, CMAME 163, 1998)
# ----------------------------------------------------------------------------

# A new direction is dropped when orthogonalisation leaves less than this
# fraction of its squared A-norm (it lies in the span up to round-off).
PROJ_DROP = 1e-20


class Projection:
    """Space of earlier solutions kept as an A-orthonormal basis x_1..x_l with
    the products b_i = A x_i stored beside it.

    project(b): for an A-orthonormal basis the A-norm-closest element of
    span{x_i} to the solution x* of A x* = b is xbar = sum_i (x_i^T A x*) x_i =
    sum_i (x_i, b) x_i, and its residual r0 = b - A xbar = b - sum_i (x_i, b) b_i
    costs no operator application.

    update(x, dx): after the solve of A dx = r0, the new direction is dx, or
    the whole solution x when the basis already holds max_vectors (the basis
    restarts from x alone). It is made A-orthogonal to the basis by classical
    Gram-Schmidt applied twice, v <- v - sum_i (x_i, A v) x_i with A v carried
    along as A v <- A v - sum_i (x_i, A v) b_i, then scaled to unit A-norm and
    appended, unless it vanished (PROJ_DROP).
    """

    def __init__(self, apply, max_vectors: int):
        self.apply = apply
        self.max_vectors = max_vectors
        self.X: list[np.ndarray] = []
        self.AX: list[np.ndarray] = []

    def project(self, b):
        xbar = np.zeros_like(b)
        r0 = b.copy()
        for xi, bi in zip(self.X, self.AX):
            a = float(xi @ b)
            xbar = xbar + a * xi
            r0 = r0 - a * bi
        return xbar, r0

    def update(self, x, dx):
        if len(self.X) == self.max_vectors:
            self.X, self.AX = [], []
            v = x.copy()
        else:
            v = dx.copy()
        w = self.apply(v)
        n0 = float(v @ w)
        for _ in range(2):
            beta = [float(xi @ w) for xi in self.X]
            for bt, xi, bi in zip(beta, self.X, self.AX):
                v = v - bt * xi
                w = w - bt * bi
        n2 = float(v @ w)
        if n2 > 0.0 and n2 > PROJ_DROP * n0:
            s = 1.0 / np.sqrt(n2)
            self.X.append(s * v)
            self.AX.append(s * w)
            return True
        return False


def solve_projected(level: Level, proj: Projection, b, h1=1.0, h2=0.0, tol=1e-8, maxit=1000,
                    precond="jacobi", mg: "PMG | None" = None) -> SolveResult:
    """Solve A x = b from the projected initial guess: xbar, r0 = proj.project(b);
    A dx = r0 by PCG from zero (flexible PCG + p-MG when precond == "pmg"),
    stopping at ||r|| <= tol ||b||; x = xbar + dx; proj.update(x, dx).
    The result's relres0 is ||r0|| / ||b||."""
    op = lambda v: level.apply(v, h1, h2)
    bnorm = float(np.linalg.norm(b))
    xbar, r0 = proj.project(b)
    if precond == "jacobi":
        dinv = np.where(level.free, 1.0 / level.diag(h1, h2), 0.0)
        res = pcg(op, r0, lambda v: dinv * v, tol, maxit, bnorm=bnorm)
    elif precond == "pmg":
        res = pcg(op, r0, mg, tol, maxit, flexible=True, bnorm=bnorm)
    else:
        raise ValueError(precond)
    x = xbar + res.x
    res.added = proj.update(x, res.x)
    res.relres0 = res.history[0]
    res.xbar = xbar
    res.x = x
    return res


# ----------------------------------------------------------------------------
# Dealiased advection operator (Section 2.1, eq. stdadv and eq. hyp, whose
# nonlinear term is evaluated on N_q^3 quadrature points; Section 3.3 "High-Order
# Kernels" on its N_q^3 dealiased evaluation)
# ----------------------------------------------------------------------------


def cubature_points(N: int, nq: int | None = None):
    """Gauss-Legendre rule of the dealiased evaluation: nq = ceil(3 (N+1) / 2) points
    by default (N=7 -> 12), exact for polynomials of degree <= 2 nq - 1
    (numpy.polynomial.legendre.leggauss)."""
    if nq is None:
        nq = (3 * (N + 1) + 1) // 2
    z, w = np.polynomial.legendre.leggauss(nq)
    return z, w


@dataclass
class Cubature:
    """Per-level data of the dealiased evaluation: the interpolation Im from the
    GLL nodes to the Gauss points, the derivative matrix Dq on the Gauss points,
    and at every Gauss point of every element the nine factors
    Gq[e, d, m] = w_q J_q dr_d/dx_m (quadrature weight, Jacobian, inverse metric)."""
    nq: int
    z: np.ndarray
    w: np.ndarray
    Im: np.ndarray
    Dq: np.ndarray
    Gq: np.ndarray


def cubature_setup(level: "Level", nq: int | None = None) -> Cubature:
    """The isoparametric map (eq. xijk) interpolated to the Gauss points and
    differentiated there (the map is a degree-N polynomial, so both steps are
    exact); the 3x3 metric is inverted pointwise (numpy.linalg.inv)."""
    z, w = cubature_points(level.N, nq)
    Im = interp_matrix(level.xi, z)
    Dq = lagrange_deriv_matrix(z)
    X = [interp_local(c - c[:, :1, :1, :1], Im) for c in (level.x, level.y, level.z)]
    d = [grad_ref(c, Dq) for c in X]                        # d[m][q] = dx_m / dr_q
    Jm = np.stack([np.stack(d[m], -1) for m in range(3)], -2)   # (..., m, q)
    det = np.linalg.det(Jm)
    inv = np.linalg.inv(Jm)                                  # (..., q, m) = dr_q / dx_m
    w3 = w[:, None, None] * w[None, :, None] * w[None, None, :]
    Gq = np.moveaxis(inv, (-2, -1), (1, 2)) * (w3 * det)[:, None, None]
    return Cubature(len(z), z, w, Im, Dq, Gq)


def advect_local(level: "Level", cub: Cubature, cL, uL):
    """w_L = the dealiased weak advection term of u with advecting field c, element
    by element: (C u)_i = sum_q w_q J_q phi_i(x_q) (c . grad u)(x_q).

    c at the Gauss points is interpolated from its nodal values, the
    contravariant field chat_d = w_q J_q sum_m (dr_d/dx_m) c_m is formed, u is
    interpolated and differentiated on the Gauss points, and the pointwise
    product sum_d chat_d du/dr_d is projected back with the transposed
    interpolation. cL: (3, E, NP, NP, NP); uL: (E, NP, NP, NP)."""
    cq = [interp_local(cL[m], cub.Im) for m in range(3)]
    chat = [sum(cub.Gq[:, dd, m] * cq[m] for m in range(3)) for dd in range(3)]
    uq = interp_local(uL, cub.Im)
    ur, us, ut = grad_ref(uq, cub.Dq)
    conv = chat[0] * ur + chat[1] * us + chat[2] * ut
    return interp_local_T(conv, cub.Im)


def advect_assembled(level: "Level", cub: Cubature, cL, ug):
    """Q^T C_L Q u on a global vector (no Dirichlet mask: the advection term is explicit)."""
    uL = q_gather(ug, level.node).reshape(level.x.shape)
    return q_scatter(advect_local(level, cub, cL, uL), level.node, level.n_G)


def char_advance(level: "Level", cub: Cubature, c0L, c1L, w0, t0: float, t1: float, nsub: int):
    """The hyperbolic subproblem of the characteristics scheme (Section 2.1, eq. hyp):
    dw/dt = -M^-1 Q^T C(c(t)) Q w on [t0, t1] from w(t0) = w0, with the assembled
    diagonal GLL mass M and the dealiased advection operator C, by nsub classical
    Runge-Kutta steps (RK4). The wind is linear in time between its values c0 at t0
    and c1 at t1 (c1 None: frozen). w0: list of global vectors (components)."""
    minv = 1.0 / level.mass()
    h = (t1 - t0) / nsub

    def wind(t):
        if c1L is None:
            return c0L
        th = (t - t0) / (t1 - t0)
        return c0L + th * (c1L - c0L)

    def f(t, w):
        cL = wind(t)
        return [-minv * advect_assembled(level, cub, cL, wc) for wc in w]

    w = [np.array(wc, dtype=np.float64) for wc in w0]
    for q in range(nsub):
        t = t0 + q * h
        k1 = f(t, w)
        k2 = f(t + 0.5 * h, [wc + 0.5 * h * kc for wc, kc in zip(w, k1)])
        k3 = f(t + 0.5 * h, [wc + 0.5 * h * kc for wc, kc in zip(w, k2)])
        k4 = f(t + h, [wc + h * kc for wc, kc in zip(w, k3)])
        w = [wc + (h / 6.0) * (a1 + 2.0 * a2 + 2.0 * a3 + a4) for wc, a1, a2, a3, a4 in zip(w, k1, k2, k3, k4)]
    return w


# ----------------------------------------------------------------------------
# Adjoint gradient with respect to nodal h1
# ----------------------------------------------------------------------------


def grad_h1_local(level: Level, uL, lamL):
    """g_L = -sum_{m,m'} (D_m lam) G_mm' (D_m' u) at every local point (G without h1).

    For A(h1) = Q^T [D^T (h1 G) D] Q with h1 nodal, dA/dh1 at a local point is the
    pointwise factor of eq. Ae, so dL/dh1 = -lam^T (dA/dh1) u with A lam = dL/du.
    """
    lr, ls, lt = grad_ref(lamL, level.D)
    ur, us, ut = grad_ref(uL, level.D)
    Gf = _g_full(level.G)
    gl = (lr, ls, lt)
    gu = (ur, us, ut)
    acc = np.zeros_like(uL)
    for m in range(3):
        for mp in range(3):
            acc += gl[m] * Gf[m][mp] * gu[mp]
    return -acc


def adjoint_loss_and_grads(level: Level, fL, h1L, h2, u_target_L, tol=1e-13, maxit=5000):
    """Loss L = 1/2 sum_l B_l (u_l - t_l)^2 over local points, u_L = Q u with A(h1, h2) u = R Q^T B_L f_L.

    For continuous u_L and t_L this is 1/2 (u - t)^T M (u - t) with the assembled
    mass M = Q^T B_L Q. Returns (L, u, lam, dL/df_L, dL/dh1_L): the adjoint solve
    A lam = R Q^T (dL/du_L) uses the symmetry of A (A = R Q^T A_L Q R^T is SPD),
    dL/df_L = B_L Q lam and dL/dh1_L is grad_h1_local.
    """
    b = level.rhs_from_nodal(fL)
    u = solve(level, b, h1L, h2, tol=tol, maxit=maxit).x
    uL = q_gather(u, level.node).reshape(level.x.shape)
    gL = level.B * (uL - u_target_L)
    loss = 0.5 * float(np.sum(level.B * (uL - u_target_L) ** 2))
    lam = solve(level, level.mask(q_scatter(gL, level.node, level.n_G)), h1L, h2, tol=tol, maxit=maxit).x
    lamL = q_gather(lam, level.node).reshape(level.x.shape)
    dfL = level.B * lamL
    dh1L = grad_h1_local(level, uL, lamL)
    return loss, u, lam, dfL, dh1L
