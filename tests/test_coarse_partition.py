"""Host-side sub-domain partition of the pipelined coarse solve (no GPU).

The one-launch coarse Jacobi-PCG splits the order-1 elements into sub-domains
and replaces the direct-stiffness summation QQ^T (Section 3.2) by a per-node
gather over every copy of the node. These tests check the structures the
library builds (sem_coarse_partition) exactly: every point maps to its own
node, every node lists all of its copies in canonical order, the published
points are exactly those whose node leaves the sub-domain, each free node is
owned once. Then a NumPy emulation of the kernel's data flow (gathers from the
sub-domain's own outputs and from the exchange buffer, which holds only the
published points) runs pipelined PCG (Ghysels and Vanroose 2014) and must give
the oracle's Jacobi-PCG iterates, as it does in exact arithmetic.
"""
import numpy as np
import pytest

import oracle as O
import sem_inputs as si

MASK = 0x7FFFFFFF


@pytest.fixture(scope="module")
def part_fn():
    from paper_2104_05829_gb300 import build, sem
    build.build()
    return sem.coarse_partition


def _inputs(L):
    nL = L.node.size
    first = np.full(L.n_G, nL)
    np.minimum.at(first, L.node, np.arange(nL))
    dmask = L.dir_g[L.node]
    owner = (first[L.node] == np.arange(nL)) & ~dmask
    return dmask, owner


def _partition(part_fn, L, nblocks):
    dmask, owner = _inputs(L)
    return part_fn(L.node, dmask, owner, L.x, L.y, L.z, L.n_G, nblocks)


def _lpos(p, E):
    return (p["el"].astype(np.int64)[:, None] * 8 + np.arange(8)).ravel()


def _pt_node(p):
    B = len(p["el_off"]) - 1
    out = np.empty(p["p2n"].size, np.int64)
    for b in range(B):
        s = slice(p["el_off"][b] * 8, p["el_off"][b + 1] * 8)
        out[s] = p["nd_off"][b] + (p["p2n"][s] & MASK)
    return out


@pytest.mark.parametrize("shape,nblocks", [((5, 4, 3), 7), ((4, 3, 3), 1), ((6, 5, 4), 16)])
def test_partition_structures_are_exact(part_fn, shape, nblocks):
    mesh = si.box_mesh(shape, 1, warp=0.1, perm_seed=3, dirichlet=("x0",))
    L = O.level_from_mesh(mesh)
    E, nL = L.E, L.node.size
    p = _partition(part_fn, L, nblocks)
    el, el_off = p["el"], p["el_off"]
    assert np.array_equal(np.sort(el), np.arange(E))
    sizes = np.diff(el_off)
    assert el_off[0] == 0 and el_off[-1] == E and sizes.min() >= 1 and sizes.max() - sizes.min() <= 1
    for b in range(nblocks):
        assert np.all(np.diff(el[el_off[b]:el_off[b + 1]]) > 0)
    lpos = _lpos(p, E)
    pt_node = _pt_node(p)
    blk_of_pt = np.repeat(np.repeat(np.arange(nblocks), sizes), 8)        # in el order
    blk_of_l = np.empty(nL, np.int64)
    blk_of_l[lpos] = blk_of_pt
    nd_src, nd_fl, cp_off, cp = p["nd_src"], p["nd_fl"], p["cp_off"], p["cp"]
    # every point maps to a node of its own sub-domain holding its unique node
    assert np.array_equal(L.node[nd_src[pt_node]], L.node[lpos])
    for b in range(nblocks):
        s = slice(el_off[b] * 8, el_off[b + 1] * 8)
        assert np.all((pt_node[s] >= p["nd_off"][b]) & (pt_node[s] < p["nd_off"][b + 1]))
    owned = np.zeros(L.n_G, np.int64)
    held = {}
    for b in range(nblocks):
        base = el_off[b] * 8
        for j in range(p["nd_off"][b], p["nd_off"][b + 1]):
            g = L.node[nd_src[j]]
            assert blk_of_l[nd_src[j]] == b
            ent = cp[cp_off[j]:cp_off[j + 1]]
            loc = np.where(ent >= 0, lpos[base + np.maximum(ent, 0)], -ent.astype(np.int64) - 1)
            assert np.array_equal(loc, np.flatnonzero(L.node == g))          # all copies, ascending
            assert np.array_equal(ent >= 0, blk_of_l[loc] == b)              # local iff in the sub-domain
            assert bool(nd_fl[j] & 2) == bool(L.dir_g[g])
            owned[g] += int(nd_fl[j] & 1)
            held.setdefault(int(g), []).append(b)
    assert np.array_equal(owned, (~L.dir_g).astype(np.int64))
    assert sorted(held) == list(range(L.n_G))
    # published points: exactly those whose node has a copy in another sub-domain
    multi = np.zeros(L.n_G, bool)
    for g, bs in held.items():
        multi[g] = len(bs) > 1
    assert np.array_equal(p["p2n"] < 0, multi[L.node[lpos]])
    assert p["max_el"] == sizes.max()
    assert p["max_nd"] == np.diff(p["nd_off"]).max()


def test_unwarped_cube_splits_into_octants(part_fn):
    mesh = si.box_mesh(4, 1, warp=0.0, perm_seed=1, dirichlet=())
    L = O.level_from_mesh(mesh)
    p = _partition(part_fn, L, 8)
    cen = np.stack([L.x.reshape(L.E, 8).mean(1), L.y.reshape(L.E, 8).mean(1), L.z.reshape(L.E, 8).mean(1)], 1)
    octs = set()
    for b in range(8):
        side = cen[p["el"][p["el_off"][b]:p["el_off"][b + 1]]] > 0.5
        assert np.all(side == side[0])
        octs.add(tuple(side[0]))
        # a 2x2x2 block of order-1 elements holds 27 nodes; its outer 26 reach other octants
        assert p["nd_off"][b + 1] - p["nd_off"][b] == 27
    assert len(octs) == 8


def _emulate(L, p, b_g, dinv_g, h1, h2, maxit, tol):
    """Pipelined Jacobi-PCG on the sub-domain structures, in the kernel's data flow."""
    E = L.E
    lpos, pt_node = _lpos(p, E), _pt_node(p)
    publish = p["p2n"] < 0
    el_off, nd_off, cp_off, cp = p["el_off"], p["nd_off"], p["cp_off"], p["cp"]
    dir_n, own_n = (p["nd_fl"] & 2) > 0, (p["nd_fl"] & 1) > 0
    nn = len(p["nd_src"])
    g_of = L.node[p["nd_src"]]
    di = np.where(dir_n, 0.0, dinv_g[g_of])
    r = np.where(dir_n, 0.0, b_g[g_of])

    def apply(mn):
        uL = np.empty(8 * E)
        uL[lpos] = mn[pt_node]
        s_pt = O.ax_local(uL.reshape(E, 2, 2, 2), L.G, L.B, L.D, h1, h2).ravel()[lpos]
        xbuf = np.full(8 * E, np.nan)                  # only published points are readable
        xbuf[lpos[publish]] = s_pt[publish]
        out = np.zeros(nn)
        for b in range(len(el_off) - 1):
            base = el_off[b] * 8
            for j in range(nd_off[b], nd_off[b + 1]):
                if dir_n[j]:
                    continue
                vals = [s_pt[base + e] if e >= 0 else xbuf[-e - 1] for e in cp[cp_off[j]:cp_off[j + 1]]]
                acc = vals[0]
                for v in vals[1:]:
                    acc = acc + v
                out[j] = acc
        return out

    u = di * r
    w = apply(u)
    x, z, q, s, pv = (np.zeros(nn) for _ in range(5))
    gam_old = pi_old = bb = tol2 = 0.0
    for it in range(maxit + 1):
        gam, dlt, rr = (float(np.sum((a * c)[own_n])) for a, c in ((r, u), (w, u), (r, r)))
        m = di * w
        n = apply(m)
        if it == 0:
            bb, tol2 = rr, tol * tol * rr
        if rr <= tol2 or it >= maxit:
            break
        beta = 0.0 if it == 0 else gam / gam_old
        pi = dlt if it == 0 else dlt - beta * beta * pi_old      # (p, A p)
        alpha = gam / pi
        z, q, s, pv = n + beta * z, m + beta * q, w + beta * s, u + beta * pv
        x, r, u, w = x + alpha * pv, r - alpha * s, u - alpha * q, w - alpha * z
        gam_old, pi_old = gam, pi
    return x, it, g_of


@pytest.mark.parametrize("nblocks", [1, 5, 12])
def test_pipelined_emulation_reproduces_jacobi_pcg(part_fn, nblocks):
    mesh = si.box_mesh((5, 4, 3), 1, warp=0.1, perm_seed=4, dirichlet=("x0",))
    L = O.level_from_mesh(mesh)
    h1, h2 = 1.0, 0.3
    p = _partition(part_fn, L, nblocks)
    b_g = L.mask(np.random.default_rng(7).standard_normal(L.n_G))
    dinv_g = np.where(L.dir_g, 0.0, 1.0 / L.diag(h1, h2))
    ref = O.pcg(lambda v: L.apply(v, h1, h2), b_g, lambda v: dinv_g * v, tol=0.0, maxit=8)
    x, it, g_of = _emulate(L, p, b_g, dinv_g, h1, h2, maxit=8, tol=0.0)
    assert it == 8
    assert np.max(np.abs(x - ref.x[g_of])) < 1e-10 * np.max(np.abs(ref.x))
    # every copy of a node holds the same bits
    for g in np.unique(g_of):
        assert np.unique(x[g_of == g]).size == 1
    # to a tolerance: the same stopping iteration as the oracle
    ref = O.pcg(lambda v: L.apply(v, h1, h2), b_g, lambda v: dinv_g * v, tol=1e-1, maxit=100)
    x, it, g_of = _emulate(L, p, b_g, dinv_g, h1, h2, maxit=100, tol=1e-1)
    assert it == ref.iters
    assert np.max(np.abs(x - ref.x[g_of])) < 1e-10 * np.max(np.abs(ref.x))


def test_partition_argument_errors(part_fn):
    from paper_2104_05829_gb300 import SemError
    mesh = si.box_mesh((2, 2, 1), 1, warp=0.0, perm_seed=0, dirichlet=())
    L = O.level_from_mesh(mesh)
    with pytest.raises(SemError):
        _partition(part_fn, L, L.E + 1)
    dmask, owner = _inputs(L)
    bad = L.node.copy()
    bad[3] = L.n_G
    with pytest.raises(SemError):
        part_fn(bad, dmask, owner, L.x, L.y, L.z, L.n_G, 2)
