"""Element partitioning across ranks and the interface exchange (Sections 3.1 and 3.2)
on gloo ranks on CPU.

The plan (recursive coordinate bisection, interface ids, buffer positions,
interface-first element order, owner flags) and the exchange (an all-reduce of the
interface buffers) are the package's own code. The rank-local device steps - the
element operator on the rank's elements, the halo gather, the rank's own gather-
scatter and the halo scatter - are emulated here with the oracle, following the
contract of sem_ax_elements / sem_halo_gather / sem_gs / sem_halo_scatter. The
assembled result on every rank must equal the oracle's whole-mesh R QQ^T A_L u on
that rank's points, and the sum over ranks of the owner-flagged products must equal
the unique-node dot product.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shape, N, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        import sem_inputs as si
        from paper_2104_05829_gb300 import dist as D

        mesh = si.box_mesh(shape, N, warp=0.1, perm_seed=3, dirichlet=("x0", "y1"))
        E = mesh["E"]
        part = D.partition(mesh, world)
        P = D.plan(mesh, part, rank)
        loc = P["local"]
        lg, dl = loc["gid"], loc["dirichlet"]
        el = P["elements"]
        u = si.uniform_field(mesh, 0) * (1 - mesh["dirichlet"])           # continuous, masked
        ul = u.reshape(E, -1)[el].reshape(loc["x"].shape)
        # element operator on the rank's elements (sem_ax_elements)
        G, B, _ = O.geometry(loc["x"], loc["y"], loc["z"], N)
        wl = O.ax_local(ul, G, B, O.deriv_matrix(N), 1.0, 0.5).ravel()
        # halo gather: the rank's partial sum of each interface node at its position
        buf = torch.zeros(max(1, P["n_iface"]), dtype=torch.float64)
        at = np.isin(lg, P["iface_gid"])
        k = np.searchsorted(P["iface_gid"], lg)
        part_sums = np.bincount(k[at], weights=wl[at], minlength=P["iface_gid"].size)
        buf[torch.as_tensor(P["iface_pos"], dtype=torch.long)] = torch.as_tensor(part_sums)
        D.exchange(buf)                                                      # the package's collective
        # the rank's own gather-scatter with the Dirichlet mask (sem_gs)
        maps = O.gs_maps(lg)
        w = O.qqt(wl, maps["node"], maps["n_G"]).ravel()
        w[dl == 1] = 0.0
        # halo scatter: every copy of an interface node <- the exchanged sum (0 at Dirichlet)
        tot = buf.numpy()[P["iface_pos"]]
        w[at] = np.where(dl[at] == 1, 0.0, tot[k[at]])
        lev = O.level_from_mesh(mesh)
        ug = O.q_scatter(u.ravel() / lev.maps["mult"], lev.node, lev.n_G)
        ref = O.q_gather(lev.apply(ug, 1.0, 0.5), lev.node).reshape(E, -1)[el].ravel()
        err = float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))
        # unique-node dot product from the owner flags
        a = si.uniform_field(mesh, 4).ravel()
        bb = si.uniform_field(mesh, 5).ravel()
        al, bl = (v.reshape(E, -1)[el].ravel() for v in (a, bb))
        d = torch.tensor([float(np.sum(P["owner"] * al * bl))], dtype=torch.float64)
        D.exchange(d)
        ag, bg = (O.q_scatter(v / lev.maps["mult"], lev.node, lev.n_G) for v in (a, bb))
        dref = float(np.sum((ag * bg)[lev.free]))
        out[rank] = {"err": err, "dot": d.item(), "dref": dref, "scale": float(np.sum(np.abs(ag * bg))),
                     "E": int(el.size), "nb": P["nb"], "n_iface": P["n_iface"], "mine": int(P["iface_gid"].size),
                     "owned": int(P["owner"].sum()), "free": int(lev.free.sum()),
                     "first_are_boundary": bool(np.all(np.isin(lg.reshape(el.size, -1)[:P["nb"]],
                                                               P["iface"]).any(axis=1))),
                     "rest_are_interior": bool(not np.isin(lg.reshape(el.size, -1)[P["nb"]:], P["iface"]).any())}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,N", [(2, (4, 3, 3), 5), (3, (5, 3, 2), 4)])
def test_partitioned_ax_gs_and_dot_match_the_oracle(world, shape, N):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, shape, N, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = [out[r] for r in range(world)]
    E = shape[0] * shape[1] * shape[2]
    assert sum(r["E"] for r in res) == E
    assert max(r["E"] for r in res) - min(r["E"] for r in res) <= 1          # balanced bisection
    for r in res:
        assert r["err"] < 1e-12, r
        assert 0 < r["nb"] <= r["E"] and 0 < r["mine"] <= r["n_iface"]
        assert r["first_are_boundary"] and r["rest_are_interior"]
        assert abs(r["dot"] - r["dref"]) <= 1e-12 * r["scale"]
        assert r["dot"] == res[0]["dot"]                                   # every rank holds the same sum
    assert sum(r["owned"] for r in res) == res[0]["free"]                  # each free node counted once


def test_partition_rcb_splits_along_the_longest_extent():
    """Two parts of an 8x2x2 box of unit elements: the cut is x = 4 (the longest extent)."""
    from paper_2104_05829_gb300.sem import partition_rcb
    ix, iy, iz = np.meshgrid(np.arange(8), np.arange(2), np.arange(2), indexing="ij")
    cx, cy, cz = (v.ravel() + 0.5 for v in (ix, iy, iz))
    part = partition_rcb(cx, cy, cz, 2)
    assert np.array_equal(part, (cx > 4).astype(np.int32))
    part4 = partition_rcb(cx, cy, cz, 4)
    assert np.array_equal(np.bincount(part4), [8, 8, 8, 8])
    for p in range(4):   # each part is a 2-element-wide slab in x
        xs = np.unique(cx[part4 == p])
        assert xs.size == 2 and xs[1] - xs[0] == 1
