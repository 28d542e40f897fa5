"""Element partitioning across GPUs and the interface exchange (Sections 3.1 and 3.2).

One process per GPU. Every rank holds the same global mesh description, splits the
elements by recursive coordinate bisection of their centroids (sem_partition_rcb)
and builds a libsem context from its own elements, keeping their global node ids.
The gather-scatter QQ^T of the whole mesh is then each rank's own QQ^T plus, at the
interface nodes (ids held by more than one rank), the other ranks' partial sums.

Exchange: one all-reduce (sum) over a buffer with one slot per interface node of the
whole mesh. A rank writes the partial sums of the interface nodes it holds into its
slots (zero elsewhere, sem_halo_gather); after the all-reduce every slot holds the
node's full sum, which sem_halo_scatter writes to every local copy. The slots'
order is the ascending global id, the same on every rank, and the all-reduce returns
the same bits to every rank, so the copies of a node agree across ranks. (gslib,
which NekRS uses, chooses at setup between pairwise exchanges, a crystal router and
this all-reduce; at a handful of GPUs the interface buffer is small and the all-
reduce is one collective.)

Overlap (the nonlocal-first ordering of Section 3.2): a rank stores the elements
that touch the interface first. It applies the element operator to them, gathers
the interface partial sums, starts the all-reduce, applies the operator to its other
elements and runs its own gather-scatter, then waits for the exchange and writes the
interface sums.

Dot products over unique nodes count each non-Dirichlet node once over all ranks:
the rank of lowest index that holds a node counts its first local copy.

Every arithmetic step runs in libsem's kernels; this module plans the partition on
the host and moves buffers through torch.distributed.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L
from .sem import Halo, SemContext, partition_rcb


def element_centroids(mesh: dict):
    """Mean of each element's nodal coordinates (x, y, z shaped [E, ...])."""
    E = int(mesh["E"])
    return tuple(np.asarray(mesh[c], dtype=np.float64).reshape(E, -1).mean(axis=1) for c in ("x", "y", "z"))


def partition(mesh: dict, nparts: int) -> np.ndarray:
    """Rank of every element: recursive coordinate bisection of the element centroids."""
    cx, cy, cz = element_centroids(mesh)
    return partition_rcb(cx, cy, cz, nparts)


def plan(mesh: dict, part: np.ndarray, rank: int) -> dict:
    """Host-side plan of one rank: its elements in storage order (interface-touching first),
    its local mesh arrays, the interface of the whole mesh and this rank's share of it,
    and the owner flags of its local points for dot products."""
    E = int(mesh["E"])
    gid = np.asarray(mesh["gid"], dtype=np.int64).reshape(E, -1)
    npe = gid.shape[1]
    part = np.asarray(part, dtype=np.int64)
    # interface ids: nonzero ids that occur in elements of at least two ranks
    g = gid.ravel()
    r = np.repeat(part, npe)
    keep = g > 0
    pairs = np.unique(np.stack([g[keep], r[keep]], axis=1), axis=0)     # unique (id, rank), sorted by id
    ids, first, counts = np.unique(pairs[:, 0], return_index=True, return_counts=True)
    iface = ids[counts > 1]
    owner_rank = pairs[first[counts > 1], 1]                           # the smallest rank holding the id
    mine = np.nonzero(part == rank)[0]
    on_iface = np.isin(gid[mine], iface).any(axis=1)
    order = np.concatenate([mine[on_iface], mine[~on_iface]])
    nb = int(on_iface.sum())
    lg = gid[order].ravel()
    my_iface = np.intersect1d(iface, lg)                                 # ascending
    pos = np.searchsorted(iface, my_iface)
    # owner flags: first local copy of each node, not Dirichlet, and this rank the lowest holder
    dirichlet = mesh.get("dirichlet")
    dl = (np.zeros(lg.size, np.uint8) if dirichlet is None
          else np.asarray(dirichlet, dtype=np.uint8).reshape(E, -1)[order].ravel())
    first_copy = np.ones(lg.size, dtype=bool)
    nz = np.nonzero(lg > 0)[0]
    _, firsts = np.unique(lg[nz], return_index=True)
    first_copy[nz] = False
    first_copy[nz[firsts]] = True
    lowest = np.ones(lg.size, dtype=bool)
    at_iface = np.isin(lg, iface)
    lowest[at_iface] = owner_rank[np.searchsorted(iface, lg[at_iface])] == rank
    owner = (first_copy & (dl == 0) & lowest).astype(np.uint8)
    local = {"E": int(order.size), "N": int(mesh["N"]),
             "x": np.asarray(mesh["x"]).reshape(E, -1)[order].reshape((order.size,) + np.shape(mesh["x"])[1:]),
             "y": np.asarray(mesh["y"]).reshape(E, -1)[order].reshape((order.size,) + np.shape(mesh["y"])[1:]),
             "z": np.asarray(mesh["z"]).reshape(E, -1)[order].reshape((order.size,) + np.shape(mesh["z"])[1:]),
             "gid": lg, "dirichlet": None if dirichlet is None else dl}
    return {"elements": order, "nb": nb, "local": local, "iface": iface, "iface_gid": my_iface, "iface_pos": pos,
            "n_iface": int(iface.size), "owner": owner}


def exchange(buf: torch.Tensor, group=None, async_op: bool = False):
    """Sum of the ranks' interface buffers (the collective of the gather-scatter)."""
    import torch.distributed as dist

    return dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group, async_op=async_op)


class DistContext:
    """One rank's share of a mesh partitioned across GPUs: Ax+gs and unique-node dot
    products of the whole mesh on this rank's elements (see the module notes)."""

    def __init__(self, mesh: dict, group=None, device=None, **opts):
        import torch.distributed as dist

        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.part = partition(mesh, self.world)
        self.plan = plan(mesh, self.part, self.rank)
        loc = self.plan["local"]
        self.ctx = SemContext(loc["x"], loc["y"], loc["z"], loc["gid"], loc["dirichlet"], loc["N"], **opts)
        self.E, self.nb, self.nL = loc["E"], self.plan["nb"], self.ctx.nL
        self.halo = Halo(self.ctx, self.plan["iface_gid"], self.plan["iface_pos"], self.plan["n_iface"])
        self.buf = torch.zeros(max(1, self.plan["n_iface"]), dtype=torch.float64, device=self.device)
        self.owner = torch.tensor(self.plan["owner"], dtype=torch.uint8, device=self.device)
        self._lib = L.load()

    def close(self):
        self.halo.close()
        self.ctx.close()

    def ax(self, u, w=None, h1=1.0, h2=0.0, mask=True, pairs=False, stream=None):
        """w = (R) QQ^T A_L u over the whole mesh, on this rank's local points."""
        w = torch.empty_like(u) if w is None else w
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.ctx.ax_elements(0, self.nb, u, w, h1=h1, h2=h2, pairs=pairs, stream=s)
            self.halo.gather(w, self.buf, stream=s)
            work = exchange(self.buf, self.group, async_op=True) if self.world > 1 else None
            self.ctx.ax_elements(self.nb, self.E, u, w, h1=h1, h2=h2, pairs=pairs, stream=s)
            self.ctx.gs(w, mask=mask, stream=s)
            if work is not None:
                work.wait()
            self.halo.scatter(self.buf, w, mask=mask, stream=s)
        return w

    def dot(self, a, b, stream=None) -> float:
        """(a, b) over the unique non-Dirichlet nodes of the whole mesh (continuous vectors)."""
        s = torch.cuda.current_stream() if stream is None else stream
        out = torch.empty(1, dtype=torch.float64, device=self.device)
        L.check(self._lib.sem_dot_static(a.data_ptr(), b.data_ptr(), self.owner.data_ptr(), C.c_int64(self.nL),
                                         out.data_ptr(), s.cuda_stream), "sem_dot_static")
        with torch.cuda.stream(s):
            if self.world > 1:
                exchange(out, self.group)
        return out.item()

    def local_from_global(self, v: np.ndarray) -> np.ndarray:
        """This rank's entries of a global L-vector (elements in this rank's storage order)."""
        E = int(self.part.size)
        return np.asarray(v).reshape(E, -1)[self.plan["elements"]].ravel()
