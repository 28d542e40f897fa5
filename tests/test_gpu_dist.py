"""The partitioned operator (Sections 3.1 and 3.2) through libsem's kernels.

Two processes share the one GPU here, each holding one rank's elements; they meet
only in the host-side gloo all-reduce of the interface buffers (no kernel waits on
another rank). Every rank's assembled R QQ^T A_L u must equal the oracle's
whole-mesh result on its points (FP64 to 1e-12, the FP32-pair kernel to its 5e-12),
and the unique-node dot product must equal the oracle's. One rank reproduces
sem_ax bit for bit.
"""
import os
import socket

import numpy as np
import pytest

from gpu_common import H, T, ctx_for, dev, relmax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SHAPE, N = (6, 5, 4), 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _mesh():
    import sem_inputs as si
    return si.box_mesh(SHAPE, N, warp=0.1, perm_seed=3, dirichlet=("x0", "y1"))


def _oracle(mesh):
    import oracle as O
    import sem_inputs as si
    lev = O.level_from_mesh(mesh)
    u = si.uniform_field(mesh, 0) * (1 - mesh["dirichlet"])
    ug = O.q_scatter(u.ravel() / lev.maps["mult"], lev.node, lev.n_G)
    ref = O.q_gather(lev.apply(ug, 1.0, 0.5), lev.node)
    a, b = si.uniform_field(mesh, 4).ravel(), si.uniform_field(mesh, 5).ravel()
    ag, bg = (O.q_scatter(v / lev.maps["mult"], lev.node, lev.n_G) for v in (a, b))
    return u.ravel(), ref, a, b, float(np.sum((ag * bg)[lev.free])), float(np.sum(np.abs(ag * bg)))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2104_05829_gb300.dist import DistContext
        mesh = _mesh()
        u, ref, a, b, dref, scale = _oracle(mesh)
        dc = DistContext(mesh, device="cuda:0", prec_copies=4)
        ul = torch.tensor(dc.local_from_global(u), device="cuda:0")
        refl = dc.local_from_global(ref)
        w = dc.ax(ul, h1=1.0, h2=0.5)
        wp = dc.ax(ul, h1=1.0, h2=0.5, pairs=True)
        d = dc.dot(torch.tensor(dc.local_from_global(a), device="cuda:0"),
                   torch.tensor(dc.local_from_global(b), device="cuda:0"))
        out[rank] = {"err": relmax(H(w), refl), "err_pairs": relmax(H(wp), refl), "dot": d, "dref": dref,
                     "scale": scale, "nb": dc.nb, "E": dc.E, "n_iface": dc.plan["n_iface"]}
        dc.close()
    finally:
        dist.destroy_process_group()


def test_two_ranks_match_the_oracle():
    dev()
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    res = [out[r] for r in range(world)]
    print(res)
    assert sum(r["E"] for r in res) == SHAPE[0] * SHAPE[1] * SHAPE[2]
    for r in res:
        assert 0 < r["nb"] < r["E"] and r["n_iface"] > 0
        assert r["err"] < 1e-12 and r["err_pairs"] < 5e-12, r
        assert abs(r["dot"] - r["dref"]) <= 1e-12 * r["scale"]
    assert res[0]["dot"] == res[1]["dot"]


def test_one_rank_is_sem_ax():
    """Without a process group the partition is the whole mesh: no interface, every element
    interior, and the result is sem_ax's (assembled, masked) bit for bit."""
    dev()
    from paper_2104_05829_gb300.dist import DistContext
    mesh = _mesh()
    u, ref, *_ = _oracle(mesh)
    dc = DistContext(mesh, device="cuda:0", prec_copies=0)
    assert dc.world == 1 and dc.nb == 0 and dc.plan["n_iface"] == 0
    assert np.array_equal(dc.plan["elements"], np.arange(mesh["E"]))
    ut = T(u)
    w = H(dc.ax(ut, h1=1.0, h2=0.5))
    ctx = ctx_for(mesh, prec_copies=0)
    w1 = H(ctx.ax(ut, h1=1.0, h2=0.5, assemble=True))
    assert np.array_equal(w, w1)
    assert relmax(w, ref) < 1e-12
