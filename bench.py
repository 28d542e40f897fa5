"""Benchmark: FP64 matrix-free Ax + gather-scatter throughput (GDOF/s) on the
warped 32^3-element N=7 box, plus the p-multigrid PCG time to a 1e-8 relative
residual on the 24^3-element N=7 pressure problem.

A step is one assembled operator application w_L = R QQ^T A_L u_L (sem_ax with
SEM_AX_ASSEMBLE: the Ax kernel then the gather-scatter+mask kernel) on inputs
resident in HBM. value = unique DOFs (n_G) per second over the timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun every rank runs an independent replica on its own GPU
(the path has no exchange step on one box): value sums the ranks' DOFs over
the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GDOF/s of Ax+gather-scatter and PCG time-to-1e-8 at N=7, vs HBM roofline"
SM_COUNT = 152
FP64_FLOP_PER_CLK_SM = 4          # GB300 nominal 1.25 TFLOP/s FP64 at 2.07 GHz over 152 SMs
SM_MAX_MHZ = 2070.0
FP32_TFLOPS = 72.0                # FFMA microbenchmark on this machine's GB300 (2 flops per FMA)


def ax_flops_per_element(N: int, helmholtz: bool = True) -> int:
    """The paper's count for A^e u^e, 12(N+1)^4 + 15(N+1)^3, plus 2(N+1)^3 for h2 B u."""
    NP = N + 1
    return 12 * NP ** 4 + 15 * NP ** 3 + (2 * NP ** 3 if helmholtz else 0)


def ax_gs_bytes(nL: int, n_shared: int, nG: int, helmholtz: bool = True) -> int:
    """Algorithmic bytes of one FP64 Ax+gs: 6 G (+B) per local point, a 4-byte id per
    non-interior local point, u read and w written once per unique node."""
    return (56 if helmholtz else 48) * nL + 4 * n_shared + 16 * nG


KERNEL_SOURCES = {"k_ax_eo<ArF64,8>": ["ax_eo.cu"], "k_ax_eo<ArPair,8>": ["ax_eo.cu", "pairs.cuh"]}


def kernel_source_hash(kernel: str) -> str:
    """SHA-256 over the sources a kernel is built from, to tell whether recorded ncu counters are current."""
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2104_05829_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, elements: int):
    """DRAM bytes per launch of `kernel` from the ncu capture recorded in profiles/traffic.json,
    scaled to `elements` (traffic grows in proportion to the elements processed); None when no
    capture exists or the kernel source changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(kernel)
    if not rec or rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    return rec["dram_bytes"] * elements / rec["elements"]


def peaks():
    p = {"hbm_gbs": 6686.5, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        p = {"hbm_gbs": d.get("hbm_gbs", 6686.5), "source": "measured"}
    p["fp64_tflops"] = SM_COUNT * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def wait_first(self, timeout=5.0):
        t0 = time.time()
        while self.proc and not self.rows and time.time() - t0 < timeout:
            time.sleep(0.05)

    def mark(self, which):
        setattr(self, which, time.time())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        t0, t1 = getattr(self, "t_start", 0.0), getattr(self, "t_end", 1e30)
        rows = [r for (t, r) in self.rows if t0 <= t <= t1 + 0.2]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ----------------------------------------------------------------------------------
# CPU oracle leg
# ----------------------------------------------------------------------------------
def oracle_ax_gs_rate(mesh, budget_s: float = 12.0):
    """Time the oracle's FP64 local Ax on a growing sample of elements (bounded CPU time)
    and scale to GDOF/s through the unique-DOF share of a local point."""
    import oracle as O

    N, E = mesh["N"], mesh["E"]
    nL = mesh["x"].size
    nG = int(mesh["gid"].max())
    D = O.deriv_matrix(N)
    u = mesh["u"]
    k = 64
    spent, pts, calls = 0.0, 0, 0
    while spent < budget_s and k <= E:
        sl = slice(0, k)
        G, B, _ = O.geometry(mesh["x"][sl], mesh["y"][sl], mesh["z"][sl], N)
        t0 = time.perf_counter()
        w = O.ax_local(u[sl], G, B, D, 1.0, 0.5)
        O.qqt(w, O.gs_maps(mesh["gid"][sl])["node"], int(w.size))
        dt = time.perf_counter() - t0
        spent += dt
        pts += w.size
        calls += 1
        k = min(E, k * 2) if k < E else E + 1
    rate_local = pts / spent
    return {"value": rate_local * nG / nL / 1e9, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle ax_local+qqt (numpy, FP64) on the first 64..{k // 2} elements of the "
                      f"{E}-element box, {calls} calls, {pts} local points in {spent:.1f} s; "
                      f"scaled by n_G/n_L = {nG / nL:.4f}"}


# ----------------------------------------------------------------------------------
def build_mesh(e1: int, N: int):
    import sem_inputs as si

    mesh = si.box_mesh(e1, N, warp=0.1, perm_seed=0)
    mesh["u"] = si.uniform_field(mesh, 0)
    return mesh


def arm_config(elements: int, E: int, nL: int, nG: int, world: int) -> dict:
    """The workload both arms report (the reference arm times the oracle on the same one)."""
    return {"workload": f"FP64 Helmholtz Ax+gs (h1=1, h2=0.5) on a {elements}^3-element warped "
                        f"unit-cube box, N=7, u ~ U[-1,1] continuous (seed 0)",
            "E": E, "N": 7, "n_L": nL, "n_G": nG, "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 ({64 * nL / 1e9:.1f} GB read per step vs 129 MB L2)"}


def run_reference(args, rank):
    if rank != 0:
        return
    mesh = build_mesh(args.elements, 7)
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(oracle_ax_gs_rate(mesh, budget_s=max(2.0, 20.0 / (args.warmup + args.steps))))
    timed = vals[args.warmup:]
    v = statistics.median([t["value"] for t in timed])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.elements, int(mesh["E"]), int(mesh["x"].size), int(mesh["n_lattice"]), args.gpus),
            "cpu_baseline": {**timed[-1], "value": v},
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(t_local: float, units_local: float, dist=None, device="cpu"):
    """Whole-job figures over ranks: the slowest rank's time and the sum of all ranks' units."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return t_local, units_local
    import torch

    dist.barrier()
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def time_events(fn, steps, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def solve_bench(ctx_cls, args, dev):
    """PCG time to ||r||/||b|| <= 1e-8 on the 24^3-element N=7 warped pressure problem."""
    import torch

    import sem_inputs as si

    mesh = si.box_mesh(args.solve_elements, 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    copts = {"coarse_mode": args.coarse_mode}
    if args.coarse_tol is not None:
        copts["coarse_tol"] = args.coarse_tol
    ctxs = {"jacobi": ctx_cls.from_mesh(mesh, **copts)}
    ctx = ctxs["jacobi"]
    b = torch.tensor(si.gaussian_assembled_rhs(mesh, 0).ravel(), device=dev)
    out = {"workload": f"{args.solve_elements}^3 warped box, N=7, x=0 Dirichlet, Gaussian zero-mean RHS, "
                       f"FCG + p-MG (7-3-1, Chebyshev degree 2 with Jacobi or Schwarz (asm_*), "
                       f"coarse Jacobi-PCG) to 1e-8",
           "n_L": int(mesh["x"].size), "n_G": int(ctx.levels[0]["nG"])}
    stream = torch.cuda.current_stream()
    variants = (("fp64", "fp64", False, "jacobi"), ("fp32", "fp32", False, "jacobi"),
                ("bf16g", "bf16g", False, "jacobi"), ("fp32_outer_pairs", "fp32", True, "jacobi"),
                ("bf16g_outer_pairs", "bf16g", True, "jacobi"),
                ("asm_fp64", "fp64", False, "asm"), ("asm_fp32", "fp32", False, "asm"),
                ("asm_fp32_outer_pairs", "fp32", True, "asm"), ("asm_bf16g_outer_pairs", "bf16g", True, "asm"))
    if args.solve_variants:
        keep = set(args.solve_variants.split(","))
        variants = tuple(v for v in variants if v[0] in keep)
    for name, prec, op, sm in variants:
        if sm not in ctxs:
            ctxs[sm] = ctx_cls.from_mesh(mesh, smoother=sm, **copts)
        c = ctxs[sm]
        solve = lambda: c.solve(b, tol=1e-8, maxit=300, precond="pmg", prec=prec, rhs="assembled", outer_pairs=op)
        solve()   # warm-up, includes the preconditioner setup for this precision
        times, info = [], None
        for _ in range(args.solve_reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        t = min(times)
        out[name] = {"time_to_1e-8_s": t, "median_s": statistics.median(times), "iters": info["iters"],
                     "ms_per_iter": 1e3 * t / max(1, info["iters"]), "relres": info["relres"],
                     "coarse_iters": info["coarse_iters"], "graph_steps": info["graph_steps"], "smoother": f"cheby-{'asm' if sm == 'asm' else 'jac'} {prec}",
                     "outer_operator": "f32x2" if op else "f64"}
    if args.jacobi:
        ctx.solve(b, tol=1e-8, maxit=20000, precond="jacobi", rhs="assembled")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, info = ctx.solve(b, tol=1e-8, maxit=20000, precond="jacobi", rhs="assembled")
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out["jacobi_fp64"] = {"time_to_1e-8_s": t, "iters": info["iters"], "ms_per_iter": 1e3 * t / info["iters"],
                              "relres": info["relres"]}
    for c in ctxs.values():
        c.close()
    return out


def proj_bench(ctx_cls, args, dev):
    """Successive right-hand sides f(x, t_k), t_k = 0.02 k (travelling waves), on the
    24^3-element N=7 pressure problem: FCG + p-MG (FP32 smoother) to 1e-8 from x0 = 0
    and from the projected initial guess (Section 3.4, projection-based initial guesses)."""
    import torch

    import sem_inputs as si
    from paper_2104_05829_gb300 import Projection

    mesh = si.box_mesh(args.solve_elements, 7, warp=0.1, perm_seed=0, dirichlet=("x0",))
    ctx = ctx_cls.from_mesh(mesh)
    modes, K, dt, nvec = 12, args.proj_steps, 0.02, 8
    a, om, cm, sm = si.travelling_modes(mesh, 7, modes=modes, kmax=3)
    cm = [torch.tensor(c.ravel(), device=dev) for c in cm]
    sm = [torch.tensor(s.ravel(), device=dev) for s in sm]

    def field(t):
        f = torch.zeros_like(cm[0])
        for m in range(modes):
            f += a[m] * (cm[m] * np.cos(om[m] * t) + sm[m] * np.sin(om[m] * t))
        return f

    fs = [field(dt * k) for k in range(K)]
    del cm, sm
    stream = torch.cuda.current_stream()
    out = {"workload": f"{args.solve_elements}^3 warped box, N=7, x=0 Dirichlet, {K} successive nodal RHS "
                       f"f(x, 0.02k) ({modes} travelling waves), FCG + p-MG (FP32 smoother) to 1e-8",
           "max_vectors": nvec}
    ctx.solve(fs[0], tol=1e-8, maxit=300, precond="pmg", prec="fp32")   # warm-up and preconditioner setup
    for name, proj in (("x0_zero", None), ("projected", Projection(ctx, nvec))):
        times, iters, rel0 = [], [], []
        for f in fs:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = ctx.solve(f, tol=1e-8, maxit=300, precond="pmg", prec="fp32", proj=proj)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(info["iters"])
            rel0.append(info.get("relres0", 1.0))
        out[name] = {"mean_s": float(np.mean(times)), "mean_s_after_3": float(np.mean(times[3:])),
                     "iters": iters, "relres0": rel0, "times_s": times}
        if proj is not None:
            proj.close()
    ctx.close()
    return out


def advect_work_per_element(N: int, ncomp: int = 3):
    """Multiply-adds of the dealiased advection kernel per element (sum-factorised, as
    executed): wind interpolation and contravariant combination once, then per
    component interpolation, three Gauss-point derivatives, the product and the
    transposed interpolation; and the bytes it must move (factors, c, u, w)."""
    NP, NQ = N + 1, (3 * (N + 1) + 1) // 2
    interp = NQ * NP ** 3 + NQ ** 2 * NP ** 2 + NQ ** 3 * NP
    mac = 3 * interp + 9 * NQ ** 3 + ncomp * (2 * interp + 3 * NQ ** 4 + 3 * NQ ** 3)
    words = 9 * NQ ** 3 + (3 + 2 * ncomp) * NP ** 3
    return 2 * mac, words


def advect_bench(ctx, u, nG, E, N, stream, pk, steps=(5, 50)):
    """Dealiased u . grad u (three components) on the Ax box, FP64 and FP32."""
    import torch

    flops_e, words_e = advect_work_per_element(N)
    out = {"workload": f"dealiased advection u . grad u, 3 components, {E} elements N={N}, "
                       f"nq={(3 * (N + 1) + 1) // 2} Gauss points per direction",
           "flops_per_element": flops_e, "words_per_element": words_e}
    for prec, dt, nstep in (("fp64", torch.float64, steps[0]), ("fp32", torch.float32, steps[1])):
        c = torch.stack([u, 0.5 * u, -u]).to(dt).contiguous()
        uu = c.clone()
        w = torch.empty_like(c)
        fn = lambda: ctx.advect(c, uu, w, prec=prec)
        fn()   # builds the cubature factors on the first call
        fn()
        t = time_events(fn, nstep, stream) / nstep
        fl = flops_e * E / t / 1e12
        byt = words_e * E * (8 if prec == "fp64" else 4) / t / 1e9
        peak = pk["fp64_tflops"] if prec == "fp64" else FP32_TFLOPS
        out[prec] = {"ms": 1e3 * t, "GDOF_per_s": 3 * nG / t / 1e9, "tflops": fl, "alu_peak_tflops": peak,
                     "alu_frac": fl / peak, "achieved_gbs": byt, "hbm_frac": byt / pk["hbm_gbs"]}
        # one RK4 substep of the characteristics subproblem (4 operator evaluations, wind linear in time)
        c1 = c.flip(0).contiguous()
        sub = lambda: ctx.char_advance(c, uu, 0.0, 1e-3, 1, c1=c1, prec=prec)
        sub()
        ts = time_events(sub, max(2, nstep // 4), stream) / max(2, nstep // 4)
        out[prec]["char_substep_ms"] = 1e3 * ts
        del c, c1, uu, w
    return out


def sweep_orders(ctx_cls, dev, stream, steps=100):
    """Ax+gs throughput across orders at about 16.8M local points (nearest cube of elements)."""
    import torch

    import sem_inputs as si

    out = []
    for N in (3, 5, 7, 9, 11):
        e1 = si.cube_for_points(N)
        mesh = si.box_mesh(e1, N, warp=0.1, perm_seed=0)
        ctx = ctx_cls.from_mesh(mesh, prec_copies=4, mg_orders=[N])
        lv = ctx.levels[0]
        u = torch.tensor(si.uniform_field(mesh, 0).ravel(), device=dev)
        w = torch.empty_like(u)
        row = {"N": N, "E": lv["E"], "n_L": lv["nL"], "n_G": lv["nG"]}
        for name, pairs in (("fp64", False), ("fp32_pairs", True)):
            fn = lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=True, pairs=pairs)
            for _ in range(3):
                fn()
            t = time_events(fn, steps, stream)
            ta = time_events(lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=False, pairs=pairs), steps, stream)
            row[name] = {"gdofs": lv["nG"] * steps / t / 1e9, "ms_per_step": 1e3 * t / steps,
                         "ax_ms": 1e3 * ta / steps,
                         "ax_tflops_paper_count": ax_flops_per_element(N) * lv["E"] / (ta / steps) / 1e12}
        out.append(row)
        ctx.close()
        del u, w
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--elements", type=int, default=32, help="elements per side of the Ax box")
    ap.add_argument("--solve-elements", type=int, default=24)
    ap.add_argument("--solve-reps", type=int, default=3)
    ap.add_argument("--solve-variants", default="", help="comma list of fp64,fp32,bf16g,fp32_outer_pairs")
    ap.add_argument("--solve-48", action="store_true", help="also time the 48^3-element (56.6M-point) solve")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-proj", action="store_true", help="skip the successive-RHS projection sequence")
    ap.add_argument("--no-advect", action="store_true", help="skip the dealiased advection timing")
    ap.add_argument("--coarse-tol", type=float, default=None, help="coarse Jacobi-PCG tolerance (default 1e-2)")
    ap.add_argument("--coarse-mode", default="auto", choices=["auto", "pipe", "cluster", "grid", "kernels"],
                    help="execution of the coarse Jacobi-PCG (same algorithm)")
    ap.add_argument("--proj-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--jacobi", action="store_true", help="also time Jacobi-PCG on the solve problem")
    ap.add_argument("--ax", default="fp64", choices=["fp64", "pairs"],
                    help="element kernel of the timed step: FP64 instructions or FP32-pair arithmetic")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="also measure Ax+gs for N in 3,5,7,9,11 at about 16.8M local points")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2104_05829_gb300 import SemContext

    mesh = build_mesh(args.elements, 7)
    ctx = SemContext.from_mesh(mesh, prec_copies=4, mg_orders=[7])
    lv = ctx.levels[0]
    nL, nG, n_shared, E = lv["nL"], lv["nG"], lv["n_seg_idx"], lv["E"]
    u = torch.tensor(mesh["u"].ravel(), device=dev)
    w = torch.empty_like(u)
    stream = torch.cuda.current_stream()

    pairs = args.ax == "pairs"
    step = lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=True, pairs=pairs)
    with ClockSampler(local) as clk:
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        clk.wait_first()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark("t_start")
        t = time_events(step, args.steps, stream)
        # dominant kernel alone: the local Ax launch, same stream, same inputs
        t_ax = time_events(lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=False, pairs=pairs), args.steps, stream)
        clk.mark("t_end")
    torch.cuda.synchronize()
    t, units = aggregate(t, nG * args.steps, dist, dev)
    ms = 1e3 * t / args.steps
    value = units / t / 1e9

    pk = peaks()
    flops = ax_flops_per_element(7) * E
    t_ax_launch = t_ax / args.steps
    achieved_tf = flops / t_ax_launch / 1e12
    bytes_alg = ax_gs_bytes(nL, n_shared, nG)
    kname = "k_ax_eo<ArPair,8>" if pairs else "k_ax_eo<ArF64,8>"
    roof = {"bound": "alu", "achieved": achieved_tf, "peak": pk["fp64_tflops"], "unit": "TFLOP/s",
            "frac": achieved_tf / pk["fp64_tflops"], "traffic": recorded_traffic(kname, E),
            "kernel": kname + (" (FP32-pair local Ax)" if pairs else " (FP64 local Ax, even-odd)"),
            "peak_source": "derived: 152 SMs x 4 FP64 FLOP/clk x 2070 MHz (nominal 1.25 TFLOP/s)",
            "hbm_view": {"bytes_per_step": bytes_alg, "achieved_gbs": bytes_alg / (ms / 1e3) / 1e9,
                         "peak_gbs": pk["hbm_gbs"], "frac": bytes_alg / (ms / 1e3) / 1e9 / pk["hbm_gbs"],
                         "peak_source": pk["source"]}}

    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2" if pairs else "f64", "data": "synthetic",
            "config": arm_config(args.elements, E, nL, nG, world),
            "roofline": roof, "gpu_launches": 2 * args.steps,
            "clocks": clk.summary()}

    if not args.no_e2e:
        # End to end through the public API, as a server would run a stream of requests:
        # every step copies its own input from pinned host memory, runs Ax+gs and copies
        # its result back to pinned host memory. Steps are pipelined over three streams
        # with two device buffer pairs, so step k+1's input copy and step k-1's output
        # copy (separate copy engines) overlap step k's kernels.
        uh = torch.tensor(mesh["u"].ravel()).pin_memory()
        ub = [u, torch.empty_like(u)]
        wb = [w, torch.empty_like(w)]
        whb = [torch.empty_like(uh).pin_memory() for _ in range(2)]
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_run(k_steps):
            for s_ in (s_in, s_cmp, s_out):
                s_.wait_stream(stream)
            for k in range(k_steps):
                b = k & 1
                s_in.wait_event(ev_cmp[b])        # step k-2 no longer reads ub[b]
                with torch.cuda.stream(s_in):
                    ub[b].copy_(uh, non_blocking=True)
                ev_in[b].record(s_in)
                s_cmp.wait_event(ev_in[b])
                s_cmp.wait_event(ev_out[b])       # step k-2's result has left wb[b]
                ctx.ax(ub[b], wb[b], h1=1.0, h2=0.5, assemble=True, pairs=pairs, stream=s_cmp)
                ev_cmp[b].record(s_cmp)
                s_out.wait_event(ev_cmp[b])
                with torch.cuda.stream(s_out):
                    whb[b].copy_(wb[b], non_blocking=True)
                ev_out[b].record(s_out)
            stream.wait_stream(s_out)

        for ev in ev_in + ev_cmp + ev_out:
            ev.record(stream)
        e2e_run(3)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_run(args.steps)
        e1.record(stream)
        e1.synchronize()
        te = e0.elapsed_time(e1) / 1e3
        ok = bool(torch.equal(whb[(args.steps - 1) & 1], w.cpu())) if args.steps > 0 else True
        line["e2e"] = {"value": world * nG * args.steps / te / 1e9, "unit": "GDOF/s",
                       "h2d_bytes_per_step": 8 * nL, "d2h_bytes_per_step": 8 * nL, "ms_per_step": 1e3 * te / args.steps,
                       "pipelined": "3 streams, 2 buffer pairs", "result_check": ok}
    if not args.no_variants:
        # the other element kernel on the same inputs (reported, not the headline)
        other = not pairs
        fn = lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=True, pairs=other)
        for _ in range(3):
            fn()
        tv = time_events(fn, args.steps, stream)
        tva = time_events(lambda: ctx.ax(u, w, h1=1.0, h2=0.5, assemble=False, pairs=other), args.steps, stream)
        line["variants"] = {("ax_fp32_pairs" if other else "ax_fp64"): {
            "value": world * nG * args.steps / tv / 1e9, "unit": "GDOF/s", "ms_per_step": 1e3 * tv / args.steps,
            "ax_kernel_ms": 1e3 * tva / args.steps, "dtype": "f32x2" if other else "f64",
            "ax_kernel_tflops_paper_count": flops / (tva / args.steps) / 1e12}}
    if not args.no_advect:
        line["advection"] = advect_bench(ctx, u, nG, E, 7, stream, pk)
    ctx.close()
    if args.sweep:
        line["sweep"] = sweep_orders(SemContext, dev, stream)
    if not args.no_solve:
        line["solve"] = solve_bench(SemContext, args, dev)
    if not args.no_solve and not args.no_proj:
        line["solve_proj"] = proj_bench(SemContext, args, dev)
    if args.solve_48:
        import copy
        a48 = copy.copy(args)
        a48.solve_elements, a48.solve_reps = 48, 1
        line["solve_48"] = solve_bench(SemContext, a48, dev)
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = oracle_ax_gs_rate(mesh)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
