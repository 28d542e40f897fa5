"""Python binding of libsem: argument marshalling over torch CUDA tensors.

Every computation runs in libsem's CUDA kernels; this module only checks
tensors, passes device pointers and the current torch stream, and converts the
read-back products to numpy. Names follow the C ABI (include/sem.h).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

_PREC = {"fp64": L.SEM_FP64, "fp32": L.SEM_FP32, "bf16g": L.SEM_BF16G, "fp64p": L.SEM_FP64P,
         L.SEM_FP64: L.SEM_FP64, L.SEM_FP32: L.SEM_FP32, L.SEM_BF16G: L.SEM_BF16G, L.SEM_FP64P: L.SEM_FP64P}
_F64 = (L.SEM_FP64, L.SEM_FP64P)
_PC = {"jacobi": L.SEM_PC_JACOBI, "pmg": L.SEM_PC_PMG}


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, n: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t.data_ptr()


def _host(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def default_opts(**kw) -> L.SemOpts:
    lib = L.load()
    o = L.SemOpts()
    lib.sem_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "mg_orders":
            o.mg_nlevels = len(v)
            for i, n in enumerate(v):
                o.mg_orders[i] = int(n)
        elif k == "smoother":
            o.smoother = {"jacobi": L.SEM_SMOOTH_JACOBI, "asm": L.SEM_SMOOTH_ASM}.get(v, v)
        elif k == "coarse_mode":
            o.coarse_mode = {"auto": L.SEM_COARSE_AUTO, "kernels": L.SEM_COARSE_KERNELS,
                             "pipe": L.SEM_COARSE_PIPE}.get(v, v)
        elif not hasattr(o, k):
            raise KeyError(k)
        else:
            setattr(o, k, v)
    return o


class SemContext:
    """A libsem context: geometry, gather-scatter maps and multigrid levels of one mesh."""

    def __init__(self, x, y, z, gid, dirichlet=None, N: int | None = None, **opts):
        self._lib = L.load()
        x = _host(x, np.float64)
        E = x.shape[0]
        if N is None:
            N = round(x[0].size ** (1 / 3)) - 1
        self.E, self.N = int(E), int(N)
        self.nL = self.E * (self.N + 1) ** 3
        self._keep = [x, _host(y, np.float64), _host(z, np.float64), _host(gid, np.int64)]
        dptr = None
        if dirichlet is not None:
            d = _host(dirichlet, np.uint8)
            self._keep.append(d)
            dptr = d.ctypes.data
        for a in self._keep[:4]:
            if a.size != self.nL:
                raise ValueError("mesh arrays must hold E*(N+1)^3 values")
        m = L.SemMesh(self.E, self.N, self._keep[0].ctypes.data, self._keep[1].ctypes.data,
                      self._keep[2].ctypes.data, self._keep[3].ctypes.data, dptr)
        o = default_opts(**opts)
        h = C.c_void_p()
        L.check(self._lib.sem_setup(C.byref(m), C.byref(o), C.byref(h)), "sem_setup")
        self._h = h
        self._keep = None
        self.levels = [self.level_info(l) for l in range(self._lib.sem_num_levels(h))]

    @classmethod
    def from_mesh(cls, mesh: dict, **opts):
        return cls(mesh["x"], mesh["y"], mesh["z"], mesh["gid"], mesh.get("dirichlet"), mesh["N"], **opts)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sem_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes -------------------------------------------------------------------
    def level_info(self, level: int) -> dict:
        d = L.SemLevelDesc()
        L.check(self._lib.sem_level_info(self._h, level, C.byref(d)), "sem_level_info")
        return {k: getattr(d, k) for k, _ in d._fields_}

    def nl(self, level=0):
        if not 0 <= level < len(self.levels):
            return self.level_info(level)["nL"]      # raises SemError (SEM_EINVAL) from the library
        return self.levels[level]["nL"]

    def empty(self, level=0, prec="fp64", device="cuda"):
        dt = torch.float64 if _PREC[prec] in _F64 else torch.float32
        return torch.empty(self.nl(level), dtype=dt, device=device)

    def zeros(self, level=0, prec="fp64", device="cuda"):
        return self.empty(level, prec, device).zero_()

    # ---- fine-level FP64 operators ---------------------------------------------
    def ax(self, u, w=None, h1=1.0, h2=0.0, h1_L=None, assemble=True, pairs=False, stream=None):
        n = self.nL
        if w is None:
            w = torch.empty_like(u)
        c = L.SemCoef(float(h1), float(h2), _dev(h1_L, torch.float64, n, "h1_L") if h1_L is not None else None)
        flags = (L.SEM_AX_ASSEMBLE if assemble else L.SEM_AX_LOCAL) | (L.SEM_AX_PAIRS if pairs else 0)
        L.check(self._lib.sem_ax(self._h, _dev(u, torch.float64, n, "u"), _dev(w, torch.float64, n, "w"),
                                 C.byref(c), flags, _stream(stream)), "sem_ax")
        return w

    def ax_elements(self, e0, e1, u, w, h1=1.0, h2=0.0, h1_L=None, pairs=False, stream=None):
        """w_L = A_L u_L on elements e0 .. e1-1 only (sem_ax_elements); other entries untouched."""
        n = self.nL
        c = L.SemCoef(float(h1), float(h2), _dev(h1_L, torch.float64, n, "h1_L") if h1_L is not None else None)
        L.check(self._lib.sem_ax_elements(self._h, int(e0), int(e1), _dev(u, torch.float64, n, "u"),
                                          _dev(w, torch.float64, n, "w"), C.byref(c),
                                          L.SEM_AX_PAIRS if pairs else 0, _stream(stream)), "sem_ax_elements")
        return w

    def gs(self, w, mask=False, stream=None):
        L.check(self._lib.sem_gs(self._h, _dev(w, torch.float64, self.nL, "w"),
                                 L.SEM_GS_ADD_MASK if mask else L.SEM_GS_ADD, _stream(stream)), "sem_gs")
        return w

    def rhs(self, f, b=None, stream=None):
        b = torch.empty_like(f) if b is None else b
        L.check(self._lib.sem_rhs(self._h, _dev(f, torch.float64, self.nL, "f"),
                                  _dev(b, torch.float64, self.nL, "b"), _stream(stream)), "sem_rhs")
        return b

    def mass_local(self, f, out=None, stream=None):
        out = torch.empty_like(f) if out is None else out
        L.check(self._lib.sem_mass_local(self._h, _dev(f, torch.float64, self.nL, "f"),
                                         _dev(out, torch.float64, self.nL, "out"), _stream(stream)), "sem_mass_local")
        return out

    def dot(self, a, b, stream=None) -> float:
        out = C.c_double()
        L.check(self._lib.sem_dot(self._h, _dev(a, torch.float64, self.nL, "a"), _dev(b, torch.float64, self.nL, "b"),
                                  C.byref(out), _stream(stream)), "sem_dot")
        return out.value

    def grad_h1(self, u, lam, g=None, sum_copies=False, stream=None):
        g = torch.empty_like(u) if g is None else g
        L.check(self._lib.sem_grad_h1(self._h, _dev(u, torch.float64, self.nL, "u"),
                                      _dev(lam, torch.float64, self.nL, "lam"), _dev(g, torch.float64, self.nL, "g"),
                                      L.SEM_GRAD_SUM if sum_copies else 0, _stream(stream)), "sem_grad_h1")
        return g

    # ---- level operators -------------------------------------------------------
    def _vec(self, t, level, prec, name):
        dt = torch.float64 if _PREC[prec] in _F64 else torch.float32
        return _dev(t, dt, self.nl(level), name)

    def level_ax(self, level, u, w=None, h1=1.0, h2=0.0, prec="fp64", assemble=True, stream=None):
        w = torch.empty_like(u) if w is None else w
        L.check(self._lib.sem_level_ax(self._h, level, _PREC[prec], self._vec(u, level, prec, "u"),
                                       self._vec(w, level, prec, "w"), float(h1), float(h2),
                                       L.SEM_AX_ASSEMBLE if assemble else L.SEM_AX_LOCAL, _stream(stream)),
                "sem_level_ax")
        return w

    def level_gs(self, level, w, prec="fp64", mask=False, stream=None):
        L.check(self._lib.sem_level_gs(self._h, level, _PREC[prec], self._vec(w, level, prec, "w"),
                                       L.SEM_GS_ADD_MASK if mask else L.SEM_GS_ADD, _stream(stream)), "sem_level_gs")
        return w

    def level_dinv(self, level, h1=1.0, h2=0.0, stream=None):
        d = self.empty(level)
        L.check(self._lib.sem_level_dinv(self._h, level, float(h1), float(h2), d.data_ptr(), _stream(stream)),
                "sem_level_dinv")
        return d

    def prolong_add(self, level, ec, xf, prec="fp64", stream=None):
        L.check(self._lib.sem_prolong_add(self._h, level, _PREC[prec], self._vec(ec, level + 1, prec, "ec"),
                                          self._vec(xf, level, prec, "xf"), _stream(stream)), "sem_prolong_add")
        return xf

    def restrict(self, level, rf, rc=None, prec="fp64", stream=None):
        rc = self.empty(level + 1, prec, rf.device) if rc is None else rc
        L.check(self._lib.sem_restrict(self._h, level, _PREC[prec], self._vec(rf, level, prec, "rf"),
                                       self._vec(rc, level + 1, prec, "rc"), _stream(stream)), "sem_restrict")
        return rc

    def precond_setup(self, h1=1.0, h2=0.0, prec="fp64", h1_L=None, stream=None):
        """sem_precond_setup, or sem_precond_setup_nodal with a nodal h1_L (fine-level tensor)."""
        if h1_L is None:
            L.check(self._lib.sem_precond_setup(self._h, float(h1), float(h2), _PREC[prec], _stream(stream)),
                    "sem_precond_setup")
        else:
            L.check(self._lib.sem_precond_setup_nodal(self._h, _dev(h1_L, torch.float64, self.nL, "h1_L"), float(h2),
                                                      _PREC[prec], _stream(stream)), "sem_precond_setup_nodal")
        self._pc_prec = prec

    def cheb_smooth(self, level, b, x, x_is_zero=False, stream=None):
        prec = getattr(self, "_pc_prec", "fp64")
        L.check(self._lib.sem_cheb_smooth(self._h, level, self._vec(b, level, prec, "b"),
                                          self._vec(x, level, prec, "x"), 1 if x_is_zero else 0, _stream(stream)),
                "sem_cheb_smooth")
        return x

    def asm_apply(self, level, r, z=None, h1=1.0, h2=0.0, prec="fp64", stream=None):
        """Weighted overlapping Schwarz z = W sum_e P_e^T F_e P_e r on `level` (sem_asm_apply)."""
        z = torch.empty_like(r) if z is None else z
        L.check(self._lib.sem_asm_apply(self._h, level, _PREC[prec], self._vec(r, level, prec, "r"),
                                        self._vec(z, level, prec, "z"), float(h1), float(h2), _stream(stream)),
                "sem_asm_apply")
        return z

    def advect(self, c, u, w=None, assemble=False, prec="fp64", stream=None):
        """Dealiased advection w = C(c) u (sem_advect). c: (3, nL) tensor; u: (ncomp, nL) or (nL,)."""
        dt = torch.float64 if _PREC[prec] in _F64 else torch.float32
        squeeze = u.dim() == 1
        u2 = u.reshape(-1, self.nL)
        w = torch.empty_like(u2) if w is None else w.reshape(-1, self.nL)
        ncomp = u2.shape[0]
        L.check(self._lib.sem_advect(self._h, _PREC[prec], _dev(c, dt, 3 * self.nL, "c"),
                                     _dev(u2, dt, ncomp * self.nL, "u"), _dev(w, dt, ncomp * self.nL, "w"), ncomp,
                                     L.SEM_ADV_ASSEMBLE if assemble else L.SEM_ADV_LOCAL, _stream(stream)),
                "sem_advect")
        return w.reshape(-1) if squeeze else w

    def char_advance(self, c0, w, t0, t1, nsub, c1=None, prec="fp64", stream=None):
        """RK4 substeps of w_t + c . grad w = 0 on [t0, t1] in place (sem_char_advance).
        c0, c1: (3, nL) winds at t0 and t1 (c1 None: frozen); w: (ncomp, nL) or (nL,)."""
        dt = torch.float64 if _PREC[prec] in _F64 else torch.float32
        w2 = w.reshape(-1, self.nL)
        ncomp = w2.shape[0]
        L.check(self._lib.sem_char_advance(self._h, _PREC[prec], _dev(c0, dt, 3 * self.nL, "c0"),
                                           _dev(c1, dt, 3 * self.nL, "c1") if c1 is not None else None,
                                           _dev(w2, dt, ncomp * self.nL, "w"), ncomp, float(t0), float(t1),
                                           int(nsub), _stream(stream)), "sem_char_advance")
        return w

    def vcycle(self, r, z=None, stream=None):
        z = torch.empty_like(r) if z is None else z
        L.check(self._lib.sem_vcycle(self._h, _dev(r, torch.float64, self.nL, "r"),
                                     _dev(z, torch.float64, self.nL, "z"), _stream(stream)), "sem_vcycle")
        return z

    def lmax(self):
        out = (C.c_double * L.SEM_MAX_LEVELS)()
        L.check(self._lib.sem_get_lmax(self._h, out, L.SEM_MAX_LEVELS), "sem_get_lmax")
        return [out[i] for i in range(len(self.levels) - 1)]

    # ---- solve -----------------------------------------------------------------
    def solve(self, f, h1=1.0, h2=0.0, h1_L=None, tol=1e-8, maxit=1000, precond="jacobi", prec="fp64",
              rhs="nodal", x0=None, u=None, outer_pairs=False, stream=None, raise_on_error=True, proj=None):
        """sem_solve, or sem_solve_proj when a Projection space `proj` is given."""
        n = self.nL
        if u is None:
            u = torch.empty_like(f) if x0 is None else x0.clone()
        elif x0 is not None:
            u.copy_(x0)
        flags = (L.SEM_RHS_ASSEMBLED if rhs == "assembled" else L.SEM_RHS_NODAL) | (L.SEM_X0_GIVEN if x0 is not None else 0)
        flags |= L.SEM_OUTER_PAIRS if outer_pairs else 0
        c = L.SemCoef(float(h1), float(h2), _dev(h1_L, torch.float64, n, "h1_L") if h1_L is not None else None)
        info = L.SemInfo()
        args = (_dev(f, torch.float64, n, "f"), C.byref(c), float(tol), int(maxit), _PC[precond], _PREC[prec], flags,
                _dev(u, torch.float64, n, "u"), C.byref(info), _stream(stream))
        if proj is None:
            rc = self._lib.sem_solve(self._h, *args)
        else:
            rc = self._lib.sem_solve_proj(self._h, proj._h, *args)
        out = {"iters": info.iters, "relres": info.relres, "bnorm": info.bnorm, "coarse_iters": info.coarse_iters,
               "lmax": [info.lmax[i] for i in range(max(0, info.nlevels - 1))], "status": rc,
               "graph_steps": info.graph_steps}
        if proj is not None:
            out["relres0"] = info.relres0
            out["proj_count"] = info.proj_count
        if raise_on_error:
            L.check(rc, "sem_solve_proj" if proj is not None else "sem_solve")
        return u, out

    # ---- read-back -------------------------------------------------------------
    def maps(self, level=0) -> dict:
        d = self.levels[level]
        ids = np.empty(d["n_ids"], np.int64)
        off = np.empty(d["n_ids"] + 1, np.int64)
        idx = np.empty(d["n_idx"], np.int32)
        mult = np.empty(d["nL"], np.int32)
        node = np.empty(d["nL"], np.int64)
        label = np.empty(d["nL"], np.int64)
        dmask = np.empty(d["nL"], np.uint8)
        ptr = lambda a: a.ctypes.data if a.size else None
        L.check(self._lib.sem_get_maps(self._h, level, ptr(ids), ptr(off), ptr(idx), ptr(mult), ptr(node),
                                       ptr(label), ptr(dmask)), "sem_get_maps")
        return {"ids": ids, "off": off, "idx": idx, "mult": mult, "node": node, "label": label, "dmask": dmask,
                "n_G": d["nG"]}

    def geom(self, level=0) -> np.ndarray:
        d = self.levels[level]
        G = np.empty((d["E"], 7, (d["N"] + 1) ** 3), np.float64)
        L.check(self._lib.sem_get_geom(self._h, level, G.ctypes.data), "sem_get_geom")
        return G

    def geom_lowp(self, level=0, prec="bf16g") -> np.ndarray:
        d = self.levels[level]
        dt = np.uint16 if _PREC[prec] == L.SEM_BF16G else np.uint32
        G = np.empty((d["E"], 7, (d["N"] + 1) ** 3), dt)
        L.check(self._lib.sem_get_geom_lowp(self._h, level, _PREC[prec], G.ctypes.data), "sem_get_geom_lowp")
        return G

    def coords(self, level=0):
        d = self.levels[level]
        out = [np.empty(d["nL"], np.float64) for _ in range(3)] + [np.empty(d["nL"], np.int64)]
        L.check(self._lib.sem_get_coords(self._h, level, *[a.ctypes.data for a in out]), "sem_get_coords")
        return out


class Projection:
    """A projection space of earlier solutions (sem_proj_*): A-orthonormal
    directions x_i with A x_i beside them, used by SemContext.solve(proj=...)."""

    def __init__(self, ctx: SemContext, max_vectors: int = 8):
        self._lib = L.load()
        self.ctx = ctx
        h = C.c_void_p()
        L.check(self._lib.sem_proj_create(ctx._h, int(max_vectors), C.byref(h)), "sem_proj_create")
        self._h = h
        self.max_vectors = int(max_vectors)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sem_proj_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        L.check(self._lib.sem_proj_reset(self._h), "sem_proj_reset")

    def __len__(self) -> int:
        n = self._lib.sem_proj_count(self._h)
        if n < 0:
            L.check(n, "sem_proj_count")
        return n

    def vectors(self, i: int):
        """(x_i, A x_i) copied into new CUDA tensors (read-back for validation)."""
        px, pa = C.c_void_p(), C.c_void_p()
        L.check(self._lib.sem_proj_vectors(self._h, int(i), C.byref(px), C.byref(pa)), "sem_proj_vectors")
        n = self.ctx.nL
        return (torch.as_tensor(_DeviceView(px.value, n), device="cuda").clone(),
                torch.as_tensor(_DeviceView(pa.value, n), device="cuda").clone())

    def project(self, b, xbar=None, r0=None, stream=None):
        n = self.ctx.nL
        xbar = torch.empty_like(b) if xbar is None else xbar
        r0 = torch.empty_like(b) if r0 is None else r0
        L.check(self._lib.sem_proj_project(self._h, _dev(b, torch.float64, n, "b"), _dev(xbar, torch.float64, n, "xbar"),
                                           _dev(r0, torch.float64, n, "r0"), _stream(stream)), "sem_proj_project")
        return xbar, r0

    def update(self, dx, x=None, h1=1.0, h2=0.0, outer_pairs=False, stream=None) -> bool:
        n = self.ctx.nL
        c = L.SemCoef(float(h1), float(h2), None)
        added = C.c_int(0)
        L.check(self._lib.sem_proj_update(self._h, C.byref(c), L.SEM_OUTER_PAIRS if outer_pairs else 0,
                                          _dev(x, torch.float64, n, "x") if x is not None else None,
                                          _dev(dx, torch.float64, n, "dx"), C.byref(added), _stream(stream)),
                "sem_proj_update")
        return bool(added.value)


class Halo:
    """Interface nodes of this rank (sem_halo_*): gather its partial sums into an exchange
    buffer at given positions, and write completed sums back to every local copy."""

    def __init__(self, ctx: SemContext, gid, pos, nbuf: int):
        self._lib = L.load()
        self.ctx = ctx
        gid = _host(gid, np.int64)
        pos = _host(pos, np.int64)
        if gid.size != pos.size:
            raise ValueError("gid and pos must have the same length")
        h = C.c_void_p()
        L.check(self._lib.sem_halo_create(ctx._h, gid.size, gid.ctypes.data if gid.size else None,
                                          pos.ctypes.data if pos.size else None, int(nbuf), C.byref(h)),
                "sem_halo_create")
        self._h = h
        self.n, self.nbuf = int(gid.size), int(nbuf)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sem_halo_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _buf(self, buf):
        if buf.numel() < self.nbuf:
            raise ValueError(f"the exchange buffer needs {self.nbuf} values")
        return _dev(buf, torch.float64, buf.numel(), "buf")

    def gather(self, w, buf, stream=None):
        L.check(self._lib.sem_halo_gather(self._h, _dev(w, torch.float64, self.ctx.nL, "w"), self._buf(buf),
                                          _stream(stream)), "sem_halo_gather")
        return buf

    def scatter(self, buf, w, mask=True, stream=None):
        L.check(self._lib.sem_halo_scatter(self._h, self._buf(buf),
                                           _dev(w, torch.float64, self.ctx.nL, "w"),
                                           L.SEM_GS_ADD_MASK if mask else L.SEM_GS_ADD, _stream(stream)),
                "sem_halo_scatter")
        return w


def partition_rcb(cx, cy, cz, nparts: int) -> np.ndarray:
    """Recursive coordinate bisection of element centroids into nparts parts (sem_partition_rcb)."""
    lib = L.load()
    cx, cy, cz = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (cx, cy, cz))
    part = np.empty(cx.size, np.int32)
    L.check(lib.sem_partition_rcb(cx.size, cx.ctypes.data, cy.ctypes.data, cz.ctypes.data, int(nparts),
                                  part.ctypes.data), "sem_partition_rcb")
    return part


class _DeviceView:
    """View of n doubles at a library-owned device address (CUDA array interface); callers
    only copy from it (torch does not accept the interface's read-only flag)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 2,
                                         "strides": None}


def measure_peaks() -> dict:
    """Measured arithmetic peaks of the current device in TFLOP/s (sem_measure_peaks)."""
    lib = L.load()
    out = (C.c_double * 3)()
    L.check(lib.sem_measure_peaks(out), "sem_measure_peaks")
    return {"fp64_fma": out[0], "fp64_mma": out[1], "fp32_fma": out[2]}


def gll(N: int):
    """GLL nodes, weights and D_hat as the library computes them (host-side)."""
    lib = L.load()
    xi, rho, D = np.empty(N + 1), np.empty(N + 1), np.empty((N + 1, N + 1))
    L.check(lib.sem_gll(N, xi.ctypes.data, rho.ctypes.data, D.ctypes.data), "sem_gll")
    return xi, rho, D


def coarse_partition(node, dmask, owner, x, y, z, n_G: int, nblocks: int) -> dict:
    """The order-1 sub-domain partition of the pipelined coarse solve (host-side,
    sem_coarse_partition); per-point inputs of length 8E, returns the arrays by name."""
    lib = L.load()
    node = np.ascontiguousarray(node, dtype=np.int32)
    dmask = np.ascontiguousarray(dmask, dtype=np.uint8)
    owner = np.ascontiguousarray(owner, dtype=np.uint8)
    x, y, z = (np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (x, y, z))
    nL = node.size
    E = nL // 8
    cap_n, cap_c = nL, 8 * nL
    out = dict(el_off=np.empty(nblocks + 1, np.int32), el=np.empty(E, np.int32), p2n=np.empty(nL, np.int32),
               nd_off=np.empty(nblocks + 1, np.int32), nd_src=np.empty(cap_n, np.int32),
               nd_fl=np.empty(cap_n, np.uint8), cp_off=np.empty(cap_n + 1, np.int32), cp=np.empty(cap_c, np.int32))
    counts = np.zeros(5, np.int64)
    p = {k: v.ctypes.data for k, v in out.items()}
    L.check(lib.sem_coarse_partition(E, int(n_G), node.ctypes.data, dmask.ctypes.data, owner.ctypes.data,
                                      x.ctypes.data, y.ctypes.data, z.ctypes.data, nblocks, cap_n, cap_c,
                                      p["el_off"], p["el"], p["p2n"], p["nd_off"], p["nd_src"], p["nd_fl"],
                                      p["cp_off"], p["cp"], counts.ctypes.data), "sem_coarse_partition")
    nn, nc = int(counts[0]), int(counts[1])
    out["nd_src"], out["nd_fl"] = out["nd_src"][:nn], out["nd_fl"][:nn]
    out["cp_off"], out["cp"] = out["cp_off"][:nn + 1], out["cp"][:nc]
    out["max_el"], out["max_nd"], out["max_cp"] = (int(c) for c in counts[2:])
    return out
