"""Seeded synthetic inputs for the SEM elliptic path: box meshes and fields.

This module produces *inputs only*: element nodal coordinates in the local
lexicographic layout, global node ids, Dirichlet flags, and right-hand-side /
coefficient fields. It holds none of the method's arithmetic (no quadrature,
no differentiation, no operator, no gather-scatter). The oracle, the tests and
the benchmark all consume what it produces; the CUDA library never imports it.

Layout (Section 2.3, eq. uijk): an L-vector holds E blocks of (N+1)^3 values,
point (i, j, k) of element e at index i + (N+1)*(j + (N+1)*(k + (N+1)*e)),
i fastest. Arrays here are shaped (E, N+1, N+1, N+1) with axes (e, k, j, i).

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
evaluated counter-style: draw c of stream s is mix(s + (c + 1) * golden).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FACES = ("x0", "x1", "y0", "y1", "z0", "z1")


def splitmix64(seed: int, counters) -> np.ndarray:
    """SplitMix64 output for each counter value (uint64, wrapping arithmetic)."""
    c = np.asarray(counters).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, counters) -> np.ndarray:
    """Standard normal draws by Box-Muller on two uniforms per counter."""
    c = np.asarray(counters).astype(np.uint64)
    u1 = uniform01(seed, np.uint64(2) * c)
    u2 = uniform01(seed, np.uint64(2) * c + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def _node_positions(N: int) -> np.ndarray:
    """Reference-element node positions used to place mesh nodes.

    The mesh is defined by nodal coordinates at the Gauss-Lobatto-Legendre
    points (eq. xijk); this generator places them with numpy's Legendre
    derivative roots (a library routine, independent of both the oracle's and
    the library's own GLL rules).
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    if N == 1:
        return np.array([-1.0, 1.0])
    r = np.polynomial.legendre.Legendre.basis(N).deriv().roots().real
    x = np.concatenate(([-1.0], np.sort(r), [1.0]))
    return 0.5 * (x - x[::-1])  # exact antisymmetry


def element_permutation(E: int, seed: int) -> np.ndarray:
    """Fisher-Yates shuffle of range(E) driven by SplitMix64 (draw i picks j in [0, i])."""
    perm = np.arange(E, dtype=np.int64)
    if E > 1:
        draws = splitmix64(seed, np.arange(E, dtype=np.uint64))
        for i in range(E - 1, 0, -1):
            j = int(draws[i] % np.uint64(i + 1))
            perm[i], perm[j] = perm[j], perm[i]
    return perm


def box_mesh(n_el, N: int, warp: float = 0.0, perm_seed: int | None = 0,
             dirichlet=FACES, interior_zero: bool = False) -> dict:
    """Unit-cube box split into Ex x Ey x Ez hexahedra of order N.

    * Coordinates: x = (ex + (xi_i + 1)/2) / Ex per direction, then, if
      ``warp`` != 0, s = warp*sin(pi x)sin(pi y)sin(pi z) (unwarped x) is added
      to every coordinate. The warp vanishes on the cube's boundary.
    * Storage order: elements are shuffled by a SplitMix64 Fisher-Yates
      permutation (``perm_seed``; None keeps the natural order). Storage slot s
      holds natural element perm[s].
    * Global ids: lattice nodes are numbered 1, 2, ... in order of first
      appearance, scanning storage slots in order and points lexicographically.
      With ``interior_zero`` the element-interior points get id 0 (singletons).
    * Dirichlet flags: a point is Dirichlet if its lattice position lies on one
      of the listed faces ('x0' is x = 0, 'x1' is x = 1, ...).
    """
    if np.isscalar(n_el):
        n_el = (int(n_el),) * 3
    Ex, Ey, Ez = (int(v) for v in n_el)
    E = Ex * Ey * Ez
    NP = N + 1
    xi = _node_positions(N)
    perm = element_permutation(E, perm_seed) if perm_seed is not None else np.arange(E)
    ex = perm % Ex
    ey = (perm // Ex) % Ey
    ez = perm // (Ex * Ey)
    t = (xi + 1.0) / 2.0
    # Broadcast to (E, k, j, i)
    x = ((ex[:, None, None, None] + t[None, None, None, :]) / Ex) * np.ones((1, NP, NP, 1))
    y = ((ey[:, None, None, None] + t[None, None, :, None]) / Ey) * np.ones((1, NP, 1, NP))
    z = ((ez[:, None, None, None] + t[None, :, None, None]) / Ez) * np.ones((1, 1, NP, NP))
    ar = np.arange(NP)
    I = (ex[:, None, None, None] * N + ar[None, None, None, :]) * np.ones((1, NP, NP, 1), dtype=np.int64)
    J = (ey[:, None, None, None] * N + ar[None, None, :, None]) * np.ones((1, NP, 1, NP), dtype=np.int64)
    K = (ez[:, None, None, None] * N + ar[None, :, None, None]) * np.ones((1, 1, NP, NP), dtype=np.int64)
    LX, LY, LZ = Ex * N + 1, Ey * N + 1, Ez * N + 1
    lattice = I + LX * (J + LY * K)
    flat = lattice.ravel()
    uniq, first, inverse = np.unique(flat, return_index=True, return_inverse=True)
    rank = np.empty(uniq.size, dtype=np.int64)
    rank[np.argsort(first, kind="stable")] = np.arange(1, uniq.size + 1)
    gid = rank[inverse].reshape(lattice.shape)
    if interior_zero and N >= 2:
        inner = np.zeros((NP, NP, NP), dtype=bool)
        inner[1:N, 1:N, 1:N] = True
        gid = np.where(inner[None], 0, gid)
    dmask = np.zeros(lattice.shape, dtype=bool)
    on = {"x0": I == 0, "x1": I == Ex * N, "y0": J == 0, "y1": J == Ey * N,
          "z0": K == 0, "z1": K == Ez * N}
    for f in dirichlet:
        dmask |= on[f]
    if warp != 0.0:
        s = warp * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        x, y, z = x + s, y + s, z + s
    return {
        "E": E, "N": N, "shape": (Ex, Ey, Ez),
        "x": np.ascontiguousarray(x), "y": np.ascontiguousarray(y), "z": np.ascontiguousarray(z),
        "gid": np.ascontiguousarray(gid, dtype=np.int64),
        "dirichlet": np.ascontiguousarray(dmask.astype(np.uint8)),
        "lattice": np.ascontiguousarray(lattice),
        "n_lattice": LX * LY * LZ,
        "perm": perm,
    }


def manufactured(mesh: dict):
    """u* = sin(pi x) sin(pi y) sin(pi z) and f = 3 pi^2 u* at the mesh nodes."""
    u = np.sin(np.pi * mesh["x"]) * np.sin(np.pi * mesh["y"]) * np.sin(np.pi * mesh["z"])
    return u, 3.0 * np.pi ** 2 * u


def uniform_field(mesh: dict, seed: int = 0, continuous: bool = True) -> np.ndarray:
    """U[-1, 1] values: per lattice node (continuous across elements) or per local point."""
    if continuous:
        c = mesh["lattice"]
    else:
        c = np.arange(mesh["lattice"].size, dtype=np.int64).reshape(mesh["lattice"].shape)
    return 2.0 * uniform01(seed, c) - 1.0


def gaussian_assembled_rhs(mesh: dict, seed: int = 0) -> np.ndarray:
    """i.i.d. N(0,1) per lattice node with the lattice mean removed, replicated to local points."""
    vals = normal(seed, np.arange(mesh["n_lattice"], dtype=np.int64))
    vals -= vals.mean()
    return vals[mesh["lattice"]]


def smooth_random_modes(seed: int, modes: int = 64, kmax: int = 4):
    """The draws of smooth_random_field: wave vectors k_m [modes, 3], amplitudes a_m, phases phi_m."""
    r = np.arange(-kmax, kmax + 1)
    kk = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n2 = (kk ** 2).sum(1)
    kk = kk[(n2 > 0) & (n2 <= kmax * kmax)]
    pick = (splitmix64(seed, np.arange(modes)) % np.uint64(len(kk))).astype(np.int64)
    k = kk[pick].astype(np.float64)
    a = np.sqrt(2.0 / modes) * normal(seed + 1, np.arange(modes))
    phi = 2.0 * np.pi * uniform01(seed + 2, np.arange(modes))
    return k, a, phi


def smooth_random_field(mesh: dict, seed: int, modes: int = 64, kmax: int = 4) -> np.ndarray:
    """g(x) = sum_m a_m cos(pi k_m . x + phi_m) at the mesh nodes.

    k_m is drawn uniformly from the integer vectors with 0 < |k| <= kmax,
    a_m ~ N(0, 2/modes) (so Var g is about 1) and phi_m ~ U[0, 2 pi).
    """
    k, a, phi = smooth_random_modes(seed, modes, kmax)
    g = np.zeros_like(mesh["x"])
    for m in range(modes):
        g += a[m] * np.cos(np.pi * (k[m, 0] * mesh["x"] + k[m, 1] * mesh["y"] + k[m, 2] * mesh["z"]) + phi[m])
    return g


def travelling_modes(mesh: dict, seed: int, modes: int = 32, kmax: int = 3, omega_max: float = 2.0 * np.pi):
    """The pieces of travelling_field: amplitudes a_m, frequencies omega_m and the
    nodal fields cos(theta_m), sin(theta_m) with theta_m = pi k_m . x + phi_m,
    so that g(x, t) = sum_m a_m (cos(theta_m) cos(omega_m t) + sin(theta_m) sin(omega_m t)).
    k_m, a_m and phi_m are drawn as in smooth_random_field; omega_m ~ U[0, omega_max)."""
    r = np.arange(-kmax, kmax + 1)
    kk = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n2 = (kk ** 2).sum(1)
    kk = kk[(n2 > 0) & (n2 <= kmax * kmax)]
    pick = (splitmix64(seed, np.arange(modes)) % np.uint64(len(kk))).astype(np.int64)
    k = kk[pick].astype(np.float64)
    a = np.sqrt(2.0 / modes) * normal(seed + 1, np.arange(modes))
    phi = 2.0 * np.pi * uniform01(seed + 2, np.arange(modes))
    omega = omega_max * uniform01(seed + 3, np.arange(modes))
    theta = [np.pi * (k[m, 0] * mesh["x"] + k[m, 1] * mesh["y"] + k[m, 2] * mesh["z"]) + phi[m] for m in range(modes)]
    return a, omega, [np.cos(t) for t in theta], [np.sin(t) for t in theta]


def travelling_field(mesh: dict, seed: int, t: float, modes: int = 32, kmax: int = 3,
                     omega_max: float = 2.0 * np.pi) -> np.ndarray:
    """g(x, t) = sum_m a_m cos(pi k_m . x + phi_m - omega_m t) at the mesh nodes:
    a field that changes smoothly in time, standing in for the right-hand
    sides of successive time steps (travelling_modes gives its pieces)."""
    a, omega, c, s = travelling_modes(mesh, seed, modes, kmax, omega_max)
    g = np.zeros_like(mesh["x"])
    for m in range(modes):
        g += a[m] * (c[m] * np.cos(omega[m] * t) + s[m] * np.sin(omega[m] * t))
    return g


def cube_for_points(N: int, target_points: int = 16_777_216) -> int:
    """Elements per side of the box whose local point count E*(N+1)^3 is closest to the target."""
    e1 = round((target_points / (N + 1) ** 3) ** (1.0 / 3.0))
    return max(1, int(e1))
