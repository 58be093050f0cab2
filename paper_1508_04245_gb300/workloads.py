"""Seeded synthetic inputs for the upwind-DG convection step.

This module only *generates inputs*: structured simplicial meshes with
optional vertex jitter, the analytic stream functions / vector potentials
from which the divergence-free winds are built, and random coefficient
vectors.  It contains none of the discretisation's arithmetic (no basis,
no quadrature, no operator), so the CUDA library and the CPU oracle can both
be fed from it without sharing any of the method.

The shapes follow the paper's workloads: affine triangles (2D) and tetrahedra
(3D) as in its Schaefer-Turek benchmarks (Sec. 4.4-4.5), with the unit square
/ cube standing in for the channel geometry, which is not available.

Mesh conventions
----------------
* vertices are numbered row-major: ``i + (n+1) j (+ (n+1)^2 l)``;
* squares are split along the diagonal (0,0)-(1,1) into two triangles,
  cubes are split into the six Kuhn (Freudenthal) tetrahedra that share the
  main diagonal (0,0,0)-(1,1,1); both give conforming meshes;
* the elements of one square / cube are consecutive, squares / cubes are
  row-major, so element order is spatially local;
* jitter moves interior vertices only, each coordinate by ``U[-J, J] * h``,
  so the domain stays exactly the unit square / cube.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def square_mesh(n: int, jitter: float = 0.0, seed: int | None = None):
    """Unit square, ``n x n`` squares, each split into 2 triangles.

    Returns ``(verts [ (n+1)^2, 2 ] float64, elems [ 2 n^2, 3 ] int32)``.
    """
    h = 1.0 / n
    g = np.arange(n + 1) * h
    X, Y = np.meshgrid(g, g, indexing="xy")          # X[j, i] = x_i
    verts = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        disp = rng.uniform(-jitter, jitter, size=verts.shape) * h
        ii = np.arange(n + 1)
        interior = ((ii[None, :] > 0) & (ii[None, :] < n) & (ii[:, None] > 0) & (ii[:, None] < n)).ravel()
        verts[interior] += disp[interior]
    vid = lambda i, j: i + (n + 1) * j                     # noqa: E731
    elems = np.empty((2 * n * n, 3), dtype=np.int32)
    e = 0
    for j in range(n):
        for i in range(n):
            v00, v10, v01, v11 = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
            elems[e] = (v00, v10, v11)
            elems[e + 1] = (v00, v11, v01)
            e += 2
    return verts, elems


def cube_mesh(n: int, jitter: float = 0.0, seed: int | None = None):
    """Unit cube, ``n^3`` cubes, each split into the 6 Kuhn tetrahedra.

    Returns ``(verts [ (n+1)^3, 3 ] float64, elems [ 6 n^3, 4 ] int32)``.
    """
    h = 1.0 / n
    g = np.arange(n + 1) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")     # X[l, j, i] = x_i
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        disp = rng.uniform(-jitter, jitter, size=verts.shape) * h
        ii = np.arange(n + 1)
        inn = (ii > 0) & (ii < n)
        interior = (inn[:, None, None] & inn[None, :, None] & inn[None, None, :]).ravel()
        verts[interior] += disp[interior]
    m = n + 1
    perms = list(itertools.permutations(range(3)))
    unit = np.eye(3, dtype=np.int64)
    elems = np.empty((6 * n ** 3, 4), dtype=np.int32)
    e = 0
    for l in range(n):
        for j in range(n):
            for i in range(n):
                base = np.array([i, j, l])
                for p in perms:
                    c0 = base
                    c1 = c0 + unit[p[0]]
                    c2 = c1 + unit[p[1]]
                    c3 = c2 + unit[p[2]]
                    elems[e] = [c[0] + m * c[1] + m * m * c[2] for c in (c0, c1, c2, c3)]
                    e += 1
    return verts, elems


# --------------------------------------------------------------------------
# analytic potentials for divergence-free winds
# --------------------------------------------------------------------------
@dataclass
class StreamModes2D:
    """psi(x, y) = sum_m a_m sin(p_m pi x) sin(q_m pi y); psi = 0 on the boundary."""
    a: np.ndarray
    p: np.ndarray
    q: np.ndarray

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros(np.broadcast(x, y).shape)
        for a, p, q in zip(self.a, self.p, self.q):
            out += a * np.sin(p * np.pi * x) * np.sin(q * np.pi * y)
        return out


def stream_single() -> StreamModes2D:
    """psi = sin(pi x) sin(pi y)."""
    return StreamModes2D(np.array([1.0]), np.array([1]), np.array([1]))


def stream_random(seed: int, n_modes: int = 8) -> StreamModes2D:
    """8 random modes, p, q in {1..4}, a ~ N(0,1) / (p^2 + q^2)."""
    rng = np.random.default_rng(seed)
    p = rng.integers(1, 5, size=n_modes)
    q = rng.integers(1, 5, size=n_modes)
    a = rng.standard_normal(n_modes) / (p ** 2 + q ** 2)
    return StreamModes2D(a, p, q)


@dataclass
class PotentialModes3D:
    """Vector potential A with vanishing tangential part on the unit cube.

    A_x = sum a cos(r pi x) sin(p pi y) sin(q pi z), and cyclically
    A_y(y, z, x), A_z(z, x, y) with their own mode sets.
    """
    modes: list   # three lists of (a, r, p, q)

    def __call__(self, x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        shape = np.broadcast(x, y, z).shape
        A = np.zeros((3,) + shape)
        coords = (x, y, z)
        for c in range(3):
            u, v, w = coords[c], coords[(c + 1) % 3], coords[(c + 2) % 3]
            for a, r, p, q in self.modes[c]:
                A[c] += a * np.cos(r * np.pi * u) * np.sin(p * np.pi * v) * np.sin(q * np.pi * w)
        return A


def potential_fixed() -> PotentialModes3D:
    """A = (sin pi y sin pi z, sin pi z sin pi x, sin pi x sin pi y)."""
    return PotentialModes3D([[(1.0, 0, 1, 1)], [(1.0, 0, 1, 1)], [(1.0, 0, 1, 1)]])


def potential_random(seed: int, n_modes: int = 8) -> PotentialModes3D:
    """Random modes r in {0..3}, p, q in {1..4}, a ~ N(0,1)/(r^2+p^2+q^2)."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(3):
        r = rng.integers(0, 4, size=n_modes)
        p = rng.integers(1, 5, size=n_modes)
        q = rng.integers(1, 5, size=n_modes)
        a = rng.standard_normal(n_modes) / (r ** 2 + p ** 2 + q ** 2)
        modes.append(list(zip(a, r, p, q)))
    return PotentialModes3D(modes)


@dataclass
class FourierField:
    """w_c(x) = sum_m b_cm cos(2 pi kappa_cm . x + phi_cm), kappa in {-4..4}^d."""
    b: np.ndarray       # [d, M]
    kappa: np.ndarray   # [d, M, d]
    phi: np.ndarray     # [d, M]

    def __call__(self, pts):
        pts = np.asarray(pts, dtype=np.float64)            # [..., d]
        d = self.b.shape[0]
        out = np.zeros(pts.shape[:-1] + (d,))
        for c in range(d):
            arg = 2.0 * np.pi * np.einsum("...k,mk->...m", pts, self.kappa[c]) + self.phi[c]
            out[..., c] = np.cos(arg) @ self.b[c]
        return out


def fourier_field(seed: int, dim: int, n_modes: int = 8) -> FourierField:
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=(dim, n_modes))
    kappa = rng.integers(-4, 5, size=(dim, n_modes, dim)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(dim, n_modes))
    return FourierField(b, kappa, phi)


def parallelogram_mesh(n: int, seed: int | None = None, stretch: float = 0.4, skew: float = 0.4,
                       reorient: bool = True):
    """``n x n`` parallelograms (uncurved quadrilaterals).

    A tensor grid with random column widths and row heights (each
    ``1 + U[-stretch, stretch]``, normalised to a unit total), every row of
    vertices shifted sideways by a random walk of steps ``U[-skew, skew]``
    times the row height: cell (i, j) is a parallelogram whose size, aspect
    ratio and shear change from cell to cell.  With ``reorient`` the vertex
    numbering is a random permutation and every cell starts its cyclic vertex
    order at a random corner, in reversed (clockwise) order for about half of
    them, so every local facet orientation and both signs of det J occur.

    Returns ``(verts [ (n+1)^2, 2 ] float64, elems [ n^2, 4 ] int32)``, the
    vertices of each element in cyclic order; cells are row-major.
    """
    rng = np.random.default_rng(seed)
    wx = 1.0 + rng.uniform(-stretch, stretch, n)
    wy = 1.0 + rng.uniform(-stretch, stretch, n)
    x = np.concatenate([[0.0], np.cumsum(wx / wx.sum())])
    y = np.concatenate([[0.0], np.cumsum(wy / wy.sum())])
    shift = np.concatenate([[0.0], np.cumsum(rng.uniform(-skew, skew, n) * np.diff(y))])
    verts = np.array([(x[i] + shift[j], y[j]) for j in range(n + 1) for i in range(n + 1)], dtype=np.float64)
    vid = lambda i, j: i + (n + 1) * j                     # noqa: E731
    elems = np.array([(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1))
                      for j in range(n) for i in range(n)], dtype=np.int64)
    if reorient:
        perm = rng.permutation(verts.shape[0])            # new id of old vertex v: perm[v]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        verts = verts[inv]
        elems = perm[elems]
        start = rng.integers(0, 4, size=elems.shape[0])
        rev = rng.random(elems.shape[0]) < 0.5
        for e in range(elems.shape[0]):
            cyc = np.roll(elems[e], -start[e])
            elems[e] = cyc[[0, 3, 2, 1]] if rev[e] else cyc
    return verts, elems.astype(np.int32)


def curved_square_mesh(n: int, jitter: float = 0.0, seed: int | None = None, delta: float = 0.15,
                       radius: float = 0.3):
    """``square_mesh`` with quadratic (P2) elements curved inside a disk.

    Every edge gets a mid-node: its chord midpoint m, moved by
    ``delta * h * w(m) * (sin(2 pi m_y + phi), cos(2 pi m_x + phi))`` with the
    cutoff ``w = (1 - r^2 / radius^2)^2`` for ``r = |m - (1/2, 1/2)| < radius``
    and 0 outside (phi seeded).  Elements with an edge inside the disk are
    curved, the others (and every boundary edge) stay straight.

    Returns ``(verts, elems, edge_nodes [n_edges, 2])`` with the edges in the
    order of their sorted vertex pairs, sorted lexicographically.
    """
    verts, elems = square_mesh(n, jitter, seed)
    pairs = sorted({tuple(sorted((int(t[a]), int(t[b])))) for t in elems for a, b in ((0, 1), (0, 2), (1, 2))})
    P = np.array(pairs)
    mid = 0.5 * (verts[P[:, 0]] + verts[P[:, 1]])
    phi = np.random.default_rng(None if seed is None else seed + 555).uniform(0.0, 2.0 * np.pi)
    r2 = np.sum((mid - 0.5) ** 2, axis=1)
    w = np.where(r2 < radius ** 2, (1.0 - r2 / radius ** 2) ** 2, 0.0)
    disp = np.stack([np.sin(2 * np.pi * mid[:, 1] + phi), np.cos(2 * np.pi * mid[:, 0] + phi)], axis=1)
    return verts, elems, mid + (delta / n) * w[:, None] * disp


def parallelepiped_mesh(n: int, seed: int | None = None, stretch: float = 0.4, skew: float = 0.3,
                        reorient: bool = True):
    """``n^3`` parallelepipeds (uncurved hexahedra).

    Vertex (i, j, l) sits at ``(x_i + a_j + b_l, y_j + c_l, z_l)`` with random
    spacings of x, y, z (each ``1 + U[-stretch, stretch]``, normalised) and
    random-walk shifts a, b, c (steps ``U[-skew, skew]`` times the layer
    thickness): separable coordinates make every cell a parallelepiped, each
    with its own size and shear.  With ``reorient`` the vertex numbering is a
    random permutation and every cell lists its vertices under one of the 48
    symmetries of the cube (axis permutation and reflections), so every face
    orientation and both signs of det J occur.

    Returns ``(verts [ (n+1)^3, 3 ], elems [ n^3, 8 ] int32)``, local vertex order
    (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1).
    """
    rng = np.random.default_rng(seed)
    axes = []
    for _ in range(3):
        w = 1.0 + rng.uniform(-stretch, stretch, n)
        axes.append(np.concatenate([[0.0], np.cumsum(w / w.sum())]))
    x, y, z = axes
    dy, dz = np.diff(y), np.diff(z)
    a = np.concatenate([[0.0], np.cumsum(rng.uniform(-skew, skew, n) * dy)])
    b = np.concatenate([[0.0], np.cumsum(rng.uniform(-skew, skew, n) * dz)])
    c = np.concatenate([[0.0], np.cumsum(rng.uniform(-skew, skew, n) * dz)])
    m = n + 1
    vid = lambda i, j, l: i + m * (j + m * l)                   # noqa: E731
    verts = np.array([(x[i] + a[j] + b[l], y[j] + c[l], z[l]) for l in range(m) for j in range(m) for i in range(m)])
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    elems = np.array([[vid(i + ci, j + cj, l + cl) for ci, cj, cl in corners]
                      for l in range(n) for j in range(n) for i in range(n)], dtype=np.int64)
    if reorient:
        perm = rng.permutation(verts.shape[0])
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        verts = verts[inv]
        elems = perm[elems]
        index = {cc: t for t, cc in enumerate(corners)}
        for e in range(elems.shape[0]):
            p = rng.permutation(3)
            fl = rng.integers(0, 2, 3)
            old = elems[e].copy()
            for t, cn in enumerate(corners):
                co = [0, 0, 0]
                for d in range(3):
                    co[p[d]] = cn[d] ^ int(fl[d])
                elems[e, t] = old[index[tuple(co)]]
    return verts, elems.astype(np.int32)


def tensor_coeffs(seed: int, n_elem: int, k: int) -> np.ndarray:
    """DG coefficients on parallelograms i.i.d. U[-1, 1], layout [E][2][(k+1)^2]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_elem, 2, (k + 1) ** 2))


# --------------------------------------------------------------------------
# coefficient vectors
# --------------------------------------------------------------------------
def dim_pk(dim: int, k: int) -> int:
    """dim P^k on a dim-simplex (a count, not arithmetic of the method)."""
    return math.comb(k + dim, dim)


def uniform_coeffs(seed: int, n_elem: int, dim: int, k: int) -> np.ndarray:
    """DG coefficients i.i.d. U[-1, 1], layout [E][d][N]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_elem, dim, dim_pk(dim, k)))


# --------------------------------------------------------------------------
# the five workload configurations (sizes only)
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    dim: int
    n: int            # squares / cubes per direction
    k: int
    jitter: float
    seed: int
    wind: str         # "single" | "random" (2D stream fn) / "fixed" | "random" (3D potential)
    state: str        # "uniform" | "fourier" | "wind" (a second divergence-free field)
    scheme: int       # 2 = SSP-RK2, 3 = SSP-RK3
    substeps: int
    cfl: float = 0.2
    unit_peak_speed: bool = False
    shape: str = "simplex"    # "simplex" | "quad" (parallelograms) | "curved" (quadratic triangles) | "hex"

    @property
    def n_elem(self) -> int:
        if self.shape == "quad":
            return self.n * self.n
        if self.shape == "hex":
            return self.n ** 3
        return (2 if self.dim == 2 else 6) * self.n ** self.dim

    def mesh(self):
        """(verts, elems), or (verts, elems, edge_nodes) for curved meshes."""
        if self.shape == "quad":
            return parallelogram_mesh(self.n, self.seed)
        if self.shape == "hex":
            return parallelepiped_mesh(self.n, self.seed)
        if self.shape == "curved":
            return curved_square_mesh(self.n, self.jitter, self.seed)
        if self.dim == 2:
            return square_mesh(self.n, self.jitter, self.seed)
        return cube_mesh(self.n, self.jitter, self.seed)

    def potential(self):
        if self.dim == 2:
            return stream_single() if self.wind == "single" else stream_random(self.seed + 1000)
        return potential_fixed() if self.wind == "fixed" else potential_random(self.seed + 1000)


WORKLOADS = {
    "square16_k2": Workload("square16_k2", 2, 16, 2, 0.0, 1, "single", "uniform", 2, 10),
    "square256_k4": Workload("square256_k4", 2, 256, 4, 0.10, 2, "random", "fourier", 3, 100),
    "cube32_k3": Workload("cube32_k3", 3, 32, 3, 0.0, 3, "fixed", "uniform", 3, 50),
    "cube48_k4": Workload("cube48_k4", 3, 48, 4, 0.05, 4, "random", "uniform", 3, 200,
                          unit_peak_speed=True),
    # the cube48_k4 recipe at 1/8 of its size (82944 tetrahedra): the case the kernel
    # profiles are captured on, small enough for a full ncu capture
    "cube24_k4": Workload("cube24_k4", 3, 24, 4, 0.05, 4, "random", "uniform", 3, 4, unit_peak_speed=True),
    # parallelograms: 256 x 256 cells of varying size and shear (3.3M DOFs at k = 4)
    "parallelogram256_k4": Workload("parallelogram256_k4", 2, 256, 4, 0.0, 6, "random", "fourier", 3, 100,
                                    shape="quad"),
    # quadratic triangles, edges inside a disk of radius 0.3 curved (about 28% of the elements)
    "curved256_k4": Workload("curved256_k4", 2, 256, 4, 0.10, 7, "random", "wind", 3, 100, shape="curved"),
    # parallelepipeds: 32^3 cells of varying size and shear (6.3M DOFs at k = 3)
    "parallelepiped32_k3": Workload("parallelepiped32_k3", 3, 32, 3, 0.0, 8, "random", "fourier", 3, 50,
                                    shape="hex"),
}


def batched_instances(seed: int = 5, count: int = 64):
    """64 independent 2D instances: n ~ U{8..128}, k ~ U{1..6}, 50 SSP-RK3 substeps."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(8, 129, size=count)
    ks = rng.integers(1, 7, size=count)
    return [Workload(f"batch{i}", 2, int(ns[i]), int(ks[i]), 0.0, 100 + i, "random", "uniform", 3, 50)
            for i in range(count)]
