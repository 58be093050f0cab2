"""Hexahedral elements for the explicit upwind-DG convection step -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The three-dimensional counterpart of ``oracle/quad.py`` (Sec. 2 admits
hexahedra; uncurved, readings A27-A29 in 3D, A32):

* an uncurved hexahedron is the affine image of [0,1]^3, a parallelepiped:
  x = X_0 + J xi, J = [X_1 - X_0, X_3 - X_0, X_4 - X_0] for the local vertex
  order (0,0,0), (1,0,0), (1,1,0), (0,1,0), (0,0,1), (1,0,1), (1,1,1), (0,1,1);
* V_h = [Q^k]^3 with psi_{abc} = l_a(xi) l_b(eta) l_c(zeta), i = (a (k+1) + b)(k+1) + c;
* W_h = the H(div)-conforming subspace of the Piola images of [Q^k]^3.  Face
  moments int_F u . n_F l_a(s_1) l_b(s_2) dS in the face's global parameter:
  origin at the face vertex with the lowest global id, s_1 towards the lower-id
  of its two face neighbours, s_2 towards the other; n_F the outward normal of
  the lower-index element.  Interior moments of u^ against (l_a l_b l_c, 0, 0),
  a <= k-2, then (0, ., 0) with b <= k-2, then (0, 0, .) with c <= k-2 (each
  ordered like psi).

Local faces: f = 0: zeta = 0, 1: eta = 0, 2: xi = 1, 3: eta = 1, 4: xi = 0,
5: zeta = 1; the local face parameter (s_1, s_2) is the pair of tangential
reference coordinates in increasing axis order.

Quadrature: Gauss-Legendre with m = floor(3k/2) + 1 points per direction
(degree 3k per variable), as on parallelograms.  The operator is evaluated in
physical coordinates with the neighbour trace found by mapping the physical
face points back into the neighbour.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .quad import dleg, gauss01, leg, n_points

CORNERS = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
FACE_AXIS = (2, 1, 0, 1, 0, 2)          # normal axis of local face f
FACE_SIDE = (0, 0, 1, 1, 0, 1)          # the reference coordinate on face f
N_REF = np.array([[0, 0, -1], [0, -1, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, 0, 1]], float)


def tangential_axes(f: int):
    return tuple(a for a in range(3) if a != FACE_AXIS[f])


def face_point(f: int, s1, s2) -> np.ndarray:
    """Reference point of local face f at local parameters (s1, s2) [Q] -> [Q, 3]."""
    s1 = np.asarray(s1, dtype=np.float64)
    xi = np.zeros((s1.size, 3))
    t1, t2 = tangential_axes(f)
    xi[:, FACE_AXIS[f]] = FACE_SIDE[f]
    xi[:, t1] = s1
    xi[:, t2] = s2
    return xi


def face_corner_vertices(f: int):
    """Local vertex ids at the face corners (s1, s2) = (0,0), (1,0), (0,1), (1,1)."""
    out = []
    for s1, s2 in ((0, 0), (1, 0), (0, 1), (1, 1)):
        p = face_point(f, [s1], [s2])[0]
        out.append(int(np.nonzero(np.all(CORNERS == p, axis=1))[0][0]))
    return out


def vbasis(k: int, xi) -> np.ndarray:
    """psi_i at xi [M, 3] -> [M, N], i = (a (k+1) + b)(k+1) + c."""
    xi = np.asarray(xi, dtype=np.float64)
    n = k + 1
    l = [np.stack([leg(a, xi[:, d]) for a in range(n)], axis=1) for d in range(3)]
    return np.einsum("ma,mb,mc->mabc", *l).reshape(-1, n ** 3)


def vgrad(k: int, xi) -> np.ndarray:
    """Reference gradient of psi_i at xi [M, 3] -> [M, N, 3]."""
    xi = np.asarray(xi, dtype=np.float64)
    n = k + 1
    l = [np.stack([leg(a, xi[:, d]) for a in range(n)], axis=1) for d in range(3)]
    dl = [np.stack([dleg(a, xi[:, d]) for a in range(n)], axis=1) for d in range(3)]
    gx = np.einsum("ma,mb,mc->mabc", dl[0], l[1], l[2]).reshape(-1, n ** 3)
    gy = np.einsum("ma,mb,mc->mabc", l[0], dl[1], l[2]).reshape(-1, n ** 3)
    gz = np.einsum("ma,mb,mc->mabc", l[0], l[1], dl[2]).reshape(-1, n ** 3)
    return np.stack([gx, gy, gz], axis=2)


def cube_rule(m: int):
    t, w = gauss01(m)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), np.einsum("a,b,c->abc", w, w, w).ravel()


def square_rule(m: int):
    t, w = gauss01(m)
    A, B = np.meshgrid(t, t, indexing="ij")
    return A.ravel(), B.ravel(), np.outer(w, w).ravel()


class HexMesh:
    """Conforming mesh of parallelepipeds (local vertex order as in the module docstring)."""

    def __init__(self, verts, elems, tol: float = 1e-12):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.elems = np.asarray(elems, dtype=np.int64)
        self.dim = 3
        E = self.n_elem = self.elems.shape[0]
        X = self.X = self.verts[self.elems]                              # [E, 8, 3]
        self.J = np.stack([X[:, 1] - X[:, 0], X[:, 3] - X[:, 0], X[:, 4] - X[:, 0]], axis=2)
        pred = X[:, :1] + np.einsum("eab,vb->eva", self.J, CORNERS)
        scale = np.abs(self.J).sum(axis=(1, 2))
        if np.any(np.abs(pred - X).max(axis=(1, 2)) > tol * scale):
            raise ValueError("element is not a parallelepiped")
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ == 0.0):
            raise ValueError("degenerate element")
        self.Jinv = np.linalg.inv(self.J)
        corners = [face_corner_vertices(f) for f in range(6)]
        table = {}
        for e in range(E):
            for f in range(6):
                key = tuple(sorted(int(self.elems[e, v]) for v in corners[f]))
                table.setdefault(key, []).append((e, f))
        keys = sorted(table)
        self.n_facets = len(keys)
        self.facet_id = np.empty((E, 6), dtype=np.int64)
        self.nbr = -np.ones((E, 6), dtype=np.int64)
        self.nbr_facet = -np.ones((E, 6), dtype=np.int64)
        self.orient = np.ones((E, 6), dtype=np.int64)
        self.facet_owner = np.empty((self.n_facets, 2), dtype=np.int64)
        for g, key in enumerate(keys):
            sides = sorted(table[key])
            if len(sides) > 2:
                raise ValueError("non-manifold face")
            self.facet_owner[g] = sides[0]
            for (e, f) in sides:
                self.facet_id[e, f] = g
            if len(sides) == 2:
                (e0, f0), (e1, f1) = sides
                self.nbr[e0, f0], self.nbr_facet[e0, f0] = e1, f1
                self.nbr[e1, f1], self.nbr_facet[e1, f1] = e0, f0
                self.orient[e1, f1] = -1
        # local -> global face parameter: (transpose, o1, o2), o = local corner of the origin
        self.fcode = np.zeros((E, 6, 3), dtype=np.int64)
        loc = ((0, 0), (1, 0), (0, 1), (1, 1))
        for e in range(E):
            for f in range(6):
                ids = [int(self.elems[e, v]) for v in corners[f]]
                o = int(np.argmin(ids))
                o1, o2 = loc[o]
                adj = [j for j in range(4) if (loc[j][0] != o1) != (loc[j][1] != o2)]   # differ in one coordinate
                g1 = min(adj, key=lambda j: ids[j])
                transpose = 0 if loc[g1][0] != o1 else 1
                self.fcode[e, f] = (transpose, o1, o2)
        centre = X.mean(axis=1)
        self.normal = np.empty((E, 6, 3))
        self.area = np.empty((E, 6))
        for f in range(6):
            c = corners[f]
            t1 = X[:, c[1]] - X[:, c[0]]
            t2 = X[:, c[2]] - X[:, c[0]]
            nv = np.cross(t1, t2)
            A = np.linalg.norm(nv, axis=1)
            nv = nv / A[:, None]
            away = np.einsum("ed,ed->e", nv, X[:, c[0]] - centre)
            self.normal[:, f] = nv * np.sign(away)[:, None]
            self.area[:, f] = A

    def to_physical(self, e, xi):
        return self.X[e, 0, :] + np.einsum("mab,mb->ma", self.J[e], xi)

    def to_reference(self, e, x):
        return np.einsum("mab,mb->ma", self.Jinv[e], x - self.X[e, 0, :])

    def shortest_edge(self):
        lens = [np.linalg.norm(self.J[:, :, a], axis=1) for a in range(3)]
        return np.minimum(np.minimum(lens[0], lens[1]), lens[2])


def global_param(code, s1, s2):
    """The face's global parameter (sigma1, sigma2) at local (s1, s2) for code (T, o1, o2)."""
    T, o1, o2 = code
    a = 1.0 - s1 if o1 else s1
    b = 1.0 - s2 if o2 else s2
    return (b, a) if T else (a, b)


# ------------------------------------------------------------------------------
# W_h
# ------------------------------------------------------------------------------
def counts(k: int):
    n = k + 1
    N = n ** 3
    return N, n * n, 3 * n * n * (n - 2), 3 * N


def layout(mesh, k):
    N, n_fm, n_int, n_w = counts(k)
    return n_fm, n_int, n_w, mesh.n_facets * n_fm + mesh.n_elem * n_int


def interior_tests(k: int, xi) -> np.ndarray:
    """[n_int, M, 3]: component d against l_a l_b l_c with the d-th degree <= k-2."""
    xi = np.asarray(xi, dtype=np.float64)
    n = k + 1
    out = []
    for d in range(3):
        for a in range(n):
            for b in range(n):
                for c in range(n):
                    if (a, b, c)[d] > k - 2:
                        continue
                    v = leg(a, xi[:, 0]) * leg(b, xi[:, 1]) * leg(c, xi[:, 2])
                    t = np.zeros((xi.shape[0], 3))
                    t[:, d] = v
                    out.append(t)
    return np.array(out).reshape(-1, xi.shape[0], 3)


@lru_cache(maxsize=None)
def _local_dof_matrix(k: int) -> np.ndarray:
    N, n_fm, n_int, n_w = counts(k)
    n = k + 1
    m = k + 2
    s1, s2, ws = square_rule(m)
    Dm = np.zeros((n_w, n_w))
    for f in range(6):
        psi = vbasis(k, face_point(f, s1, s2))
        lm = np.stack([leg(a, s1) * leg(b, s2) for a in range(n) for b in range(n)], axis=1)   # mode a n + b
        for c in range(3):
            if N_REF[f, c] != 0.0:
                Dm[f * n_fm:(f + 1) * n_fm, c * N:(c + 1) * N] = N_REF[f, c] * np.einsum("q,qm,qi->mi", ws, lm, psi)
    if n_int:
        xq, wq = cube_rule(m)
        psi = vbasis(k, xq)
        T = interior_tests(k, xq)
        for c in range(3):
            Dm[6 * n_fm:, c * N:(c + 1) * N] = np.einsum("q,jq,qi->ji", wq, T[:, :, c], psi)
    Dm.setflags(write=False)
    return Dm


def local_dof_matrix(k: int) -> np.ndarray:
    return np.array(_local_dof_matrix(k))


def dof_map(mesh, k):
    """Global index and sign [E, n_w] of every local DOF: local face moment (alpha, beta)
    = orient sign(det J) (-1)^(alpha o1 + beta o2) times global moment (alpha, beta), or
    (beta, alpha) when the face parameter is transposed."""
    N, n_fm, n_int, n_w = counts(k)
    n = k + 1
    E = mesh.n_elem
    idx = np.empty((E, n_w), dtype=np.int64)
    sgn = np.ones((E, n_w))
    sd = np.sign(mesh.detJ)
    for f in range(6):
        T, o1, o2 = mesh.fcode[:, f, 0], mesh.fcode[:, f, 1], mesh.fcode[:, f, 2]
        for al in range(n):
            for be in range(n):
                j = f * n_fm + al * n + be
                gm = np.where(T == 1, be * n + al, al * n + be)
                idx[:, j] = mesh.facet_id[:, f] * n_fm + gm
                sgn[:, j] = mesh.orient[:, f] * sd * (-1.0) ** (al * o1 + be * o2)
    base = mesh.n_facets * n_fm
    for j in range(n_int):
        idx[:, 6 * n_fm + j] = base + np.arange(E) * n_int + j
    return idx, sgn


def ref_coeffs(mesh, k, u_hdiv, sel=None) -> np.ndarray:
    N = (k + 1) ** 3
    idx, sgn = dof_map(mesh, k)
    if sel is not None:
        idx, sgn = idx[sel], sgn[sel]
    loc = sgn * np.asarray(u_hdiv)[idx]
    return np.linalg.solve(local_dof_matrix(k), loc.T).T.reshape(-1, 3, N)


def evaluate(mesh, k, u_hdiv, e, xi) -> np.ndarray:
    e = np.asarray(e)
    coef = ref_coeffs(mesh, k, u_hdiv, sel=e)
    uref = np.einsum("mci,mi->mc", coef, vbasis(k, xi))
    return np.einsum("mab,mb->ma", mesh.J[e], uref) / mesh.detJ[e][:, None]


def dofs_of_field(mesh, k, field_e) -> np.ndarray:
    """DOFs of a physical field, field_e(e [S], xi [Q, 3]) -> [S, Q, 3]: face moments from
    the owner in the face's global parameter, interior moments of u^ = det J J^{-1} u."""
    n_fm, n_int, n_w, n_hdiv = layout(mesh, k)
    n = k + 1
    m = k + 2
    s1, s2, ws = square_rule(m)
    out = np.zeros(n_hdiv)
    e_own, f_own = mesh.facet_owner[:, 0], mesh.facet_owner[:, 1]
    for f in range(6):
        gs = np.nonzero(f_own == f)[0]
        if gs.size == 0:
            continue
        eo = e_own[gs]
        u = field_e(eo, face_point(f, s1, s2))                         # [g, Q, 3]
        un = np.einsum("gqd,gd->gq", u, mesh.normal[eo, f])
        for gi, g in enumerate(gs):
            sig1, sig2 = global_param(mesh.fcode[eo[gi], f], s1, s2)
            lm = np.stack([leg(a, sig1) * leg(b, sig2) for a in range(n) for b in range(n)], axis=1)
            out[g * n_fm:(g + 1) * n_fm] = mesh.area[eo[gi], f] * (ws * un[gi]) @ lm
    if n_int:
        xq, wq = cube_rule(m)
        T = interior_tests(k, xq)
        u = field_e(np.arange(mesh.n_elem), xq)
        uref = mesh.detJ[:, None, None] * np.einsum("eab,eqb->eqa", mesh.Jinv, u)
        out[mesh.n_facets * n_fm:] = np.einsum("eqa,jqa,q->ej", uref, T, wq).ravel()
    return out


def dofs_of_function(mesh, k, func) -> np.ndarray:
    def field_e(e, xi):
        S, Q = e.shape[0], xi.shape[0]
        x = mesh.to_physical(np.repeat(e, Q), np.tile(xi, (S, 1)))
        return func(x).reshape(S, Q, 3)
    return dofs_of_field(mesh, k, field_e)


def lagrange_nodes(k: int) -> np.ndarray:
    """Equispaced Q^k nodes, index (a (k+1) + b)(k+1) + c."""
    t = np.arange(k + 1) / k
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def wind_from_potential(mesh, k, pot) -> np.ndarray:
    """Divergence-free wind: the curl of the continuous [Q^k]^3 interpolant of a vector
    potential given at the element nodes, pot [E, (k+1)^3, 3] (reading A29 in 3D)."""
    n = k + 1
    t = np.arange(n) / k
    Lc = np.linalg.inv(np.vander(t, n, increasing=True))
    pot = np.asarray(pot, dtype=np.float64).reshape(mesh.n_elem, n, n, n, 3)

    def L1(x):
        return np.vander(x, n, increasing=True) @ Lc

    def dL1(x):
        V = np.zeros((x.size, n))
        for p in range(1, n):
            V[:, p] = p * x ** (p - 1)
        return V @ Lc

    def field_e(e, xi):
        lx, ly, lz = L1(xi[:, 0]), L1(xi[:, 1]), L1(xi[:, 2])
        dx, dy, dz = dL1(xi[:, 0]), dL1(xi[:, 1]), dL1(xi[:, 2])
        g = np.stack([np.einsum("sabcd,qa,qb,qc->sqd", pot[e], dx, ly, lz),
                      np.einsum("sabcd,qa,qb,qc->sqd", pot[e], lx, dy, lz),
                      np.einsum("sabcd,qa,qb,qc->sqd", pot[e], lx, ly, dz)], axis=3)   # [S, Q, comp, ref axis]
        gp = np.einsum("sba,sqcb->sqca", mesh.Jinv[e], g)                          # d A_c / d x_a
        return np.stack([gp[..., 2, 1] - gp[..., 1, 2], gp[..., 0, 2] - gp[..., 2, 0],
                         gp[..., 1, 0] - gp[..., 0, 1]], axis=-1)
    return dofs_of_field(mesh, k, field_e)


# ------------------------------------------------------------------------------
# convection, transfers
# ------------------------------------------------------------------------------
class HexConvectionOracle:
    """(M^V)^{-1} C^V(u) on parallelepipeds, as ``quad.QuadConvectionOracle`` in 3D."""

    def __init__(self, mesh, k, u_hdiv, sel=None):
        self.mesh, self.k, self.d = mesh, k, 3
        self.N = (k + 1) ** 3
        sel = np.arange(mesh.n_elem) if sel is None else np.asarray(sel, dtype=np.int64)
        self.sel = sel
        S = sel.size
        J, Jinv, detJ = mesh.J[sel], mesh.Jinv[sel], mesh.detJ[sel]
        self.absdet = np.abs(detJ)
        Ucoef = ref_coeffs(mesh, k, u_hdiv, sel=sel)
        m = n_points(k)
        xq, wq = cube_rule(m)
        self.Psi = vbasis(k, xq)
        self.dPsi = vgrad(k, xq)
        uphys = np.einsum("sab,sqb->sqa", J, np.einsum("sci,qi->sqc", Ucoef, self.Psi)) / detJ[:, None, None]
        self.vol_g = wq[None, :, None] * self.absdet[:, None, None] * np.einsum("sab,sqb->sqa", Jinv, uphys)
        s1, s2, ws = square_rule(m)
        Qf = ws.size
        self.psi_own = np.empty((S, 6, Qf, self.N))
        self.psi_nb = np.zeros((S, 6, Qf, self.N))
        self.un = np.empty((S, 6, Qf))
        self.wt = np.empty((S, 6, Qf))
        self.nbr = mesh.nbr[sel]
        for f in range(6):
            xi = face_point(f, s1, s2)
            x = mesh.to_physical(np.repeat(sel, Qf), np.tile(xi, (S, 1)))
            B = vbasis(k, xi)
            self.psi_own[:, f] = B[None]
            u_at = np.einsum("sab,sqb->sqa", J, np.einsum("sci,qi->sqc", Ucoef, B)) / detJ[:, None, None]
            self.un[:, f] = np.einsum("sqa,sa->sq", u_at, mesh.normal[sel, f])
            self.wt[:, f] = mesh.area[sel, f][:, None] * ws[None, :]
            nb = self.nbr[:, f]
            inner = nb >= 0
            if np.any(inner):
                xi_n = mesh.to_reference(np.repeat(nb[inner], Qf), x.reshape(S, Qf, 3)[inner].reshape(-1, 3))
                self.psi_nb[inner, f] = vbasis(k, xi_n).reshape(-1, Qf, self.N)

    def apply(self, w) -> np.ndarray:
        w = np.asarray(w)
        ws = w[self.sel]
        Wq = np.einsum("sci,qi->scq", ws, self.Psi)
        vol = -np.einsum("scq,sqa,qia->sci", Wq, self.vol_g, self.dPsi, optimize=True)
        w_own = np.einsum("sci,sfqi->sfqc", ws, self.psi_own)
        w_nb = np.einsum("sfci,sfqi->sfqc", w[np.maximum(self.nbr, 0)], self.psi_nb)
        hat = np.where((self.un >= 0)[..., None], w_own, w_nb)
        flux = (self.wt * self.un)[..., None] * hat
        return (vol + np.einsum("sfqc,sfqi->sci", flux, self.psi_own)) / self.absdet[:, None, None]


def transfer(mesh, k, u_hdiv) -> np.ndarray:
    xq, wq = cube_rule(k + 1)
    psi = vbasis(k, xq)
    coef = ref_coeffs(mesh, k, u_hdiv)
    u = np.einsum("eab,eqb->eqa", mesh.J, np.einsum("eci,qi->eqc", coef, psi)) / mesh.detJ[:, None, None]
    return np.einsum("q,eqc,qi->eci", wq, u, psi)


def transfer_T(mesh, k, f_dg) -> np.ndarray:
    N, n_fm, n_int, n_w = counts(k)
    xq, wq = cube_rule(k + 1)
    psi = vbasis(k, xq)
    Binv = np.linalg.inv(local_dof_matrix(k))
    phi = np.einsum("qi,cij->qcj", psi, Binv.reshape(3, N, n_w))
    R = np.einsum("q,qdj,qi->dij", wq, phi, psi)
    y = np.einsum("ecd,eci->edi", mesh.J, np.asarray(f_dg)) / mesh.detJ[:, None, None]
    z = np.einsum("dij,edi->ej", R, y)
    idx, sgn = dof_map(mesh, k)
    g = np.zeros(layout(mesh, k)[3])
    np.add.at(g, idx.ravel(), (sgn * z).ravel())
    return g


def max_wind_speed(mesh, k, u_hdiv) -> float:
    xq, _ = cube_rule(n_points(k))
    coef = ref_coeffs(mesh, k, u_hdiv)
    u = np.einsum("eab,eqb->eqa", mesh.J, np.einsum("eci,qi->eqc", coef, vbasis(k, xq))) / mesh.detJ[:, None, None]
    return float(np.linalg.norm(u, axis=2).max())


def cfl_ds(mesh, k, u_hdiv, cfl: float) -> float:
    return cfl * float(mesh.shortest_edge().min()) / ((2 * k + 1) * max_wind_speed(mesh, k, u_hdiv))


def integrals(mesh, k, w):
    """mass[c] = sum_T int_T w_c dx and energy = sum_T int_T |w|^2 dx on
    parallelepipeds (Sec. 2.3), Gauss rule on [0,1]^3 exact for degree 2k per
    direction, times |det J|."""
    xq, wq = cube_rule(k + 1)
    vals = np.einsum("eci,qi->ecq", np.asarray(w), vbasis(k, xq))
    ad = np.abs(mesh.detJ)
    return np.einsum("e,q,ecq->c", ad, wq, vals), float(np.einsum("e,q,ecq->", ad, wq, vals ** 2))


def upwind_energy(mesh, k, u_hdiv, w) -> float:
    s1, s2, ws = square_rule(n_points(k))
    total = 0.0
    for g in range(mesh.n_facets):
        e, f = mesh.facet_owner[g]
        x = mesh.to_physical(np.full(ws.size, e), face_point(f, s1, s2))
        xi = mesh.to_reference(np.full(ws.size, e), x)
        un = evaluate(mesh, k, u_hdiv, np.full(ws.size, e), xi) @ mesh.normal[e, f]
        wa = np.einsum("ci,qi->qc", w[e], vbasis(k, xi))
        e2 = mesh.nbr[e, f]
        wb = np.einsum("ci,qi->qc", w[e2], vbasis(k, mesh.to_reference(np.full(ws.size, e2), x))) if e2 >= 0 else 0.0
        total += 0.5 * mesh.area[e, f] * np.sum(ws * np.abs(un) * np.sum((wa - wb) ** 2, axis=1))
    return total
