"""Curved triangles for the explicit upwind-DG convection step -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Remark "Curved elements" of Sec. 2.4: on curved elements the Piola map makes W_h
leave V_h, so I becomes the L2 projection, and M^V is block diagonal with
non-diagonal blocks on the curved elements only.  Readings (A30, A31):

* a curved triangle is the image of the reference triangle under the quadratic
  (P2) map x = F(xi) = sum_j X_j phi_j(xi) through its three vertices
  (sorted by global id, as for affine simplices) and three edge nodes: nodes
  [v_0, v_1, v_2, m_01, m_02, m_12] at xi = (0,0), (1,0), (0,1), (1/2,0),
  (0,1/2), (1/2,1/2), phi_a = lambda_a (2 lambda_a - 1), phi_ab =
  4 lambda_a lambda_b.  The edge node of every facet is given per global facet
  (facets numbered as for affine simplices); an element whose three edge nodes
  are the chord midpoints is affine.
* V_h = mapped polynomials psi^_i o F^{-1} per velocity component (the Dubiner
  basis on the reference triangle), M^V_T = int_T psi_i psi_j dx (dense on
  curved elements); W_h = Piola images of BDM_k with the reference DOFs of the
  affine case, so the H(div) coefficient layout is unchanged.

Everything here is evaluated in physical coordinates: the Jacobian J(xi) and
det J(xi) pointwise, facet normals and arc length from the mapped facet curve,
the neighbour trace by Newton inversion of the neighbour's map at the physical
facet points; I = (M^V)^{-1} M^{U,V} with the physical mixed mass matrix.
"""
from __future__ import annotations

import math

import numpy as np

from . import basis as B
from . import hdiv as H
from .mesh import Mesh
from .quadrature import simplex_rule

REF_NODES = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.5, 0.0], [0.0, 0.5], [0.5, 0.5]])
EDGE_OF_FACET = {0: 5, 1: 4, 2: 3}          # facet f (opposite vertex f) -> its edge node


def p2_values(xi) -> np.ndarray:
    """P2 Lagrange basis at reference points [M, 2] -> [M, 6]."""
    xi = np.asarray(xi, dtype=np.float64)
    l1, l2 = xi[:, 0], xi[:, 1]
    l0 = 1.0 - l1 - l2
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1), 4 * l0 * l1, 4 * l0 * l2, 4 * l1 * l2],
                    axis=1)


def p2_grads(xi) -> np.ndarray:
    """Reference gradients of the P2 basis [M, 6, 2]."""
    xi = np.asarray(xi, dtype=np.float64)
    l1, l2 = xi[:, 0], xi[:, 1]
    l0 = 1.0 - l1 - l2
    g = np.empty((xi.shape[0], 6, 2))
    g[:, 0, 0] = g[:, 0, 1] = -(4 * l0 - 1)
    g[:, 1, 0], g[:, 1, 1] = 4 * l1 - 1, 0.0
    g[:, 2, 0], g[:, 2, 1] = 0.0, 4 * l2 - 1
    g[:, 3, 0], g[:, 3, 1] = 4 * (l0 - l1), -4 * l1
    g[:, 4, 0], g[:, 4, 1] = -4 * l2, 4 * (l0 - l2)
    g[:, 5, 0], g[:, 5, 1] = 4 * l2, 4 * l1
    return g


class CurvedMesh:
    """Quadratic triangles: an affine simplicial mesh (connectivity, orientation)
    plus one edge node per global facet."""

    def __init__(self, verts, elems, edge_nodes):
        self.base = Mesh(verts, elems)
        b = self.base
        self.dim, self.n_elem, self.n_facets = 2, b.n_elem, b.n_facets
        edge_nodes = np.asarray(edge_nodes, dtype=np.float64)
        assert edge_nodes.shape == (b.n_facets, 2)
        self.nodes = np.empty((b.n_elem, 6, 2))
        self.nodes[:, :3] = b.X
        for f, j in EDGE_OF_FACET.items():
            self.nodes[:, j] = edge_nodes[b.facet_id[:, f]]
        mid = {5: (1, 2), 4: (0, 2), 3: (0, 1)}
        dev = np.max(np.stack([np.abs(self.nodes[:, j] - 0.5 * (b.X[:, a] + b.X[:, c])).max(axis=1)
                               for j, (a, c) in mid.items()]), axis=0)
        self.curved = dev > 1e-14 * b.shortest_edge()
        self.sign = np.sign(b.detJ)
        xq, _ = simplex_rule(2, 8)
        if np.any(np.sign(self.detJ(np.arange(self.n_elem), xq)) != self.sign[:, None]):
            raise ValueError("the quadratic map folds over inside an element")

    def J(self, e, xi) -> np.ndarray:
        """J(xi) [S, Q, 2, 2] for elements e [S] at points xi [Q, 2]."""
        return np.einsum("sja,qjb->sqab", self.nodes[e], p2_grads(xi))

    def detJ(self, e, xi) -> np.ndarray:
        J = self.J(e, xi)
        return J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]

    def to_physical(self, e, xi) -> np.ndarray:
        """x = F_e(xi) for elements e [S] at points xi [Q, 2] -> [S, Q, 2]."""
        return np.einsum("sja,qj->sqa", self.nodes[e], p2_values(xi))

    def to_reference(self, e, x, iters: int = 40) -> np.ndarray:
        """Newton inversion of F_e at physical points x [M, 2] (one element each, e [M])."""
        e = np.asarray(e)
        xi = self.base.to_reference(e, x)                         # affine guess
        for _ in range(iters):
            F = np.einsum("mja,mj->ma", self.nodes[e], p2_values(xi))
            G = np.einsum("mja,mjb->mab", self.nodes[e], p2_grads(xi))
            step = np.linalg.solve(G, (x - F)[..., None])[..., 0]
            xi = xi + step
            if np.abs(step).max() < 1e-15:
                break
        return xi

    def mass(self, k) -> np.ndarray:
        """M^V_T [E, N, N] = sum_q w_q |det J(xi_q)| psi_i psi_j (exact: degree 2k + 2)."""
        xq, wq = simplex_rule(2, 2 * k + 2)
        psi = B.dubiner_values(2, k, xq)
        dj = np.abs(self.detJ(np.arange(self.n_elem), xq))
        return np.einsum("q,eq,qi,qj->eij", wq, dj, psi, psi)

    def facet_points(self, e, f, s):
        """Physical points, unit outward normals and arc-length weights |dx/ds| on
        local facet f of element e at parameters s [Q]."""
        xi = B.facet_param_to_ref(2, f, s[:, None])
        fv = B.facet_vertices(2, f)
        dxi = B.ref_vertices(2)[fv[1]] - B.ref_vertices(2)[fv[0]]
        x = self.to_physical(np.array([e]), xi)[0]
        t = np.einsum("qab,b->qa", self.J(np.array([e]), xi)[0], dxi)   # dx/ds
        L = np.linalg.norm(t, axis=1)
        n = np.stack([t[:, 1], -t[:, 0]], axis=1) / L[:, None]
        inward = self.to_physical(np.array([e]), xi + 1e-3 * (np.array([1.0, 1.0]) / 3 - xi))[0] - x
        n = n * np.where(np.einsum("qa,qa->q", n, inward) > 0, -1.0, 1.0)[:, None]
        return xi, x, n, L


def evaluate(cm: CurvedMesh, k, u_hdiv, e, xi) -> np.ndarray:
    """Physical u = J(xi) u^(xi) / det J(xi) at points xi [Q, 2] of element e."""
    coef = H.ref_coeffs(cm.base, k, u_hdiv, sel=np.array([e]))[0]     # [2, N]
    uref = np.einsum("ci,qi->qc", coef, B.dubiner_values(2, k, xi))
    J = cm.J(np.array([e]), xi)[0]
    return np.einsum("qab,qb->qa", J, uref) / cm.detJ(np.array([e]), xi)[0][:, None]


def dofs_of_field(cm: CurvedMesh, k, field_e) -> np.ndarray:
    """BDM DOFs of a physical field, field_e(e, xi [Q, 2]) -> [Q, 2]: facet moments
    int_F u . n_F q_m dS on the curved facet (owner's outward normal, arc length),
    interior moments int u^ . t_m dxi of u^ = det J J^{-1} u."""
    n_fm, n_int, n_w, n_hdiv = H.layout(cm.base, k)
    s, ws = simplex_rule(1, 2 * k + 4)
    s = s[:, 0]
    qm = B.dubiner_values(1, k, s[:, None])
    out = np.zeros(n_hdiv)
    for g in range(cm.n_facets):
        e, f = cm.base.facet_owner[g]
        xi, x, n, L = cm.facet_points(e, f, s)
        un = np.einsum("qa,qa->q", field_e(e, xi), n)
        out[g * n_fm:(g + 1) * n_fm] = (ws * L * un) @ qm
    if n_int:
        xq, wq = simplex_rule(2, 2 * k + 4)
        T = np.stack([np.stack([B.P.evaluate(t[c], xq) for c in range(2)], axis=1)
                      for t in B.nedelec_interior_fields(2, k)])          # [n_int, Q, 2]
        base = cm.n_facets * n_fm
        for e in range(cm.n_elem):
            J = cm.J(np.array([e]), xq)[0]
            dj = cm.detJ(np.array([e]), xq)[0]
            uref = dj[:, None] * np.linalg.solve(J, field_e(e, xq)[..., None])[..., 0]
            out[base + e * n_int: base + (e + 1) * n_int] = np.einsum("qa,mqa,q->m", uref, T, wq)
    return out


def wind_from_potential(cm: CurvedMesh, k, pot) -> np.ndarray:
    """Divergence-free wind: the physical curl of the P^{k+1} Lagrange interpolant of
    a stream function given at the mapped nodes, pot [E, n_lag] (reading A13)."""
    order = k + 1
    L = H._lagrange_polys(2, order)
    dL = [[B.P.deriv(p, a) for a in range(2)] for p in L]
    pot = np.asarray(pot, dtype=np.float64)

    def field_e(e, xi):
        gl = np.stack([np.stack([B.P.evaluate(dL[n][a], xi) for a in range(2)], axis=1) for n in range(len(L))],
                      axis=1)                                             # [Q, n_lag, 2]
        g_ref = np.einsum("n,qna->qa", pot[e], gl)
        J = cm.J(np.array([e]), xi)[0]
        g = np.linalg.solve(np.transpose(J, (0, 2, 1)), g_ref[..., None])[..., 0]   # J^{-T} grad^
        return np.stack([g[:, 1], -g[:, 0]], axis=1)
    return dofs_of_field(cm, k, field_e)


def lagrange_points(cm: CurvedMesh, k) -> np.ndarray:
    """Physical positions of the P^{k+1} Lagrange nodes of every element [E, n_lag, 2]."""
    return cm.to_physical(np.arange(cm.n_elem), H.lagrange_nodes_ref(2, k + 1))


class CurvedConvectionOracle:
    """(M^V)^{-1} C^V(u) on curved triangles, evaluated in physical coordinates.

    C(u; w, z) = sum_T -int_T w (u . grad z) dx + int_dT (u . n) w^ z ds, the
    upwind value w^ taken from the side the wind comes from (zero inflow datum,
    interior trace on a tie), then the block-diagonal inverse mass matrix."""

    def __init__(self, cm: CurvedMesh, k, u_hdiv):
        self.mesh, self.k, self.d = cm, k, 2
        self.sel = np.arange(cm.n_elem)
        N = self.N = B.dim_pk(2, k)
        E = cm.n_elem
        self.Minv = np.linalg.inv(cm.mass(k))
        # the rules of the method (reading A1): the upwind switch inside a facet makes
        # the discrete operator depend on the facet points, so these are not raised
        xq, wq = simplex_rule(2, 3 * k - 1)
        self.Psi = B.dubiner_values(2, k, xq)
        polys = B.dubiner_polys(2, k)
        dpolys = B.grad_polys(polys, 2)
        dPsi = np.stack([np.stack([B.P.evaluate(g[a], xq) for a in range(2)], axis=1) for g in dpolys], axis=1)
        # volume: V[e][q][i] = w_q |det J| (u . grad psi_i)(x_q), grad psi = J^{-T} grad^ psi^
        self.V = np.empty((E, xq.shape[0], N))
        for e in range(E):
            J = cm.J(np.array([e]), xq)[0]
            dj = cm.detJ(np.array([e]), xq)[0]
            u = evaluate(cm, k, u_hdiv, e, xq)
            ginv = np.linalg.inv(J)                                       # [Q, 2, 2]
            gpsi = np.einsum("qba,qib->qia", ginv, dPsi)                  # J^{-T} grad^
            self.V[e] = (wq * np.abs(dj))[:, None] * np.einsum("qa,qia->qi", u, gpsi)
        s, ws = simplex_rule(1, 3 * k)
        s = s[:, 0]
        Qf = s.size
        self.psi_own = np.empty((E, 3, Qf, N))
        self.psi_nb = np.zeros((E, 3, Qf, N))
        self.flux = np.empty((E, 3, Qf))
        self.nbr = cm.base.nbr
        for e in range(E):
            for f in range(3):
                xi, x, n, L = cm.facet_points(e, f, s)
                self.psi_own[e, f] = B.dubiner_values(2, k, xi)
                self.flux[e, f] = ws * L * np.einsum("qa,qa->q", evaluate(cm, k, u_hdiv, e, xi), n)
                e2 = self.nbr[e, f]
                if e2 >= 0:
                    xi2 = cm.to_reference(np.full(Qf, e2), x)
                    self.psi_nb[e, f] = B.dubiner_values(2, k, xi2)

    def apply(self, w) -> np.ndarray:
        w = np.asarray(w)
        Wq = np.einsum("eci,qi->ecq", w, self.Psi)
        vol = -np.einsum("ecq,eqi->eci", Wq, self.V)
        w_own = np.einsum("eci,efqi->efqc", w, self.psi_own)
        w_nb = np.einsum("efci,efqi->efqc", w[np.maximum(self.nbr, 0)], self.psi_nb)
        hat = np.where((self.flux >= 0)[..., None], w_own, w_nb)
        fac = np.einsum("efq,efqc,efqi->eci", self.flux, hat, self.psi_own)
        return np.einsum("eij,ecj->eci", self.Minv, vol + fac)


def transfer(cm: CurvedMesh, k, u_hdiv) -> np.ndarray:
    """I u = (M^V)^{-1} int_T u psi_i dx, the L2 projection (remark on curved elements)."""
    xq, wq = simplex_rule(2, 2 * k + 2)
    psi = B.dubiner_values(2, k, xq)
    Minv = np.linalg.inv(cm.mass(k))
    out = np.empty((cm.n_elem, 2, psi.shape[1]))
    for e in range(cm.n_elem):
        u = evaluate(cm, k, u_hdiv, e, xq)
        dj = np.abs(cm.detJ(np.array([e]), xq)[0])
        out[e] = np.einsum("ij,cj->ci", Minv[e], np.einsum("q,qc,qj->cj", wq * dj, u, psi))
    return out


def transfer_T(cm: CurvedMesh, k, f_dg) -> np.ndarray:
    """g = I^T f: per element the local matrix of I, column j the transfer of the
    local BDM function s_j phi_j (its Piola image projected, (M^V_T)^{-1} int (J phi^_j / det J)
    psi_i |det J| dxi), transposed and accumulated into the global DOFs."""
    n_fm, n_int, n_w, n_hdiv = H.layout(cm.base, k)
    N = B.dim_pk(2, k)
    xq, wq = simplex_rule(2, 2 * k + 2)
    psi = B.dubiner_values(2, k, xq)
    Cb = np.asarray(B.bdm_element(2, k), dtype=np.float64)
    phi = np.einsum("qi,cij->qcj", psi, Cb.reshape(2, N, n_w))              # phi^_j(x_q)
    idx, sgn = H.dof_map(cm.base, k)
    M = cm.mass(k)
    f = np.asarray(f_dg)
    g = np.zeros(n_hdiv)
    for e in range(cm.n_elem):
        J = cm.J(np.array([e]), xq)[0]
        dj = cm.detJ(np.array([e]), xq)[0]
        piola = np.einsum("qab,qbj->qaj", J, phi) * np.sign(dj)[:, None, None]   # |det J| J phi^ / det J
        Be = np.einsum("q,qaj,qi->aij", wq, piola, psi)                    # [2, N, n_w]
        cols = np.stack([np.linalg.solve(M[e], Be[a]) for a in range(2)])
        z = np.einsum("aij,ai->j", cols, f[e])
        np.add.at(g, idx[e], sgn[e] * z)
    return g


def mass_apply(cm: CurvedMesh, k, v) -> np.ndarray:
    return np.einsum("eij,ecj->eci", cm.mass(k), np.asarray(v))


def upwind_energy(cm: CurvedMesh, k, u_hdiv, w) -> float:
    """1/2 sum_F int_F |u.n| [[w]]^2 + 1/2 int_{dOmega} |u.n| w^2 on the curved facets."""
    s, ws = simplex_rule(1, 3 * k)
    s = s[:, 0]
    total = 0.0
    for g in range(cm.n_facets):
        e, f = cm.base.facet_owner[g]
        xi, x, n, L = cm.facet_points(e, f, s)
        un = np.einsum("qa,qa->q", evaluate(cm, k, u_hdiv, e, xi), n)
        wa = np.einsum("ci,qi->qc", w[e], B.dubiner_values(2, k, xi))
        e2 = cm.base.nbr[e, f]
        wb = np.einsum("ci,qi->qc", w[e2], B.dubiner_values(2, k, cm.to_reference(np.full(s.size, e2), x))) \
            if e2 >= 0 else 0.0
        total += 0.5 * np.sum(ws * L * np.abs(un) * np.sum((wa - wb) ** 2, axis=1))
    return total


def max_wind_speed(cm: CurvedMesh, k, u_hdiv) -> float:
    xq, _ = simplex_rule(2, 3 * k - 1)
    return float(max(np.linalg.norm(evaluate(cm, k, u_hdiv, e, xq), axis=1).max() for e in range(cm.n_elem)))


def cfl_ds(cm: CurvedMesh, k, u_hdiv, cfl: float) -> float:
    return cfl * float(cm.base.shortest_edge().min()) / ((2 * k + 1) * max_wind_speed(cm, k, u_hdiv))


def integrals(cm: CurvedMesh, k, w):
    """mass[c] = sum_T int_T w_c dx and energy = sum_T int_T |w|^2 dx on the curved
    mesh (Sec. 2.3), the reference rule weighted by |det J(xi_q)| of the quadratic
    map (exact: degree 2k + 2)."""
    xq, wq = simplex_rule(2, 2 * k + 2)
    vals = np.einsum("eci,qi->ecq", np.asarray(w), B.dubiner_values(2, k, xq))
    dj = np.abs(cm.detJ(np.arange(cm.n_elem), xq))
    return np.einsum("q,eq,ecq->c", wq, dj, vals), float(np.einsum("q,eq,ecq->", wq, dj, vals ** 2))


def dg_energy(cm: CurvedMesh, k, v) -> float:
    """||v||^2_{L2} = sum_T v_c^T M_T v_c."""
    return float(np.einsum("eci,eij,ecj->", v, cm.mass(k), v))
