"""The H(div)-conforming velocity space W_h = BDM_k (Sec. 2.1.1) -- oracle.

Test infrastructure only.

Global coefficient vector (reading A3): the facet block
[n_facets][n_fm] -- value of int_F u . n_F q_m dS with n_F the owner's outward
normal and q_m the facet Dubiner basis in the facet's sorted-vertex
parametrisation -- followed by the interior block [E][n_int] of moments
int_T^ u^ . t_m dx of the reference field.  The tangential facet unknowns
F_h of the HDG space carry no convection and are never represented
(Sec. 2.4: I ignores them, I^T returns zero for them).

Element view: u(x) = (1/det J) J u^(xi) (contravariant Piola) with
u^ = sum_j s_j u_g(j) phi^_j, s_j = orient(e, f) * sign(det J) on the facet
moments of local facet f and +1 on interior moments (the Piola map turns
int_F u . n_T q dS into sign(det J) times the reference facet moment).
"""
from __future__ import annotations

import math

import numpy as np

from . import basis as B
from . import polynomials as P
from .quadrature import simplex_rule


def layout(mesh, k):
    """(n_fm, n_int, n_w, n_hdiv)."""
    n_fm, n_int, n_w = B.hdiv_counts(mesh.dim, k)
    return n_fm, n_int, n_w, mesh.n_facets * n_fm + mesh.n_elem * n_int


def local_signs(mesh) -> np.ndarray:
    return mesh.orient * np.sign(mesh.detJ)[:, None]


def dof_map(mesh, k):
    """Global index [E, n_w] and sign [E, n_w] of every local BDM DOF."""
    d = mesh.dim
    n_fm, n_int, n_w, _ = layout(mesh, k)
    E = mesh.n_elem
    idx = np.empty((E, n_w), dtype=np.int64)
    sgn = np.ones((E, n_w))
    s = local_signs(mesh)
    for f in range(d + 1):
        for m in range(n_fm):
            idx[:, f * n_fm + m] = mesh.facet_id[:, f] * n_fm + m
            sgn[:, f * n_fm + m] = s[:, f]
    base = mesh.n_facets * n_fm
    for m in range(n_int):
        idx[:, (d + 1) * n_fm + m] = base + np.arange(E) * n_int + m
    return idx, sgn


def ref_coeffs(mesh, k, u_hdiv, sel=None) -> np.ndarray:
    """Reference field u^ of each element on the vector Dubiner basis: [S, d, N]."""
    d = mesh.dim
    N = B.dim_pk(d, k)
    idx, sgn = dof_map(mesh, k)
    if sel is not None:
        idx, sgn = idx[sel], sgn[sel]
    loc = sgn * np.asarray(u_hdiv)[idx]                       # [S, n_w]
    Cb = np.asarray(B.bdm_element(d, k), dtype=np.float64)    # [n_w(basis b), n_w(dof j)]
    coef = loc @ Cb.T                                          # [S, n_w] on e_c psi_i
    return coef.reshape(-1, d, N)


def evaluate(mesh, k, u_hdiv, e, xi) -> np.ndarray:
    """Physical u at reference points xi [M, d] of elements e [M]."""
    e = np.asarray(e)
    coef = ref_coeffs(mesh, k, u_hdiv, sel=e)                  # [M, d, N]
    psi = B.dubiner_values(mesh.dim, k, xi)                    # [M, N]
    uref = np.einsum("mci,mi->mc", coef, psi)
    return np.einsum("mab,mb->ma", mesh.J[e], uref) / mesh.detJ[e][:, None]


def dofs_of_field(mesh, k, field_e, degree=None, elems=None) -> np.ndarray:
    """BDM DOFs of a field given per element.

    ``field_e(e [S], xi [Q, d]) -> u [S, Q, d]`` returns the physical field at
    the reference points xi of every element in e.  Facet moments are taken
    from the facet's owner element:
    int_F u . n_F q_m dS = |F| (d-1)! sum_q w_q (u . n_F)(x_q) q_m(s_q).
    Interior moments: int_T^ u^ . t_m dxi with u^ = det J J^{-1} u.

    ``elems`` restricts the work to the facets owned by those elements and to
    their interiors (the other entries stay zero); the restrictions to a
    partition of the elements add up to the full vector.
    """
    d = mesh.dim
    n_fm, n_int, n_w, n_hdiv = layout(mesh, k)
    degree = 2 * k + 2 if degree is None else degree
    out = np.zeros(n_hdiv)
    s, ws = simplex_rule(d - 1, degree)
    qm = B.dubiner_values(d - 1, k, s)                          # [Qf, n_fm]
    G = mesh.n_facets
    E = mesh.n_elem
    e_own = mesh.facet_owner[:, 0]
    f_own = mesh.facet_owner[:, 1]
    fact = math.factorial(d - 1)
    es = np.arange(E) if elems is None else np.unique(np.asarray(elems, dtype=np.int64))
    mine = np.zeros(E, dtype=bool)
    mine[es] = True
    for f in range(d + 1):
        gs = np.nonzero((f_own == f) & mine[e_own])[0]
        if gs.size == 0:
            continue
        xi_f = B.facet_param_to_ref(d, f, s)                    # [Qf, d]
        u = field_e(e_own[gs], xi_f)                            # [g, Qf, d]
        un = np.einsum("gqd,gd->gq", u, mesh.normal[e_own[gs], f])
        mom = fact * mesh.area[e_own[gs], f][:, None] * ((un * ws[None, :]) @ qm)   # [g, n_fm]
        out[(gs[:, None] * n_fm + np.arange(n_fm)[None, :]).ravel()] = mom.ravel()
    if n_int:
        xq, wq = simplex_rule(d, degree)
        fields = B.nedelec_interior_fields(d, k)
        T = np.stack([np.stack([P.evaluate(t[c], xq) for c in range(d)], axis=1) for t in fields])  # [n_int, Q, d]
        u = field_e(es, xq)                                     # [S, Q, d]
        uref = mesh.detJ[es, None, None] * np.einsum("eab,eqb->eqa", mesh.Jinv[es], u)
        mom = np.einsum("eqa,mqa,q->em", uref, T, wq)
        out[G * n_fm + (es[:, None] * n_int + np.arange(n_int)[None, :]).ravel()] = mom.ravel()
    return out


def dofs_of_function(mesh, k, func, degree=None, elems=None) -> np.ndarray:
    """BDM DOFs of an analytic field func(x [M, d]) -> [M, d] (``elems`` as in ``dofs_of_field``)."""
    def field_e(e, xi):
        S, Q = e.shape[0], xi.shape[0]
        x = mesh.to_physical(np.repeat(e, Q), np.tile(xi, (S, 1)))
        return func(x).reshape(S, Q, mesh.dim)
    return dofs_of_field(mesh, k, field_e, degree, elems=elems)


def lagrange_nodes_ref(dim: int, order: int) -> np.ndarray:
    """Equispaced P^order nodes on the reference simplex."""
    pts = []
    if dim == 2:
        for j in range(order + 1):
            for i in range(order + 1 - j):
                pts.append((i / order, j / order))
    else:
        for l in range(order + 1):
            for j in range(order + 1 - l):
                for i in range(order + 1 - l - j):
                    pts.append((i / order, j / order, l / order))
    return np.array(pts)


def _lagrange_polys(dim: int, order: int):
    """Lagrange basis of P^order at the equispaced nodes (monomial arrays)."""
    nodes = lagrange_nodes_ref(dim, order)
    exps = [e for e in np.ndindex(*(order + 1,) * dim) if sum(e) <= order]
    Vm = np.array([[np.prod([LDpow(x[i], e[i]) for i in range(dim)]) for e in exps] for x in nodes],
                  dtype=np.longdouble)
    coef = B._solve_ld(Vm, np.eye(len(nodes), dtype=np.longdouble))   # columns: Lagrange functions
    polys = []
    for n in range(len(nodes)):
        c = P.zeros(dim, order + 1)
        for j, e in enumerate(exps):
            c[e] = coef[j, n]
        polys.append(c)
    return polys


def LDpow(x, e):
    return np.longdouble(x) ** e


def wind_from_potential(mesh, k, potential, elems=None) -> np.ndarray:
    """Exactly divergence-free wind in W_h as the curl of an interpolated potential.

    Reading A13: interpolate the stream function psi (2D) or each component of
    the vector potential A (3D) by continuous P^{k+1} Lagrange elements
    (element-wise equispaced nodes, which coincide on shared facets), take the
    curl element by element (a [P^k]^d field with continuous normal component
    and zero divergence) and return its BDM_k DOFs.  ``elems`` restricts the
    DOFs computed as in ``dofs_of_field`` (the potential is then interpolated
    on those elements only).
    """
    d = mesh.dim
    order = k + 1
    nodes = lagrange_nodes_ref(d, order)
    L = _lagrange_polys(d, order)
    dL = [[P.deriv(p, a) for a in range(d)] for p in L]
    E = mesh.n_elem
    es = np.arange(E) if elems is None else np.unique(np.asarray(elems, dtype=np.int64))
    loc = np.full(E, -1, dtype=np.int64)
    loc[es] = np.arange(es.size)
    S = es.size
    ee = np.repeat(es, nodes.shape[0])
    X = mesh.to_physical(ee, np.tile(nodes, (S, 1)))
    if d == 2:
        vals = potential(X[:, 0], X[:, 1]).reshape(S, -1)           # [S, n_lag]
    else:
        vals = potential(X[:, 0], X[:, 1], X[:, 2]).reshape(3, S, -1).transpose(1, 2, 0)  # [S, n_lag, 3]

    def field_e(e, xi):
        # reference gradients of the Lagrange functions at xi -> [Q, n_lag, d]
        gl = np.stack([np.stack([P.evaluate(dL[n][a], xi) for a in range(d)], axis=1) for n in range(len(L))], axis=1)
        gphys = np.einsum("sba,qnb->sqna", mesh.Jinv[e], gl)       # J^{-T} grad^ -> [S, Q, n_lag, d]
        if d == 2:
            gpsi = np.einsum("sn,sqna->sqa", vals[loc[e]], gphys)
            return np.stack([gpsi[..., 1], -gpsi[..., 0]], axis=-1)
        gA = np.einsum("snc,sqna->sqca", vals[loc[e]], gphys)       # dA_c/dx_a
        return np.stack([gA[..., 2, 1] - gA[..., 1, 2], gA[..., 0, 2] - gA[..., 2, 0],
                         gA[..., 1, 0] - gA[..., 0, 1]], axis=-1)

    return dofs_of_field(mesh, k, field_e, elems=elems)
