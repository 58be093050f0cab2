"""Upwind DG convection, its explicit propagation and the transfer operators.

Test infrastructure only (see ``oracle/__init__``).

Definitions followed (Lehrenfeld & Schoeberl, arXiv:1508.04245):

* Sec. 2.3: V_h = [P^k(T)]^d per element, mass form M^V (diagonal with the
  orthonormal basis: M^V_T = |det J_T| Id), and the upwind trilinear form
      C(u; w, z) = sum_T  - int_T (w (x) u) : grad z dx
                          + int_{dT} (u . n) w^ z ds,
  w^ the upwind value, i.e. the trace from the side the wind comes from.
  With (w (x) u) : grad z = sum_c w_c (u . grad z_c), every velocity
  component is transported as an independent scalar.
* Sec. 3.2.2: the propagation problem dv/ds + (M^V)^{-1} C^V v = 0 with a
  frozen wind; integrated here by SSP-RK2 (Heun) or SSP-RK3 (Shu-Osher)
  (reading A6).
* Sec. 3.3.2: the implicit convection problem v + tau (M^V)^{-1} C^V v = g
  of the modified fractional-step-theta scheme, solved by the pseudo-time
  (Richardson) iteration (readings A9, A23, A24).
* Sec. 2.4: the embedding I: W_h -> V_h through the L2 problem
  int (I u) v = int u v for all v in V_h, and its transpose I^T.

Readings: exact quadrature (A1); ``apply`` returns +(M^V)^{-1} C^V w, the
ODE uses its negative (A8); a zero inflow datum on the domain boundary (A5);
the interior trace on a tie u . n = 0 (A4).

The operator is evaluated in physical coordinates: physical quadrature
points, normals and facet measures, the wind by the Piola map, and the
neighbour trace by mapping the physical facet point back into the neighbour
with the inverse of its affine map (no permutation tables).
"""
from __future__ import annotations

import math

import numpy as np

from . import basis as B
from . import hdiv as H
from .quadrature import simplex_rule


class ConvectionOracle:
    """(M^V)^{-1} C^V(u) for one fixed wind u in W_h, on a set of elements.

    ``sel`` restricts the output to a subset of elements (the input state is
    always the full vector, as neighbours are needed).
    """

    def __init__(self, mesh, k, u_hdiv, sel=None):
        self.mesh, self.k = mesh, k
        d = self.d = mesh.dim
        self.N = B.dim_pk(d, k)
        sel = np.arange(mesh.n_elem) if sel is None else np.asarray(sel, dtype=np.int64)
        self.sel = sel
        S = sel.size
        J, Jinv, detJ = mesh.J[sel], mesh.Jinv[sel], mesh.detJ[sel]
        self.absdet = np.abs(detJ)
        Ucoef = H.ref_coeffs(mesh, k, u_hdiv, sel=sel)                  # [S, d, N]

        # ---- volume: int_T w_c (u . grad psi_i) dx at exact quadrature -------
        xq, wq = simplex_rule(d, 3 * k - 1)
        polys = B.dubiner_polys(d, k)
        self.Psi = B.eval_polys(polys, xq)                                # [Q, N]
        dpolys = B.grad_polys(polys, d)
        self.dPsi = np.stack([np.stack([B.P.evaluate(g[a], xq) for a in range(d)], axis=1)
                              for g in dpolys], axis=1)                   # [Q, N, d]
        uref = np.einsum("sci,qi->sqc", Ucoef, self.Psi)
        uphys = np.einsum("sab,sqb->sqa", J, uref) / detJ[:, None, None]  # Piola
        # u . grad psi_i = u . J^{-T} grad^ psi^_i = (J^{-1} u) . grad^ psi^_i
        self.vol_g = (wq[None, :, None] * self.absdet[:, None, None]
                      * np.einsum("sab,sqb->sqa", Jinv, uphys))           # [S, Q, d]

        # ---- facets ---------------------------------------------------------
        s, ws = simplex_rule(d - 1, 3 * k)
        Qf = s.shape[0]
        fact = math.factorial(d - 1)
        X = mesh.X[sel]
        self.psi_own = np.empty((S, d + 1, Qf, self.N))
        self.psi_nb = np.zeros((S, d + 1, Qf, self.N))
        self.un = np.empty((S, d + 1, Qf))
        self.wt = np.empty((S, d + 1, Qf))
        self.nbr = mesh.nbr[sel]
        for f in range(d + 1):
            fv = [v for v in range(d + 1) if v != f]
            x = np.repeat(X[:, fv[0], None, :], Qf, axis=1)
            for j in range(d - 1):
                x = x + s[None, :, j, None] * (X[:, fv[j + 1], None, :] - X[:, fv[0], None, :])
            xf = x.reshape(-1, d)                                          # physical facet points
            ee = np.repeat(sel, Qf)
            xi = mesh.to_reference(ee, xf)
            self.psi_own[:, f] = B.dubiner_values(d, k, xi).reshape(S, Qf, self.N)
            u_at = np.einsum("mab,mb->ma", mesh.J[ee],
                             np.einsum("mci,mi->mc", np.repeat(Ucoef, Qf, axis=0),
                                       self.psi_own[:, f].reshape(-1, self.N))) / mesh.detJ[ee][:, None]
            self.un[:, f] = np.einsum("sqa,sa->sq", u_at.reshape(S, Qf, d), mesh.normal[sel, f])
            self.wt[:, f] = fact * mesh.area[sel, f][:, None] * ws[None, :]
            nb = self.nbr[:, f]
            inner = nb >= 0
            if np.any(inner):
                ne = np.repeat(nb[inner], Qf)
                xi_n = mesh.to_reference(ne, x[inner].reshape(-1, d))
                self.psi_nb[inner, f] = B.dubiner_values(d, k, xi_n).reshape(-1, Qf, self.N)

    def apply(self, w) -> np.ndarray:
        """r = (M^V)^{-1} C^V(u) w on the selected elements; w: [E, d, N] -> [S, d, N]."""
        w = np.asarray(w)
        ws = w[self.sel]
        # volume:  - sum_q w_q |det J| w_c(x_q) (u . grad psi_i)(x_q)
        Wq = np.einsum("sci,qi->scq", ws, self.Psi)
        vol = -np.einsum("scq,sqa,qia->sci", Wq, self.vol_g, self.dPsi, optimize=True)
        # facets:  sum_f sum_q |F| w_q (u.n) w^_c psi_i
        w_own = np.einsum("sci,sfqi->sfqc", ws, self.psi_own)
        nbw = w[np.maximum(self.nbr, 0)]                                  # [S, d+1, d, N]
        w_nb = np.einsum("sfci,sfqi->sfqc", nbw, self.psi_nb)             # 0 where boundary
        hat = np.where((self.un >= 0)[..., None], w_own, w_nb)
        flux = (self.wt * self.un)[..., None] * hat                       # [S, d+1, Qf, d]
        fac = np.einsum("sfqc,sfqi->sci", flux, self.psi_own)
        return (vol + fac) / self.absdet[:, None, None]

    def magnitude(self, w) -> np.ndarray:
        """The summand scale of ``apply``: the same sums taken over the absolute
        values of their summands, sum |a| / |det J| per output entry.

        A sum evaluated in floating point with unit roundoff eps is off by at most
        about (number of terms) * eps * sum |a|; this is the scale against which
        two evaluations of ``apply`` are compared when the result is a cancellation
        (smooth states on fine meshes, where the volume and facet parts are each
        about 1/h times the residual)."""
        w = np.asarray(w)
        ws = w[self.sel]
        Wq = np.einsum("sci,qi->scq", ws, self.Psi)
        vol = np.einsum("scq,sqa,qia->sci", np.abs(Wq), np.abs(self.vol_g), np.abs(self.dPsi), optimize=True)
        w_own = np.einsum("sci,sfqi->sfqc", ws, self.psi_own)
        nbw = w[np.maximum(self.nbr, 0)]
        w_nb = np.einsum("sfci,sfqi->sfqc", nbw, self.psi_nb)
        hat = np.where((self.un >= 0)[..., None], w_own, w_nb)
        flux = np.abs((self.wt * self.un)[..., None] * hat)
        fac = np.einsum("sfqc,sfqi->sci", flux, np.abs(self.psi_own))
        return (vol + fac) / self.absdet[:, None, None]


def rk_substeps(op: ConvectionOracle, v, ds: float, nsteps: int, scheme: int) -> np.ndarray:
    """nsteps explicit substeps of dv/ds = L v, L = -(M^V)^{-1} C^V (Sec. 3.2.2)."""
    assert op.sel.size == op.mesh.n_elem
    v = np.array(v, dtype=np.float64)
    L = lambda x: -op.apply(x)                                            # noqa: E731
    for _ in range(nsteps):
        if scheme == 2:          # SSP-RK2 (Heun)
            v1 = v + ds * L(v)
            v = 0.5 * v + 0.5 * (v1 + ds * L(v1))
        elif scheme == 3:        # SSP-RK3 (Shu-Osher)
            v1 = v + ds * L(v)
            v2 = 0.75 * v + 0.25 * (v1 + ds * L(v1))
            v = v / 3.0 + 2.0 / 3.0 * (v2 + ds * L(v2))
        else:
            raise ValueError(scheme)
    return v


def transfer(mesh, k, u_hdiv, sel=None) -> np.ndarray:
    """w = I u: w_{c,i} = (1/|det J|) int_T u_c psi_i dx   (Sec. 2.4, L2 problem);
    ``sel`` restricts the output to a subset of elements."""
    d = mesh.dim
    xq, wq = simplex_rule(d, 2 * k)
    sel = np.arange(mesh.n_elem) if sel is None else np.asarray(sel, dtype=np.int64)
    psi = B.dubiner_values(d, k, xq)                                     # [Q, N]
    u = np.stack([H.evaluate(mesh, k, u_hdiv, np.full(xq.shape[0], e), xq) for e in sel]) \
        if sel.size <= 64 else _eval_all(mesh, k, u_hdiv, xq, sel)        # [S, Q, d]
    return np.einsum("q,eqc,qi->eci", wq, u, psi)


def _eval_all(mesh, k, u_hdiv, xq, sel=None):
    sel = np.arange(mesh.n_elem) if sel is None else sel
    coef = H.ref_coeffs(mesh, k, u_hdiv, sel=sel)                         # [S, d, N]
    psi = B.dubiner_values(mesh.dim, k, xq)
    uref = np.einsum("eci,qi->eqc", coef, psi)
    return np.einsum("eab,eqb->eqa", mesh.J[sel], uref) / mesh.detJ[sel][:, None, None]


def transfer_T(mesh, k, f_dg) -> np.ndarray:
    """g = I^T f: g_j = sum_T sum_{c,i} f_{T,c,i} (I phi_j)_{T,c,i}  (Sec. 2.4).

    Per element the local matrix column for the local BDM function s_j phi^_j
    (Piola-mapped) is its transfer, (1/det J) J int_T^ phi^_j psi^_i dxi,
    computed here by quadrature; the transpose is accumulated into the
    global DOFs with np.add.at.
    """
    d = mesh.dim
    N = B.dim_pk(d, k)
    n_fm, n_int, n_w, n_hdiv = H.layout(mesh, k)
    xq, wq = simplex_rule(d, 2 * k)
    psi = B.dubiner_values(d, k, xq)                                     # [Q, N]
    Cb = np.asarray(B.bdm_element(d, k), dtype=np.float64)               # phi_j = sum_b Cb[b, j] b_b
    phi = np.einsum("qi,cib->qcb", psi, Cb.reshape(d, N, n_w))           # phi^_j(x_q) [Q, d, n_w]
    R = np.einsum("q,qdj,qi->dij", wq, phi, psi)                         # int phi^_{j,dd} psi^_i
    f = np.asarray(f_dg)
    y = np.einsum("ecd,eci->edi", mesh.J, f) / mesh.detJ[:, None, None]  # (J / det J)^T f
    z = np.einsum("dij,edi->ej", R, y)                                   # [E, n_w]
    idx, sgn = H.dof_map(mesh, k)
    g = np.zeros(n_hdiv)
    np.add.at(g, idx.ravel(), (sgn * z).ravel())
    return g


def mass(mesh, v) -> np.ndarray:
    """M^V v = |det J| v per element."""
    return np.abs(mesh.detJ)[:, None, None] * np.asarray(v)


def integrals(mesh, k, w):
    """Mass and energy of a DG field, the quantities of the conservation and
    stability statements of Sec. 2.3: mass[c] = sum_T int_T w_c dx per component,
    energy = sum_T int_T |w|^2 dx; by a reference rule exact for degree 2k, the
    element integral being |det J| times the reference one (affine map)."""
    d = mesh.dim
    xq, wq = simplex_rule(d, 2 * k)
    vals = np.einsum("eci,qi->ecq", np.asarray(w), B.dubiner_values(d, k, xq))
    ad = np.abs(mesh.detJ)
    return np.einsum("e,q,ecq->c", ad, wq, vals), float(np.einsum("e,q,ecq->", ad, wq, vals ** 2))


def upwind_energy(mesh, k, u_hdiv, w) -> float:
    """1/2 sum_F int_F |u.n| [[w]]^2 + 1/2 int_{dOmega} |u.n| w^2, by facet quadrature.

    Computed facet by facet from physical facet points, with both traces
    found by affine inversion; the right-hand side of the upwind energy
    identity that follows from the stability statement of Sec. 2.3.
    """
    d = mesh.dim
    s, ws = simplex_rule(d - 1, 3 * k)
    fact = math.factorial(d - 1)
    total = 0.0
    for g in range(mesh.n_facets):
        e, f = mesh.facet_owner[g]
        fv = [v for v in range(d + 1) if v != f]
        X = mesh.X[e]
        x = X[fv[0]] + s @ (X[fv[1:]] - X[fv[0]])
        xi = mesh.to_reference(np.full(len(s), e), x)
        un = H.evaluate(mesh, k, u_hdiv, np.full(len(s), e), xi) @ mesh.normal[e, f]
        wa = np.einsum("ci,qi->qc", w[e], B.dubiner_values(d, k, xi))
        e2 = mesh.nbr[e, f]
        if e2 >= 0:
            xi2 = mesh.to_reference(np.full(len(s), e2), x)
            wb = np.einsum("ci,qi->qc", w[e2], B.dubiner_values(d, k, xi2))
        else:
            wb = 0.0
        total += 0.5 * fact * mesh.area[e, f] * np.sum(ws * np.abs(un) * np.sum((wa - wb) ** 2, axis=1))
    return total


def assemble(op: ConvectionOracle) -> np.ndarray:
    """Dense matrix of w -> (M^V)^{-1} C^V w, column by column (tiny meshes)."""
    E, d, N = op.mesh.n_elem, op.d, op.N
    n = E * d * N
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = op.apply(e.reshape(E, d, N)).ravel()
    return A


def max_wind_speed(mesh, k, u_hdiv, sel=None) -> float:
    """max |u(x_q)| over the volume quadrature points (degree 3k-1 rule), over the
    elements ``sel`` (default all)."""
    xq, _ = simplex_rule(mesh.dim, 3 * k - 1)
    return float(np.linalg.norm(_eval_all(mesh, k, u_hdiv, xq, sel), axis=2).max())


def cfl_ds(mesh, k, u_hdiv, cfl: float) -> float:
    """Substep size (reading A7): cfl * min_T h_T / ((2k+1) max |u|), h_T the shortest edge."""
    return cfl * float(mesh.shortest_edge().min()) / ((2 * k + 1) * max_wind_speed(mesh, k, u_hdiv))


# ---------------------------------------------------------------------------------
# implicit convection step by pseudo-time stepping (Sec. 3.3.2)
# ---------------------------------------------------------------------------------
def dg_norm(mesh, x) -> float:
    """L2 norm of a DG function in the orthonormal basis: sqrt(sum_T |det J_T| sum_{c,i} x^2)."""
    x = np.asarray(x)
    return math.sqrt(float(np.sum(np.abs(mesh.detJ) * np.sum(x.reshape(x.shape[0], -1) ** 2, axis=1))))


def richardson(op: ConvectionOracle, g, v0, tau: float, ds: float, reduction: float, max_iter: int):
    """Solve v + tau (M^V)^{-1} C^V v = g (Sec. 3.3.2) by explicit Euler steps in
    pseudo-time s of dv/ds + v + tau (M^V)^{-1} C^V v = g, i.e. the Richardson
    iteration (reading A9 of the garbled sign)

        rho_i = g - v_i - tau (M^V)^{-1} C^V v_i,     v_{i+1} = v_i + ds rho_i,

    stopped at the first i with ||rho_i|| <= reduction ||rho_0|| or i = max_iter
    (reading A23: the DG L2 norm ``dg_norm``).

    Returns (v_i, i, [||rho_0||, ..., ||rho_i||]).
    """
    assert op.sel.size == op.mesh.n_elem
    v = np.array(v0, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    history = []
    i = 0
    while True:
        rho = g - v - tau * op.apply(v)
        history.append(dg_norm(op.mesh, rho))
        if history[-1] <= reduction * history[0] or i == max_iter:
            return v, i, history
        v = v + ds * rho
        i += 1


def richardson_ds(mesh, k, u_hdiv, tau: float) -> float:
    """Pseudo-time step (reading A24): 1 / (1 + beta^2), beta = tau (2k+1) max|u| / min_T h_T.

    The eigenvalues 1 + tau mu of Id + tau (M^V)^{-1} C^V have Re mu >= 0 (upwind
    energy) and |Im mu| up to about (2k+1) max|u| / h; an explicit Euler step
    ds contracts such a mode while ds < 2 Re(1 + tau mu) / |1 + tau mu|^2,
    which 1 / (1 + beta^2) satisfies for Re mu = 0 and |Im mu| <= beta / tau.
    """
    beta = tau * (2 * k + 1) * max_wind_speed(mesh, k, u_hdiv) / float(mesh.shortest_edge().min())
    return 1.0 / (1.0 + beta * beta)


# ---------------------------------------------------------------------------------
# compositions on the H(div) side (Sec. 3.2, OIFS; Sec. 2.4)
# ---------------------------------------------------------------------------------
def extrapolation_coefs(j: int, ds: float, dt_prev: float):
    """Weights (a, b) of u^n and u^{n-1} in the wind of substep j (reading A25): the
    linear extrapolation u^n + theta (u^n - u^{n-1}) through the two previous
    velocities (time levels t^n and t^n - dt_prev) evaluated at the substep's
    midpoint t^n + (j + 1/2) ds, theta = (j + 1/2) ds / dt_prev."""
    theta = (j + 0.5) * ds / dt_prev
    return 1.0 + theta, -theta


def oifs_rhs(mesh, k, u_hdiv, wind, ds: float, nsteps: int, scheme: int, wind_prev=None, dt_prev=None):
    """The OIFS right-hand side M^{V,U} Q I u (Sec. 3.2): transfer u into V_h,
    propagate it over nsteps substeps of the problem of Sec. 3.2.2 and map the
    result back as a functional on W_h, I^T M^V (M^{V,U} = I^T M^V).

    Without wind_prev the wind is frozen; with it, substep j uses the wind
    extrapolated from (wind, wind_prev) to its midpoint (reading A25)."""
    v = transfer(mesh, k, u_hdiv)
    if wind_prev is None:
        if nsteps > 0:
            v = rk_substeps(ConvectionOracle(mesh, k, wind), v, ds, nsteps, scheme)
    else:
        for j in range(nsteps):
            a, b = extrapolation_coefs(j, ds, dt_prev)
            v = rk_substeps(ConvectionOracle(mesh, k, extrapolate([wind, wind_prev], [a, b])), v, ds, 1, scheme)
    return transfer_T(mesh, k, mass(mesh, v))


def conv_hdiv(op: ConvectionOracle, u_hdiv) -> np.ndarray:
    """C^U u = I^T C^V I u, the convection operator on W_h (Sec. 2.4: C^U is the
    Galerkin restriction of C^V through the embedding); C^V = M^V (M^V)^{-1} C^V."""
    mesh, k = op.mesh, op.k
    return transfer_T(mesh, k, mass(mesh, op.apply(transfer(mesh, k, u_hdiv))))


def extrapolate(fields, coefs) -> np.ndarray:
    """sum_j c_j u_j: the extrapolated convection velocity as a linear combination
    of earlier exactly divergence-free velocities (Sec. 3.3)."""
    out = np.zeros_like(np.asarray(fields[0], dtype=np.float64))
    for f, c in zip(fields, coefs):
        out = out + c * np.asarray(f, dtype=np.float64)
    return out
