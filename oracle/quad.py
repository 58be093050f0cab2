"""Quadrilateral elements for the explicit upwind-DG convection step -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2 ("Preliminaries") admits quadrilaterals besides simplices and takes all
elements uncurved.  Readings for them (A27-A29):

* an uncurved quadrilateral is the affine image of the reference square
  [0,1]^2, i.e. a parallelogram: x = X_0 + J xi with J[:, 0] = X_1 - X_0,
  J[:, 1] = X_3 - X_0 for the vertices (X_0, X_1, X_2, X_3) in cyclic order,
  X_2 = X_1 + X_3 - X_0 (det J keeps its sign);
* V_h = [Q^k(T)]^2 (physical components, tensor-product polynomials of degree
  k in each reference variable), with the L2-orthonormal basis
  psi_{ab}(xi, eta) = l_a(xi) l_b(eta), i = a (k+1) + b, l_a the orthonormal
  shifted Legendre polynomial on [0,1]; so M^V_T = |det J_T| Id (Sec. 2.3);
* W_h = { u in prod_T Piola([Q^k]^2) : [[u . n]] = 0 }: the H(div)-conforming
  subspace of V_h, so that W_h is contained in V_h and I is an embedding
  (Sec. 2.4).  DOFs: facet moments int_F u . n_F l_m(s) dS, m = 0..k, with s
  running from the facet's lower to its higher global vertex id and n_F the
  outward normal of the lower-index element; interior moments
  int_T^ u^ . q^ dxi of the reference field against q^ = (l_a l_b, 0),
  a <= k-2, b <= k, then q^ = (0, l_a l_b), a <= k, b <= k-2.

Local facets: f = 0: eta = 0 (X_0 -> X_1), 1: xi = 1 (X_1 -> X_2),
2: eta = 1 (X_3 -> X_2), 3: xi = 0 (X_0 -> X_3); each with the local
parameter s = xi (f = 0, 2) or eta (f = 1, 3).  Global facets are numbered by
sorting their sorted vertex pairs.

Quadrature is exact: Gauss-Legendre with m = floor(3k/2) + 1 points per
direction integrates degree 3k in each variable, the degree of
w u . grad z (volume) and of (u . n) w z (facets) for w, u, z in Q^k.
The operator is evaluated, as for simplices, in physical coordinates with the
neighbour trace found by mapping the physical facet points back into the
neighbour (no orientation tables).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg

from .quadrature import gauss_jacobi

F_LOC = ((0, 1), (1, 2), (3, 2), (0, 3))        # local facet -> (start, end) local vertices
N_REF = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])   # reference outward normals


def facet_point(f: int, s) -> np.ndarray:
    """Reference point of local facet f at local parameter s [Q] -> [Q, 2]."""
    s = np.asarray(s, dtype=np.float64)
    one, zero = np.ones_like(s), np.zeros_like(s)
    return np.stack([(s, zero), (one, s), (s, one), (zero, s)][f], axis=1)


# ------------------------------------------------------------------------------
# 1D building blocks
# ------------------------------------------------------------------------------
def gauss01(m: int):
    """m-point Gauss-Legendre rule on [0, 1] (Golub-Welsch on [-1, 1], mapped)."""
    t, w = gauss_jacobi(m, 0.0, 0.0)
    return 0.5 * (t + 1.0), 0.5 * w


def n_points(k: int) -> int:
    """Points per direction of the exact rules (degree 3k per variable)."""
    return (3 * k) // 2 + 1


def leg(a: int, t) -> np.ndarray:
    """Orthonormal shifted Legendre l_a(t) = sqrt(2a+1) P_a(2t-1) on [0,1]."""
    c = np.zeros(a + 1)
    c[a] = np.sqrt(2 * a + 1)
    return npleg.legval(2.0 * np.asarray(t, dtype=np.float64) - 1.0, c)


def dleg(a: int, t) -> np.ndarray:
    """d/dt l_a(t)."""
    c = np.zeros(a + 1)
    c[a] = np.sqrt(2 * a + 1)
    return 2.0 * npleg.legval(2.0 * np.asarray(t, dtype=np.float64) - 1.0, npleg.legder(c))


def vbasis(k: int, xi) -> np.ndarray:
    """psi_i at reference points xi [M, 2] -> [M, N], i = a (k+1) + b."""
    xi = np.asarray(xi, dtype=np.float64)
    n = k + 1
    lx = np.stack([leg(a, xi[:, 0]) for a in range(n)], axis=1)
    ly = np.stack([leg(b, xi[:, 1]) for b in range(n)], axis=1)
    return np.einsum("ma,mb->mab", lx, ly).reshape(-1, n * n)


def vgrad(k: int, xi) -> np.ndarray:
    """Reference gradient of psi_i at xi [M, 2] -> [M, N, 2]."""
    xi = np.asarray(xi, dtype=np.float64)
    n = k + 1
    lx = np.stack([leg(a, xi[:, 0]) for a in range(n)], axis=1)
    ly = np.stack([leg(b, xi[:, 1]) for b in range(n)], axis=1)
    dx = np.stack([dleg(a, xi[:, 0]) for a in range(n)], axis=1)
    dy = np.stack([dleg(b, xi[:, 1]) for b in range(n)], axis=1)
    gx = np.einsum("ma,mb->mab", dx, ly).reshape(-1, n * n)
    gy = np.einsum("ma,mb->mab", lx, dy).reshape(-1, n * n)
    return np.stack([gx, gy], axis=2)


def square_rule(m: int):
    """Tensor Gauss rule on [0,1]^2: points [m*m, 2] (xi index major), weights [m*m]."""
    t, w = gauss01(m)
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1), np.outer(w, w).ravel()


# ------------------------------------------------------------------------------
# mesh
# ------------------------------------------------------------------------------
class QuadMesh:
    """Conforming mesh of parallelograms, vertices of each element in cyclic order."""

    def __init__(self, verts, elems, tol: float = 1e-12):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.elems = np.asarray(elems, dtype=np.int64)
        self.dim = 2
        E = self.n_elem = self.elems.shape[0]
        X = self.X = self.verts[self.elems]                            # [E, 4, 2]
        scale = np.max(np.abs(X[:, 1] - X[:, 0]) + np.abs(X[:, 3] - X[:, 0]), axis=1)
        if np.any(np.linalg.norm(X[:, 0] + X[:, 2] - X[:, 1] - X[:, 3], axis=1) > tol * scale):
            raise ValueError("element is not a parallelogram")
        self.J = np.stack([X[:, 1] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)   # J[e][:, j]
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ == 0.0):
            raise ValueError("degenerate element")
        self.Jinv = np.linalg.inv(self.J)
        # facets by brute-force matching of sorted vertex pairs
        table = {}
        for e in range(E):
            for f, (a, b) in enumerate(F_LOC):
                key = tuple(sorted((int(self.elems[e, a]), int(self.elems[e, b]))))
                table.setdefault(key, []).append((e, f))
        keys = sorted(table)
        self.n_facets = len(keys)
        self.facet_verts = np.array(keys, dtype=np.int64)
        self.facet_id = np.empty((E, 4), dtype=np.int64)
        self.nbr = -np.ones((E, 4), dtype=np.int64)
        self.nbr_facet = -np.ones((E, 4), dtype=np.int64)
        self.orient = np.ones((E, 4), dtype=np.int64)
        self.facet_owner = np.empty((self.n_facets, 2), dtype=np.int64)
        for g, key in enumerate(keys):
            sides = sorted(table[key])
            if len(sides) > 2:
                raise ValueError("non-manifold facet")
            self.facet_owner[g] = sides[0]
            for (e, f) in sides:
                self.facet_id[e, f] = g
            if len(sides) == 2:
                (e0, f0), (e1, f1) = sides
                self.nbr[e0, f0], self.nbr_facet[e0, f0] = e1, f1
                self.nbr[e1, f1], self.nbr_facet[e1, f1] = e0, f0
                self.orient[e1, f1] = -1
        # local parameter runs against the global one (higher -> lower vertex id)
        self.flip = np.stack([(self.elems[:, a] > self.elems[:, b]).astype(np.int64) for (a, b) in F_LOC], axis=1)
        # outward unit normals and lengths
        self.normal = np.empty((E, 4, 2))
        self.length = np.empty((E, 4))
        centre = X.mean(axis=1)
        for f, (a, b) in enumerate(F_LOC):
            t = X[:, b] - X[:, a]
            nvec = np.stack([t[:, 1], -t[:, 0]], axis=1)
            L = np.linalg.norm(nvec, axis=1)
            nvec = nvec / L[:, None]
            away = np.einsum("ed,ed->e", nvec, X[:, a] - centre)
            self.normal[:, f] = nvec * np.sign(away)[:, None]
            self.length[:, f] = L

    def to_physical(self, e, xi):
        return self.X[e, 0, :] + np.einsum("mab,mb->ma", self.J[e], xi)

    def to_reference(self, e, x):
        return np.einsum("mab,mb->ma", self.Jinv[e], x - self.X[e, 0, :])

    def shortest_edge(self):
        return self.length.min(axis=1)


# ------------------------------------------------------------------------------
# H(div) space W_h (reading A28)
# ------------------------------------------------------------------------------
def counts(k: int):
    """(N, n_fm, n_int, n_w)."""
    N = (k + 1) ** 2
    return N, k + 1, 2 * (k + 1) * (k - 1), 2 * N


def layout(mesh, k):
    N, n_fm, n_int, n_w = counts(k)
    return n_fm, n_int, n_w, mesh.n_facets * n_fm + mesh.n_elem * n_int


def interior_tests(k: int, xi) -> np.ndarray:
    """Interior test fields q^_j at reference points xi [M, 2] -> [n_int, M, 2]."""
    xi = np.asarray(xi, dtype=np.float64)
    out = []
    for a in range(k - 1):
        for b in range(k + 1):
            v = leg(a, xi[:, 0]) * leg(b, xi[:, 1])
            out.append(np.stack([v, 0.0 * v], axis=1))
    for a in range(k + 1):
        for b in range(k - 1):
            v = leg(a, xi[:, 0]) * leg(b, xi[:, 1])
            out.append(np.stack([0.0 * v, v], axis=1))
    return np.array(out).reshape(-1, xi.shape[0], 2)


@lru_cache(maxsize=None)
def _local_dof_matrix(k: int) -> np.ndarray:
    Dm = _build_local_dof_matrix(k)
    Dm.setflags(write=False)
    return Dm


def local_dof_matrix(k: int) -> np.ndarray:
    """D[j, (c, i)]: local DOF j of the reference field e_c psi_i (exact quadrature)."""
    return np.array(_local_dof_matrix(k))


def _build_local_dof_matrix(k: int) -> np.ndarray:
    N, n_fm, n_int, n_w = counts(k)
    m = k + 2
    s, ws = gauss01(m)
    Dm = np.zeros((n_w, n_w))
    for f in range(4):
        psi = vbasis(k, facet_point(f, s))                       # [Q, N]
        lm = np.stack([leg(mm, s) for mm in range(n_fm)], axis=1)   # [Q, n_fm]
        for c in range(2):
            # int_0^1 (e_c psi_i) . n^_f l_m(s) ds
            Dm[f * n_fm:(f + 1) * n_fm, c * N:(c + 1) * N] = N_REF[f, c] * np.einsum("q,qm,qi->mi", ws, lm, psi)
    if n_int:
        xq, wq = square_rule(m)
        psi = vbasis(k, xq)
        T = interior_tests(k, xq)                                 # [n_int, Q, 2]
        for c in range(2):
            Dm[4 * n_fm:, c * N:(c + 1) * N] = np.einsum("q,jq,qi->ji", wq, T[:, :, c], psi)
    return Dm


def dof_map(mesh, k):
    """Global index and sign [E, n_w] of every local DOF (reading A28):
    local facet moment m = orient sign(det J) (-1)^(m flip) times the global one."""
    N, n_fm, n_int, n_w = counts(k)
    E = mesh.n_elem
    idx = np.empty((E, n_w), dtype=np.int64)
    sgn = np.ones((E, n_w))
    sd = np.sign(mesh.detJ)
    for f in range(4):
        for m in range(n_fm):
            idx[:, f * n_fm + m] = mesh.facet_id[:, f] * n_fm + m
            sgn[:, f * n_fm + m] = mesh.orient[:, f] * sd * np.where(mesh.flip[:, f] == 1, (-1.0) ** m, 1.0)
    base = mesh.n_facets * n_fm
    for j in range(n_int):
        idx[:, 4 * n_fm + j] = base + np.arange(E) * n_int + j
    return idx, sgn


def ref_coeffs(mesh, k, u_hdiv, sel=None) -> np.ndarray:
    """Reference field u^ on [psi_i e_c]: [S, 2, N] (solves the local DOF system)."""
    N = (k + 1) ** 2
    idx, sgn = dof_map(mesh, k)
    if sel is not None:
        idx, sgn = idx[sel], sgn[sel]
    loc = sgn * np.asarray(u_hdiv)[idx]                           # [S, n_w]
    coef = np.linalg.solve(local_dof_matrix(k), loc.T).T
    return coef.reshape(-1, 2, N)


def evaluate(mesh, k, u_hdiv, e, xi) -> np.ndarray:
    """Physical u = J u^ / det J at reference points xi [M, 2] of elements e [M]."""
    e = np.asarray(e)
    coef = ref_coeffs(mesh, k, u_hdiv, sel=e)
    uref = np.einsum("mci,mi->mc", coef, vbasis(k, xi))
    return np.einsum("mab,mb->ma", mesh.J[e], uref) / mesh.detJ[e][:, None]


def dofs_of_field(mesh, k, field_e) -> np.ndarray:
    """DOFs of a physical field given per element, field_e(e [S], xi [Q, 2]) -> [S, Q, 2].

    Facet moments from the owner element in physical terms,
    int_F u . n_F l_m(s) dS = |F| sum_q w_q (u . n_F)(x_q) l_m(s_q) with s the
    global (lower -> higher vertex id) parameter; interior moments of the
    reference field u^ = det J J^{-1} u."""
    n_fm, n_int, n_w, n_hdiv = layout(mesh, k)
    m = k + 2
    s, ws = gauss01(m)
    out = np.zeros(n_hdiv)
    e_own, f_own = mesh.facet_owner[:, 0], mesh.facet_owner[:, 1]
    for f in range(4):                                             # facets grouped by the owner's local facet
        gs = np.nonzero(f_own == f)[0]
        if gs.size == 0:
            continue
        eo = e_own[gs]
        u = field_e(eo, facet_point(f, s))                         # [g, Q, 2]
        un = np.einsum("gqd,gd->gq", u, mesh.normal[eo, f])
        sg = np.where(mesh.flip[eo, f][:, None] == 1, 1.0 - s[None, :], s[None, :])   # global parameter
        lm = np.stack([leg(mm, sg) for mm in range(n_fm)], axis=2)                   # [g, Q, n_fm]
        mom = mesh.length[eo, f][:, None] * np.einsum("q,gq,gqm->gm", ws, un, lm)
        out[(gs[:, None] * n_fm + np.arange(n_fm)[None, :]).ravel()] = mom.ravel()
    if n_int:
        xq, wq = square_rule(m)
        T = interior_tests(k, xq)
        E = mesh.n_elem
        u = field_e(np.arange(E), xq)
        uref = mesh.detJ[:, None, None] * np.einsum("eab,eqb->eqa", mesh.Jinv, u)
        out[mesh.n_facets * n_fm:] = np.einsum("eqa,jqa,q->ej", uref, T, wq).ravel()
    return out


def dofs_of_function(mesh, k, func) -> np.ndarray:
    """DOFs of an analytic field func(x [M, 2]) -> [M, 2]."""
    def field_e(e, xi):
        S, Q = e.shape[0], xi.shape[0]
        x = mesh.to_physical(np.repeat(e, Q), np.tile(xi, (S, 1)))
        return func(x).reshape(S, Q, 2)
    return dofs_of_field(mesh, k, field_e)


def lagrange_nodes(k: int) -> np.ndarray:
    """Equispaced Q^k nodes (a/k, b/k), index a (k+1) + b."""
    t = np.arange(k + 1) / k
    X, Y = np.meshgrid(t, t, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def wind_from_potential(mesh, k, pot) -> np.ndarray:
    """Exactly divergence-free wind in W_h (reading A29): the curl of the
    continuous Q^k interpolant of a stream function given by its values at the
    element nodes ``pot`` [E, (k+1)^2]; curl psi = (d_y psi, -d_x psi) lies in
    [Q^k]^2 with a continuous normal component (the tangential derivative of a
    continuous psi)."""
    n = k + 1
    t = np.arange(n) / k
    # 1D Lagrange basis at the equispaced nodes, as power-series coefficients
    Lc = np.linalg.inv(np.vander(t, n, increasing=True))        # column j: coefficients of L_j
    pot = np.asarray(pot, dtype=np.float64).reshape(mesh.n_elem, n, n)

    def L1(x):
        return np.vander(x, n, increasing=True) @ Lc

    def dL1(x):
        V = np.zeros((x.size, n))
        for p in range(1, n):
            V[:, p] = p * x ** (p - 1)
        return V @ Lc

    def field_e(e, xi):
        gx = np.einsum("qa,qb->qab", dL1(xi[:, 0]), L1(xi[:, 1]))      # d/dxi of L_a(xi) L_b(eta)
        gy = np.einsum("qa,qb->qab", L1(xi[:, 0]), dL1(xi[:, 1]))
        dref = np.stack([np.einsum("sab,qab->sq", pot[e], gx),
                         np.einsum("sab,qab->sq", pot[e], gy)], axis=2)    # [S, Q, 2] reference gradient
        gphys = np.einsum("sba,sqb->sqa", mesh.Jinv[e], dref)             # J^{-T} grad^
        return np.stack([gphys[..., 1], -gphys[..., 0]], axis=-1)

    return dofs_of_field(mesh, k, field_e)


# ------------------------------------------------------------------------------
# convection, transfers
# ------------------------------------------------------------------------------
class QuadConvectionOracle:
    """(M^V)^{-1} C^V(u) for one frozen wind u in W_h on parallelograms (Sec. 2.3).

    Same form and readings as ``dg.ConvectionOracle``: volume term
    -int_T w_c (u . grad psi_i) dx, facet term int_dT (u . n) w^ psi_i ds with
    the upwind trace w^ (zero inflow datum, interior trace on a tie), divided
    by |det J|.  ``sel`` restricts the output to a subset of elements."""

    def __init__(self, mesh, k, u_hdiv, sel=None):
        self.mesh, self.k, self.d = mesh, k, 2
        self.N = (k + 1) ** 2
        sel = np.arange(mesh.n_elem) if sel is None else np.asarray(sel, dtype=np.int64)
        self.sel = sel
        S = sel.size
        J, Jinv, detJ = mesh.J[sel], mesh.Jinv[sel], mesh.detJ[sel]
        self.absdet = np.abs(detJ)
        Ucoef = ref_coeffs(mesh, k, u_hdiv, sel=sel)                  # [S, 2, N]
        m = n_points(k)
        xq, wq = square_rule(m)
        self.Psi = vbasis(k, xq)                                       # [Q, N]
        self.dPsi = vgrad(k, xq)                                       # [Q, N, 2]
        uref = np.einsum("sci,qi->sqc", Ucoef, self.Psi)
        uphys = np.einsum("sab,sqb->sqa", J, uref) / detJ[:, None, None]
        # |det J| w_q J^{-1} u: the wind against reference gradients
        self.vol_g = wq[None, :, None] * self.absdet[:, None, None] * np.einsum("sab,sqb->sqa", Jinv, uphys)
        s, ws = gauss01(m)
        Qf = s.size
        self.psi_own = np.empty((S, 4, Qf, self.N))
        self.psi_nb = np.zeros((S, 4, Qf, self.N))
        self.un = np.empty((S, 4, Qf))
        self.wt = np.empty((S, 4, Qf))
        self.nbr = mesh.nbr[sel]
        for f in range(4):
            xi = facet_point(f, s)
            x = mesh.to_physical(np.repeat(sel, Qf), np.tile(xi, (S, 1)))   # physical facet points
            self.psi_own[:, f] = vbasis(k, xi)[None]
            u_at = np.einsum("sab,sqb->sqa", J, np.einsum("sci,qi->sqc", Ucoef, vbasis(k, xi))) / detJ[:, None, None]
            self.un[:, f] = np.einsum("sqa,sa->sq", u_at, mesh.normal[sel, f])
            self.wt[:, f] = mesh.length[sel, f][:, None] * ws[None, :]
            nb = self.nbr[:, f]
            inner = nb >= 0
            if np.any(inner):
                ne = np.repeat(nb[inner], Qf)
                xi_n = mesh.to_reference(ne, x.reshape(S, Qf, 2)[inner].reshape(-1, 2))
                self.psi_nb[inner, f] = vbasis(k, xi_n).reshape(-1, Qf, self.N)

    def apply(self, w) -> np.ndarray:
        """r = (M^V)^{-1} C^V(u) w on the selected elements; w: [E, 2, N] -> [S, 2, N]."""
        w = np.asarray(w)
        ws = w[self.sel]
        Wq = np.einsum("sci,qi->scq", ws, self.Psi)
        vol = -np.einsum("scq,sqa,qia->sci", Wq, self.vol_g, self.dPsi, optimize=True)
        w_own = np.einsum("sci,sfqi->sfqc", ws, self.psi_own)
        nbw = w[np.maximum(self.nbr, 0)]
        w_nb = np.einsum("sfci,sfqi->sfqc", nbw, self.psi_nb)
        hat = np.where((self.un >= 0)[..., None], w_own, w_nb)
        flux = (self.wt * self.un)[..., None] * hat
        fac = np.einsum("sfqc,sfqi->sci", flux, self.psi_own)
        return (vol + fac) / self.absdet[:, None, None]

    def magnitude(self, w) -> np.ndarray:
        """Summand scale of ``apply`` (sum of |summands| / |det J| per entry)."""
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


def transfer(mesh, k, u_hdiv) -> np.ndarray:
    """w = I u: w_{c,i} = (1/|det J|) int_T u_c psi_i dx (Sec. 2.4, the L2 problem)."""
    xq, wq = square_rule(k + 1)
    psi = vbasis(k, xq)
    coef = ref_coeffs(mesh, k, u_hdiv)
    uref = np.einsum("eci,qi->eqc", coef, psi)
    u = np.einsum("eab,eqb->eqa", mesh.J, uref) / mesh.detJ[:, None, None]
    return np.einsum("q,eqc,qi->eci", wq, u, psi)


def transfer_T(mesh, k, f_dg) -> np.ndarray:
    """g = I^T f: g_j = sum_T sum_{c,i} f_{T,c,i} (I phi_j)_{T,c,i} (Sec. 2.4);
    the local columns (1/det J) J int_T^ phi^_j psi^_i dxi by quadrature."""
    N, n_fm, n_int, n_w = counts(k)
    n_hdiv = layout(mesh, k)[3]
    xq, wq = square_rule(k + 1)
    psi = vbasis(k, xq)
    Binv = np.linalg.inv(local_dof_matrix(k))                      # column j: local basis fn j on e_c psi_i
    phi = np.einsum("qi,cij->qcj", psi, Binv.reshape(2, N, n_w))   # phi^_j(x_q)
    R = np.einsum("q,qdj,qi->dij", wq, phi, psi)
    f = np.asarray(f_dg)
    y = np.einsum("ecd,eci->edi", mesh.J, f) / mesh.detJ[:, None, None]
    z = np.einsum("dij,edi->ej", R, y)
    idx, sgn = dof_map(mesh, k)
    g = np.zeros(n_hdiv)
    np.add.at(g, idx.ravel(), (sgn * z).ravel())
    return g


def max_wind_speed(mesh, k, u_hdiv) -> float:
    """max |u(x_q)| over the volume quadrature points."""
    xq, _ = square_rule(n_points(k))
    coef = ref_coeffs(mesh, k, u_hdiv)
    uref = np.einsum("eci,qi->eqc", coef, vbasis(k, xq))
    u = np.einsum("eab,eqb->eqa", mesh.J, uref) / mesh.detJ[:, None, None]
    return float(np.linalg.norm(u, axis=2).max())


def cfl_ds(mesh, k, u_hdiv, cfl: float) -> float:
    """Substep size of reading A7 with h_T the shortest edge of the parallelogram."""
    return cfl * float(mesh.shortest_edge().min()) / ((2 * k + 1) * max_wind_speed(mesh, k, u_hdiv))


def integrals(mesh, k, w):
    """mass[c] = sum_T int_T w_c dx and energy = sum_T int_T |w|^2 dx on
    parallelograms (Sec. 2.3), Gauss rule on [0,1]^2 exact for degree 2k per
    direction, times |det J|."""
    xq, wq = square_rule(k + 1)
    vals = np.einsum("eci,qi->ecq", np.asarray(w), vbasis(k, xq))
    ad = np.abs(mesh.detJ)
    return np.einsum("e,q,ecq->c", ad, wq, vals), float(np.einsum("e,q,ecq->", ad, wq, vals ** 2))


def upwind_energy(mesh, k, u_hdiv, w) -> float:
    """1/2 sum_F int_F |u.n| [[w]]^2 + 1/2 int_{dOmega} |u.n| w^2 by facet
    quadrature, both traces found by affine inversion of physical points."""
    s, ws = gauss01(n_points(k))
    total = 0.0
    for g in range(mesh.n_facets):
        e, f = mesh.facet_owner[g]
        a, b = F_LOC[f]
        x = mesh.X[e, a] + s[:, None] * (mesh.X[e, b] - mesh.X[e, a])
        xi = mesh.to_reference(np.full(s.size, e), x)
        un = evaluate(mesh, k, u_hdiv, np.full(s.size, e), xi) @ mesh.normal[e, f]
        wa = np.einsum("ci,qi->qc", w[e], vbasis(k, xi))
        e2 = mesh.nbr[e, f]
        wb = np.einsum("ci,qi->qc", w[e2], vbasis(k, mesh.to_reference(np.full(s.size, e2), x))) if e2 >= 0 else 0.0
        total += 0.5 * mesh.length[e, f] * np.sum(ws * np.abs(un) * np.sum((wa - wb) ** 2, axis=1))
    return total
