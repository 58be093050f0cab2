"""Reference-element bases of the oracle (test infrastructure only).

Reference simplex: vertices v_0 = 0, v_i = e_i (i = 1..dim); barycentric
coordinates lambda_0 = 1 - sum x_i, lambda_i = x_i.

DG basis (Sec. 2.3): an L2-orthonormal basis of P^k on the reference simplex,
the Dubiner basis (collapsed-coordinate products of Jacobi polynomials, the
basis the paper cites in Sec. 2.2.3).  Orthonormality makes the DG mass
matrix diagonal, M^V_T = |det J_T| Id (reading A2).  Index order: by total
degree n, then (2D) q ascending with p = n - q; (3D) r ascending, then q
ascending, with p = n - q - r.

   2D  psi_pq  = c * v^p P_p(u/v) * P_q^{(2p+1,0)}(2y-1),
       u = 2x-1+y, v = 1-y,             c^2 = (2p+1) 2(p+q+1)
   3D  psi_pqr = c * v^p P_p(u/v) * v2^q P_q^{(2p+1,0)}(u2/v2) * P_r^{(2p+2q+2,0)}(2z-1),
       u = 2x-1+y+z, v = 1-y-z, u2 = 2y-1+z, v2 = 1-z,
       c^2 = (2p+1) 2(p+q+1) (2(p+q+r)+3)
   1D  psi_p   = sqrt(2p+1) P_p(2x-1)

H(div) space (Sec. 2.1.1): BDM_k = [P^k]^dim with the degrees of freedom
(reading A3)

* facet f (opposite v_f), mode m:  int_{param} (v . (-grad lambda_f)) q_m ds,
  where the facet is parametrised by its vertices in increasing local order,
  x(s) = v_a + sum_j s_j (v_{b_j} - v_a), and q_m is the (dim-1)-dimensional
  Dubiner basis in s.  (-grad lambda_f) ds is the area-weighted outward normal
  times the facet measure, so this is int_F v.n q_m dS on the reference facet.
* interior: int_T v . t_m dx with t_m running over the first-kind Nedelec
  space N_{k-1} = [P^{k-2}]^dim + S_{k-1} (Boffi-Brezzi-Fortin):
  [P^{k-2}]^dim as e_c psi_m (c outer, m inner, m < dim P^{k-2}); then S_{k-1}:
  2D: (-y, x) x^a y^(k-2-a), a = 0..k-2;
  3D: for each monomial x^a y^b z^c of degree k-2, ordered by c ascending then
  b ascending, the fields (x cross e_0) m, (x cross e_1) m and, only when c = 0,
  (x cross e_2) m.  Every interior test field is divided by its L2 norm on
  the reference simplex (this keeps the dual basis well scaled up to k = 6).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from scipy.special import eval_jacobi

from . import polynomials as P
from .quadrature import simplex_rule

LD = np.longdouble


def dim_pk(dim: int, k: int) -> int:
    return math.comb(k + dim, dim) if k >= 0 else 0


def dubiner_indices(dim: int, k: int):
    if dim == 1:
        return [(p,) for p in range(k + 1)]
    if dim == 2:
        return [(n - q, q) for n in range(k + 1) for q in range(n + 1)]
    return [(n - q - r, q, r) for n in range(k + 1) for r in range(n + 1) for q in range(n - r + 1)]


def _norm(idx) -> float:
    if len(idx) == 1:
        (p,) = idx
        return math.sqrt(2 * p + 1)
    if len(idx) == 2:
        p, q = idx
        return math.sqrt((2 * p + 1) * 2 * (p + q + 1))
    p, q, r = idx
    return math.sqrt((2 * p + 1) * 2 * (p + q + 1) * (2 * (p + q + r) + 3))


@lru_cache(maxsize=None)
def dubiner_polys(dim: int, k: int):
    """Dubiner basis as dense long-double monomial arrays (list of N arrays)."""
    out = []
    for idx in dubiner_indices(dim, k):
        c = LD(_norm(idx))
        if dim == 1:
            (p,) = idx
            poly = P.compose_1d(P.jacobi_coeffs(p, 0, 0), P.linear(1, -1, [2]))
        elif dim == 2:
            p, q = idx
            u = P.linear(2, -1, [2, 1])
            v = P.linear(2, 1, [0, -1])
            A = P.homogenised(P.jacobi_coeffs(p, 0, 0), u, v, p)
            B = P.compose_1d(P.jacobi_coeffs(q, 2 * p + 1, 0), P.linear(2, -1, [0, 2]))
            poly = P.mul(A, B)
        else:
            p, q, r = idx
            u = P.linear(3, -1, [2, 1, 1])
            v = P.linear(3, 1, [0, -1, -1])
            u2 = P.linear(3, -1, [0, 2, 1])
            v2 = P.linear(3, 1, [0, 0, -1])
            A = P.homogenised(P.jacobi_coeffs(p, 0, 0), u, v, p)
            B = P.homogenised(P.jacobi_coeffs(q, 2 * p + 1, 0), u2, v2, q)
            C = P.compose_1d(P.jacobi_coeffs(r, 2 * p + 2 * q + 2, 0), P.linear(3, -1, [0, 0, 2]))
            poly = P.mul(P.mul(A, B), C)
        out.append(P.scale(poly, c))
    return out


def dubiner_values(dim: int, k: int, pts) -> np.ndarray:
    """psi_i(x) at points [M, dim] -> [M, N], float64, by the collapsed formula.

    Stable direct evaluation (Jacobi polynomials of the collapsed
    coordinates); valid wherever the collapse denominators are non-zero,
    i.e. away from the top vertex / edge, which no quadrature point touches.
    """
    pts = np.asarray(pts, dtype=np.float64)
    M = pts.shape[0]
    idxs = dubiner_indices(dim, k)
    out = np.empty((M, len(idxs)))
    if dim == 1:
        x = pts[:, 0]
        for j, (p,) in enumerate(idxs):
            out[:, j] = _norm((p,)) * eval_jacobi(p, 0, 0, 2 * x - 1)
        return out
    if dim == 2:
        x, y = pts[:, 0], pts[:, 1]
        v = 1 - y
        a = (2 * x - 1 + y) / v
        for j, (p, q) in enumerate(idxs):
            out[:, j] = (_norm((p, q)) * eval_jacobi(p, 0, 0, a) * v ** p
                         * eval_jacobi(q, 2 * p + 1, 0, 2 * y - 1))
        return out
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    v = 1 - y - z
    a = (2 * x - 1 + y + z) / v
    v2 = 1 - z
    b = (2 * y - 1 + z) / v2
    for j, (p, q, r) in enumerate(idxs):
        out[:, j] = (_norm((p, q, r)) * eval_jacobi(p, 0, 0, a) * v ** p
                     * eval_jacobi(q, 2 * p + 1, 0, b) * v2 ** q
                     * eval_jacobi(r, 2 * p + 2 * q + 2, 0, 2 * z - 1))
    return out


def eval_polys(polys, pts) -> np.ndarray:
    """Evaluate a list of polynomials at points -> [M, len(polys)]."""
    return np.stack([P.evaluate(p, pts) for p in polys], axis=1)


def grad_polys(polys, dim: int):
    """Gradients: list over functions of lists over axes of polynomials."""
    return [[P.deriv(p, a) for a in range(dim)] for p in polys]


# --------------------------------------------------------------------------
# reference simplex geometry
# --------------------------------------------------------------------------
def ref_vertices(dim: int) -> np.ndarray:
    return np.vstack([np.zeros(dim), np.eye(dim)])


def facet_vertices(dim: int, f: int):
    """Local vertex ids of facet f (opposite vertex f), increasing."""
    return [v for v in range(dim + 1) if v != f]


def minus_grad_lambda(dim: int, f: int) -> np.ndarray:
    """-grad lambda_f: area-weighted outward normal of facet f times (dim-1)!."""
    if f == 0:
        return np.ones(dim)
    g = np.zeros(dim)
    g[f - 1] = -1.0
    return g


def facet_param_to_ref(dim: int, f: int, s) -> np.ndarray:
    """Map facet parameters s [M, dim-1] to reference points [M, dim]."""
    V = ref_vertices(dim)
    fv = facet_vertices(dim, f)
    s = np.asarray(s, dtype=np.float64)
    x = np.repeat(V[fv[0]][None, :], s.shape[0], axis=0)
    for j in range(dim - 1):
        x = x + s[:, j:j + 1] * (V[fv[j + 1]] - V[fv[0]])[None, :]
    return x


# --------------------------------------------------------------------------
# interior test space N_{k-1}
# --------------------------------------------------------------------------
def nedelec_interior_fields(dim: int, k: int):
    """List of vector fields (tuples of dim polynomials) spanning N_{k-1}."""
    fields = []
    if k < 2:
        return fields
    base = dubiner_polys(dim, k)[:dim_pk(dim, k - 2)]
    zero = P.zeros(dim, 1)
    for c in range(dim):
        for m in base:
            fields.append(tuple(m if cc == c else zero for cc in range(dim)))
    deg = k - 2

    def mono(exps):
        c = P.zeros(dim, deg + 1)
        c[tuple(exps)] = 1
        return c

    X = [P.linear(dim, 0, np.eye(dim)[i]) for i in range(dim)]
    if dim == 2:
        for a in range(deg + 1):
            m = mono((a, deg - a))
            fields.append((P.mul(P.scale(X[1], -1), m), P.mul(X[0], m)))
    else:
        # x cross e_0 = (0, z, -y); x cross e_1 = (-z, 0, x); x cross e_2 = (y, -x, 0)
        cross = [
            (zero, X[2], P.scale(X[1], -1)),
            (P.scale(X[2], -1), zero, X[0]),
            (X[1], P.scale(X[0], -1), zero),
        ]
        for c3 in range(deg + 1):
            for b in range(deg - c3 + 1):
                a = deg - c3 - b
                m = mono((a, b, c3))
                for e in range(3):
                    if e == 2 and c3 > 0:
                        continue
                    fields.append(tuple(P.mul(cross[e][i], m) for i in range(3)))
    # every test field is scaled to unit L2 norm on the reference simplex
    xq, wq = simplex_rule(dim, 2 * k)
    wq = wq.astype(LD)
    out = []
    for t in fields:
        nrm2 = sum((wq * P.evaluate(t[c], xq, LD) ** 2).sum() for c in range(dim))
        out.append(tuple(P.scale(t[c], LD(1) / np.sqrt(nrm2)) for c in range(dim)))
    return out


def hdiv_counts(dim: int, k: int):
    """(facet moments per facet, interior moments, local dimension N_W)."""
    n_fm = dim_pk(dim - 1, k)
    n_w = dim * dim_pk(dim, k)
    n_int = n_w - (dim + 1) * n_fm
    return n_fm, n_int, n_w


def _solve_ld(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Gauss-Jordan elimination with partial pivoting in long double."""
    A = np.array(A, dtype=LD)
    B = np.array(B, dtype=LD)
    n = A.shape[0]
    for col in range(n):
        piv = col + int(np.argmax(np.abs(A[col:, col])))
        if A[piv, col] == 0:
            raise np.linalg.LinAlgError("singular DOF matrix")
        if piv != col:
            A[[col, piv]] = A[[piv, col]]
            B[[col, piv]] = B[[piv, col]]
        inv = LD(1) / A[col, col]
        A[col] *= inv
        B[col] *= inv
        for r in range(n):
            if r != col and A[r, col] != 0:
                f = A[r, col]
                A[r] -= f * A[col]
                B[r] -= f * B[col]
    return B


@lru_cache(maxsize=None)
def bdm_element(dim: int, k: int):
    """BDM_k reference basis as coefficients on the vector Dubiner basis.

    The vector Dubiner basis is b_(c,i) = e_c psi_i, flattened as c*N + i.
    Returns ``Cb`` [N_W, N_W] (long double) with phi_j = sum_b Cb[b, j] b_b,
    i.e. the inverse of the DOF matrix V[dof, b] = dof(b_b).
    """
    N = dim_pk(dim, k)
    n_fm, n_int, n_w = hdiv_counts(dim, k)
    polys = dubiner_polys(dim, k)
    V = np.zeros((n_w, n_w), dtype=LD)
    # facet moments, exact for degree 2k on the facet
    s, ws = simplex_rule(dim - 1, 2 * k + 2)
    facet_basis = dubiner_polys(dim - 1, k)
    for f in range(dim + 1):
        xref = facet_param_to_ref(dim, f, s)
        psi = np.stack([P.evaluate(p, xref, LD) for p in polys], axis=1)   # [Q, N]
        qm = np.stack([P.evaluate(p, s, LD) for p in facet_basis], axis=1)  # [Q, n_fm]
        g = minus_grad_lambda(dim, f)
        for m in range(n_fm):
            for c in range(dim):
                if g[c] == 0:
                    continue
                row = f * n_fm + m
                V[row, c * N:(c + 1) * N] += LD(g[c]) * ((ws.astype(LD) * qm[:, m]) @ psi)
    # interior moments
    fields = nedelec_interior_fields(dim, k)
    assert len(fields) == n_int
    if n_int:
        xq, wq = simplex_rule(dim, 2 * k + 2)
        psi = np.stack([P.evaluate(p, xq, LD) for p in polys], axis=1)
        for m, t in enumerate(fields):
            row = (dim + 1) * n_fm + m
            for c in range(dim):
                tv = P.evaluate(t[c], xq, LD)
                V[row, c * N:(c + 1) * N] += (wq.astype(LD) * tv) @ psi
    Cb = _solve_ld(V, np.eye(n_w, dtype=LD))
    return Cb
