"""Quadrature rules of the oracle (test infrastructure only).

* Gauss-Jacobi rules on [-1, 1] for the weight (1-t)^alpha (1+t)^beta by the
  Golub-Welsch method: nodes are the eigenvalues of the Jacobi matrix of the
  monic Jacobi recurrence, weights are mu_0 times the squared first
  eigenvector components.
* Collapsed (Duffy) tensor rules on the unit simplex: Gauss-Legendre in the
  first collapsed coordinate, Gauss-Jacobi(1,0) in the second and
  Gauss-Jacobi(2,0) in the third absorb the Jacobian of the collapse, so an
  n-point rule per direction integrates total degree 2n-1 exactly.

The paper does not state a quadrature order (reading A1): the oracle uses
exact rules, degree 3k-1 in volumes (w, u in P^k, grad z in P^{k-1}) and 3k
on facets, so any other exact rule gives the same discrete operator.
"""
from __future__ import annotations

from math import gamma

import numpy as np


def gauss_jacobi(n: int, alpha: float, beta: float):
    """n-point Gauss-Jacobi rule on [-1, 1] (Golub-Welsch)."""
    ab = alpha + beta
    diag = np.empty(n)
    for i in range(n):
        den = (2 * i + ab) * (2 * i + ab + 2)
        diag[i] = (beta - alpha) / (ab + 2) if i == 0 else (beta ** 2 - alpha ** 2) / den
    off = np.empty(max(n - 1, 0))
    for i in range(1, n):
        num = 4.0 * i * (i + alpha) * (i + beta) * (i + ab)
        den = (2 * i + ab) ** 2 * (2 * i + ab + 1) * (2 * i + ab - 1)
        off[i - 1] = np.sqrt(num / den)
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(T)
    mu0 = 2.0 ** (ab + 1) * gamma(alpha + 1) * gamma(beta + 1) / gamma(ab + 2)
    weights = mu0 * vecs[0, :] ** 2
    return nodes, weights


def points_for_degree(degree: int) -> int:
    """Smallest n with 2n-1 >= degree."""
    return max(degree, 0) // 2 + 1


def simplex_rule(dim: int, degree: int):
    """Collapsed rule on the unit simplex {x_i >= 0, sum x_i <= 1}.

    Returns (points [Q, dim], weights [Q]); the weights sum to 1/dim!.
    ``dim == 1`` is Gauss-Legendre on [0, 1].
    """
    n = points_for_degree(degree)
    t0, w0 = gauss_jacobi(n, 0.0, 0.0)
    s0, v0 = (1 + t0) / 2, w0 / 2                 # int_0^1 g(s) ds
    if dim == 1:
        return s0[:, None], v0
    t1, w1 = gauss_jacobi(n, 1.0, 0.0)
    s1, v1 = (1 + t1) / 2, w1 / 4                 # int_0^1 g(s) (1-s) ds
    if dim == 2:
        A, B = np.meshgrid(s0, s1, indexing="ij")
        WA, WB = np.meshgrid(v0, v1, indexing="ij")
        x = A * (1 - B)
        y = B
        return np.stack([x.ravel(), y.ravel()], axis=1), (WA * WB).ravel()
    t2, w2 = gauss_jacobi(n, 2.0, 0.0)
    s2, v2 = (1 + t2) / 2, w2 / 8                 # int_0^1 g(s) (1-s)^2 ds
    A, B, C = np.meshgrid(s0, s1, s2, indexing="ij")
    WA, WB, WC = np.meshgrid(v0, v1, v2, indexing="ij")
    x = A * (1 - B) * (1 - C)
    y = B * (1 - C)
    z = C
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1), (WA * WB * WC).ravel()
