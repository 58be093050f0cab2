"""Pins of the oracle's quadrature and reference bases (CPU only).

Each check compares the oracle against something other than itself:
closed-form monomial integrals, scipy's Gauss-Jacobi routine, numpy's
Legendre polynomials, orthonormality under the (separately pinned)
quadrature, and polynomial reproduction.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre
from scipy.special import roots_jacobi

from oracle import basis as B
from oracle import polynomials as P
from oracle import quadrature as Q


@pytest.mark.parametrize("n,a,b", [(1, 0, 0), (5, 0, 0), (7, 1, 0), (9, 2, 0), (4, 2.5, 1.0)])
def test_gauss_jacobi_matches_scipy(n, a, b):
    x, w = Q.gauss_jacobi(n, a, b)
    xr, wr = roots_jacobi(n, a, b)
    assert np.allclose(x, xr, atol=1e-14, rtol=0)
    assert np.allclose(w, wr, atol=0, rtol=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("degree", [0, 1, 5, 11, 12, 17])
def test_simplex_rule_integrates_monomials(dim, degree):
    """int_T x^a y^b z^c = a! b! c! / (a+b+c+dim)!  (closed form on the unit simplex)."""
    pts, w = Q.simplex_rule(dim, degree)
    for exps in np.ndindex(*(degree + 1,) * dim):
        if sum(exps) > degree:
            continue
        exact = math.prod(math.factorial(e) for e in exps) / math.factorial(sum(exps) + dim)
        got = np.sum(w * np.prod(pts ** np.array(exps), axis=1))
        assert abs(got - exact) <= 1e-15 * max(1.0, exact) + 1e-16, (exps, got, exact)


def test_simplex_rule_degree_is_sharp():
    """The n-point collapsed rule is not exact one degree beyond 2n-1."""
    pts, w = Q.simplex_rule(2, 5)          # n = 3
    exact = math.factorial(6) / math.factorial(8)
    got = np.sum(w * pts[:, 0] ** 6)
    assert abs(got - exact) > 1e-8


@pytest.mark.parametrize("dim,k", [(1, 6), (2, 6), (3, 5)])
def test_dubiner_orthonormal(dim, k):
    pts, w = Q.simplex_rule(dim, 2 * k)
    V = B.dubiner_values(dim, k, pts)
    M = V.T @ (w[:, None] * V)
    assert np.abs(M - np.eye(M.shape[0])).max() < 1e-13


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dubiner_constant_mode(dim):
    """psi_0 = sqrt(dim!) so that it has unit L2 norm on a simplex of volume 1/dim!."""
    pts = np.random.default_rng(0).uniform(0, 0.3, size=(5, dim))
    assert np.allclose(B.dubiner_values(dim, 3, pts)[:, 0], math.sqrt(math.factorial(dim)))


@pytest.mark.parametrize("dim,k", [(2, 5), (3, 4)])
def test_dubiner_hierarchical_span(dim, k):
    """The first dim P^m functions span P^m: monomials of degree m are reproduced exactly."""
    rng = np.random.default_rng(1)
    pts, w = Q.simplex_rule(dim, 2 * k)
    test = rng.dirichlet(np.ones(dim + 1), size=40)[:, :dim]
    for m in range(k + 1):
        n_m = B.dim_pk(dim, m)
        V = B.dubiner_values(dim, k, pts)[:, :n_m]
        Vt = B.dubiner_values(dim, k, test)[:, :n_m]
        for exps in np.ndindex(*(m + 1,) * dim):
            if sum(exps) != m:
                continue
            f = np.prod(pts ** np.array(exps), axis=1)
            coef = V.T @ (w * f)                    # orthonormal projection
            ft = np.prod(test ** np.array(exps), axis=1)
            assert np.abs(Vt @ coef - ft).max() < 1e-13


def test_dubiner_edge_restriction_is_legendre():
    """On y = 0 the modes psi_(p,0) reduce to c_p P_p(2x-1) (numpy's Legendre)."""
    x = np.linspace(0.01, 0.99, 7)
    pts = np.stack([x, np.zeros_like(x)], axis=1)
    V = B.dubiner_values(2, 5, pts)
    for j, (p, q) in enumerate(B.dubiner_indices(2, 5)):
        if q:
            continue
        c = np.zeros(p + 1)
        c[p] = 1
        ref = math.sqrt(2 * (2 * p + 1) * (p + 1)) * legendre.legval(2 * x - 1, c)
        assert np.allclose(V[:, j], ref, atol=1e-13)


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_monomial_and_collapsed_forms_agree(dim, k):
    pts = np.random.default_rng(2).dirichlet(np.ones(dim + 1), size=30)[:, :dim]
    a = B.eval_polys(B.dubiner_polys(dim, k), pts)
    b = B.dubiner_values(dim, k, pts)
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 4), (2, 6), (3, 1), (3, 2), (3, 4)])
def test_bdm_counts_and_duality(dim, k):
    """BDM_k has dim (k+1)(k+2) (2D) / (k+1)(k+2)(k+3)/2 (3D); DOFs of the basis = Id."""
    n_fm, n_int, n_w = B.hdiv_counts(dim, k)
    expect = (k + 1) * (k + 2) if dim == 2 else (k + 1) * (k + 2) * (k + 3) // 2
    assert n_w == expect
    assert len(B.nedelec_interior_fields(dim, k)) == n_int
    Cb = np.asarray(B.bdm_element(dim, k), dtype=np.float64)
    assert np.isfinite(Cb).all() and np.linalg.matrix_rank(Cb) == n_w


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 3)])
def test_nedelec_fields_are_independent_and_normalised(dim, k):
    fields = B.nedelec_interior_fields(dim, k)
    pts, w = Q.simplex_rule(dim, 2 * k)
    F = np.stack([np.concatenate([P.evaluate(t[c], pts) for c in range(dim)]) for t in fields])
    Wd = np.tile(w, dim)
    G = F @ (Wd[:, None] * F.T)
    assert np.allclose(np.diag(G), 1.0, atol=1e-13)
    assert np.linalg.matrix_rank(G, tol=1e-10) == len(fields)
