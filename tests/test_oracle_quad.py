"""Pins of the quadrilateral (parallelogram) oracle against closed forms, library
routines, invariants and brute force -- never against itself.  CPU only.

What each test would catch:
* 1D rule / basis: wrong nodes, weights, normalisation or derivative;
* mesh: wrong normals, orientation flags or neighbour pairing;
* H(div) DOFs: a wrong sign (orientation, flip, det J) on any element makes
  the reconstruction of a smooth field fail there, a wrong pairing breaks the
  normal continuity;
* transfer: a transposed Piola matrix or a wrong scale fails the embedding;
* convection: a dropped term or a wrong sign fails the closed form of
  u . grad w for continuous polynomial states, a wrong upwind side or
  neighbour fails the energy identity and the conservation balance.
"""
import numpy as np
import pytest

from oracle import dg
from oracle import quad as Q
from paper_1508_04245_gb300 import workloads as W


def mesh(n=3, seed=1, reorient=True):
    v, e = W.parallelogram_mesh(n, seed, reorient=reorient)
    return Q.QuadMesh(v, e)


# ----------------------------------------------------------------------------- 1D
@pytest.mark.parametrize("m", [1, 2, 5, 10])
def test_gauss01_matches_numpy_leggauss_and_integrates_monomials(m):
    t, w = Q.gauss01(m)
    tn, wn = np.polynomial.legendre.leggauss(m)
    assert np.allclose(t, 0.5 * (tn + 1.0), atol=1e-14) and np.allclose(w, 0.5 * wn, atol=1e-14)
    for p in range(2 * m):
        assert abs(np.sum(w * t ** p) - 1.0 / (p + 1)) < 1e-14


def test_legendre_closed_forms_and_orthonormality():
    t = np.linspace(0.0, 1.0, 11)
    assert np.allclose(Q.leg(0, t), 1.0)
    assert np.allclose(Q.leg(1, t), np.sqrt(3.0) * (2 * t - 1))
    assert np.allclose(Q.leg(2, t), np.sqrt(5.0) * (6 * t * t - 6 * t + 1))
    assert np.allclose(Q.dleg(2, t), np.sqrt(5.0) * (12 * t - 6))
    assert np.allclose(Q.dleg(3, t), np.sqrt(7.0) * (60 * t * t - 60 * t + 12))
    x, w = Q.gauss01(9)
    Lm = np.stack([Q.leg(a, x) for a in range(8)])
    assert np.allclose((Lm * w) @ Lm.T, np.eye(8), atol=1e-13)


# ----------------------------------------------------------------------------- mesh
def test_mesh_geometry_normals_and_pairing():
    M = mesh(4, 3)
    v, e = W.parallelogram_mesh(4, 3, reorient=False)
    # shoelace area of every cell of the same grid without renumbering
    area = sum(0.5 * abs(sum(v[q[j]][0] * v[q[(j + 1) % 4]][1] - v[q[(j + 1) % 4]][0] * v[q[j]][1]
                             for j in range(4))) for q in e)
    assert np.isclose(np.abs(M.detJ).sum(), area)
    assert (M.detJ < 0).any() and (M.detJ > 0).any()
    assert M.flip.min() == 0 and M.flip.max() == 1
    centre = M.X.mean(axis=1)
    for e_ in range(M.n_elem):
        for f, (a, b) in enumerate(Q.F_LOC):
            mid = 0.5 * (M.X[e_, a] + M.X[e_, b])
            assert np.dot(M.normal[e_, f], mid - centre[e_]) > 0
            nb = M.nbr[e_, f]
            if nb >= 0:
                f2 = M.nbr_facet[e_, f]
                assert M.nbr[nb, f2] == e_
                assert np.allclose(M.normal[nb, f2], -M.normal[e_, f])
                assert M.orient[e_, f] * M.orient[nb, f2] == -1
    # interior facets 2 n (n-1), boundary 4 n
    assert M.n_facets == 2 * 4 * 3 + 4 * 4
    with pytest.raises(ValueError):
        bad = v.copy()
        bad[e[5, 2]] += 0.01
        Q.QuadMesh(bad, e)


# ----------------------------------------------------------------------------- H(div)
def test_local_dof_matrix_interior_rows_are_unit_vectors():
    for k in (1, 2, 4):
        N, n_fm, n_int, n_w = Q.counts(k)
        Dm = Q.local_dof_matrix(k)
        rows = Dm[4 * n_fm:]
        expect = np.zeros_like(rows)
        j = 0
        for a in range(k - 1):
            for b in range(k + 1):
                expect[j, a * (k + 1) + b] = 1.0
                j += 1
        for a in range(k + 1):
            for b in range(k - 1):
                expect[j, N + a * (k + 1) + b] = 1.0
                j += 1
        assert np.allclose(rows, expect, atol=1e-14)
        # facet moments of psi_0 e_c: n^_c of the facet times 1 for m = 0
        assert np.allclose(Dm[0:4 * n_fm:n_fm, 0], Q.N_REF[:, 0]) and np.allclose(Dm[0:4 * n_fm:n_fm, N], Q.N_REF[:, 1])
        assert abs(np.linalg.det(Dm)) > 1e-8


def poly_field(k, seed):
    """A physical polynomial field of total degree k (so in [Q^k]^2 on parallelograms)."""
    rng = np.random.default_rng(seed)
    exps = [(p, q) for p in range(k + 1) for q in range(k + 1 - p)]
    C = rng.normal(size=(2, len(exps)))

    def f(x):
        return np.stack([sum(C[c, j] * x[:, 0] ** p * x[:, 1] ** q for j, (p, q) in enumerate(exps))
                         for c in range(2)], axis=1)
    return f


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_dofs_reconstruct_polynomial_fields_on_every_orientation(k):
    M = mesh(3, 7 + k)
    f = poly_field(k, k)
    u = Q.dofs_of_function(M, k, f)
    rng = np.random.default_rng(k)
    xi = rng.random((6, 2))
    for e in range(M.n_elem):
        got = Q.evaluate(M, k, u, np.full(6, e), xi)
        assert np.allclose(got, f(M.to_physical(np.full(6, e), xi)), atol=1e-11)


@pytest.mark.parametrize("k", [1, 3])
def test_random_dof_vectors_have_continuous_normal_component(k):
    M = mesh(3, 11)
    n_hdiv = Q.layout(M, k)[3]
    u = np.random.default_rng(5).normal(size=n_hdiv)
    s = np.array([0.1, 0.45, 0.8])
    for g in range(M.n_facets):
        e, f = M.facet_owner[g]
        e2 = M.nbr[e, f]
        if e2 < 0:
            continue
        a, b = Q.F_LOC[f]
        x = M.X[e, a] + s[:, None] * (M.X[e, b] - M.X[e, a])
        ua = Q.evaluate(M, k, u, np.full(3, e), M.to_reference(np.full(3, e), x)) @ M.normal[e, f]
        ub = Q.evaluate(M, k, u, np.full(3, e2), M.to_reference(np.full(3, e2), x)) @ M.normal[e, f]
        assert np.allclose(ua, ub, atol=1e-11)


@pytest.mark.parametrize("k", [2, 4])
def test_wind_from_potential_is_the_exact_curl_and_divergence_free(k):
    M = mesh(3, 2)
    # a stream function of total degree k is reproduced by the Q^k interpolant
    psi = lambda x, y: 0.3 + x * y ** (k - 1) - 0.7 * x ** k + 1.3 * y ** 2 * (k >= 2)   # noqa: E731
    curl = lambda x, y: np.stack([(k - 1) * x * y ** (k - 2) + 2.6 * y * (k >= 2),        # noqa: E731
                                  -(y ** (k - 1) - 0.7 * k * x ** (k - 1))], axis=-1)
    nodes = Q.lagrange_nodes(k)
    X = np.stack([M.to_physical(np.full(nodes.shape[0], e), nodes) for e in range(M.n_elem)])
    u = Q.wind_from_potential(M, k, psi(X[..., 0], X[..., 1]))
    rng = np.random.default_rng(0)
    xi = rng.random((5, 2))
    coef = Q.ref_coeffs(M, k, u)
    G = Q.vgrad(k, xi)
    for e in range(M.n_elem):
        x = M.to_physical(np.full(5, e), xi)
        assert np.allclose(Q.evaluate(M, k, u, np.full(5, e), xi), curl(x[:, 0], x[:, 1]), atol=1e-10)
        div = np.einsum("i,qi->q", coef[e, 0], G[:, :, 0]) + np.einsum("i,qi->q", coef[e, 1], G[:, :, 1])
        assert np.abs(div).max() < 1e-10


# ----------------------------------------------------------------------------- transfer
@pytest.mark.parametrize("k", [1, 3])
def test_transfer_is_the_embedding_and_transfer_T_its_adjoint(k):
    M = mesh(3, 4)
    rng = np.random.default_rng(k)
    n_hdiv = Q.layout(M, k)[3]
    u = rng.normal(size=n_hdiv)
    w = Q.transfer(M, k, u)
    xi = rng.random((7, 2))
    for e in range(M.n_elem):
        dgv = np.einsum("ci,qi->qc", w[e], Q.vbasis(k, xi))
        assert np.allclose(dgv, Q.evaluate(M, k, u, np.full(7, e), xi), atol=1e-11)
    f = rng.normal(size=w.shape)
    assert np.isclose(np.dot(Q.transfer_T(M, k, f), u), np.sum(f * w), rtol=1e-12)


# ----------------------------------------------------------------------------- convection
def project(M, k, func):
    """Coefficients of the L2 projection of an analytic [E]-wise field onto V_h."""
    xq, wq = Q.square_rule(k + 2)
    psi = Q.vbasis(k, xq)
    out = np.empty((M.n_elem, 2, (k + 1) ** 2))
    for e in range(M.n_elem):
        x = M.to_physical(np.full(xq.shape[0], e), xq)
        out[e] = np.einsum("q,qc,qi->ci", wq, func(x), psi)
    return out


@pytest.mark.parametrize("k", [1, 2, 4])
def test_continuous_polynomial_state_gives_u_dot_grad_w_away_from_inflow(k):
    M = mesh(4, 9)
    a = np.array([0.8, -0.55])
    u = Q.dofs_of_function(M, k, lambda x: np.tile(a, (x.shape[0], 1)))
    rng = np.random.default_rng(k)
    exps = [(p, q) for p in range(k + 1) for q in range(k + 1 - p)]
    C = rng.normal(size=(2, len(exps)))
    wfun = lambda x: np.stack([sum(C[c, j] * x[:, 0] ** p * x[:, 1] ** q for j, (p, q) in enumerate(exps))  # noqa
                               for c in range(2)], axis=1)

    def adv(x):
        gx = np.stack([sum(C[c, j] * p * x[:, 0] ** max(p - 1, 0) * x[:, 1] ** q for j, (p, q) in enumerate(exps))
                       for c in range(2)], axis=1)
        gy = np.stack([sum(C[c, j] * q * x[:, 0] ** p * x[:, 1] ** max(q - 1, 0) for j, (p, q) in enumerate(exps))
                       for c in range(2)], axis=1)
        return a[0] * gx + a[1] * gy
    w = project(M, k, wfun)
    r = Q.QuadConvectionOracle(M, k, u).apply(w)
    expect = project(M, k, adv)
    inner = np.all(M.nbr >= 0, axis=1)
    assert inner.sum() >= 4
    assert np.allclose(r[inner], expect[inner], atol=1e-10 * (1 + np.abs(expect).max()))
    # and not the same on elements with an inflow facet (the zero datum enters there)
    assert not np.allclose(r[~inner], expect[~inner], atol=1e-6)


@pytest.mark.parametrize("k", [1, 3, 4])
def test_upwind_energy_identity_for_discontinuous_states(k):
    M = mesh(3, 13)
    nodes = Q.lagrange_nodes(k)
    X = np.stack([M.to_physical(np.full(nodes.shape[0], e), nodes) for e in range(M.n_elem)])
    u = Q.wind_from_potential(M, k, W.stream_random(3)(X[..., 0], X[..., 1]))
    w = W.tensor_coeffs(4, M.n_elem, k)
    r = Q.QuadConvectionOracle(M, k, u).apply(w)
    lhs = float(np.sum(np.abs(M.detJ)[:, None, None] * w * r))
    rhs = Q.upwind_energy(M, k, u, w)
    assert rhs > 0 and abs(lhs - rhs) < 1e-11 * rhs


@pytest.mark.parametrize("k", [2, 3])
def test_total_balance_is_the_outflow_flux(k):
    M = mesh(4, 17)
    nodes = Q.lagrange_nodes(k)
    X = np.stack([M.to_physical(np.full(nodes.shape[0], e), nodes) for e in range(M.n_elem)])
    u = Q.wind_from_potential(M, k, W.stream_random(8)(X[..., 0], X[..., 1]))
    w = W.tensor_coeffs(9, M.n_elem, k)
    r = Q.QuadConvectionOracle(M, k, u).apply(w)
    total = np.einsum("e,ec->c", np.abs(M.detJ), r[:, :, 0])       # int (M^-1 C w)_c dx, psi_0 = 1
    # the upwind trace switches sides where u . n changes sign inside a facet, so
    # the balance holds for the facet rule of the method (reading A1), not for
    # the exact integral of the kinked integrand
    s, ws = Q.gauss01(Q.n_points(k))
    flux = np.zeros(2)
    for e in range(M.n_elem):
        for f, (a, b) in enumerate(Q.F_LOC):
            if M.nbr[e, f] >= 0:
                continue
            x = M.X[e, a] + s[:, None] * (M.X[e, b] - M.X[e, a])
            xi = M.to_reference(np.full(s.size, e), x)
            un = Q.evaluate(M, k, u, np.full(s.size, e), xi) @ M.normal[e, f]
            wv = np.einsum("ci,qi->qc", w[e], Q.vbasis(k, xi))
            flux += M.length[e, f] * np.einsum("q,q,qc->c", ws, np.maximum(un, 0.0), wv)
    assert np.allclose(total, flux, atol=1e-11 * np.abs(flux).max())


def test_rk_substeps_dissipate_energy_on_quads():
    k = 3
    M = mesh(4, 21)
    nodes = Q.lagrange_nodes(k)
    X = np.stack([M.to_physical(np.full(nodes.shape[0], e), nodes) for e in range(M.n_elem)])
    u = Q.wind_from_potential(M, k, W.stream_random(2)(X[..., 0], X[..., 1]))
    op = Q.QuadConvectionOracle(M, k, u)
    ds = Q.cfl_ds(M, k, u, 0.2)
    v = W.tensor_coeffs(1, M.n_elem, k)
    energy = lambda x: float(np.sum(np.abs(M.detJ)[:, None, None] * x * x))   # noqa: E731
    e0 = energy(v)
    for _ in range(4):
        v = dg.rk_substeps(op, v, ds, 1, 3)
        e1 = energy(v)
        assert e1 < e0
        e0 = e1
