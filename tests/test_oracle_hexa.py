"""Pins of the hexahedral (parallelepiped) oracle against closed forms,
invariants and brute force -- never against itself.  CPU only.

As for parallelograms: a wrong sign, transpose or flip of a face moment fails
the reconstruction of smooth fields on every face orientation or the normal
continuity; a wrong term of the operator fails the closed form u . grad w for
continuous polynomial states or the upwind energy identity.
"""
import numpy as np
import pytest

from oracle import dg as ODG
from oracle import hexa as X
from paper_1508_04245_gb300 import workloads as W


def mesh(n=2, seed=1, reorient=True):
    v, e = W.parallelepiped_mesh(n, seed, reorient=reorient)
    return X.HexMesh(v, e)


def poly_field(k, seed):
    rng = np.random.default_rng(seed)
    exps = [(p, q, r) for p in range(k + 1) for q in range(k + 1 - p) for r in range(k + 1 - p - q)]
    C = rng.normal(size=(3, len(exps)))
    return lambda x: np.stack([sum(C[c, j] * x[:, 0] ** p * x[:, 1] ** q * x[:, 2] ** r
                                   for j, (p, q, r) in enumerate(exps)) for c in range(3)], axis=1)


def test_mesh_volume_normals_pairing_and_face_codes():
    M = mesh(3, 2)
    v, e = W.parallelepiped_mesh(3, 2, reorient=False)
    vol = sum(abs(np.linalg.det(np.stack([v[q[1]] - v[q[0]], v[q[3]] - v[q[0]], v[q[4]] - v[q[0]]]))) for q in e)
    assert np.isclose(np.abs(M.detJ).sum(), vol)
    assert (M.detJ < 0).any() and (M.detJ > 0).any()
    assert len({tuple(c) for c in M.fcode.reshape(-1, 3)}) == 8
    centre = M.X.mean(axis=1)
    for el in range(M.n_elem):
        for f in range(6):
            c = X.face_corner_vertices(f)
            mid = M.X[el, c].mean(axis=0)
            assert np.dot(M.normal[el, f], mid - centre[el]) > 0
            nb = M.nbr[el, f]
            if nb >= 0:
                f2 = M.nbr_facet[el, f]
                assert M.nbr[nb, f2] == el and np.allclose(M.normal[nb, f2], -M.normal[el, f])
    assert M.n_facets == 3 * 3 * 3 * 4
    with pytest.raises(ValueError):
        bad = v.copy()
        bad[e[4, 6]] += 0.01
        X.HexMesh(bad, e)


def test_local_dof_matrix_interior_rows_are_unit_vectors():
    for k in (1, 2, 3):
        N, n_fm, n_int, n_w = X.counts(k)
        n = k + 1
        rows = X.local_dof_matrix(k)[6 * n_fm:]
        expect = np.zeros_like(rows)
        j = 0
        for d in range(3):
            for a in range(n):
                for b in range(n):
                    for c in range(n):
                        if (a, b, c)[d] <= k - 2:
                            expect[j, d * N + (a * n + b) * n + c] = 1.0
                            j += 1
        assert j == n_int and np.allclose(rows, expect, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_dofs_reconstruct_polynomial_fields_on_every_face_orientation(k):
    M = mesh(2, 5 + k)
    f = poly_field(k, k)
    u = X.dofs_of_function(M, k, f)
    xi = np.random.default_rng(k).random((5, 3))
    for el in range(M.n_elem):
        assert np.allclose(X.evaluate(M, k, u, np.full(5, el), xi), f(M.to_physical(np.full(5, el), xi)), atol=1e-11)


@pytest.mark.parametrize("k", [1, 2])
def test_random_dof_vectors_have_continuous_normal_component(k):
    M = mesh(2, 9)
    u = np.random.default_rng(5).normal(size=X.layout(M, k)[3])
    s1, s2 = np.array([0.2, 0.7, 0.4]), np.array([0.3, 0.15, 0.8])
    for g in range(M.n_facets):
        el, f = M.facet_owner[g]
        e2 = M.nbr[el, f]
        if e2 < 0:
            continue
        x = M.to_physical(np.full(3, el), X.face_point(f, s1, s2))
        ua = X.evaluate(M, k, u, np.full(3, el), M.to_reference(np.full(3, el), x)) @ M.normal[el, f]
        ub = X.evaluate(M, k, u, np.full(3, e2), M.to_reference(np.full(3, e2), x)) @ M.normal[el, f]
        assert np.allclose(ua, ub, atol=1e-11)


def test_wind_from_potential_is_the_exact_curl_and_divergence_free():
    k = 2
    M = mesh(2, 3)
    A = lambda x: np.stack([x[:, 1] * x[:, 2], 0.5 * x[:, 0] ** 2 - x[:, 2], x[:, 0] * x[:, 1] + 0.3 * x[:, 1] ** 2],   # noqa
                           axis=1)
    curl = lambda x: np.stack([x[:, 0] + 0.6 * x[:, 1] + 1.0, x[:, 1] - x[:, 1], x[:, 0] - x[:, 2]], axis=1)     # noqa
    nodes = X.lagrange_nodes(k)
    P = np.stack([A(M.to_physical(np.full(nodes.shape[0], el), nodes)) for el in range(M.n_elem)])
    u = X.wind_from_potential(M, k, P)
    xi = np.random.default_rng(0).random((4, 3))
    coef = X.ref_coeffs(M, k, u)
    G = X.vgrad(k, xi)
    for el in range(M.n_elem):
        x = M.to_physical(np.full(4, el), xi)
        assert np.allclose(X.evaluate(M, k, u, np.full(4, el), xi), curl(x), atol=1e-10)
        assert np.abs(sum(np.einsum("i,qi->q", coef[el, d], G[:, :, d]) for d in range(3))).max() < 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_transfer_is_the_embedding_and_transfer_T_its_adjoint(k):
    M = mesh(2, 4)
    rng = np.random.default_rng(k)
    u = rng.normal(size=X.layout(M, k)[3])
    w = X.transfer(M, k, u)
    xi = rng.random((5, 3))
    for el in range(M.n_elem):
        assert np.allclose(np.einsum("ci,qi->qc", w[el], X.vbasis(k, xi)), X.evaluate(M, k, u, np.full(5, el), xi),
                           atol=1e-11)
    f = rng.normal(size=w.shape)
    assert np.isclose(np.dot(X.transfer_T(M, k, f), u), np.sum(f * w), rtol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_continuous_polynomial_state_gives_u_dot_grad_w_away_from_inflow(k):
    M = mesh(3, 6)
    a = np.array([0.8, -0.55, 0.3])
    u = X.dofs_of_function(M, k, lambda x: np.tile(a, (x.shape[0], 1)))
    rng = np.random.default_rng(k)
    exps = [(p, q, r) for p in range(k + 1) for q in range(k + 1 - p) for r in range(k + 1 - p - q)]
    C = rng.normal(size=(3, len(exps)))

    def wfun(x, dd=None):
        out = []
        for c in range(3):
            acc = 0.0
            for j, e in enumerate(exps):
                if dd is None:
                    acc = acc + C[c, j] * x[:, 0] ** e[0] * x[:, 1] ** e[1] * x[:, 2] ** e[2]
                elif e[dd] > 0:
                    ee = list(e)
                    ee[dd] -= 1
                    acc = acc + C[c, j] * e[dd] * x[:, 0] ** ee[0] * x[:, 1] ** ee[1] * x[:, 2] ** ee[2]
            out.append(acc + 0 * x[:, 0])
        return np.stack(out, axis=1)

    def project(func):
        xq, wq = X.cube_rule(k + 2)
        psi = X.vbasis(k, xq)
        return np.stack([np.einsum("q,qc,qi->ci", wq, func(M.to_physical(np.full(len(wq), el), xq)), psi)
                         for el in range(M.n_elem)])
    w = project(wfun)
    expect = project(lambda x: sum(a[d] * wfun(x, d) for d in range(3)))
    r = X.HexConvectionOracle(M, k, u).apply(w)
    inner = np.all(M.nbr >= 0, axis=1)
    assert inner.sum() == 1
    assert np.allclose(r[inner], expect[inner], atol=1e-10 * (1 + np.abs(expect).max()))
    assert not np.allclose(r[~inner], expect[~inner], atol=1e-6)


@pytest.mark.parametrize("k", [1, 2])
def test_upwind_energy_identity(k):
    M = mesh(2, 8)
    nodes = X.lagrange_nodes(k)
    pot = W.potential_random(4)
    P = np.stack([np.moveaxis(np.asarray(pot(*M.to_physical(np.full(nodes.shape[0], el), nodes).T)), 0, -1)
                  for el in range(M.n_elem)])
    u = X.wind_from_potential(M, k, P)
    w = np.random.default_rng(3).uniform(-1, 1, size=(M.n_elem, 3, (k + 1) ** 3))
    r = X.HexConvectionOracle(M, k, u).apply(w)
    lhs = float(np.sum(np.abs(M.detJ)[:, None, None] * w * r))
    rhs = X.upwind_energy(M, k, u, w)
    assert rhs > 0 and abs(lhs - rhs) < 1e-10 * rhs
    ds = X.cfl_ds(M, k, u, 0.2)
    v = ODG.rk_substeps(X.HexConvectionOracle(M, k, u), w, ds, 2, 3)
    assert np.sum(np.abs(M.detJ)[:, None, None] * v * v) < np.sum(np.abs(M.detJ)[:, None, None] * w * w)
