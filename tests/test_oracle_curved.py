"""Pins of the curved-triangle oracle (remark on curved elements, Sec. 2.4) against
the pinned affine oracle (the special case of straight edges), closed forms,
invariants and brute force -- never against itself.  CPU only.

What each test would catch:
* P2 map: wrong basis, node order or Jacobian (partition of unity, nodal
  values, exact reproduction of a global quadratic map and its area);
* straight edges: any difference from the affine oracle (a wrong mass block,
  Piola factor, normal or arc length shows up here first);
* winds: a wrong pointwise Jacobian breaks the divergence-free property or the
  normal continuity across curved facets;
* transfer: the L2 projection reproduces constant fields exactly, and I^T is
  its adjoint;
* convection: constant and coordinate states give closed forms, the upwind
  energy identity and energy decay hold on curved facets.
"""
import numpy as np
import pytest

from oracle import basis as OB
from oracle import curved as C
from oracle import dg as ODG
from oracle import hdiv as OH
from oracle import mesh as OM
from oracle.quadrature import simplex_rule
from paper_1508_04245_gb300 import workloads as W


def straight(n=3, jitter=0.15, seed=4):
    v, e = W.square_mesh(n, jitter, seed)
    om = OM.Mesh(v, e)
    mids = 0.5 * (v[om.facet_verts[:, 0]] + v[om.facet_verts[:, 1]])
    return v, e, om, C.CurvedMesh(v, e, mids)


def curved(n=4, seed=3, delta=0.25):
    v, e, en = W.curved_square_mesh(n, 0.1, seed, delta)
    return C.CurvedMesh(v, e, en)


def stream_values(cm, k, psi):
    X = C.lagrange_points(cm, k)
    return psi(X[..., 0], X[..., 1])


# ----------------------------------------------------------------------------- P2 map
def test_p2_basis_partition_of_unity_and_nodal_values():
    rng = np.random.default_rng(0)
    xi = rng.random((20, 2)) * 0.5
    assert np.allclose(C.p2_values(xi).sum(axis=1), 1.0) and np.allclose(C.p2_grads(xi).sum(axis=1), 0.0)
    assert np.allclose(C.p2_values(C.REF_NODES), np.eye(6), atol=1e-15)
    h = 1e-6
    for a in range(2):
        d = np.zeros(2)
        d[a] = h
        fd = (C.p2_values(xi + d) - C.p2_values(xi - d)) / (2 * h)
        assert np.allclose(fd, C.p2_grads(xi)[:, :, a], atol=1e-8)


def test_global_quadratic_map_is_reproduced_with_its_area():
    a, b = 0.3, -0.2
    phi = lambda x: np.stack([x[..., 0] + a * x[..., 0] * x[..., 1], x[..., 1] + b * x[..., 0] ** 2], axis=-1)  # noqa
    v, e = W.square_mesh(4)
    om = OM.Mesh(v, e)
    mids = 0.5 * (v[om.facet_verts[:, 0]] + v[om.facet_verts[:, 1]])
    cm = C.CurvedMesh(phi(v), e, phi(mids))
    rng = np.random.default_rng(1)
    xi = rng.random((6, 2)) * 0.5
    for el in range(cm.n_elem):
        straight_x = om.to_physical(np.full(6, el), xi)
        assert np.allclose(cm.to_physical(np.array([el]), xi)[0], phi(straight_x), atol=1e-14)
    area = np.sum(C.CurvedMesh.mass(cm, 1)[:, 0, 0]) / 2.0              # psi_0 = sqrt(2)
    assert abs(area - (1 + a / 2 - 2 * a * b / 3)) < 1e-14
    assert cm.curved.all()


# ----------------------------------------------------------------------------- straight edges
@pytest.mark.parametrize("k", [1, 3])
def test_straight_edges_reduce_to_the_affine_oracle(k):
    v, e, om, cm = straight(3)
    pot = W.stream_random(5)
    wind = OH.wind_from_potential(om, k, pot)
    assert not cm.curved.any()
    assert np.allclose(C.wind_from_potential(cm, k, stream_values(cm, k, pot)), wind, atol=1e-12)
    assert np.allclose(cm.mass(k), np.abs(om.detJ)[:, None, None] * np.eye(OB.dim_pk(2, k)), atol=1e-15)
    w = W.uniform_coeffs(2, om.n_elem, 2, k)
    ref = ODG.ConvectionOracle(om, k, wind).apply(w)
    assert np.abs(C.CurvedConvectionOracle(cm, k, wind).apply(w) - ref).max() < 1e-12 * np.abs(ref).max()
    u = np.random.default_rng(3).normal(size=wind.size)
    assert np.allclose(C.transfer(cm, k, u), ODG.transfer(om, k, u), atol=1e-12)
    f = np.random.default_rng(4).normal(size=w.shape)
    assert np.allclose(C.transfer_T(cm, k, f), ODG.transfer_T(om, k, f), atol=1e-11)


# ----------------------------------------------------------------------------- winds
@pytest.mark.parametrize("k", [2, 4])
def test_winds_on_curved_elements_are_divergence_free_and_normal_continuous(k):
    cm = curved(4, 3)
    u = C.wind_from_potential(cm, k, stream_values(cm, k, W.stream_random(7)))
    rng = np.random.default_rng(k)
    h = 1e-5
    for el in np.nonzero(cm.curved)[0][:6]:
        xi = 0.2 + 0.5 * rng.random((3, 2)) * 0.5
        x = cm.to_physical(np.array([el]), xi)[0]
        div = 0.0
        for a in range(2):
            d = np.zeros(2)
            d[a] = h
            up = C.evaluate(cm, k, u, el, cm.to_reference(np.full(3, el), x + d))[:, a]
            um = C.evaluate(cm, k, u, el, cm.to_reference(np.full(3, el), x - d))[:, a]
            div = div + (up - um) / (2 * h)
        assert np.abs(div).max() < 1e-6
    s = np.array([0.15, 0.5, 0.85])
    for g in range(cm.n_facets):
        el, f = cm.base.facet_owner[g]
        e2 = cm.base.nbr[el, f]
        if e2 < 0:
            continue
        xi, x, n, L = cm.facet_points(el, f, s)
        ua = C.evaluate(cm, k, u, el, xi) @ n.T
        ub = C.evaluate(cm, k, u, e2, cm.to_reference(np.full(3, e2), x)) @ n.T
        assert np.allclose(np.diag(ua), np.diag(ub), atol=1e-11)


def test_curl_of_a_quadratic_stream_function_is_exact_for_k3():
    k = 3
    cm = curved(3, 5)
    psi = lambda x, y: 0.4 * x * x - 0.3 * x * y + 0.9 * y * y + 0.2 * x     # noqa: E731
    u = C.wind_from_potential(cm, k, stream_values(cm, k, psi))
    xi = np.array([[0.2, 0.3], [0.6, 0.1], [0.1, 0.7]])
    for el in range(cm.n_elem):
        x = cm.to_physical(np.array([el]), xi)[0]
        exact = np.stack([-0.3 * x[:, 0] + 1.8 * x[:, 1], -(0.8 * x[:, 0] - 0.3 * x[:, 1] + 0.2)], axis=1)
        assert np.allclose(C.evaluate(cm, k, u, el, xi), exact, atol=1e-11)


# ----------------------------------------------------------------------------- transfer
@pytest.mark.parametrize("k", [1, 2, 4])
def test_transfer_projects_constant_fields_exactly_and_transfer_T_is_adjoint(k):
    cm = curved(3, 8)
    c = np.array([0.7, -1.3])
    u = C.dofs_of_field(cm, k, lambda e, xi: np.tile(c, (xi.shape[0], 1)))
    w = C.transfer(cm, k, u)
    expect = np.zeros_like(w)
    expect[:, :, 0] = c / np.sqrt(2.0)                                      # psi_0 = sqrt(2)
    assert np.allclose(w, expect, atol=1e-12)
    rng = np.random.default_rng(k)
    uu = rng.normal(size=u.size)
    f = rng.normal(size=w.shape)
    assert np.isclose(np.dot(C.transfer_T(cm, k, f), uu), np.sum(f * C.transfer(cm, k, uu)), rtol=1e-11)


# ----------------------------------------------------------------------------- convection
def interior(cm):
    return np.all(cm.base.nbr >= 0, axis=1)


@pytest.mark.parametrize("k", [2, 3])
def test_constant_and_coordinate_states_give_closed_forms(k):
    cm = curved(4, 11)
    u = C.wind_from_potential(cm, k, stream_values(cm, k, W.stream_random(2)))
    op = C.CurvedConvectionOracle(cm, k, u)
    N = OB.dim_pk(2, k)
    inner = interior(cm) & cm.curved
    assert inner.sum() >= 3
    w = np.zeros((cm.n_elem, 2, N))
    w[:, :, 0] = [1.5, -0.5]
    r = op.apply(w)
    assert np.abs(r[interior(cm)]).max() < 1e-11
    # the x coordinate (a P2 function of xi on every element) is continuous:
    # (M^V)^{-1} C^V x = I u restricted to its first component
    xq, wq = simplex_rule(2, 2 * k + 2)
    psi = OB.dubiner_values(2, k, xq)
    X = cm.to_physical(np.arange(cm.n_elem), xq)                           # [E, Q, 2]
    w = np.zeros((cm.n_elem, 2, N))
    w[:, 0, :] = np.einsum("q,eq,qi->ei", wq, X[..., 0], psi)               # reference-orthonormal coefficients
    r = op.apply(w)
    Iu = C.transfer(cm, k, u)
    assert np.allclose(r[inner, 0], Iu[inner, 0], atol=1e-11 * np.abs(Iu).max())
    assert np.abs(r[interior(cm), 1]).max() < 1e-11


@pytest.mark.parametrize("k", [1, 3])
def test_upwind_energy_identity_and_decay_on_curved_elements(k):
    cm = curved(3, 13)
    u = C.wind_from_potential(cm, k, stream_values(cm, k, W.stream_random(6)))
    op = C.CurvedConvectionOracle(cm, k, u)
    w = W.uniform_coeffs(7, cm.n_elem, 2, k)
    r = op.apply(w)
    lhs = float(np.einsum("eci,eij,ecj->", w, cm.mass(k), r))
    rhs = C.upwind_energy(cm, k, u, w)
    assert rhs > 0 and abs(lhs - rhs) < 1e-10 * rhs
    ds = C.cfl_ds(cm, k, u, 0.2)
    e0 = C.dg_energy(cm, k, w)
    v = w
    for _ in range(3):
        v = ODG.rk_substeps(op, v, ds, 1, 3)
        e1 = C.dg_energy(cm, k, v)
        assert e1 < e0
        e0 = e1
