"""Pins of the oracle's mass and energy integrals (the conserved and the
dissipated quantity of Sec. 2.3) against closed forms.

A polynomial field of degree <= k is represented exactly by its DG
coefficients; those are fitted here by least squares at many points per
element, independently of the integration rule under test, and the integrals
are compared with the exact values over the domain: the unit square or cube
for simplices and curved triangles, and per-element centroid formulas
(|P| times the mean vertex) for parallelograms and parallelepipeds.
"""
import numpy as np
import pytest

from oracle import basis as B
from oracle import curved as C
from oracle import dg as ODG
from oracle import hexa as OX
from oracle import mesh as OM
from oracle import quad as OQ
from oracle.quadrature import simplex_rule
from paper_1508_04245_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def fit(psi, x_of_e, f, n_elem, dim):
    """DG coefficients [E, dim, N] of f by least squares at the points of each element."""
    out = np.zeros((n_elem, dim, psi.shape[1]))
    for e in range(n_elem):
        vals = f(x_of_e(e))                                   # [Q, dim]
        out[e] = np.linalg.lstsq(psi, vals, rcond=None)[0].T
    return out


def field_linear(x):
    return x.copy()


def field_quadratic(x):
    if x.shape[1] == 2:
        return np.stack([x[:, 0] ** 2, x[:, 0] * x[:, 1]], axis=1)
    return np.stack([x[:, 0] ** 2, x[:, 1] * x[:, 2], np.ones(len(x))], axis=1)


# exact integrals over the unit square / cube
EXACT = {
    (2, "linear"): ([0.5, 0.5], 2.0 / 3.0),
    (3, "linear"): ([0.5, 0.5, 0.5], 1.0),
    (2, "quadratic"): ([1.0 / 3.0, 0.25], 1.0 / 5.0 + 1.0 / 9.0),
    (3, "quadratic"): ([1.0 / 3.0, 0.25, 1.0], 1.0 / 5.0 + 1.0 / 9.0 + 1.0),
}


@pytest.mark.parametrize("dim,k,kind", [(2, 1, "linear"), (2, 3, "quadratic"), (3, 1, "linear"),
                                        (3, 2, "quadratic"), (3, 4, "quadratic")])
def test_simplex_integrals_closed_forms(dim, k, kind):
    verts, elems = W.square_mesh(5, 0.1, 3) if dim == 2 else W.cube_mesh(2, 0.05, 3)
    om = OM.Mesh(verts, elems)
    xi, _ = simplex_rule(dim, 2 * k + 4)
    psi = B.dubiner_values(dim, k, xi)
    f = field_linear if kind == "linear" else field_quadratic
    w = fit(psi, lambda e: om.to_physical(np.full(len(xi), e), xi), f, om.n_elem, dim)
    mass, energy = ODG.integrals(om, k, w)
    m_ex, e_ex = EXACT[(dim, kind)]
    assert np.allclose(mass, m_ex, rtol=0, atol=1e-12)
    assert energy == pytest.approx(e_ex, rel=1e-12)


def test_simplex_integrals_of_a_random_field_scale_with_the_element():
    """A reference-element field: the integral over T is |det J| times the
    reference one, computed here by a rule of much higher degree."""
    verts, elems = W.cube_mesh(2, 0.05, 5)
    om = OM.Mesh(verts, elems)
    k = 3
    w = np.random.default_rng(4).uniform(-1, 1, (om.n_elem, 3, B.dubiner_values(3, k, np.zeros((1, 3))).shape[1]))
    xi, wq = simplex_rule(3, 4 * k + 3)
    vals = np.einsum("eci,qi->ecq", w, B.dubiner_values(3, k, xi))
    ref_mass = np.einsum("e,q,ecq->c", np.abs(om.detJ), wq, vals)
    ref_energy = np.einsum("e,q,ecq->", np.abs(om.detJ), wq, vals ** 2)
    mass, energy = ODG.integrals(om, k, w)
    assert np.allclose(mass, ref_mass, rtol=1e-13, atol=1e-15)
    assert energy == pytest.approx(ref_energy, rel=1e-13)


@pytest.mark.parametrize("shape", ["quad", "hex"])
def test_tensor_element_integrals_closed_forms(shape):
    if shape == "quad":
        verts, elems = W.parallelogram_mesh(4, 3)
        om, O, dim, k = OQ.QuadMesh(verts, elems), OQ, 2, 2
        pts, _ = OQ.square_rule(k + 3)
    else:
        verts, elems = W.parallelepiped_mesh(2, 3)
        om, O, dim, k = OX.HexMesh(verts, elems), OX, 3, 1
        pts, _ = OX.cube_rule(k + 3)
    psi = O.vbasis(k, pts)
    w = fit(psi, lambda e: om.to_physical(np.full(len(pts), e), pts), field_linear, om.n_elem, dim)
    mass, energy = O.integrals(om, k, w)
    # int_P x dx = |P| times the centroid (the mean of the vertices of a parallelotope)
    X = np.asarray(verts)[np.asarray(elems)]                   # [E, 2^dim, dim]
    vol = np.abs(om.detJ)
    m_ex = np.einsum("e,ec->c", vol, X.mean(axis=1))
    assert np.allclose(mass, m_ex, rtol=1e-12, atol=1e-14)
    assert vol.sum() == pytest.approx(1.0, rel=1e-12)
    # energy of the constant field 1 in every component: dim times the measure
    ones = fit(psi, lambda e: om.to_physical(np.full(len(pts), e), pts),
               lambda x: np.ones_like(x), om.n_elem, dim)
    assert O.integrals(om, k, ones)[1] == pytest.approx(dim * 1.0, rel=1e-12)


def test_curved_integrals_closed_forms():
    """Curved triangles filling the unit square: a field that is linear in x is
    quadratic in the reference coordinates, so k = 2 represents it exactly."""
    verts, elems, en = W.curved_square_mesh(5, 0.1, 3)
    cm = C.CurvedMesh(verts, elems, en)
    k = 2
    xi, _ = simplex_rule(2, 2 * k + 4)
    psi = B.dubiner_values(2, k, xi)
    w = fit(psi, lambda e: cm.to_physical(np.array([e]), xi)[0], field_linear, cm.n_elem, 2)
    mass, energy = C.integrals(cm, k, w)
    assert np.allclose(mass, [0.5, 0.5], rtol=0, atol=1e-12)
    assert energy == pytest.approx(2.0 / 3.0, rel=1e-12)
