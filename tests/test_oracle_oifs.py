"""Pins of the oracle's H(div)-side compositions (CPU only):

* C^U = I^T C^V I (Sec. 2.4): u . C^U u equals the upwind energy of I u, an
  independent facet-by-facet jump integral (Sec. 2.3 stability statement), and
  a constant field has zero convection;
* the OIFS right-hand side I^T M^V Q I u (Sec. 3.2): without substeps,
  z . (I^T M^V I u) is the L2 product of the two H(div) fields by direct
  quadrature; with a tangential wind (frozen or extrapolated) the functional
  against a constant field is conserved over the substeps;
* the extrapolation weights (reading A25) are consistent (sum 1), give 2u^n -
  u^{n-1} one previous step ahead, and a steady wind reproduces the frozen run.
"""
import numpy as np
import pytest

from oracle import dg
from oracle import hdiv as H
from oracle import mesh as OM
from oracle.quadrature import simplex_rule
from paper_1508_04245_gb300 import workloads as W


def setup(dim=2, k=2, n=3, seed=3):
    if dim == 2:
        mesh = OM.Mesh(*W.square_mesh(n, 0.1, seed))
        pots = [W.stream_random(seed + 10), W.stream_random(seed + 11)]
    else:
        mesh = OM.Mesh(*W.cube_mesh(1, 0.0, seed))
        pots = [W.potential_random(seed + 10), W.potential_random(seed + 11)]
    winds = [H.wind_from_potential(mesh, k, p) for p in pots]
    field = W.fourier_field(seed + 20, dim)
    u = H.dofs_of_function(mesh, k, field)
    return mesh, winds, u


def l2_product(mesh, k, a, b):
    """int_Omega a_h . b_h dx by a degree-2k rule in every element (physical weights)."""
    xq, wq = simplex_rule(mesh.dim, 2 * k)
    tot = 0.0
    for e in range(mesh.n_elem):
        ee = np.full(len(wq), e)
        tot += abs(mesh.detJ[e]) * np.sum(wq * np.sum(H.evaluate(mesh, k, a, ee, xq) * H.evaluate(mesh, k, b, ee, xq),
                                                      axis=1))
    return tot


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_conv_hdiv_energy_is_the_upwind_jump_integral(dim, k):
    mesh, winds, u = setup(dim, k)
    op = dg.ConvectionOracle(mesh, k, winds[0])
    e = float(u @ dg.conv_hdiv(op, u))
    ref = dg.upwind_energy(mesh, k, winds[0], dg.transfer(mesh, k, u))
    assert e == pytest.approx(ref, rel=1e-11, abs=1e-14)


def test_conv_hdiv_of_a_constant_field_vanishes():
    mesh, winds, _ = setup(2, 2)
    op = dg.ConvectionOracle(mesh, 2, winds[0])
    c = H.dofs_of_function(mesh, 2, lambda x: np.tile([0.3, -1.1], (x.shape[0], 1)))
    assert np.abs(dg.conv_hdiv(op, c)).max() < 1e-12


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 1)])
def test_oifs_rhs_without_substeps_is_the_hdiv_mass_form(dim, k):
    mesh, winds, u = setup(dim, k)
    z = H.dofs_of_function(mesh, k, W.fourier_field(77, dim))
    out = dg.oifs_rhs(mesh, k, u, winds[0], 0.1, 0, 3)
    assert float(z @ out) == pytest.approx(l2_product(mesh, k, z, u), rel=1e-12)


@pytest.mark.parametrize("extrapolated", [False, True])
def test_oifs_rhs_conserves_the_functional_of_a_constant_field(extrapolated):
    mesh, winds, u = setup(2, 2, n=4)
    ds = 0.2 * dg.cfl_ds(mesh, 2, winds[0], 1.0)
    c = H.dofs_of_function(mesh, 2, lambda x: np.tile([0.7, 0.4], (x.shape[0], 1)))
    base = float(c @ dg.oifs_rhs(mesh, 2, u, winds[0], ds, 0, 3))
    kw = dict(wind_prev=winds[1], dt_prev=4 * ds) if extrapolated else {}
    out = dg.oifs_rhs(mesh, 2, u, winds[0], ds, 4, 3, **kw)
    assert float(c @ out) == pytest.approx(base, rel=1e-12)
    assert not np.allclose(out, dg.oifs_rhs(mesh, 2, u, winds[0], ds, 0, 3))


def test_extrapolation_weights_and_steady_wind():
    for j, ds, dt in ((0, 0.1, 0.4), (3, 0.05, 0.2), (7, 1.0, 1.0)):
        a, b = dg.extrapolation_coefs(j, ds, dt)
        assert a + b == pytest.approx(1.0, abs=1e-15)
        assert a * 0.0 + b * (-dt) == pytest.approx((j + 0.5) * ds, rel=1e-14)   # linear in time: exact
    a, b = dg.extrapolation_coefs(0, 2.0, 1.0)
    assert (a, b) == (2.0, -1.0)
    mesh, winds, u = setup(2, 2)
    ds = 0.2 * dg.cfl_ds(mesh, 2, winds[0], 1.0)
    frozen = dg.oifs_rhs(mesh, 2, u, winds[0], ds, 3, 3)
    steady = dg.oifs_rhs(mesh, 2, u, winds[0], ds, 3, 3, wind_prev=winds[0], dt_prev=ds)
    assert np.allclose(steady, frozen, rtol=0, atol=1e-13 * np.abs(frozen).max())
    f = dg.extrapolate([winds[0], winds[1]], [2.0, -1.0])
    assert np.array_equal(f, 2.0 * winds[0] - winds[1])
