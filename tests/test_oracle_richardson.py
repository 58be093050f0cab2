"""Pins of the oracle's pseudo-time (Richardson) solve of the implicit
convection problem v + tau (M^V)^{-1} C^V v = g (Sec. 3.3.2), CPU only.

* tau = 0: the iteration is v_{i+1} = v_i + ds (g - v_i), with the closed form
  v_i = g + (1 - ds)^i (v_0 - g) and the stop index ceil(log r / log|1 - ds|);
* the fixed point is the solution of the dense linear system (Id + tau A) v = g,
  A the assembled operator, from numpy's LU solve (a sign error in tau, a
  dropped -v term or a wrong update would move it);
* the residual history follows rho_{i+1} = (Id - ds (Id + tau A)) rho_i;
* the stop rule (first index below the reduction, iteration cap, zero
  data), and the DG norm against the mass form;
* the pseudo-time step of reading A24 gives a converging iteration.
"""
import math

import numpy as np
import pytest

from oracle import dg
from oracle import hdiv as H
from oracle import mesh as OM
from paper_1508_04245_gb300 import workloads as W


def setup(dim=2, k=2, n=3, seed=4):
    if dim == 2:
        mesh = OM.Mesh(*W.square_mesh(n, 0.1, seed))
        pot = W.stream_random(seed + 10)
    else:
        mesh = OM.Mesh(*W.cube_mesh(1, 0.0, seed))
        pot = W.potential_random(seed + 10)
    u = H.wind_from_potential(mesh, k, pot)
    op = dg.ConvectionOracle(mesh, k, u)
    rng = np.random.default_rng(seed)
    shape = (mesh.n_elem, dim, op.N)
    return mesh, u, op, rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)


def test_dg_norm_is_the_mass_form():
    mesh, _, _, g, _ = setup()
    assert dg.dg_norm(mesh, g) ** 2 == pytest.approx(float(np.sum(g * dg.mass(mesh, g))), rel=1e-14)


@pytest.mark.parametrize("ds", [0.3, 0.9, 1.4])
def test_tau_zero_closed_form(ds):
    mesh, _, op, g, v0 = setup()
    red = 3e-6                                   # away from the powers of |1 - ds| (no ties)
    v, it, hist = dg.richardson(op, g, v0, 0.0, ds, red, 500)
    q = abs(1.0 - ds)
    assert it == math.ceil(math.log(red) / math.log(q) - 1e-12)
    assert np.allclose(v, g + (1.0 - ds) ** it * (v0 - g), rtol=0, atol=1e-13)
    r0 = dg.dg_norm(mesh, g - v0)
    assert np.allclose(hist, [r0 * q ** i for i in range(it + 1)], rtol=1e-10, atol=0)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 1)])
def test_fixed_point_is_the_linear_solve(dim, k):
    mesh, u, op, g, v0 = setup(dim, k)
    A = dg.assemble(op)
    tau = 0.1 * float(mesh.shortest_edge().min())
    n = A.shape[0]
    v_star = np.linalg.solve(np.eye(n) + tau * A, g.ravel())
    ds = dg.richardson_ds(mesh, k, u, tau)
    v, it, hist = dg.richardson(op, g, v0, tau, ds, 1e-13, 5000)
    assert hist[-1] <= 1e-13 * hist[0] and it < 5000
    assert np.abs(v.ravel() - v_star).max() < 1e-10 * np.abs(v_star).max()


def test_residual_history_follows_the_iteration_matrix():
    mesh, u, op, g, v0 = setup(2, 2)
    A = dg.assemble(op)
    tau = 0.5 * float(mesh.shortest_edge().min())
    ds = dg.richardson_ds(mesh, 2, u, tau)
    n = A.shape[0]
    _, it, hist = dg.richardson(op, g, v0, tau, ds, 1e-3, 40)
    P = np.eye(n) - ds * (np.eye(n) + tau * A)
    rho = g.ravel() - (np.eye(n) + tau * A) @ v0.ravel()
    for i in range(it + 1):
        assert hist[i] == pytest.approx(dg.dg_norm(mesh, rho.reshape(g.shape)), rel=1e-11)
        rho = P @ rho


def test_stop_rule_cap_and_zero_data():
    mesh, u, op, g, v0 = setup(2, 2)
    tau = 0.5 * float(mesh.shortest_edge().min())
    ds = dg.richardson_ds(mesh, 2, u, tau)
    red = 1e-4
    v, it, hist = dg.richardson(op, g, v0, tau, ds, red, 1000)
    assert len(hist) == it + 1 and hist[-1] <= red * hist[0]
    assert all(h > red * hist[0] for h in hist[:-1])
    # the iteration cap returns v_max and its residual
    v3, it3, hist3 = dg.richardson(op, g, v0, tau, ds, red, 3)
    assert it3 == 3 and np.allclose(hist3, hist[:4], rtol=1e-14)
    # zero data: zero initial residual, no iteration (the criterion is relative, so
    # any nonzero initial residual, however small, is reduced by the factor)
    z = np.zeros_like(g)
    assert dg.richardson(op, z, z, tau, ds, red, 10)[1] == 0


def test_pseudo_time_step_converges():
    """With ds = 1 / (1 + beta^2) every mode contracts; the slowest (Re = 1)
    at the rate 1 - ds, so the count grows like beta^2."""
    mesh, u, op, g, v0 = setup(2, 3, n=4)
    for tau in (0.1, 1.0):
        tau_s = tau * float(mesh.shortest_edge().min())
        ds = dg.richardson_ds(mesh, 3, u, tau_s)
        _, it, hist = dg.richardson(op, g, v0, tau_s, ds, 1e-6, 20000)
        assert hist[-1] <= 1e-6 * hist[0], (tau, it)
