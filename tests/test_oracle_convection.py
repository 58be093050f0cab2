"""Pins of the oracle's convection operator and explicit propagation (CPU only).

* constant states give a zero residual (div u = 0 and continuous u.n);
* the upwind energy identity w^T M^V r = 1/2 sum_F |u.n| [[w]]^2 + boundary
  term, against an independent facet-by-facet jump integral (Sec. 2.3
  stability statement);
* mass conservation when u.n = 0 on the boundary;
* the mean mode of a piecewise-constant state is the textbook first-order
  upwind finite-volume residual (golden fixture, derived by hand);
* linearity; consistency with u . grad w at the expected rate; the summand
  scale of the residual (a rounding-error scale) bounds it and grows like 1/h
  relative to it on a smooth state;
* an RK substep equals the Taylor polynomial of the assembled operator
  (SSP-RK2/3 are exact for linear autonomous ODEs up to their order);
  energy does not increase at CFL 0.2.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import basis as B
from oracle import dg
from oracle import hdiv as H
from oracle import mesh as OM
from oracle.quadrature import simplex_rule
from paper_1508_04245_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def setup(dim, k, jitter=0.1, n=None, seed=1):
    if dim == 2:
        mesh = OM.Mesh(*W.square_mesh(n or 4, jitter, seed))
        pot = W.stream_random(seed + 10)
    else:
        mesh = OM.Mesh(*W.cube_mesh(n or 2, jitter, seed))
        pot = W.potential_random(seed + 10)
    u = H.wind_from_potential(mesh, k, pot)
    return mesh, u, dg.ConvectionOracle(mesh, k, u)


CASES = [(2, 1), (2, 2), (2, 4), (2, 6), (3, 1), (3, 2), (3, 3)]


@pytest.mark.parametrize("dim,k", CASES)
def test_constant_state_has_zero_residual(dim, k):
    mesh, u, op = setup(dim, k)
    w = np.zeros((mesh.n_elem, dim, op.N))
    w[:, :, 0] = np.arange(1, dim + 1) * math.sqrt(math.factorial(dim))
    r = op.apply(w)
    scale = np.abs(op.apply(np.random.default_rng(0).uniform(-1, 1, w.shape))).max()
    assert np.abs(r).max() < 1e-12 * scale


@pytest.mark.parametrize("dim,k", CASES)
def test_upwind_energy_identity(dim, k):
    mesh, u, op = setup(dim, k)
    w = np.random.default_rng(1).uniform(-1, 1, (mesh.n_elem, dim, op.N))
    lhs = np.sum(dg.mass(mesh, w) * op.apply(w))
    rhs = dg.upwind_energy(mesh, k, u, w)
    assert rhs > 0
    assert abs(lhs - rhs) < 1e-12 * rhs


def test_energy_identity_fails_for_a_downwind_flux():
    """Negative control: the identity detects a flipped upwind choice."""
    mesh, u, op = setup(2, 2)
    w = np.random.default_rng(2).uniform(-1, 1, (mesh.n_elem, 2, op.N))
    rhs = dg.upwind_energy(mesh, 2, u, w)
    wt = op.wt.copy()
    op.wt[:] = 0.0
    r_vol = op.apply(w)                  # volume part alone
    op.wt[:] = wt
    op.un = -op.un                       # planted flip: selects the downwind trace, negates the flux
    r_down = 2.0 * r_vol - op.apply(w)   # volume + (downwind trace) flux
    lhs = np.sum(dg.mass(mesh, w) * r_down)
    assert abs(lhs + rhs) < 1e-12 * rhs  # the downwind form anti-dissipates exactly


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_mass_conservation_with_tangential_wind(dim, k):
    mesh, u, op = setup(dim, k)
    w = np.random.default_rng(3).uniform(-1, 1, (mesh.n_elem, dim, op.N))
    r = op.apply(w)
    total = np.sum(dg.mass(mesh, r)[:, :, 0], axis=0)
    assert np.abs(total).max() < 1e-12 * np.abs(r).max()


def test_mean_mode_is_finite_volume_golden():
    g = json.load(open(os.path.join(GOLDEN, "fv_two_triangles.json")))
    mesh = OM.Mesh(np.array(g["verts"]), np.array(g["elems"]))
    k = 1
    wind = np.array(g["wind"])
    u = H.dofs_of_function(mesh, k, lambda x: np.tile(wind, (x.shape[0], 1)))
    op = dg.ConvectionOracle(mesh, k, u)
    w = np.zeros((2, 2, op.N))
    w[:, 0, 0] = np.array(g["means"]) / math.sqrt(2.0)         # mean value m has coefficient m / psi_0
    r = op.apply(w)
    mean_res = r[:, 0, 0] * math.sqrt(2.0)
    assert np.allclose(mean_res, g["mean_residual"], atol=1e-13)


@pytest.mark.parametrize("dim,k", [(2, 1), (3, 2)])
def test_mean_mode_matches_finite_volume_on_jittered_mesh(dim, k):
    """Constant wind, random piecewise-constant state: r_{c,0} psi_0 = FV residual."""
    mesh = OM.Mesh(*(W.square_mesh(4, 0.1, 3) if dim == 2 else W.cube_mesh(2, 0.05, 3)))
    wind = np.array([0.7, -0.4, 0.25][:dim])
    u = H.dofs_of_function(mesh, k, lambda x: np.tile(wind, (x.shape[0], 1)))
    op = dg.ConvectionOracle(mesh, k, u)
    means = np.random.default_rng(4).uniform(-1, 1, mesh.n_elem)
    psi0 = math.sqrt(math.factorial(dim))
    w = np.zeros((mesh.n_elem, dim, op.N))
    w[:, 0, 0] = means / psi0
    r = op.apply(w)
    fv = np.zeros(mesh.n_elem)
    vol = np.abs(mesh.detJ) / math.factorial(dim)
    for e in range(mesh.n_elem):
        for f in range(dim + 1):
            flux = wind @ mesh.normal[e, f] * mesh.area[e, f]
            nb = mesh.nbr[e, f]
            up = means[e] if flux >= 0 else (means[nb] if nb >= 0 else 0.0)
            fv[e] += flux * up / vol[e]
    assert np.allclose(r[:, 0, 0] * psi0, fv, atol=1e-12)


def test_linearity_in_the_state():
    mesh, u, op = setup(2, 3)
    rng = np.random.default_rng(5)
    a, b = rng.uniform(-1, 1, (2, mesh.n_elem, 2, op.N))
    assert np.allclose(op.apply(2.5 * a - 0.5 * b), 2.5 * op.apply(a) - 0.5 * op.apply(b), atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_consistency_rate_against_u_grad_w(k):
    """r_h -> Pi_h(u . grad w) for smooth w at rate ~k in L2 (solid-body rotation wind)."""
    def rot(x):
        return 2 * np.pi * np.stack([-(x[:, 1] - 0.5), x[:, 0] - 0.5], axis=1)

    def wfun(x):
        return np.exp(-40 * ((x[:, 0] - 0.45) ** 2 + (x[:, 1] - 0.55) ** 2))

    def grad_w(x):
        g = wfun(x)
        return np.stack([-80 * (x[:, 0] - 0.45) * g, -80 * (x[:, 1] - 0.55) * g], axis=1)

    errs = []
    for n in (8, 16):
        mesh = OM.Mesh(*W.square_mesh(n, 0.0))
        u = H.dofs_of_function(mesh, k, rot)
        op = dg.ConvectionOracle(mesh, k, u)
        xq, wq = simplex_rule(2, 2 * k + 6)
        psi = B.dubiner_values(2, k, xq)
        E = mesh.n_elem
        X = mesh.to_physical(np.repeat(np.arange(E), len(wq)), np.tile(xq, (E, 1)))
        wq_vals = wfun(X).reshape(E, -1)
        adv = np.sum(rot(X) * grad_w(X), axis=1).reshape(E, -1)
        w = np.zeros((E, 2, op.N))
        w[:, 0] = np.einsum("q,eq,qi->ei", wq, wq_vals, psi)          # L2 projection (orthonormal basis)
        target = np.einsum("q,eq,qi->ei", wq, adv, psi)
        r = op.apply(w)[:, 0]
        errs.append(math.sqrt(np.sum(np.abs(mesh.detJ) * np.sum((r - target) ** 2, axis=1))))
    rate = math.log2(errs[0] / errs[1])
    assert rate > k - 0.6, (errs, rate)


def test_summand_magnitude_bounds_and_scales_with_one_over_h():
    """The summand scale bounds the residual entrywise, is absolutely homogeneous,
    and for a fixed smooth state grows like 1/h over the residual (the volume and
    facet parts each scale like |u| |w| / h while their sum stays ~ u . grad w)."""
    def rot(x):
        return 2 * np.pi * np.stack([-(x[:, 1] - 0.5), x[:, 0] - 0.5], axis=1)

    k = 2
    ratios = []
    for n in (8, 16, 32):
        mesh = OM.Mesh(*W.square_mesh(n, 0.0))
        u = H.dofs_of_function(mesh, k, rot)
        op = dg.ConvectionOracle(mesh, k, u)
        xq, wq = simplex_rule(2, 2 * k + 6)
        psi = B.dubiner_values(2, k, xq)
        E = mesh.n_elem
        X = mesh.to_physical(np.repeat(np.arange(E), len(wq)), np.tile(xq, (E, 1)))
        vals = np.stack([np.sin(2 * X[:, 0] + X[:, 1]), np.cos(X[:, 0] - 3 * X[:, 1])], axis=1).reshape(E, -1, 2)
        w = np.einsum("q,eqc,qi->eci", wq, vals, psi)
        r, m = op.apply(w), op.magnitude(w)
        assert np.all(np.abs(r) <= m * (1 + 1e-14))
        assert np.allclose(op.magnitude(-3.0 * w), 3.0 * m, rtol=1e-14)
        inner = np.all(mesh.nbr >= 0, axis=1)          # the zero inflow datum makes r ~ 1/h at the boundary
        ratios.append(m[inner].max() / np.abs(r[inner]).max())
    assert 1.6 < ratios[1] / ratios[0] < 2.4 and 1.6 < ratios[2] / ratios[1] < 2.4, ratios


@pytest.mark.parametrize("scheme", [2, 3])
def test_rk_step_is_the_taylor_polynomial(scheme):
    mesh, u, op = setup(2, 2, n=2)
    A = -dg.assemble(op)                                  # L = -(M^V)^{-1} C^V
    v = np.random.default_rng(6).uniform(-1, 1, (mesh.n_elem, 2, op.N))
    h = 0.01
    x = v.ravel()
    ref = x.copy()
    term = x.copy()
    for p in range(1, scheme + 1):
        term = h * (A @ term) / p
        ref = ref + term
    got = dg.rk_substeps(op, v, h, 1, scheme).ravel()
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dim,k,scheme", [(2, 2, 2), (2, 3, 3), (3, 2, 3)])
def test_rk_conserves_mass_and_dissipates_energy(dim, k, scheme):
    mesh, u, op = setup(dim, k)
    v = np.random.default_rng(7).uniform(-1, 1, (mesh.n_elem, dim, op.N))
    xq, _ = simplex_rule(dim, 3 * k - 1)
    umax = np.abs(dg._eval_all(mesh, k, u, xq)).max()
    ds = 0.2 * mesh.shortest_edge().min() / ((2 * k + 1) * umax)
    mass0 = np.sum(dg.mass(mesh, v)[:, :, 0], axis=0)
    energy = np.sum(dg.mass(mesh, v) * v)
    for _ in range(5):
        v = dg.rk_substeps(op, v, ds, 1, scheme)
        e_new = np.sum(dg.mass(mesh, v) * v)
        assert e_new <= energy * (1 + 1e-14)
        energy = e_new
    assert np.allclose(np.sum(dg.mass(mesh, v)[:, :, 0], axis=0), mass0, atol=1e-12)


def test_element_subset_matches_full_operator():
    mesh, u, op = setup(2, 3)
    sel = np.array([0, 5, 17, mesh.n_elem - 1])
    sub = dg.ConvectionOracle(mesh, 3, u, sel=sel)
    w = np.random.default_rng(8).uniform(-1, 1, (mesh.n_elem, 2, op.N))
    assert np.allclose(sub.apply(w), op.apply(w)[sel], atol=1e-14)


def _rotation_solve(n, k, op_scale=1.0, sigma=0.08, t_end=0.1):
    """Solid-body rotation of a narrow Gaussian through SSP-RK3 substeps of the
    propagation problem of Sec. 3.2.2 (CFL 0.2), with the L2 error at t_end
    against the closed form w(x, t) = w_0(R(-2 pi t) (x - c) + c).

    The wind u = 2 pi (-(y - 1/2), x - 1/2) is the curl of the quadratic stream
    function -pi |x - c|^2, so the interpolated wind (reading A13) is exact for
    k >= 1.  The Gaussian stays 4.4 sigma away from the boundary, where the zero
    inflow datum (reading A5) would otherwise differ from the closed form.
    ``op_scale`` multiplies the operator (a planted mistake for the pin)."""
    centre = np.array([0.5, 0.65])

    def w0(x):
        return np.exp(-np.sum((x - centre) ** 2, axis=1) / (2 * sigma ** 2))

    mesh = OM.Mesh(*W.square_mesh(n, 0.1, 3))
    u = H.wind_from_potential(mesh, k, lambda x, y: -np.pi * ((x - 0.5) ** 2 + (y - 0.5) ** 2))
    op = dg.ConvectionOracle(mesh, k, u)
    if op_scale != 1.0:
        base = op.apply
        op.apply = lambda w: op_scale * base(w)          # noqa: E731
    xq, wq = simplex_rule(2, 2 * k + 8)
    psi = B.dubiner_values(2, k, xq)
    E = mesh.n_elem
    X = mesh.to_physical(np.repeat(np.arange(E), len(wq)), np.tile(xq, (E, 1)))
    p0 = np.einsum("q,eq,qi->ei", wq, w0(X).reshape(E, -1), psi)   # L2 projection (orthonormal basis)
    v = np.stack([p0, -0.5 * p0], axis=1)                        # both components, different amplitudes
    nsteps = int(math.ceil(t_end / dg.cfl_ds(mesh, k, u, 0.2)))
    vT = dg.rk_substeps(op, v, t_end / nsteps, nsteps, 3)
    a = -2 * np.pi * t_end
    rot = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    ex = w0((X - 0.5) @ rot.T + 0.5).reshape(E, -1)
    wh = np.einsum("eci,qi->ecq", vT, psi)
    err2 = np.abs(mesh.detJ)[:, None] * wq[None, :] * ((wh[:, 0] - ex) ** 2 + (wh[:, 1] + 0.5 * ex) ** 2)
    return math.sqrt(float(err2.sum()))


@pytest.mark.parametrize("k,meshes", [(1, (16, 32)), (2, (8, 16)), (3, (8, 16))])
def test_convergence_of_solid_body_rotation_against_the_closed_form(k, meshes):
    """h^(k+1) convergence of the upwind DG transport (Sec. 2.3; the DG theory the
    paper cites for hyperbolic problems gives at least k + 1/2 in L2): the L2 error
    of the propagated state against the rotated closed form halves the mesh size
    at a rate of at least k + 1/2 (measured about k + 1 on these jittered meshes).
    A dropped term, a wrong sign, a wrong Piola or facet scaling or a low-order
    integrator leaves an error that does not converge at that rate."""
    e0, e1 = (_rotation_solve(n, k) for n in meshes)
    rate = math.log2(e0 / e1)
    assert rate >= k + 0.5, (e0, e1, rate)


def test_convergence_pin_rejects_a_one_percent_speed_error():
    """Planted mistake: the operator scaled by 1.01 (for example a wrong facet
    measure or weight normalisation) transports at the wrong speed; the error
    then stalls and the rate of the pin above falls below k + 1/2."""
    k = 2
    e0, e1 = (_rotation_solve(n, k, op_scale=1.01) for n in (8, 16))
    assert math.log2(e0 / e1) < k + 0.5, (e0, e1)
