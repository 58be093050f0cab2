"""Pins of the oracle's H(div) space, divergence-free winds and transfer operators.

Against closed forms (polynomial fields are reproduced exactly by BDM_k and
by V_h), against properties the paper states (normal continuity of W_h,
div W_h-fields from curls are zero, W_h is embedded in V_h, I^T is the
transpose of I, M^U = I^T M^V I), and against a direct assembly of M^U.
"""
import numpy as np
import pytest

from oracle import basis as B
from oracle import dg
from oracle import hdiv as H
from oracle import mesh as OM
from oracle import polynomials as P
from paper_1508_04245_gb300 import workloads as W


def small_mesh(dim, jitter=0.1, n=None, seed=1):
    if dim == 2:
        return OM.Mesh(*W.square_mesh(n or 3, jitter, seed))
    return OM.Mesh(*W.cube_mesh(n or 2, jitter, seed))


def poly_field(dim, k, seed=0):
    """A random global polynomial vector field of degree k (closed form)."""
    rng = np.random.default_rng(seed)
    exps = [e for e in np.ndindex(*(k + 1,) * dim) if sum(e) <= k]
    C = rng.standard_normal((dim, len(exps)))
    E = np.array(exps)

    def f(x):
        mon = np.prod(x[:, None, :] ** E[None, :, :], axis=2)     # [M, n_exp]
        return mon @ C.T
    return f


def random_points(mesh, count, seed=3):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, mesh.n_elem, size=count)
    xi = rng.dirichlet(np.ones(mesh.dim + 1), size=count)[:, :mesh.dim]
    return e, xi


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (2, 5), (3, 1), (3, 3)])
def test_bdm_reproduces_polynomial_fields(dim, k):
    mesh = small_mesh(dim)
    f = poly_field(dim, k)
    u = H.dofs_of_function(mesh, k, f)
    e, xi = random_points(mesh, 60)
    got = H.evaluate(mesh, k, u, e, xi)
    ref = f(mesh.to_physical(e, xi))
    assert np.abs(got - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 2)])
def test_random_hdiv_vector_has_continuous_normal_component(dim, k):
    mesh = small_mesh(dim)
    _, _, _, n = H.layout(mesh, k)
    u = np.random.default_rng(4).standard_normal(n)
    s = np.random.default_rng(5).dirichlet(np.ones(dim), size=6)[:, : dim - 1]
    checked = 0
    for e in range(mesh.n_elem):
        for f in range(dim + 1):
            e2 = mesh.nbr[e, f]
            if e2 < e:
                continue
            fv = [v for v in range(dim + 1) if v != f]
            X = mesh.X[e]
            x = X[fv[0]] + s @ (X[fv[1:]] - X[fv[0]])
            ua = H.evaluate(mesh, k, u, np.full(len(s), e), mesh.to_reference(np.full(len(s), e), x))
            ub = H.evaluate(mesh, k, u, np.full(len(s), e2), mesh.to_reference(np.full(len(s), e2), x))
            nrm = mesh.normal[e, f]
            assert np.abs((ua - ub) @ nrm).max() < 1e-11
            checked += 1
    assert checked > 0


def divergence(mesh, k, u, e, xi):
    """div u = (1/det J) div^ u^ at reference points (Piola), by the Dubiner gradients."""
    d = mesh.dim
    coef = H.ref_coeffs(mesh, k, u, sel=e)
    grads = B.grad_polys(B.dubiner_polys(d, k), d)
    dv = np.zeros(len(e))
    for i, g in enumerate(grads):
        for c in range(d):
            dv += coef[:, c, i] * P.evaluate(g[c], xi)
    return dv / mesh.detJ[e]


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 4), (3, 2), (3, 3)])
def test_wind_from_potential_is_divergence_free_and_tangential(dim, k):
    mesh = small_mesh(dim)
    pot = W.stream_random(7) if dim == 2 else W.potential_random(7)
    u = H.wind_from_potential(mesh, k, pot)
    e, xi = random_points(mesh, 50)
    assert np.abs(divergence(mesh, k, u, e, xi)).max() < 1e-10
    # u . n = 0 on the boundary of the unit square / cube: the boundary facet DOFs vanish
    n_fm = H.layout(mesh, k)[0]
    bnd = np.nonzero(mesh.nbr[mesh.facet_owner[:, 0], mesh.facet_owner[:, 1]] < 0)[0]
    assert np.abs(u[(bnd[:, None] * n_fm + np.arange(n_fm)).ravel()]).max() < 1e-12


def test_wind_from_polynomial_stream_function_is_its_exact_curl():
    """psi of degree k+1 is interpolated exactly, so u = curl psi exactly (closed form)."""
    k = 3
    mesh = small_mesh(2)
    psi = lambda x, y: x ** 2 * y * (1 - y) + 0.5 * x * y ** 3            # noqa: E731, degree 4
    curl = lambda x: np.stack([x[:, 0] ** 2 * (1 - 2 * x[:, 1]) + 1.5 * x[:, 0] * x[:, 1] ** 2,
                               -(2 * x[:, 0] * x[:, 1] * (1 - x[:, 1]) + 0.5 * x[:, 1] ** 3)], axis=1)  # noqa: E731
    u = H.wind_from_potential(mesh, k, psi)
    e, xi = random_points(mesh, 40)
    assert np.abs(H.evaluate(mesh, k, u, e, xi) - curl(mesh.to_physical(e, xi))).max() < 1e-12


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 4), (3, 2)])
def test_transfer_is_the_embedding(dim, k):
    """I u evaluated in V_h equals u evaluated in W_h (W_h subset V_h on affine meshes)."""
    mesh = small_mesh(dim)
    _, _, _, n = H.layout(mesh, k)
    u = np.random.default_rng(8).standard_normal(n)
    w = dg.transfer(mesh, k, u)
    e, xi = random_points(mesh, 50)
    wv = np.einsum("mci,mi->mc", w[e], B.dubiner_values(dim, k, xi))
    assert np.abs(wv - H.evaluate(mesh, k, u, e, xi)).max() < 1e-11 * np.abs(wv).max()


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_transfer_T_is_the_adjoint(dim, k):
    mesh = small_mesh(dim)
    _, _, _, n = H.layout(mesh, k)
    rng = np.random.default_rng(9)
    g = rng.standard_normal(n)
    f = rng.standard_normal((mesh.n_elem, dim, B.dim_pk(dim, k)))
    lhs = g @ dg.transfer_T(mesh, k, f)
    rhs = np.sum(dg.transfer(mesh, k, g) * f)
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("dim,k", [(2, 2), (3, 1)])
def test_mass_identity_MU_equals_IT_MV_I(dim, k):
    """M^U = I^T M^V I, with M^U assembled directly from the global basis functions."""
    mesh = small_mesh(dim, n=2)
    _, _, _, n = H.layout(mesh, k)
    from oracle.quadrature import simplex_rule
    xq, wq = simplex_rule(dim, 2 * k)
    # field values of every global basis function at every element's quadrature points
    F = np.empty((n, mesh.n_elem, len(wq), dim))
    for g in range(n):
        eg = np.zeros(n)
        eg[g] = 1
        F[g] = dg._eval_all(mesh, k, eg, xq)
    MU = np.einsum("geqa,heqa,q,e->gh", F, F, wq, np.abs(mesh.detJ))
    IT_MV_I = np.stack([dg.transfer_T(mesh, k, dg.mass(mesh, dg.transfer(mesh, k, np.eye(n)[h])))
                        for h in range(n)], axis=1)
    assert np.abs(IT_MV_I - MU).max() < 1e-12 * np.abs(MU).max()


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_dofs_restricted_to_an_element_partition_add_up(dim, k):
    """The element-subset restriction of the DOF builders (used to split large
    meshes over processes) computes each entry as the full call does: the
    restrictions to a partition of the elements sum to the full vector (up to
    the summation order numpy picks for a batch of another size)."""
    mesh = OM.Mesh(*(W.square_mesh(5, 0.1, 2) if dim == 2 else W.cube_mesh(2, 0.05, 2)))
    pot = W.stream_random(3) if dim == 2 else W.potential_random(3)
    full = H.wind_from_potential(mesh, k, pot)
    parts = np.array_split(np.random.default_rng(1).permutation(mesh.n_elem), 3)
    tol = 4 * np.finfo(np.float64).eps
    got = sum(H.wind_from_potential(mesh, k, pot, elems=p) for p in parts)
    assert np.abs(got - full).max() <= tol * np.abs(full).max()
    field = W.fourier_field(4, dim)
    full_f = H.dofs_of_function(mesh, k, field)
    got_f = sum(H.dofs_of_function(mesh, k, field, elems=p) for p in parts)
    assert np.abs(got_f - full_f).max() <= tol * np.abs(full_f).max()


def test_transfer_restricted_to_elements_matches_the_full_transfer():
    mesh = OM.Mesh(*W.square_mesh(9, 0.1, 3))
    u = np.random.default_rng(2).standard_normal(H.layout(mesh, 3)[3])
    full = dg.transfer(mesh, 3, u)
    for sel in (np.array([0, 5, mesh.n_elem - 1]), np.arange(70, 150)):
        assert np.allclose(dg.transfer(mesh, 3, u, sel=sel), full[sel], rtol=0, atol=1e-14 * np.abs(full).max())
