"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Sizes span several thread blocks with a ragged tail; every order the library
supports is covered in both dimensions and both contraction precisions.
Tolerances are max-norm relative errors (reading A17): 1e-12 for FP64,
1e-5 for FP32 contractions with FP64 stage accumulation.
"""
import numpy as np
import pytest

from gpu_common import TC_PRECS, TOL, make_case, maxrel, oracle_ds, oracle_state, tc_ok
from oracle import dg as ODG
from oracle import hdiv as OH
from paper_1508_04245_gb300 import build, dgconv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDERS = [(2, k) for k in range(1, 7)] + [(3, k) for k in range(1, 6)]


def mesh_n(dim, k):
    return 12 if dim == 2 else (4 if k <= 3 else 3)


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def cases():
    cache = {}

    def get(dim, k):
        if (dim, k) not in cache:
            verts, elems, pot, om, wind = make_case(dim, k, mesh_n(dim, k))
            gm = dgconv.Mesh(dim, k, verts, elems)
            cache[(dim, k)] = (verts, elems, pot, om, wind, gm)
        return cache[(dim, k)]
    return get


@pytest.mark.parametrize("dim,k", ORDERS)
def test_wind_from_potential(cases, dim, k):
    verts, elems, pot, om, wind, gm = cases(dim, k)
    got = gm.wind_from_potential(cu(dgconv.potential_values(gm, pot)))
    assert maxrel(host(got), wind) < 1e-12


@pytest.mark.parametrize("dim,k", ORDERS)
def test_transfer(cases, dim, k):
    verts, elems, pot, om, wind, gm = cases(dim, k)
    u = np.random.default_rng(11).standard_normal(gm.n_hdiv)
    assert maxrel(host(gm.transfer(cu(u))), ODG.transfer(om, k, u)) < 1e-12


@pytest.mark.parametrize("dim,k", ORDERS)
def test_transfer_T(cases, dim, k):
    verts, elems, pot, om, wind, gm = cases(dim, k)
    f = np.random.default_rng(12).standard_normal((om.n_elem, dim, gm.N))
    assert maxrel(host(gm.transfer_T(cu(f))), ODG.transfer_T(om, k, f)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("dim,k", ORDERS)
def test_conv_apply(cases, dim, k, prec):
    if prec in TC_PRECS and not tc_ok(dim, k, prec):
        pytest.skip("tensor-core paths: triangles k <= 6, tetrahedra k <= 4 in bf16x3")
    verts, elems, pot, om, wind, gm = cases(dim, k)
    w = oracle_state(om, k)
    ref = ODG.ConvectionOracle(om, k, wind).apply(w)
    got = host(gm.conv_apply(cu(wind), cu(w), prec=prec))
    assert maxrel(got, ref) < TOL[prec]
    gm.check()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("dim,k,scheme", [(2, 1, 3), (2, 2, 2), (2, 3, 3), (2, 4, 3), (2, 6, 3), (3, 1, 2), (3, 3, 3),
                                          (3, 4, 3)])
def test_rk_substeps(cases, dim, k, scheme, prec):
    if prec in TC_PRECS and not tc_ok(dim, k, prec):
        pytest.skip("tensor-core paths: triangles k <= 6, tetrahedra k <= 4 in bf16x3")
    verts, elems, pot, om, wind, gm = cases(dim, k)
    v0 = oracle_state(om, k, seed=5)
    ds = oracle_ds(om, k, wind)
    op = ODG.ConvectionOracle(om, k, wind)
    ref = ODG.rk_substeps(op, v0, ds, 4, scheme)
    v = cu(v0)
    gm.rk_substeps(cu(wind), v, ds, 4, scheme, prec)
    assert maxrel(host(v), ref) < TOL[prec]
    gm.check()


def test_rk_graph_replay_matches_fresh_launch(cases):
    """A replayed graph gives bit-identical results to the first (captured) call."""
    verts, elems, pot, om, wind, gm = cases(2, 3)
    v0 = oracle_state(om, 3, seed=6)
    ds = oracle_ds(om, 3, wind)
    wt = cu(wind)
    a = cu(v0)
    gm.rk_substeps(wt, a, ds, 3, 3, "fp64")
    first = host(a).copy()
    a.copy_(cu(v0))
    gm.rk_substeps(wt, a, ds, 3, 3, "fp64")
    assert np.array_equal(host(a), first)


def test_tc_unsupported_orders_are_rejected(cases):
    """Tetrahedra k = 5 have no tensor-core path; tetrahedra take bf16x3 only."""
    for dim, k in ((3, 5),):
        verts, elems, pot, om, wind, gm = cases(dim, k)
        w = cu(oracle_state(om, k))
        for prec in TC_PRECS:
            with pytest.raises(dgconv.DgcError):
                gm.conv_apply(cu(wind), w, prec=prec)
    verts, elems, pot, om, wind, gm = cases(3, 2)
    with pytest.raises(dgconv.DgcError):
        gm.conv_apply(cu(wind), cu(oracle_state(om, 2)), prec="tf32x3")


def test_mass_and_geometry(cases):
    verts, elems, pot, om, wind, gm = cases(3, 2)
    v = oracle_state(om, 2, seed=8)
    gm.geometry()
    assert maxrel(host(gm.mass(cu(v))), ODG.mass(om, v)) < 1e-14
    assert maxrel(host(gm.mass(cu(v), inverse=True)), v / np.abs(om.detJ)[:, None, None]) < 1e-14


def test_max_wind_speed_and_min_edge(cases):
    verts, elems, pot, om, wind, gm = cases(2, 4)
    assert abs(gm.max_wind_speed(cu(wind)) - ODG.max_wind_speed(om, 4, wind)) < 1e-12 * ODG.max_wind_speed(om, 4, wind)
    assert gm.min_edge() == pytest.approx(float(om.shortest_edge().min()), rel=1e-15)


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 5), (3, 2), (3, 4)])
def test_hdiv_interpolate_and_project(cases, dim, k):
    """BDM interpolation and L2 projection of a seeded Fourier field."""
    from oracle import basis as OB
    from oracle.quadrature import simplex_rule
    from paper_1508_04245_gb300 import workloads as W
    verts, elems, pot, om, wind, gm = cases(dim, k)
    field = W.fourier_field(21, dim)
    got = host(gm.hdiv_interpolate(cu(field(gm.point_coords(2)))))
    ref = OH.dofs_of_function(om, k, lambda x: field(x))
    assert maxrel(got, ref) < 1e-12
    # projection: w_{c,i} = sum_q w_q f_c(x_q) psi_i(xi_q), degree 2k+2 collapsed rule
    xq, wq = simplex_rule(dim, 2 * k + 2)
    E = om.n_elem
    X = om.to_physical(np.repeat(np.arange(E), len(wq)), np.tile(xq, (E, 1)))
    fv = field(X).reshape(E, len(wq), dim)
    pref = np.einsum("q,eqc,qi->eci", wq, fv, OB.dubiner_values(dim, k, xq))
    pgot = host(gm.project(cu(field(gm.point_coords(1)))))
    assert maxrel(pgot, pref) < 1e-12
