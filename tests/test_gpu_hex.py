"""GPU parity of the parallelepiped path (block-per-element sum-factorised stage
kernel, W_h in [Q^k]^3) through the C-ABI against the FP64 hexahedral oracle.

Meshes: seeded parallelepipeds of varying size and shear, random vertex
numbering and a random cube symmetry per element, so all eight face
orientations and both signs of det J occur (125 elements).  Tolerances as for
simplices (reading A17).
"""
import numpy as np
import pytest

from gpu_common import TOL, maxrel
from oracle import dg as ODG
from oracle import hexa as OX
from paper_1508_04245_gb300 import build, dgconv
from paper_1508_04245_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDERS = [1, 2, 3]


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


def potential_at(M, k, pot):
    nodes = OX.lagrange_nodes(k)
    return np.stack([np.moveaxis(np.asarray(pot(*M.to_physical(np.full(nodes.shape[0], el), nodes).T)), 0, -1)
                     for el in range(M.n_elem)])


@pytest.fixture(scope="module")
def cases():
    cache = {}

    def get(k, n=5, seed=3):
        if (k, n, seed) not in cache:
            verts, elems = W.parallelepiped_mesh(n, seed + k)
            om = OX.HexMesh(verts, elems)
            pot = W.potential_random(seed + 40)
            wind = OX.wind_from_potential(om, k, potential_at(om, k, pot))
            gm = dgconv.Mesh(3, k, verts, elems, shape="hex")
            cache[(k, n, seed)] = (verts, elems, pot, om, wind, gm)
        return cache[(k, n, seed)]
    return get


def state(om, k, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(om.n_elem, 3, (k + 1) ** 3))


@pytest.mark.parametrize("k", ORDERS)
def test_wind_from_potential(cases, k):
    verts, elems, pot, om, wind, gm = cases(k)
    got = gm.wind_from_potential(cu(dgconv.potential_values(gm, pot)))
    assert maxrel(host(got), wind) < 1e-12


@pytest.mark.parametrize("k", ORDERS)
def test_transfer_and_transpose(cases, k):
    verts, elems, pot, om, wind, gm = cases(k)
    rng = np.random.default_rng(11 + k)
    u = rng.standard_normal(gm.n_hdiv)
    assert maxrel(host(gm.transfer(cu(u))), OX.transfer(om, k, u)) < 1e-12
    f = rng.standard_normal((om.n_elem, 3, gm.N))
    assert maxrel(host(gm.transfer_T(cu(f))), OX.transfer_T(om, k, f)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", ORDERS)
def test_conv_apply(cases, k, prec):
    verts, elems, pot, om, wind, gm = cases(k)
    w = state(om, k, 3 + k)
    ref = OX.HexConvectionOracle(om, k, wind).apply(w)
    got = host(gm.conv_apply(cu(wind), cu(w), prec=prec))
    assert maxrel(got, ref) < TOL[prec]
    gm.check()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,scheme", [(1, 3), (2, 2), (3, 3)])
def test_rk_substeps(cases, k, scheme, prec):
    verts, elems, pot, om, wind, gm = cases(k)
    v0 = state(om, k, 20 + k)
    ds = OX.cfl_ds(om, k, wind, 0.2)
    ref = ODG.rk_substeps(OX.HexConvectionOracle(om, k, wind), v0, ds, 3, scheme)
    v = cu(v0)
    gm.rk_substeps(cu(wind), v, ds, 3, scheme, prec)
    assert maxrel(host(v), ref) < TOL[prec]


def test_interpolation_projection_mass_speed(cases):
    k = 2
    verts, elems, pot, om, wind, gm = cases(k)
    field = W.fourier_field(21, 3)
    got = host(gm.hdiv_interpolate(cu(field(gm.point_coords(2)))))
    assert maxrel(got, OX.dofs_of_function(om, k, lambda x: field(x))) < 1e-12
    xq, wq = OX.cube_rule(k + 2)
    psi = OX.vbasis(k, xq)
    pref = np.stack([np.einsum("q,qc,qi->ci", wq, field(om.to_physical(np.full(len(wq), el), xq)), psi)
                     for el in range(om.n_elem)])
    assert maxrel(host(gm.project(cu(field(gm.point_coords(1))))), pref) < 1e-12
    v = state(om, k, 8)
    assert maxrel(host(gm.mass(cu(v))), np.abs(om.detJ)[:, None, None] * v) < 1e-14
    ref = OX.max_wind_speed(om, k, wind)
    assert abs(gm.max_wind_speed(cu(wind)) - ref) < 1e-12 * ref
    assert gm.min_edge() == pytest.approx(float(om.shortest_edge().min()), rel=1e-15)


def test_richardson_and_oifs(cases):
    k = 2
    verts, elems, pot, om, wind, gm = cases(k)
    op = OX.HexConvectionOracle(om, k, wind)
    g = state(om, k, 31)
    tau = 2.0 * OX.cfl_ds(om, k, wind, 0.2)
    beta = tau * (2 * k + 1) * OX.max_wind_speed(om, k, wind) / float(om.shortest_edge().min())
    ds = 1.0 / (1.0 + beta * beta)
    ref, it_ref, hist = ODG.richardson(op, g, np.zeros_like(g), tau, ds, 1e-3, 60)
    v = cu(np.zeros_like(g))
    iters, res = gm.richardson(cu(wind), cu(g), v, tau, ds, 1e-3, 60, "fp64")
    assert int(host(iters)[0]) == it_ref and maxrel(host(v), ref) < 1e-12
    u = np.random.default_rng(9).standard_normal(gm.n_hdiv)
    dss = OX.cfl_ds(om, k, wind, 0.2)
    vv = ODG.rk_substeps(op, OX.transfer(om, k, u), dss, 2, 3)
    expect = OX.transfer_T(om, k, np.abs(om.detJ)[:, None, None] * vv)
    assert maxrel(host(gm.oifs_rhs(cu(u), cu(wind), dss, 2, 3, "fp64")), expect) < 1e-11


def test_rejections(cases):
    verts, elems, pot, om, wind, gm = cases(1)
    w = cu(state(om, 1, 1))
    for prec in ("tf32x3", "bf16x3"):
        with pytest.raises(dgconv.DgcError):
            gm.conv_apply(cu(wind), w, prec=prec)
    with pytest.raises(dgconv.DgcError):
        dgconv.Mesh(3, 4, verts, elems, shape="hex")
    bad = verts.copy()
    bad[elems[7, 6]] += np.array([0.011, -0.004, 0.002])
    with pytest.raises(dgconv.DgcError):
        dgconv.Mesh(3, 1, bad, elems, shape="hex")
