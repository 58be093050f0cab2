"""GPU parity of the parallelogram path (sum-factorised stage kernel, W_h in
[Q^k]^2) through the C-ABI against the FP64 quadrilateral oracle.

Meshes are seeded parallelograms of varying size and shear with random vertex
numbering, random starting corners and both senses of rotation, so every facet
orientation and both signs of det J occur; 81 elements give 162 threads, two
blocks with a ragged tail.  Tolerances as for simplices (reading A17): 1e-12
for FP64, 1e-5 for FP32 contractions with FP64 stage accumulation.
"""
import numpy as np
import pytest

from gpu_common import TOL, maxrel
from oracle import dg as ODG
from oracle import quad as OQ
from paper_1508_04245_gb300 import build, dgconv
from paper_1508_04245_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDERS = list(range(1, 7))


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

    def get(k, n=9, seed=3):
        if (k, n, seed) not in cache:
            verts, elems = W.parallelogram_mesh(n, seed + k)
            om = OQ.QuadMesh(verts, elems)
            pot = W.stream_random(seed + 40)
            nodes = OQ.lagrange_nodes(k)
            X = np.stack([om.to_physical(np.full(nodes.shape[0], e), nodes) for e in range(om.n_elem)])
            wind = OQ.wind_from_potential(om, k, pot(X[..., 0], X[..., 1]))
            gm = dgconv.Mesh(2, k, verts, elems, shape="quad")
            cache[(k, n, seed)] = (verts, elems, pot, om, wind, gm)
        return cache[(k, n, seed)]
    return get


def test_sizes_and_layout(cases):
    verts, elems, pot, om, wind, gm = cases(3)
    assert gm.N == 16 and gm.n_fm == 4 and gm.n_int == 2 * 4 * 2
    assert gm.n_hdiv == om.n_facets * 4 + om.n_elem * 16 and gm.n_dg == om.n_elem * 2 * 16


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
    assert maxrel(host(gm.transfer(cu(u))), OQ.transfer(om, k, u)) < 1e-12
    f = rng.standard_normal((om.n_elem, 2, gm.N))
    assert maxrel(host(gm.transfer_T(cu(f))), OQ.transfer_T(om, k, f)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", ORDERS)
def test_conv_apply(cases, k, prec):
    verts, elems, pot, om, wind, gm = cases(k)
    w = W.tensor_coeffs(3 + k, om.n_elem, k)
    ref = OQ.QuadConvectionOracle(om, k, wind).apply(w)
    got = host(gm.conv_apply(cu(wind), cu(w), prec=prec))
    assert maxrel(got, ref) < TOL[prec]
    gm.check()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,scheme", [(1, 3), (2, 2), (3, 3), (4, 3), (5, 2), (6, 3)])
def test_rk_substeps(cases, k, scheme, prec):
    verts, elems, pot, om, wind, gm = cases(k)
    v0 = W.tensor_coeffs(20 + k, om.n_elem, k)
    ds = OQ.cfl_ds(om, k, wind, 0.2)
    ref = ODG.rk_substeps(OQ.QuadConvectionOracle(om, k, wind), v0, ds, 4, scheme)
    v = cu(v0)
    gm.rk_substeps(cu(wind), v, ds, 4, scheme, prec)
    assert maxrel(host(v), ref) < TOL[prec]
    gm.check()


@pytest.mark.parametrize("k", [2, 5])
def test_hdiv_interpolate_and_project(cases, k):
    verts, elems, pot, om, wind, gm = cases(k)
    field = W.fourier_field(21, 2)
    got = host(gm.hdiv_interpolate(cu(field(gm.point_coords(2)))))
    assert maxrel(got, OQ.dofs_of_function(om, k, lambda x: field(x))) < 1e-12
    # projection: w_{c,i} = sum_q w_q f_c(x_q) psi_i(xi_q) on the (k+2)^2 Gauss rule
    xq, wq = OQ.square_rule(k + 2)
    psi = OQ.vbasis(k, xq)
    pref = np.stack([np.einsum("q,qc,qi->ci", wq, field(om.to_physical(np.full(len(wq), e), xq)), psi)
                     for e in range(om.n_elem)])
    assert maxrel(host(gm.project(cu(field(gm.point_coords(1))))), pref) < 1e-12


def test_mass_speed_edge_and_geometry(cases):
    verts, elems, pot, om, wind, gm = cases(4)
    v = W.tensor_coeffs(8, om.n_elem, 4)
    gm.geometry()
    assert maxrel(host(gm.mass(cu(v))), np.abs(om.detJ)[:, None, None] * v) < 1e-14
    ref = OQ.max_wind_speed(om, 4, wind)
    assert abs(gm.max_wind_speed(cu(wind)) - ref) < 1e-12 * ref
    assert gm.min_edge() == pytest.approx(float(om.shortest_edge().min()), rel=1e-15)


def test_richardson_on_parallelograms(cases):
    k = 3
    verts, elems, pot, om, wind, gm = cases(k)
    op = OQ.QuadConvectionOracle(om, k, wind)
    g = W.tensor_coeffs(31, om.n_elem, k)
    tau = 2.0 * OQ.cfl_ds(om, k, wind, 0.2)
    beta = tau * (2 * k + 1) * OQ.max_wind_speed(om, k, wind) / float(om.shortest_edge().min())
    ds = 1.0 / (1.0 + beta * beta)
    ref, it_ref, hist = ODG.richardson(op, g, np.zeros_like(g), tau, ds, 1e-3, 60)
    v = cu(np.zeros_like(g))
    iters, res = gm.richardson(cu(wind), cu(g), v, tau, ds, 1e-3, 60, "fp64")
    assert int(host(iters)[0]) == it_ref
    assert maxrel(host(v), ref) < 1e-12
    assert maxrel(host(res)[:it_ref + 1], hist) < 1e-12


def test_oifs_rhs_on_parallelograms(cases):
    k = 2
    verts, elems, pot, om, wind, gm = cases(k)
    u = np.random.default_rng(9).standard_normal(gm.n_hdiv)
    ds = OQ.cfl_ds(om, k, wind, 0.2)
    v = ODG.rk_substeps(OQ.QuadConvectionOracle(om, k, wind), OQ.transfer(om, k, u), ds, 3, 3)
    ref = OQ.transfer_T(om, k, np.abs(om.detJ)[:, None, None] * v)
    got = host(gm.oifs_rhs(cu(u), cu(wind), ds, 3, 3, "fp64"))
    assert maxrel(got, ref) < 1e-11


def test_rejections(cases):
    verts, elems, pot, om, wind, gm = cases(2)
    w = cu(W.tensor_coeffs(1, om.n_elem, 2))
    for prec in ("tf32x3", "bf16x3"):
        with pytest.raises(dgconv.DgcError):
            gm.conv_apply(cu(wind), w, prec=prec)
    bad = verts.copy()
    bad[elems[4, 2]] += np.array([0.013, -0.007])
    with pytest.raises(dgconv.DgcError):
        dgconv.Mesh(2, 2, bad, elems, shape="quad")
    with pytest.raises(dgconv.DgcError):
        dgconv.Mesh(2, 7, verts, elems, shape="quad")
    assert gm.autotune(cu(wind), "fp64") == 0
