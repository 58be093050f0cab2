"""GPU parity of curved (quadratic) triangles (remark on curved elements, Sec. 2.4)
through the C-ABI against the FP64 curved oracle.

Meshes: ``curved_square_mesh`` -- jittered triangles whose edges inside a disk
carry displaced mid-nodes, so curved and affine elements mix (200 elements:
two thread blocks of the stage kernel with a ragged tail).  Tolerances as for
affine simplices (reading A17), 1e-12 for FP64 and 1e-5 for FP32 contractions.
"""
import numpy as np
import pytest

from gpu_common import TOL, maxrel
from oracle import curved as C
from oracle import dg as ODG
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

    def get(k, n=10, seed=3):
        if (k, n, seed) not in cache:
            verts, elems, en = W.curved_square_mesh(n, 0.1, seed + k)
            cm = C.CurvedMesh(verts, elems, en)
            pot = W.stream_random(seed + 70)
            X = C.lagrange_points(cm, k)
            wind = C.wind_from_potential(cm, k, pot(X[..., 0], X[..., 1]))
            gm = dgconv.Mesh(2, k, verts, elems, shape="curved", edge_nodes=en)
            cache[(k, n, seed)] = (verts, elems, en, pot, cm, wind, gm)
        return cache[(k, n, seed)]
    return get


def test_mesh_has_curved_and_affine_elements(cases):
    verts, elems, en, pot, cm, wind, gm = cases(2)
    assert 0 < cm.curved.sum() < cm.n_elem
    X = gm.point_coords(0)
    assert np.allclose(X, C.lagrange_points(cm, 2), atol=1e-14)


@pytest.mark.parametrize("k", ORDERS)
def test_wind_from_potential(cases, k):
    verts, elems, en, pot, cm, wind, gm = cases(k)
    got = gm.wind_from_potential(cu(dgconv.potential_values(gm, pot)))
    assert maxrel(host(got), wind) < 1e-12


@pytest.mark.parametrize("k", ORDERS)
def test_transfer_transpose_and_mass(cases, k):
    verts, elems, en, pot, cm, wind, gm = cases(k)
    rng = np.random.default_rng(11 + k)
    u = rng.standard_normal(gm.n_hdiv)
    assert maxrel(host(gm.transfer(cu(u))), C.transfer(cm, k, u)) < 1e-12
    f = rng.standard_normal((cm.n_elem, 2, gm.N))
    assert maxrel(host(gm.transfer_T(cu(f))), C.transfer_T(cm, k, f)) < 1e-11
    M = cm.mass(k)
    assert maxrel(host(gm.mass(cu(f))), np.einsum("eij,ecj->eci", M, f)) < 1e-13
    assert maxrel(host(gm.mass(cu(f), inverse=True)), np.linalg.solve(M[:, None], f[..., None])[..., 0]) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", ORDERS)
def test_conv_apply(cases, k, prec):
    verts, elems, en, pot, cm, wind, gm = cases(k)
    w = W.uniform_coeffs(3 + k, cm.n_elem, 2, k)
    ref = C.CurvedConvectionOracle(cm, k, wind).apply(w)
    got = host(gm.conv_apply(cu(wind), cu(w), prec=prec))
    assert maxrel(got, ref) < TOL[prec]
    gm.check()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,scheme", [(1, 3), (2, 2), (4, 3), (6, 3)])
def test_rk_substeps(cases, k, scheme, prec):
    verts, elems, en, pot, cm, wind, gm = cases(k)
    v0 = W.uniform_coeffs(20 + k, cm.n_elem, 2, k)
    ds = C.cfl_ds(cm, k, wind, 0.2)
    ref = ODG.rk_substeps(C.CurvedConvectionOracle(cm, k, wind), v0, ds, 4, scheme)
    v = cu(v0)
    gm.rk_substeps(cu(wind), v, ds, 4, scheme, prec)
    assert maxrel(host(v), ref) < TOL[prec]


def test_max_wind_speed_and_oifs(cases):
    k = 3
    verts, elems, en, pot, cm, wind, gm = cases(k)
    ref = C.max_wind_speed(cm, k, wind)
    assert abs(gm.max_wind_speed(cu(wind)) - ref) < 1e-12 * ref
    u = np.random.default_rng(9).standard_normal(gm.n_hdiv)
    ds = C.cfl_ds(cm, k, wind, 0.2)
    v = ODG.rk_substeps(C.CurvedConvectionOracle(cm, k, wind), C.transfer(cm, k, u), ds, 3, 3)
    expect = C.transfer_T(cm, k, C.mass_apply(cm, k, v))
    assert maxrel(host(gm.oifs_rhs(cu(u), cu(wind), ds, 3, 3, "fp64")), expect) < 1e-11


def test_rejections(cases):
    verts, elems, en, pot, cm, wind, gm = cases(2)
    w = cu(W.uniform_coeffs(1, cm.n_elem, 2, 2))
    for prec in ("tf32x3", "bf16x3"):
        with pytest.raises(dgconv.DgcError):
            gm.conv_apply(cu(wind), w, prec=prec)
    with pytest.raises(dgconv.DgcError):
        gm.richardson(cu(wind), w, w.clone(), 0.01, 0.5, 1e-3, 5)
    with pytest.raises(dgconv.DgcError):
        gm.project(cu(np.zeros((cm.n_elem, gm.n_proj, 2))))
    folded = en.copy()
    j = int(np.argmax(np.linalg.norm(en - 0.5 * (verts[cm.base.facet_verts[:, 0]] + verts[cm.base.facet_verts[:, 1]]),
                                     axis=1)))
    a, b = cm.base.facet_verts[j]
    folded[j] = verts[a] + 0.02 * (verts[b] - verts[a])          # mid-node next to a vertex: the map folds
    with pytest.raises(dgconv.DgcError):
        dgconv.Mesh(2, 2, verts, elems, shape="curved", edge_nodes=folded)
