"""GPU parity of the tensor-core stage kernels on meshes that exercise their
persistent multi-tile pipelines, against the FP64 oracle at the BF16x3
tolerance (1e-6 of the max norm, reading A17) with no cancellation scale:

* tetrahedra: 13182 elements = 330 tiles of 40 elements on one CTA per SM,
  so every CTA runs two or three tiles through the double-buffered TMEM
  stages; conv_apply at k = 4 on sampled elements and three SSP-RK3 substeps
  at k = 3 on the whole mesh;
* triangles: 51200 elements = 400 tiles of 128 on two CTAs per SM, so the
  one-tile-ahead refill and the two-slot ring of the triangle kernel run;
  three SSP-RK3 substeps at k = 4 on the whole mesh.

States are uniform random coefficients (every mode excited), so the residual
is not a cancellation and the plain max-norm error applies.
"""
import numpy as np
import pytest

from gpu_common import TOL, make_case, maxrel, oracle_ds, oracle_state
from oracle import dg as ODG
from paper_1508_04245_gb300 import build, dgconv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_tetrahedra_conv_apply_330_tiles_sampled():
    k = 4
    verts, elems, pot, om, wind = make_case(3, k, 13, jitter=0.05, seed=9)
    assert om.n_elem == 13182
    gm = dgconv.Mesh(3, k, verts, elems)
    w = oracle_state(om, k, seed=4)
    sel = np.random.default_rng(0).choice(om.n_elem, size=1500, replace=False)
    sel = np.unique(np.concatenate([sel, [0, 39, 40, om.n_elem - 1]]))   # tile edges and the ragged tail
    ref = ODG.ConvectionOracle(om, k, wind, sel=sel).apply(w)
    got = host(gm.conv_apply(cu(wind), cu(w), prec="bf16x3"))[sel]
    gm.check()
    assert maxrel(got, ref) < TOL["bf16x3"]


def test_tetrahedra_rk_330_tiles():
    k = 3
    verts, elems, pot, om, wind = make_case(3, k, 13, jitter=0.05, seed=9)
    gm = dgconv.Mesh(3, k, verts, elems)
    v0 = oracle_state(om, k, seed=5)
    ds = oracle_ds(om, k, wind)
    ref = ODG.rk_substeps(ODG.ConvectionOracle(om, k, wind), v0, ds, 3, 3)
    v = cu(v0)
    gm.rk_substeps(cu(wind), v, ds, 3, 3, "bf16x3")
    gm.check()
    assert maxrel(host(v), ref) < TOL["bf16x3"]


def test_triangles_rk_400_tiles():
    k = 4
    verts, elems, pot, om, wind = make_case(2, k, 160, jitter=0.1, seed=9)
    assert om.n_elem == 51200
    gm = dgconv.Mesh(2, k, verts, elems)
    v0 = oracle_state(om, k, seed=5)
    ds = oracle_ds(om, k, wind)
    ref = ODG.rk_substeps(ODG.ConvectionOracle(om, k, wind), v0, ds, 3, 3)
    for prec in ("bf16x3", "tf32x3"):
        v = cu(v0)
        gm.rk_substeps(cu(wind), v, ds, 3, 3, prec)
        gm.check()
        assert maxrel(host(v), ref) < TOL[prec], prec


def test_triangles_order6_400_tiles_one_cta_per_sm_sampled():
    """k = 6: the triangle kernel runs one CTA per SM (its shared memory and TMEM
    exceed half of the SM's) and reads its gradient table from global memory, so
    400 tiles put two or three tiles through every CTA."""
    k = 6
    verts, elems, pot, om, wind = make_case(2, k, 160, jitter=0.1, seed=9)
    gm = dgconv.Mesh(2, k, verts, elems)
    w = oracle_state(om, k, seed=4)
    sel = np.random.default_rng(0).choice(om.n_elem, size=1500, replace=False)
    sel = np.unique(np.concatenate([sel, [0, 127, 128, om.n_elem - 1]]))   # tile edges and the last element
    ref = ODG.ConvectionOracle(om, k, wind, sel=sel).apply(w)
    for prec in ("bf16x3", "tf32x3"):
        got = host(gm.conv_apply(cu(wind), cu(w), prec=prec))[sel]
        assert maxrel(got, ref) < TOL[prec], prec
    gm.check()


def test_triangles_order5_rk_169_tiles_one_cta_per_sm():
    k = 5
    verts, elems, pot, om, wind = make_case(2, k, 104, jitter=0.1, seed=9)
    assert (om.n_elem + 127) // 128 == 169
    gm = dgconv.Mesh(2, k, verts, elems)
    v0 = oracle_state(om, k, seed=5)
    ds = oracle_ds(om, k, wind)
    ref = ODG.rk_substeps(ODG.ConvectionOracle(om, k, wind), v0, ds, 2, 3)
    for prec in ("bf16x3", "tf32x3"):
        v = cu(v0)
        gm.rk_substeps(cu(wind), v, ds, 2, 3, prec)
        assert maxrel(host(v), ref) < TOL[prec], prec
    gm.check()
