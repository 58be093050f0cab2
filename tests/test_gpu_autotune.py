"""GPU tests of the autotuner of the CUDA-core stage kernel (dgc_autotune):
the choice is one of the candidate block shapes, results are bit-identical
before and after tuning (every element is computed independently of the block
shape), and the tensor-core precision has nothing to tune."""
import numpy as np
import pytest

from paper_1508_04245_gb300 import build, dgconv
from paper_1508_04245_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def case(dim, k, n, seed):
    verts, elems = W.square_mesh(n, 0.1, seed) if dim == 2 else W.cube_mesh(n, 0.05, seed)
    gm = dgconv.Mesh(dim, k, verts, elems)
    pot = W.stream_random(seed + 3) if dim == 2 else W.potential_random(seed + 3)
    wind = gm.wind_from_potential(torch.tensor(dgconv.potential_values(gm, pot), dtype=torch.float64,
                                               device="cuda"))
    v0 = torch.tensor(W.uniform_coeffs(seed, gm.n_elem, dim, k), dtype=torch.float64, device="cuda")
    return gm, wind, v0


@pytest.mark.parametrize("dim,k,n,prec", [(2, 5, 24, "fp32"), (2, 6, 16, "fp64"), (3, 2, 6, "fp64"),
                                          (3, 4, 4, "fp32")])
def test_autotune_keeps_results_bit_identical(dim, k, n, prec):
    gm, wind, v0 = case(dim, k, n, 3)
    ds = gm.cfl_ds(wind, 0.2)
    before = v0.clone()
    gm.rk_substeps(wind, before, ds, 3, 3, prec)
    r_before = gm.conv_apply(wind, v0, prec=prec)
    block = gm.autotune(wind, prec, reps=3)
    assert block in (64, 128, 192, 256)
    after = v0.clone()
    gm.rk_substeps(wind, after, ds, 3, 3, prec)
    r_after = gm.conv_apply(wind, v0, prec=prec)
    torch.cuda.synchronize()
    assert torch.equal(before, after) and torch.equal(r_before, r_after)
    gm.check()


def test_autotune_tensor_core_precision_and_arguments():
    gm, wind, v0 = case(2, 3, 8, 4)
    assert gm.autotune(wind, "tf32x3") == 0
    with pytest.raises(dgconv.DgcError):
        gm.autotune(wind, "fp64", reps=0)
    g3, w3, _ = case(3, 2, 2, 5)
    with pytest.raises(dgconv.DgcError):                      # no tensor-core path for tetrahedra
        g3.autotune(w3, "tf32x3")
