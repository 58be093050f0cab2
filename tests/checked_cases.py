"""Small cases run against the checked build (libdgconv_checked.so, every gather
index bounds-checked on the device): full parity with the oracle and a clean
status word on triangles, tetrahedra, parallelograms and parallelepipeds of 1 to
8 elements, then an injected out-of-range facet id that the checks must catch.
Run by tests/test_gpu_checked.py in a process of its own with DGC_LIBRARY=checked."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from gpu_common import TOL, make_case, maxrel, oracle_ds, oracle_state  # noqa: E402
from oracle import dg as ODG  # noqa: E402
from oracle import hexa as OX  # noqa: E402
from oracle import quad as OQ  # noqa: E402
from paper_1508_04245_gb300 import dgconv  # noqa: E402
from paper_1508_04245_gb300 import workloads as W  # noqa: E402

assert dgconv.LIB_PATH.endswith("libdgconv_checked.so"), dgconv.LIB_PATH


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def simplex(dim, k, n, precs):
    verts, elems, pot, om, wind = make_case(dim, k, n)
    assert om.n_elem <= 8
    gm = dgconv.Mesh(dim, k, verts, elems)
    w = oracle_state(om, k)
    assert maxrel(host(gm.transfer(cu(wind))), ODG.transfer(om, k, wind)) < 1e-12
    op = ODG.ConvectionOracle(om, k, wind)
    for prec in precs:
        assert maxrel(host(gm.conv_apply(cu(wind), cu(w), prec=prec)), op.apply(w)) < TOL[prec], (dim, k, prec)
        v = cu(w)
        ds = oracle_ds(om, k, wind)
        gm.rk_substeps(cu(wind), v, ds, 2, 3, prec)
        assert maxrel(host(v), ODG.rk_substeps(op, w, ds, 2, 3)) < TOL[prec], (dim, k, prec)
    assert maxrel(host(gm.transfer_T(cu(w))), ODG.transfer_T(om, k, w)) < 1e-12
    gm.check()
    return verts, elems, gm, wind


def tensor(shape):
    if shape == "quad":
        verts, elems = W.parallelogram_mesh(2, 3)
        om, O, dim, k, N = OQ.QuadMesh(verts, elems), OQ, 2, 2, 9
        op = OQ.QuadConvectionOracle
    else:
        verts, elems = W.parallelepiped_mesh(2, 3)
        om, O, dim, k, N = OX.HexMesh(verts, elems), OX, 3, 1, 8
        op = OX.HexConvectionOracle
    assert om.n_elem <= 8
    gm = dgconv.Mesh(dim, k, verts, elems, shape=shape)
    u = np.random.default_rng(3).standard_normal(gm.n_hdiv)
    w = np.random.default_rng(4).uniform(-1, 1, (om.n_elem, dim, N))
    assert maxrel(host(gm.transfer(cu(u))), O.transfer(om, k, u)) < 1e-12
    wind = O.dofs_of_function(om, k, lambda x: np.stack([np.sin(3 * x[:, 1]), np.cos(2 * x[:, 0])] +
                                                        ([np.sin(x[:, 0] + x[:, 1])] if dim == 3 else []), axis=1))
    assert maxrel(host(gm.conv_apply(cu(wind), cu(w))), op(om, k, wind).apply(w)) < 1e-12
    assert maxrel(host(gm.transfer_T(cu(w))), O.transfer_T(om, k, w)) < 1e-12
    gm.check()


simplex(2, 2, 2, ["fp64", "fp32", "bf16x3"])
simplex(2, 4, 1, ["fp64", "tf32x3"])
verts, elems, gm, wind = simplex(3, 2, 1, ["fp64", "fp32", "bf16x3"])
tensor("quad")
tensor("hex")
# an out-of-range facet id (element 0's, offset by the facet count) is caught and
# skipped: DGC_ERR_BOUNDS from dgc_check, then a clean run on a new handle
os.environ["DGC_FAULT"] = "gather"
bad = dgconv.Mesh(3, 2, verts, elems)
bad.transfer(cu(wind))
try:
    bad.check()
    raise SystemExit("the injected gather index was not reported")
except dgconv.DgcError as e:
    assert "status -7" in str(e), e
os.environ.pop("DGC_FAULT")
simplex(3, 2, 1, ["fp64"])
print("checked build: all cases OK")
