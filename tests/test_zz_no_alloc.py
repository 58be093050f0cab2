"""GPU test of dgc_transfer_T_noalloc, the variant of I^T for callers that
cannot allocate device memory at call time (applications that reserve their
device memory at start-up, host loops that must not block on the device-wide
synchronisation of cudaMalloc / cudaFree).

It must give the same result as dgc_transfer_T, call after call (the shared
fixed scratch keeps the previous call's contents), and reject meshes whose
scratch would not fit.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1508_04245_gb300 import build, dgconv
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dgconv


def _call(dgconv, mesh, f, g):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = dgconv.lib().dgc_transfer_T_noalloc(mesh._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                             stream)
    return rc


def _mesh(lib, shape, dim, k):
    from paper_1508_04245_gb300 import workloads as W
    if shape == "simplex":
        verts, elems = W.square_mesh(9, 0.1, 4) if dim == 2 else W.cube_mesh(3, 0.05, 4)
        return lib.Mesh(dim, k, verts, elems)
    if shape == "quad":
        return lib.Mesh(2, k, *W.parallelogram_mesh(6, 4), shape="quad")
    if shape == "hex":
        return lib.Mesh(3, k, *W.parallelepiped_mesh(3, 4), shape="hex")
    verts, elems, nodes = W.curved_square_mesh(8, 0.1, 4)
    return lib.Mesh(2, k, verts, elems, shape="curved", edge_nodes=nodes)


# every element shape: triangles, tetrahedra, parallelograms (4 facets),
# parallelepipeds (6 faces) and curved triangles (a second kernel rewrites the
# scratch of the curved elements)
@pytest.mark.parametrize("shape,dim,k", [("simplex", 2, 4), ("simplex", 3, 3), ("quad", 2, 3), ("hex", 3, 2),
                                         ("curved", 2, 3)])
def test_noalloc_matches_transfer_T_twice(lib, shape, dim, k):
    mesh = _mesh(lib, shape, dim, k)
    rng = np.random.default_rng(31)
    for call in range(2):
        f = torch.tensor(rng.standard_normal((mesh.n_elem, dim, mesh.N)), dtype=torch.float64, device="cuda")
        ref = mesh.transfer_T(f)
        got = torch.full_like(ref, np.nan)
        assert _call(lib, mesh, f, got) == 0, lib.last_error()
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err < 1e-12, (shape, call, err)


def test_noalloc_rejects_meshes_beyond_its_scratch(lib):
    from paper_1508_04245_gb300 import workloads as W
    # 2 * 230^2 triangles * 3 facets * 7 moments (k = 6) = 2.2e6 > 2^21 scratch doubles
    verts, elems = W.square_mesh(230, 0.0)
    mesh = lib.Mesh(2, 6, verts, elems)
    f = mesh.dg_zeros()
    g = mesh.hdiv_zeros()
    assert _call(lib, mesh, f, g) == -1
    assert "fixed maximum" in lib.last_error()
