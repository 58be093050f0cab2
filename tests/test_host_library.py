"""CPU checks of the CUDA library's host side (no GPU needed).

* the shared library loads and exports every entry point of include/dgconv.h;
* its reference tables (Newton-iteration quadrature, dual-number Dubiner
  basis, BDM inverse) agree with the oracle's independent construction and
  with closed-form monomial integrals;
* its facet connectivity agrees with the oracle's brute-force matching.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import basis as OB
from oracle import mesh as OM
from paper_1508_04245_gb300 import build, dgconv
from paper_1508_04245_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "dgconv.h")).read()
    return sorted(set(re.findall(r"^dgc_status\s+(dgc_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    syms = header_symbols()
    assert len(syms) >= 15
    lib = ctypes.CDLL(dgconv.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(dgconv.SIGNATURES), set(syms) ^ set(dgconv.SIGNATURES)


def test_header_uses_plain_c_types_only():
    text = open(os.path.join(ROOT, "include", "dgconv.h")).read()
    for bad in ("torch", "at::", "Tensor", "std::"):
        assert bad not in text


CASES = [(2, 1), (2, 2), (2, 4), (2, 6), (3, 1), (3, 3), (3, 4), (3, 5)]


@pytest.mark.parametrize("dim,k", CASES)
def test_volume_rule_integrates_monomials(dim, k):
    x = dgconv.table(dim, k, "xv").reshape(-1, dim)
    w = dgconv.table(dim, k, "wv")
    deg = 3 * k - 1
    for exps in np.ndindex(*(deg + 1,) * dim):
        if sum(exps) > deg:
            continue
        exact = math.prod(math.factorial(e) for e in exps) / math.factorial(sum(exps) + dim)
        assert abs(np.sum(w * np.prod(x ** np.array(exps), axis=1)) - exact) < 1e-15


@pytest.mark.parametrize("dim,k", CASES)
def test_basis_tables_match_oracle(dim, k):
    x = dgconv.table(dim, k, "xv").reshape(-1, dim)
    N = OB.dim_pk(dim, k)
    Bv = dgconv.table(dim, k, "Bv").reshape(-1, N)
    assert np.abs(Bv - OB.dubiner_values(dim, k, x)).max() < 1e-12
    Gv = dgconv.table(dim, k, "Gv").reshape(-1, N, dim)
    grads = OB.grad_polys(OB.dubiner_polys(dim, k), dim)
    for a in range(dim):
        ref = np.stack([OB.P.evaluate(g[a], x) for g in grads], axis=1)
        assert np.abs(Gv[:, :, a] - ref).max() < 1e-11 * max(1, np.abs(ref).max())


@pytest.mark.parametrize("dim,k", CASES)
def test_facet_tables_match_oracle(dim, k):
    N = OB.dim_pk(dim, k)
    nfm = OB.dim_pk(dim - 1, k)
    s = dgconv.table(dim, k, "sf").reshape(-1, dim - 1)
    Qt = dgconv.table(dim, k, "Qt").reshape(-1, nfm)
    assert np.abs(Qt - OB.dubiner_values(dim - 1, k, s)).max() < 1e-12
    Ef = dgconv.table(dim, k, "Ef").reshape(dim + 1, nfm, N)
    from oracle.quadrature import simplex_rule
    sq, wq = simplex_rule(dim - 1, 2 * k + 2)
    qm = OB.dubiner_values(dim - 1, k, sq)
    for f in range(dim + 1):
        psi = OB.dubiner_values(dim, k, OB.facet_param_to_ref(dim, f, sq))
        ref = np.einsum("q,qm,qi->mi", wq, qm, psi)
        assert np.abs(Ef[f] - ref).max() < 1e-12


@pytest.mark.parametrize("dim,k", CASES)
def test_bdm_basis_matches_oracle(dim, k):
    nw = dim * OB.dim_pk(dim, k)
    Cb = dgconv.table(dim, k, "Cb").reshape(nw, nw)
    ref = np.asarray(OB.bdm_element(dim, k), dtype=np.float64)
    assert np.abs(Cb - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_connectivity_matches_oracle(dim):
    verts, elems = (W.square_mesh(5, 0.1, 2) if dim == 2 else W.cube_mesh(3, 0.05, 2))
    # scramble the local vertex order: the library must sort it
    rng = np.random.default_rng(0)
    elems = np.array([rng.permutation(e) for e in elems], dtype=np.int32)
    fid, nbr, ori, nf = dgconv.connectivity(dim, verts.shape[0], elems)
    om = OM.Mesh(verts, elems)
    assert nf == om.n_facets
    assert np.array_equal(fid, om.facet_id)
    assert np.array_equal(ori, om.orient)
    ne = np.where(nbr >= 0, nbr >> 2, -1)
    nfacet = np.where(nbr >= 0, nbr & 3, -1)
    assert np.array_equal(ne, om.nbr)
    assert np.array_equal(nfacet, om.nbr_facet)


def test_connectivity_rejects_bad_meshes():
    with pytest.raises(dgconv.DgcError):
        dgconv.connectivity(2, 4, np.array([[0, 1, 1]]))                   # repeated vertex
    with pytest.raises(dgconv.DgcError):
        dgconv.connectivity(2, 3, np.array([[0, 1, 5]]))                   # out of range
    with pytest.raises(dgconv.DgcError):                                    # facet in 3 triangles
        dgconv.connectivity(2, 5, np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]]))


def test_unsupported_order_is_rejected():
    with pytest.raises(dgconv.DgcError):
        dgconv.table(3, 6, "Bv")
    with pytest.raises(dgconv.DgcError):
        dgconv.table(2, 0, "Bv")


# ---- parallelograms -------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_quad_tables_match_oracle(k):
    from oracle import quad as OQ
    m = OQ.n_points(k)
    xq, wq = OQ.square_rule(m)
    N = (k + 1) ** 2
    Bv = dgconv.quad_table(k, "Bv").reshape(m * m, N)
    assert np.abs(Bv - OQ.vbasis(k, xq)).max() < 1e-13 * np.abs(Bv).max()
    assert np.allclose(dgconv.quad_table(k, "wv"), wq, atol=1e-15)
    t, w = OQ.gauss01(m)
    assert np.allclose(dgconv.quad_table(k, "sf"), t, atol=1e-15) and np.allclose(dgconv.quad_table(k, "wf"), w)
    L = dgconv.quad_table(k, "q1L").reshape(m, k + 1)
    Dl = dgconv.quad_table(k, "q1D").reshape(m, k + 1)
    E = dgconv.quad_table(k, "q1E").reshape(2, k + 1)
    for a in range(k + 1):
        assert np.allclose(L[:, a], OQ.leg(a, t), atol=1e-13) and np.allclose(Dl[:, a], OQ.dleg(a, t), atol=1e-11)
        assert np.allclose(E[:, a], OQ.leg(a, np.array([0.0, 1.0])), atol=1e-13)
    Cb = dgconv.quad_table(k, "Cb").reshape(2 * N, 2 * N)
    ref = np.linalg.inv(OQ.local_dof_matrix(k))
    assert np.abs(Cb - ref).max() < 1e-12 * np.abs(ref).max()


def test_quad_connectivity_matches_oracle():
    from oracle import quad as OQ
    v, e = W.parallelogram_mesh(6, 4)
    M = OQ.QuadMesh(v, e)
    fid, nbr, ori, flip, nf = dgconv.quad_connectivity(v.shape[0], e)
    assert nf == M.n_facets
    assert (fid == M.facet_id).all() and (ori == M.orient).all() and (flip == M.flip).all()
    inner = nbr >= 0
    assert (inner == (M.nbr >= 0)).all()
    assert (np.where(inner, nbr >> 3, -1) == M.nbr).all() and (np.where(inner, nbr & 3, -1) == M.nbr_facet).all()
    rev = (nbr >> 2) & 1
    nb_flip = M.flip[np.maximum(M.nbr, 0), np.maximum(M.nbr_facet, 0)]
    assert (rev[inner] == (M.flip[inner] != nb_flip[inner])).all()
    bad = e.copy()
    bad[3, 1] = bad[3, 0]
    with pytest.raises(dgconv.DgcError):
        dgconv.quad_connectivity(v.shape[0], bad)


# ---- parallelepipeds ------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3])
def test_hex_tables_match_oracle(k):
    from oracle import hexa as OX
    from oracle import quad as OQ
    m = OQ.n_points(k)
    xq, wq = OX.cube_rule(m)
    N = (k + 1) ** 3
    Bv = dgconv.hex_table(k, "Bv").reshape(m ** 3, N)
    assert np.abs(Bv - OX.vbasis(k, xq)).max() < 1e-13 * np.abs(Bv).max()
    assert np.allclose(dgconv.hex_table(k, "wv"), wq, atol=1e-15)
    s1, s2, ws = OX.square_rule(m)
    Bf = dgconv.hex_table(k, "Bf").reshape(6, m * m, N)
    for f in range(6):
        assert np.abs(Bf[f] - OX.vbasis(k, OX.face_point(f, s1, s2))).max() < 1e-13 * np.abs(Bv).max()
    Cb = dgconv.hex_table(k, "Cb").reshape(3 * N, 3 * N)
    ref = np.linalg.inv(OX.local_dof_matrix(k))
    assert np.abs(Cb - ref).max() < 1e-12 * np.abs(ref).max()


def test_hex_connectivity_matches_oracle():
    from oracle import hexa as OX
    v, e = W.parallelepiped_mesh(3, 6)
    M = OX.HexMesh(v, e)
    fid, nbr, ori, fc, nf = dgconv.hex_connectivity(v.shape[0], e)
    assert nf == M.n_facets and (fid == M.facet_id).all() and (ori == M.orient).all()
    code = M.fcode[..., 0] | (M.fcode[..., 1] << 1) | (M.fcode[..., 2] << 2)
    assert (fc == code).all()
    inner = nbr >= 0
    assert (np.where(inner, nbr >> 3, -1) == M.nbr).all() and (np.where(inner, nbr & 7, -1) == M.nbr_facet).all()


def test_quad_and_hex_host_inputs_are_validated():
    v, e = W.parallelogram_mesh(3, 1, reorient=False)
    # a third element on an existing edge: not conforming
    extra = np.array([[e[0, 0], e[0, 1], v.shape[0], v.shape[0] + 1]], dtype=np.int32)
    with pytest.raises(dgconv.DgcError):
        dgconv.quad_connectivity(v.shape[0] + 2, np.vstack([e, extra, extra[:, [1, 0, 3, 2]]]))
    bad = e.copy()
    bad[0, 3] = v.shape[0] + 5                                  # vertex out of range
    with pytest.raises(dgconv.DgcError):
        dgconv.quad_connectivity(v.shape[0], bad)
    hv, he = W.parallelepiped_mesh(2, 1, reorient=False)
    bad = he.copy()
    bad[1, 7] = bad[1, 0]                                       # repeated vertex
    with pytest.raises(dgconv.DgcError):
        dgconv.hex_connectivity(hv.shape[0], bad)
    for fn in (dgconv.quad_table, dgconv.hex_table):
        with pytest.raises(dgconv.DgcError):
            fn(2, "no_such_table")
    with pytest.raises(dgconv.DgcError):
        dgconv.hex_table(4, "Bv")                               # parallelepipeds: k <= 3
    with pytest.raises(dgconv.DgcError):
        dgconv.quad_table(7, "Bv")
