"""GPU parity of the H(div)-side compositions against the oracle, through the
C ABI: the OIFS right-hand side I^T M^V Q I u (frozen and extrapolated wind,
Sec. 3.2), C^U = I^T C^V I (Sec. 2.4) and the velocity extrapolation."""
import numpy as np
import pytest

from gpu_common import TC_PRECS, TOL, make_case, maxrel, oracle_ds, tc_ok, tol_hdiv_chain
from oracle import dg as ODG
from oracle import hdiv as OH
from paper_1508_04245_gb300 import build, dgconv
from paper_1508_04245_gb300 import workloads as W

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


def case(dim, k, n, seed):
    verts, elems, pot, om, wind = make_case(dim, k, n, seed=seed)
    pot2 = W.stream_random(seed + 31) if dim == 2 else W.potential_random(seed + 31)
    wind2 = OH.wind_from_potential(om, k, pot2)
    u = OH.dofs_of_function(om, k, W.fourier_field(seed + 41, dim))
    return verts, elems, om, wind, wind2, u


CASES = [(2, 1, 5, 1), (2, 3, 4, 2), (2, 4, 4, 3), (2, 6, 2, 4), (3, 2, 2, 5)]


@pytest.mark.parametrize("dim,k,n,seed", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_conv_apply_hdiv(dim, k, n, seed, prec):
    if prec in TC_PRECS and not tc_ok(dim, k, prec):
        pytest.skip("tensor-core paths: triangles k <= 6, tetrahedra k <= 4 in bf16x3")
    verts, elems, om, wind, _, u = case(dim, k, n, seed)
    ref = ODG.conv_hdiv(ODG.ConvectionOracle(om, k, wind), u)
    gm = dgconv.Mesh(dim, k, verts, elems)
    got = host(gm.conv_apply_hdiv(cu(wind), cu(u), prec=prec))
    assert maxrel(got, ref) < tol_hdiv_chain(dim, k, prec)


@pytest.mark.parametrize("dim,k,n,seed", CASES)
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("extrapolated", [False, True])
def test_oifs_rhs(dim, k, n, seed, prec, extrapolated):
    if prec in TC_PRECS and not tc_ok(dim, k, prec):
        pytest.skip("tensor-core paths: triangles k <= 6, tetrahedra k <= 4 in bf16x3")
    verts, elems, om, wind, wind2, u = case(dim, k, n, seed)
    ds = oracle_ds(om, k, wind)
    kw = dict(wind_prev=wind2, dt_prev=3 * ds) if extrapolated else {}
    ref = ODG.oifs_rhs(om, k, u, wind, ds, 3, 3, **kw)
    gm = dgconv.Mesh(dim, k, verts, elems)
    gkw = dict(wind_prev=cu(wind2), dt_prev=3 * ds) if extrapolated else {}
    got = host(gm.oifs_rhs(cu(u), cu(wind), ds, 3, 3, prec=prec, **gkw))
    gm.check()
    assert maxrel(got, ref) < tol_hdiv_chain(dim, k, prec)


def test_oifs_rhs_without_substeps_and_rk2():
    verts, elems, om, wind, _, u = case(2, 2, 5, 6)
    gm = dgconv.Mesh(2, 2, verts, elems)
    ds = oracle_ds(om, 2, wind)
    for nsteps, scheme in ((0, 3), (4, 2)):
        ref = ODG.oifs_rhs(om, 2, u, wind, ds, nsteps, scheme)
        got = host(gm.oifs_rhs(cu(u), cu(wind), ds, nsteps, scheme))
        assert maxrel(got, ref) < 1e-12


def test_oifs_rhs_is_the_composition_of_the_single_calls():
    """Bit for bit: the fused call runs the same kernels in the same order."""
    verts, elems, om, wind, _, u = case(2, 4, 6, 7)
    gm = dgconv.Mesh(2, 4, verts, elems)
    w, uu = cu(wind), cu(u)
    ds = oracle_ds(om, 4, wind)
    for prec in ("fp64", "tf32x3", "bf16x3"):
        fused = host(gm.oifs_rhs(uu, w, ds, 5, 3, prec=prec))
        v = gm.transfer(uu)
        gm.rk_substeps(w, v, ds, 5, 3, prec)
        single = host(gm.transfer_T(gm.mass(v)))
        assert np.array_equal(fused, single)
        again = host(gm.oifs_rhs(uu, w, ds, 5, 3, prec=prec))    # graph replay
        assert np.array_equal(again, fused)


def test_wind_extrapolate():
    verts, elems, om, wind, wind2, u = case(2, 3, 4, 8)
    gm = dgconv.Mesh(2, 3, verts, elems)
    fields = [cu(wind), cu(wind2), cu(u)]
    coefs = [3.0, -3.0, 1.0]
    ref = ODG.extrapolate([wind, wind2, u], coefs)
    got = host(gm.wind_extrapolate(fields, coefs))
    assert maxrel(got, ref) < 1e-15
    # in place on the first field
    gm.wind_extrapolate(fields[:2], [2.0, -1.0], out=fields[0])
    assert maxrel(host(fields[0]), ODG.extrapolate([wind, wind2], [2.0, -1.0])) < 1e-15


def test_rejects_bad_arguments():
    verts, elems, om, wind, wind2, u = case(2, 2, 3, 9)
    gm = dgconv.Mesh(2, 2, verts, elems)
    w, w2, uu = cu(wind), cu(wind2), cu(u)
    with pytest.raises(dgconv.DgcError):
        gm.wind_extrapolate([], [])
    with pytest.raises(dgconv.DgcError):
        gm.wind_extrapolate([w] * 9, [1.0] * 9)
    with pytest.raises(dgconv.DgcError):                      # extrapolation needs dt_prev > 0
        gm.oifs_rhs(uu, w, 0.01, 2, 3, wind_prev=w2, dt_prev=0.0)
    with pytest.raises(dgconv.DgcError):                      # out aliases u
        gm.oifs_rhs(uu, w, 0.01, 2, 3, out=uu)
    with pytest.raises(dgconv.DgcError):
        gm.conv_apply_hdiv(w, uu, out=uu)
    with pytest.raises(dgconv.DgcError):
        gm.oifs_rhs(uu, w, -1.0, 2, 3)
