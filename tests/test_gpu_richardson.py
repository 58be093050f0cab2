"""GPU parity of the pseudo-time (Richardson) solve of the implicit convection
problem (Sec. 3.3.2) against the oracle, through the C ABI.

The iteration count is an integer decided by floating point; the tests choose
the reduction factor between two consecutive oracle residuals, so that the
decision has a margin far above the precision of the path (and assert that
margin), then compare the count exactly, the residual history and the
returned state element by element.
"""
import numpy as np
import pytest

from gpu_common import TC_PRECS, TOL, make_case, maxrel, oracle_state, tc_ok
from oracle import dg as ODG
from oracle import hdiv as OH
from oracle import mesh as OM
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


def problem(dim, k, n, seed):
    verts, elems, pot, om, wind = make_case(dim, k, n, seed=seed)
    op = ODG.ConvectionOracle(om, k, wind)
    g = oracle_state(om, k, seed=seed + 1)
    v0 = oracle_state(om, k, seed=seed + 2)
    tau = 0.3 * float(om.shortest_edge().min())
    ds = ODG.richardson_ds(om, k, wind, tau)
    return verts, elems, om, op, wind, g, v0, tau, ds


def reduction_for(op, g, v0, tau, ds, target):
    """A reduction factor that stops the oracle at `target` with a wide margin."""
    _, _, hist = ODG.richardson(op, g, v0, tau, ds, 0.0, target + 1)
    red = float(np.sqrt(hist[target] * hist[target - 1]) / hist[0])
    _, it, hist = ODG.richardson(op, g, v0, tau, ds, red, 10 * target)
    margin = min(abs(h / (red * hist[0]) - 1.0) for h in hist)
    return red, it, hist, margin


CASES = [(2, 1, 5, 1), (2, 2, 6, 2), (2, 4, 4, 3), (2, 6, 3, 4), (3, 2, 2, 5)]


@pytest.mark.parametrize("dim,k,n,seed", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_richardson_matches_oracle(dim, k, n, seed, prec):
    if prec in TC_PRECS and not tc_ok(dim, k, prec):
        pytest.skip("tensor-core paths: triangles k <= 6, tetrahedra k <= 4 in bf16x3")
    verts, elems, om, op, wind, g, v0, tau, ds = problem(dim, k, n, seed)
    red, it_o, hist_o, margin = reduction_for(op, g, v0, tau, ds, 12)
    assert margin > 1e-3
    v_o, _, _ = ODG.richardson(op, g, v0, tau, ds, red, 100)
    gm = dgconv.Mesh(dim, k, verts, elems)
    v = cu(v0)
    iters, res = gm.richardson(cu(wind), cu(g), v, tau, ds, red, 100, prec=prec)
    gm.check()
    assert int(host(iters)[0]) == it_o
    res = host(res)
    assert np.abs(res[:it_o + 1] - hist_o).max() <= TOL[prec] * hist_o[0]
    assert np.all(res[it_o + 1:] == 0.0)                     # untouched after the stop
    assert maxrel(host(v), v_o) < TOL[prec]


def test_richardson_iteration_cap_and_zero_data():
    verts, elems, om, op, wind, g, v0, tau, ds = problem(2, 3, 5, 7)
    gm = dgconv.Mesh(2, 3, verts, elems)
    v_o, it_o, hist_o = ODG.richardson(op, g, v0, tau, ds, 0.0, 5)
    assert it_o == 5
    v = cu(v0)
    iters, res = gm.richardson(cu(wind), cu(g), v, tau, ds, 0.0, 5)
    assert int(host(iters)[0]) == 5
    assert maxrel(host(v), v_o) < 1e-12
    assert maxrel(host(res), hist_o) < 1e-12
    # max_iter = 0: no update, only the initial residual
    v = cu(v0)
    iters, res = gm.richardson(cu(wind), cu(g), v, tau, ds, 0.5, 0)
    assert int(host(iters)[0]) == 0 and np.array_equal(host(v), v0)
    assert abs(host(res)[0] - hist_o[0]) <= 1e-12 * hist_o[0]
    # zero data and zero guess: zero residual, stop at once
    z = gm.dg_zeros()
    iters, res = gm.richardson(cu(wind), gm.dg_zeros(), z, tau, ds, 1e-6, 10)
    assert int(host(iters)[0]) == 0 and host(res)[0] == 0.0 and not host(z).any()
    gm.check()


def test_richardson_graph_replay_is_deterministic():
    verts, elems, om, op, wind, g, v0, tau, ds = problem(2, 4, 6, 8)
    gm = dgconv.Mesh(2, 4, verts, elems)
    w, gg = cu(wind), cu(g)
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = torch.zeros(41, dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(3):
        v = cu(v0)
        gm.richardson(w, gg, v, tau, ds, 1e-5, 40, prec="tf32x3", iters=iters, res=res)
        outs.append((host(v).copy(), int(host(iters)[0]), host(res).copy()))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1] == outs[0][1] and np.array_equal(o[2], outs[0][2])


def test_richardson_rejects_bad_arguments():
    verts, elems, om, op, wind, g, v0, tau, ds = problem(2, 2, 3, 9)
    gm = dgconv.Mesh(2, 2, verts, elems)
    w, gg, v = cu(wind), cu(g), cu(v0)
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = [(0.0, ds, 1e-3, 10), (tau, 2.0, 1e-3, 10), (tau, 0.0, 1e-3, 10), (tau, ds, -1.0, 10),
           (tau, ds, 1e-3, -1), (float("nan"), ds, 1e-3, 10)]
    for t_, d_, r_, m_ in bad:
        rc = dgconv.lib().dgc_richardson(gm._h, dgconv._ptr(w), dgconv._ptr(gg), dgconv._ptr(v), t_, d_, r_, m_,
                                         dgconv.DGC_FP64, dgconv.ctypes.c_void_p(iters.data_ptr()), None,
                                         dgconv._stream(None))
        assert rc == -1, (t_, d_, r_, m_)
    with pytest.raises(dgconv.DgcError):                      # g and v alias
        gm.richardson(w, v, v, tau, ds, 1e-3, 10)
    assert np.array_equal(host(v), v0)                         # nothing ran


def test_richardson_full_size_residual_property():
    """square256_k4 (131072 triangles, k = 4), 20 capped iterations on the
    tensor-core path and in FP64: the residual norm each run reports for its
    returned state equals the oracle's residual norm of that state."""
    wl = W.WORKLOADS["square256_k4"]
    verts, elems = wl.mesh()
    gm = dgconv.Mesh(2, wl.k, verts, elems)
    om = OM.Mesh(verts, elems)
    wind_o = OH.wind_from_potential(om, wl.k, wl.potential())
    wind = cu(wind_o)
    op = ODG.ConvectionOracle(om, wl.k, wind_o)
    g = cu(W.uniform_coeffs(wl.seed + 11, gm.n_elem, 2, wl.k))
    tau = 2.0 * ODG.cfl_ds(om, wl.k, wind_o, 1.0)
    ds = ODG.richardson_ds(om, wl.k, wind_o, tau)
    for prec, tol in (("fp64", 1e-12), ("tf32x3", 1e-5), ("bf16x3", 1e-6)):
        v = gm.dg_zeros()
        iters, res = gm.richardson(wind, g, v, tau, ds, 0.0, 20, prec=prec)
        gm.check()
        assert int(host(iters)[0]) == 20
        vh, gh = host(v), host(g)
        rho = gh - vh - tau * op.apply(vh)
        assert abs(host(res)[20] - ODG.dg_norm(om, rho)) <= tol * host(res)[0]
        assert host(res)[20] < host(res)[0]
