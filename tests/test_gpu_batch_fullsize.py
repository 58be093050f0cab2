"""GPU tests of the batched entry point and of the full-size workloads.

* dgc_batch_rk_substeps: every instance equals its own dgc_rk_substeps run
  (bit for bit: same kernels, same order), replaying the cached graph gives
  the same result, and instances are checked against the oracle;
* the benchmark workload (131072 jittered triangles, k = 4) at full size, in
  the launch configuration bench.py times: conv_apply on sampled elements
  against the oracle (error against the summand scale of the residual, which
  on this smooth state is a strong cancellation), and after 100 SSP-RK3 substeps the invariants that hold
  at any size (mass conservation, non-increasing upwind energy) and the
  tensor-core path against the FP64 path;
* the 3D workloads at full size (196608 and 663552 tetrahedra): invariants.
"""
import math

import numpy as np
import pytest

from gpu_common import TOL, make_case, maxrel, oracle_ds, oracle_state, tc_ok
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


def gpu_case(dim, k, n, seed):
    verts, elems = W.square_mesh(n, 0.1, seed) if dim == 2 else W.cube_mesh(n, 0.05, seed)
    gm = dgconv.Mesh(dim, k, verts, elems)
    pot = W.stream_random(seed + 3) if dim == 2 else W.potential_random(seed + 3)
    wind = gm.wind_from_potential(cu(dgconv.potential_values(gm, pot)))
    v0 = cu(W.uniform_coeffs(seed, gm.n_elem, dim, k))
    return gm, wind, v0


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_batch_equals_single_instances(prec):
    specs = [(2, 1, 5, 1), (2, 2, 9, 2), (2, 3, 6, 3), (2, 4, 11, 4), (2, 5, 4, 5), (2, 6, 3, 6), (3, 2, 2, 7)]
    cases = [gpu_case(*s) for s in specs]
    ds = [0.2 * m.min_edge() / ((2 * m.k + 1) * m.max_wind_speed(w)) for m, w, _ in cases]
    nsteps = [3, 2, 4, 3, 2, 1, 2]
    singles = []
    for (m, w, v0), d, n in zip(cases, ds, nsteps):
        x = v0.clone()
        m.rk_substeps(w, x, d, n, 3, prec if (prec == "fp64" or tc_ok(m.dim, m.k, prec)) else "fp32")
        singles.append(host(x).copy())
    states = [v0.clone() for _, _, v0 in cases]
    dgconv.batch_rk_substeps([c[0] for c in cases], [c[1] for c in cases], states, ds, nsteps, 3, prec)
    for got, ref in zip(states, singles):
        assert np.array_equal(host(got), ref)
    # replay of the cached graph
    states2 = [v0.clone() for _, _, v0 in cases]
    dgconv.batch_rk_substeps([c[0] for c in cases], [c[1] for c in cases], states2, ds, nsteps, 3, prec)
    for got, ref in zip(states2, singles):
        assert np.array_equal(host(got), ref)
    for m, _, _ in cases:
        m.check()


@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_merged_batch_launch_equals_single_instances(prec, scheme):
    """Triangle instances of one order share each stage launch (a work list over all of
    their tiles): several meshes per order of uneven size, more tiles than resident CTAs
    (k = 2: 309 tiles on two CTAs per SM), meshes that stop stepping early (the launch
    shrinks to the ones still stepping), one CTA per SM at k = 6; each result equals the
    instance's own rk_substeps run bit for bit."""
    specs = [(2, 2, 100, 21), (2, 2, 90, 22), (2, 2, 40, 23), (2, 4, 20, 24), (2, 4, 5, 25), (2, 4, 33, 26),
             (2, 6, 9, 27), (2, 6, 4, 28)]
    nsteps = [2, 3, 1, 3, 1, 2, 2, 1]
    cases = [gpu_case(*s) for s in specs]
    ds = [0.2 * m.min_edge() / ((2 * m.k + 1) * m.max_wind_speed(w)) for m, w, _ in cases]
    singles = []
    for (m, w, v0), d, n in zip(cases, ds, nsteps):
        x = v0.clone()
        m.rk_substeps(w, x, d, n, scheme, prec)
        singles.append(host(x).copy())
    for rep in range(2):   # capture, then replay of the cached graph
        states = [v0.clone() for _, _, v0 in cases]
        dgconv.batch_rk_substeps([c[0] for c in cases], [c[1] for c in cases], states, ds, nsteps, scheme, prec)
        for got, ref in zip(states, singles):
            assert np.array_equal(host(got), ref)
    for m, _, _ in cases:
        m.check()


def test_batch_instances_match_oracle():
    insts = []
    for k, n, seed in [(2, 6, 11), (4, 5, 12)]:
        verts, elems, pot, om, wind = make_case(2, k, n, seed=seed)
        gm = dgconv.Mesh(2, k, verts, elems)
        v0 = oracle_state(om, k, seed=seed)
        ds = oracle_ds(om, k, wind)
        ref = ODG.rk_substeps(ODG.ConvectionOracle(om, k, wind), v0, ds, 3, 3)
        insts.append((gm, cu(wind), cu(v0), ds, ref))
    states = [i[2] for i in insts]
    dgconv.batch_rk_substeps([i[0] for i in insts], [i[1] for i in insts], states, [i[3] for i in insts], [3, 3],
                             3, "fp64")
    for (gm, w, v, ds, ref) in insts:
        assert maxrel(host(v), ref) < 1e-12


def test_batch_rejects_shared_meshes():
    m, w, v = gpu_case(2, 2, 4, 1)
    with pytest.raises(dgconv.DgcError):
        dgconv.batch_rk_substeps([m, m], [w, w], [v, v.clone()], [1e-3, 1e-3], [1, 1])


# ---------------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def square256():
    wl = W.WORKLOADS["square256_k4"]
    verts, elems = wl.mesh()
    gm = dgconv.Mesh(2, wl.k, verts, elems)
    wind = gm.wind_from_potential(cu(dgconv.potential_values(gm, wl.potential())))
    field = W.fourier_field(wl.seed + 2000, 2)
    u_n = gm.hdiv_interpolate(cu(field(gm.point_coords(2))))
    return wl, verts, elems, gm, wind, u_n


def test_square256_conv_apply_sampled_against_oracle(square256):
    wl, verts, elems, gm, wind, u_n = square256
    om = OM.Mesh(verts, elems)
    wind_o = OH.wind_from_potential(om, wl.k, wl.potential())
    assert maxrel(host(wind), wind_o) < 1e-12
    w = gm.transfer(u_n)
    sel = np.random.default_rng(0).choice(om.n_elem, size=300, replace=False)
    sel = np.unique(np.concatenate([sel, [0, 1, om.n_elem - 1]]))
    op = ODG.ConvectionOracle(om, wl.k, wind_o, sel=sel)
    ref, scale = op.apply(host(w)), op.magnitude(host(w)).max()
    # The state is smooth and h = 1/256: the volume and facet sums are each ~1/h
    # times the residual (summand scale / max |r| is about 640 here), so the
    # error of either evaluation is a rounding error of the summands and is
    # measured against their scale (the forward-error bound of a sum).
    assert scale > 100 * np.abs(ref).max()
    for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
        got = host(gm.conv_apply(cu(wind_o), w, prec=prec))[sel]
        assert np.abs(got - ref).max() < TOL[prec] * scale, prec


def _mass_energy(gm, v):
    """Per component: sum_T |det J| w_{c,0} (the mean mode carries the mass), the
    scale sum_T |det J| |w_{c,0}|, and the energy sum_T |det J| |w|^2."""
    a = host(gm.mass(v))
    x = host(v)
    return a[:, :, 0].sum(axis=0), np.abs(a[:, :, 0]).sum(axis=0), float((a * x).sum())


def test_square256_rk_bench_configuration(square256):
    wl, verts, elems, gm, wind, u_n = square256
    ds = gm.cfl_ds(wind, wl.cfl)
    v64 = gm.transfer(u_n)
    m0, s0, e0 = _mass_energy(gm, v64)
    gm.rk_substeps(wind, v64, ds, wl.substeps, 3, "fp64")
    m1, s1, e64 = _mass_energy(gm, v64)
    # the wind is tangential on the boundary: the total of each component is conserved
    assert np.all(np.abs(m1 - m0) < 1e-13 * s0)
    # On this smooth state the upwind dissipation (jumps ~ h^(k+1)) and the
    # damping of SSP-RK3 on the skew part ((lambda ds)^4 / 12 per substep) are
    # below the tensor-core paths' rounding; only the FP64 run can show the
    # energy not increasing, and the tensor-core energy follows from its state error.
    assert e64 <= e0 * (1 + 1e-12)
    for prec in ("tf32x3", "bf16x3"):
        vtc = gm.transfer(u_n)
        gm.rk_substeps(wind, vtc, ds, wl.substeps, 3, prec)
        gm.check()
        m1, s1, e1 = _mass_energy(gm, vtc)
        assert np.all(np.abs(m1 - m0) < 1e-6 * s0)
        err = maxrel(host(vtc), host(v64))
        assert err < 1e-6, prec
        assert abs(e1 - e64) <= 3 * err * e64


def test_bf16x3_meets_1e_6_on_rough_states():
    """Uniform random coefficients (all modes excited), 50 SSP-RK3 substeps at CFL
    0.2, every tensor-core order: the BF16x3 path (operands split exactly)
    stays within 1e-6 of the FP64 path; TF32x3 (22-bit operands) is only
    required to stay within its FP32-level tolerance here."""
    for k in (1, 2, 3, 4):
        m, w, v0 = gpu_case(2, k, 40, 20 + k)
        ds = m.cfl_ds(w, 0.2)
        ref = v0.clone()
        m.rk_substeps(w, ref, ds, 50, 3, "fp64")
        for prec, tol in (("bf16x3", 1e-6), ("tf32x3", 1e-5)):
            v = v0.clone()
            m.rk_substeps(w, v, ds, 50, 3, prec)
            m.check()
            assert maxrel(host(v), host(ref)) < tol, (k, prec)


@pytest.mark.parametrize("name,prec", [("cube32_k3", "fp32"), ("cube48_k4", "fp32")])
def test_cube_full_size_invariants(name, prec):
    wl = W.WORKLOADS[name]
    verts, elems = wl.mesh()
    gm = dgconv.Mesh(3, wl.k, verts, elems)
    wind = gm.wind_from_potential(cu(dgconv.potential_values(gm, wl.potential())))
    if wl.unit_peak_speed:
        wind /= gm.max_wind_speed(wind)
    ds = gm.cfl_ds(wind, wl.cfl)
    # a constant state is steady (exactly divergence-free wind, zero residual)
    c = gm.dg_zeros()
    c[:, :, 0] = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda") * math.sqrt(6.0)
    r = host(gm.conv_apply(wind, c, prec=prec))
    assert np.abs(r).max() < 1e-4 * np.abs(host(gm.conv_apply(wind, cu(W.uniform_coeffs(1, gm.n_elem, 3, wl.k)),
                                                              prec=prec))).max()
    v = cu(W.uniform_coeffs(wl.seed, gm.n_elem, 3, wl.k))
    m0, s0, e0 = _mass_energy(gm, v)
    gm.rk_substeps(wind, v, ds, 2, 3, prec)
    gm.check()
    m1, s1, e1 = _mass_energy(gm, v)
    assert np.all(np.abs(m1 - m0) < 1e-6 * s0)
    assert e1 <= e0
