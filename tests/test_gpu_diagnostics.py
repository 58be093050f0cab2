"""GPU parity of dgc_diagnostics (mass per component, energy, non-finite count)
against the oracle's integrals (Sec. 2.3), on simplices, parallelograms,
parallelepipeds and curved triangles; the invariants of an RK run read through
it; the non-finite report through dgc_check; bitwise repetition."""
import numpy as np
import pytest

from gpu_common import make_case, oracle_state
from oracle import curved as C
from oracle import dg as ODG
from oracle import hexa as OX
from oracle import quad as OQ
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


def compare(got, mass, energy, volume):
    """Masses to 1e-12 of their Cauchy-Schwarz bound sqrt(volume energy), energy to 1e-12."""
    d = len(mass)
    bound = np.sqrt(volume * energy)
    assert np.all(np.abs(got[:d] - mass) <= 1e-12 * bound)
    assert abs(got[d] - energy) <= 1e-12 * energy
    assert got[d + 1] == 0.0


@pytest.mark.parametrize("dim,k,n", [(2, 1, 6), (2, 2, 5), (2, 4, 4), (2, 6, 3), (3, 1, 3), (3, 3, 2), (3, 5, 2)])
def test_simplex_diagnostics_match_oracle(dim, k, n):
    verts, elems, pot, om, wind = make_case(dim, k, n)
    gm = dgconv.Mesh(dim, k, verts, elems)
    w = oracle_state(om, k, seed=k + 10)
    mass, energy = ODG.integrals(om, k, w)
    compare(host(gm.diagnostics(cu(w))), mass, energy, np.abs(om.detJ).sum() / (2 if dim == 2 else 6))


def test_parallelogram_parallelepiped_and_curved_diagnostics_match_oracle():
    rng = np.random.default_rng(12)
    verts, elems = W.parallelogram_mesh(6, 5)
    om = OQ.QuadMesh(verts, elems)
    w = rng.uniform(-1, 1, (om.n_elem, 2, 9))
    gm = dgconv.Mesh(2, 2, verts, elems, shape="quad")
    compare(host(gm.diagnostics(cu(w))), *OQ.integrals(om, 2, w), np.abs(om.detJ).sum())
    verts, elems = W.parallelepiped_mesh(3, 5)
    om = OX.HexMesh(verts, elems)
    w = rng.uniform(-1, 1, (om.n_elem, 3, 27))
    gm = dgconv.Mesh(3, 2, verts, elems, shape="hex")
    compare(host(gm.diagnostics(cu(w))), *OX.integrals(om, 2, w), np.abs(om.detJ).sum())
    verts, elems, en = W.curved_square_mesh(6, 0.1, 5)
    cm = C.CurvedMesh(verts, elems, en)
    w = rng.uniform(-1, 1, (cm.n_elem, 2, 6))
    gm = dgconv.Mesh(2, 2, verts, elems, shape="curved", edge_nodes=en)
    compare(host(gm.diagnostics(cu(w))), *C.integrals(cm, 2, w), 1.0)


@pytest.mark.parametrize("dim,k,n,prec,tol", [(2, 3, 8, "fp64", 1e-13), (3, 2, 3, "fp64", 1e-13),
                                               (2, 4, 8, "bf16x3", 1e-5), (3, 4, 3, "bf16x3", 1e-5)])
def test_rk_run_conserves_mass_and_dissipates_energy(dim, k, n, prec, tol):
    """Zero inflow (the wind is tangential on the boundary): the mass of every
    component stays, the energy does not grow (Sec. 2.3), read on the device.
    FP64 keeps the mass to rounding; the split-BF16 stages add increments carrying
    FP32 accuracy, whose rounding the FP64 state sums over the 12 stages, so the
    mixed path is held to 1e-5 of the mass bound sqrt(|Omega| energy)."""
    verts, elems, pot, om, wind = make_case(dim, k, n)
    gm = dgconv.Mesh(dim, k, verts, elems)
    v = cu(oracle_state(om, k, seed=7))
    ds = ODG.cfl_ds(om, k, wind, 0.2)
    before = host(gm.diagnostics(v)).copy()
    energies = [before[dim]]
    for _ in range(4):
        gm.rk_substeps(cu(wind), v, ds, 3, 3, prec)
        energies.append(host(gm.diagnostics(v))[dim])
    after = host(gm.diagnostics(v))
    gm.check()
    bound = np.sqrt(before[dim])
    assert np.all(np.abs(after[:dim] - before[:dim]) <= tol * bound)
    assert all(b <= a * (1 + min(tol, 1e-6)) for a, b in zip(energies, energies[1:]))
    assert energies[-1] < energies[0]


def test_non_finite_coefficients_are_counted_and_reported():
    verts, elems, pot, om, wind = make_case(2, 2, 4)
    gm = dgconv.Mesh(2, 2, verts, elems)
    v = cu(oracle_state(om, 2))
    gm.check()
    good = host(gm.diagnostics(v)).copy()
    again = host(gm.diagnostics(v))
    assert np.array_equal(good, again)                      # fixed reduction order: bit for bit
    v[3, 1, 2] = float("nan")
    v[5, 0, 0] = float("inf")
    out = host(gm.diagnostics(v))
    assert out[3] == 2.0
    with pytest.raises(dgconv.DgcError, match="non-finite coefficient"):
        gm.check()
    gm.check()                                              # reported once, then cleared
