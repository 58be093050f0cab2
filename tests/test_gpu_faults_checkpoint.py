"""GPU tests of the auxiliary subsystems: checkpoint / resume of a DG state and
the host-side fault injection (DGC_FAULT) for error propagation.  No GPU is
made to fault: the injected failures happen on the host before the CUDA call."""
import os

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


def case(k=3, n=8, seed=2):
    verts, elems = W.square_mesh(n, 0.1, seed)
    gm = dgconv.Mesh(2, k, verts, elems)
    wind = gm.wind_from_potential(torch.tensor(dgconv.potential_values(gm, W.stream_random(seed + 3)),
                                               dtype=torch.float64, device="cuda"))
    v0 = torch.tensor(W.uniform_coeffs(seed, gm.n_elem, 2, k), dtype=torch.float64, device="cuda")
    return verts, elems, gm, wind, v0


class fault:
    def __init__(self, what):
        self.what = what

    def __enter__(self):
        os.environ["DGC_FAULT"] = self.what

    def __exit__(self, *exc):
        os.environ.pop("DGC_FAULT", None)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_resume_from_checkpoint_is_bit_identical(prec):
    verts, elems, gm, wind, v0 = case()
    ds = gm.cfl_ds(wind, 0.2)
    ref = v0.clone()
    gm.rk_substeps(wind, ref, ds, 10, 3, prec)
    half = v0.clone()
    gm.rk_substeps(wind, half, ds, 5, 3, prec)
    blob = gm.state_save(half, t=5 * ds, step=5)
    # a new handle, as after a restart
    g2 = dgconv.Mesh(2, 3, verts, elems)
    v, t, step = g2.state_load(blob)
    assert step == 5 and t == 5 * ds
    g2.rk_substeps(wind, v, ds, 5, 3, prec)
    torch.cuda.synchronize()
    assert torch.equal(v, ref)


def test_checkpoint_rejects_corrupt_and_foreign_blobs():
    verts, elems, gm, wind, v0 = case()
    blob = bytearray(gm.state_save(v0, t=1.5, step=7))
    target = gm.dg_zeros()
    bad = bytearray(blob)
    bad[-3] ^= 0x40                                          # payload byte
    with pytest.raises(dgconv.DgcError):
        gm.state_load(bytes(bad), out=target)
    with pytest.raises(dgconv.DgcError):                     # truncated
        gm.state_load(bytes(blob[:-8]), out=target)
    bad = bytearray(blob)
    bad[0:4] = b"XXXX"
    with pytest.raises(dgconv.DgcError):
        gm.state_load(bytes(bad), out=target)
    _, _, g3, _, _ = case(k=2)                               # another order
    with pytest.raises(dgconv.DgcError):
        g3.state_load(bytes(blob))
    torch.cuda.synchronize()
    assert not target.any()                                  # nothing written by a failed load
    v, t, step = gm.state_load(bytes(blob), out=target)
    assert torch.equal(v, v0) and (t, step) == (1.5, 7)


def test_injected_faults_return_errors_and_leave_the_handle_usable():
    verts, elems, gm, wind, v0 = case()
    ds = gm.cfl_ds(wind, 0.2)
    ref = v0.clone()
    gm.rk_substeps(wind, ref, ds, 3, 3, "fp64")
    ref_apply = gm.conv_apply(wind, v0)
    torch.cuda.synchronize()
    # allocation: a fresh handle needs scratch for its first substeps
    with fault("alloc"):
        with pytest.raises(dgconv.DgcError):
            dgconv.Mesh(2, 3, verts, elems)
    fresh = dgconv.Mesh(2, 3, verts, elems)
    with fault("alloc"):
        with pytest.raises(dgconv.DgcError):
            fresh.rk_substeps(wind, v0.clone(), ds, 3, 3, "fp64")
    # capture: a call that needs a new graph
    with fault("capture"):
        with pytest.raises(dgconv.DgcError):
            gm.rk_substeps(wind, v0.clone(), ds, 4, 3, "fp64")
        with pytest.raises(dgconv.DgcError):
            dgconv.batch_rk_substeps([gm], [wind], [v0.clone()], [ds], [2], 3, "fp64")
    # launch: the stage kernels of either path
    with fault("launch"):
        for prec in ("fp64", "bf16x3"):
            with pytest.raises(dgconv.DgcError):
                gm.conv_apply(wind, v0, prec=prec)
    # after the faults every call works and gives the same results
    for h in (gm, fresh):
        v = v0.clone()
        h.rk_substeps(wind, v, ds, 3, 3, "fp64")
        torch.cuda.synchronize()
        assert torch.equal(v, ref)
        assert torch.equal(h.conv_apply(wind, v0), ref_apply)
        h.check()
    v = v0.clone()
    gm.rk_substeps(wind, v, ds, 4, 3, "fp64")
    w = v0.clone()
    gm.rk_substeps(wind, w, ds, 4, 3, "fp64")
    torch.cuda.synchronize()
    assert torch.equal(v, w)
    assert np.isfinite(v.cpu().numpy()).all()


def mesh_case(dim, k, n, seed=4):
    verts, elems = W.square_mesh(n, 0.1, seed) if dim == 2 else W.cube_mesh(n, 0.05, seed)
    gm = dgconv.Mesh(dim, k, verts, elems)
    pot = W.stream_random(seed + 3) if dim == 2 else W.potential_random(seed + 3)
    wind = gm.wind_from_potential(torch.tensor(dgconv.potential_values(gm, pot), dtype=torch.float64,
                                               device="cuda"))
    v0 = torch.tensor(W.uniform_coeffs(seed, gm.n_elem, dim, k), dtype=torch.float64, device="cuda")
    return verts, elems, gm, wind, v0


@pytest.mark.parametrize("dim,k,n,prec", [(2, 3, 12, "tf32x3"), (2, 4, 12, "bf16x3"), (3, 2, 3, "bf16x3"),
                                          (3, 4, 3, "bf16x3")])
def test_bounded_wait_timeout_is_reported_and_handle_recovers(dim, k, n, prec):
    """DGC_FAULT=stall: the tensor-core stage kernel issues no bulk copy, so its
    bounded mbarrier waits run out (nothing in flight); the timeout reaches the
    status word, dgc_check reports DGC_ERR_TIMEOUT once, and the same handle then
    reproduces a fresh handle's run bit for bit."""
    verts, elems, gm, wind, v0 = mesh_case(dim, k, n)
    ds = gm.cfl_ds(wind, 0.2)
    ref_mesh = dgconv.Mesh(dim, k, verts, elems)
    ref = v0.clone()
    ref_mesh.rk_substeps(wind, ref, ds, 3, 3, prec)
    ref_mesh.check()
    v = v0.clone()
    with fault("stall"):
        gm.rk_substeps(wind, v, ds, 3, 3, prec)   # launches; the waits give up on the device
    torch.cuda.synchronize()
    with pytest.raises(dgconv.DgcError, match="status -4"):
        gm.check()
    gm.check()   # the word was cleared by the report
    v = v0.clone()
    gm.rk_substeps(wind, v, ds, 3, 3, prec)
    gm.check()
    torch.cuda.synchronize()
    assert torch.equal(v, ref)
