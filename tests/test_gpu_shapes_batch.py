"""GPU: one batched graph over instances of every element shape, and checkpoints
of the new shapes.

The batch advances each instance with the same kernels and launch sequence as
its own dgc_rk_substeps call, so the results must be bit-identical to the
single calls (which the per-shape parity tests pin to the oracles); in the
tensor-core precision the non-triangle instances run their stages in FP32.
"""
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


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def instances():
    out = []
    v, e = W.square_mesh(8, 0.1, 1)
    m = dgconv.Mesh(2, 3, v, e)
    out.append((m, m.wind_from_potential(cu(dgconv.potential_values(m, W.stream_random(2))))))
    v, e = W.parallelogram_mesh(6, 2)
    m = dgconv.Mesh(2, 3, v, e, shape="quad")
    out.append((m, m.wind_from_potential(cu(dgconv.potential_values(m, W.stream_random(3))))))
    v, e = W.parallelepiped_mesh(3, 3)
    m = dgconv.Mesh(3, 2, v, e, shape="hex")
    out.append((m, m.wind_from_potential(cu(dgconv.potential_values(m, W.potential_random(4))))))
    v, e, en = W.curved_square_mesh(6, 0.1, 3)
    m = dgconv.Mesh(2, 2, v, e, shape="curved", edge_nodes=en)
    out.append((m, m.wind_from_potential(cu(dgconv.potential_values(m, W.stream_random(5))))))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_mixed_shape_batch_matches_single_calls(instances, prec):
    rng = np.random.default_rng(7)
    states0 = [rng.uniform(-1, 1, size=(m.n_elem, m.dim, m.N)) for m, _ in instances]
    ds = [m.cfl_ds(w, 0.2) for m, w in instances]
    steps = [3, 2, 2, 4]
    ref = []
    for (m, w), s0, d, n in zip(instances, states0, ds, steps):
        v = cu(s0)
        m.rk_substeps(w, v, d, n, 3, "fp32" if (prec == "bf16x3" and m is not instances[0][0]) else prec)
        ref.append(v)
    states = [cu(s0) for s0 in states0]
    dgconv.batch_rk_substeps([m for m, _ in instances], [w for _, w in instances], states, ds, steps, 3, prec)
    torch.cuda.synchronize()
    for got, want in zip(states, ref):
        assert torch.equal(got, want)


def test_checkpoints_of_the_new_shapes(instances):
    for m, w in instances[1:]:
        v = torch.rand(m.n_elem, m.dim, m.N, dtype=torch.float64, device="cuda")
        blob = m.state_save(v, t=0.25, step=3)
        got, t, step = m.state_load(blob)
        assert torch.equal(got, v) and t == 0.25 and step == 3
