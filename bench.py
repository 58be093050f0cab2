"""Benchmark of the explicit upwind-DG convection step on one GB300.

Workload (default): 2D unit square, 256 x 256 squares split into 131072
triangles, interior vertices jittered +-10% of h, order k = 4, wind = curl of a
seeded 8-mode stream function, state = the BDM_k interpolant of a seeded
8-mode Fourier velocity field; 100 SSP-RK3 substeps at CFL 0.2.

One step is one pass of the whole hot path, the OIFS right-hand side of the
paper's Sec. 3.2 for this velocity:
    a1 geometry -> a2 v = I u^n -> 100 x (a3..a7 RK3 substep, frozen wind)
    -> a6 M^V v -> a8 g = I^T M^V v.
The metric counts DOF-stage updates: E * N * dim * 3 stages * 100 substeps.

``value`` is measured with every input resident in HBM; ``e2e`` repeats the
step through the same public calls with u^n and the wind copied from pinned
host memory and g copied back inside the timed region.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1508_04245_gb300 import workloads as W  # noqa: E402

METRIC = "DG convection DOF-stage updates/s, plain FP64 vs mixed/batched at ≤1e-6 err"
TC_PRECS = ("tf32x3", "bf16x3")
WORKLOAD = "square256_k4"
FP64_TFLOPS = 1.25          # nominal dense FP64 rate of a GB300 (no measured figure in the peaks file)
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgconv", choices=["dgconv", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "fp64", "tf32x3", "bf16x3"])
    ap.add_argument("--no-other-precisions", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--substeps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-shapes", action="store_true",
                    help="skip the parallelogram and curved-triangle sections")
    args = ap.parse_args()
    if args.impl == "dgconv" and W.WORKLOADS[args.workload].shape != "simplex" and args.prec in TC_PRECS:
        ap.error("the tensor-core precisions cover affine triangles; use --prec fp32 or fp64 on other shapes")
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# several GPUs: one independent problem per rank (weak scaling, no data-path
# collective); the step time of the job is the slowest rank's
# ---------------------------------------------------------------------------
def rank_workload(wl, rank: int):
    """The workload of one rank: same sizes, its own seeds (rank 0 keeps the configured ones)."""
    return wl if rank == 0 else dataclasses.replace(wl, seed=wl.seed + 7919 * rank)


def max_over_ranks(x: float, world: int, device) -> float:
    """The maximum of a per-rank time over all ranks (an all-reduce on the default group)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, world: int, ms_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's step time."""
    return world * units_per_rank_step / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload construction (untimed)
# ---------------------------------------------------------------------------
def make_inputs(wl, torch, dgconv):
    m = wl.mesh()
    mesh = dgconv.Mesh(wl.dim, wl.k, m[0], m[1], shape=wl.shape, edge_nodes=m[2] if len(m) > 2 else None)
    pot = dgconv.potential_values(mesh, wl.potential())
    wind = mesh.wind_from_potential(torch.tensor(pot, dtype=torch.float64, device="cuda"))
    if wl.unit_peak_speed:
        wind /= mesh.max_wind_speed(wind)
    if wl.state == "wind":
        # the transported velocity: another exactly divergence-free field
        pot2 = dgconv.potential_values(mesh, W.stream_random(wl.seed + 2000))
        u_n = mesh.wind_from_potential(torch.tensor(pot2, dtype=torch.float64, device="cuda"))
    else:
        field = W.fourier_field(wl.seed + 2000, wl.dim)
        X = mesh.point_coords(2)
        u_n = mesh.hdiv_interpolate(torch.tensor(field(X), dtype=torch.float64, device="cuda"))
    ds = mesh.cfl_ds(wind, wl.cfl)
    return mesh, wind, u_n, ds


def stage_bytes_flops(wl):
    """Algorithmic bytes and flops per element per RK stage (method's own work).

    bytes: read v^(i), read v^n, write v^(i+1) (FP64), the wind's N_W
    coefficients, d^2+1 geometry values, d+1 neighbour ids.
    flops: wind and state at the volume points, the gradient test
    contraction, traces and facet test contraction.
    """
    d, k = wl.dim, wl.k
    if wl.shape == "quad":
        # parallelograms, sum-factorised: per component m rows of (trace, m points,
        # two row projections, outer update) and 4 facets of (own and neighbour
        # trace, m points, scatter); the same bytes convention with 4 facets
        n, m = k + 1, (3 * k) // 2 + 1
        N = n * n
        fma_c = m * (3 * n * n + m * (3 * n + 2)) + 4 * (3 * n * n + m * (3 * n + 1))
        byts = 3 * N * d * 8 + d * N * 8 + (d * d + 1) * 8 + 4 * 4
        return byts, 2 * d * fma_c, N
    if wl.shape == "hex":
        # parallelepipeds, sum-factorised per component: three contractions to the m^3
        # points, the wind products, three back; per face the two traces (own and
        # neighbour), values at the m^2 points, projection back and the scatter
        n, m = k + 1, (3 * k) // 2 + 1
        N = n ** 3
        vol = m * n ** 3 + m * m * n * n + m ** 3 * n + 3 * m ** 3 + 3 * m ** 3 * n + 3 * m * m * n * n + 2 * m * n ** 3
        face = 3 * n ** 3 + 3 * m * n * n + 3 * m * m * n
        byts = 3 * N * d * 8 + d * N * 8 + (d * d + 1) * 8 + 6 * 4
        return byts, 2 * d * (vol + 6 * face), N
    N = math.comb(k + d, d)
    nq = (3 * k - 1) // 2 + 1
    nf = (3 * k) // 2 + 1
    Qv = nq ** d
    Qf = nf ** (d - 1)
    NW = d * N
    byts = 3 * N * d * 8 + NW * 8 + (d * d + 1) * 8 + (d + 1) * 4
    flops = 2 * Qv * N * d + 2 * Qv * N * d + 2 * Qv * N * d * d + 4 * (d + 1) * Qf * N * d
    return byts, flops, N


# committed ncu summaries: (workload, precision) -> (summary file, kernel source it measured)
PROFILES = {
    ("square256_k4", "bf16x3"): ("stage_tc_kernel_square256_k4.md", "dgc_stage_tc.cuh"),
    ("square256_k4", "fp32"): ("stage_kernel_square256_k4_fp32.md", "dgc_stage.cuh"),
    ("parallelogram256_k4", "fp32"): ("stage_quad_kernel_parallelogram256_k4.md", "dgc_stage_quad.cu"),
    ("parallelepiped32_k3", "fp32"): ("stage_hex_kernel_parallelepiped32_k3.md", "dgc_stage_hex.cu"),
}


def ncu_traffic(wl, prec):
    """DRAM bytes per stage launch from the committed ncu capture, if it still applies.

    The capture records the sha1 of the kernel source it measured and the
    precision; after any change of that source the figure is stale and None is
    returned.
    """
    entry = PROFILES.get((wl.name, prec))
    if entry is None:
        return None
    import hashlib
    prof = os.path.join(ROOT, "profiles", entry[0])
    src = os.path.join(ROOT, "paper_1508_04245_gb300", "csrc", entry[1])
    try:
        text = open(prof).read()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    fields = dict(ln.split(":", 1) for ln in text.splitlines()
                  if ln.startswith(("kernel_source_sha1:", "traffic_bytes_per_launch:", "prec:")))
    if fields.get("kernel_source_sha1", "").split()[0:1] != [sha]:
        return None
    if fields.get("prec", "").strip() != prec:
        return None
    return float(fields["traffic_bytes_per_launch"].strip())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        return m.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# batched workload: 64 independent 2D instances of uneven size and order
# ---------------------------------------------------------------------------
def measure_batched(torch, dgconv, rank: int, world: int, flush, stream, mixed_prec: str, reps: int = 3):
    """The batched instances in one graph launch (mixed precision: the tensor-core
    split precision where it covers the order, FP32 otherwise) against one FP64
    rk_substeps launch per instance; same inputs, errors against the FP64 run."""
    insts = W.batched_instances(seed=5 + 1000 * rank)
    meshes, winds, v0s, ds, nsteps = [], [], [], [], []
    units = 0
    byts = 0
    for wl in insts:
        verts, elems = wl.mesh()
        m = dgconv.Mesh(2, wl.k, verts, elems)
        pot = dgconv.potential_values(m, wl.potential())
        w = m.wind_from_potential(torch.tensor(pot, dtype=torch.float64, device="cuda"))
        meshes.append(m)
        winds.append(w)
        v0s.append(torch.tensor(W.uniform_coeffs(wl.seed, m.n_elem, 2, wl.k), dtype=torch.float64, device="cuda"))
        ds.append(m.cfl_ds(w, wl.cfl))
        nsteps.append(wl.substeps)
        b, _, n = stage_bytes_flops(wl)
        units += m.n_elem * n * 2 * 3 * wl.substeps
        byts += b * m.n_elem * 3 * wl.substeps
    # autotuned block shapes of the CUDA-core kernel for the orders that use it
    # (k = 5, 6 in mixed precision; every order in the FP64 comparison), each tuned
    # on the largest instance of its order
    tuned = {}
    for k in sorted({wl.k for wl in insts}):
        j = max((i for i, wl in enumerate(insts) if wl.k == k), key=lambda i: meshes[i].n_elem)
        for prec in (("fp32", "fp64") if k > 4 else ("fp64",)):
            tuned[f"k{k}/{prec}"] = meshes[j].autotune(winds[j], prec)
    states = [v.clone() for v in v0s]

    def reset():
        for s_, v in zip(states, v0s):
            s_.copy_(v)

    def timed(fn):
        ts = []
        for rep in range(reps + 1):
            reset()
            flush.zero_()
            a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            b0.record(stream)
            torch.cuda.synchronize()
            if rep > 0:                                    # the first call builds the graphs
                ts.append(a0.elapsed_time(b0))
        return max_over_ranks(min(ts), world, "cuda")

    def mixed():
        dgconv.batch_rk_substeps(meshes, winds, states, ds, nsteps, 3, mixed_prec)

    def fp64():
        for m, w, s_, d, n in zip(meshes, winds, states, ds, nsteps):
            m.rk_substeps(w, s_, d, n, 3, "fp64")

    ms_mixed = timed(mixed)
    out_mixed = [s_.clone() for s_ in states]
    # the same graph restricted to the tensor-core orders and to the others
    sub_ms = {}
    for name, keep in (("k<=4 (tensor cores)", lambda k: k <= 4), ("k>=5 (CUDA cores, fp32)", lambda k: k > 4)):
        idx = [i for i, wl in enumerate(insts) if keep(wl.k)]
        if idx:
            sub_ms[name] = timed(lambda idx=idx: dgconv.batch_rk_substeps(
                [meshes[i] for i in idx], [winds[i] for i in idx], [states[i] for i in idx],
                [ds[i] for i in idx], [nsteps[i] for i in idx], 3, mixed_prec))
    ms_fp64 = timed(fp64)
    errs = [float((a - b).abs().max() / b.abs().max()) for a, b in zip(out_mixed, states)]
    err = max(errs)
    err_by_k = {f"k{k}": max(e for e, wl in zip(errs, insts) if wl.k == k) for k in sorted({wl.k for wl in insts})}
    units_by_k = {f"k{k}": sum(m.n_elem * math.comb(k + 2, 2) * 2 * 3 * 50 for m, wl in zip(meshes, insts)
                               if wl.k == k) for k in sorted({wl.k for wl in insts})}
    for m in meshes:
        m.check()
    hbm, _ = peaks()
    return {"instances": len(insts), "elements": sum(m.n_elem for m in meshes),
            "orders": sorted({wl.k for wl in insts}), "substeps": 50, "scheme": "SSP-RK3",
            "mixed": {"value": job_throughput(units, world, ms_mixed), "ms": ms_mixed,
                      "prec": f"{mixed_prec} (k <= 4), fp32 (k = 5, 6)", "launch": "one cached multi-branch CUDA graph",
                      "roofline_frac": byts / (ms_mixed * 1e-3) / 1e9 / hbm},
            "fp64_per_instance": {"value": job_throughput(units, world, ms_fp64), "ms": ms_fp64,
                                  "launch": "one cached graph per instance, in sequence"},
            "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed, "max_rel_err_vs_fp64": err,
            "autotuned_block": tuned, "max_rel_err_by_order": err_by_k, "units_by_order": units_by_k,
            "sub_batch_ms": sub_ms,
            "unit": "DOF-stage updates/s"}


def measure_shape(torch, dgconv, name: str, rank: int, world: int, flush, stream, steps: int = 2):
    """Another element shape in FP32 and FP64 (parallelograms: the sum-factorised stage
    kernel; curved triangles: the CUDA-core kernel with inverse mass blocks): the same
    step as the headline (a1, a2, 100 SSP-RK3 substeps, M^V, a8), the stage time from two
    graph lengths, and the stage kernel against its roofline."""
    wl = rank_workload(W.WORKLOADS[name], rank)
    mesh, wind, u_n, ds = make_inputs(wl, torch, dgconv)
    v, mv, g = mesh.dg_zeros(), mesh.dg_zeros(), mesh.hdiv_zeros()
    kernel = {"quad": "stage_quad_kernel", "hex": "stage_hex_kernel"}.get(wl.shape, "stage_kernel")
    byts, flops, N = stage_bytes_flops(wl)
    curved_frac = mesh.n_curved / wl.n_elem if wl.shape == "curved" else None
    if curved_frac:
        # the curved elements' inverse mass block: read once per stage (FP32 or FP64 like
        # the contraction; counted at 8 bytes) and multiplied into the residual
        byts = byts + curved_frac * N * N * 8
        flops = flops + curved_frac * 2 * N * N * wl.dim
    units = wl.n_elem * N * wl.dim * 3 * wl.substeps
    hbm, hbm_src = peaks()
    out = {"workload": wl.name, "elements": wl.n_elem, "k": wl.k, "substeps": wl.substeps,
           "unit": "DOF-stage updates/s", "alg_bytes_per_elem_stage": byts, "alg_flops_per_elem_stage": flops,
           "by_prec": {}}
    if curved_frac is not None:
        out["curved_elements"] = mesh.n_curved
    ref = None
    for prec in ("fp64", "fp32"):
        def step(p=prec):
            mesh.geometry()
            mesh.transfer(u_n, out=v)
            mesh.rk_substeps(wind, v, ds, wl.substeps, 3, p)
            mesh.mass(v, out=mv)
            mesh.transfer_T(mv, out=g)
        step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        x = mesh.transfer(u_n)
        mesh.rk_substeps(wind, x, ds, wl.substeps, 3, prec)
        torch.cuda.synchronize()
        if ref is None:
            ref = x
        err = float((x - ref).abs().max() / ref.abs().max())

        def time_rk(n, p=prec):
            best = None
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                a.record(stream)
                mesh.rk_substeps(wind, v, ds, n, 3, p)
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                best = t if best is None else min(best, t)
            return best
        n_lo = wl.substeps // 2
        mesh.rk_substeps(wind, v, ds, n_lo, 3, prec)
        t_lo = time_rk(n_lo)
        t_hi = time_rk(wl.substeps)
        stage_ms = (t_hi - t_lo) / (3 * (wl.substeps - n_lo))
        ms = max_over_ranks(statistics.mean(ts), world, "cuda")
        achieved = byts * wl.n_elem / (stage_ms * 1e-3) / 1e9
        tflops = flops * wl.n_elem / (stage_ms * 1e-3) / 1e12
        roof = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_source": hbm_src, "achieved_tflops": tflops,
                "traffic": ncu_traffic(wl, prec)}
        if prec == "fp64":
            # FP64 FMAs bound this variant: against the nominal FP64 rate of the part
            roof = {"bound": "alu", "kernel": kernel, "achieved": tflops, "peak": FP64_TFLOPS,
                    "unit": "TFLOP/s", "frac": tflops / FP64_TFLOPS, "peak_source": "nominal FP64 (no measured peak)",
                    "hbm_frac": achieved / hbm}
        out["by_prec"][prec] = {
            "value": job_throughput(units, world, ms), "ms_per_step": ms, "max_rel_err_vs_fp64": err,
            "stage_ms": stage_ms, "roofline": roof}
    return out


# ---------------------------------------------------------------------------
# oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def _oracle_setup(wl):
    """Mesh, wind, initial state and substep of a workload, by the oracle (untimed)."""
    from oracle import dg as ODG
    from oracle import hdiv as OH
    from oracle import mesh as OM
    verts, elems = wl.mesh()[:2]
    field = W.fourier_field(wl.seed + 2000, wl.dim)
    if wl.shape == "quad":
        from oracle import quad as OQ
        om = OQ.QuadMesh(verts, elems)
        nodes = OQ.lagrange_nodes(wl.k)
        X = om.to_physical(np.repeat(np.arange(om.n_elem), nodes.shape[0]), np.tile(nodes, (om.n_elem, 1)))
        wind = OQ.wind_from_potential(om, wl.k, wl.potential()(X[:, 0], X[:, 1]).reshape(om.n_elem, -1))
        v = OQ.transfer(om, wl.k, OQ.dofs_of_function(om, wl.k, lambda x: field(x)))
        return om, wind, v, OQ.cfl_ds(om, wl.k, wind, wl.cfl), (wl.k + 1) ** 2
    if wl.shape == "hex":
        from oracle import hexa as OX
        om = OX.HexMesh(verts, elems)
        nodes = OX.lagrange_nodes(wl.k)
        X = om.to_physical(np.repeat(np.arange(om.n_elem), nodes.shape[0]), np.tile(nodes, (om.n_elem, 1)))
        pot = np.moveaxis(np.asarray(wl.potential()(X[:, 0], X[:, 1], X[:, 2])), 0, -1).reshape(om.n_elem, -1, 3)
        wind = OX.wind_from_potential(om, wl.k, pot)
        v = OX.transfer(om, wl.k, OX.dofs_of_function(om, wl.k, lambda x: field(x)))
        return om, wind, v, OX.cfl_ds(om, wl.k, wind, wl.cfl), (wl.k + 1) ** 3
    om = OM.Mesh(verts, elems)
    wind = OH.wind_from_potential(om, wl.k, wl.potential())
    if wl.unit_peak_speed:
        wind = wind / ODG.max_wind_speed(om, wl.k, wind)
    v = ODG.transfer(om, wl.k, OH.dofs_of_function(om, wl.k, lambda x: field(x)))
    return om, wind, v, ODG.cfl_ds(om, wl.k, wind, wl.cfl), math.comb(wl.k + wl.dim, wl.dim)


def _oracle_block(wl_name, lo, hi, wind, v, ds, warm, steps, barrier, queue):
    """One process of the oracle timing: the operator on elements [lo, hi) (its own
    ``sel``), warm untimed and `steps` timed explicit stages, in lockstep with the others."""
    wl = W.WORKLOADS[wl_name]
    verts, elems = wl.mesh()[:2]
    sel = np.arange(lo, hi)
    if wl.shape == "quad":
        from oracle import quad as OQ
        op = OQ.QuadConvectionOracle(OQ.QuadMesh(verts, elems), wl.k, wind, sel=sel)
    elif wl.shape == "hex":
        from oracle import hexa as OX
        op = OX.HexConvectionOracle(OX.HexMesh(verts, elems), wl.k, wind, sel=sel)
    else:
        from oracle import dg as ODG
        from oracle import mesh as OM
        op = ODG.ConvectionOracle(OM.Mesh(verts, elems), wl.k, wind, sel=sel)
    for _ in range(warm):
        op.apply(v)
    times = []
    for _ in range(steps):
        if barrier is not None:
            barrier.wait()
        t0 = time.perf_counter()
        _ = v[sel] + ds * (-op.apply(v))
        times.append(time.perf_counter() - t0)
    queue.put((lo, hi, times))


class OracleTimer:
    """The FP64 numpy oracle, as it stands, timed on the host cores: P spawned processes
    (one BLAS thread each) each apply the operator to their own contiguous block of
    elements (``sel``), in lockstep; a stage takes the slowest block's time.  The 1-core
    rate times one block alone."""

    def __init__(self, wl):
        if wl.shape == "curved":
            raise ValueError("the timed oracle covers affine simplices, parallelograms and parallelepipeds")
        self.wl = wl
        om, self.wind, self.v, self.ds, N = _oracle_setup(wl)
        self.E = om.n_elem
        self.units_per_stage = self.E * N * wl.dim
        try:
            self.cores = len(os.sched_getaffinity(0))
        except AttributeError:
            self.cores = os.cpu_count() or 1

    def _run(self, blocks, warm, steps):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"                         # inherited by the spawned processes
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        bar = ctx.Barrier(len(blocks)) if len(blocks) > 1 else None
        procs = [ctx.Process(target=_oracle_block, args=(self.wl.name, lo, hi, self.wind, self.v, self.ds, warm,
                                                         steps, bar, q)) for lo, hi in blocks]
        for pr in procs:
            pr.start()
        res = [q.get() for _ in procs]
        for pr in procs:
            pr.join()
        return res

    def rates(self, warm: int = 1, steps: int = 2):
        """(all-core rate, its per-stage seconds, 1-core rate) in DOF-stage updates/s."""
        P = self.cores
        edges = np.linspace(0, self.E, P + 1).astype(int)
        blocks = [(int(edges[j]), int(edges[j + 1])) for j in range(P)]
        res = self._run(blocks, warm, steps)
        stage_s = [max(r[2][i] for r in res) for i in range(steps)]
        all_core = self.units_per_stage / statistics.mean(stage_s)
        lo, hi = blocks[0]
        one = self._run([(lo, hi)], warm, steps)[0]
        one_core = self.units_per_stage * (hi - lo) / self.E / statistics.mean(one[2])
        return all_core, stage_s, one_core


def run_reference(args, rank):
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    timer = OracleTimer(wl)
    value, stage_s, one_core = timer.rates(warm=args.warmup, steps=args.steps)
    sample = (f"per step one explicit stage (E*N*dim DOF updates) of the FP64 numpy oracle on the full mesh, "
              f"split into {timer.cores} element blocks timed in lockstep by {timer.cores} processes "
              f"(1 BLAS thread each)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-stage updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(stage_s), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "elements": wl.n_elem, "k": wl.k, "dim": wl.dim, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "DOF-stage updates/s", "cores": timer.cores, "kind": "oracle",
                         "sample": sample, "one_core_value": one_core},
        "e2e": {"value": value, "unit": "DOF-stage updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    from paper_1508_04245_gb300 import build, dgconv
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = rank_workload(W.WORKLOADS[args.workload], rank)
    substeps = args.substeps or wl.substeps
    mesh, wind, u_n, ds = make_inputs(wl, torch, dgconv)
    stream = torch.cuda.current_stream()
    v = mesh.dg_zeros()
    mv = mesh.dg_zeros()
    g = mesh.hdiv_zeros()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(un=u_n, wnd=wind):
        mesh.geometry()                                   # a1
        mesh.transfer(un, out=v)                          # a2
        mesh.rk_substeps(wnd, v, ds, substeps, 3, args.prec)   # a3..a7
        mesh.mass(v, out=mv)                              # a6 (M^V)
        mesh.transfer_T(mv, out=g)                        # a8
    # geometry, transfer, [wind prep (+ layout in/out on the tensor-core path), stages], mass, transfer_T (2)
    # (+1 in FP32: the FP32 copy of the state at the start of the RK sequence)
    launches_per_step = 1 + 1 + (1 + 3 * substeps + (2 if args.prec in TC_PRECS else 0)
                                 + (1 if args.prec == "fp32" else 0)) + 1 + 2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()                                     # evict L2 between timed steps
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]

    # stage-kernel duration: difference of two graph lengths cancels the per-call kernels
    def time_rk(n, reps=3):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            mesh.rk_substeps(wind, v, ds, n, 3, args.prec)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)
    n_lo = max(substeps // 2, 1)
    mesh.rk_substeps(wind, v, ds, n_lo, 3, args.prec)
    t_lo = time_rk(n_lo)
    mesh.rk_substeps(wind, v, ds, substeps, 3, args.prec)
    t_hi = time_rk(substeps)
    stage_ms = (t_hi - t_lo) / (3 * (substeps - n_lo))

    # end to end through the public calls with host buffers
    u_host = torch.empty(mesh.n_hdiv, dtype=torch.float64, pin_memory=True)
    w_host = torch.empty(mesh.n_hdiv, dtype=torch.float64, pin_memory=True)
    g_host = torch.empty(mesh.n_hdiv, dtype=torch.float64, pin_memory=True)
    u_host.copy_(u_n)
    w_host.copy_(wind)
    u_dev = torch.empty_like(u_n)
    w_dev = torch.empty_like(wind)
    e2e_ms = []
    for i in range(max(args.steps, 1)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        u_dev.copy_(u_host, non_blocking=True)
        w_dev.copy_(w_host, non_blocking=True)
        step(u_dev, w_dev)
        g_host.copy_(g, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))

    # error of the mixed path against the FP64 GPU path (itself pinned to the oracle)
    err = None
    if args.prec != "fp64":
        v64 = mesh.transfer(u_n)
        mesh.rk_substeps(wind, v64, ds, substeps, 3, "fp64")
        vmx = mesh.transfer(u_n)
        mesh.rk_substeps(wind, vmx, ds, substeps, 3, args.prec)
        torch.cuda.synchronize()
        err = float((vmx - v64).abs().max() / v64.abs().max())

    ms = max_over_ranks(statistics.mean(step_ms), world, "cuda")
    e2e_ms_max = max_over_ranks(statistics.mean(e2e_ms), world, "cuda")
    byts, flops, N = stage_bytes_flops(wl)
    units_per_step = wl.n_elem * N * wl.dim * 3 * substeps
    value = job_throughput(units_per_step, world, ms)
    e2e_val = job_throughput(units_per_step, world, e2e_ms_max)
    hbm, hbm_src = peaks()
    achieved = byts * wl.n_elem / (stage_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": ncu_traffic(wl, args.prec), "peak_source": hbm_src,
            "kernel": ("stage_tc_kernel" if args.prec in TC_PRECS
                       else {"quad": "stage_quad_kernel", "hex": "stage_hex_kernel"}.get(wl.shape, "stage_kernel")),
            "stage_ms": stage_ms, "alg_bytes_per_elem_stage": byts, "alg_flops_per_elem_stage": flops,
            "achieved_tflops": flops * wl.n_elem / (stage_ms * 1e-3) / 1e12}
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stage updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": {"workload": wl.name, "elements": wl.n_elem, "dim": wl.dim, "k": wl.k, "substeps": substeps,
                   "scheme": "SSP-RK3", "prec": args.prec, "l2": "flushed between timed steps",
                   "step": "a1 geometry, a2 I, 100x RK3 (a3-a7), M^V, a8 I^T"},
        "max_rel_err_vs_fp64": err,
        "e2e": {"value": e2e_val, "unit": "DOF-stage updates/s", "h2d_bytes_per_step": 2 * mesh.n_hdiv * 8,
                "d2h_bytes_per_step": mesh.n_hdiv * 8},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
    }
    if not args.no_other_precisions:
        # the same step at the other contraction precisions (1 warm-up, 2 timed steps each)
        others = {}
        for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
            if prec == args.prec or (prec in TC_PRECS and not (wl.dim == 2 and wl.k <= 4 and wl.shape == "simplex")):
                continue

            def step_p(p=prec):
                mesh.geometry()
                mesh.transfer(u_n, out=v)
                mesh.rk_substeps(wind, v, ds, substeps, 3, p)
                mesh.mass(v, out=mv)
                mesh.transfer_T(mv, out=g)
            step_p()
            torch.cuda.synchronize()
            ts = []
            for _ in range(2):
                flush.zero_()
                a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                step_p()
                b0.record(stream)
                torch.cuda.synchronize()
                ts.append(a0.elapsed_time(b0))
            v64 = mesh.transfer(u_n)
            mesh.rk_substeps(wind, v64, ds, substeps, 3, "fp64")
            vp = mesh.transfer(u_n)
            mesh.rk_substeps(wind, vp, ds, substeps, 3, prec)
            torch.cuda.synchronize()
            e_p = float((vp - v64).abs().max() / v64.abs().max())
            ms_p = max_over_ranks(statistics.mean(ts), world, "cuda")
            others[prec] = {"value": job_throughput(units_per_step, world, ms_p),
                            "ms_per_step": ms_p, "max_rel_err_vs_fp64": e_p}
        line["other_precisions"] = others
    # the implicit convection step by pseudo-time iteration (Sec. 3.3.2): 20 capped
    # Richardson iterations on the same mesh and wind, timed as one graph launch
    rich_iters = 20
    tau = 2.0 * mesh.cfl_ds(wind, 1.0)
    ds_r = mesh.richardson_ds(wind, tau)
    g_r = mesh.transfer(u_n)
    v_r = mesh.dg_zeros()
    it_r = torch.zeros(1, dtype=torch.int32, device="cuda")
    res_r = torch.zeros(rich_iters + 1, dtype=torch.float64, device="cuda")
    rich = {}
    for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
        if prec in TC_PRECS and not (wl.dim == 2 and wl.k <= 4 and wl.shape == "simplex"):
            continue
        if wl.shape == "curved":        # the pseudo-time solve takes affine meshes
            break
        ts = []
        for rep in range(4):
            v_r.zero_()
            flush.zero_()
            a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            mesh.richardson(wind, g_r, v_r, tau, ds_r, 0.0, rich_iters, prec=prec, iters=it_r, res=res_r)
            b0.record(stream)
            torch.cuda.synchronize()
            if rep > 0:                                    # the first call builds the graph
                ts.append(a0.elapsed_time(b0))
        ms_it = max_over_ranks(min(ts), world, "cuda") / (rich_iters + 1)   # operator evaluations
        rich[prec] = {"ms_per_iteration": ms_it,
                      "value": job_throughput(wl.n_elem * N * wl.dim, world, ms_it),
                      "roofline_frac": byts * wl.n_elem / (ms_it * 1e-3) / 1e9 / hbm,
                      "residual_reduction": float(res_r[rich_iters] / res_r[0])}
    line["richardson"] = {"unit": "DOF updates/s (one residual + update per iteration)", "iterations": rich_iters,
                          "tau": tau, "ds": ds_r, "by_prec": rich,
                          "note": "operator evaluations = iterations + 1; roofline against the same "
                                  "algorithmic bytes per element as one stage"}
    if not args.no_batched:
        line["batched"] = measure_batched(torch, dgconv, rank, world, flush, stream,
                                          args.prec if args.prec in TC_PRECS else "bf16x3")
    if not args.no_shapes and wl.shape == "simplex":
        line["parallelogram"] = measure_shape(torch, dgconv, "parallelogram256_k4", rank, world, flush, stream)
        line["curved"] = measure_shape(torch, dgconv, "curved256_k4", rank, world, flush, stream)
        line["parallelepiped"] = measure_shape(torch, dgconv, "parallelepiped32_k3", rank, world, flush, stream)
    # clocks sampled from before the first timed step to the end of the GPU measurements
    line["clocks"] = clocks.stop()
    if rank == 0 and world == 1 and not args.no_cpu_baseline and wl.shape != "curved":
        timer = OracleTimer(wl)
        rate, stage_s, one_core = timer.rates(warm=1, steps=2)
        line["cpu_baseline"] = {"value": rate, "unit": "DOF-stage updates/s", "cores": timer.cores,
                                "kind": "oracle", "one_core_value": one_core,
                                "sample": f"2 explicit stages of the FP64 numpy oracle on the full {wl.n_elem}-element "
                                          f"mesh in {timer.cores} element blocks, one process (1 BLAS thread) each, "
                                          f"in lockstep ({sum(stage_s):.1f} s); one_core_value: one block alone"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
