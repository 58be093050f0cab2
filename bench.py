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
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other simplex configurations (square16_k2, cube32_k3, cube48_k4)")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle runs (errors against the oracle and the cpu_baseline)")
    args = ap.parse_args()
    if args.impl == "dgconv" and args.prec in TC_PRECS and not tc_covers(W.WORKLOADS[args.workload], args.prec):
        ap.error("the tensor-core precisions cover affine triangles with k <= 6 and tetrahedra with k <= 4 (bf16x3 only); "
                 "use --prec fp32 or fp64 here")
    return args


def tc_covers(wl, prec) -> bool:
    """Whether the tensor-core path of the library covers a workload at a precision."""
    return wl.shape == "simplex" and (wl.k <= 6 if wl.dim == 2 else (wl.k <= 4 and prec == "bf16x3"))


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
    ("cube48_k4", "bf16x3"): ("stage_tc3_kernel_cube48_k4.md", "dgc_stage_tc3.cuh"),
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


def bf16_peak():
    """Dense bf16 tensor rate (TFLOP/s) for a kernel timed inside a long step: the
    sustained measured figure, else the burst one, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        for key in ("bf16_tflops_sustained", "bf16_tflops"):
            if m.get(key):
                return float(m[key]), f"measured ({key})"
    return 1700.0, "fallback (sustained)"


def measure_fp64_peak(torch):
    """FP64 rate of this GPU (TFLOP/s), measured here: a cuBLAS DGEMM of 4096^3, best of 5."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


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
    for name, keep in (("k<=4 (two CTAs per SM)", lambda k: k <= 4), ("k>=5 (one CTA per SM)", lambda k: k >= 5)):
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
                      "prec": f"{mixed_prec} (every order on the tensor cores)",
                      "launch": "one cached CUDA graph; per order one persistent launch per RK stage over "
                                "the element tiles of all instances of that order; k <= 4 (two CTAs per "
                                "SM) first, then k = 5, 6 (one CTA per SM), the orders of a phase "
                                "concurrently",
                      "roofline_frac": byts / (ms_mixed * 1e-3) / 1e9 / hbm},
            "fp64_per_instance": {"value": job_throughput(units, world, ms_fp64), "ms": ms_fp64,
                                  "launch": "one cached graph per instance, in sequence"},
            "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed, "max_rel_err_vs_fp64": err,
            "autotuned_block": tuned, "max_rel_err_by_order": err_by_k, "units_by_order": units_by_k,
            "sub_batch_ms": sub_ms,
            "unit": "DOF-stage updates/s"}


def measure_shape(torch, dgconv, name: str, rank: int, world: int, flush, stream, steps: int = 2,
                  fp64_tflops=None):
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
            # FP64 FMAs bound this variant: against the FP64 rate measured in this run (a
            # DGEMM), else the nominal FP64 rate of the part
            peak64 = fp64_tflops or FP64_TFLOPS
            roof = {"bound": "alu", "kernel": kernel, "achieved": tflops, "peak": peak64,
                    "unit": "TFLOP/s", "frac": tflops / peak64,
                    "peak_source": "FP64 DGEMM measured in this run" if fp64_tflops else "nominal FP64 (no measured peak)",
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

    def one_core_rate(self, warm: int = 1, steps: int = 1):
        """DOF-stage updates/s of one block of E / cores elements timed alone (one core)."""
        hi = max(1, self.E // self.cores)
        one = self._run([(0, hi)], warm, steps)[0]
        return self.units_per_stage * hi / self.E / statistics.mean(one[2])


# ---------------------------------------------------------------------------
# the oracle on the whole mesh over the host cores: the reference result of a
# workload's RK sequence and the cpu_baseline rate
# ---------------------------------------------------------------------------
def _shm_view(name, shape):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf)


def _oracle_rk_worker(wl, p, lo, hi, nsteps, names, shapes, barrier, queue):
    """Process p of the parallel oracle run: elements [lo, hi) of workload wl.

    Every process builds the oracle's mesh; the wind, its peak speed and the
    initial state are computed over the process's elements (the element
    restrictions of the oracle's builders, in sub-blocks for memory) into
    shared arrays; then each stage of every substep applies the oracle's
    operator to the block (its ``sel``) between barriers, so the shared state
    goes through the SSP-RK sequence of ``oracle.dg.rk_substeps``."""
    from oracle import dg as ODG
    from oracle import hdiv as OH
    from oracle import mesh as OM
    views = {key: _shm_view(nm, shapes[key]) for key, nm in names.items()}
    A = {key: v[1] for key, v in views.items()}
    verts, elems = wl.mesh()[:2]
    om = OM.Mesh(verts, elems)
    k, d = wl.k, wl.dim
    block = np.arange(lo, hi)
    subs = np.array_split(block, max(1, (hi - lo) // 2048))
    t0 = time.perf_counter()
    for sub in subs:                       # the wind's DOFs owned by this block
        w = OH.wind_from_potential(om, k, wl.potential(), elems=sub)
        nz = np.nonzero(w)[0]
        A["wind"][nz] = w[nz]
    barrier.wait()
    wind = A["wind"].copy()
    A["speed"][p] = ODG.max_wind_speed(om, k, wind, sel=block)
    barrier.wait()
    if wl.unit_peak_speed:
        wind = wind / A["speed"].max()
        barrier.wait()
        A["speed"][p] = ODG.max_wind_speed(om, k, wind, sel=block)
        barrier.wait()
    ds = wl.cfl * float(om.shortest_edge().min()) / ((2 * k + 1) * A["speed"].max())   # reading A7
    v, v1, v2 = A["v"], A["v1"], A["v2"]
    if wl.state == "fourier":
        field = W.fourier_field(wl.seed + 2000, d)
        for sub in subs:
            u = OH.dofs_of_function(om, k, lambda x: field(x), elems=sub)
            nz = np.nonzero(u)[0]
            A["un"][nz] = u[nz]
        barrier.wait()
        for sub in subs:
            v[sub] = ODG.transfer(om, k, A["un"], sel=sub)
    else:
        v[block] = W.uniform_coeffs(wl.seed, om.n_elem, d, k)[block]
    barrier.wait()
    op = ODG.ConvectionOracle(om, k, wind, sel=block)
    setup_s = time.perf_counter() - t0
    L = lambda x: -op.apply(x)            # noqa: E731
    stage_s = []

    def stage(f):
        t = time.perf_counter()
        f()
        stage_s.append(time.perf_counter() - t)
        barrier.wait()
    if wl.name == "square16_k2":           # this configuration also applies the operator once
        A["apply"][block] = op.apply(v)
        barrier.wait()
    for _ in range(nsteps):
        if wl.scheme == 2:
            stage(lambda: v1.__setitem__(block, v[block] + ds * L(v)))
            stage(lambda: v.__setitem__(block, 0.5 * v[block] + 0.5 * (v1[block] + ds * L(v1))))
        else:
            stage(lambda: v1.__setitem__(block, v[block] + ds * L(v)))
            stage(lambda: v2.__setitem__(block, 0.75 * v[block] + 0.25 * (v1[block] + ds * L(v1))))
            stage(lambda: v.__setitem__(block, v[block] / 3.0 + 2.0 / 3.0 * (v2[block] + ds * L(v2))))
    queue.put((p, ds, setup_s, stage_s))
    for shm, _ in views.values():
        shm.close()


def oracle_rk(wl, nsteps: int, procs: int | None = None):
    """The oracle's RK sequence of workload wl (its wind, initial state and CFL
    substep) on the whole mesh, split over the host cores.  Returns a dict with
    the final state, the operator applied to the initial state (square16_k2),
    the substep size, the stage times (slowest process) and the core count."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    from oracle import basis as OB
    from oracle import mesh as OM
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    P = min(procs or cores, wl.n_elem)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"                             # inherited by the spawned processes
    N = OB.dim_pk(wl.dim, wl.k)
    verts, elems = wl.mesh()[:2]
    n_hdiv = OM.Mesh(verts, elems).n_facets * OB.hdiv_counts(wl.dim, wl.k)[0] + \
        wl.n_elem * OB.hdiv_counts(wl.dim, wl.k)[1]
    shapes = {"wind": (n_hdiv,), "un": (n_hdiv,), "speed": (P,), "v": (wl.n_elem, wl.dim, N),
              "v1": (wl.n_elem, wl.dim, N), "v2": (wl.n_elem, wl.dim, N), "apply": (wl.n_elem, wl.dim, N)}
    shms = {key: shared_memory.SharedMemory(create=True, size=max(8, int(np.prod(sh)) * 8))
            for key, sh in shapes.items()}
    try:
        for key, sh in shapes.items():
            np.ndarray(sh, dtype=np.float64, buffer=shms[key].buf)[...] = 0.0
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        bar = ctx.Barrier(P)
        edges = np.linspace(0, wl.n_elem, P + 1).astype(int)
        names = {key: sm.name for key, sm in shms.items()}
        ps = [ctx.Process(target=_oracle_rk_worker, args=(wl, p, int(edges[p]), int(edges[p + 1]), nsteps,
                                                           names, shapes, bar, q)) for p in range(P)]
        t0 = time.perf_counter()
        for pr in ps:
            pr.start()
        res = [q.get() for _ in ps]
        for pr in ps:
            pr.join()
        wall = time.perf_counter() - t0
        out = {"v": np.ndarray(shapes["v"], dtype=np.float64, buffer=shms["v"].buf).copy(),
               "apply": np.ndarray(shapes["apply"], dtype=np.float64, buffer=shms["apply"].buf).copy(),
               "ds": res[0][1], "setup_s": max(r[2] for r in res), "cores": P, "wall_s": wall}
        n_st = len(res[0][3])
        out["stage_s"] = [max(r[3][i] for r in res) for i in range(n_st)]
        return out
    finally:
        for sm in shms.values():
            sm.close()
            sm.unlink()


def oracle_apply_sample(wl, w, sel):
    """The oracle's operator on the elements sel of workload wl (its unscaled wind,
    computed only where those elements need it) applied to the state w."""
    from oracle import dg as ODG
    from oracle import hdiv as OH
    from oracle import mesh as OM
    verts, elems = wl.mesh()[:2]
    om = OM.Mesh(verts, elems)
    nb = om.nbr[sel]
    need = np.unique(np.concatenate([sel, nb[nb >= 0]]))   # owners of the selected elements' facets
    wind = OH.wind_from_potential(om, wl.k, wl.potential(), elems=need)
    return ODG.ConvectionOracle(om, wl.k, wind, sel=sel).apply(w)


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


class OracleJobs(threading.Thread):
    """The oracle runs of the benchmark, one after another on the host cores while
    the GPU measurements proceed (spawned processes; none of them touches CUDA)."""

    def __init__(self, jobs):
        super().__init__(daemon=True)
        self.jobs = jobs
        self.results = {}

    def run(self):
        for key, fn in self.jobs:
            t0 = time.perf_counter()
            try:
                self.results[key] = fn()
            except Exception as ex:            # reported in the JSON line, never silent
                self.results[key] = {"error": repr(ex)}
            self.results[key]["job_s"] = time.perf_counter() - t0


# the slice of the RK sequence the oracle runs on the full mesh, per configuration
# (square256_k4 and square16_k2 in full; cube32_k3 the first 4 substeps of 50)
ORACLE_SUBSTEPS = {"square16_k2": 10, "square256_k4": 100, "cube32_k3": 4}
SAMPLE_ELEMS = 1024     # cube48_k4: one operator application on sampled elements


def sample_elements(wl):
    """Seeded element sample of a workload (first and last tile edges included)."""
    sel = np.random.default_rng(wl.seed + 77).choice(wl.n_elem, size=SAMPLE_ELEMS, replace=False)
    return np.unique(np.concatenate([sel, [0, 39, 40, wl.n_elem - 1]]))


def oracle_jobs_for(names):
    jobs = []
    for name in names:
        wl = W.WORKLOADS[name]
        if name in ORACLE_SUBSTEPS:
            jobs.append((name, lambda wl=wl: oracle_rk(wl, ORACLE_SUBSTEPS[wl.name])))
        else:
            def sample(wl=wl):
                w = W.uniform_coeffs(wl.seed, wl.n_elem, wl.dim, wl.k)
                sel = sample_elements(wl)
                return {"apply": oracle_apply_sample(wl, w, sel), "sel": sel}
            jobs.append((name, sample))
    return jobs


def stage_roofline(wl, stage_ms, hbm, hbm_src, bf16, bf16_src, prec, fp64_tflops=None):
    """Roofline of one stage launch: the algorithmic bytes at the HBM rate, and the
    algorithmic flops at the rate of the arithmetic that carries them (the split
    BF16x3 contractions issue six tensor-core products per FP32 product; FP64 runs
    on the FP64 pipe); the binding bound is the larger time."""
    byts, flops, _ = stage_bytes_flops(wl)
    t_hbm = byts * wl.n_elem / (hbm * 1e9)
    out = {"kernel": ("stage_tc3_kernel" if wl.dim == 3 else "stage_tc_kernel") if prec in TC_PRECS
           else "stage_kernel", "stage_ms": stage_ms,
           "alg_bytes_per_elem_stage": byts, "alg_flops_per_elem_stage": flops,
           "hbm_bound_ms": 1e3 * t_hbm, "achieved_gbs": byts * wl.n_elem / (stage_ms * 1e-3) / 1e9}
    if prec in TC_PRECS:
        t_t = 6.0 * flops * wl.n_elem / (bf16 * 1e12)
        out["tensor_bound_ms"] = 1e3 * t_t
        if t_t > t_hbm:
            out.update(bound="tensor", achieved=6.0 * flops * wl.n_elem / (stage_ms * 1e-3) / 1e12, peak=bf16,
                       unit="TFLOP/s", peak_source=bf16_src + ", 6 bf16 products per FP32 product")
        else:
            out.update(bound="hbm", achieved=out["achieved_gbs"], peak=hbm, unit="GB/s", peak_source=hbm_src)
    elif prec == "fp64" and fp64_tflops:
        out.update(bound="alu", achieved=flops * wl.n_elem / (stage_ms * 1e-3) / 1e12, peak=fp64_tflops,
                   unit="TFLOP/s", peak_source="FP64 DGEMM measured in this run")
    else:
        out.update(bound="hbm", achieved=out["achieved_gbs"], peak=hbm, unit="GB/s", peak_source=hbm_src)
    out["frac"] = out["achieved"] / out["peak"]
    out["traffic"] = ncu_traffic(wl, prec)
    out["traffic_source"] = ("committed ncu capture of this kernel source, scaled to this workload's elements as its "
                             "summary states (None once the source changed or without a capture)")
    return out


def measure_config(torch, dgconv, name, rank, world, flush, stream, fp64_tflops):
    """One of the simplex configurations (square16_k2, cube32_k3, cube48_k4): the
    configured RK sequence per precision (its step time, or for long FP64 runs the
    step extrapolated from the stage time), the stage kernel against its roofline,
    and the inputs of the comparison with the oracle (run afterwards)."""
    wl = rank_workload(W.WORKLOADS[name], rank)
    verts, elems = wl.mesh()[:2]
    mesh = dgconv.Mesh(wl.dim, wl.k, verts, elems)
    wind = mesh.wind_from_potential(torch.tensor(dgconv.potential_values(mesh, wl.potential()),
                                                 dtype=torch.float64, device="cuda"))
    wind_raw = wind.clone()
    if wl.unit_peak_speed:
        wind /= mesh.max_wind_speed(wind)
    ds = mesh.cfl_ds(wind, wl.cfl)
    v0 = torch.tensor(W.uniform_coeffs(wl.seed, wl.n_elem, wl.dim, wl.k), dtype=torch.float64, device="cuda")
    byts, flops, N = stage_bytes_flops(wl)
    stages = wl.scheme * wl.substeps
    units = wl.n_elem * N * wl.dim * (stages + (1 if name == "square16_k2" else 0))
    hbm, hbm_src = peaks()
    bf16, bf16_src = bf16_peak()
    v = mesh.dg_zeros()
    out = {"workload": wl.name, "elements": wl.n_elem, "dim": wl.dim, "k": wl.k, "substeps": wl.substeps,
           "scheme": f"SSP-RK{wl.scheme}", "unit": "DOF-stage updates/s", "by_prec": {}}

    def step(p):
        if name == "square16_k2":
            mesh.conv_apply(wind, v0, out=v, prec=p)
        v.copy_(v0)
        mesh.rk_substeps(wind, v, ds, wl.substeps, wl.scheme, p)

    def time_rk(n, p, reps=3):
        best = 1e30
        for _ in range(reps):
            v.copy_(v0)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            mesh.rk_substeps(wind, v, ds, n, wl.scheme, p)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best
    for prec in ("bf16x3", "fp32", "fp64"):
        if prec in TC_PRECS and not tc_covers(wl, prec):
            continue
        # two graph lengths whose difference is a few hundred milliseconds of stages
        mesh.rk_substeps(wind, v, ds, 1, wl.scheme, prec)
        est = time_rk(1, prec, reps=1) / wl.scheme
        n_hi = max(2, min(wl.substeps // 2, int(300.0 / (wl.scheme * max(est, 1e-3)))))
        n_lo = max(1, n_hi // 3)
        mesh.rk_substeps(wind, v, ds, n_lo, wl.scheme, prec)          # graphs built outside the timing
        mesh.rk_substeps(wind, v, ds, n_hi, wl.scheme, prec)
        t_lo, t_hi = time_rk(n_lo, prec), time_rk(n_hi, prec)
        stage_ms = max((t_hi - t_lo) / (wl.scheme * (n_hi - n_lo)), 1e-6)
        rec = {"stage_ms": stage_ms}
        if stage_ms * stages < 5000.0:                                # the whole configured step, timed
            step(prec)
            torch.cuda.synchronize()
            ts = []
            for _ in range(2):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step(prec)
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = max_over_ranks(min(ts), world, "cuda")
            rec.update(ms_per_step=ms, value=job_throughput(units, world, ms))
        else:
            ms = stage_ms * stages
            rec.update(ms_per_step_from_stage=ms, value=job_throughput(units, world, ms),
                       value_note="step extrapolated from the stage time (the full FP64 run takes minutes)")
        rec["roofline"] = stage_roofline(wl, stage_ms, hbm, hbm_src, bf16, bf16_src, prec, fp64_tflops)
        mesh.check()
        out["by_prec"][prec] = rec
    out["_gpu"] = {"mesh": mesh, "wind": wind, "wind_raw": wind_raw, "v0": v0, "ds": ds}
    return out


def config_errors(torch, cfg, orc):
    """The configuration's GPU results against the oracle's (reading A17, max-norm
    relative): the oracle's RK slice from the same initial state with the oracle's
    substep, or (cube48_k4) one operator application on sampled elements with the
    unscaled wind; plus the whole configured run of each mixed precision against the
    FP64 GPU run (short for cube48_k4, whose FP64 run takes minutes)."""
    g = cfg.pop("_gpu")
    mesh, wind, v0 = g["mesh"], g["wind"], g["v0"]
    wl = W.WORKLOADS[cfg["workload"]]
    errs = {}
    if orc is None or "error" in orc:
        errs["oracle"] = {"error": None if orc is None else orc["error"]}
    elif "sel" in orc:
        sel = orc["sel"]
        ref = orc["apply"]
        for prec in cfg["by_prec"]:
            got = mesh.conv_apply(g["wind_raw"], v0, prec=prec).cpu().numpy()[sel]
            errs[prec] = float(np.abs(got - ref).max() / np.abs(ref).max())
        errs["oracle"] = {"what": f"conv_apply on {sel.size} sampled elements (unscaled wind)",
                          "oracle_s": orc["job_s"]}
    else:
        ns = ORACLE_SUBSTEPS[wl.name]
        for prec in cfg["by_prec"]:
            x = v0.clone()
            mesh.rk_substeps(wind if not wl.unit_peak_speed else wind, x, orc["ds"], ns, wl.scheme, prec)
            got = x.cpu().numpy()
            errs[prec] = float(np.abs(got - orc["v"]).max() / np.abs(orc["v"]).max())
        if wl.name == "square16_k2":
            for prec in cfg["by_prec"]:
                got = mesh.conv_apply(wind, v0, prec=prec).cpu().numpy()
                errs[f"conv_apply/{prec}"] = float(np.abs(got - orc["apply"]).max() / np.abs(orc["apply"]).max())
        errs["oracle"] = {"what": f"{ns} of {wl.substeps} substeps on the full mesh from the same state, the "
                                  f"oracle's substep {orc['ds']:.6g}", "cores": orc["cores"],
                          "oracle_s": orc["job_s"]}
    cfg["max_rel_err_vs_oracle"] = errs
    # the whole configured run of the mixed precisions against FP64 on the GPU
    ns = wl.substeps if wl.name != "cube48_k4" else 4
    ref = v0.clone()
    mesh.rk_substeps(wind, ref, g["ds"], ns, wl.scheme, "fp64")
    vs = {}
    for prec in cfg["by_prec"]:
        if prec == "fp64":
            continue
        x = v0.clone()
        mesh.rk_substeps(wind, x, g["ds"], ns, wl.scheme, prec)
        vs[prec] = float((x - ref).abs().max() / ref.abs().max())
    cfg["max_rel_err_vs_fp64_gpu"] = {"substeps": ns, **vs}
    mesh.check()


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    # the oracle runs on the host cores while the GPU is measured (rank 0 of a 1-GPU run)
    use_oracle = rank == 0 and world == 1 and not args.no_oracle and args.workload == WORKLOAD
    config_names = [] if (args.no_configs or args.workload != WORKLOAD) else ["square16_k2", "cube32_k3", "cube48_k4"]
    oracle = None
    if use_oracle:
        oracle = OracleJobs(oracle_jobs_for([WORKLOAD] + config_names))
        oracle.start()
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
    n_hi = max(substeps, n_lo + 1)
    mesh.rk_substeps(wind, v, ds, n_lo, 3, args.prec)
    t_lo = time_rk(n_lo)
    mesh.rk_substeps(wind, v, ds, n_hi, 3, args.prec)
    t_hi = time_rk(n_hi)
    stage_ms = (t_hi - t_lo) / (3 * (n_hi - n_lo))

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

    # error of the mixed path against the FP64 GPU path (itself pinned to the oracle);
    # the error against the oracle follows once its run has finished
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
    bf16, bf16_src = bf16_peak()
    roof = stage_roofline(wl, stage_ms, hbm, hbm_src, bf16, bf16_src, args.prec)
    if args.prec not in TC_PRECS:
        roof["kernel"] = {"quad": "stage_quad_kernel", "hex": "stage_hex_kernel"}.get(wl.shape, "stage_kernel")
    roof["traffic"] = ncu_traffic(wl, args.prec)
    roof["traffic_source"] = "committed ncu capture of this kernel source (None once the source changed)"
    roof["achieved_tflops"] = flops * wl.n_elem / (stage_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stage updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}[args.prec],
        "data": "synthetic",
        "config": {"workload": wl.name, "elements": wl.n_elem, "dim": wl.dim, "k": wl.k, "substeps": substeps,
                   "scheme": "SSP-RK3", "prec": args.prec, "l2": "flushed between timed steps",
                   "step": "a1 geometry, a2 I, 100x RK3 (a3-a7), M^V, a8 I^T"},
        "max_rel_err_vs_fp64_gpu": err,
        "e2e": {"value": e2e_val, "unit": "DOF-stage updates/s", "h2d_bytes_per_step": 2 * mesh.n_hdiv * 8,
                "d2h_bytes_per_step": mesh.n_hdiv * 8},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roof,
    }
    if not args.no_other_precisions:
        # the same step at the other contraction precisions (1 warm-up, 2 timed steps each)
        others = {}
        for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
            if prec == args.prec or (prec in TC_PRECS and not tc_covers(wl, prec)):
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
        if prec in TC_PRECS and not tc_covers(wl, prec):
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
    fp64_tflops = measure_fp64_peak(torch)
    line["fp64_peak_tflops"] = {"value": fp64_tflops, "source": "cuBLAS DGEMM 4096^3 in this run"}
    if not args.no_shapes and wl.shape == "simplex":
        for key, shape_wl in (("parallelogram", "parallelogram256_k4"), ("curved", "curved256_k4"),
                              ("parallelepiped", "parallelepiped32_k3")):
            line[key] = measure_shape(torch, dgconv, shape_wl, rank, world, flush, stream, fp64_tflops=fp64_tflops)
    configs = {}
    for name in config_names:
        configs[name] = measure_config(torch, dgconv, name, rank, world, flush, stream, fp64_tflops)
    # clocks sampled from before the first timed step to the end of the GPU measurements
    line["clocks"] = clocks.stop()
    if oracle is not None:
        oracle.join()
        orc = oracle.results.get(WORKLOAD)
        if orc is None or "error" in orc:
            line["max_rel_err_vs_oracle"] = {"error": None if orc is None else orc["error"]}
        else:
            # the configured RK sequence from the GPU's own I u^n with the oracle's substep
            errs = {}
            ns_o = ORACLE_SUBSTEPS[WORKLOAD]
            for prec in ("fp64", "fp32", "tf32x3", "bf16x3"):
                if prec in TC_PRECS and not tc_covers(wl, prec):
                    continue
                x = mesh.transfer(u_n)
                mesh.rk_substeps(wind, x, orc["ds"], ns_o, 3, prec)
                got = x.cpu().numpy()
                errs[prec] = float(np.abs(got - orc["v"]).max() / np.abs(orc["v"]).max())
            errs["oracle"] = {"what": f"the oracle's {ns_o}-substep SSP-RK3 run of the full mesh from its own "
                                      f"I u^n (substep {orc['ds']:.6g}), {orc['cores']} processes",
                              "oracle_s": orc["job_s"]}
            line["max_rel_err_vs_oracle"] = errs
            units_stage = wl.n_elem * N * wl.dim
            line["cpu_baseline"] = {
                "value": units_stage / statistics.mean(orc["stage_s"]), "unit": "DOF-stage updates/s",
                "cores": orc["cores"], "kind": "oracle",
                "sample": f"the FP64 numpy oracle's {len(orc['stage_s'])} SSP-RK3 stages of the full "
                          f"{wl.n_elem}-element mesh (the reference run of max_rel_err_vs_oracle), {orc['cores']} "
                          f"processes on element blocks, one BLAS thread each, a barrier per stage; value = DOF "
                          f"updates per stage over the mean stage time ({sum(orc['stage_s']):.1f} s of stages); "
                          f"one_core_value: one block of E / cores elements timed alone"}
            if not args.no_cpu_baseline:
                line["cpu_baseline"]["one_core_value"] = OracleTimer(wl).one_core_rate()
    for name, cfg in configs.items():
        config_errors(torch, cfg, None if oracle is None else oracle.results.get(name))
    if configs:
        line["configs"] = configs
    if rank == 0 and world == 1 and not args.no_cpu_baseline and "cpu_baseline" not in line \
            and wl.shape != "curved":
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
