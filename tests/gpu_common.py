"""Shared setup of the GPU parity tests: seeded meshes, winds and states, and
the oracle's side of every comparison (the oracle never sees CUDA output)."""
from __future__ import annotations

import numpy as np

from oracle import dg as ODG
from oracle import hdiv as OH
from oracle import mesh as OM
from paper_1508_04245_gb300 import workloads as W

TOL = {"fp64": 1e-12, "fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-6}
TC_PRECS = ("tf32x3", "bf16x3")


def tol_hdiv_chain(dim, k, prec):
    """Tolerance of outputs that pass through I and I^T (reading A26): in FP64
    max(1e-12, 16 eps ||Cb||_inf), Cb the BDM_k dual-basis coefficients (each
    transfer rounds at about eps ||Cb||_inf; two transfers, two independent
    evaluations, slack 4 for the sum lengths); the mixed paths keep TOL."""
    if prec != "fp64":
        return TOL[prec]
    from oracle import basis as B
    cb = np.abs(np.asarray(B.bdm_element(dim, k), dtype=np.float64)).sum(axis=0).max()
    return max(1e-12, 16 * np.finfo(np.float64).eps / 2 * cb)


def tc_ok(dim, k, prec="bf16x3"):
    """The tensor-core paths cover affine triangles with k <= 6 in tf32x3 and
    bf16x3, and tetrahedra with k <= 4 in bf16x3."""
    return k <= 6 if dim == 2 else (k <= 4 and prec == "bf16x3")


def maxrel(got, ref) -> float:
    """Max-norm relative error over the whole vector (reading A17)."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def make_case(dim, k, n, jitter=0.1, seed=1, potential=None):
    verts, elems = W.square_mesh(n, jitter, seed) if dim == 2 else W.cube_mesh(n, jitter, seed)
    if potential is None:
        potential = W.stream_random(seed + 7) if dim == 2 else W.potential_random(seed + 7)
    omesh = OM.Mesh(verts, elems)
    wind = OH.wind_from_potential(omesh, k, potential)
    return verts, elems, potential, omesh, wind


def oracle_state(omesh, k, seed=3):
    return W.uniform_coeffs(seed, omesh.n_elem, omesh.dim, k)


def oracle_ds(omesh, k, wind, cfl=0.2):
    return ODG.cfl_ds(omesh, k, wind, cfl)
