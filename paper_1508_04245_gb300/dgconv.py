"""Python binding of libdgconv (ctypes; argument marshalling only).

Every computation runs in the CUDA library.  Tensors are torch CUDA tensors
of dtype float64 (contiguous); streams default to torch's current stream.
If the shared library is missing this module raises at first use: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DGC_LIBRARY=checked selects the test build whose kernels bounds-check every gather
LIB_PATH = os.path.join(_HERE, "libdgconv_checked.so" if os.environ.get("DGC_LIBRARY") == "checked"
                        else "libdgconv.so")

DGC_FP64, DGC_FP32, DGC_BF16X3, DGC_TF32X3 = 0, 1, 2, 3
DGC_SSPRK2, DGC_SSPRK3 = 2, 3
PREC = {"fp64": DGC_FP64, "fp32": DGC_FP32, "bf16x3": DGC_BF16X3, "tf32x3": DGC_TF32X3}

# symbol name -> (restype, argtypes); mirrors include/dgconv.h
_vp, _dp, _i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "dgc_mesh_upload": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                        ctypes.POINTER(ctypes.c_void_p)],
    "dgc_mesh_upload_quad": [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                             ctypes.POINTER(ctypes.c_void_p)],
    "dgc_mesh_upload_curved": [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp,
                               ctypes.POINTER(ctypes.c_void_p)],
    "dgc_mesh_upload_hex": [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                            ctypes.POINTER(ctypes.c_void_p)],
    "dgc_mesh_free": [_vp],
    "dgc_sizes": [_vp, _i64p, _i64p],
    "dgc_mesh_info": [_vp, _i64p],
    "dgc_geometry": [_vp, _vp],
    "dgc_transfer": [_vp, _vp, _vp, _vp],
    "dgc_transfer_T": [_vp, _vp, _vp, _vp],
    "dgc_transfer_T_noalloc": [_vp, _vp, _vp, _vp],
    "dgc_mass_apply": [_vp, _vp, _vp, ctypes.c_int, _vp],
    "dgc_diagnostics": [_vp, _vp, _vp, _vp],
    "dgc_conv_apply": [_vp, _vp, _vp, _vp, ctypes.c_int, _vp],
    "dgc_rk_substeps": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "dgc_richardson": [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                       ctypes.c_int, _vp, _vp, _vp],
    "dgc_oifs_rhs": [_vp, _vp, _vp, _vp, ctypes.c_double, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                     ctypes.c_int, _vp],
    "dgc_conv_apply_hdiv": [_vp, _vp, _vp, _vp, ctypes.c_int, _vp],
    "dgc_wind_extrapolate": [_vp, ctypes.c_int, _vp, _vp, _vp, _vp],
    "dgc_autotune": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp],
    "dgc_state_save": [_vp, _vp, ctypes.c_double, ctypes.c_int64, _vp, _i64p, _vp],
    "dgc_state_load": [_vp, _vp, ctypes.c_int64, _vp, _dp, _i64p, _vp],
    "dgc_batch_rk_substeps": [ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp],
    "dgc_point_coords": [_vp, ctypes.c_int, _vp, _i64p],
    "dgc_wind_from_potential": [_vp, _vp, _vp, _vp],
    "dgc_project": [_vp, _vp, _vp, _vp],
    "dgc_hdiv_interpolate": [_vp, _vp, _vp, _vp],
    "dgc_max_wind_speed": [_vp, _vp, _dp, _vp],
    "dgc_min_edge": [_vp, _dp],
    "dgc_check": [_vp, _vp],
    "dgc_table": [ctypes.c_int, ctypes.c_int, ctypes.c_char_p, _vp, _i64p],
    "dgc_connectivity": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                         ctypes.POINTER(ctypes.c_int32)],
    "dgc_quad_table": [ctypes.c_int, ctypes.c_char_p, _vp, _i64p],
    "dgc_quad_connectivity": [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int32)],
    "dgc_hex_table": [ctypes.c_int, ctypes.c_char_p, _vp, _i64p],
    "dgc_hex_connectivity": [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int32)],
    "dgc_last_error": [ctypes.c_char_p, ctypes.c_int],
}

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(the dgconv path has no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        _lib = handle
    return _lib


class DgcError(RuntimeError):
    pass


def last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib().dgc_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(rc: int):
    if rc != 0:
        raise DgcError(f"dgconv status {rc}: {last_error()}")


def _ptr(t, n=None, name="tensor"):
    """Device pointer of a contiguous float64 CUDA tensor (length check)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Mesh:
    """A dgc_mesh handle, order k, device geometry: affine simplices (``shape="simplex"``,
    elems [E][dim+1]), parallelograms (``shape="quad"``, dim 2, elems [E][4] in cyclic order),
    parallelepipeds (``shape="hex"``, dim 3, elems [E][8] in the reference-cube order) or
    quadratic triangles (``shape="curved"``, dim 2, plus ``edge_nodes`` [n_facets][2])."""

    def __init__(self, dim: int, k: int, verts, elems, stream=None, shape: str = "simplex", edge_nodes=None):
        verts = np.ascontiguousarray(verts, dtype=np.float64)
        elems = np.ascontiguousarray(elems, dtype=np.int32)
        h = ctypes.c_void_p()
        self.shape = shape
        if shape == "quad":
            if dim != 2:
                raise ValueError("parallelogram meshes are two-dimensional")
            check(lib().dgc_mesh_upload_quad(k, verts.shape[0], verts.ctypes.data_as(ctypes.c_void_p),
                                             elems.shape[0], elems.ctypes.data_as(ctypes.c_void_p),
                                             _stream(stream), ctypes.byref(h)))
        elif shape == "hex":
            if dim != 3:
                raise ValueError("parallelepiped meshes are three-dimensional")
            check(lib().dgc_mesh_upload_hex(k, verts.shape[0], verts.ctypes.data_as(ctypes.c_void_p),
                                            elems.shape[0], elems.ctypes.data_as(ctypes.c_void_p),
                                            _stream(stream), ctypes.byref(h)))
        elif shape == "curved":
            if dim != 2 or edge_nodes is None:
                raise ValueError("curved meshes are two-dimensional and need edge_nodes [n_facets, 2]")
            en = np.ascontiguousarray(edge_nodes, dtype=np.float64)
            check(lib().dgc_mesh_upload_curved(k, verts.shape[0], verts.ctypes.data_as(ctypes.c_void_p),
                                               elems.shape[0], elems.ctypes.data_as(ctypes.c_void_p),
                                               en.ctypes.data_as(ctypes.c_void_p), _stream(stream),
                                               ctypes.byref(h)))
        elif shape == "simplex":
            check(lib().dgc_mesh_upload(dim, k, verts.shape[0], verts.ctypes.data_as(ctypes.c_void_p),
                                        elems.shape[0], elems.ctypes.data_as(ctypes.c_void_p), _stream(stream),
                                        ctypes.byref(h)))
        else:
            raise ValueError(f"unknown element shape {shape!r}")
        self._h = h
        info = (ctypes.c_int64 * 13)()
        check(lib().dgc_mesh_info(self._h, info))
        (self.dim, self.k, self.n_elem, self.n_facets, self.N, self.NW, self.n_fm, self.n_int,
         self.n_lagrange, self.n_proj, self.n_dofpts, _shape, self.n_curved) = [int(x) for x in info]
        a, b = ctypes.c_int64(), ctypes.c_int64()
        check(lib().dgc_sizes(self._h, ctypes.byref(a), ctypes.byref(b)))
        self.n_dg, self.n_hdiv = a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dgc_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- tensors -----------------------------------------------------------
    def dg_zeros(self):
        import torch
        return torch.zeros(self.n_elem, self.dim, self.N, dtype=torch.float64, device="cuda")

    def hdiv_zeros(self):
        import torch
        return torch.zeros(self.n_hdiv, dtype=torch.float64, device="cuda")

    # ---- operators ---------------------------------------------------------
    def geometry(self, stream=None):
        check(lib().dgc_geometry(self._h, _stream(stream)))

    def transfer(self, u_hdiv, out=None, stream=None):
        out = self.dg_zeros() if out is None else out
        check(lib().dgc_transfer(self._h, _ptr(u_hdiv, self.n_hdiv, "u_hdiv"), _ptr(out, self.n_dg, "out"),
                                 _stream(stream)))
        return out

    def transfer_T(self, f_dg, out=None, stream=None):
        out = self.hdiv_zeros() if out is None else out
        check(lib().dgc_transfer_T(self._h, _ptr(f_dg, self.n_dg, "f_dg"), _ptr(out, self.n_hdiv, "out"),
                                   _stream(stream)))
        return out

    def mass(self, v_dg, out=None, inverse=False, stream=None):
        out = self.dg_zeros() if out is None else out
        check(lib().dgc_mass_apply(self._h, _ptr(v_dg, self.n_dg, "v_dg"), _ptr(out, self.n_dg, "out"),
                                   int(inverse), _stream(stream)))
        return out

    def diagnostics(self, v_dg, out=None, stream=None):
        """[mass per component..., energy, non-finite count] of v_dg (device, float64)."""
        import torch
        out = torch.empty(self.dim + 2, dtype=torch.float64, device="cuda") if out is None else out
        check(lib().dgc_diagnostics(self._h, _ptr(v_dg, self.n_dg, "v_dg"), _ptr(out, self.dim + 2, "out"),
                                    _stream(stream)))
        return out

    def conv_apply(self, wind, w_dg, out=None, prec="fp64", stream=None):
        out = self.dg_zeros() if out is None else out
        check(lib().dgc_conv_apply(self._h, _ptr(wind, self.n_hdiv, "wind"), _ptr(w_dg, self.n_dg, "w_dg"),
                                   _ptr(out, self.n_dg, "out"), PREC[prec], _stream(stream)))
        return out

    def rk_substeps(self, wind, v_dg, ds: float, nsteps: int, scheme: int = 3, prec="fp64", stream=None):
        check(lib().dgc_rk_substeps(self._h, _ptr(wind, self.n_hdiv, "wind"), _ptr(v_dg, self.n_dg, "v_dg"),
                                    float(ds), int(nsteps), int(scheme), PREC[prec], _stream(stream)))
        return v_dg

    def richardson(self, wind, g_dg, v_dg, tau: float, ds: float, reduction: float, max_iter: int, prec="fp64",
                   iters=None, res=None, stream=None):
        """Pseudo-time solve of v + tau (M^V)^-1 C^V v = g in place on v_dg (see dgc_richardson).

        Returns the device tensors (iters int32[1], res float64[max_iter + 1]); read
        them after the stream has reached the end of the call."""
        import torch
        if iters is None:
            iters = torch.zeros(1, dtype=torch.int32, device=v_dg.device)
        if res is None:
            res = torch.zeros(max_iter + 1, dtype=torch.float64, device=v_dg.device)
        if iters.dtype != torch.int32 or not iters.is_cuda or iters.numel() < 1:
            raise TypeError("iters must be an int32 CUDA tensor with at least one entry")
        check(lib().dgc_richardson(self._h, _ptr(wind, self.n_hdiv, "wind"), _ptr(g_dg, self.n_dg, "g_dg"),
                                   _ptr(v_dg, self.n_dg, "v_dg"), float(tau), float(ds), float(reduction),
                                   int(max_iter), PREC[prec], ctypes.c_void_p(iters.data_ptr()),
                                   _ptr(res, max_iter + 1, "res"), _stream(stream)))
        return iters, res

    def oifs_rhs(self, u_hdiv, wind, ds: float, nsteps: int, scheme: int = 3, prec="fp64", wind_prev=None,
                 dt_prev: float = 0.0, out=None, stream=None):
        """out = I^T M^V Q I u with a frozen or extrapolated wind (see dgc_oifs_rhs)."""
        out = self.hdiv_zeros() if out is None else out
        wp = _ptr(wind_prev, self.n_hdiv, "wind_prev") if wind_prev is not None else None
        check(lib().dgc_oifs_rhs(self._h, _ptr(u_hdiv, self.n_hdiv, "u_hdiv"), _ptr(wind, self.n_hdiv, "wind"), wp,
                                 float(dt_prev), _ptr(out, self.n_hdiv, "out"), float(ds), int(nsteps), int(scheme),
                                 PREC[prec], _stream(stream)))
        return out

    def conv_apply_hdiv(self, wind, u_hdiv, out=None, prec="fp64", stream=None):
        """out = I^T C^V(wind) I u (see dgc_conv_apply_hdiv)."""
        out = self.hdiv_zeros() if out is None else out
        check(lib().dgc_conv_apply_hdiv(self._h, _ptr(wind, self.n_hdiv, "wind"), _ptr(u_hdiv, self.n_hdiv, "u_hdiv"),
                                        _ptr(out, self.n_hdiv, "out"), PREC[prec], _stream(stream)))
        return out

    def wind_extrapolate(self, fields, coefs, out=None, stream=None):
        """out = sum_t coefs[t] fields[t] over H(div) vectors (see dgc_wind_extrapolate)."""
        out = self.hdiv_zeros() if out is None else out
        n = len(fields)
        if len(coefs) != n:
            raise ValueError("fields and coefs differ in length")
        hp = (ctypes.c_void_p * n)(*[_ptr(f, self.n_hdiv, "field").value for f in fields])
        hc = (ctypes.c_double * n)(*[float(c) for c in coefs])
        check(lib().dgc_wind_extrapolate(self._h, n, hp, hc, _ptr(out, self.n_hdiv, "out"), _stream(stream)))
        return out

    def autotune(self, wind, prec="fp64", reps: int = 5, stream=None) -> int:
        """Pick the CUDA-core stage kernel's block shape for this (dim, k, prec) (see dgc_autotune)."""
        b = ctypes.c_int()
        check(lib().dgc_autotune(self._h, _ptr(wind, self.n_hdiv, "wind"), PREC[prec], int(reps), ctypes.byref(b),
                                 _stream(stream)))
        return b.value

    def state_save(self, v_dg, t: float = 0.0, step: int = 0, stream=None) -> bytes:
        """Checkpoint blob of a DG state (see dgc_state_save)."""
        size = ctypes.c_int64()
        check(lib().dgc_state_save(self._h, _ptr(v_dg, self.n_dg, "v_dg"), float(t), int(step), None,
                                   ctypes.byref(size), _stream(stream)))
        buf = ctypes.create_string_buffer(size.value)
        check(lib().dgc_state_save(self._h, _ptr(v_dg, self.n_dg, "v_dg"), float(t), int(step), buf,
                                   ctypes.byref(size), _stream(stream)))
        return buf.raw[:size.value]

    def state_load(self, blob: bytes, out=None, stream=None):
        """Restore a DG state from a checkpoint blob; returns (v_dg, t, step)."""
        out = self.dg_zeros() if out is None else out
        t, step = ctypes.c_double(), ctypes.c_int64()
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        check(lib().dgc_state_load(self._h, buf, len(blob), _ptr(out, self.n_dg, "out"), ctypes.byref(t),
                                   ctypes.byref(step), _stream(stream)))
        return out, t.value, step.value

    def richardson_ds(self, wind, tau: float) -> float:
        """Pseudo-time step 1 / (1 + beta^2), beta = tau (2k+1) max|u| / min h_T (stable for every mode)."""
        beta = tau * (2 * self.k + 1) * self.max_wind_speed(wind) / self.min_edge()
        return 1.0 / (1.0 + beta * beta)

    # ---- inputs --------------------------------------------------------------
    def point_coords(self, kind: int) -> np.ndarray:
        cnt = ctypes.c_int64()
        check(lib().dgc_point_coords(self._h, kind, None, ctypes.byref(cnt)))
        out = np.empty((cnt.value, self.dim))
        check(lib().dgc_point_coords(self._h, kind, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
        per = (self.n_lagrange, self.n_proj, self.n_dofpts)[kind]
        return out.reshape(self.n_elem, per, self.dim)

    def wind_from_potential(self, pot, out=None, stream=None):
        out = self.hdiv_zeros() if out is None else out
        n = self.n_elem * self.n_lagrange * (1 if self.dim == 2 else 3)
        check(lib().dgc_wind_from_potential(self._h, _ptr(pot, n, "pot"), _ptr(out, self.n_hdiv, "out"),
                                            _stream(stream)))
        return out

    def hdiv_interpolate(self, vals, out=None, stream=None):
        out = self.hdiv_zeros() if out is None else out
        check(lib().dgc_hdiv_interpolate(self._h, _ptr(vals, self.n_elem * self.n_dofpts * self.dim, "vals"),
                                         _ptr(out, self.n_hdiv, "out"), _stream(stream)))
        return out

    def project(self, vals, out=None, stream=None):
        out = self.dg_zeros() if out is None else out
        check(lib().dgc_project(self._h, _ptr(vals, self.n_elem * self.n_proj * self.dim, "vals"),
                                _ptr(out, self.n_dg, "out"), _stream(stream)))
        return out

    def max_wind_speed(self, wind, stream=None) -> float:
        v = ctypes.c_double()
        check(lib().dgc_max_wind_speed(self._h, _ptr(wind, self.n_hdiv, "wind"), ctypes.byref(v), _stream(stream)))
        return v.value

    def check(self, stream=None):
        """Raise if a bounded device-side wait gave up since the last check (synchronizes)."""
        check(lib().dgc_check(self._h, _stream(stream)))

    def min_edge(self) -> float:
        v = ctypes.c_double()
        check(lib().dgc_min_edge(self._h, ctypes.byref(v)))
        return v.value

    def cfl_ds(self, wind, cfl: float) -> float:
        """Substep size cfl * min h_T / ((2k+1) max |u|)  (CFL rule; the paper gives none)."""
        return cfl * self.min_edge() / ((2 * self.k + 1) * self.max_wind_speed(wind))


def batch_rk_substeps(meshes, winds, states, ds, nsteps, scheme: int = 3, prec="tf32x3", stream=None):
    """Advance many independent instances in one graph launch (see dgc_batch_rk_substeps)."""
    n = len(meshes)
    if not (len(winds) == len(states) == len(ds) == len(nsteps) == n):
        raise ValueError("batch arrays differ in length")
    hm = (ctypes.c_void_p * n)(*[m._h.value for m in meshes])
    hw = (ctypes.c_void_p * n)(*[_ptr(w, m.n_hdiv, "wind").value for m, w in zip(meshes, winds)])
    hs = (ctypes.c_void_p * n)(*[_ptr(v, m.n_dg, "state").value for m, v in zip(meshes, states)])
    hd = (ctypes.c_double * n)(*[float(x) for x in ds])
    hn = (ctypes.c_int * n)(*[int(x) for x in nsteps])
    check(lib().dgc_batch_rk_substeps(n, hm, hw, hs, hd, hn, int(scheme), PREC[prec], _stream(stream)))
    return states


def table(dim: int, k: int, name: str) -> np.ndarray:
    """A reference table of the library (host only, no GPU needed)."""
    cnt = ctypes.c_int64()
    check(lib().dgc_table(dim, k, name.encode(), None, ctypes.byref(cnt)))
    out = np.empty(cnt.value)
    check(lib().dgc_table(dim, k, name.encode(), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    return out


def connectivity(dim: int, n_vert: int, elems):
    """(facet_id, nbr, orient, n_facets) exactly as the mesh upload builds them (host only)."""
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    E = elems.shape[0]
    fid = np.empty((E, dim + 1), np.int32)
    nbr = np.empty((E, dim + 1), np.int32)
    ori = np.empty((E, dim + 1), np.int8)
    nf = ctypes.c_int32()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)      # noqa: E731
    check(lib().dgc_connectivity(dim, n_vert, E, vp(elems), vp(fid), vp(nbr), vp(ori), ctypes.byref(nf)))
    return fid, nbr, ori, nf.value


def quad_table(k: int, name: str) -> np.ndarray:
    """A reference table of the parallelogram element (host only, no GPU needed)."""
    cnt = ctypes.c_int64()
    check(lib().dgc_quad_table(k, name.encode(), None, ctypes.byref(cnt)))
    out = np.empty(cnt.value)
    check(lib().dgc_quad_table(k, name.encode(), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    return out


def quad_connectivity(n_vert: int, elems):
    """(facet_id, nbr codes, orient, flip, n_facets) as the parallelogram upload builds them (host only)."""
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    E = elems.shape[0]
    fid = np.empty((E, 4), np.int32)
    nbr = np.empty((E, 4), np.int32)
    ori = np.empty((E, 4), np.int8)
    flip = np.empty((E, 4), np.int8)
    nf = ctypes.c_int32()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)      # noqa: E731
    check(lib().dgc_quad_connectivity(n_vert, E, vp(elems), vp(fid), vp(nbr), vp(ori), vp(flip), ctypes.byref(nf)))
    return fid, nbr, ori, flip, nf.value


def hex_table(k: int, name: str) -> np.ndarray:
    """A reference table of the parallelepiped element (host only, no GPU needed)."""
    cnt = ctypes.c_int64()
    check(lib().dgc_hex_table(k, name.encode(), None, ctypes.byref(cnt)))
    out = np.empty(cnt.value)
    check(lib().dgc_hex_table(k, name.encode(), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    return out


def hex_connectivity(n_vert: int, elems):
    """(facet_id, nbr codes, orient, fcode, n_faces) as the parallelepiped upload builds them (host only)."""
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    E = elems.shape[0]
    fid = np.empty((E, 6), np.int32)
    nbr = np.empty((E, 6), np.int32)
    ori = np.empty((E, 6), np.int8)
    fc = np.empty((E, 6), np.int8)
    nf = ctypes.c_int32()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)      # noqa: E731
    check(lib().dgc_hex_connectivity(n_vert, E, vp(elems), vp(fid), vp(nbr), vp(ori), vp(fc), ctypes.byref(nf)))
    return fid, nbr, ori, fc, nf.value


def potential_values(mesh: Mesh, potential) -> np.ndarray:
    """Evaluate a workload potential at the mesh's Lagrange nodes: [E, n_lag] or [E, n_lag, 3]."""
    X = mesh.point_coords(0)
    if mesh.dim == 2:
        return np.ascontiguousarray(potential(X[..., 0], X[..., 1]))
    A = potential(X[..., 0], X[..., 1], X[..., 2])        # [3, E, n_lag]
    return np.ascontiguousarray(np.moveaxis(A, 0, -1))
