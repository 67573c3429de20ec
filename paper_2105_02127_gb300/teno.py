"""Thin ctypes binding of libteno.so (C ABI in include/teno.h).

Argument marshalling only: every step of the residual, the RK3 update and the
adjoint runs in the CUDA library.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA; CUDA tensors are passed as device pointers and use the
current torch stream).  There is no fallback: if the library is missing or
was not built, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TENO_OK, TENO_EINVAL, TENO_ENOMEM, TENO_ECUDA = 0, -1, -2, -3
TENO_EMESH, TENO_ESTENCIL, TENO_ENONPHYS, TENO_ETIMEOUT, TENO_ESTATE = -4, -5, -6, -7, -8
FLUX_UPWIND, FLUX_HLL, FLUX_HLLC = 0, 1, 2
FP64, FP32_MIXED, FP64_NATIVE = 0, 1, 2
SEL_LARGE = 8
DEBUG_FORCE_FALLBACK, DEBUG_ZERO_POLL_WAITS = 1, 2

_NAMES = {0: "TENO_OK", -1: "TENO_EINVAL", -2: "TENO_ENOMEM", -3: "TENO_ECUDA", -4: "TENO_EMESH",
          -5: "TENO_ESTENCIL", -6: "TENO_ENONPHYS", -7: "TENO_ETIMEOUT", -8: "TENO_ESTATE"}


class TenoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class teno_params(C.Structure):
    _fields_ = [("order", C.c_int32), ("n_var", C.c_int32), ("flux", C.c_int32),
                ("precision", C.c_int32), ("linear", C.c_int32), ("nq", C.c_int32),
                ("recon_variant", C.c_int32),
                ("ct", C.c_double), ("eps", C.c_double), ("gamma", C.c_double),
                ("adv_x", C.c_double), ("adv_y", C.c_double), ("cfl", C.c_double),
                ("adv_field", C.c_int32), ("adv_cx", C.c_double), ("adv_cy", C.c_double),
                ("adv_omega", C.c_double), ("adv_r1", C.c_double), ("adv_r2", C.c_double),
                ("scheme", C.c_int32), ("cweno_dk", C.c_double), ("charvar", C.c_int32),
                ("positivity", C.c_int32), ("debug", C.c_int32)]


_lib = None
_vp = C.c_void_p


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libteno.so; raises if it is not built (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libteno.so not built at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    sig = {
        "teno_default_params": (None, [_vp]),
        "teno_create": (C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
        "teno_destroy": (C.c_int, [_vp]),
        "teno_last_error": (C.c_char_p, [_vp]),
        "teno_set_stream": (C.c_int, [_vp, _vp]),
        "teno_mesh_load": (C.c_int, [_vp, C.c_int64, _vp, C.c_int64, _vp, C.c_int64, _vp, _vp]),
        "teno_get_permutation": (C.c_int, [_vp, _vp]),
        "teno_precompute_stencils": (C.c_int, [_vp, _vp]),
        "teno_get_stencils": (C.c_int, [_vp, _vp, _vp]),
        "teno_get_sizes": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "teno_set_state": (C.c_int, [_vp, _vp, C.c_int]),
        "teno_get_state": (C.c_int, [_vp, _vp, C.c_int]),
        "teno_set_time": (C.c_int, [_vp, C.c_double]),
        "teno_residual": (C.c_int, [_vp, _vp, _vp, C.c_int]),
        "teno_set_selection_override": (C.c_int, [_vp, _vp, C.c_int]),
        "teno_cfl_dt": (C.c_int, [_vp, _vp]),
        "teno_rk3_step": (C.c_int, [_vp, C.c_double, _vp]),
        "teno_rk3_steps": (C.c_int, [_vp, C.c_int32, C.c_double]),
        "teno_get_stage_state": (C.c_int, [_vp, C.c_int32, _vp, C.c_int]),
        "teno_check_state": (C.c_int, [_vp]),
        "teno_residual_vjp": (C.c_int, [_vp, _vp, _vp, C.c_int]),
        "teno_adjoint_step": (C.c_int, [_vp, C.c_double, _vp, _vp, C.c_int]),
        "teno_edge_values": (C.c_int, [_vp, _vp]),
        "teno_cfl_dt_noalloc": (C.c_int, [C.c_int, _vp, C.c_int32, C.c_int64, _vp, _vp,
                                          C.c_double, C.c_double, C.c_double, C.c_double, _vp,
                                          C.c_int]),
        "teno_colour_slots": (C.c_int, [C.c_int32, C.c_int32, _vp, _vp]),
        "teno_fma_peak": (C.c_int, [C.c_int, _vp, C.c_int, _vp]),
        "teno_precompute_partition": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32]),
        "teno_tape_reserve": (C.c_int, [_vp, C.c_int32]),
        "teno_rk3_step_record": (C.c_int, [_vp, C.c_int32, C.c_double]),
        "teno_adjoint_step_tape": (C.c_int, [_vp, C.c_int32, _vp, _vp, C.c_int]),
        "teno_partition_sizes": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "teno_partition_cells": (C.c_int, [_vp, _vp]),
        "teno_partition_recv_cells": (C.c_int, [_vp, C.c_int32, _vp]),
        "teno_partition_set_send": (C.c_int, [_vp, C.c_int32, C.c_int64, _vp]),
        "teno_halo_pack": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp]),
        "teno_halo_unpack": (C.c_int, [_vp, C.c_int32, C.c_int32, _vp]),
        "teno_rk3_stage": (C.c_int, [_vp, C.c_int32, C.c_double]),
        "teno_local_max_speed": (C.c_int, [_vp, _vp]),
        "teno_group_rk3_step": (C.c_int, [_vp, C.c_int32, C.c_double, _vp]),
        "teno_group_residual_vjp": (C.c_int, [_vp, C.c_int32, _vp, _vp]),
        "teno_profile": (C.c_int, [_vp, C.c_int]),
        "teno_profile_read": (C.c_int, [_vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
        return None
    return getattr(stream, "cuda_stream", stream)


NOALLOC_MAX_CELLS = 8388608


def cfl_dt_noalloc(U, cell_len, dt_out=None, gamma: float = 1.4, adv=(1.0, 1.0),
                   cfl: float = 0.4, device: int = 0, stream=None) -> float | None:
    """CFL step through teno_cfl_dt_noalloc, which allocates no device memory.
    U: CUDA tensor [n_var][n_cell]; cell_len: CUDA tensor [n_cell] (4|V|/perimeter);
    dt_out: None (the host value is returned) or a CUDA float64 tensor of one element."""
    n_var, n_cell = int(U.shape[0]), int(U.shape[1])
    up, udev = _ptr(U)
    lp, ldev = _ptr(cell_len)
    if not (udev and ldev):
        raise ValueError("U and cell_len must be device tensors")
    if dt_out is None:
        out = C.c_double()
        rc = lib().teno_cfl_dt_noalloc(device, _stream_handle(stream), n_var, n_cell, up, lp,
                                       gamma, adv[0], adv[1], cfl, C.addressof(out), 0)
        if rc != 0:
            raise TenoError(rc, "teno_cfl_dt_noalloc failed")
        return out.value
    op, odev = _ptr(dt_out)
    if not odev:
        raise ValueError("dt_out must be a device tensor")
    rc = lib().teno_cfl_dt_noalloc(device, _stream_handle(stream), n_var, n_cell, up, lp, gamma,
                                   adv[0], adv[1], cfl, op, 1)
    if rc != 0:
        raise TenoError(rc, "teno_cfl_dt_noalloc failed")
    return None


def fma_peak(precision: int = 1, device: int = 0, stream=None) -> float:
    """Measured FMA rate (flop/s) on every SM: precision 0 FP32, 1 FP64."""
    out = C.c_double()
    rc = lib().teno_fma_peak(device, _stream_handle(stream), int(precision), C.addressof(out))
    if rc != 0:
        raise TenoError(rc, "teno_fma_peak failed")
    return out.value


def colour_slots(members):
    """teno_colour_slots: slot of every stencil member so that no cell sits
    in the same slot of two lanes.  members: int array [n_lanes][n_slots]
    (distinct within a row).  Returns the int32 array of slots, or None when
    some cell is a member of more than n_slots lanes."""
    m = np.ascontiguousarray(members, dtype=np.int32)
    if m.ndim != 2:
        raise ValueError("members must be [n_lanes][n_slots]")
    out = np.empty_like(m)
    rc = lib().teno_colour_slots(m.shape[0], m.shape[1], m.ctypes.data, out.ctypes.data)
    if rc < 0:
        raise TenoError(rc, "teno_colour_slots: invalid members")
    return out if rc == 1 else None


SCHEME_TENO, SCHEME_CWENO = 0, 1


def default_params(**kw) -> teno_params:
    """Library defaults overridden by keyword: teno_params fields, plus
    adv=(ax, ay), rotation=(x_c, y_c, omega[, r1, r2]) and scheme='teno' |
    'cweno' (CWENO takes eps = 1e-14, the paper's value, unless eps is given)."""
    p = teno_params()
    lib().teno_default_params(C.byref(p))
    if isinstance(kw.get("scheme"), str):
        name = kw.pop("scheme")
        if name not in ("teno", "cweno"):
            raise ValueError("scheme must be 'teno' or 'cweno'")
        p.scheme = SCHEME_CWENO if name == "cweno" else SCHEME_TENO
        if p.scheme == SCHEME_CWENO and "eps" not in kw:
            p.eps = 1e-14
    for k, v in kw.items():
        if k == "adv":
            p.adv_x, p.adv_y = float(v[0]), float(v[1])
        elif k == "rotation":  # (x_c, y_c, omega[, r1, r2]): rigid rotation, n_var = 1
            if v is None:
                p.adv_field = 0
            else:
                p.adv_field = 1
                p.adv_cx, p.adv_cy, p.adv_omega = float(v[0]), float(v[1]), float(v[2])
                p.adv_r1, p.adv_r2 = (float(v[3]), float(v[4])) if len(v) > 3 else (0.0, 0.0)
        else:
            setattr(p, k, v)
    return p


class Teno:
    """One library context: a mesh, a scheme and a state on one GPU.

    device=-1 creates a host-only context (mesh and stencil preprocessing)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = _vp()
        self.device = device
        rc = lib().teno_create(C.byref(self._h), device,
                               _stream_handle(stream) if device >= 0 else None)
        if rc != 0:
            raise TenoError(rc, "teno_create failed")
        self.n_cell = 0
        self.n_var = 0

    def close(self):
        if self._h:
            lib().teno_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc: int):
        if rc != 0:
            raise TenoError(rc, lib().teno_last_error(self._h).decode())

    def set_stream(self, stream):
        self._chk(lib().teno_set_stream(self._h, _stream_handle(stream)))

    # -- mesh and precompute
    def mesh_load(self, xy, tri, bface=None, period=None):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        nb = 0
        bp = None
        if bface is not None and len(bface):
            bface = np.ascontiguousarray(bface, dtype=np.int32)
            nb, bp = bface.shape[0], bface.ctypes.data
        per = None if period is None else np.ascontiguousarray(period, dtype=np.float64)
        self._chk(lib().teno_mesh_load(self._h, xy.shape[0], xy.ctypes.data, tri.shape[0],
                                       tri.ctypes.data, nb, bp,
                                       None if per is None else per.ctypes.data))
        self.n_cell = tri.shape[0]
        return self

    def load(self, mesh):
        return self.mesh_load(mesh.xy, mesh.tri, mesh.bface, mesh.period)

    def precompute_stencils(self, params: teno_params | None = None, **kw):
        p = params if params is not None else default_params(**kw)
        self._chk(lib().teno_precompute_stencils(self._h, C.byref(p)))
        self.params = p
        self.n_var = p.n_var
        n = C.c_int64()
        nv, m, ns = C.c_int32(), C.c_int32(), C.c_int32()
        self._chk(lib().teno_get_sizes(self._h, C.byref(n), C.byref(nv), C.byref(m),
                                       C.byref(ns)))
        self.m, self.ns = m.value, ns.value
        self.n_out = self.n_cell
        return self

    def precompute_partition(self, n_parts: int, part: int, params: teno_params | None = None,
                             **kw):
        """Stencils and matrices of part `part` of n_parts of the mesh (a range
        of whole tiles of the Hilbert order; see teno_precompute_partition)."""
        p = params if params is not None else default_params(**kw)
        self._chk(lib().teno_precompute_partition(self._h, C.byref(p), int(n_parts), int(part)))
        self.params = p
        self.n_var = p.n_var
        n = C.c_int64()
        nv, m, ns = C.c_int32(), C.c_int32(), C.c_int32()
        self._chk(lib().teno_get_sizes(self._h, C.byref(n), C.byref(nv), C.byref(m),
                                       C.byref(ns)))
        self.m, self.ns = m.value, ns.value
        self.n_parts, self.part = int(n_parts), int(part)
        self.n_out = self.partition_sizes()[0]  # a partition returns its owned cells
        return self

    def partition_sizes(self):
        """(n_owned, n_state, recv_counts[n_parts], send_counts[n_parts])"""
        P = getattr(self, "n_parts", 1)
        a, b = C.c_int64(), C.c_int64()
        rc_, sc_ = np.zeros(P, dtype=np.int64), np.zeros(P, dtype=np.int64)
        self._chk(lib().teno_partition_sizes(self._h, C.byref(a), C.byref(b), rc_.ctypes.data,
                                             sc_.ctypes.data))
        return a.value, b.value, rc_, sc_

    def partition_cells(self):
        """user ids of the owned cells, in the order of the owned arrays"""
        out = np.empty(self.partition_sizes()[0], dtype=np.int32)
        self._chk(lib().teno_partition_cells(self._h, out.ctypes.data))
        return out

    def partition_recv_cells(self, peer: int):
        n = int(self.partition_sizes()[2][peer])
        out = np.empty(max(n, 1), dtype=np.int32)
        self._chk(lib().teno_partition_recv_cells(self._h, int(peer), out.ctypes.data))
        return out[:n]

    def partition_set_send(self, peer: int, user_ids):
        u = np.ascontiguousarray(user_ids, dtype=np.int32)
        self._chk(lib().teno_partition_set_send(self._h, int(peer), len(u),
                                                u.ctypes.data if len(u) else None))

    def halo_pack(self, peer: int, what: int, buf):
        p, dev = _ptr(buf)
        self._chk(lib().teno_halo_pack(self._h, int(peer), int(what), p))

    def halo_unpack(self, peer: int, what: int, buf):
        p, dev = _ptr(buf)
        self._chk(lib().teno_halo_unpack(self._h, int(peer), int(what), p))

    def rk3_stage(self, stage: int, dt: float):
        self._chk(lib().teno_rk3_stage(self._h, int(stage), float(dt)))

    def local_max_speed(self) -> float:
        lam = C.c_double()
        self._chk(lib().teno_local_max_speed(self._h, C.byref(lam)))
        return lam.value

    def permutation(self):
        out = np.empty(self.n_cell, dtype=np.int32)
        self._chk(lib().teno_get_permutation(self._h, out.ctypes.data))
        return out

    def stencils(self):
        large = np.empty((self.n_cell, self.ns), dtype=np.int32)
        small = np.empty((self.n_cell, 3, 12), dtype=np.int32)
        self._chk(lib().teno_get_stencils(self._h, large.ctypes.data, small.ctypes.data))
        return large, small

    # -- state
    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
        p, dev = _ptr(U)
        self._chk(lib().teno_set_state(self._h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.n_var, getattr(self, "n_out", self.n_cell)))
        p, dev = _ptr(out)
        self._chk(lib().teno_get_state(self._h, p, dev))
        return out

    def set_time(self, t: float):
        self._chk(lib().teno_set_time(self._h, float(t)))

    # -- compute
    def residual(self, out=None, sel=None, want_sel: bool = False):
        """R [n_var][n_cell] of the current state; returns (R, sel or None)."""
        if out is None:
            n = getattr(self, "n_out", self.n_cell)
            out = np.empty((self.n_var, n))
            if want_sel and sel is None:
                sel = np.empty((self.n_var, n), dtype=np.uint8)
        p, dev = _ptr(out)
        sp, sdev = _ptr(sel)
        if sel is not None and sdev != dev:
            raise ValueError("R and sel must both be host or both be device arrays")
        self._chk(lib().teno_residual(self._h, p, sp, dev))
        return out, sel

    def set_selection_override(self, sel=None):
        if sel is None:
            self._chk(lib().teno_set_selection_override(self._h, None, 0))
            return
        if isinstance(sel, np.ndarray):
            sel = np.ascontiguousarray(sel, dtype=np.uint8)
        p, dev = _ptr(sel)
        self._chk(lib().teno_set_selection_override(self._h, p, dev))

    def cfl_dt(self) -> float:
        dt = C.c_double()
        self._chk(lib().teno_cfl_dt(self._h, C.byref(dt)))
        return dt.value

    def rk3_step(self, dt: float = 0.0, sync: bool = True) -> float | None:
        if sync:
            used = C.c_double()
            self._chk(lib().teno_rk3_step(self._h, float(dt), C.byref(used)))
            return used.value
        self._chk(lib().teno_rk3_step(self._h, float(dt), None))
        return None

    def stage_state(self, stage: int, out=None):
        """Input state of stage 1 or 2 of the last SSP-RK3 step (U^(1), U^(2))."""
        if out is None:
            out = np.empty((self.n_var, getattr(self, "n_out", self.n_cell)))
        p, dev = _ptr(out)
        self._chk(lib().teno_get_stage_state(self._h, int(stage), p, dev))
        return out

    def rk3_steps(self, n: int, dt: float = 0.0):
        self._chk(lib().teno_rk3_steps(self._h, int(n), float(dt)))

    def check_state(self):
        self._chk(lib().teno_check_state(self._h))

    def edge_values(self):
        """Gauss-point values of the last reconstruction, [n_cell][3][nq][n_var]."""
        nq = 2 if self.params.order <= 4 else 3
        out = np.empty((self.n_cell, 3, nq, self.n_var))
        self._chk(lib().teno_edge_values(self._h, out.ctypes.data))
        return out

    def profile(self, enable: bool = True):
        self._chk(lib().teno_profile(self._h, int(enable)))

    def profile_read(self):
        """(ms[8], launches[8]) per kernel kind: recon, face flux, gather/update,
        CFL reduction, other, flux adjoint, recon adjoint, reverse gather."""
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        self._chk(lib().teno_profile_read(self._h, ms.ctypes.data, n.ctypes.data))
        return ms, n

    def residual_vjp(self, w, out=None):
        if isinstance(w, np.ndarray):
            w = np.ascontiguousarray(w, dtype=np.float64)
        if out is None:
            out = np.empty((self.n_var, self.n_cell))
        wp, wdev = _ptr(w)
        op, odev = _ptr(out)
        if wdev != odev:
            raise ValueError("w and out must both be host or both be device arrays")
        self._chk(lib().teno_residual_vjp(self._h, wp, op, wdev))
        return out

    def tape_reserve(self, n_slots: int):
        """Room for n_slots recorded SSP-RK3 steps (teno_tape_reserve)."""
        self._chk(lib().teno_tape_reserve(self._h, int(n_slots)))

    def rk3_step_record(self, slot: int, dt: float):
        """One SSP-RK3 step recorded in tape slot `slot`."""
        self._chk(lib().teno_rk3_step_record(self._h, int(slot), float(dt)))

    def adjoint_step_tape(self, slot: int, lam_np1, out=None):
        """The adjoint of the step recorded in `slot` (no reconstruction)."""
        if isinstance(lam_np1, np.ndarray):
            lam_np1 = np.ascontiguousarray(lam_np1, dtype=np.float64)
        if out is None:
            out = np.empty((self.n_var, self.n_cell))
        lp, ldev = _ptr(lam_np1)
        op, odev = _ptr(out)
        if ldev != odev:
            raise ValueError("lam_np1 and out must both be host or both be device arrays")
        self._chk(lib().teno_adjoint_step_tape(self._h, int(slot), lp, op, ldev))
        return out

    def adjoint_step(self, dt: float, lam_np1, out=None):
        if isinstance(lam_np1, np.ndarray):
            lam_np1 = np.ascontiguousarray(lam_np1, dtype=np.float64)
        if out is None:
            out = np.empty((self.n_var, self.n_cell))
        lp, ldev = _ptr(lam_np1)
        op, odev = _ptr(out)
        if ldev != odev:
            raise ValueError("lam_np1 and out must both be host or both be device arrays")
        self._chk(lib().teno_adjoint_step(self._h, float(dt), lp, op, ldev))
        return out


def _group(parts):
    arr = (_vp * len(parts))(*[p._h for p in parts])
    return arr


def group_rk3_step(parts, dt: float = 0.0) -> float:
    """One SSP-RK3 step of all parts of a partitioned mesh in this process
    (teno_group_rk3_step); returns the step."""
    used = C.c_double()
    rc = lib().teno_group_rk3_step(_group(parts), len(parts), float(dt), C.byref(used))
    if rc != 0:
        raise TenoError(rc, lib().teno_last_error(parts[0]._h).decode())
    return used.value


def group_residual_vjp(parts, w):
    """v = (dR/dU)^T w over all parts (host [n_var][n_cell] arrays, user order)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    v = np.zeros_like(w)
    rc = lib().teno_group_residual_vjp(_group(parts), len(parts), w.ctypes.data, v.ctypes.data)
    if rc != 0:
        raise TenoError(rc, lib().teno_last_error(parts[0]._h).decode())
    return v
