"""ctypes front end of the C oracle (teno_oracle.c).

Test infrastructure: only the tests, the package smoke check and the
benchmark's CPU-baseline leg may use it.  Marshalling only; all arithmetic is
in teno_oracle.c.  Arrays are SoA [n_var][n_cell] in user cell order.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

FLUX_UPWIND, FLUX_HLL, FLUX_HLLC = 0, 1, 2
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def _opt(p):
    """nullable pointer argument"""
    return None if p is None else p.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        L.oracle_new.restype = C.c_void_p
        L.oracle_new.argtypes = [C.c_int64, _dp, C.c_int64, _ip, C.c_int64, C.c_void_p, C.c_void_p,
                                 _ip, _dp, C.POINTER(C.c_int32)]
        L.oracle_free.argtypes = [C.c_void_p]
        L.oracle_prepare.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        L.oracle_stencils.argtypes = [C.c_void_p, _ip, _ip]
        L.oracle_recon_matrix.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]
        L.oracle_reference_data.argtypes = [C.c_void_p, _dp, _dp, _dp, _ip, _dp, _dp]
        L.oracle_recon_cell.argtypes = [C.c_void_p, _dp, C.c_int64, _dp, _dp, _bp, _dp]
        L.oracle_residual.argtypes = [C.c_void_p, _dp, C.c_double, _dp, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
        L.oracle_residual_cells.argtypes = [C.c_void_p, _dp, C.c_double, C.c_int64, _lp, _dp,
                                            C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_cfl_dt.restype = C.c_double
        L.oracle_cfl_dt.argtypes = [C.c_void_p, _dp, C.c_double]
        L.oracle_rk3_step.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double]
        L.oracle_residual_vjp.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp, C.c_void_p]
        L.oracle_rk3_vjp.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp]
        L.oracle_flux.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                  C.c_double, _dp, C.c_void_p, C.c_void_p]
        L.oracle_geometry.argtypes = [C.c_void_p, _dp, _dp, _ip]
        L.oracle_ghost.argtypes = [C.c_void_p, C.c_int, _dp, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, _dp]
        L.oracle_face_flux.argtypes = [C.c_void_p, _dp, C.c_double, C.c_int64, C.c_int, _dp]
        L.oracle_char_basis.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp]
        L.oracle_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
    return _lib


def default_nq(order: int) -> int:
    return 2 if order <= 4 else 3


def n_unknowns(order: int) -> int:
    r = order - 1
    return (r + 1) * (r + 2) // 2 - 1


class OracleError(RuntimeError):
    pass


class Oracle:
    """One mesh + scheme configuration of the CPU oracle."""

    def __init__(self, mesh, order: int = 3, n_var: int = 1, flux: int = FLUX_UPWIND,
                 linear: bool = False, ct: float = 1e-6, eps: float = 1e-12, gamma: float = 1.4,
                 adv=(1.0, 1.0), nq: int | None = None, rotation=None, scheme: str = "teno",
                 cweno_dk: float = 1e4, charvar: bool = False, positivity: bool = False):
        """rotation: (x_c, y_c, omega) or (x_c, y_c, omega, r1, r2) for scalar
        advection by the rigid rotation v = omega phi(r) (-(y - y_c), x - x_c)
        (the solid-body case of Sec. 5 is (0.5, 0.5, 1.0)), phi a smoothstep
        taper from 1 at r1 to 0 at r2 (none when omitted); otherwise the
        constant velocity adv.  charvar: Euler reconstruction in characteristic
        variables per face (TENO only).  positivity: Euler, scale each cell's
        reconstruction towards its average so that density and pressure stay
        positive at its face Gauss points (Zhang and Shu's scaling; not in the
        paper; the adjoint entry points refuse it)."""
        self.mesh = mesh
        self.order, self.n_var = order, n_var
        self.m = n_unknowns(order)
        self.ns = 2 * (self.m + 1)
        self.nq = default_nq(order) if nq is None else nq
        self._xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self._bf = np.ascontiguousarray(mesh.bface, dtype=np.int32)
        self._per = None if mesh.period is None else np.asarray(mesh.period, dtype=np.float64)
        rot = (0.0, 0.0, 0.0, 0.0, 0.0) if rotation is None else tuple(rotation)
        if len(rot) == 3:
            rot = rot + (0.0, 0.0)
        if scheme not in ("teno", "cweno"):
            raise ValueError("scheme must be 'teno' or 'cweno'")
        iopt = np.array([order, self.nq, n_var, flux, int(linear), int(rotation is not None),
                         int(scheme == "cweno"), int(charvar), int(positivity)], dtype=np.int32)
        dopt = np.array([ct, eps, gamma, adv[0], adv[1], rot[0], rot[1], rot[2], rot[3], rot[4],
                         cweno_dk], dtype=np.float64)
        st = C.c_int32(0)
        self._h = lib().oracle_new(self._xy.shape[0], self._xy, self._tri.shape[0], self._tri,
                                   self._bf.shape[0], _opt(self._bf if len(self._bf) else None),
                                   _opt(self._per), iopt, dopt, C.byref(st))
        if st.value != 0:
            lib().oracle_free(self._h)
            self._h = None
            raise OracleError(f"oracle_new failed: {st.value}")
        self.n_cell = self._tri.shape[0]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oracle_free(self._h)
            self._h = None

    def _chk(self, rc, what):
        if rc != 0:
            raise OracleError(f"{what} failed: {rc}")

    def prepare(self, cells=None):
        if cells is None:
            self._chk(lib().oracle_prepare(self._h, 0, None), "prepare")
        else:
            c = np.ascontiguousarray(cells, dtype=np.int64)
            self._chk(lib().oracle_prepare(self._h, len(c), c.ctypes.data_as(C.c_void_p)),
                      "prepare")

    def stencils(self):
        large = np.empty((self.n_cell, self.ns), dtype=np.int32)
        small = np.empty((self.n_cell, 3, 12), dtype=np.int32)
        self._chk(lib().oracle_stencils(self._h, large, small), "stencils")
        return large, small

    def recon_matrix(self, cell: int, which: int = 0):
        n = self.ns if which == 0 else 12
        mm = self.m if which == 0 else 5
        A = np.empty((n, mm))
        Ah = np.empty((mm, n))
        vol = np.empty(n)
        ids = np.empty(n, dtype=np.int32)
        self._chk(lib().oracle_recon_matrix(self._h, cell, which, _opt(A), _opt(Ah), _opt(vol),
                                            _opt(ids)), "recon_matrix")
        return A, Ah, vol, ids

    def reference_data(self):
        m = self.m
        mean0, Br, B2 = np.empty(m), np.empty((m, m)), np.empty((5, 5))
        ex = np.empty((m, 2), dtype=np.int32)
        gt, gw = np.empty(self.nq), np.empty(self.nq)
        lib().oracle_reference_data(self._h, mean0, Br, B2, ex, gt, gw)
        return dict(mean0=mean0, Br=Br, B2=B2, ex=ex, gt=gt, gw=gw)

    def recon_cell(self, U, cell: int):
        U = np.ascontiguousarray(U, dtype=np.float64)
        coef = np.empty((self.n_var, self.m))
        beta = np.empty((self.n_var, 4))
        sel = np.empty(self.n_var, dtype=np.uint8)
        margin = np.empty(self.n_var)
        self._chk(lib().oracle_recon_cell(self._h, U, cell, coef, beta, sel, margin), "recon_cell")
        return coef, beta, sel, margin

    def residual(self, U, time: float = 0.0, sel_override=None):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.n_var, self.n_cell)
        R = np.empty_like(U)
        sel = np.empty(U.shape, dtype=np.uint8)
        margin = np.empty(U.shape)
        so = None if sel_override is None else np.ascontiguousarray(sel_override, dtype=np.uint8)
        self._chk(lib().oracle_residual(self._h, U, time, R, _opt(sel), _opt(margin), _opt(so)),
                  "residual")
        return R, sel, margin

    def residual_cells(self, U, cells, time: float = 0.0, flux_scale: bool = False):
        """(R, sel, margin) of the listed cells, [n][n_var] each; with
        flux_scale also sum_faces |K_f| / |V| per cell and variable."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        R = np.empty((len(cells), self.n_var))
        sel = np.empty((len(cells), self.n_var), dtype=np.uint8)
        margin = np.empty((len(cells), self.n_var))
        sc = np.empty((len(cells), self.n_var)) if flux_scale else None
        self._chk(lib().oracle_residual_cells(self._h, U, time, len(cells), cells, R, _opt(sel),
                                              _opt(margin), _opt(sc)), "residual_cells")
        return (R, sel, margin, sc) if flux_scale else (R, sel, margin)

    def cfl_dt(self, U, cfl: float) -> float:
        U = np.ascontiguousarray(U, dtype=np.float64)
        return float(lib().oracle_cfl_dt(self._h, U, cfl))

    def rk3_step(self, U, dt: float, time: float = 0.0):
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        self._chk(lib().oracle_rk3_step(self._h, U, time, dt), "rk3_step")
        return U

    def residual_vjp(self, U, w, time: float = 0.0, sel_override=None):
        U = np.ascontiguousarray(U, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        v = np.empty_like(w)
        so = None if sel_override is None else np.ascontiguousarray(sel_override, dtype=np.uint8)
        self._chk(lib().oracle_residual_vjp(self._h, U, time, w, v, _opt(so)), "residual_vjp")
        return v

    def rk3_vjp(self, Un, lam_np1, dt: float, time: float = 0.0):
        Un = np.ascontiguousarray(Un, dtype=np.float64)
        lam = np.ascontiguousarray(lam_np1, dtype=np.float64)
        out = np.empty_like(lam)
        self._chk(lib().oracle_rk3_vjp(self._h, Un, time, dt, lam, out), "rk3_vjp")
        return out

    def flux(self, UL, UR, nx: float, ny: float, jac: bool = False, x: float = 0.0,
             y: float = 0.0):
        """numerical flux at face point (x, y) (the point matters only for the
        rotation field of scalar advection)"""
        UL = np.ascontiguousarray(UL, dtype=np.float64)
        UR = np.ascontiguousarray(UR, dtype=np.float64)
        F = np.empty(self.n_var)
        if jac:
            JL = np.empty((self.n_var, self.n_var))
            JR = np.empty((self.n_var, self.n_var))
            lib().oracle_flux(self._h, UL, UR, nx, ny, x, y, F, _opt(JL), _opt(JR))
            return F, JL, JR
        lib().oracle_flux(self._h, UL, UR, nx, ny, x, y, F, None, None)
        return F

    def face_flux(self, U, cell: int, edge: int, time: float = 0.0):
        """K = |A| sum_k w_k F(U_L, U_R) of the face on local edge `edge` of
        `cell` (which must own the face)"""
        U = np.ascontiguousarray(U, dtype=np.float64)
        K = np.empty(self.n_var)
        self._chk(lib().oracle_face_flux(self._h, U, time, cell, edge, K), "face_flux")
        return K

    def ghost(self, tag: int, UL, nx: float, ny: float, x: float = 0.0, y: float = 0.0,
              time: float = 0.0):
        """boundary ghost state of the shock case (tag 1 wall, 2 inflow, 3
        outflow, 4 top) at face point (x, y), outward normal (nx, ny), time t"""
        UL = np.ascontiguousarray(UL, dtype=np.float64)
        UR = np.empty(self.n_var)
        lib().oracle_ghost(self._h, tag, UL, nx, ny, x, y, time, UR)
        return UR

    def char_basis(self, W, nx: float, ny: float):
        """left / right eigenvector matrices (4x4) of the Euler flux in
        direction (nx, ny) at conservative state W"""
        W = np.ascontiguousarray(W, dtype=np.float64)
        Lm, Rm = np.empty(16), np.empty(16)
        lib().oracle_char_basis(self._h, W, nx, ny, Lm, Rm)
        return Lm.reshape(4, 4), Rm.reshape(4, 4)

    def geometry(self):
        area = np.empty(self.n_cell)
        cen = np.empty((self.n_cell, 2))
        fnbr = np.empty((self.n_cell, 3), dtype=np.int32)
        lib().oracle_geometry(self._h, area, cen, fnbr)
        return area, cen, fnbr


def gauss_legendre(n: int):
    x, w = np.empty(n), np.empty(n)
    if lib().oracle_gauss_legendre(n, x, w) != 0:
        raise OracleError("gauss_legendre")
    return x, w
