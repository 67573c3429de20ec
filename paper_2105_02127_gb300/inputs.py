"""Seeded synthetic inputs: jittered triangular meshes and initial cell averages.

This module is shared by the library's tests/benchmark and by the CPU oracle's
tests.  It holds none of the finite-volume method's arithmetic: it only builds
meshes (vertex coordinates and triangle connectivity) and the initial cell
averages of analytic fields, which are the *inputs* of the method (the
semi-discrete scheme of Sec. 2.1 starts from given cell averages).

Random numbers come from a counter-based splitmix64 stream:
    z_n = mix(seed + (n + 1) * 0x9E3779B97F4A7C15),  u_n = (z_n >> 11) * 2**-53.

Meshes: an nx-by-ny quad grid, every vertex displaced by an i.i.d. uniform
offset in [-jitter*h, +jitter*h] per coordinate (periodic meshes jitter every
vertex; on non-periodic domains interior vertices move freely, boundary vertices
only tangentially and corners not at all).  Each quad is split along one of its
two diagonals, picked by a seeded coin flip.  Triangles are counter-clockwise.
Periodic meshes share vertex ids across the wrap, so the mesh is a torus; the
period (Lx, Ly) tells the consumer how to unwrap coordinates.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
GAMMA = 1.4


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """splitmix64 output for state seed + (n+1)*golden, n = counters (uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) from counters start .. start+n-1."""
    z = splitmix64(seed, np.arange(start, start + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class Mesh:
    """Triangular mesh: xy [n_vert,2] float64, tri [n_cell,3] int32 (CCW),
    bface [n_bface,3] int32 (v0, v1, tag) for non-periodic domains,
    period (Lx, Ly) or None."""

    def __init__(self, xy, tri, bface, period, nx, ny, Lx, Ly, x0=0.0, y0=0.0):
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.bface = np.ascontiguousarray(bface, dtype=np.int32)
        self.period = None if period is None else (float(period[0]), float(period[1]))
        self.nx, self.ny, self.Lx, self.Ly = nx, ny, Lx, Ly
        self.x0, self.y0 = x0, y0

    @property
    def n_cell(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.xy.shape[0])

    def unwrapped_vertices(self) -> np.ndarray:
        """[n_cell,3,2] vertex coordinates with periodic wrap undone so that
        every vertex of a triangle lies within half a period of its first
        vertex (the convention both the library and the oracle document)."""
        v = self.xy[self.tri].copy()
        if self.period is not None:
            for ax, L in enumerate(self.period):
                d = v[:, 1:, ax] - v[:, :1, ax]
                v[:, 1:, ax] -= L * np.round(d / L)
        return v


# boundary tags for non-periodic domains
BC_WALL, BC_INFLOW, BC_OUTFLOW, BC_TOP = 1, 2, 3, 4


def jittered_mesh(nx: int, ny: int, Lx: float = 1.0, Ly: float = 1.0, seed: int = 1001,
                  periodic: bool = True, jitter: float = 0.1, x0: float = 0.0,
                  y0: float = 0.0, bc_tagger=None) -> Mesh:
    """Jittered split-quad triangular mesh of an nx-by-ny quad grid on
    [x0, x0+Lx] x [y0, y0+Ly]; 2*nx*ny triangles."""
    hx, hy = Lx / nx, Ly / ny
    if periodic:
        nvx, nvy = nx, ny
    else:
        nvx, nvy = nx + 1, ny + 1
    nv = nvx * nvy
    jj, ii = np.meshgrid(np.arange(nvy), np.arange(nvx), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    u = uniform(seed, 0, 2 * nv).reshape(nv, 2)
    dx = (2.0 * u[:, 0] - 1.0) * jitter * hx
    dy = (2.0 * u[:, 1] - 1.0) * jitter * hy
    if not periodic:
        onx = (ii == 0) | (ii == nx)
        ony = (jj == 0) | (jj == ny)
        dx = np.where(onx, 0.0, dx)
        dy = np.where(ony, 0.0, dy)
    xy = np.stack([x0 + ii * hx + dx, y0 + jj * hy + dy], axis=1)

    qj, qi = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    qi = qi.ravel()
    qj = qj.ravel()
    flip = uniform(seed, 2 * nv, nx * ny) < 0.5

    def vid(i, j):
        if periodic:
            return (j % nvy) * nvx + (i % nvx)
        return j * nvx + i

    v00 = vid(qi, qj)
    v10 = vid(qi + 1, qj)
    v11 = vid(qi + 1, qj + 1)
    v01 = vid(qi, qj + 1)
    t1 = np.where(flip[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(flip[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    tri = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2

    bface = np.zeros((0, 3), dtype=np.int32)
    if not periodic:
        faces = []
        # bottom (y=y0), right (x=x0+Lx), top, left; edge direction follows the
        # counter-clockwise orientation of the interior triangle.
        for i in range(nx):
            faces.append((vid(i, 0), vid(i + 1, 0), "bottom", x0 + (i + 0.5) * hx))
            faces.append((vid(i + 1, ny), vid(i, ny), "top", x0 + (i + 0.5) * hx))
        for j in range(ny):
            faces.append((vid(nx, j), vid(nx, j + 1), "right", y0 + (j + 0.5) * hy))
            faces.append((vid(0, j + 1), vid(0, j), "left", y0 + (j + 0.5) * hy))
        rows = []
        for a, b, side, s in faces:
            tag = bc_tagger(side, s) if bc_tagger is not None else BC_OUTFLOW
            rows.append((a, b, tag))
        bface = np.asarray(rows, dtype=np.int32)
    return Mesh(xy, tri, bface, (Lx, Ly) if periodic else None, nx, ny, Lx, Ly, x0, y0)


# ---------------------------------------------------------------------------
# cell averages of analytic fields (collapsed Gauss-Legendre rule on triangles)


def _duffy_rule(n: int):
    """Points (u, v) and weights on the unit triangle {u,v>=0, u+v<=1} from an
    n x n collapsed Gauss-Legendre rule; weights sum to 1/2."""
    x, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (x + 1.0)
    ws = 0.5 * w
    a, b = np.meshgrid(s, s, indexing="ij")
    wa, wb = np.meshgrid(ws, ws, indexing="ij")
    u = a.ravel()
    v = (b * (1.0 - a)).ravel()
    wt = (wa * wb * (1.0 - a)).ravel()
    return u, v, wt


def cell_average(mesh: Mesh, func, n_quad: int = 6, n_var: int | None = None) -> np.ndarray:
    """Cell averages of func(x, y) -> array [..., n_var] (or scalar field) over
    every triangle.  Returns [n_var, n_cell] float64 (SoA, user cell order)."""
    V = mesh.unwrapped_vertices()
    u, v, wt = _duffy_rule(n_quad)
    p0 = V[:, 0, :]
    e1 = V[:, 1, :] - p0
    e2 = V[:, 2, :] - p0
    X = p0[:, None, 0] + u[None, :] * e1[:, None, 0] + v[None, :] * e2[:, None, 0]
    Y = p0[:, None, 1] + u[None, :] * e1[:, None, 1] + v[None, :] * e2[:, None, 1]
    f = np.asarray(func(X, Y), dtype=np.float64)
    if f.ndim == 2:
        f = f[None]
    avg = 2.0 * np.einsum("vcq,q->vc", f, wt)
    return np.ascontiguousarray(avg)


def prim_to_cons(rho, u, v, p, gamma: float = GAMMA):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def advection_sine(x, y):
    """u0 = sin(2 pi (x + y))."""
    return np.sin(2.0 * np.pi * (x + y))


def advection_sine_product(x, y):
    """u0 = sin(2 pi x) sin(2 pi y) (the accuracy test field of Sec. 5.1)."""
    return np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y)


def solid_bodies(x, y):
    """Initial field of the solid-body rotation case (Sec. 5, table of the
    rotation case): a cosine hump centred (0.25, 0.5), a sharp cone at
    (0.5, 0.25) and a slotted cylinder at (0.5, 0.75), each of radius 0.15.
    Readings of the garbled table: r is the distance to the body's centre
    divided by r_0 and capped at 1, so every body is zero outside its disc
    (the hump as 1/4 (1 + cos(pi r)), the cone as 1 - r); the cylinder is 1 in
    its disc except the slot |x - x_0| < 0.025, y < 0.85."""
    r0 = 0.15

    def rr(x0, y0):
        return np.minimum(np.hypot(x - x0, y - y0), r0) / r0

    hump = 0.25 * (1.0 + np.cos(np.pi * rr(0.25, 0.5)))
    cone = 1.0 - rr(0.5, 0.25)
    inside = np.hypot(x - 0.5, y - 0.75) <= r0
    cyl = np.where(inside & ((np.abs(x - 0.5) >= 0.025) | (y >= 0.85)), 1.0, 0.0)
    return hump + cone + cyl


def isentropic_vortex(x, y, t: float = 0.0, strength: float = 5.0, gamma: float = GAMMA,
                      L: float = 10.0, images: int = 1):
    """Isentropic vortex of Sec. 5.2 (centre (5,5), free stream (1,1,1,1)),
    advected to time t on the periodic [0,L]^2 square; the perturbations of the
    nearest (2*images+1)^2 periodic copies are superposed."""
    du = np.zeros_like(x)
    dv = np.zeros_like(x)
    dT = np.zeros_like(x)
    cx = (5.0 + t) % L
    cy = (5.0 + t) % L
    for ix in range(-images, images + 1):
        for iy in range(-images, images + 1):
            xr = x - cx - ix * L
            yr = y - cy - iy * L
            r2 = xr * xr + yr * yr
            f = np.exp(0.5 * (1.0 - r2))
            du += -strength / (2.0 * np.pi) * f * yr
            dv += strength / (2.0 * np.pi) * f * xr
            dT += -(gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * f * f
    T = 1.0 + dT
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return prim_to_cons(rho, 1.0 + du, 1.0 + dv, p, gamma)


def shear_layer(seed: int = 2005, gamma: float = GAMMA):
    """Periodic shear layer on [0,1]^2 (density 2 inside |y-0.5|<0.25, 1 outside,
    u = -+0.5 with tanh thickness 0.01, p = 2.5, 8-mode seeded v perturbation of
    amplitude 0.01 localised at the two layers)."""
    a = uniform(seed, 0, 8)
    a = a / a.sum()
    phi = 2.0 * np.pi * uniform(seed, 8, 8)

    def f(x, y):
        dyc = np.abs(y - 0.5)
        rho = 1.5 + 0.5 * np.tanh((0.25 - dyc) / 0.01)
        u = 0.5 * np.tanh((dyc - 0.25) / 0.01)
        env = np.exp(-((y - 0.25) / 0.05) ** 2) + np.exp(-((y - 0.75) / 0.05) ** 2)
        v = np.zeros_like(x)
        for m in range(8):
            v += a[m] * np.sin(2.0 * np.pi * (m + 1) * x + phi[m])
        v = 0.01 * v * env
        p = 2.5 * np.ones_like(x)
        return prim_to_cons(rho, u, v, p, gamma)

    return f


def dmr_state(x, y, t: float = 0.0, gamma: float = GAMMA):
    """Double-Mach-reflection initial state (Sec. 5.8): post-shock state left of
    the 60-degree shock line y = 1.732 (x - 0.1667 - 20 t / 1.732), pre-shock
    state (1.4, 0, 0, 1) right of it."""
    post = (8.0, 7.145, -4.125, 116.8333)
    pre = (1.4, 0.0, 0.0, 1.0)
    xs = 0.1667 + 20.0 * t / 1.732
    behind = y >= 1.732 * (x - xs)
    rho = np.where(behind, post[0], pre[0])
    u = np.where(behind, post[1], pre[1])
    v = np.where(behind, post[2], pre[2])
    p = np.where(behind, post[3], pre[3])
    return prim_to_cons(rho, u, v, p, gamma)


def dmr_bc_tagger(side: str, s: float) -> int:
    if side == "bottom":
        return BC_INFLOW if s < 0.1667 else BC_WALL
    if side == "left":
        return BC_INFLOW
    if side == "right":
        return BC_OUTFLOW
    return BC_TOP


def random_directions(seed: int, n_dir: int, n_val: int) -> np.ndarray:
    """n_dir seeded directions of length n_val with entries uniform in [-1,1)."""
    return (2.0 * uniform(seed, 0, n_dir * n_val) - 1.0).reshape(n_dir, n_val)


def smooth_directions(seed: int, n_dir: int, mesh: Mesh, n_var: int, n_modes: int = 4,
                      k_max: int = 2) -> np.ndarray:
    """n_dir seeded smooth directions [n_dir, n_var, n_cell]: per direction and
    variable a sum of n_modes periodic Fourier modes a sin(2 pi (kx x / Lx +
    ky y / Ly) + phi) at the cell centroids, with integer wavenumbers |kx|,
    |ky| <= k_max (not both zero), amplitudes uniform in [-1, 1) and phases
    uniform in [0, 2 pi).  Unlike cell-wise random entries they do not roughen
    a nearly uniform state at the scale of the cells."""
    c = mesh.unwrapped_vertices().mean(axis=1)
    Lx, Ly = (mesh.period if mesh.period is not None else (1.0, 1.0))
    per = n_var * n_modes
    r = uniform(seed, 0, n_dir * per * 4).reshape(n_dir, n_var, n_modes, 4)
    out = np.zeros((n_dir, n_var, c.shape[0]))
    span = 2 * k_max + 1
    for d in range(n_dir):
        for v in range(n_var):
            for m in range(n_modes):
                kx = int(r[d, v, m, 0] * span) - k_max
                ky = int(r[d, v, m, 1] * span) - k_max
                if kx == 0 and ky == 0:
                    kx = 1
                a = 2.0 * r[d, v, m, 2] - 1.0
                phi = 2.0 * np.pi * r[d, v, m, 3]
                out[d, v] += a * np.sin(2.0 * np.pi * (kx * c[:, 0] / Lx + ky * c[:, 1] / Ly) + phi)
    return out
