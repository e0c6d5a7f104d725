"""Seeded synthetic inputs for the surfactant step (shared by the tests, the
benchmark and both implementations).

This module only builds inputs: grids, VoF fractions of circles and spheres
(exact cell areas / volumes), discretely divergence-free face velocities from
stream functions or vector potentials, kinetic parameters and seeded random
fields.  It holds none of the method's arithmetic (no phase field, no
transport, no kinetics) and imports neither the CUDA library nor the oracle.

Layout conventions (shared with both implementations):
  cell arrays are float64 numpy arrays of shape (nz, ny, nx), x fastest;
  2D planar and axisymmetric grids have nz = 1 (axisymmetric: x = r with the
  axis at r = 0, y = z);
  face velocities: ux (nz, ny, nx+1), uy (nz, ny+1, nx), uz (nz+1, ny, nx).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

PLANAR, AXI, CART3D = 0, 1, 2
EOS_LANGMUIR, EOS_LINEAR, EOS_TANH = 0, 1, 2


@dataclasses.dataclass
class Grid:
    geom: int
    nx: int
    ny: int
    nz: int
    h: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    @property
    def ndim(self):
        return 3 if self.geom == CART3D else 2


@dataclasses.dataclass
class Params:
    ka: float = 1.0
    kd: float = 0.1
    gamma_inf: float = 1.0
    Df: float = 1e-2
    DF: float = 1e-2
    eps: float = 0.0
    eta: float = 1e-6
    sigma0: float = 1.0
    E: float = 0.2
    eos: int = EOS_LANGMUIR
    literal_upwind: int = 0
    bc_F: float = 1.0
    bc_f: float = 0.0


@dataclasses.dataclass
class Case:
    """One synthetic workload: grid, VoF fraction, initial state, velocity."""
    name: str
    grid: Grid
    params: Params
    C: np.ndarray
    F0: np.ndarray
    gamma0: Optional[np.ndarray]  # interfacial concentration to load as f0 = gamma0 * delta
    ux: Optional[np.ndarray] = None
    uy: Optional[np.ndarray] = None
    uz: Optional[np.ndarray] = None
    dt: float = 1e-3
    steps: int = 1
    tol: float = 1e-10
    redist_iters: int = 24
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def dtau(self):
        return redist_dtau(self.grid)


def redist_dtau(g: Grid) -> float:
    """Pseudo-time step of the redistancing iterations (a CFL-limited choice)."""
    return g.h / 3.0 if g.geom == CART3D else 0.5 * g.h


# --------------------------------------------------------------- VoF areas
def _prim_chord(x, R):
    """Antiderivative of sqrt(R^2 - x^2)."""
    x = np.clip(x, -R, R)
    return 0.5 * (x * np.sqrt(np.maximum(R * R - x * x, 0.0)) + R * R * np.arcsin(x / R))


def circle_rect_area(x0, x1, y0, y1, R):
    """Exact area of the disk of radius R centred at the origin inside the
    rectangle [x0,x1] x [y0,y1] (vectorised over the rectangle bounds).

    The overlap length in y at abscissa x is clip(min(y1, s) - max(y0, -s), 0)
    with s = sqrt(R^2 - x^2); between break points each branch integrates in
    closed form."""
    x0, x1, y0, y1 = (np.asarray(v, dtype=np.float64) for v in (x0, x1, y0, y1))
    x0, x1, y0, y1 = np.broadcast_arrays(x0, x1, y0, y1)
    out = np.zeros(x0.shape)
    flat = [a.ravel() for a in (x0, x1, y0, y1)]
    res = out.ravel()
    for n in range(res.size):
        a, b, c, d = (float(v[n]) for v in flat)
        lo, hi = max(a, -R), min(b, R)
        if hi <= lo:
            continue
        bps = {lo, hi}
        for yy in (c, d):
            if abs(yy) < R:
                xx = math.sqrt(R * R - yy * yy)
                for v in (-xx, xx):
                    if lo < v < hi:
                        bps.add(v)
        bps = sorted(bps)
        tot = 0.0
        for p, q in zip(bps[:-1], bps[1:]):
            m = 0.5 * (p + q)
            s = math.sqrt(max(R * R - m * m, 0.0))
            top_is_s = s < d       # upper limit min(d, s)
            bot_is_s = -s > c      # lower limit max(c, -s)
            top = s if top_is_s else d
            bot = -s if bot_is_s else c
            if top <= bot:
                continue
            S = float(_prim_chord(q, R) - _prim_chord(p, R))
            val = 0.0
            val += S if top_is_s else d * (q - p)
            val -= -S if bot_is_s else c * (q - p)
            tot += val
        res[n] = tot
    return out


def circle_vof(nx, ny, h, xc, yc, R, x0=0.0, y0=0.0):
    """Volume fraction of a disk (fluid 1) in each cell of a planar grid."""
    C = np.zeros((1, ny, nx))
    xs = x0 + np.arange(nx + 1) * h - xc
    ys = y0 + np.arange(ny + 1) * h - yc
    for j in range(ny):
        for i in range(nx):
            xa, xb, ya, yb = xs[i], xs[i + 1], ys[j], ys[j + 1]
            # nearest and farthest corner distances decide full / empty cells
            dx_n = 0.0 if xa <= 0 <= xb else min(abs(xa), abs(xb))
            dy_n = 0.0 if ya <= 0 <= yb else min(abs(ya), abs(yb))
            dx_f, dy_f = max(abs(xa), abs(xb)), max(abs(ya), abs(yb))
            if dx_n * dx_n + dy_n * dy_n >= R * R:
                continue
            if dx_f * dx_f + dy_f * dy_f <= R * R:
                C[0, j, i] = 1.0
                continue
            C[0, j, i] = float(circle_rect_area(xa, xb, ya, yb, R)) / (h * h)
    return np.clip(C, 0.0, 1.0)


def ring_vof(nr, nz, h, zc, R):
    """Volume fraction of a sphere of radius R centred on the axis at z = zc,
    in the ring cells [ih,(i+1)h] x [jh,(j+1)h] of an axisymmetric grid.

    The ring volume inside the sphere is pi * int (clip(R^2 - z^2, r0^2,
    r1^2) - r0^2) dz over the cell's z-range (z measured from zc); the
    integrand is piecewise constant or quadratic, so its antiderivative G is
    exact: with z1 = sqrt(R^2 - r1^2) and z0 = sqrt(R^2 - r0^2) (0 when
    negative), G(z) = r1^2 z for z <= z1, + R^2 (z - z1) - (z^3 - z1^3)/3 up to
    z0, + r0^2 (z - z0) beyond, odd in z."""
    r0 = (np.arange(nr) * h)[None, :]
    r1 = ((np.arange(nr) + 1) * h)[None, :]
    za = (np.arange(nz) * h - zc)[:, None]
    zb = ((np.arange(nz) + 1) * h - zc)[:, None]
    z1 = np.sqrt(np.maximum(R * R - r1 * r1, 0.0))
    z0 = np.sqrt(np.maximum(R * R - r0 * r0, 0.0))

    def G(z):
        a = np.abs(z)
        g = np.where(a <= z1, r1 * r1 * a,
                     np.where(a <= z0,
                              r1 * r1 * z1 + R * R * (a - z1) - (a ** 3 - z1 ** 3) / 3.0,
                              r1 * r1 * z1 + R * R * (z0 - z1) - (z0 ** 3 - z1 ** 3) / 3.0
                              + r0 * r0 * (a - z0)))
        return np.sign(z) * g

    vol = G(zb) - G(za) - r0 * r0 * (zb - za)
    C = vol / ((r1 * r1 - r0 * r0) * h)
    return np.clip(C, 0.0, 1.0)[None]


_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)


def sphere_vof(n, h, centre, R):
    """Volume fraction of a sphere in each cell of an n^3 grid.

    Cells cut by the sphere are integrated with 16-point Gauss-Legendre in y
    (split at the sphere's poles) of the exact disk-rectangle area in the
    x-z cross-section."""
    xc, yc, zc = centre
    C = np.zeros((n, n, n))
    e = np.arange(n + 1) * h
    X, Y, Zc = e - xc, e - yc, e - zc
    # classify by nearest / farthest corner distance
    def near(a):
        lo, hi = a[:-1], a[1:]
        return np.where((lo <= 0) & (hi >= 0), 0.0, np.minimum(np.abs(lo), np.abs(hi)))

    def far(a):
        return np.maximum(np.abs(a[:-1]), np.abs(a[1:]))

    nx_, ny_, nz_ = near(X), near(Y), near(Zc)
    fx_, fy_, fz_ = far(X), far(Y), far(Zc)
    dn = nz_[:, None, None] ** 2 + ny_[None, :, None] ** 2 + nx_[None, None, :] ** 2
    df = fz_[:, None, None] ** 2 + fy_[None, :, None] ** 2 + fx_[None, None, :] ** 2
    C[df <= R * R] = 1.0
    cut = np.argwhere((dn < R * R) & (df > R * R))
    for k, j, i in cut:
        ya, yb = Y[j], Y[j + 1]
        lo, hi = max(ya, -R), min(yb, R)
        if hi <= lo:
            continue
        tot = 0.0
        ys = 0.5 * (hi + lo) + 0.5 * (hi - lo) * _GL_X
        for y, w in zip(ys, _GL_W):
            rho = math.sqrt(max(R * R - y * y, 0.0))
            if rho <= 0:
                continue
            a = float(circle_rect_area(X[i], X[i + 1], Zc[k], Zc[k + 1], rho))
            tot += w * a
        C[k, j, i] = 0.5 * (hi - lo) * tot / h ** 3
    return np.clip(C, 0.0, 1.0)


# ----------------------------------------------------------- velocities
def single_vortex_faces(n, h, t, T):
    """Face velocities of the single-vortex flow from the vertex stream
    function psi = sin^2(pi x) sin^2(pi y) cos(pi t/T) / pi
    (u = dpsi/dy, v = -dpsi/dx), exactly divergence-free per cell."""
    x = np.arange(n + 1) * h
    s = np.sin(np.pi * x) ** 2
    psi = (s[None, :] * s[:, None]) * math.cos(math.pi * t / T) / math.pi  # [y][x]
    ux = (psi[1:, :] - psi[:-1, :]) / h          # (n, n+1)
    uy = -(psi[:, 1:] - psi[:, :-1]) / h         # (n+1, n)
    return ux[None], uy[None]


def hr_stream(r, cos_t, R, U, lam):
    """Hadamard-Rybczynski Stokes stream function divided by sin^2(theta):
    returns psi / (r sin theta)^2 (regular on the axis).  Drop frame,
    far-field velocity U e_z, viscosity ratio lam = mu_in / mu_out."""
    A = (2 + 3 * lam) / (2 * (1 + lam))
    B = lam / (2 * (1 + lam))
    r = np.maximum(r, 1e-30)
    out = 0.5 * U * (1.0 - A * R / r + B * R ** 3 / r ** 3)
    inn = U / (4 * (1 + lam)) * (r * r / (R * R) - 1.0)
    return np.where(r >= R, out, inn)


def hr_faces_3d(n, h, centre, R, U=1.0, lam=0.01):
    """Face velocities of the Hadamard-Rybczynski flow on an n^3 grid from the
    edge vector potential A = (psi/w^2)(-y, x, 0), w the distance to the
    drop axis; the face fluxes are circulations of A, so every cell's net
    flux cancels exactly."""
    xc, yc, zc = centre
    v = np.arange(n + 1) * h
    m = (np.arange(n) + 0.5) * h

    def pot(x, y, z):
        r = np.sqrt(x * x + y * y + z * z)
        return hr_stream(r, None, R, U, lam)

    # A_y on y-edges at (x_i, y_{j+1/2}, z_k): shape (n+1 z, n y, n+1 x)
    Z, Yh, X = np.meshgrid(v - zc, m - yc, v - xc, indexing="ij")
    Ay = pot(X, Yh, Z) * X
    # A_x on x-edges at (x_{i+1/2}, y_j, z_k): shape (n+1, n+1, n)
    Z2, Y2, Xh = np.meshgrid(v - zc, v - yc, m - xc, indexing="ij")
    Ax = -pot(Xh, Y2, Z2) * Y2
    # x-face (i, j+1/2, k+1/2): h [A_y(z_k) - A_y(z_{k+1})]
    ux = h * (Ay[:-1, :, :] - Ay[1:, :, :]) / (h * h)           # (n, n, n+1)
    # y-face (i+1/2, j, k+1/2): h [A_x(z_{k+1}) - A_x(z_k)]
    uy = h * (Ax[1:, :, :] - Ax[:-1, :, :]) / (h * h)           # (n, n+1, n)
    # z-face (i+1/2, j+1/2, k): h [A_x(y_j) + A_y(x_{i+1}) - A_x(y_{j+1}) - A_y(x_i)]
    uz = h * (Ax[:, :-1, :] + Ay[:, :, 1:] - Ax[:, 1:, :] - Ay[:, :, :-1]) / (h * h)
    return ux, uy, uz


def hr_faces_axi(nr, nz, h, zc, R, U=1.0, lam=0.01):
    """Axisymmetric face velocities from the Stokes stream function
    Psi(r, z) = w^2 * hr_stream: ring fluxes are 2 pi differences of Psi."""
    rv = np.arange(nr + 1) * h
    zv = np.arange(nz + 1) * h - zc
    Z, Rr = np.meshgrid(zv, rv, indexing="ij")                  # (nz+1, nr+1)
    Psi = Rr * Rr * hr_stream(np.sqrt(Rr * Rr + Z * Z), None, R, U, lam)
    # r-face at r_i, z in [z_j, z_j+1]: flux = -2 pi (Psi(z_j+1) - Psi(z_j))
    flux_r = -2 * np.pi * (Psi[1:, :] - Psi[:-1, :])           # (nz, nr+1)
    area_r = 2 * np.pi * rv[None, :] * h
    ur = np.where(area_r > 0, flux_r / np.where(area_r > 0, area_r, 1.0), 0.0)
    # z-face at z_j, r in [r_i, r_i+1]: flux = 2 pi (Psi(r_i+1) - Psi(r_i))
    flux_z = 2 * np.pi * (Psi[:, 1:] - Psi[:, :-1])            # (nz+1, nr)
    area_z = np.pi * (rv[1:] ** 2 - rv[:-1] ** 2)[None, :]
    uz = flux_z / area_z
    return ur[None], uz[None]


def ring_vortex_faces_axi(nr, nz, h):
    """A closed axisymmetric ring vortex: ring fluxes from the stream
    function Psi = r^2 sin^2(pi r/R) sin^2(pi z/Z) on the box [0, R] x
    [0, Z] (R = nr h, Z = nz h), zero on every wall, so no flow crosses
    them and every ring cell is divergence-free."""
    rv = np.arange(nr + 1) * h
    zv = np.arange(nz + 1) * h
    Z, Rr = np.meshgrid(zv, rv, indexing="ij")
    Psi = Rr ** 2 * np.sin(np.pi * Rr / rv[-1]) ** 2 * np.sin(np.pi * Z / zv[-1]) ** 2
    Psi[:, -1] = 0.0
    Psi[0, :] = Psi[-1, :] = 0.0
    flux_r = -2 * np.pi * (Psi[1:, :] - Psi[:-1, :])
    area_r = 2 * np.pi * rv[None, :] * h
    ur = np.where(area_r > 0, flux_r / np.where(area_r > 0, area_r, 1.0), 0.0)
    flux_z = 2 * np.pi * (Psi[:, 1:] - Psi[:, :-1])
    uz = flux_z / (np.pi * (rv[1:] ** 2 - rv[:-1] ** 2)[None, :])
    return ur[None], uz[None]


def solid_rotation_faces(n, h, centre, omega):
    """Solid-body rotation about `centre` from psi = -omega/2 |x - c|^2 on
    an n x n grid (n an int) or an nx x ny grid (n = (nx, ny))."""
    nx, ny = (n, n) if np.isscalar(n) else n
    x = np.arange(nx + 1) * h - centre[0]
    y = np.arange(ny + 1) * h - centre[1]
    psi = -0.5 * omega * (x[None, :] ** 2 + y[:, None] ** 2)
    ux = (psi[1:, :] - psi[:-1, :]) / h
    uy = -(psi[:, 1:] - psi[:, :-1]) / h
    return ux[None], uy[None]


def radial_expansion_faces(shape, h, origin, K):
    """Face velocities of the isotropic expansion u = K (x - c) of Sec. 4.1
    (u = K r e_r) on a 3D grid whose lower corner sits at `origin` relative
    to the centre c; each face carries the normal component at its centre.
    Not divergence-free (div u = 3 K)."""
    nz, ny, nx = shape
    xf = origin[0] + np.arange(nx + 1) * h
    yf = origin[1] + np.arange(ny + 1) * h
    zf = origin[2] + np.arange(nz + 1) * h
    ux = np.broadcast_to(K * xf[None, None, :], (nz, ny, nx + 1)).copy()
    uy = np.broadcast_to(K * yf[None, :, None], (nz, ny + 1, nx)).copy()
    uz = np.broadcast_to(K * zf[:, None, None], (nz + 1, ny, nx)).copy()
    return ux, uy, uz


def cell_centre_offsets(shape, h, origin):
    """Coordinates (x, y, z) of every cell centre, arrays of the cell shape
    (nz, ny, nx), for a grid whose lower corner lies at `origin`."""
    nz, ny, nx = shape
    x = origin[0] + (np.arange(nx) + 0.5) * h
    y = origin[1] + (np.arange(ny) + 0.5) * h
    z = origin[2] + (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def expanding_sphere(N, ds=0.5, half=1.0, K=1.0, octant=True):
    """Expanding sphere of Sec. 4.1: a sphere of diameter ds at the centre of
    the box [-half, half]^3 resolved by N cells per side, in the flow
    u = K r e_r.  With octant=True only the octant [0, half]^3 is gridded
    (N/2 cells per side): its three inner walls are mirror planes of the
    problem (zero normal velocity, zero-gradient walls).  Returns the grid,
    the cell-centre radius r (cell shape) and the face velocities."""
    h = 2.0 * half / N
    n = N // 2 if octant else N
    g = Grid(CART3D, n, n, n, h)
    org = (0.0, 0.0, 0.0) if octant else (-half, -half, -half)
    X, Y, Z = cell_centre_offsets(g.shape, h, org)
    faces = radial_expansion_faces(g.shape, h, org, K)
    return g, np.sqrt(X * X + Y * Y + Z * Z), faces


def rotating_circle(N, db=1.0, domain_over_db=2.0, omega=1.0):
    """Rotating circle of Sec. 4.2: a circle of diameter db at the centre of
    the square [0, L]^2, L = domain_over_db * db, N cells per side, in the
    solid-body rotation of angular velocity omega about the centre.
    Returns the grid, the cell-centre radius and polar angle (cell shape)
    and the face velocities (ux, uy)."""
    L = domain_over_db * db
    h = L / N
    g = Grid(PLANAR, N, N, 1, h)
    X, Y, _ = cell_centre_offsets((1, N, N), h, (-0.5 * L, -0.5 * L, 0.0))
    ux, uy = solid_rotation_faces(N, h, (0.5 * L, 0.5 * L), omega)
    return g, np.sqrt(X * X + Y * Y), np.arctan2(Y, X), (ux, uy)


def uniform_faces(grid: Grid, vel):
    """Uniform translation velocity on every face."""
    nz, ny, nx = grid.shape
    ux = np.full((nz, ny, nx + 1), float(vel[0]))
    uy = np.full((nz, ny + 1, nx), float(vel[1]))
    uz = np.full((nz + 1, ny, nx), float(vel[2])) if grid.geom == CART3D else None
    return ux, uy, uz


# ------------------------------------------------------ seeded random
def smooth_noise(shape2d, seed, corr_cells):
    """White noise N(0,1) convolved with a Gaussian of std corr_cells
    (reflecting boundaries), rescaled to max |g| = 1."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    g = gaussian_filter(rng.standard_normal(shape2d), corr_cells, mode="reflect")
    return g / np.abs(g).max()


# ------------------------------------------------------------ configs
def case_adsorption_2d(n=128, seed=0, steps=1000, tol=1e-10, dt=1e-3):
    """2D planar no-flow diffusion-driven adsorption: unit box, circle R=0.25
    centred, phase-field width 1.5 cells (eps = 0.75 h); bulk 1 outside and
    0 inside (cell average 1 - C), clean interface; Langmuir kinetics
    k_a = 1, k_d = 0.1, Gamma_inf = 1, D = 1e-2; dt = 1e-3."""
    h = 1.0 / n
    g = Grid(PLANAR, n, n, 1, h)
    C = circle_vof(n, n, h, 0.5, 0.5, 0.25)
    p = Params(ka=1.0, kd=0.1, gamma_inf=1.0, Df=1e-2, DF=1e-2, eps=0.75 * h,
               sigma0=1.0, E=0.2, eos=EOS_LANGMUIR)
    return Case("adsorption2d_%d" % n, g, p, C, 1.0 - C, np.zeros_like(C),
                dt=dt, steps=steps, tol=tol)


HR3D_DT = {256: 5e-5}


def case_hr_3d(n=256, Bi=1.0, Da=1.0, steps=2000, tol=1e-10):
    """3D bubble-like transport: n^3 unit cube, sphere R = 0.125 centred,
    prescribed Hadamard-Rybczynski Stokes flow (viscosity ratio 0.01, unit
    far-field velocity), F = 1 and Gamma = 0 initially, Langmuir EOS
    sigma0 = 1, E = 0.2.  Rates from Bi and Da with the bubble diameter
    d = 0.25 and U = 1: k_d = Bi U/d, k_a = Da U/(d F0) (F0 = 1); Peclet
    numbers Pe_F = 10, Pe_f = 100 give D = U d / Pe."""
    h = 1.0 / n
    g = Grid(CART3D, n, n, n, h)
    R, d, U = 0.125, 0.25, 1.0
    C = sphere_vof(n, h, (0.5, 0.5, 0.5), R)
    ux, uy, uz = hr_faces_3d(n, h, (0.5, 0.5, 0.5), R, U, 0.01)
    DF, Df = U * d / 10.0, U * d / 100.0
    p = Params(ka=Da * U / d, kd=Bi * U / d, gamma_inf=1.0, Df=Df, DF=DF,
               eps=0.75 * h, sigma0=1.0, E=0.2, eos=EOS_LANGMUIR, bc_F=1.0,
               bc_f=0.0)
    umax = max(np.abs(ux).max(), np.abs(uy).max(), np.abs(uz).max())
    # dt fixed per resolution, within the Sec. 3.3 bound (checked by a test)
    dt = HR3D_DT.get(n, 3.2 * h * h)
    return Case("hr3d_%d" % n, g, p, C, np.ones_like(C), np.zeros_like(C), ux,
                uy, uz, dt=dt, steps=steps, tol=tol,
                extra=dict(Bi=Bi, Da=Da, umax=umax))


def case_vortex_2d(n=512, t=0.0, T=4.0, soluble=False):
    """2D single vortex: circle R = 0.15 at (0.5, 0.75); insoluble phase
    Gamma0 = 1, D_f = 1e-4; soluble phase Bi = Da = 1 with d = 0.3."""
    h = 1.0 / n
    g = Grid(PLANAR, n, n, 1, h)
    C = circle_vof(n, n, h, 0.5, 0.75, 0.15)
    ux, uy = single_vortex_faces(n, h, t, T)
    d, U = 0.3, 1.0
    if soluble:
        p = Params(ka=1.0 * U / d, kd=1.0 * U / d, gamma_inf=1.0, Df=1e-4,
                   DF=1e-4, eps=0.75 * h)
        F0 = 1.0 - C
        g0 = np.zeros_like(C)
    else:
        p = Params(ka=0.0, kd=0.0, gamma_inf=1.0, Df=1e-4, DF=1e-4, eps=0.75 * h)
        F0 = np.zeros_like(C)
        g0 = np.ones_like(C)
    # dt = T / (8.6 n): about half the Sec. 3.3 advective bound (checked by a test)
    steps = int(round(8.6 * n))
    return Case("vortex2d_%d" % n, g, p, C, F0, g0, ux, uy, None, dt=T / steps,
                steps=steps, extra=dict(T=T))


AXI_DT = {64: 4e-3, 128: 1.5e-3, 256: 4e-4}


def case_axi(nr, nz, Bi, Da, Pe=100.0, R=0.2, steps=500):
    """Axisymmetric instance: (r, z) in [0, nr h] x [0, nz h] with h = 1/nr,
    sphere R on the axis at mid-height, HR Stokes flow, F = 1, Gamma = 0."""
    h = 1.0 / nr
    g = Grid(AXI, nr, nz, 1, h)
    zc = 0.5 * nz * h
    C = ring_vof(nr, nz, h, zc, R)
    ur, uz = hr_faces_axi(nr, nz, h, zc, R, 1.0, 0.01)
    d, U = 2 * R, 1.0
    D = U * d / Pe
    p = Params(ka=Da * U / d, kd=Bi * U / d, gamma_inf=1.0, Df=D, DF=D,
               eps=0.75 * h, bc_F=1.0, bc_f=0.0)
    umax = max(np.abs(ur).max(), np.abs(uz).max())
    # dt fixed per resolution, within the Sec. 3.3 bound (checked by a test)
    dt = AXI_DT.get(nr, 0.1 * h)
    return Case("axi_%dx%d" % (nr, nz), g, p, C, np.ones_like(C),
                np.zeros_like(C), ur, uz, None, dt=dt, steps=steps,
                extra=dict(Bi=Bi, Da=Da, umax=umax))


def batch_axi(n_inst=64, seed=3, steps=500):
    """64 axisymmetric instances with grids drawn from {64x128, 128x256,
    256x512} and log10 Bi, log10 Da uniform in [-2, 2]."""
    rng = np.random.default_rng(seed)
    sizes = [(64, 128), (128, 256), (256, 512)]
    out = []
    for _ in range(n_inst):
        nr, nz = sizes[int(rng.integers(0, 3))]
        Bi, Da = 10.0 ** rng.uniform(-2, 2), 10.0 ** rng.uniform(-2, 2)
        out.append((nr, nz, Bi, Da))
    return out


def case_flat_kinetics(ny, Bi, Da, nx=8, eps_cells=0.75, dt=1e-3, steps=100):
    """Flat-interface kinetics of Sec. 4.3 as a planar column: y in [-4, 4]
    (L = 1), interface at y = 0 with fluid 1 (no bulk surfactant) below, no
    flow, a clean interface and F = 1 above it.  Langmuir kinetics with
    Gamma_inf = F_inf = D_F = D_f = 1, so that Da = r_a Gamma_inf^2/(D_F
    F_inf) = k_a and Bi = r_d = k_d in the scalings of Sec. 4.3."""
    h = 8.0 / ny
    g = Grid(PLANAR, nx, ny, 1, h)
    y = -4.0 + (np.arange(ny) + 0.5) * h
    C = np.zeros(g.shape)
    C[0, y < 0.0, :] = 1.0
    p = Params(ka=Da, kd=Bi, gamma_inf=1.0, Df=1.0, DF=1.0, eps=eps_cells * h,
               bc_F=1.0, bc_f=0.0)
    return Case("flat_%dx%d" % (nx, ny), g, p, C, 1.0 - C, np.zeros_like(C), dt=dt,
                steps=steps, extra=dict(Bi=Bi, Da=Da))


def batch_flat_kinetics(n_inst=512, ny=256, nx=8, seed=5, steps=100, dt=2.5e-4):
    """A sweep of flat-interface columns with log10 Bi, log10 Da uniform in
    [-2, 2] (seeded); dt = 2.5e-4 keeps D dt/h^2 = 0.26 at ny = 256."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        Bi, Da = 10.0 ** rng.uniform(-2, 2), 10.0 ** rng.uniform(-2, 2)
        out.append(case_flat_kinetics(ny, Bi, Da, nx=nx, steps=steps, dt=dt))
    return out


def case_adjoint_2d(n=256, seed=4, corr=4.0):
    """Adjoint workload: the 2D adsorption physics at n^2 with a seeded
    interfacial perturbation Gamma0 = 0.05 (1 + g), g smooth noise."""
    c = case_adsorption_2d(n=n, steps=200)
    gn = smooth_noise((n, n), seed, corr)
    c.gamma0 = (0.05 * (1.0 + gn))[None]
    c.name = "adjoint2d_%d" % n
    return c
