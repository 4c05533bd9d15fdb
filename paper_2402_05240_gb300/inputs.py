"""Seeded synthetic initial conditions for the VL+CT ideal-MHD step.

This module generates inputs only.  It holds none of the integrator's
arithmetic (no reconstruction, Riemann solver, EMF or update); it builds a
conserved state ``U`` in the library's layout from a physical description:

* layout ``U[8, nz, ny, nx]`` float64, fields ``rho, mx, my, mz, E, Bx, By, Bz``
  (Sec. 2.1, the conserved vector U);
* ``Bx[k, j, i]`` is the face value at ``x_{i+1/2}`` (upper face), likewise
  ``By`` at ``y_{j+1/2}`` and ``Bz`` at ``z_{k+1/2}`` (Sec. 2.2, staggered grid);
* cell ``(i, j, k)`` has its centre at ``((i+1/2)dx, (j+1/2)dy, (k+1/2)dz)``
  on a periodic box ``[0, Lx) x [0, Ly) x [0, Lz)``.

All random draws use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA_DEFAULT = 5.0 / 3.0


@dataclass
class Box:
    """A periodic box: cell counts and lengths (x, y, z)."""

    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def dz(self) -> float:
        return self.lz / self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def centres(self):
        """Cell-centre coordinate arrays broadcastable to (nz, ny, nx)."""
        x = (np.arange(self.nx) + 0.5) * self.dx
        y = (np.arange(self.ny) + 0.5) * self.dy
        z = (np.arange(self.nz) + 0.5) * self.dz
        return x[None, None, :], y[None, :, None], z[:, None, None]


def assemble(box: Box, rho, vel, pres, bface, gamma=GAMMA_DEFAULT):
    """Conserved state from density, velocity, pressure and face fields.

    ``vel`` is (vx, vy, vz) cell values, ``bface`` is (Bx, By, Bz) on the upper
    faces.  The total energy uses the cell-centred field, the average of the two
    faces of each component (Sec. 2.2.1), and the ideal-gas law P = (gamma-1) eps.
    """
    shape = box.shape
    rho = np.broadcast_to(np.asarray(rho, np.float64), shape)
    vx, vy, vz = (np.broadcast_to(np.asarray(v, np.float64), shape) for v in vel)
    pres = np.broadcast_to(np.asarray(pres, np.float64), shape)
    bx, by, bz = (np.broadcast_to(np.asarray(b, np.float64), shape).copy() for b in bface)
    bcx = 0.5 * (bx + np.roll(bx, 1, axis=2))
    bcy = 0.5 * (by + np.roll(by, 1, axis=1))
    bcz = 0.5 * (bz + np.roll(bz, 1, axis=0))
    U = np.empty((8,) + shape, np.float64)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = (pres / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
            + 0.5 * (bcx * bcx + bcy * bcy + bcz * bcz))
    U[5] = bx
    U[6] = by
    U[7] = bz
    return U


def uniform(box: Box, rho=1.0, vel=(0.0, 0.0, 0.0), pres=1.0, b=(0.0, 0.0, 0.0), gamma=GAMMA_DEFAULT):
    """A uniform state (every cell and face equal)."""
    return assemble(box, rho, vel, pres, b, gamma)


# ---------------------------------------------------------------------------
# Linear waves (Sec. 3.1.1): q = qbar + A R_w sin(2 pi x / lambda)
# ---------------------------------------------------------------------------

def _primitive_jacobian(rho, u, v, w, p, bn, bt1, bt2, gamma):
    """Matrix A of the 1-D primitive ideal-MHD system dW/dt + A dW/dx = 0.

    Variables (rho, u, v, w, P, B_t1, B_t2); B_n is constant along the normal.
    This is the PDE of Sec. 2.1 rewritten in primitive form; it is used here only
    to obtain the wave eigenvector numerically.
    """
    A = np.zeros((7, 7))
    A[0, 0], A[0, 1] = u, rho
    A[1, 1], A[1, 4], A[1, 5], A[1, 6] = u, 1.0 / rho, bt1 / rho, bt2 / rho
    A[2, 2], A[2, 5] = u, -bn / rho
    A[3, 3], A[3, 6] = u, -bn / rho
    A[4, 1], A[4, 4] = gamma * p, u
    A[5, 1], A[5, 2], A[5, 5] = bt1, -bn, u
    A[6, 1], A[6, 3], A[6, 6] = bt2, -bn, u
    return A


WAVES = ("fast-", "alfven-", "slow-", "entropy", "slow+", "alfven+", "fast+")


def wave_eigenvector(rho, vel, p, b, gamma=GAMMA_DEFAULT, wave="fast+"):
    """Conserved-variable right eigenvector along x for one wave family.

    Returns (speed, r) with r over (rho, mx, my, mz, E, By, Bz), unit Euclidean
    norm and a positive density component where it has one.  The primitive
    eigenvector comes from a numerical eigen-decomposition of the primitive
    Jacobian; it is mapped to conserved variables with dU/dW.
    """
    u, v, w = vel
    bn, bt1, bt2 = b
    A = _primitive_jacobian(rho, u, v, w, p, bn, bt1, bt2, gamma)
    lam, vec = np.linalg.eig(A)
    order = np.argsort(lam.real)
    lam = lam.real[order]
    vec = vec.real[:, order]
    k = WAVES.index(wave)
    dw = vec[:, k]
    drho, du, dv, dw_, dp, dby, dbz = dw
    dU = np.array([
        drho,
        u * drho + rho * du,
        v * drho + rho * dv,
        w * drho + rho * dw_,
        dp / (gamma - 1.0) + 0.5 * (u * u + v * v + w * w) * drho
        + rho * (u * du + v * dv + w * dw_) + bt1 * dby + bt2 * dbz,
        dby,
        dbz,
    ])
    dU /= np.linalg.norm(dU)
    lead = dU[0] if abs(dU[0]) > 1e-12 else (dU[5] if abs(dU[5]) > 1e-12 else dU[2])
    if lead < 0:
        dU = -dU
    return lam[k], dU


def linear_wave(box: Box, amp=1e-6, rho=1.0, vel=(0.0, 0.0, 0.0), pres=None,
                b=(1.0, math.sqrt(2.0), 0.5), gamma=GAMMA_DEFAULT, wave="fast+"):
    """A sinusoidal linear wave along x with one wavelength across the box.

    Cell averages of sin(2 pi x) are used: sin(2 pi x_i) * sin(pi dx)/(pi dx)
    for unit wavelength.  Transverse face fields (By on y-faces, Bz on z-faces)
    sit at the cell's x-range and take the same average; Bx is uniform, so the
    discrete divergence is zero.
    """
    if pres is None:
        pres = 1.0 / gamma
    speed, r = wave_eigenvector(rho, vel, pres, b, gamma, wave)
    x, _, _ = box.centres()
    k = 2.0 * math.pi / box.lx
    avg = math.sin(0.5 * k * box.dx) / (0.5 * k * box.dx)
    s = np.broadcast_to(np.sin(k * x) * avg, box.shape)
    bg = uniform(box, rho, vel, pres, b, gamma)
    U = bg.copy()
    for f, comp in zip((0, 1, 2, 3, 4, 6, 7), r):
        U[f] = bg[f] + amp * comp * s
    return U, speed


# ---------------------------------------------------------------------------
# Turbulent box: k^-2 shell spectrum, divergence-free field from a vector
# potential on cell edges.
# ---------------------------------------------------------------------------

def _spectral_field(shape, rng, kmin=1.0, kmax=16.0, slope=-4.0):
    """Real random field with per-mode power |k|^slope for kmin <= |k| <= kmax.

    A shell spectrum E(k) ~ k^-2 corresponds to per-mode power ~ |k|^-4.
    Gaussian white noise is filtered in Fourier space; the k = 0 mode is
    removed, so the mean is zero.
    """
    nz, ny, nx = shape
    noise = rng.standard_normal(shape)
    fk = np.fft.rfftn(noise)
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    filt = np.zeros_like(kk)
    sel = (kk >= kmin) & (kk <= kmax)
    filt[sel] = kk[sel] ** (0.5 * slope)
    return np.fft.irfftn(fk * filt, s=shape, axes=(0, 1, 2))


def turbulent_box(box: Box, seed_v=1, seed_b=2, rho=1.0, pres=1.0, b0=(0.5, 0.0, 0.0),
                  mach=1.0, db_rms=0.1, kmax=16.0, gamma=GAMMA_DEFAULT):
    """Turbulent periodic box: rho, P uniform; random k^-2 velocity at rms Mach
    ``mach``; B = b0 + curl(A) with A on cell edges, scaled to rms |dB_cc| =
    ``db_rms``.  The face field is the discrete curl of edge values, so its
    discrete divergence vanishes to round-off."""
    shape = box.shape
    kmax_eff = min(kmax, 0.5 * min(shape) - 1.0)
    rng_v = np.random.Generator(np.random.PCG64(seed_v))
    vel = [_spectral_field(shape, rng_v, 1.0, kmax_eff) for _ in range(3)]
    vrms = math.sqrt(float(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)))
    cs = math.sqrt(gamma * pres / rho)
    vel = [v * (mach * cs / vrms) for v in vel]

    rng_b = np.random.Generator(np.random.PCG64(seed_b))
    # A_x at (i, j+1/2, k+1/2), A_y at (i+1/2, j, k+1/2), A_z at (i+1/2, j+1/2, k),
    # each stored at index [k, j, i].
    ax, ay, az = (_spectral_field(shape, rng_b, 1.0, kmax_eff) for _ in range(3))
    dx, dy, dz = box.dx, box.dy, box.dz
    # Bx(i+1/2,j,k) = (Az(i+1/2,j+1/2) - Az(i+1/2,j-1/2))/dy - (Ay(i+1/2,k+1/2) - Ay(i+1/2,k-1/2))/dz
    bx = (az - np.roll(az, 1, axis=1)) / dy - (ay - np.roll(ay, 1, axis=0)) / dz
    # By(i,j+1/2,k) = (Ax(j+1/2,k+1/2) - Ax(j+1/2,k-1/2))/dz - (Az(i+1/2,j+1/2) - Az(i-1/2,j+1/2))/dx
    by = (ax - np.roll(ax, 1, axis=0)) / dz - (az - np.roll(az, 1, axis=2)) / dx
    # Bz(i,j,k+1/2) = (Ay(i+1/2,k+1/2) - Ay(i-1/2,k+1/2))/dx - (Ax(j+1/2,k+1/2) - Ax(j-1/2,k+1/2))/dy
    bz = (ay - np.roll(ay, 1, axis=2)) / dx - (ax - np.roll(ax, 1, axis=1)) / dy
    bcx = 0.5 * (bx + np.roll(bx, 1, axis=2))
    bcy = 0.5 * (by + np.roll(by, 1, axis=1))
    bcz = 0.5 * (bz + np.roll(bz, 1, axis=0))
    brms = math.sqrt(float(np.mean(bcx ** 2 + bcy ** 2 + bcz ** 2)))
    s = db_rms / brms
    bface = (b0[0] + s * bx, b0[1] + s * by, b0[2] + s * bz)
    return assemble(box, rho, vel, pres, bface, gamma)


def blast(box: Box, seed=4, rho=1.0, b0=(2.5, 0.0, 0.0), beta=0.1, over=100.0, radius=0.1,
          gamma=GAMMA_DEFAULT):
    """Strongly magnetised periodic blast: P = P0 (1 + (over-1) exp(-r^2/R^2)) with
    P0 = beta |B0|^2 / 2, a Gaussian over-pressure of peak ratio ``over`` centred
    at a seeded point; r is the periodic (minimum-image) distance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = rng.uniform(0.25, 0.75, size=3) * np.array([box.lx, box.ly, box.lz])
    x, y, z = box.centres()

    def dist(c, L, q):
        d = np.abs(q - c)
        return np.minimum(d, L - d)

    r2 = (dist(centre[0], box.lx, x) ** 2 + dist(centre[1], box.ly, y) ** 2
          + dist(centre[2], box.lz, z) ** 2)
    p0 = beta * (b0[0] ** 2 + b0[1] ** 2 + b0[2] ** 2) / 2.0
    pres = p0 * (1.0 + (over - 1.0) * np.exp(-r2 / radius ** 2))
    return assemble(box, rho, (0.0, 0.0, 0.0), pres, b0, gamma)


def shock_tube(box: Box, left, right, bn, gamma=GAMMA_DEFAULT, axis=0):
    """Two states split at the box mid-plane along x (a periodic double interface).

    ``left``/``right`` are (rho, vx, vy, vz, P, By, Bz); ``bn`` is the uniform Bx.
    Used for stationary contact / rotational-discontinuity checks.
    """
    assert axis == 0
    x, _, _ = box.centres()
    mask = np.broadcast_to(x < 0.5 * box.lx, box.shape)
    vals = [np.where(mask, l, r) for l, r in zip(left, right)]
    rho, vx, vy, vz, p, by, bz = vals
    return assemble(box, rho, (vx, vy, vz), p, (np.full(box.shape, bn), by, bz), gamma)


# ---------------------------------------------------------------------------
# The paper's periodic system problems (Sec. 3.1).  Face fields are discrete
# curls of vector potentials on cell edges, so their discrete divergence is
# zero to round-off; a uniform field is added face by face.
# ---------------------------------------------------------------------------

def edge_positions(box: Box, origin=(0.0, 0.0, 0.0)):
    """Coordinates of the edges that carry A_x (i, j+1/2, k+1/2), A_y
    (i+1/2, j, k+1/2) and A_z (i+1/2, j+1/2, k), as (x, y, z) triples of arrays
    broadcastable to (nz, ny, nx)."""
    x, y, z = box.centres()
    x, y, z = x + origin[0], y + origin[1], z + origin[2]
    xf, yf, zf = x + 0.5 * box.dx, y + 0.5 * box.dy, z + 0.5 * box.dz
    return (x, yf, zf), (xf, y, zf), (xf, yf, z)


def faces_from_potential(box: Box, ax, ay, az):
    """Face fields (Bx, By, Bz) on the upper faces from edge potentials (each
    broadcast to the grid, layout [k, j, i], positions of edge_positions)."""
    ax, ay, az = (np.broadcast_to(np.asarray(a, np.float64), box.shape) for a in (ax, ay, az))
    dx, dy, dz = box.dx, box.dy, box.dz
    bx = (az - np.roll(az, 1, axis=1)) / dy - (ay - np.roll(ay, 1, axis=0)) / dz
    by = (ax - np.roll(ax, 1, axis=0)) / dz - (az - np.roll(az, 1, axis=2)) / dx
    bz = (ay - np.roll(ay, 1, axis=2)) / dx - (ax - np.roll(ax, 1, axis=1)) / dy
    return bx, by, bz


# wave-frame basis of the circularly polarised Alfven wave: e1 = (1, 2, 2)/3
# (sin a = 2/3, sin b = 2/sqrt5), the normal for which one wavelength fits the
# 3 x 1.5 x 1.5 box along every axis
_CPAW_E1 = np.array([1.0, 2.0, 2.0]) / 3.0
_CPAW_E2 = np.array([-2.0, 1.0, 0.0]) / math.sqrt(5.0)
_CPAW_E3 = np.cross(_CPAW_E1, _CPAW_E2)


def cpaw(n: int, amp=0.1, v_par=0.0, gamma=GAMMA_DEFAULT):
    """Circularly polarised Alfven wave (Sec. 3.1.2) on 3 x 1.5 x 1.5 with
    2n x n x n cells: rho = 1, P = 0.1, B_par = 1, and in the wave frame
    v_perp = B_perp = amp (sin 2 pi x1, cos 2 pi x1), x1 = e1 . r, lambda = 1.
    v_par = 0 travels at v_A = 1 (period 1); v_par = -1 stands.
    Returns (box, U)."""
    box = Box(2 * n, n, n, 3.0, 1.5, 1.5)
    k = 2.0 * math.pi
    x, y, z = box.centres()
    x1 = _CPAW_E1[0] * x + _CPAW_E1[1] * y + _CPAW_E1[2] * z
    s, c = np.sin(k * x1), np.cos(k * x1)
    vel = [v_par * _CPAW_E1[d] + amp * (s * _CPAW_E2[d] + c * _CPAW_E3[d]) for d in range(3)]
    pots = []
    for d, (ex, ey, ez) in enumerate(edge_positions(box)):
        q = _CPAW_E1[0] * ex + _CPAW_E1[1] * ey + _CPAW_E1[2] * ez
        # dA = (amp/k)(sin(k x1) e2 + cos(k x1) e3): curl gives amp (sin e2 + cos e3)
        pots.append((amp / k) * (np.sin(k * q) * _CPAW_E2[d] + np.cos(k * q) * _CPAW_E3[d]))
    bx, by, bz = faces_from_potential(box, *pots)
    bface = (bx + _CPAW_E1[0], by + _CPAW_E1[1], bz + _CPAW_E1[2])
    return box, assemble(box, 1.0, vel, 0.1, bface, gamma)


def field_loop(n: int, amp=1e-3, radius=0.3, vel=(1.0, 1.0, 2.0), centre=(0.0, 0.0, 0.0), b0=(0.0, 0.0, 0.0),
               gamma=GAMMA_DEFAULT):
    """Advecting field loop (Sec. 3.1.3) on [-1/2, 1/2]^2 x [-1, 1] with
    n x n x 2n cells: rho = 1, P = 1, v = (1, 1, 2), A_x = 0,
    A_y = A_z = amp (R - r) inside r < R = 0.3 (r: distance from ``centre``,
    the domain centre in the paper), plus a uniform field ``b0`` (zero in the
    paper).  One period is t = 1.  Returns (box, U)."""
    box = Box(n, n, 2 * n, 1.0, 1.0, 2.0)
    origin = (-0.5 - centre[0], -0.5 - centre[1], -1.0 - centre[2])
    (_, _, _), (yx, yy, yz), (zx, zy, zz) = edge_positions(box, origin)

    def pot(px, py, pz):
        r = np.sqrt(px * px + py * py + pz * pz)
        return np.where(r < radius, amp * (radius - r), 0.0)

    bx, by, bz = faces_from_potential(box, 0.0, pot(yx, yy, yz), pot(zx, zy, zz))
    return box, assemble(box, 1.0, vel, 1.0, (bx + b0[0], by + b0[1], bz + b0[2]), gamma)


def orszag_tang(n: int, nz: int = 4, gamma=GAMMA_DEFAULT):
    """Orszag-Tang vortex (Sec. 3.1.6) on the unit box with n x n x nz cells
    (uniform along z): rho = 25/(36 pi), P = 5/(12 pi), v = (sin 2 pi y,
    -sin 2 pi x, 0), A_z = (B0 / 4 pi)(cos 4 pi x + 2 cos 2 pi y) with
    B0 = 1/sqrt(4 pi).  Returns (box, U)."""
    box = Box(n, n, nz)
    x, y, _ = box.centres()
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    (_, _, _), (_, _, _), (zx, zy, _) = edge_positions(box)
    az = (b0 / (4.0 * math.pi)) * (np.cos(4.0 * math.pi * zx) + 2.0 * np.cos(2.0 * math.pi * zy))
    bface = faces_from_potential(box, 0.0, 0.0, az)
    vel = (np.sin(2.0 * math.pi * y), -np.sin(2.0 * math.pi * x), 0.0)
    return box, assemble(box, 25.0 / (36.0 * math.pi), vel, 5.0 / (12.0 * math.pi), bface, gamma)


# The paper's Riemann problems (Sec. 3.1.4, table of initial conditions):
# gamma, t_max, B_x, and the left / right states (rho, P, vx, vy, vz, By, Bz).
_S4PI = math.sqrt(4.0 * math.pi)
RIEMANN = {
    "brio_wu": (2.0, 0.1, 0.75, (1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0), (0.125, 0.1, 0.0, 0.0, 0.0, -1.0, 0.0)),
    "dai_woodward": (5.0 / 3.0, 0.2, 2.0 / _S4PI,
                     (1.08, 0.95, 1.2, 0.01, 0.5, 3.6 / _S4PI, 2.0 / _S4PI),
                     (1.0, 1.0, 0.0, 0.0, 0.0, 4.0 / _S4PI, 2.0 / _S4PI)),
    "ryu_jones_1a": (5.0 / 3.0, 0.08, 5.0 / _S4PI, (1.0, 20.0, 10.0, 0.0, 0.0, 5.0 / _S4PI, 0.0),
                     (1.0, 1.0, -10.0, 0.0, 0.0, 5.0 / _S4PI, 0.0)),
    "ryu_jones_4d": (5.0 / 3.0, 0.16, 0.7, (1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0), (0.3, 0.2, 0.0, 0.0, 1.0, 1.0, 0.0)),
    "einfeldt": (1.4, 0.16, 0.0, (1.0, 0.45, -2.0, 0.0, 0.0, 0.5, 0.0), (1.0, 0.45, 2.0, 0.0, 0.0, 0.5, 0.0)),
}


def riemann(name: str, n=512, ntrans=16, mirror=False, skew=0.0):
    """One of the paper's Riemann problems along x on the unit box with
    n x ntrans x ntrans cells, the states split at x = 1/2 (run with outflow
    boundaries along x).  ``mirror``: the same problem reflected, x -> 1 - x
    with v_x -> -v_x and B_x -> -B_x (left and right swapped).  ``skew``
    scales the right state's rho and P by (1 + skew) (0 in the paper).
    Returns (box, U, gamma, t_max)."""
    gamma, t_max, bx, left, right = RIEMANN[name]
    right = (right[0] * (1.0 + skew), right[1] * (1.0 + skew)) + tuple(right[2:])
    box = Box(n, ntrans, ntrans)
    x, _, _ = box.centres()
    if mirror:
        left, right = right, left
    lmask = np.broadcast_to(x < 0.5, box.shape)
    f = [np.where(lmask, a, b) for a, b in zip(left, right)]
    rho, p, vx, vy, vz, by, bz = f
    sx = -1.0 if mirror else 1.0
    U = assemble(box, rho, (sx * vx, vy, vz), p, (np.full(box.shape, sx * bx), by, bz), gamma)
    return box, U, gamma, t_max


def blast_paper(nx=200, ny=300, nz=200, centre=(0.5, 0.75, 0.5), gamma=GAMMA_DEFAULT):
    """MHD blast wave in a strongly magnetised medium (Sec. 3.1.5) on
    1 x 1.5 x 1: rho = 1, P = 0.1 (beta = 0.2), B = (1, 1, 0)/sqrt2, v = 0,
    P = 10 inside the sphere r < 0.1 about ``centre`` (the domain centre in
    the paper; cell centres decide).  Returns (box, U)."""
    box = Box(nx, ny, nz, 1.0, 1.5, 1.0)
    x, y, z = box.centres()
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    pres = np.where(r2 < 0.01, 10.0, 0.1)
    b = 1.0 / math.sqrt(2.0)
    return box, assemble(box, 1.0, (0.0, 0.0, 0.0), pres, (b, b, 0.0), gamma)


def l1_error_norm(U, U0):
    """The paper's error measure (Sec. 3.1.1): the L2 norm over the conserved
    variables of their mean absolute differences."""
    d = np.abs(np.asarray(U) - np.asarray(U0)).reshape(U.shape[0], -1).mean(axis=1)
    return float(np.sqrt(np.sum(d * d)))


# ---------------------------------------------------------------------------
# Axis relabelling (for symmetry checks)
# ---------------------------------------------------------------------------

def cycle_axes(U):
    """Relabel axes x->y, y->z, z->x: returns the state of the rotated problem.

    New field component y is old x, etc.; array axes (z, y, x) are permuted so
    that the old x-axis becomes the new y-axis.  Face arrays move with their
    component, so the upper-face convention is kept.
    """
    # old array axes: (z, y, x) -> new (z', y', x') with x' = old z, y' = old x, z' = old y
    def perm(a):
        return np.ascontiguousarray(np.transpose(a, (1, 2, 0)))

    V = np.empty((U.shape[0],) + perm(U[0]).shape, dtype=U.dtype)
    V[0] = perm(U[0])
    V[1] = perm(U[3])  # new mx = old mz
    V[2] = perm(U[1])  # new my = old mx
    V[3] = perm(U[2])  # new mz = old my
    V[4] = perm(U[4])
    V[5] = perm(U[7])
    V[6] = perm(U[5])
    V[7] = perm(U[6])
    return V
