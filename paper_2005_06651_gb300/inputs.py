"""Seeded synthetic initial states for the VL2 MHD step.

This module holds only problem set-up: primitive cell values (rho, v, p) and face-centred magnetic
fields.  It contains none of the integration method's arithmetic, imports nothing from the CUDA
binding or from the CPU oracle, and is the one module both sides may share.

Face fields are always built as the discrete curl of an edge-centred vector potential sampled on a
periodic node lattice, so that the discrete divergence of B vanishes to round-off and periodic
duplicate faces (face N and face 0) are bitwise equal.

Array conventions (global active region, C order):
  w  : [5][NZ][NY][NX]  rho, vx, vy, vz, p at cell centres
  b1 : [NZ][NY][NX+1]   B_x on x-faces (face i sits at the lower side of cell i)
  b2 : [NZ][NY+1][NX]   B_y on y-faces
  b3 : [NZ+1][NY][NX]   B_z on z-faces
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PERIODIC = 0
OUTFLOW = 1


@dataclasses.dataclass
class Problem:
    """A complete initial state plus the mesh it lives on."""

    name: str
    nx: tuple  # global active cells (NX, NY, NZ)
    mb: tuple  # MeshBlock active cells
    xmin: tuple
    xmax: tuple
    gamma: float
    w: np.ndarray
    b1: np.ndarray
    b2: np.ndarray
    b3: np.ndarray
    bc: tuple = (PERIODIC,) * 6
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def dx(self):
        return tuple((self.xmax[d] - self.xmin[d]) / self.nx[d] for d in range(3))

    @property
    def ncells(self):
        return int(self.nx[0] * self.nx[1] * self.nx[2])


# ------------------------------------------------------------------------------------------------
# geometry helpers
# ------------------------------------------------------------------------------------------------

def _centres(nx, xmin, xmax):
    """Cell-centre and node coordinates along each dimension (node n is the lower face of cell n)."""
    cc, nodes = [], []
    for d in range(3):
        h = (xmax[d] - xmin[d]) / nx[d]
        cc.append(xmin[d] + (np.arange(nx[d]) + 0.5) * h)
        nodes.append(xmin[d] + np.arange(nx[d]) * h)
    return cc, nodes


def faces_from_potential(nx, xmin, xmax, ax, ay, az):
    """Face fields = discrete curl of an edge-centred vector potential (Stokes on each face).

    ax[k][j][i] is A_x on the x-edge through cell centre x_i at node (y_j, z_k); ay[k][j][i] is A_y
    at (x_i node, y_j centre, z_k node); az[k][j][i] is A_z at (x_i node, y_j node, z_k centre).
    All three are periodic node arrays of shape (NZ, NY, NX); node N is node 0.
    """
    NX, NY, NZ = nx
    hx, hy, hz = ((xmax[d] - xmin[d]) / nx[d] for d in range(3))
    rollx = lambda a: np.roll(a, -1, axis=2)  # value at i+1 (periodic)
    rolly = lambda a: np.roll(a, -1, axis=1)
    rollz = lambda a: np.roll(a, -1, axis=0)
    bx = (rolly(az) - az) / hy - (rollz(ay) - ay) / hz
    by = (rollz(ax) - ax) / hz - (rollx(az) - az) / hx
    bz = (rollx(ay) - ay) / hx - (rolly(ax) - ax) / hy
    b1 = np.concatenate([bx, bx[:, :, :1]], axis=2)
    b2 = np.concatenate([by, by[:, :1, :]], axis=1)
    b3 = np.concatenate([bz, bz[:1, :, :]], axis=0)
    return (np.ascontiguousarray(b1), np.ascontiguousarray(b2), np.ascontiguousarray(b3))


def uniform_faces(nx, b0):
    NX, NY, NZ = nx
    return (np.full((NZ, NY, NX + 1), float(b0[0])), np.full((NZ, NY + 1, NX), float(b0[1])),
            np.full((NZ + 1, NY, NX), float(b0[2])))


def _edge_coords(nx, xmin, xmax):
    cc, nodes = _centres(nx, xmin, xmax)
    # grids (z, y, x) for the three edge families
    ex = np.meshgrid(nodes[2], nodes[1], cc[0], indexing="ij")
    ey = np.meshgrid(nodes[2], cc[1], nodes[0], indexing="ij")
    ez = np.meshgrid(cc[2], nodes[1], nodes[0], indexing="ij")
    # reorder to (x, y, z) tuples
    return ((ex[2], ex[1], ex[0]), (ey[2], ey[1], ey[0]), (ez[2], ez[1], ez[0]))


def _cell_coords(nx, xmin, xmax):
    cc, _ = _centres(nx, xmin, xmax)
    z, y, x = np.meshgrid(cc[2], cc[1], cc[0], indexing="ij")
    return x, y, z


# ------------------------------------------------------------------------------------------------
# Orszag-Tang-style 3D vortex (seeded phases)
# ------------------------------------------------------------------------------------------------

def orszag_tang(n=256, mb=32, seed=2005, b0=0.5, gamma=5.0 / 3.0):
    """3D Orszag-Tang-style vortex on the unit periodic cube with seeded random phases.

    rho = 1, p = 1; v = (-sin(2 pi y + f1), sin(2 pi x + f2), 0.2 sin(2 pi (x + y) + f3));
    A = (b0 / 2 pi) (sin(2 pi z + f4), sin(2 pi x + f5), cos(4 pi x + f6) / 2 + cos(2 pi y + f7)),
    f_i ~ U[0, 2 pi) from numpy PCG64(seed).
    """
    nx = (n, n, n) if np.isscalar(n) else tuple(n)
    mbt = (mb, mb, mb) if np.isscalar(mb) else tuple(mb)
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=7)
    tp = 2.0 * math.pi
    x, y, z = _cell_coords(nx, xmin, xmax)
    w = np.empty((5,) + x.shape)
    w[0] = 1.0
    w[1] = -np.sin(tp * y + ph[0])
    w[2] = np.sin(tp * x + ph[1])
    w[3] = 0.2 * np.sin(tp * (x + y) + ph[2])
    w[4] = 1.0
    (exx, exy, exz), (eyx, eyy, eyz), (ezx, ezy, ezz) = _edge_coords(nx, xmin, xmax)
    c = b0 / tp
    ax = c * np.sin(tp * exz + ph[3])
    ay = c * np.sin(tp * eyx + ph[4])
    az = c * (0.5 * np.cos(2.0 * tp * ezx + ph[5]) + np.cos(tp * ezy + ph[6]))
    b1, b2, b3 = faces_from_potential(nx, xmin, xmax, ax, ay, az)
    return Problem("orszag_tang", nx, mbt, xmin, xmax, gamma, np.ascontiguousarray(w), b1, b2, b3,
                   meta={"seed": seed, "phases": ph.tolist(), "b0": b0})


# ------------------------------------------------------------------------------------------------
# Linear MHD waves
# ------------------------------------------------------------------------------------------------

def primitive_jacobian(rho, vn, vt1, vt2, p, bn, bt1, bt2, gamma):
    """7x7 matrix A of the 1D primitive system W_t + A W_x = 0, W = (rho, vn, vt1, vt2, p, bt1, bt2)."""
    A = np.zeros((7, 7))
    A[0, 0], A[0, 1] = vn, rho
    A[1, 1], A[1, 4], A[1, 5], A[1, 6] = vn, 1.0 / rho, bt1 / rho, bt2 / rho
    A[2, 2], A[2, 5] = vn, -bn / rho
    A[3, 3], A[3, 6] = vn, -bn / rho
    A[4, 1], A[4, 4] = gamma * p, vn
    A[5, 1], A[5, 2], A[5, 5] = bt1, -bn, vn
    A[6, 1], A[6, 3], A[6, 6] = bt2, -bn, vn
    return A


WAVES = ("fast", "alfven", "slow", "entropy")


def wave_eigen(kind, rho, v, p, b, gamma):
    """Right-going eigenpair (speed, right eigenvector) of the primitive system in the wave frame.

    `v` and `b` are (normal, t1, t2) components.  The eigenvector is normalised to unit max-norm.
    """
    A = primitive_jacobian(rho, v[0], v[1], v[2], p, b[0], b[1], b[2], gamma)
    lam, R = np.linalg.eig(A)
    lam = lam.real
    R = R.real
    order = np.argsort(lam)
    lam, R = lam[order], R[:, order]
    # ascending: u-cf, u-ca, u-cs, u, u+cs, u+ca, u+cf
    idx = {"fast": 6, "alfven": 5, "slow": 4, "entropy": 3}[kind]
    r = R[:, idx]
    r = r / r[np.argmax(np.abs(r))]
    return float(lam[idx]), r


def linear_wave(n=32, mb=None, kind="alfven", amp=1.0e-6, geometry="cube", b_unit=True,
                v0=(0.0, 0.0, 0.0), gamma=5.0 / 3.0, phase=0.0):
    """Linear MHD wave on a periodic box, propagating along a grid diagonal.

    geometry "cube": unit cube, n^3 cells, k = 2 pi (1, 1, 1) (wavelength 1/sqrt(3)).
    geometry "paper": box (3, 1.5, 1.5) with 2n x n x n cells and wavelength 1; the periodic
    diagonal direction is k_hat = (1, 2, 2)/3, i.e. k = 2 pi (1/3, 2/3, 2/3).
    Background (wave frame): rho = 1, p = 1/gamma, b = (1, sqrt 2, 1/2) (c_f = 2, c_A = 1, c_s = 1/2),
    scaled to |b| = 1 when b_unit.  `v0` is a uniform background flow in the grid frame; `phase` shifts the
    profile sin(k.x + phase) (with phase 0 the extrema and zeros sit on cell symmetry points of the grid).
    Returns the Problem; meta holds the wave speed, the period and the exact (initial) state.
    """
    if geometry == "cube":
        nx = (n, n, n)
        xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
        kvec = 2.0 * math.pi * np.array([1.0, 1.0, 1.0])
    elif geometry == "paper":
        nx = (2 * n, n, n)
        xmin, xmax = (0.0, 0.0, 0.0), (3.0, 1.5, 1.5)
        kvec = 2.0 * math.pi * np.array([1.0, 2.0, 2.0]) / 3.0
    else:
        raise ValueError(geometry)
    mbt = nx if mb is None else ((mb, mb, mb) if np.isscalar(mb) else tuple(mb))
    kmag = float(np.linalg.norm(kvec))
    nhat = kvec / kmag
    t1 = np.array([nhat[1], -nhat[0], 0.0])
    if np.linalg.norm(t1) < 1e-12:
        t1 = np.array([0.0, nhat[2], -nhat[1]])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nhat, t1)
    bw = np.array([1.0, math.sqrt(2.0), 0.5])
    if b_unit:
        bw = bw / np.linalg.norm(bw)
    rho0, p0 = 1.0, 1.0 / gamma
    v0 = np.asarray(v0, dtype=float)
    vw = np.array([v0 @ nhat, v0 @ t1, v0 @ t2])
    speed, r = wave_eigen(kind, rho0, vw, p0, bw, gamma)
    x, y, z = _cell_coords(nx, xmin, xmax)
    ph = kvec[0] * x + kvec[1] * y + kvec[2] * z + phase
    s = amp * np.sin(ph)
    w = np.empty((5,) + x.shape)
    w[0] = rho0 + r[0] * s
    vel_wave = [vw[0] + r[1] * s, vw[1] + r[2] * s, vw[2] + r[3] * s]
    for d in range(3):
        w[1 + d] = vel_wave[0] * nhat[d] + vel_wave[1] * t1[d] + vel_wave[2] * t2[d]
    w[4] = p0 + r[4] * s
    # field: uniform background plus curl of A = cos(k.x) (alpha t1 + beta t2)
    alpha = -amp * r[6] / kmag
    beta = amp * r[5] / kmag
    avec = alpha * t1 + beta * t2
    (exx, exy, exz), (eyx, eyy, eyz), (ezx, ezy, ezz) = _edge_coords(nx, xmin, xmax)
    ax = avec[0] * np.cos(kvec[0] * exx + kvec[1] * exy + kvec[2] * exz + phase)
    ay = avec[1] * np.cos(kvec[0] * eyx + kvec[1] * eyy + kvec[2] * eyz + phase)
    az = avec[2] * np.cos(kvec[0] * ezx + kvec[1] * ezy + kvec[2] * ezz + phase)
    b1, b2, b3 = faces_from_potential(nx, xmin, xmax, ax, ay, az)
    bg = bw[0] * nhat + bw[1] * t1 + bw[2] * t2
    b1 += bg[0]
    b2 += bg[1]
    b3 += bg[2]
    wavelength = 2.0 * math.pi / kmag
    # the pattern moves at (speed) along nhat in the grid frame (speed includes the background flow)
    period = wavelength / abs(speed)
    return Problem("linear_wave_" + kind, nx, mbt, xmin, xmax, gamma, np.ascontiguousarray(w), b1, b2, b3,
                   meta={"speed": speed, "period": period, "wavelength": wavelength, "amp": amp,
                         "eigvec": r.tolist(), "kind": kind, "geometry": geometry})


# ------------------------------------------------------------------------------------------------
# Random-phase turbulence (Gaussian velocity field, k^-2 amplitude spectrum)
# ------------------------------------------------------------------------------------------------

def _irfftn(a, shape):
    try:  # multithreaded when scipy is present; same transform either way
        import scipy.fft

        return scipy.fft.irfftn(a, s=shape, axes=(0, 1, 2), workers=-1)
    except ImportError:
        return np.fft.irfftn(a, s=shape, axes=(0, 1, 2))


def turbulence(n=64, mb=None, seed=3003, mach=1.0, beta=1.0, gamma=5.0 / 3.0):
    """Gaussian random velocity field on the unit periodic cube.

    rho = 1, p = 1/gamma (sound speed 1).  Fourier modes have complex-Gaussian amplitudes with
    |v_hat(k)| proportional to |k|^-2 for 1 <= |k|/(2 pi) <= n/8; the real field is scaled to
    rms |v| = mach.  B is uniform along x with plasma beta = 2 p / B^2.
    """
    nx = (n, n, n) if np.isscalar(n) else tuple(n)
    mbt = nx if mb is None else ((mb, mb, mb) if np.isscalar(mb) else tuple(mb))
    rng = np.random.Generator(np.random.PCG64(seed))
    NX, NY, NZ = nx
    kx = np.fft.fftfreq(NX, 1.0 / NX)
    ky = np.fft.fftfreq(NY, 1.0 / NY)
    kz = np.fft.rfftfreq(NZ, 1.0 / NZ)
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    kmax = max(1.0, min(nx) / 8.0)
    mask = (kk >= 1.0) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[mask] = kk[mask] ** -2.0
    vel = []
    for _ in range(3):
        re = rng.standard_normal(kk.shape)
        im = rng.standard_normal(kk.shape)
        field = _irfftn(amp * (re + 1j * im), (NX, NY, NZ))  # Hermitian by construction
        field -= field.mean()
        vel.append(np.transpose(field, (2, 1, 0)))  # (x, y, z) -> (z, y, x)
    vrms = math.sqrt(sum(float(np.mean(v ** 2)) for v in vel))
    scale = mach / vrms if vrms > 0 else 0.0
    p0 = 1.0 / gamma
    bmag = math.sqrt(2.0 * p0 / beta)
    w = np.empty((5, NZ, NY, NX))
    w[0] = 1.0
    for d in range(3):
        w[1 + d] = vel[d] * scale
    w[4] = p0
    b1, b2, b3 = uniform_faces(nx, (bmag, 0.0, 0.0))
    return Problem("turbulence", nx, mbt, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), gamma, np.ascontiguousarray(w),
                   b1, b2, b3, meta={"seed": seed, "mach": mach, "beta": beta})


def forcing_field(n=64, seed=4004, amp=1.0, kmax=2.0):
    """Fixed solenoidal acceleration field a(x) on the unit periodic cube, for driven turbulence (a forcing
    the paper does not define; see the forcing reading): complex-Gaussian Fourier modes on the shell
    1 <= |k|/(2 pi) <= kmax, each projected onto the plane normal to its wave vector (div a = 0 mode by mode),
    mean removed, scaled to rms |a| = amp.  Returns a (3, NZ, NY, NX) at the cell centres."""
    nx = (n, n, n) if np.isscalar(n) else tuple(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    NX, NY, NZ = nx
    kx = np.fft.fftfreq(NX, 1.0 / NX)
    ky = np.fft.fftfreq(NY, 1.0 / NY)
    kz = np.fft.rfftfreq(NZ, 1.0 / NZ)
    K = np.meshgrid(kx, ky, kz, indexing="ij")
    kk2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    mask = (kk2 >= 1.0) & (kk2 <= kmax * kmax)
    modes = [np.where(mask, rng.standard_normal(kk2.shape) + 1j * rng.standard_normal(kk2.shape), 0.0)
             for _ in range(3)]
    kdot = sum(K[d] * modes[d] for d in range(3))
    inv = np.where(kk2 > 0, 1.0 / np.where(kk2 > 0, kk2, 1.0), 0.0)
    modes = [modes[d] - K[d] * kdot * inv for d in range(3)]
    acc = []
    for d in range(3):
        field = _irfftn(modes[d], (NX, NY, NZ))
        field -= field.mean()
        acc.append(np.transpose(field, (2, 1, 0)))
    arms = math.sqrt(sum(float(np.mean(a ** 2)) for a in acc))
    scale = amp / arms if arms > 0 else 0.0
    return np.ascontiguousarray(np.stack(acc) * scale)


# ------------------------------------------------------------------------------------------------
# Blast wave (Sec. 3.4, 3D blast wave tests; the paper's performance problem)
# ------------------------------------------------------------------------------------------------

def blast(n=256, mb=32, r0=0.01, e_tot=1.0, p_ambient=1e-3, magnetized=True, gamma=5.0 / 3.0):
    """Periodic unit cube, rho = 1 and p = p_ambient everywhere, except the cells whose centres lie within
    r0 of the centre.  Those hold the total internal energy e_tot = sum p/(gamma-1) dV exactly (the
    discrete form of the paper's integral; for r0 = 0.01 and e_tot = 1 the sphere's pressure is 1.6e5).
    The field is uniform, B = (sqrt 3, 1, 0) when magnetized.  Raises if no cell centre lies inside r0."""
    nx = (n, n, n) if np.isscalar(n) else tuple(n)
    mbt = (mb, mb, mb) if np.isscalar(mb) else tuple(mb)
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    x, y, z = _cell_coords(nx, xmin, xmax)
    inside = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 < r0 * r0
    nin = int(inside.sum())
    if nin == 0:
        raise ValueError("no cell centre lies within r0 = %g at this resolution" % r0)
    dv = 1.0 / (nx[0] * nx[1] * nx[2])
    p_in = (gamma - 1.0) * e_tot / (nin * dv)
    w = np.zeros((5,) + x.shape)
    w[0] = 1.0
    w[4] = np.where(inside, p_in, p_ambient)
    b0 = (math.sqrt(3.0), 1.0, 0.0) if magnetized else (0.0, 0.0, 0.0)
    b1, b2, b3 = uniform_faces(nx, b0)
    return Problem("blast", nx, mbt, xmin, xmax, gamma, np.ascontiguousarray(w), b1, b2, b3,
                   meta={"r0": r0, "p_in": p_in, "cells_inside": nin, "magnetized": magnetized})


# ------------------------------------------------------------------------------------------------
# Shock tubes (one-dimensional along a chosen axis, periodic double tube)
# ------------------------------------------------------------------------------------------------

def shock_tube(n=256, axis=0, left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.1),
               b_left=(0.0, 0.0, 0.0), b_right=(0.0, 0.0, 0.0), gamma=1.4):
    """Periodic double shock tube on [0, 1) along `axis`: the left state fills [1/4, 3/4), the right
    state the rest, so Riemann problems sit at x = 3/4 (left | right) and at x = 1/4 (right | left).

    States are (rho, v_n, v_t1, v_t2, p) and fields (b_n, b_t1, b_t2) in the sweep frame of `axis`
    (t1, t2 cyclic).  b_n must be equal on both sides.  Transverse fields are set through a vector
    potential so that the discrete divergence is zero.
    """
    if b_left[0] != b_right[0]:
        raise ValueError("normal field must be continuous")
    nx = [1, 1, 1]
    nx[axis] = n
    nx = tuple(nx)
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    x3 = _cell_coords(nx, xmin, xmax)
    s = x3[axis]
    inside = (s >= 0.25) & (s < 0.75)
    t1, t2 = (axis + 1) % 3, (axis + 2) % 3
    w = np.empty((5,) + s.shape)
    w[0] = np.where(inside, left[0], right[0])
    w[1 + axis] = np.where(inside, left[1], right[1])
    w[1 + t1] = np.where(inside, left[2], right[2])
    w[1 + t2] = np.where(inside, left[3], right[3])
    w[4] = np.where(inside, left[4], right[4])
    # transverse field is piecewise constant in the sweep coordinate: set face values directly
    # (faces normal to t1/t2 have no dependence on those directions, so div B = 0 exactly)
    faces = list(uniform_faces(nx, (0.0, 0.0, 0.0)))
    bvec = [0.0, 0.0, 0.0]
    bvec[axis] = b_left[0]
    faces[axis][...] = b_left[0]
    for comp, (bl, br) in ((t1, (b_left[1], b_right[1])), (t2, (b_left[2], b_right[2]))):
        shape = faces[comp].shape
        cc = _centres(nx, xmin, xmax)[0][axis]
        prof = np.where((cc >= 0.25) & (cc < 0.75), bl, br)
        # broadcast the profile along the sweep axis of the face array
        view_shape = [1, 1, 1]
        view_shape[2 - axis] = n
        faces[comp][...] = np.broadcast_to(prof.reshape(view_shape), shape)
    return Problem("shock_tube", nx, nx, xmin, xmax, gamma, np.ascontiguousarray(w),
                   *(np.ascontiguousarray(f) for f in faces),
                   meta={"axis": axis, "left": left, "right": right, "b_left": b_left, "b_right": b_right})


# ------------------------------------------------------------------------------------------------
# Mirror-symmetric random state
# ------------------------------------------------------------------------------------------------

def mirror_symmetric(n=16, mb=None, axis=0, seed=7, gamma=5.0 / 3.0, amp=0.3):
    """Smooth random periodic state that is exactly (bitwise) symmetric under x_axis -> -x_axis about
    the domain's lower face: rho, p, transverse v and transverse B even; normal v and normal B odd.
    """
    nx = (n, n, n) if np.isscalar(n) else tuple(n)
    mbt = nx if mb is None else ((mb, mb, mb) if np.isscalar(mb) else tuple(mb))
    rng = np.random.Generator(np.random.PCG64(seed))
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    x, y, z = _cell_coords(nx, xmin, xmax)
    tp = 2.0 * math.pi

    def smooth(xx, yy, zz):
        c = rng.uniform(-1.0, 1.0, size=(4,))
        ph = rng.uniform(0.0, tp, size=(4,))
        return (c[0] * np.sin(tp * xx + ph[0]) + c[1] * np.sin(tp * yy + ph[1]) + c[2] * np.sin(tp * zz + ph[2])
                + c[3] * np.sin(tp * (xx + yy + zz) + ph[3]))

    w = np.empty((5,) + x.shape)
    w[0] = 1.0 + 0.5 * amp * smooth(x, y, z)
    for d in range(3):
        w[1 + d] = amp * smooth(x, y, z)
    w[4] = 1.0 + 0.5 * amp * smooth(x, y, z)
    (exx, exy, exz), (eyx, eyy, eyz), (ezx, ezy, ezz) = _edge_coords(nx, xmin, xmax)
    ax = 0.05 * smooth(exx, exy, exz)
    ay = 0.05 * smooth(eyx, eyy, eyz)
    az = 0.05 * smooth(ezx, ezy, ezz)
    b1, b2, b3 = faces_from_potential(nx, xmin, xmax, ax, ay, az)
    b = [b1 + 0.3, b2 + 0.2, b3 - 0.1]
    # symmetrise about the plane x_axis = 0 (periodic): cell c <-> N-1-c, face f <-> N-f
    npa = 2 - axis  # numpy axis of the mirrored direction

    def mirror_cells(a):
        return np.flip(a, axis=npa)

    def mirror_faces(a):
        # face index f -> N - f (face N == face 0 periodic)
        return np.flip(a, axis=npa)

    out = np.empty_like(w)
    for v in range(5):
        m = mirror_cells(w[v])
        if v == 1 + axis:
            out[v] = 0.5 * (w[v] - m)
        else:
            out[v] = 0.5 * (w[v] + m)
    bs = []
    for c in range(3):
        if c == axis:
            m = mirror_faces(b[c])
            bs.append(np.ascontiguousarray(0.5 * (b[c] - m)))
        else:
            m = mirror_cells(b[c])
            bs.append(np.ascontiguousarray(0.5 * (b[c] + m)))
    return Problem("mirror_symmetric", nx, mbt, xmin, xmax, gamma, np.ascontiguousarray(out), *bs,
                   meta={"axis": axis, "seed": seed})
