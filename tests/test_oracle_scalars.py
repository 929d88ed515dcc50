"""Pins of the oracle's passive scalars (Sec. 3.1, eq. passive_scalars: d(rho C)/dt + div(rho v C) = 0)
against what the equation fixes, without a GPU.

- a scalar with C = 1 is the density: rho C equals rho bitwise, cycle after cycle (the scalar flux is the
  mass flux times the upwind concentration)
- the scalar mass is conserved on a periodic mesh
- a profile carried by a uniform flow converges to its translate at second order (PLM), with PPM closer
- donor cell keeps the concentration within its initial bounds (the update is a convex combination)
- mirror symmetry and MeshBlock independence hold bitwise for the scalars too
"""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

G = 5.0 / 3.0


def _scalar_fields(prob, seed, n=2):
    rng = np.random.default_rng(seed)
    nz, ny, nx = prob.w.shape[1:]
    z, y, x = np.meshgrid(*[(np.arange(m) + 0.5) / m for m in (nz, ny, nx)], indexing="ij")
    c = np.empty((n, nz, ny, nx))
    c[0] = 0.5 + 0.4 * np.sin(2 * np.pi * (x + 2 * y) + rng.uniform(0, 2 * np.pi)) * np.cos(2 * np.pi * z)
    c[1] = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    return c


@pytest.mark.parametrize("integrator,recon,riemann", [("VL2", "PLM", 1), ("RK3", "PPM", 0), ("RK1", "PLM", 1)])
def test_unit_concentration_is_the_density(oracle, integrator, recon, riemann):
    prob = inputs.orszag_tang(n=(16, 12, 8), mb=(8, 6, 4), seed=31)
    m = oracle.Mesh.from_problem(prob, riemann=riemann, integrator=getattr(oracle, integrator),
                                 recon=getattr(oracle, recon), nscalars=2)
    c = _scalar_fields(prob, 1)
    c[0] = 1.0
    m.set_scalars(c)
    for _ in range(3):
        m.step(m.new_dt(0.3))
    rc = m.get_scalars()
    np.testing.assert_array_equal(rc[0], m.get_cons()[0][0])


def test_scalar_mass_is_conserved(oracle):
    prob = inputs.orszag_tang(n=16, mb=8, seed=32)
    m = oracle.Mesh.from_problem(prob, nscalars=2)
    m.set_scalars(_scalar_fields(prob, 2))
    s0 = m.get_scalars().sum(axis=(1, 2, 3))
    for _ in range(5):
        m.step(m.new_dt(0.3))
    s1 = m.get_scalars().sum(axis=(1, 2, 3))
    np.testing.assert_allclose(s1, s0, rtol=1e-13)


def _cell_avg_sine(n, t, v):
    """Cell averages on an n x n x 1 grid of the unit square of 0.5 + 0.4 sin(2 pi (x + y - (vx + vy) t)),
    by 4 x 4 Gauss points per cell (error far below the scheme's)."""
    gp, gw = np.polynomial.legendre.leggauss(4)
    h = 1.0 / n
    x0 = np.arange(n) * h
    out = np.zeros((1, n, n))
    for a, wa in zip(gp, gw):
        for b, wb in zip(gp, gw):
            xx = x0[None, :] + (a + 1) * h / 2
            yy = x0[:, None] + (b + 1) * h / 2
            out[0] += wa * wb / 4 * (0.5 + 0.4 * np.sin(2 * np.pi * (xx + yy - (v[0] + v[1]) * t)))
    return out


def _advect_error(oracle, n, recon, integrator):
    nx = (n, n, 1)
    w = np.empty((5, 1, n, n))
    v = (0.7, 0.4, 0.0)
    w[0], w[1], w[2], w[3], w[4] = 1.0, v[0], v[1], v[2], 1.0
    b1, b2, b3 = inputs.uniform_faces(nx, (0.3, 0.2, 0.1))
    m = oracle.Mesh(nx, nx, riemann=oracle.HLLD, integrator=getattr(oracle, integrator),
                    recon=getattr(oracle, recon), nscalars=1)
    m.set_prims(w, b1, b2, b3)
    m.set_scalars(_cell_avg_sine(n, 0.0, v)[None])
    t_end = 0.5 / (v[0] + v[1])  # the profile moves half a period along x + y
    m.run(t_end, cfl=0.3)
    return float(np.mean(np.abs(m.get_scalars()[0] - _cell_avg_sine(n, t_end, v))))


@pytest.mark.parametrize("integrator", ["VL2", "RK3"])
def test_advected_scalar_converges(oracle, integrator):
    e = {r: [_advect_error(oracle, n, r, integrator) for n in (24, 48)] for r in ("PLM", "PPM")}
    slope = math.log2(e["PLM"][0] / e["PLM"][1])
    print("%s scalar advection L1: PLM %s (slope %.2f), PPM %s" % (integrator, e["PLM"], slope, e["PPM"]))
    assert 1.8 <= slope <= 2.6
    assert e["PPM"][1] < e["PLM"][1]


def test_donor_cell_keeps_bounds(oracle):
    prob = inputs.orszag_tang(n=16, mb=8, seed=33)
    m = oracle.Mesh.from_problem(prob, integrator=oracle.RK1, nscalars=2)
    c = _scalar_fields(prob, 3)
    m.set_scalars(c)
    lo, hi = c.min(axis=(1, 2, 3)), c.max(axis=(1, 2, 3))
    for _ in range(5):
        m.step(m.new_dt(0.3))
    conc = m.get_scalars() / m.get_cons()[0][0][None]
    assert np.all(conc.min(axis=(1, 2, 3)) >= lo - 1e-13)
    assert np.all(conc.max(axis=(1, 2, 3)) <= hi + 1e-13)


@pytest.mark.parametrize("axis", [0, 2])
def test_scalar_mirror_symmetry_and_blocks(oracle, axis):
    p = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=37 + axis)
    rng = np.random.default_rng(5)
    c = rng.uniform(0.0, 1.0, size=(1,) + p.w.shape[1:])
    npa = 3 - axis  # numpy axis of a (var, z, y, x) array
    half = c.shape[npa] // 2
    sl = [slice(None)] * 4
    sl[npa] = slice(half, None)
    c[tuple(sl)] = np.flip(c, axis=npa)[tuple(sl)]  # symmetric about the mid plane
    ms = [oracle.Mesh.from_problem(p, recon=oracle.PPM, integrator=oracle.RK3, nscalars=1, mb=mb)
          for mb in ((8, 8, 8), (16, 16, 16))]
    for m in ms:
        m.set_scalars(c)
    for _ in range(3):
        dt = ms[0].new_dt(0.3)
        for m in ms:
            m.step(dt)
    rc = ms[0].get_scalars()
    np.testing.assert_array_equal(rc, np.flip(rc, axis=npa))
    np.testing.assert_array_equal(rc, ms[1].get_scalars())
