"""Pins of the oracle's forcing source terms (a body force a(x): rho a in the momentum, M . a in the energy,
on every stage's state; the paper defines no forcing, this is the reading the library takes), without a GPU.

- a uniform state under a uniform acceleration: no flux divergence, so each cycle is the integrator applied to
  dM/dt = rho a, dE/dt = M . a.  VL2, RK2 and RK3 integrate that exactly: v = v0 + a dt and the pressure is
  unchanged (the kinetic-energy gain M0 . a dt + rho |a|^2 dt^2 / 2 is reproduced); RK1 leaves the pressure
  lower by (gamma - 1) rho |a|^2 dt^2 / 2 (first order in time), also exactly
- a non-uniform periodic state under a uniform acceleration a0: the mass is unchanged by every stage, so a
  VL2 cycle changes the total momentum by exactly dt m a0 (m the total mass) and the total energy by
  dt a0 . M_total + dt^2 m |a0|^2 / 2 (the corrector's source uses the predictor state)
- a zero acceleration field gives bitwise the unforced cycle; a solenoidal forcing field keeps the mass,
  div B and the bitwise MeshBlock invariance
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

G = 5.0 / 3.0


def uniform_problem(n=8, v0=(0.3, -0.2, 0.1), rho=1.3, p=0.7, b=(0.4, 0.2, -0.3)):
    nx = (n, n, n)
    w = np.empty((5, n, n, n))
    w[0] = rho
    for d in range(3):
        w[1 + d] = v0[d]
    w[4] = p
    b1, b2, b3 = inputs.uniform_faces(nx, b)
    return inputs.Problem("uniform", nx, (4, 4, 4), (0.0,) * 3, (1.0,) * 3, G, w, b1, b2, b3)


def prims(m):
    u, b1, b2, b3 = m.get_cons()
    rho = u[0]
    v = u[1:4] / rho
    bc = (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:] + b2[:, :-1]), 0.5 * (b3[1:] + b3[:-1]))
    p = (G - 1) * (u[4] - 0.5 * rho * (v ** 2).sum(0) - 0.5 * sum(c ** 2 for c in bc))
    return rho, v, p


@pytest.mark.parametrize("integrator", ["vl2", "rk2", "rk3", "rk1"])
def test_uniform_acceleration_is_integrated_exactly(oracle, integrator):
    prob = uniform_problem()
    itg = {"vl2": oracle.VL2, "rk1": oracle.RK1, "rk2": oracle.RK2, "rk3": oracle.RK3}[integrator]
    m = oracle.Mesh.from_problem(prob, integrator=itg)
    a0 = np.array([0.5, -1.25, 0.75])
    m.set_forcing(np.broadcast_to(a0[:, None, None, None], (3,) + prob.w.shape[1:]))
    rho0, v0, p0 = prims(m)
    dt = 0.02
    m.step(dt)
    rho, v, p = prims(m)
    np.testing.assert_allclose(rho, rho0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(v, v0 + a0[:, None, None, None] * dt, rtol=0, atol=1e-14)
    dp = 0.0 if integrator != "rk1" else -(G - 1) * 0.5 * rho0 * (a0 @ a0) * dt * dt
    np.testing.assert_allclose(p, p0 + dp, rtol=0, atol=1e-14)


def test_totals_under_a_uniform_acceleration(oracle):
    prob = inputs.turbulence(n=16, mb=8, seed=7, mach=1.0, beta=1.0)
    m = oracle.Mesh.from_problem(prob)
    a0 = np.array([0.3, 0.7, -0.4])
    m.set_forcing(np.broadcast_to(a0[:, None, None, None], (3,) + prob.w.shape[1:]))
    for _ in range(3):
        t0 = m.totals()
        dt = m.new_dt(0.3)
        m.step(dt)
        t1 = m.totals()
        mass, mom = t0[0], t0[1:4]
        assert abs(t1[0] - mass) <= 1e-14 * mass
        np.testing.assert_allclose(t1[1:4], mom + dt * mass * a0, rtol=0, atol=1e-13 * (1 + np.abs(mom).max()))
        de = dt * (a0 @ mom) + 0.5 * dt * dt * mass * (a0 @ a0)
        assert abs((t1[4] - t0[4]) - de) <= 1e-13 * abs(t0[4])


def test_zero_forcing_is_the_unforced_cycle_and_forcing_keeps_invariants(oracle):
    prob = inputs.turbulence(n=16, mb=8, seed=8, mach=1.0, beta=1.0)
    a = inputs.forcing_field(16, seed=4004, amp=2.0)
    free = oracle.Mesh.from_problem(prob)
    zero = oracle.Mesh.from_problem(prob)
    zero.set_forcing(np.zeros_like(a))
    forced = [oracle.Mesh.from_problem(prob, mb=mb) for mb in ((8, 8, 8), (16, 16, 16))]
    for f in forced:
        f.set_forcing(a)
    mass0 = forced[0].totals()[0]
    for _ in range(4):
        dt = free.new_dt(0.3)
        free.step(dt)
        zero.step(dt)
        for f in forced:
            f.step(dt)
    assert all(np.array_equal(x, y) for x, y in zip(free.get_cons(), zero.get_cons()))
    assert all(np.array_equal(x, y) for x, y in zip(forced[0].get_cons(), forced[1].get_cons()))
    assert not np.array_equal(forced[0].get_cons()[0], free.get_cons()[0])
    assert abs(forced[0].totals()[0] - mass0) <= 1e-14 * mass0
    assert forced[0].divb_norm() <= 1e-13
