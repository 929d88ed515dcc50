"""Pins of the oracle's smoothed CT upwind weight, an option beside the paper's sign switch (Sec. 3.1): the
corner corrections take w = (1 + tanh(m / delta)) / 2 on the upwind-side gradient.

- a vanishing delta is the sign switch itself, bitwise (w saturates to 0 or 1, and is 1/2 at m = 0)
- with delta well below the flow's mass fluxes the scheme keeps second-order convergence
- delta makes the corner a smooth function of the mass flux: the magnetized blast, whose zero mass fluxes
  make the sharp switch ill-conditioned, then moves by round-off only under round-off changes of its input
- the tangent-linear (dual numbers) carries dw/dm and matches central differences of the smoothed cycle;
  on the magnetized blast the sharp cycle has a jump (finite differences grow as 1/h), the smoothed one
  none
"""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_gpu_parity import state_diff
from test_oracle_mesh import _inclined, rms_l1_error


def test_vanishing_delta_is_the_sign_switch(oracle):
    p = inputs.orszag_tang(n=24, mb=12, seed=5)
    a = oracle.Mesh.from_problem(p)
    b = oracle.Mesh.from_problem(p, ct_delta=1e-300)
    for _ in range(3):
        dt = a.new_dt(0.3)
        a.step(dt)
        b.step(dt)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_cons(), b.get_cons()))
    with pytest.raises(ValueError):
        oracle.Mesh(p.nx, p.mb, ct_delta=-1.0)


def test_small_delta_keeps_second_order(oracle):
    errs = []
    for n in (32, 64):
        prob = _inclined("fast", (n, n, 2), (2 * math.pi, 2 * math.pi, 0.0), (0.0, 0.0, 0.0))
        m = oracle.Mesh.from_problem(prob, ct_delta=1e-9)  # the wave's mass fluxes are ~1e-6
        ref = m.get_cons()
        m.run(prob.meta["period"], cfl=0.3)
        errs.append(rms_l1_error(m.get_cons(), ref))
    slope = math.log2(errs[0] / errs[1])
    print("smoothed CT (delta 1e-9) fast wave: L1 %s, slope %.3f" % (errs, slope))
    assert 1.8 <= slope <= 2.2


def _blast_spread(oracle, delta, seeds=(1, 2)):
    prob = inputs.blast(32, mb=16, r0=0.1, magnetized=True)
    spread = 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)
        a = oracle.Mesh.from_problem(prob, ct_delta=delta)
        w = prob.w.copy()
        w[4] *= 1.0 + 1e-15 * rng.uniform(-1.0, 1.0, w[4].shape)
        b = oracle.Mesh(prob.nx, prob.mb, prob.xmin, prob.xmax, prob.gamma, bc=prob.bc, ct_delta=delta)
        b.set_prims(w, prob.b1, prob.b2, prob.b3)
        for _ in range(2):
            dt = a.new_dt(0.3)
            a.step(dt)
            a.new_dt(0.3)
            b.step(dt)
            b.new_dt(0.3)
        spread = max(spread, float(np.max(state_diff(b.get_cons(), a.get_cons()))))
    return spread


def test_smoothing_makes_the_blast_well_conditioned(oracle):
    sharp, smooth = _blast_spread(oracle, 0.0), _blast_spread(oracle, 1e-4)
    print("magnetized blast, 2 cycles, spread under 1e-15 pressure noise: sharp %.2e, delta 1e-4 %.2e" % (sharp, smooth))
    assert sharp >= 1e-6
    assert smooth <= 1e-12


def _direction(x, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(x[0].shape),) + tuple(np.full_like(b, rng.standard_normal()) for b in x[1:])


def _tl_vs_fd(oracle, prob, delta, d, h, riemann=1):
    geom = (prob.nx, prob.mb, prob.xmin, prob.xmax, prob.bc)
    x = oracle.Mesh.from_problem(prob).get_cons()
    dt = oracle.Mesh.from_problem(prob).new_dt(0.3)
    if callable(d):
        d = d(x)
    y, j = oracle.tl_step(geom, dt, x, d, gamma=prob.gamma, riemann=riemann, ct_delta=delta)
    y0 = oracle.step_cons(geom, dt, x, gamma=prob.gamma, riemann=riemann, ct_delta=delta)
    assert all(np.array_equal(a, b) for a, b in zip(y, y0))  # the value part is the plain cycle
    yp = oracle.step_cons(geom, dt, tuple(a + h * t for a, t in zip(x, d)), gamma=prob.gamma, riemann=riemann,
                          ct_delta=delta)
    ym = oracle.step_cons(geom, dt, tuple(a - h * t for a, t in zip(x, d)), gamma=prob.gamma, riemann=riemann,
                          ct_delta=delta)
    return max(float(np.max(np.abs((a - b) / (2 * h) - t))) / (float(np.max(np.abs(t))) + 1e-300)
               for a, b, t in zip(yp, ym, j))


@pytest.mark.parametrize("v0,delta", [((0.7, 0.4, 0.2), 0.3), ((0.0, 0.0, 0.0), 1e-2)])
def test_smoothed_tangent_linear_matches_central_differences(oracle, v0, delta):
    # mass fluxes ~ delta, so every weight sits on the slope of tanh; a tangent that dropped dw/dm misses
    # these differences by 1.6e-5 (advected wave) to 3e-2 (wave at rest)
    prob = inputs.linear_wave(8, mb=4, kind="fast", amp=1e-2, v0=v0)
    for riemann in (1, 0):
        err = _tl_vs_fd(oracle, prob, delta, lambda x: _direction(x, 1), 1e-7, riemann)
        print("smoothed CT (delta %g, v0 %s, riemann %d): tangent-linear vs central differences %.2e"
              % (delta, v0, riemann, err))
        assert err <= 1e-6


def test_smoothing_removes_the_blast_jump(oracle):
    prob = inputs.blast(16, mb=8, r0=0.2, magnetized=True)

    def d(x):
        rng = np.random.default_rng(1)
        return (1e-3 * rng.standard_normal(x[0].shape),) + tuple(np.zeros_like(b) for b in x[1:])

    sharp = [_tl_vs_fd(oracle, prob, 0.0, d, h, 0) for h in (1e-6, 1e-8)]
    smooth = [_tl_vs_fd(oracle, prob, 1e-3, d, h, 0) for h in (1e-6, 1e-8)]
    print("magnetized blast, |FD - TL| / |TL| at h = 1e-6, 1e-8: sharp %s, delta 1e-3 %s" % (sharp, smooth))
    assert sharp[1] >= 50.0 * sharp[0] and sharp[0] >= 1e3  # a jump: central differences grow as 1/h
    # no jump: the difference stays bounded as h falls (what is left is the PLM limiter's kink on the
    # uniform ambient gas, where both one-sided slopes vanish)
    assert smooth[1] <= 1.5 * smooth[0] and smooth[1] <= 10.0
