"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances.  FP64 results are compared per conserved variable with the maximum absolute difference
divided by a scale fixed by the state: rho by max rho, E by max E, each momentum component by
max sqrt(2 rho E) and each field component by max sqrt(2 E) (upper bounds of |M| and |B|).  Bounds:
<= 1e-12 after one step, <= 1e-9 after 100 steps of a smooth problem.  Fluxes of one stage are
compared against the largest oracle flux of their sweep (the normal-momentum flux, which carries the
total pressure: every flux component is formed from terms of that size), and corner EMFs against the
largest oracle EMF of their family, at 1e-12.  Rounding differs only by FMA contraction and reciprocal-multiply
forms, each a few units in the last place per operation.
"""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vl2():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06651_gb300 import build, vl2 as mod

    build.build()
    mod.load()
    return mod


def scales(u, b1, b2, b3):
    rho, E = u[0], u[4]
    sm = float(np.max(np.sqrt(2.0 * np.abs(rho * E))))
    sb = float(np.max(np.sqrt(2.0 * np.abs(E))))
    return [float(np.max(np.abs(rho))), sm, sm, sm, float(np.max(np.abs(E)))], sb


def state_diff(gpu, orc):
    """max normalised difference per variable: rho, M1, M2, M3, E, B1, B2, B3."""
    su, sb = scales(*orc)
    d = [float(np.max(np.abs(gpu[0][v] - orc[0][v]))) / su[v] for v in range(5)]
    d += [float(np.max(np.abs(gpu[1 + c] - orc[1 + c]))) / sb for c in range(3)]
    return np.array(d)


def pair(vl2, oracle, prob, **kw):
    g = vl2.Mesh.from_problem(prob, **kw)
    o = oracle.Mesh.from_problem(prob, riemann=kw.get("riemann", 1))
    return g, o


CASES = {
    "ot32_8blk": lambda: inputs.orszag_tang(n=32, mb=16, seed=2005),
    "ot_ragged": lambda: inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=9),
    "wave_1blk": lambda: inputs.linear_wave(16, kind="fast", amp=1e-3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_set_prims_get_cons_and_prims(vl2, oracle, case):
    prob = CASES[case]()
    g, o = pair(vl2, oracle, prob)
    gc, oc = g.get_cons(), o.get_cons()
    for a, b in zip(gc[1:], oc[1:]):
        np.testing.assert_array_equal(a, b)  # face fields are copied, bit for bit
    assert np.max(state_diff(gc, oc)) <= 1e-15
    gw, ow = g.get_prims(), o.get_prims()
    np.testing.assert_allclose(gw, ow, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("recon", [0, 1])
@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("case", sorted(CASES))
def test_stage_fluxes_and_emfs(vl2, oracle, case, recon, riemann):
    prob = CASES[case]()
    g, o = pair(vl2, oracle, prob, riemann=riemann)
    gf, of = g.debug_fluxes(recon), o.debug_fluxes(recon)
    for d in range(3):
        scale = float(np.max(np.abs(of[d])))
        for c in range(7):
            err = float(np.max(np.abs(gf[d][c] - of[d][c]))) / scale
            assert err <= 1e-12, (d, c, err)
    ge, oe = g.debug_emfs(recon), o.debug_emfs(recon)
    for e in range(3):
        scale = float(np.max(np.abs(oe[e]))) + 1e-12
        err = float(np.max(np.abs(ge[e] - oe[e]))) / scale
        assert err <= 1e-12, (e, err)


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("case", sorted(CASES))
def test_one_step(vl2, oracle, case, riemann):
    prob = CASES[case]()
    g, o = pair(vl2, oracle, prob, riemann=riemann)
    dtg, dto = g.new_dt(), o.new_dt(0.3)
    assert dtg == pytest.approx(dto, rel=1e-13)
    g.step(dto)
    o.step(dto)
    d = state_diff(g.get_cons(), o.get_cons())
    print("one cycle, %s, riemann %d: max normalised difference %.2e" % (case, riemann, np.max(d)))
    assert np.max(d) <= 1e-12, d
    assert g.new_dt() == pytest.approx(o.new_dt(0.3), rel=1e-12)
    assert g.floor_count() == 0


def test_hundred_steps_smooth(vl2, oracle):
    """Smooth nonlinear wave (amplitude 1e-2, advected by a background flow): 100 steps, <= 1e-9."""
    prob = inputs.linear_wave(16, mb=8, kind="fast", amp=1e-2, v0=(0.3, -0.2, 0.1))
    g, o = pair(vl2, oracle, prob)
    for _ in range(100):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    print("100 cycles, smooth wave: max normalised difference %.2e" % np.max(d))
    assert np.max(d) <= 1e-9, d


def test_hundred_steps_orszag_tang_small(vl2, oracle):
    """The vortex itself at 24^3 (8 blocks), 100 CFL steps on each side independently (each path
    takes its own dt), compared at the end: FP64 rounding differences stay far below the scheme's
    truncation error."""
    prob = inputs.orszag_tang(n=24, mb=12, seed=2005)
    g, o = pair(vl2, oracle, prob)
    for _ in range(100):
        g.step(g.new_dt())
        o.step(o.new_dt(0.3))
    d = state_diff(g.get_cons(), o.get_cons())
    print("100 cycles, vortex 24^3: max normalised difference %.2e" % np.max(d))
    assert np.max(d) <= 1e-9, d


def test_diagnostics(vl2, oracle):
    prob = inputs.orszag_tang(n=32, mb=16, seed=5)
    g, o = pair(vl2, oracle, prob)
    for _ in range(3):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    assert g.divb_norm() <= 1e-13
    tg, to = g.totals(), o.totals()
    su = np.array([abs(to[0]), abs(to[4]), abs(to[4]), abs(to[4]), abs(to[4]), 1, 1, 1])
    assert np.all(np.abs(tg - to) <= 1e-13 * su), (tg, to)


def test_conservation_on_gpu(vl2):
    prob = inputs.orszag_tang(n=32, mb=8, seed=4)
    g = vl2.Mesh.from_problem(prob)
    t0 = g.totals()
    for s in range(20):
        g.step(g.new_dt())
    t = g.totals()
    assert abs(t[0] - t0[0]) <= 1e-13 * 20 * abs(t0[0])
    assert np.all(np.abs(t[1:4] - t0[1:4]) <= 1e-13 * 20 * abs(t0[4]))
    assert abs(t[4] - t0[4]) <= 1e-13 * 20 * abs(t0[4])
    assert g.divb_norm() <= 1e-13


def test_block_decomposition_bitwise_on_gpu(vl2):
    prob = inputs.orszag_tang(n=32, seed=2005)
    outs = []
    for mb in [(32, 32, 32), (16, 16, 16), (8, 16, 32)]:
        g = vl2.Mesh.from_problem(prob, mb=mb)
        for _ in range(3):
            g.step(0.004)
        outs.append(g.get_cons())
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def test_outflow_boundaries(vl2, oracle):
    """Shock tube along y with outflow faces in y: parity through the outflow ghost fill."""
    prob = inputs.shock_tube(n=64, axis=1, b_left=(0.7, 0.5, 0.0), b_right=(0.7, -0.5, 0.2), gamma=5.0 / 3.0)
    prob.bc = (0, 0, 1, 1, 0, 0)
    prob.mb = (1, 16, 1)
    g, o = pair(vl2, oracle, prob)
    for _ in range(30):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    assert np.max(d) <= 1e-11, d


def test_device_buffers_round_trip(vl2, oracle):
    import torch

    prob = inputs.orszag_tang(n=16, mb=8, seed=1)
    g = vl2.Mesh(prob.nx, prob.mb)
    dev = [torch.from_numpy(a).cuda() for a in (prob.w, prob.b1, prob.b2, prob.b3)]
    g.set_prims(*dev)
    out = (torch.empty((5,) + g.shape, dtype=torch.float64, device="cuda"),
           *[torch.empty(s, dtype=torch.float64, device="cuda") for s in g.face_shapes()])
    g.get_cons(out)
    torch.cuda.synchronize()
    o = oracle.Mesh.from_problem(prob)
    oc = o.get_cons()
    assert np.max(state_diff([x.cpu().numpy() for x in out], oc)) <= 1e-15


def test_error_statuses(vl2):
    prob = inputs.orszag_tang(n=16, mb=8, seed=1)
    g = vl2.Mesh(prob.nx, prob.mb)
    with pytest.raises(vl2.VL2Error) as e:
        g.step(0.01)
    assert e.value.status == vl2.VL2_E_STATE
    bad = prob.b1.copy()
    bad[0, 0, -1] += 1.0  # periodic duplicate face differs
    with pytest.raises(vl2.VL2Error) as e:
        g.set_prims(prob.w, bad, prob.b2, prob.b3)
    assert e.value.status == vl2.VL2_E_ARG
    g.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
    for dt in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(vl2.VL2Error) as e:
            g.step(dt)
        assert e.value.status == vl2.VL2_E_ARG


def test_floor_reported_and_matches_oracle(vl2, oracle):
    prob = inputs.orszag_tang(n=16, mb=8, seed=1)
    w = prob.w.copy()
    w[4, 3, 4, 5] = -0.5  # a negative pressure: the pressure floor fires on set-up
    prob.w = w
    g = vl2.Mesh.from_problem(prob)
    o = oracle.Mesh.from_problem(prob)
    with pytest.raises(vl2.VL2Error) as e:
        g.new_dt()
    assert e.value.status == vl2.VL2_E_NONPHYS
    o.new_dt(0.3)
    assert g.floor_count() == o.floor_count() >= 1
    np.testing.assert_allclose(g.get_prims()[4], o.get_prims()[4], rtol=1e-14, atol=1e-14)


def test_pinned_host_buffers_match_pageable(vl2):
    """Page-locked host buffers (torch pinned tensors) in and out give bitwise the state of pageable numpy
    buffers."""
    import torch

    prob = inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=9)
    a = vl2.Mesh.from_problem(prob)
    b = vl2.Mesh(prob.nx, prob.mb)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    b.set_prims(*(pin(x) for x in (prob.w, prob.b1, prob.b2, prob.b3)))
    for _ in range(2):
        dt = a.new_dt()
        assert b.new_dt() == dt
        a.step(dt)
        b.step(dt)
    outs = (torch.zeros((5,) + b.shape, dtype=torch.float64).pin_memory(),
            *[torch.zeros(s, dtype=torch.float64).pin_memory() for s in b.face_shapes()])
    b.get_cons(outs)
    for x, y in zip(a.get_cons(), outs):
        np.testing.assert_array_equal(x, y.numpy())
