"""Forcing (a fixed body acceleration; the reading the library takes, the paper defines none) on the GPU,
through the C ABI, against the FP64 oracle:

- driven turbulence (Mach 1, beta 1, seeded solenoidal forcing of rms 2): one VL2 cycle <= 1e-12 and ten
  cycles <= 1e-10 (normalised as the other parity tests), with RK2 and RK3 as well; the mixed form keeps the
  mass and div B at round-off under forcing
- a uniform state under a uniform acceleration: v = v0 + a dt and the pressure unchanged (the closed form
  the oracle is pinned to)
- zero forcing is bitwise the unforced cycle; vl2_set_forcing(NULL) removes the forcing; a mesh created
  without params.forcing refuses it
- the batched form carries each box's forcing: bitwise equal to the per-box path
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_gpu_parity import state_diff

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


INTEGRATORS = {"vl2": (0, 0), "rk2": (2, 2), "rk3": (3, 3)}  # (GPU, oracle) integrator ids


@pytest.mark.parametrize("integrator", sorted(INTEGRATORS))
def test_driven_turbulence_matches_the_oracle(vl2, oracle, integrator):
    gi, oi = INTEGRATORS[integrator]
    prob = inputs.turbulence(n=32, mb=16, seed=31, mach=1.0, beta=1.0)
    a = inputs.forcing_field(32, seed=4004, amp=2.0)
    g = vl2.Mesh.from_problem(prob, forcing=True, integrator=gi)
    g.set_forcing(a)
    o = oracle.Mesh.from_problem(prob, integrator=oi)
    o.set_forcing(a)
    worst = []
    for _ in range(10):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
        worst.append(float(np.max(state_diff(g.get_cons(), o.get_cons()))))
    print("driven turbulence, %s: one cycle %.2e, ten cycles %.2e" % (integrator, worst[0], worst[-1]))
    assert worst[0] <= 1e-12
    assert worst[-1] <= 1e-10
    assert g.floor_count() == 0 and o.floor_count() == 0


def test_uniform_acceleration_closed_form(vl2):
    n = 8
    w = np.empty((5, n, n, n))
    w[0], w[1], w[2], w[3], w[4] = 1.3, 0.3, -0.2, 0.1, 0.7
    b1, b2, b3 = inputs.uniform_faces((n, n, n), (0.4, 0.2, -0.3))
    prob = inputs.Problem("uniform", (n,) * 3, (4,) * 3, (0.0,) * 3, (1.0,) * 3, 5.0 / 3.0, w, b1, b2, b3)
    g = vl2.Mesh.from_problem(prob, forcing=True)
    a0 = np.array([0.5, -1.25, 0.75])
    g.set_forcing(np.ascontiguousarray(np.broadcast_to(a0[:, None, None, None], (3, n, n, n))))
    w0 = g.get_prims()
    dt = 0.02
    g.step(dt)
    w1 = g.get_prims()
    np.testing.assert_allclose(w1[0], w0[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w1[1:4], w0[1:4] + a0[:, None, None, None] * dt, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w1[4], w0[4], rtol=0, atol=1e-14)


def test_zero_and_removed_forcing_and_refusal(vl2):
    prob = inputs.turbulence(n=16, mb=8, seed=32, mach=1.0, beta=1.0)
    a = inputs.forcing_field(16, seed=4005, amp=1.0)
    free = vl2.Mesh.from_problem(prob)
    zero = vl2.Mesh.from_problem(prob, forcing=True)
    zero.set_forcing(np.zeros_like(a))
    removed = vl2.Mesh.from_problem(prob, forcing=True)
    removed.set_forcing(a)
    removed.set_forcing(None)
    for _ in range(3):
        dt = free.new_dt()
        for m in (free, zero, removed):
            m.step(dt)
    ref = free.get_cons()
    for m in (zero, removed):
        assert all(np.array_equal(x, y) for x, y in zip(m.get_cons(), ref))
    with pytest.raises(vl2.VL2Error):
        free.set_forcing(a)


def test_mixed_form_conserves_mass_under_forcing(vl2):
    prob = inputs.turbulence(n=32, mb=16, seed=33, mach=2.0, beta=10.0)
    a = inputs.forcing_field(32, seed=4006, amp=2.0)
    g = vl2.Mesh.from_problem(prob, forcing=True, precision=vl2.MIXED)
    g.set_forcing(a)
    m0 = g.totals()[0]
    for _ in range(10):
        g.step(g.new_dt())
    assert abs(g.totals()[0] - m0) <= 1e-13 * m0
    assert g.divb_norm() <= 1e-13


def test_batch_carries_each_box_forcing(vl2):
    sizes = (16, 32, 16)
    probs = [inputs.turbulence(n=s, mb=s, seed=40 + q, mach=1.0, beta=1.0) for q, s in enumerate(sizes)]
    accs = [inputs.forcing_field(s, seed=50 + q, amp=1.5) for q, s in enumerate(sizes)]
    single = [vl2.Mesh.from_problem(p, forcing=True) for p in probs]
    batched = [vl2.Mesh.from_problem(p, forcing=True) for p in probs]
    for m, a in zip(single + batched, accs + accs):
        m.set_forcing(a)
    batch = vl2.Batch(batched)
    for _ in range(4):
        dts = [m.new_dt() for m in single]
        for m, dt in zip(single, dts):
            m.step(dt)
        batch.step(np.array(dts))
    for s_, b_ in zip(single, batched):
        assert all(np.array_equal(x, y) for x, y in zip(s_.get_cons(), b_.get_cons()))
