"""GPU parity of the RK1 / RK2 / RK3 integrators (Sec. 3.2.3, eq. rk-2s with the listed coefficients)
against the FP64 oracle, with the same tolerances as the VL2 parity tests: <= 1e-12 after one cycle,
<= 1e-9 after 100 cycles of a smooth problem."""
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


def pair(vl2, oracle, prob, integrator, riemann=1):
    g = vl2.Mesh.from_problem(prob, integrator=integrator, riemann=riemann)
    o = oracle.Mesh.from_problem(prob, integrator=integrator, riemann=riemann)
    return g, o


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("integrator", [1, 2, 3])
def test_rk_one_cycle(vl2, oracle, integrator, riemann):
    prob = inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=9)
    g, o = pair(vl2, oracle, prob, integrator, riemann)
    dt = o.new_dt(0.3)
    assert g.new_dt() == pytest.approx(dt, rel=1e-13)
    g.step(dt)
    o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    print("RK%d riemann %d, one cycle: max normalised difference %.2e" % (integrator, riemann, np.max(d)))
    assert np.max(d) <= 1e-12, d
    assert g.floor_count() == 0


@pytest.mark.parametrize("integrator", [2, 3])
def test_rk_hundred_cycles_smooth(vl2, oracle, integrator):
    prob = inputs.linear_wave(16, mb=8, kind="fast", amp=1e-2, v0=(0.3, -0.2, 0.1))
    g, o = pair(vl2, oracle, prob, integrator)
    for _ in range(100):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    print("RK%d, 100 cycles, smooth wave: max normalised difference %.2e" % (integrator, np.max(d)))
    assert np.max(d) <= 1e-9, d


def test_rk_conserves_and_keeps_divb(vl2):
    prob = inputs.orszag_tang(n=32, mb=16, seed=4)
    for integrator in (2, 3):
        for precision in (vl2.FP64, vl2.MIXED):
            g = vl2.Mesh.from_problem(prob, integrator=integrator, precision=precision)
            t0 = g.totals()
            for _ in range(10):
                g.step(g.new_dt())
            t = g.totals()
            assert abs(t[0] - t0[0]) <= 1e-13 * 10 * abs(t0[0])
            assert np.all(np.abs(t[1:5] - t0[1:5]) <= 1e-13 * 10 * abs(t0[4]))
            assert g.divb_norm() <= 1e-13


def test_rk_meshes_are_refused_by_the_vl2_only_paths(vl2):
    prob = inputs.linear_wave(8, mb=8, kind="fast", amp=1e-3)
    with pytest.raises(vl2.VL2Error) as e:
        vl2.Mesh.from_problem(prob, integrator=2, adjoint=True)
    assert e.value.status == vl2.VL2_E_ARG
    g = vl2.Mesh.from_problem(prob, integrator=2)
    with pytest.raises(vl2.VL2Error) as e:
        vl2.Batch([g])
    assert e.value.status == vl2.VL2_E_ARG
