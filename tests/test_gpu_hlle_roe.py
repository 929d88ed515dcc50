"""HLLE with Einfeldt's Roe-averaged outer speeds (VL2_HLLE_ROE) on the GPU, through the C ABI, against
the FP64 oracle.

- stage fluxes and corner EMFs (donor cell, PLM, characteristic PLM) equal the oracle's to rounding
- one VL2 / RK3 cycle equals the oracle's to 1e-12 (or 4x the oracle's own spread); the Brio-Wu tube
  over ten cycles; 100 smooth cycles within 1e-9
- the option changes the fluxes (Einfeldt's speeds differ from the states' own); the mixed form
  conserves; the adjoint refuses it
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_gpu_char import CASES, brio_wu
from test_gpu_parity import state_diff
from test_gpu_ppm import oracle_spread

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


@pytest.mark.parametrize("recon", ["DC", "PLM", "PLM_CHAR"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_hlle_roe_stage_fluxes_and_emfs(vl2, oracle, case, recon):
    prob = CASES[case]()
    g = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE)
    o = oracle.Mesh.from_problem(prob, riemann=oracle.HLLE_ROE)
    rg, ro = getattr(vl2, recon), getattr(oracle, recon)
    gf, of = g.debug_fluxes(rg), o.debug_fluxes(ro)
    worst = 0.0
    for d in range(3):
        scale = float(np.max(np.abs(of[d])))
        for c in range(7):
            err = float(np.max(np.abs(gf[d][c] - of[d][c]))) / scale
            worst = max(worst, err)
            assert err <= 1e-12, (d, c, err)
    ge, oe = g.debug_emfs(rg), o.debug_emfs(ro)
    for e in range(3):
        scale = float(np.max(np.abs(oe[e]))) + 1e-12
        err = float(np.max(np.abs(ge[e] - oe[e]))) / scale
        worst = max(worst, err)
        assert err <= 1e-12, (e, err)
    davis = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE).debug_fluxes(rg)
    moved = max(float(np.max(np.abs(davis[d] - gf[d]))) for d in range(3))
    print("Einfeldt HLLE stage terms, %s, %s: max normalised difference %.2e (differs from HLLE by %.2e)"
          % (case, recon, worst, moved))
    assert moved > 1e-10  # second order in the amplitude on the 1e-3 wave, 1e-5 .. 1e-2 on the vortex


@pytest.mark.parametrize("integrator", ["VL2", "RK3"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_hlle_roe_one_cycle(vl2, oracle, case, integrator):
    prob = CASES[case]()
    g = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE, integrator=getattr(vl2, integrator))
    okw = dict(riemann=oracle.HLLE_ROE, integrator=getattr(oracle, integrator))
    o = oracle.Mesh.from_problem(prob, **okw)
    dt = o.new_dt(0.3)
    g.step(dt)
    o.step(dt)
    d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
    spread = oracle_spread(oracle, prob, **okw)
    print("Einfeldt HLLE, one %s cycle, %s: GPU vs oracle %.2e, oracle spread %.2e" % (integrator, case, d, spread))
    assert d <= max(1e-12, 4.0 * spread)


def test_hlle_roe_brio_wu_and_smooth(vl2, oracle):
    prob = brio_wu()
    g = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE, mb=(16, 1, 1))
    o = oracle.Mesh.from_problem(prob, riemann=oracle.HLLE_ROE, mb=(16, 1, 1))
    for _ in range(10):
        dt = o.new_dt(0.4)
        g.step(dt)
        o.step(dt)
    d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
    prob = inputs.linear_wave(16, mb=8, kind="fast", amp=1e-2, v0=(0.3, -0.2, 0.1), phase=0.37)
    g2 = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE)
    o2 = oracle.Mesh.from_problem(prob, riemann=oracle.HLLE_ROE)
    for _ in range(100):
        dt = o2.new_dt(0.3)
        g2.step(dt)
        o2.step(dt)
    d2 = float(np.max(state_diff(g2.get_cons(), o2.get_cons())))
    print("Einfeldt HLLE: Brio-Wu 10 cycles %.2e, 100 smooth cycles %.2e" % (d, d2))
    assert d <= 1e-12
    assert d2 <= 1e-9


def test_hlle_roe_mixed_and_refusals(vl2):
    prob = inputs.orszag_tang(n=32, mb=16, seed=2005)
    m = vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE, precision=vl2.MIXED)
    t0 = m.totals()
    for _ in range(10):
        m.step(m.new_dt())
    assert abs(m.totals()[0] - t0[0]) <= 1e-13 * abs(t0[0])
    assert m.divb_norm() <= 1e-13
    with pytest.raises(vl2.VL2Error):
        vl2.Mesh.from_problem(prob, riemann=vl2.HLLE_ROE, adjoint=True)
    with pytest.raises(vl2.VL2Error):
        vl2.Mesh.from_problem(prob, riemann=3)
