"""Mixed-precision form (FP32 reconstruction, Riemann fluxes and CT EMFs; FP64 state, cons->prim and
accumulation) against the FP64 oracle.

The error of the mixed form against the FP64 oracle is a result to state, not a rounding-level parity:
bounds below are set a decade above the observed errors and the tests print the observed values.
What the FP64 accumulation guarantees exactly is checked at FP64 round-off: conservation of the totals
(face fluxes are shared by the two cells they separate and differenced in FP64) and div B (the CT curl
of any edge values is divergence free).
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


def rel_err_rho_e(gpu, orc):
    """max relative error of rho and of E, cell by cell."""
    return (float(np.max(np.abs(gpu[0][0] - orc[0][0]) / np.abs(orc[0][0]))),
            float(np.max(np.abs(gpu[0][4] - orc[0][4]) / np.abs(orc[0][4]))))


def test_mixed_one_step(vl2, oracle):
    prob = inputs.orszag_tang(n=32, mb=16, seed=2005)
    g = vl2.Mesh.from_problem(prob, precision=vl2.MIXED)
    o = oracle.Mesh.from_problem(prob)
    dt = o.new_dt(0.3)
    assert g.new_dt() == pytest.approx(dt, rel=1e-13)  # dt comes from the FP64 cons->prim
    g.step(dt)
    o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    print("mixed one-step normalised differences:", d)
    assert np.max(d) <= 1e-6


def test_mixed_turbulence_50_steps(vl2, oracle):
    """Decaying turbulence (Mach 2, beta 10) at 32^3: 50 steps, each path with its own CFL dt."""
    prob = inputs.turbulence(n=32, mb=16, seed=3003, mach=2.0, beta=10.0)
    g = vl2.Mesh.from_problem(prob, precision=vl2.MIXED)
    o = oracle.Mesh.from_problem(prob)
    for _ in range(50):
        g.step(g.new_dt())
        o.step(o.new_dt(0.3))
    er, ee = rel_err_rho_e(g.get_cons(), o.get_cons())
    print("mixed vs FP64 oracle after 50 steps: max rel rho %.3e, max rel E %.3e" % (er, ee))
    assert er <= 1e-3 and ee <= 1e-3
    assert g.floor_count() == 0


def test_mixed_conserves_and_keeps_divb_at_fp64_roundoff(vl2):
    prob = inputs.orszag_tang(n=32, mb=8, seed=4)
    g = vl2.Mesh.from_problem(prob, precision=vl2.MIXED)
    t0 = g.totals()
    for _ in range(20):
        g.step(g.new_dt())
    t = g.totals()
    assert abs(t[0] - t0[0]) <= 1e-13 * 20 * abs(t0[0])
    assert np.all(np.abs(t[1:5] - t0[1:5]) <= 1e-13 * 20 * abs(t0[4]))
    assert g.divb_norm() <= 1e-13


def test_mixed_fluxes_match_fp64_fluxes_to_fp32_rounding(vl2, oracle):
    prob = inputs.orszag_tang(n=16, mb=8, seed=3)
    g = vl2.Mesh.from_problem(prob, precision=vl2.MIXED)
    o = oracle.Mesh.from_problem(prob)
    for recon in (0, 1):
        gf, of = g.debug_fluxes(recon), o.debug_fluxes(recon)
        for d in range(3):
            scale = float(np.max(np.abs(of[d])))
            err = float(np.max(np.abs(gf[d] - of[d]))) / scale
            assert err <= 1e-5, (recon, d, err)


def test_mixed_linear_wave_error_floor(vl2, oracle):
    """A linear wave of amplitude 1e-3 at 32^3 for one period: the mixed form's L1 error stays within
    a few times the FP64 error (FP32 rounding sits below the truncation error at this amplitude)."""
    from test_oracle_mesh import rms_l1_error

    prob = inputs.linear_wave(32, mb=16, kind="alfven", amp=1e-3)
    errs = {}
    for name, kw in (("fp64", {}), ("mixed", {"precision": vl2.MIXED})):
        g = vl2.Mesh.from_problem(prob, **kw)
        ref = g.get_cons()
        g.run(prob.meta["period"])
        errs[name] = rms_l1_error(g.get_cons(), ref)
    print("linear Alfven wave, A = 1e-3, 32^3: L1 error FP64 %.4e, mixed %.4e" % (errs["fp64"], errs["mixed"]))
    assert errs["mixed"] <= 3.0 * errs["fp64"]
