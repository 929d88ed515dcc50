"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

- 256^3 vortex in 512 MeshBlocks of 32^3, FP64 VL2 + PLM + HLLD + CT: two cycles on the GPU against two
  cycles of the oracle (FP64, all host cores), every output element compared after each (<= 1e-12,
  normalised as in the other parity tests); and the vortex at 64^3 in 8 MeshBlocks of 32^3 over 100 CFL
  cycles, each side taking its own dt (<= 1e-9).
- 512^3 decaying turbulence in 4096 MeshBlocks of 32^3, mixed precision: the oracle does not fit this
  size in a test, so what holds at any size is checked: conservation of the totals and div B at FP64
  round-off over two cycles.
- The later rows at 256^3 in 512 MeshBlocks, one cycle against the oracle (<= 1e-12): VL2 + PPM on the
  vortex (three ghost layers), the vortex carrying two passive scalars, and the hydrodynamic blast wave
  (r0 = 0.01, 56 cells), whose uniform regions run the solvers' equal-state branch; and the options on
  the vortex: PLM on characteristic variables, HLLE with Einfeldt's speeds, the smoothed CT weight.
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_gpu_parity import state_diff

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def vl2():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06651_gb300 import build, vl2 as mod

    build.build()
    mod.load()
    return mod


def test_orszag_tang_256cubed_two_cycles_match_oracle(vl2, oracle):
    prob = inputs.orszag_tang(n=256, mb=32, seed=2005)
    g = vl2.Mesh.from_problem(prob)
    o = oracle.Mesh.from_problem(prob)
    for cycle in range(2):
        dt = o.new_dt(0.3)
        assert g.new_dt() == pytest.approx(dt, rel=1e-13)
        g.step(dt)
        o.step(dt)
        d = state_diff(g.get_cons(), o.get_cons())
        print("256^3, 512 blocks, cycle %d: max normalised difference %.2e" % (cycle + 1, np.max(d)))
        assert np.max(d) <= 1e-12, d
    assert g.floor_count() == 0 and o.floor_count() == 0
    assert g.divb_norm() <= 1e-13


def test_orszag_tang_64cubed_hundred_cycles_match_oracle(vl2, oracle):
    """The vortex at 64^3 in 8 MeshBlocks of 32^3 (the benchmark's block size), 100 CFL cycles: each side
    forms its own dt, so the rounding differences of every cycle feed the next one."""
    prob = inputs.orszag_tang(n=64, mb=32, seed=2005)
    g = vl2.Mesh.from_problem(prob)
    o = oracle.Mesh.from_problem(prob)
    for _ in range(100):
        g.step(g.new_dt())
        o.step(o.new_dt(0.3))
    d = state_diff(g.get_cons(), o.get_cons())
    print("64^3, 8 blocks, 100 cycles: max normalised difference %.2e" % np.max(d))
    assert np.max(d) <= 1e-9, d
    assert g.floor_count() == 0 and o.floor_count() == 0


def test_mixed_512cubed_conserves_and_keeps_divb(vl2):
    import torch

    prob = inputs.turbulence(n=512, mb=32, seed=3003, mach=2.0, beta=10.0)
    g = vl2.Mesh.from_problem(prob, precision=vl2.MIXED)
    t0 = g.totals()
    for _ in range(2):
        g.step(g.new_dt())
    t = g.totals()
    print("512^3 mixed, 2 cycles: d(mass)/mass %.2e, div B %.2e" % (abs(t[0] - t0[0]) / t0[0], g.divb_norm()))
    # the totals are FP64 sums over 1.3e8 cells: their own round-off (~1e-13 relative) sets the bound
    assert abs(t[0] - t0[0]) <= 2e-12 * abs(t0[0])
    assert np.all(np.abs(t[1:5] - t0[1:5]) <= 2e-12 * abs(t0[4]))
    assert g.divb_norm() <= 1e-13
    g.close()
    del g
    torch.cuda.empty_cache()


def _one_cycle(vl2, oracle, prob, label, scalars=None, **kw):
    g = vl2.Mesh.from_problem(prob, **kw)
    o = oracle.Mesh.from_problem(prob, **kw)
    if scalars is not None:
        g.set_scalars(scalars)
        o.set_scalars(scalars)
    dt = o.new_dt(0.3)
    assert g.new_dt() == pytest.approx(dt, rel=1e-13)
    g.step(dt)
    o.step(dt)
    d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
    ds = 0.0
    if scalars is not None:
        os_ = o.get_scalars()
        ds = float(np.max(np.abs(g.get_scalars() - os_))) / float(np.max(np.abs(os_)))
    print("%s: max normalised difference %.2e (scalars %.2e)" % (label, d, ds))
    assert d <= 1e-12 and ds <= 1e-12
    assert g.floor_count() == 0 and g.divb_norm() <= 1e-13
    g.close()


def test_ppm_256cubed_one_cycle_matches_oracle(vl2, oracle):
    prob = inputs.orszag_tang(n=256, mb=32, seed=2005)
    _one_cycle(vl2, oracle, prob, "256^3 VL2 + PPM, one cycle", recon=vl2.PPM)


def test_scalars_256cubed_one_cycle_match_oracle(vl2, oracle):
    prob = inputs.orszag_tang(n=256, mb=32, seed=2005)
    rng = np.random.default_rng(4004)
    c = rng.uniform(0.0, 1.0, size=(2, 256, 256, 256))
    _one_cycle(vl2, oracle, prob, "256^3 with 2 passive scalars, one cycle", scalars=c, nscalars=2)


def test_hydro_blast_256cubed_one_cycle_matches_oracle(vl2, oracle):
    prob = inputs.blast(n=256, mb=32, r0=0.01, magnetized=False)
    _one_cycle(vl2, oracle, prob, "256^3 hydrodynamic blast, one cycle")


@pytest.mark.parametrize("option", ["plm_char", "hlle_roe", "ct_smooth"])
def test_options_256cubed_one_cycle_match_oracle(vl2, oracle, option):
    prob = inputs.orszag_tang(n=256, mb=32, seed=2005)
    kw = {"plm_char": dict(recon=vl2.PLM_CHAR), "hlle_roe": dict(riemann=vl2.HLLE_ROE),
          "ct_smooth": dict(ct_delta=1e-4)}[option]
    _one_cycle(vl2, oracle, prob, "256^3 VL2, %s, one cycle" % option, **kw)
