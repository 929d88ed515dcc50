"""Passive scalars (eq. passive_scalars) on the GPU, through the C ABI, against the FP64 oracle.

- one cycle of the state and the scalar masses equals the oracle's to rounding (VL2 + PLM, RK3 + PPM, RK1)
- a scalar with C = 1 stays bitwise equal to the density (its flux is the mass flux, its update the
  density's arithmetic)
- 100 smooth cycles stay within 1e-9; scalar mass is conserved; scalars leave the MHD state bitwise
  unchanged; the batch and the adjoint refuse meshes with scalars
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


def concentrations(prob, seed, n=2):
    rng = np.random.default_rng(seed)
    nz, ny, nx = prob.w.shape[1:]
    z, y, x = np.meshgrid(*[(np.arange(m) + 0.5) / m for m in (nz, ny, nx)], indexing="ij")
    c = np.empty((n, nz, ny, nx))
    c[0] = 0.5 + 0.4 * np.sin(2 * np.pi * (x + 2 * y) + rng.uniform(0, 2 * np.pi)) * np.cos(2 * np.pi * z + 0.3)
    c[1] = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    return c


CONFIGS = [("VL2", "PLM", 1), ("RK3", "PPM", 0), ("RK1", "PLM", 1), ("VL2", "PPM", 1)]


@pytest.mark.parametrize("integrator,recon,riemann", CONFIGS)
def test_scalars_one_cycle(vl2, oracle, integrator, recon, riemann):
    prob = inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=41)
    kw = dict(riemann=riemann, nscalars=2)
    g = vl2.Mesh.from_problem(prob, integrator=getattr(vl2, integrator), recon=getattr(vl2, recon), **kw)
    o = oracle.Mesh.from_problem(prob, integrator=getattr(oracle, integrator), recon=getattr(oracle, recon), **kw)
    c = concentrations(prob, 3)
    g.set_scalars(c)
    o.set_scalars(c)
    np.testing.assert_array_equal(g.get_scalars(), o.get_scalars())
    dt = o.new_dt(0.3)
    g.step(dt)
    o.step(dt)
    d = state_diff(g.get_cons(), o.get_cons())
    gs, os_ = g.get_scalars(), o.get_scalars()
    ds = float(np.max(np.abs(gs - os_))) / float(np.max(np.abs(os_)))
    print("scalars, one %s + %s cycle, riemann %d: state %.2e, scalars %.2e" % (integrator, recon, riemann,
                                                                             np.max(d), ds))
    assert np.max(d) <= 1e-12
    assert ds <= 1e-12


@pytest.mark.parametrize("integrator,recon,riemann", CONFIGS)
def test_unit_scalar_is_the_density(vl2, integrator, recon, riemann):
    prob = inputs.orszag_tang(n=(16, 12, 8), mb=(8, 6, 4), seed=31)
    g = vl2.Mesh.from_problem(prob, riemann=riemann, integrator=getattr(vl2, integrator),
                              recon=getattr(vl2, recon), nscalars=2)
    c = concentrations(prob, 1)
    c[0] = 1.0
    g.set_scalars(c)
    for _ in range(5):
        g.step(g.new_dt())
    np.testing.assert_array_equal(g.get_scalars()[0], g.get_cons()[0][0])


def test_scalars_hundred_smooth_cycles(vl2, oracle):
    prob = inputs.linear_wave(16, mb=8, kind="fast", amp=1e-2, v0=(0.3, -0.2, 0.1), phase=0.37)
    g = vl2.Mesh.from_problem(prob, nscalars=2)
    o = oracle.Mesh.from_problem(prob, nscalars=2)
    c = concentrations(prob, 5)
    c[1] = 0.5 + 0.3 * np.cos(2 * np.pi * np.arange(16) / 16)[None, None, :] * np.ones((16, 16, 16))
    g.set_scalars(c)
    o.set_scalars(c)
    for _ in range(100):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    gs, os_ = g.get_scalars(), o.get_scalars()
    ds = float(np.max(np.abs(gs - os_))) / float(np.max(np.abs(os_)))
    print("scalars, 100 smooth cycles: %.2e" % ds)
    assert ds <= 1e-9


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_scalar_mass_conserved_and_state_untouched(vl2, precision):
    prob = inputs.orszag_tang(n=32, mb=16, seed=2005)
    a = vl2.Mesh.from_problem(prob, precision=getattr(vl2, precision), nscalars=3)
    b = vl2.Mesh.from_problem(prob, precision=getattr(vl2, precision))
    c = np.concatenate([concentrations(prob, 7), np.full((1, 32, 32, 32), 0.25)])
    a.set_scalars(c)
    s0 = a.get_scalars().sum(axis=(1, 2, 3))
    for _ in range(10):
        dt = a.new_dt()
        assert b.new_dt() == dt
        a.step(dt)
        b.step(dt)
    s1 = a.get_scalars().sum(axis=(1, 2, 3))
    np.testing.assert_allclose(s1, s0, rtol=1e-13)
    for x, y in zip(a.get_cons(), b.get_cons()):
        np.testing.assert_array_equal(x, y)


def test_scalar_refusals(vl2):
    prob = inputs.orszag_tang(n=16, mb=8, seed=1)
    m = vl2.Mesh(prob.nx, prob.mb, nscalars=1)
    with pytest.raises(vl2.VL2Error):  # state not set yet
        m.set_scalars(np.zeros((1, 16, 16, 16)))
    plain = vl2.Mesh.from_problem(prob)
    with pytest.raises(vl2.VL2Error):  # no scalars on this mesh
        plain.set_scalars(np.zeros((1, 16, 16, 16)))
    with pytest.raises(vl2.VL2Error):
        vl2.Mesh.from_problem(prob, adjoint=True, nscalars=1)
    with pytest.raises(vl2.VL2Error):
        vl2.Mesh.from_problem(prob, nscalars=17)
    with pytest.raises(vl2.VL2Error):
        vl2.Batch([vl2.Mesh.from_problem(prob, nscalars=1)])
