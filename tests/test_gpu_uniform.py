"""Regions at rest or in uniform motion on the GPU.

- The Riemann flux of two bitwise-equal states is the physical flux of that state: the GPU forms it
  directly, where the oracle runs the full solver, so both are checked against the physical flux.
- The CFL maximum is screened in single precision and then taken in FP64 over the cells near the CTA's
  maximum; a uniform state with a few raised cells makes every cell such a candidate.
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, MB = (24, 20, 16), (8, 10, 8)  # ragged: 3 x 2 x 2 MeshBlocks
W0 = (1.3, 0.4, -0.2, 0.1, 0.7)  # rho, vx, vy, vz, p
B0 = (0.9, -0.5, 0.3)
G = 5.0 / 3.0


@pytest.fixture(scope="module")
def vl2():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06651_gb300 import build, vl2 as mod

    build.build()
    mod.load()
    return mod


def uniform_prims():
    w = np.empty((5, NX[2], NX[1], NX[0]))
    for v in range(5):
        w[v] = W0[v]
    return w


def sweep_state(d):
    """(rho, v_n, v_t1, v_t2, p, b_t1, b_t2) and b_n of the uniform state in the frame of direction d."""
    v, b = W0[1:4], B0
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    return np.array([W0[0], v[d], v[t1], v[t2], W0[4], b[t1], b[t2]]), b[d]


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("recon", [0, 1])
def test_uniform_state_fluxes_are_the_physical_flux(vl2, oracle, riemann, recon):
    b1, b2, b3 = inputs.uniform_faces(NX, B0)
    g = vl2.Mesh(NX, MB, riemann=riemann)
    g.set_prims(uniform_prims(), b1, b2, b3)
    o = oracle.Mesh(NX, MB, riemann=riemann)
    o.set_prims(uniform_prims(), b1, b2, b3)
    fg, fo = g.debug_fluxes(recon), o.debug_fluxes(recon)
    for d in range(3):
        w, bn = sweep_state(d)
        _, pf = oracle.physical_flux(w, bn, G)
        scale = np.max(np.abs(pf))
        for n in range(7):
            # every face carries the physical flux: one value, within rounding of the oracle's formula
            assert np.ptp(fg[d][n]) == 0.0
            assert abs(fg[d][n].flat[0] - pf[n]) <= 2e-15 * scale, (d, n)
            # the oracle's full solver on the same faces agrees to its own rounding
            assert np.max(np.abs(fg[d][n] - fo[d][n])) <= 1e-13 * scale, (d, n)
    # the stage's EMFs are -(v x B), uniform
    eg = g.debug_emfs(recon)
    v, b = W0[1:4], B0
    emf = -np.cross(v, b)
    for e in range(3):
        assert np.max(np.abs(eg[e] - emf[e])) <= 1e-15


@pytest.mark.parametrize("riemann", [1, 0])
def test_uniform_state_is_steady(vl2, riemann):
    """A uniform state advected across the periodic mesh stays uniform (every face flux equal, every EMF
    equal): ten cycles change no conserved value by more than rounding."""
    b1, b2, b3 = inputs.uniform_faces(NX, B0)
    g = vl2.Mesh(NX, MB, riemann=riemann)
    g.set_prims(uniform_prims(), b1, b2, b3)
    u0 = g.get_cons()
    for _ in range(10):
        g.step(g.new_dt())
    u1 = g.get_cons()
    for a, b in zip(u0, u1):
        assert np.max(np.abs(a - b)) <= 1e-14 * max(1.0, np.max(np.abs(a)))
    assert g.floor_count() == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cfl_max_with_many_equal_cells(vl2, oracle, seed):
    """A uniform state in which a few cells carry pressures raised by up to 1e-7 (all of them within the
    single-precision screen of the maximum, several sharing a state): the CFL step is the oracle's."""
    rng = np.random.default_rng(seed)
    w = uniform_prims()
    n = NX[0] * NX[1] * NX[2]
    picks = rng.choice(n, size=40, replace=False)
    levels = 1.0 + 1e-7 * rng.integers(1, 5, size=40) / 4.0  # four distinct raised pressures
    w[4].reshape(-1)[picks] *= levels
    b1, b2, b3 = inputs.uniform_faces(NX, B0)
    g = vl2.Mesh(NX, MB)
    g.set_prims(w, b1, b2, b3)
    o = oracle.Mesh(NX, MB)
    o.set_prims(w, b1, b2, b3)
    dt_g, dt_o = g.new_dt(), o.new_dt(0.3)
    assert dt_g == pytest.approx(dt_o, rel=1e-14)
    # and the uniform state without the raised cells has a longer step, by more than the tolerance
    g2 = vl2.Mesh(NX, MB)
    g2.set_prims(uniform_prims(), b1, b2, b3)
    assert g2.new_dt() > dt_g * (1.0 + 1e-9)
