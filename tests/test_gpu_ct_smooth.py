"""The smoothed CT upwind weight (an option beside the paper's sign switch) on the GPU, through the C ABI,
against the FP64 oracle.

- a vanishing delta gives bitwise the results of the sign switch, in FP64 and in the mixed form
- one cycle of the vortex with a delta comparable to its mass fluxes (so that many corners take partial
  weights) equals the oracle's to rounding
- the magnetized blast, bounded only by the oracle's own spread with the sharp switch, agrees to rounding
  with delta = 1e-4 over two cycles, floors included
- the adjoint of the smoothed cycle (vl2_step_vjp) carries dw/dm: the dot-product test against the
  oracle's dual-number tangent-linear holds to 1e-12 with the weights on the slope of tanh (a wave
  advected at mass fluxes ~ delta, and a wave at rest), and central differences of the GPU cycle agree
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


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_vanishing_delta_is_bitwise_the_switch(vl2, precision):
    # in the mixed form delta = 1e-300 underflows to 0 in FP32: every weight is then 0, 1 or 1/2 (m = 0)
    prob = inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=9)
    a = vl2.Mesh.from_problem(prob, precision=getattr(vl2, precision))
    b = vl2.Mesh.from_problem(prob, precision=getattr(vl2, precision), ct_delta=1e-300)
    for _ in range(3):
        dt = a.new_dt()
        a.step(dt)
        b.step(dt)
    for x, y in zip(a.get_cons(), b.get_cons()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("riemann", [1, 0])
def test_smooth_weight_one_cycle(vl2, oracle, riemann):
    prob = inputs.orszag_tang(n=(24, 20, 12), mb=(8, 10, 6), seed=9)
    g = vl2.Mesh.from_problem(prob, riemann=riemann, ct_delta=0.3)
    o = oracle.Mesh.from_problem(prob, riemann=riemann, ct_delta=0.3)
    dt = o.new_dt(0.3)
    g.step(dt)
    o.step(dt)
    d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
    sharp = oracle.Mesh.from_problem(prob, riemann=riemann)
    sharp.step(dt)
    moved = float(np.max(state_diff(sharp.get_cons(), o.get_cons())))
    print("smoothed CT (delta 0.3), one cycle, riemann %d: GPU vs oracle %.2e (smoothing moved the state %.2e)"
          % (riemann, d, moved))
    assert d <= 1e-12
    assert moved > 1e-8  # the option is exercised, not a no-op


@pytest.mark.parametrize("riemann", [1, 0])
def test_smooth_weight_makes_the_blast_parity_exact(vl2, oracle, riemann):
    prob = inputs.blast(32, mb=16, r0=0.1, magnetized=True)
    g = vl2.Mesh.from_problem(prob, riemann=riemann, ct_delta=1e-4)
    o = oracle.Mesh.from_problem(prob, riemann=riemann, ct_delta=1e-4)
    for c in range(2):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
        o.new_dt(0.3)
        d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
        print("magnetized blast, delta 1e-4, riemann %d, cycle %d: GPU vs oracle %.2e" % (riemann, c, d))
        assert d <= 1e-12
    assert g.divb_norm() <= 1e-13


def test_smooth_weight_refusals_and_mixed(vl2):
    prob = inputs.orszag_tang(n=16, mb=8, seed=1)
    for kw in (dict(ct_delta=-1.0), dict(ct_delta=float("inf")), dict(ct_delta=float("nan"))):
        with pytest.raises(vl2.VL2Error):
            vl2.Mesh.from_problem(prob, **kw)
    # a batch whose meshes share delta is bitwise the per-mesh path; mixing deltas is refused
    probs = [inputs.orszag_tang(n=n, mb=n, seed=80 + n) for n in (16, 24, 32)]
    solo = [vl2.Mesh.from_problem(p, ct_delta=0.05) for p in probs]
    dts = [m.new_dt() for m in solo]
    for m, dt in zip(solo, dts):
        m.step(dt)
    meshes = [vl2.Mesh.from_problem(p, ct_delta=0.05) for p in probs]
    vl2.Batch(meshes).step(dts)
    for a, b in zip(solo, meshes):
        for x, y in zip(a.get_cons(), b.get_cons()):
            np.testing.assert_array_equal(x, y)
    with pytest.raises(vl2.VL2Error):
        vl2.Batch([vl2.Mesh.from_problem(probs[0], ct_delta=1e-3), vl2.Mesh.from_problem(probs[1])])
    m = vl2.Mesh.from_problem(prob, precision=vl2.MIXED, ct_delta=0.1)
    t0 = m.totals()
    for _ in range(5):
        m.step(m.new_dt())
    assert abs(m.totals()[0] - t0[0]) <= 1e-13 * abs(t0[0])
    assert m.divb_norm() <= 1e-13


def _periodic_direction(state, rng):
    u, b1, b2, b3 = state
    du = rng.standard_normal(u.shape)
    d1 = rng.standard_normal(b1.shape)
    d1[:, :, -1] = d1[:, :, 0]
    d2 = rng.standard_normal(b2.shape)
    d2[:, -1, :] = d2[:, 0, :]
    d3 = rng.standard_normal(b3.shape)
    d3[-1, :, :] = d3[0, :, :]
    return du, d1, d2, d3


def _to_dev(arrs):
    import torch

    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


def _absdot(a, b):
    return sum(float(np.sum(np.abs(x * y))) for x, y in zip(a, b))


SMOOTH_ADJ = [((0.7, 0.4, 0.2), 0.3, 1), ((0.7, 0.4, 0.2), 0.3, 0), ((0.0, 0.0, 0.0), 1e-2, 1),
              ((0.0, 0.0, 0.0), 1e-2, 0)]


@pytest.mark.parametrize("v0,delta,riemann", SMOOTH_ADJ)
def test_smoothed_adjoint_dot_product(vl2, oracle, v0, delta, riemann):
    prob = inputs.linear_wave(12, mb=6, kind="fast", amp=1e-2, v0=v0)
    g = vl2.Mesh.from_problem(prob, adjoint=True, riemann=riemann, ct_delta=delta)
    x = g.get_cons()
    dt = g.new_dt()
    rng = np.random.default_rng(7)
    dx = _periodic_direction(x, rng)
    y = tuple(rng.standard_normal(a.shape) for a in x)
    geom = (prob.nx, prob.mb, prob.xmin, prob.xmax, prob.bc)
    _, jdx = oracle.tl_step(geom, dt, x, dx, gamma=prob.gamma, riemann=riemann, ct_delta=delta)
    lhs = _dot(jdx, y)
    rhs = _dot(dx, [t.cpu().numpy() for t in g.step_vjp(dt, _to_dev(y))])
    scale = _absdot(jdx, y)
    # the test tells the smoothed derivative from the sharp switch's: their <J dx, y> differ by far more
    # than the tolerance
    _, jdx0 = oracle.tl_step(geom, dt, x, dx, gamma=prob.gamma, riemann=riemann)
    moved = abs(_dot(jdx0, y) - lhs) / scale
    print("smoothed adjoint (delta %g, v0 %s, riemann %d): <J dx, y> vs <dx, J^T y> rel %.2e "
          "(smoothing moves <J dx, y> by %.2e)" % (delta, v0, riemann, abs(lhs - rhs) / scale, moved))
    assert abs(lhs - rhs) <= 1e-12 * scale
    assert moved > 1e-6


def test_smoothed_adjoint_matches_central_differences_of_the_gpu_cycle(vl2):
    prob = inputs.linear_wave(12, mb=6, kind="fast", amp=1e-2, v0=(0.0, 0.0, 0.0))
    g = vl2.Mesh.from_problem(prob, adjoint=True, ct_delta=1e-2)
    x = g.get_cons()
    dt = g.new_dt()
    rng = np.random.default_rng(11)
    y = tuple(rng.standard_normal(a.shape) for a in x)
    g.set_cons(*x)
    jty = tuple(t.cpu().numpy() for t in g.step_vjp(dt, _to_dev(y)))
    def central(d, h):
        vals = []
        for sgn in (1.0, -1.0):
            g.set_cons(*[a + sgn * h * b for a, b in zip(x, d)])
            g.step(dt)
            vals.append(_dot(g.get_cons(), y))
        return (vals[0] - vals[1]) / (2 * h)

    for trial in range(3):
        d = _periodic_direction(x, rng)
        # Richardson: the h^2 term of the central difference grows as delta^-3 through tanh, so it is
        # cancelled with the difference at 2h
        h = 1e-6
        fd = (4.0 * central(d, h) - central(d, 2 * h)) / 3.0
        ad = _dot(jty, d)
        print("smoothed adjoint vs central differences of the GPU cycle, trial %d: rel %.2e"
              % (trial, abs(fd - ad) / abs(ad)))
        assert abs(fd - ad) <= 1e-6 * abs(ad), (trial, fd, ad)
