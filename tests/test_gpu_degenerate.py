"""GPU parity on the method's degenerate and discontinuous cases, against the FP64 oracle:

- Sod tubes with only a normal field (b_t = 0 on both sides: the HLLD single-star states take the
  degenerate branch), along x, y and z;
- a Brio-Wu-type MHD tube (gamma = 2, b_n = 0.75, b_t flipping sign: rotational discontinuities and a
  compound fan);
- outflow boundaries on a tube.
One cycle <= 1e-12 and 10 cycles <= 1e-10 (normalised as in the other parity tests); floors never fire.

Mirror-symmetric states are a separate case.  On their symmetry planes the face mass flux is exactly zero
in the oracle (which is bitwise mirror-symmetric), and the upwind CT takes the average of both cells
there.  The fast GPU build is not bitwise symmetric (contracted FMAs, Newton-refined reciprocals).  With
HLLD its contact speed and the averaged S_M = 0 flux still give an exactly zero mass flux on the plane, but
with HLLE the flux combination leaves a mass flux of rounding size with either sign after the predictor,
and the upwind switch, discontinuous at zero mass flux, picks one cell.  The two then differ near the
planes by the size of the upwind correction, and only there: that test bounds the difference elsewhere at
1e-12 and states the difference at the planes.  The value-safe build of the same sources (IEEE division and square root, no
contraction; Sec. 3.3.5 asks for value-safe arithmetic where symmetry must hold bitwise) stays bitwise
mirror-symmetric over 10 cycles along x, y and z, and matches the oracle to 1e-12 everywhere, planes
included."""
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


def sod_normal_field(axis):
    return inputs.shock_tube(64, axis=axis, b_left=(0.7, 0.0, 0.0), b_right=(0.7, 0.0, 0.0))


def brio_wu(axis):
    return inputs.shock_tube(64, axis=axis, left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.1),
                             b_left=(0.75, 1.0, 0.0), b_right=(0.75, -1.0, 0.0), gamma=2.0)


CASES = {
    "sod_bn_x": lambda: sod_normal_field(0),
    "sod_bn_y": lambda: sod_normal_field(1),
    "sod_bn_z": lambda: sod_normal_field(2),
    "brio_wu_x": lambda: brio_wu(0),
    "brio_wu_z": lambda: brio_wu(2),
}


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("case", sorted(CASES))
def test_degenerate_cases(vl2, oracle, case, riemann):
    prob = CASES[case]()
    g = vl2.Mesh.from_problem(prob, riemann=riemann)
    o = oracle.Mesh.from_problem(prob, riemann=riemann)
    worst = []
    for k in range(10):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
        d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
        worst.append(d)
        if k == 0:
            assert d <= 1e-12, (case, d)
    print("%s riemann %d: first cycle %.2e, 10 cycles %.2e" % (case, riemann, worst[0], worst[-1]))
    assert worst[-1] <= 1e-10, (case, worst)
    assert g.floor_count() == 0 and o.floor_count() == 0


def test_outflow_tube(vl2, oracle):
    prob = brio_wu(0)
    bc = (vl2.OUTFLOW, vl2.OUTFLOW, vl2.PERIODIC, vl2.PERIODIC, vl2.PERIODIC, vl2.PERIODIC)
    g = vl2.Mesh(prob.nx, (16, 1, 1), prob.xmin, prob.xmax, prob.gamma, bc=bc)
    g.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
    o = oracle.Mesh(prob.nx, (16, 1, 1), prob.xmin, prob.xmax, prob.gamma, bc=bc)
    o.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
    for _ in range(10):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
    d = float(np.max(state_diff(g.get_cons(), o.get_cons())))
    print("Brio-Wu tube, outflow x, 4 blocks: 10 cycles %.2e" % d)
    assert d <= 1e-10


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("n", [16, 32])
def test_mirror_states_differ_only_at_the_symmetry_planes(vl2, oracle, n, axis, riemann):
    from test_gpu_parity import scales

    prob = inputs.mirror_symmetric(n, mb=n // 2, axis=axis)
    g = vl2.Mesh.from_problem(prob, riemann=riemann)
    o = oracle.Mesh.from_problem(prob, riemann=riemann)
    dt = o.new_dt(0.3)
    g.step(dt)
    o.step(dt)
    gs, os_ = g.get_cons(), o.get_cons()
    su, sb = scales(*os_)

    def band(arr_shape, face_dir):
        # elements whose index along `axis` lies within 4 of a symmetry plane (x_axis = 0, 1/2, 1)
        m = arr_shape[2 - axis]
        idx = np.arange(m)
        plane = np.minimum(np.minimum(idx, n - idx), np.abs(idx - n // 2))
        near = plane < 4 if face_dir == axis else np.minimum(plane, np.minimum(idx + 1, n - 1 - idx)) < 4
        shape = [1, 1, 1]
        shape[2 - axis] = m
        return np.broadcast_to(near.reshape(shape), arr_shape)

    away, at = 0.0, 0.0
    for v in range(5):
        d = np.abs(gs[0][v] - os_[0][v]) / su[v]
        bmask = band(d.shape, -1)
        away, at = max(away, float(np.max(d[~bmask]))), max(at, float(np.max(d[bmask])))
    for fd in range(3):
        d = np.abs(gs[1 + fd] - os_[1 + fd]) / sb
        bmask = band(d.shape, fd)
        away, at = max(away, float(np.max(d[~bmask]))), max(at, float(np.max(d[bmask])))
    print("mirror %d^3 axis %d riemann %d: max difference away from the planes %.2e, at the planes %.2e"
          % (n, axis, riemann, away, at))
    assert away <= 1e-12
    assert g.floor_count() == 0


def mirror_max_asymmetry(cons, axis):
    """0 when the state is bitwise symmetric under x_axis -> -x_axis (about the domain's lower face): cells
    c <-> N-1-c, faces f <-> N-f, the normal momentum and normal field odd, the rest even."""
    u, b1, b2, b3 = cons
    npa = 3 - axis
    bad = 0
    for v in range(5):
        flipped = np.flip(u[v], axis=npa - 1)
        bad += int(np.count_nonzero(u[v] != (-flipped if v == 1 + axis else flipped)))
    for c, b in enumerate((b1, b2, b3)):
        flipped = np.flip(b, axis=2 - axis)
        bad += int(np.count_nonzero(b != (-flipped if c == axis else flipped)))
    return bad


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_value_safe_build_keeps_mirror_symmetry_bitwise(vl2, axis, riemann):
    prob = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=7 + axis)
    g = vl2.Mesh.from_problem(prob, riemann=riemann, value_safe=True)
    assert mirror_max_asymmetry(g.get_cons(), axis) == 0
    for k in range(10):
        g.step(g.new_dt())
        bad = mirror_max_asymmetry(g.get_cons(), axis)
        assert bad == 0, (k, bad)
    assert g.floor_count() == 0


@pytest.mark.parametrize("riemann", [1, 0])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("n", [16, 32])
def test_value_safe_mirror_states_match_the_oracle_everywhere(vl2, oracle, n, axis, riemann):
    prob = inputs.mirror_symmetric(n, mb=n // 2, axis=axis)
    g = vl2.Mesh.from_problem(prob, riemann=riemann, value_safe=True)
    o = oracle.Mesh.from_problem(prob, riemann=riemann)
    worst = []
    for k in range(10):
        dt = o.new_dt(0.3)
        g.step(dt)
        o.step(dt)
        worst.append(float(np.max(state_diff(g.get_cons(), o.get_cons()))))
    print("value-safe mirror %d^3 axis %d riemann %d: one cycle %.2e, 10 cycles %.2e (planes included)"
          % (n, axis, riemann, worst[0], worst[-1]))
    assert worst[0] <= 1e-12
    assert worst[-1] <= 1e-10
    assert g.floor_count() == 0
