"""Pins of the oracle's PPM reconstruction (Sec. 3.2.1: eq. ppm-uniform-weights and the smooth-extremum
preserving limiter) against what the mathematics fixes, without a GPU.

- the fourth-order face values are exact for the cell averages of any cubic (this fixes 7/12 and -1/12)
- where the face value leaves its two cells' range and the second differences disagree in sign, the
  limited face value is the mean of the two cells
- smooth extrema are kept: the edge values of a sine converge at third order or better everywhere,
  including the cells at its extrema (a limiter that clips extrema converges at first order there)
- a step stays monotone: no edge value leaves the range of the cell and its neighbours
- the full scheme: bitwise mirror symmetry and MeshBlock independence, N_G = 3 with PLM equal to
  N_G = 2 bitwise, and on the inclined fast wave second-order convergence with an error below PLM's
"""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_oracle_mesh import _inclined, rms_l1_error

G = 5.0 / 3.0


def cell_averages(antider, edges):
    h = np.diff(edges)
    return (antider(edges[1:]) - antider(edges[:-1])) / h


def test_face_values_exact_for_cubics(oracle):
    # a monotone cubic, so that neither limiter acts: p(x) = x^3 + 2x + 1 on [0.3, 1.3]
    p = lambda x: x ** 3 + 2 * x + 1
    P = lambda x: x ** 4 / 4 + x ** 2 + x
    for n in (10, 37):
        edges = np.linspace(0.3, 1.3, n + 1)
        q = cell_averages(P, edges)
        for i in range(2, n - 1):
            f = oracle.ppm_face(q[i - 2:i + 2])  # face between cells i-1 and i, at edges[i]
            assert f == pytest.approx(p(edges[i]), rel=1e-13, abs=1e-13)
        for i in range(2, n - 2):
            ql, qr = oracle.ppm_edges(q[i - 2:i + 3])
            assert ql == pytest.approx(p(edges[i]), rel=1e-13, abs=1e-13)
            assert qr == pytest.approx(p(edges[i + 1]), rel=1e-13, abs=1e-13)
    # a quadratic is reproduced by the parabola: edges exact, even at its extremum cell when the
    # second differences agree (x^2 around 0: every second difference is 2 h^2)
    P2 = lambda x: x ** 3 / 3
    edges = np.linspace(-1.0, 1.0, 22)
    q = cell_averages(P2, edges)
    for i in range(2, 19):
        ql, qr = oracle.ppm_edges(q[i - 2:i + 3])
        assert ql == pytest.approx(edges[i] ** 2, abs=1e-13)
        assert qr == pytest.approx(edges[i + 1] ** 2, abs=1e-13)


def test_face_limiter_falls_back_to_the_mean(oracle):
    rng = np.random.default_rng(11)
    seen = 0
    for _ in range(4000):
        q = rng.normal(size=4)
        f4 = 7.0 / 12.0 * (q[1] + q[2]) - 1.0 / 12.0 * (q[0] + q[3])
        f = oracle.ppm_face(q)
        inside = (f4 - q[1]) * (q[2] - f4) >= 0.0
        if inside:
            assert f == f4
            continue
        d2 = 3.0 * ((q[1] + q[2]) - 2.0 * f4)
        d2l = (q[0] + q[2]) - 2.0 * q[1]
        d2r = (q[1] + q[3]) - 2.0 * q[2]
        if not (np.sign(d2) == np.sign(d2l) == np.sign(d2r)):
            assert f == 0.5 * (q[1] + q[2])
            seen += 1
        else:
            lim = np.sign(d2) * min(abs(d2), 1.25 * abs(d2l), 1.25 * abs(d2r))
            assert f == pytest.approx(0.5 * (q[1] + q[2]) - lim / 6.0, rel=1e-14, abs=1e-15)
    assert seen > 100


def _edge_errors(oracle, n, limiter):
    edges = np.linspace(0.0, 1.0, n + 1)
    h = 1.0 / n
    centres = 0.5 * (edges[1:] + edges[:-1])
    # periodic sine, cell averages exact
    q = (np.cos(2 * np.pi * (centres - h / 2)) - np.cos(2 * np.pi * (centres + h / 2))) / (2 * np.pi * h)
    err = 0.0
    for i in range(n):
        idx = [(i + o) % n for o in range(-2, 3)]
        if limiter == "ppm":
            ql, qr = oracle.ppm_edges(q[idx])
        else:
            s = oracle.vanleer_slope(q[idx[1]], q[idx[2]], q[idx[3]])
            ql, qr = q[i] - 0.5 * s, q[i] + 0.5 * s
        err = max(err, abs(ql - np.sin(2 * np.pi * edges[i])), abs(qr - np.sin(2 * np.pi * edges[i + 1])))
    return err


def test_smooth_extrema_are_kept(oracle):
    e = [_edge_errors(oracle, n, "ppm") for n in (32, 64, 128)]
    orders = [math.log2(e[0] / e[1]), math.log2(e[1] / e[2])]
    v = [_edge_errors(oracle, n, "plm") for n in (32, 64, 128)]
    print("PPM max edge error %s (orders %s); PLM %s" % (e, orders, v))
    assert min(orders) >= 2.8
    assert e[2] < 0.01 * v[2]


def test_step_stays_monotone(oracle):
    rng = np.random.default_rng(12)
    for _ in range(500):
        # a random non-decreasing sequence with a jump somewhere
        q = np.sort(rng.normal(size=5)) * (1 + 10 * (rng.random() < 0.5))
        ql, qr = oracle.ppm_edges(q)
        lo, hi = min(q[1], q[2]), max(q[2], q[3])
        assert lo - 1e-15 <= ql <= q[2] + 1e-15
        assert q[2] - 1e-15 <= qr <= hi + 1e-15
    # the classic step: the cells on either side of the jump stay flat
    q = np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 1.0])
    assert oracle.ppm_edges(q[0:5]) == (0.0, 0.0)
    assert oracle.ppm_edges(q[1:6]) == (1.0, 1.0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ppm_mirror_symmetry_bitwise(oracle, axis):
    p = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=17 + axis)
    m = oracle.Mesh.from_problem(p, recon=oracle.PPM, integrator=oracle.RK3)
    for _ in range(3):
        m.step(m.new_dt(0.3))
    u, b1, b2, b3 = m.get_cons()
    npa = 3 - axis
    for v in range(5):
        flipped = np.flip(u[v], axis=npa - 1)
        np.testing.assert_array_equal(u[v], -flipped if v == 1 + axis else flipped)
    for c, b in enumerate((b1, b2, b3)):
        flipped = np.flip(b, axis=2 - axis)
        np.testing.assert_array_equal(b, -flipped if c == axis else flipped)


def test_ppm_block_decomposition_and_ghost_width(oracle):
    p = inputs.orszag_tang(n=24, mb=12, seed=19)
    ms = [oracle.Mesh.from_problem(p, recon=oracle.PPM, mb=mb) for mb in ((12, 12, 12), (8, 6, 24), (24, 24, 24))]
    for _ in range(3):
        dt = ms[0].new_dt(0.3)
        for m in ms:
            m.step(dt)
    s = [m.get_cons() for m in ms]
    for t in s[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(s[0], t))
    # three ghost layers do not change PLM
    a = oracle.Mesh.from_problem(p)
    b = oracle.Mesh.from_problem(p, ng=3)
    for _ in range(3):
        dt = a.new_dt(0.3)
        a.step(dt)
        b.step(dt)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_cons(), b.get_cons()))
    with pytest.raises(ValueError):
        oracle.Mesh(p.nx, p.mb, recon=oracle.PPM, ng=2)


@pytest.mark.parametrize("integrator", ["VL2", "RK3"])
def test_ppm_linear_wave_second_order_and_below_plm(oracle, integrator):
    """Inclined fast wave, one period: PPM converges at second order (CT and the time integrators bound
    it there, Sec. 3.2.1) with an error below PLM's at the same resolution."""
    errs = {}
    for recon in ("PLM", "PPM"):
        errs[recon] = []
        for n in (32, 64):
            prob = _inclined("fast", (n, n, 2), (2 * math.pi, 2 * math.pi, 0.0), (0.0, 0.0, 0.0))
            m = oracle.Mesh.from_problem(prob, integrator=getattr(oracle, integrator), recon=getattr(oracle, recon))
            ref = m.get_cons()
            m.run(prob.meta["period"], cfl=0.3)
            assert m.floor_count() == 0
            errs[recon].append(rms_l1_error(m.get_cons(), ref))
    slope = math.log2(errs["PPM"][0] / errs["PPM"][1])
    print("%s fast wave L1: PLM %s, PPM %s (PPM slope %.3f)" % (integrator, errs["PLM"], errs["PPM"], slope))
    assert slope >= 1.8
    assert errs["PPM"][1] < errs["PLM"][1]
