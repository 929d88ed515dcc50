"""Pins of the oracle's characteristic reconstruction (Sec. 3.2.1: PLM on C = L W, L the left
eigenvectors of the primitive ideal-MHD system) against what the mathematics fixes, without a GPU.

- the system matrix A of the primitive equations, typed here from the equations, equals the Jacobian of
  the oracle's physical flux mapped to primitives (central differences), so A is pinned independently
- the eigensystem: A R = R diag(lam) and L R = I at random states and at the degenerate ones (b_t = 0,
  b_n = 0, c_a = a with b_t = 0, negative b_n); the speeds solve the magnetosonic quartic
- the reconstruction: linear data is reproduced exactly; data made of two waves (fast and slow) is
  limited wave by wave, slope = vl(fast amplitudes) r_f + vl(slow amplitudes) r_s
- the scheme: mirror symmetry to round-off, MeshBlock independence bitwise, second-order convergence on
  the inclined fast wave, and on the Brio-Wu tube fewer oscillations than primitive PLM (Sec. 3.3)
"""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs
from test_oracle_mesh import _inclined, rms_l1_error

G = 5.0 / 3.0


def system_matrix(w, bn, gamma):
    """A of W_t + A W_n = 0, W = (rho, v_n, v_t1, v_t2, p, b_t1, b_t2), from the ideal-MHD equations."""
    rho, v, _, _, p, b1, b2 = w
    return np.array([
        [v, rho, 0, 0, 0, 0, 0],
        [0, v, 0, 0, 1 / rho, b1 / rho, b2 / rho],
        [0, 0, v, 0, 0, -bn / rho, 0],
        [0, 0, 0, v, 0, 0, -bn / rho],
        [0, gamma * p, 0, 0, v, 0, 0],
        [0, b1, -bn, 0, 0, v, 0],
        [0, b2, 0, -bn, 0, 0, v]], dtype=float)


def cons_of(w, bn, gamma):
    rho, v, t1, t2, p, b1, b2 = w
    e = p / (gamma - 1) + 0.5 * rho * (v * v + t1 * t1 + t2 * t2) + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    return np.array([rho, rho * v, rho * t1, rho * t2, e, b1, b2])


def random_states(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w = np.array([rng.uniform(0.2, 3), rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-2, 2),
                      rng.uniform(0.05, 3), rng.uniform(-2, 2), rng.uniform(-2, 2)])
        out.append((w, rng.uniform(-2, 2)))
    return out


DEGENERATE = [
    (np.array([1.0, 0.3, 0.1, -0.2, 0.6, 0.0, 0.0]), 1.3),  # b_t = 0, c_a > a
    (np.array([1.0, 0.3, 0.1, -0.2, 0.6, 0.0, 0.0]), 0.4),  # b_t = 0, c_a < a
    (np.array([1.0, 0.0, 0.0, 0.0, 0.6, 0.0, 0.0]), math.sqrt(G * 0.6)),  # b_t = 0, c_a = a (triple)
    (np.array([1.2, -0.5, 0.0, 0.3, 0.9, 0.7, -0.4]), 0.0),  # b_n = 0
    (np.array([0.8, 0.1, 0.2, 0.3, 1.1, -0.3, 0.9]), -0.7),  # b_n < 0
    (np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0]), 0.0),  # hydrodynamics
]


def test_system_matrix_is_the_flux_jacobian(oracle):
    for w, bn in random_states(1, 20):
        h = 1e-6
        dF, dU = np.zeros((7, 7)), np.zeros((7, 7))
        for q in range(7):
            e = np.zeros(7)
            e[q] = h * max(1.0, abs(w[q]))
            fp, fm = oracle.riemann(0, w + e, w + e, bn, G), oracle.riemann(0, w - e, w - e, bn, G)
            dF[:, q] = (fp - fm) / (2 * e[q])
            dU[:, q] = (cons_of(w + e, bn, G) - cons_of(w - e, bn, G)) / (2 * e[q])
        A = np.linalg.solve(dU, dF)
        np.testing.assert_allclose(A, system_matrix(w, bn, G), atol=1e-7 * (1 + np.max(np.abs(A))))


@pytest.mark.parametrize("case", ["random", "degenerate"])
def test_eigensystem(oracle, case):
    states = random_states(2, 200) if case == "random" else DEGENERATE
    worst = 0.0
    for w, bn in states:
        R, L, lam = oracle.mhd_eigensystem(w, bn, G)
        A = system_matrix(w, bn, G)
        scale = np.max(np.abs(A)) * np.max(np.abs(R))
        worst = max(worst, np.max(np.abs(A @ R - R * lam[None, :])) / scale)
        np.testing.assert_allclose(A @ R, R * lam[None, :], atol=1e-13 * scale)
        np.testing.assert_allclose(L @ R, np.eye(7), atol=1e-12)
        assert np.all(np.diff(lam) >= 0.0)
        assert np.linalg.cond(R) < 1e6
        # the magnetosonic speeds solve (c^2 - a^2)(c^2 - c_a^2) = c_t^2 c^2
        rho, v, p = w[0], w[1], w[4]
        a2, ca2, ct2 = G * p / rho, bn * bn / rho, (w[5] ** 2 + w[6] ** 2) / rho
        for c in (lam[6] - v, lam[4] - v):
            assert abs((c * c - a2) * (c * c - ca2) - ct2 * c * c) <= 1e-12 * (a2 + ca2 + ct2) ** 2
        assert abs((lam[5] - v) ** 2 - ca2) <= 1e-13 * (1 + ca2)
    print("eigensystem (%s): max |A R - R lam| / scale %.2e" % (case, worst))


def test_linear_data_is_reproduced(oracle):
    rng = np.random.default_rng(3)
    for w, bn in random_states(4, 50) + DEGENERATE:
        d = 0.01 * rng.standard_normal(7) * np.maximum(1.0, np.abs(w))
        s = oracle.char_slope(w - d, w, w + d, bn, G)
        np.testing.assert_allclose(s, d, atol=1e-13 * np.max(np.abs(d)) + 1e-16)


def test_two_waves_are_limited_wave_by_wave(oracle):
    def vl(x, y):
        return 2 * x * y / (x + y) if x * y > 0 else 0.0

    rng = np.random.default_rng(5)
    seen_difference = 0
    for w, bn in random_states(6, 100):
        R, _, _ = oracle.mhd_eigensystem(w, bn, G)
        rf, rs = R[:, 6], R[:, 4]
        e1, e2 = rng.uniform(-1, 1, 2) * 1e-2
        g1, g2 = rng.uniform(-1, 1, 2) * 1e-2
        qm = w - (e1 * rf + e2 * rs)
        qp = w + (g1 * rf + g2 * rs)
        s = oracle.char_slope(qm, w, qp, bn, G)
        want = vl(e1, g1) * rf + vl(e2, g2) * rs
        np.testing.assert_allclose(s, want, atol=1e-12 * (np.max(np.abs(want)) + 1e-3))
        prim = np.array([oracle.vanleer_slope(a, b, c) for a, b, c in zip(qm, w, qp)])
        seen_difference += int(np.max(np.abs(prim - want)) > 1e-6)
    assert seen_difference > 50  # primitive limiting gives other slopes on these data


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_char_mirror_symmetry(oracle, axis):
    # to round-off, not bitwise: L = R^-1 is eliminated in another pivot order for the mirrored state.
    # Faces on the mirror plane carry a mass flux that is zero in exact arithmetic; the sharp CT switch
    # turns its round-off into a one-sided pick and the asymmetry grows to 2e-4 within two cycles, so the
    # corners take the smoothed weight (delta 1e-3), under which it stays at round-off
    p = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=57 + axis)
    m = oracle.Mesh.from_problem(p, recon=oracle.PLM_CHAR, ct_delta=1e-3)
    for _ in range(3):
        m.step(m.new_dt(0.3))
    u, b1, b2, b3 = m.get_cons()
    npa = 3 - axis
    worst = 0.0
    for v in range(5):
        flipped = np.flip(u[v], axis=npa - 1)
        want = -flipped if v == 1 + axis else flipped
        worst = max(worst, float(np.max(np.abs(u[v] - want))) / float(np.max(np.abs(u[v])) + 1e-300))
    for c, b in enumerate((b1, b2, b3)):
        flipped = np.flip(b, axis=2 - axis)
        want = -flipped if c == axis else flipped
        worst = max(worst, float(np.max(np.abs(b - want))) / float(np.max(np.abs(b)) + 1e-300))
    print("characteristic PLM mirror symmetry (axis %d): %.2e" % (axis, worst))
    assert worst <= 1e-13


def test_char_block_decomposition(oracle):
    p = inputs.orszag_tang(n=24, mb=12, seed=59)
    ms = [oracle.Mesh.from_problem(p, recon=oracle.PLM_CHAR, mb=mb) for mb in ((12, 12, 12), (8, 6, 24))]
    for _ in range(3):
        dt = ms[0].new_dt(0.3)
        for m in ms:
            m.step(dt)
    assert all(np.array_equal(a, b) for a, b in zip(ms[0].get_cons(), ms[1].get_cons()))


_WAVE_ERRORS = {}


def _wave_errors(oracle, recon):
    """L1 errors of the inclined fast wave after one period at 32^2 and 64^2 (computed once per run)."""
    if recon not in _WAVE_ERRORS:
        errs = []
        for n in (32, 64):
            prob = _inclined("fast", (n, n, 2), (2 * math.pi, 2 * math.pi, 0.0), (0.0, 0.0, 0.0))
            m = oracle.Mesh.from_problem(prob, recon=getattr(oracle, recon))
            ref = m.get_cons()
            m.run(prob.meta["period"], cfl=0.3)
            errs.append(rms_l1_error(m.get_cons(), ref))
        _WAVE_ERRORS[recon] = errs
    return _WAVE_ERRORS[recon]


def test_char_linear_wave_second_order(oracle):
    errs = _wave_errors(oracle, "PLM_CHAR")
    slope = math.log2(errs[0] / errs[1])
    print("characteristic PLM fast wave L1 %s, slope %.3f" % (errs, slope))
    assert slope >= 1.8


def _extrema(a, tol):
    d = np.diff(a)
    d = d[np.abs(d) > tol]
    return int(np.sum(np.sign(d[1:]) != np.sign(d[:-1])))


def test_brio_wu_fewer_oscillations(oracle):
    """Sec. 3.3: primitive reconstruction oscillates behind the fast rarefaction of the Brio-Wu tube,
    characteristic reconstruction much less (VL2 + PLM + HLLD, 256 cells, t = 0.1)."""
    n = 256
    prob = inputs.shock_tube(n, axis=0, left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.1),
                             b_left=(0.75, 1.0, 0.0), b_right=(0.75, -1.0, 0.0), gamma=2.0)
    out = {}
    for name, rec in (("prim", oracle.PLM), ("char", oracle.PLM_CHAR)):
        m = oracle.Mesh.from_problem(prob, recon=rec, mb=(64, 1, 1))
        m.run(0.1, cfl=0.4)
        u = m.get_cons()[0][:, 0, 0, n // 2:]  # the tube at x = 3/4
        rho = u[0]
        out[name] = (_extrema(rho, 1e-6), _extrema(u[2] / rho, 1e-6),
                     float(np.sum(np.abs(np.diff(u[1] / rho)))))
    print("Brio-Wu extrema of rho, v_y and total variation of v_x: primitive %s, characteristic %s"
          % (out["prim"], out["char"]))
    assert out["char"][0] <= out["prim"][0] // 2
    assert out["char"][1] < out["prim"][1]
    assert out["char"][2] < out["prim"][2]


# ---- characteristic PPM ----------------------------------------------------------------------------

def _face_values(oracle, prob, recon):
    m = oracle.Mesh.from_problem(prob, recon=recon)
    return m.debug_fluxes(recon)


def test_char_ppm_scheme(oracle):
    """PPM on characteristic variables: MeshBlock independence bitwise; mirror symmetry up to the PPM
    extremum test's ties (smoothed CT, as for PLM); second order on the inclined fast wave with an error
    below characteristic PLM's; fluxes that differ from primitive PPM on the vortex (several waves
    overlap)."""
    p = inputs.orszag_tang(n=24, mb=12, seed=61)
    ms = [oracle.Mesh.from_problem(p, recon=oracle.PPM_CHAR, mb=mb) for mb in ((12, 12, 12), (8, 6, 24))]
    for _ in range(2):
        dt = ms[0].new_dt(0.3)
        for m in ms:
            m.step(dt)
    assert all(np.array_equal(a, b) for a, b in zip(ms[0].get_cons(), ms[1].get_cons()))
    fa = _face_values(oracle, p, oracle.PPM_CHAR)
    fb = _face_values(oracle, p, oracle.PPM)
    assert max(float(np.max(np.abs(a - b))) for a, b in zip(fa, fb)) > 1e-8

    q = inputs.mirror_symmetric(n=16, mb=8, axis=1, seed=63)
    m = oracle.Mesh.from_problem(q, recon=oracle.PPM_CHAR, ct_delta=1e-3)
    for _ in range(3):
        m.step(m.new_dt(0.3))
    u = m.get_cons()[0]
    worst = 0.0
    for v in range(5):
        flipped = np.flip(u[v], axis=1)
        want = -flipped if v == 2 else flipped
        worst = max(worst, float(np.max(np.abs(u[v] - want))) / float(np.max(np.abs(u[v]))))
    print("characteristic PPM mirror symmetry: %.2e" % worst)
    # Even fields take equal values in the two cells astride the mirror plane: a tie of the PPM extremum
    # test, which switches discontinuously there (Colella & Sekora).  The characteristic projection breaks
    # the tie with round-off that differs on the two sides, so symmetry holds only to 3e-5 here; a sign
    # or index mistake would break it at O(1)
    assert worst <= 1e-3

    errs = {recon: _wave_errors(oracle, recon) for recon in ("PLM_CHAR", "PPM_CHAR")}
    slope = math.log2(errs["PPM_CHAR"][0] / errs["PPM_CHAR"][1])
    print("fast wave L1: characteristic PLM %s, characteristic PPM %s (slope %.3f)"
          % (errs["PLM_CHAR"], errs["PPM_CHAR"], slope))
    assert slope >= 1.8
    assert errs["PPM_CHAR"][1] < errs["PLM_CHAR"][1]


def test_char_ppm_single_wave_equals_primitive_ppm(oracle):
    """On data made of one eigenmode of the cell (q_j = q_0 + alpha_j r_k) the characteristic and the
    primitive PPM limit the same amplitude, so the two give the same face fluxes (to rounding); a
    mistake in L or R (not inverse to each other, or not eigenvectors) breaks this."""
    n = 32
    rng = np.random.default_rng(65)
    w0 = np.array([1.1, 0.2, -0.1, 0.15, 0.7, 0.4, -0.3])
    bn = 0.8
    R, _, _ = oracle.mhd_eigensystem(w0, bn, G)
    for k in (0, 2, 6):
        alpha = 1e-3 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n + rng.uniform(0, 6.3))
        cells = w0[None, :] + alpha[:, None] * R[:, k][None, :]
        worst = 0.0
        for i in range(3, n - 3):
            qs = cells[i - 3:i + 3]
            # primitive PPM edges of cells i-1 and i, per component, and the characteristic ones
            for c in (i - 1, i):
                st = cells[c - 2:c + 3]
                prim = np.array([oracle.ppm_edges(st[:, v]) for v in range(7)])
                chars = oracle.char_ppm_edges(st, bn, G)
                worst = max(worst, float(np.max(np.abs(prim - chars))))
        print("single eigenmode %d: |characteristic - primitive| PPM edges %.2e" % (k, worst))
        assert worst <= 1e-14


def test_brio_wu_char_ppm_fewer_oscillations(oracle):
    n = 256
    prob = inputs.shock_tube(n, axis=0, left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.1),
                             b_left=(0.75, 1.0, 0.0), b_right=(0.75, -1.0, 0.0), gamma=2.0)
    out = {}
    for name, rec in (("prim", oracle.PPM), ("char", oracle.PPM_CHAR)):
        m = oracle.Mesh.from_problem(prob, recon=rec, integrator=oracle.RK3, mb=(64, 1, 1))
        m.run(0.1, cfl=0.4)
        u = m.get_cons()[0][:, 0, 0, n // 2:]
        out[name] = (_extrema(u[0], 1e-6), _extrema(u[2] / u[0], 1e-6))
    print("Brio-Wu, RK3 + PPM, extrema of rho and v_y: primitive %s, characteristic %s" % (out["prim"], out["char"]))
    assert out["char"][0] < out["prim"][0]
    assert out["char"][1] < out["prim"][1]
