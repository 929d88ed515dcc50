"""Pins of the oracle's pointwise pieces against what the mathematics fixes (no GPU).

Riemann solvers (Sec. 3.2.2): consistency F(W, W) = F(W); upwinding for supersonic states; exact
resolution of isolated contacts and rotational discontinuities by HLLD (a property of the method of
Miyoshi & Kusano that the paper uses); exact mirror symmetry.  PLM (Sec. 3.2.1): exact on linear
data, zero at extrema, bounded by neighbours.  Upwind CT (Sec. 3.1, 2.1.1): exact for quadratic
fields for every upwind choice.  Fast speed: closed forms in the three textbook limits.
"""
import math

import numpy as np
import pytest

G = 5.0 / 3.0


def rand_state(rng, vmax=1.0):
    return np.array([rng.uniform(0.5, 2.0), rng.uniform(-vmax, vmax), rng.uniform(-vmax, vmax),
                     rng.uniform(-vmax, vmax), rng.uniform(0.3, 2.0), rng.uniform(-1, 1), rng.uniform(-1, 1)])


def flux_def(w, bn, gamma):
    """Ideal-MHD flux along the normal written straight from eq. cons / eq. total_energy."""
    d, u, v, ww, p, by, bz = w
    b2 = bn * bn + by * by + bz * bz
    E = p / (gamma - 1) + 0.5 * d * (u * u + v * v + ww * ww) + 0.5 * b2
    pt = p + 0.5 * b2
    vb = u * bn + v * by + ww * bz
    return np.array([d * u, d * u * u + pt - bn * bn, d * u * v - bn * by, d * u * ww - bn * bz,
                     (E + pt) * u - bn * vb, by * u - bn * v, bz * u - bn * ww])


def cons_def(w, bn, gamma):
    d, u, v, ww, p, by, bz = w
    E = p / (gamma - 1) + 0.5 * d * (u * u + v * v + ww * ww) + 0.5 * (bn * bn + by * by + bz * bz)
    return np.array([d, d * u, d * v, d * ww, E, by, bz])


@pytest.mark.parametrize("solver", [0, 1])
def test_physical_flux_matches_equations(oracle, solver):
    rng = np.random.default_rng(11)
    for _ in range(50):
        w = rand_state(rng)
        bn = rng.uniform(-1, 1)
        u, f = oracle.physical_flux(w, bn, G)
        np.testing.assert_allclose(f, flux_def(w, bn, G), rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(u, cons_def(w, bn, G), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("solver", [0, 1])
def test_consistency(oracle, solver):
    rng = np.random.default_rng(1)
    for _ in range(200):
        w = rand_state(rng)
        bn = rng.uniform(-1, 1) if _ % 5 else 0.0
        f = oracle.riemann(solver, w, w, bn, G)
        ref = flux_def(w, bn, G)
        scale = np.max(np.abs(ref)) + 1.0
        assert np.max(np.abs(f - ref)) <= 2e-14 * scale


@pytest.mark.parametrize("solver", [0, 1])
def test_supersonic_upwind(oracle, solver):
    rng = np.random.default_rng(2)
    for _ in range(100):
        wl, wr = rand_state(rng, 0.2), rand_state(rng, 0.2)
        bn = rng.uniform(-1, 1)
        cmax = max(oracle.fast_speed(wl[0], wl[4], bn, wl[5], wl[6], G),
                   oracle.fast_speed(wr[0], wr[4], bn, wr[5], wr[6], G))
        # both states supersonic to the right: the flux is the left physical flux exactly
        wl[1] = wr[1] = cmax + 1.0 + rng.uniform(0, 1)
        wr[1] = wl[1] + 0.1
        # HLLD returns the outer flux itself; HLLE forms b+ F_L / b+ (equal up to one rounding)
        check = (np.testing.assert_array_equal if solver == 1 else
                 (lambda a, b: np.testing.assert_allclose(a, b, rtol=3e-16, atol=1e-300)))
        f = oracle.riemann(solver, wl, wr, bn, G)
        check(f, oracle.physical_flux(wl, bn, G)[1])
        np.testing.assert_allclose(f, flux_def(wl, bn, G), rtol=1e-14, atol=1e-14)
        wl[1] = wr[1] = -(cmax + 1.0 + rng.uniform(0, 1))
        wl[1] = wr[1] - 0.1
        f = oracle.riemann(solver, wl, wr, bn, G)
        check(f, oracle.physical_flux(wr, bn, G)[1])


@pytest.mark.parametrize("bn", [0.0, 0.8, -0.6])
@pytest.mark.parametrize("u0", [0.0, 0.35, -0.4])
def test_hlld_resolves_contact_exactly(oracle, bn, u0):
    """Isolated contact (equal u, p, B; jump in rho and transverse v only when bn = 0): the HLLD flux is
    the physical flux of the upwind state; HLLE smears it (non-zero spurious mass flux)."""
    wl = np.array([1.0, u0, 0.2, -0.1, 0.8, 0.5, -0.3])
    wr = np.array([0.25, u0, 0.2, -0.1, 0.8, 0.5, -0.3])
    if bn == 0.0:
        wr[2], wr[3] = -0.4, 0.7  # tangential discontinuity in v allowed without normal field
    f = oracle.riemann(1, wl, wr, bn, G)
    up = wl if u0 > 0 else wr
    ref = flux_def(up, bn, G)
    if u0 == 0.0:
        # stationary contact: mass flux and energy flux vanish exactly
        ref = flux_def(wl, bn, G)
        assert abs(f[0]) <= 1e-15
    np.testing.assert_allclose(f, ref, rtol=0, atol=5e-15 * (1 + np.max(np.abs(ref))))
    fe = oracle.riemann(0, wl, wr, bn, G)
    assert np.max(np.abs(fe - ref)) > 1e-3


@pytest.mark.parametrize("family", [+1, -1])
@pytest.mark.parametrize("side", ["left", "right"])
@pytest.mark.parametrize("bn", [0.9, -0.7])
def test_hlld_resolves_rotational_discontinuity_exactly(oracle, family, side, bn):
    """Isolated Alfven (rotational) discontinuity: same rho, p, u_n, |b_t|; b_t rotated and
    [v_t] = -sign(b_n) * family * [b_t] / sqrt(rho) (Rankine-Hugoniot).  It moves at
    S = u_n + family |b_n| / sqrt(rho); the exact interface flux is F(W_L) if S > 0, F(W_R) if S < 0."""
    rho, p = 1.3, 0.7
    ca = abs(bn) / math.sqrt(rho)
    s_target = 0.4 * ca if side == "left" else -0.4 * ca
    un = s_target - family * ca
    bt_l = np.array([0.6, 0.3])
    th = 1.1
    bt_r = np.array([math.cos(th) * bt_l[0] - math.sin(th) * bt_l[1], math.sin(th) * bt_l[0] + math.cos(th) * bt_l[1]])
    vt_l = np.array([0.1, -0.2])
    vt_r = vt_l - np.sign(bn) * family * (bt_r - bt_l) / math.sqrt(rho)
    wl = np.array([rho, un, vt_l[0], vt_l[1], p, bt_l[0], bt_l[1]])
    wr = np.array([rho, un, vt_r[0], vt_r[1], p, bt_r[0], bt_r[1]])
    # the jump satisfies the Rankine-Hugoniot condition of the flux definition
    S = un + family * ca
    np.testing.assert_allclose(flux_def(wr, bn, G) - flux_def(wl, bn, G),
                               S * (cons_def(wr, bn, G) - cons_def(wl, bn, G)), atol=1e-14)
    f = oracle.riemann(1, wl, wr, bn, G)
    ref = flux_def(wl if S > 0 else wr, bn, G)
    np.testing.assert_allclose(f, ref, rtol=0, atol=2e-14)


def mirror(w):
    m = w.copy()
    m[1] = -m[1]
    return m


@pytest.mark.parametrize("solver", [0, 1])
def test_riemann_mirror_symmetry_bitwise(oracle, solver):
    """Reflecting the normal axis (swap L and R, negate v_n and b_n) negates the fluxes of the
    even conserved variables and keeps those of the odd ones: exactly, in IEEE arithmetic."""
    rng = np.random.default_rng(3)
    sign = np.array([-1, 1, -1, -1, -1, -1, -1], dtype=float)  # parity of each flux component
    for n in range(300):
        wl, wr = rand_state(rng), rand_state(rng)
        bn = rng.uniform(-1, 1)
        if n % 7 == 0:
            wr = mirror(wl)  # symmetric face: S_M == 0 exactly
            bn = 0.0 if n % 2 else bn
        f = oracle.riemann(solver, wl, wr, bn, G)
        g = oracle.riemann(solver, mirror(wr), mirror(wl), -bn, G)
        np.testing.assert_array_equal(g, sign * f)
        if n % 7 == 0 and bn == 0.0:
            assert f[0] == 0.0


def test_fast_speed_closed_forms(oracle):
    rng = np.random.default_rng(4)
    for _ in range(50):
        d, p = rng.uniform(0.5, 2), rng.uniform(0.3, 2)
        a = math.sqrt(G * p / d)
        assert oracle.fast_speed(d, p, 0.0, 0.0, 0.0, G) == pytest.approx(a, rel=1e-15)
        bn = rng.uniform(-2, 2)
        assert oracle.fast_speed(d, p, bn, 0.0, 0.0, G) == pytest.approx(max(a, abs(bn) / math.sqrt(d)), rel=1e-14)
        bt1, bt2 = rng.uniform(-2, 2), rng.uniform(-2, 2)
        assert oracle.fast_speed(d, p, 0.0, bt1, bt2, G) == pytest.approx(math.sqrt(a * a + (bt1 ** 2 + bt2 ** 2) / d),
                                                                        rel=1e-14)


def test_vanleer_limiter(oracle):
    rng = np.random.default_rng(5)
    for _ in range(300):
        # linear data: the limited slope is the exact slope (dyadic data: every step is exact)
        q0, h = rng.integers(-64, 64) / 16.0, rng.integers(1, 32) / 32.0 * rng.choice([-1, 1])
        assert oracle.vanleer_slope(q0 - h, q0, q0 + h) == h
        q0, h = rng.uniform(-2, 2), rng.uniform(-1, 1)
        assert oracle.vanleer_slope(q0 - h, q0, q0 + h) == pytest.approx(h, rel=1e-15)
        # local extremum: zero slope
        e = abs(rng.uniform(0.01, 1))
        assert oracle.vanleer_slope(q0 - e, q0, q0 - 2 * e) == 0.0
        # boundedness: face values q0 -+ slope/2 stay within the neighbours
        qm, qp = q0 + rng.uniform(-1, 1), q0 + rng.uniform(-1, 1)
        s = oracle.vanleer_slope(qm, q0, qp)
        lo, hi = min(qm, q0, qp), max(qm, q0, qp)
        for face in (q0 - 0.5 * s, q0 + 0.5 * s):
            assert lo - 1e-15 <= face <= hi + 1e-15
        # symmetry: reversing the stencil negates the slope exactly
        assert oracle.vanleer_slope(qp, q0, qm) == -s


@pytest.mark.parametrize("seed", range(6))
def test_ct_corner_exact_for_quadratics(oracle, seed):
    """Point values of a quadratic E(x, y) at the cell centres and face centres around a corner give
    E(corner) exactly: for a separable quadratic (no x y term) whatever the upwind directions, and for
    the full quadratic whenever both halves of each edge upwind from the same side (the correction
    of the x y term is (x_I0 - x_I1) / 2).  This fixes the sign and weight of each correction term."""
    rng = np.random.default_rng(100 + seed)
    c = rng.uniform(-1, 1, 6)

    def stencil(E):
        ea = [E(0.0, -0.5), E(0.0, 0.5)]      # x-faces (i-1/2, j-1), (i-1/2, j)
        eb = [E(-0.5, 0.0), E(0.5, 0.0)]      # y-faces (i-1, j-1/2), (i, j-1/2)
        ec = [E(-0.5, -0.5), E(0.5, -0.5), E(-0.5, 0.5), E(0.5, 0.5)]
        return ea, eb, ec

    sep = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[5] * y * y
    full = lambda x, y: sep(x, y) + c[4] * x * y
    signs = (-1.0, 0.0, 1.0)
    ea, eb, ec = stencil(sep)
    for ma0 in signs:
        for ma1 in signs:
            for mb0 in signs:
                for mb1 in signs:
                    v = oracle.ct_corner(ea, eb, ec, [ma0, ma1], [mb0, mb1])
                    assert v == pytest.approx(sep(0.0, 0.0), abs=1e-14)
    ea, eb, ec = stencil(full)
    for ma in signs:
        for mb in signs:
            v = oracle.ct_corner(ea, eb, ec, [ma, ma], [mb, mb])
            assert v == pytest.approx(full(0.0, 0.0), abs=1e-14)
    # a kink (|x| + |y|) is not reproduced, and the upwind choice changes the answer
    K = lambda x, y: abs(x) + 2 * abs(y) + x * y * y
    ea, eb, ec = stencil(K)
    vals = {oracle.ct_corner(ea, eb, ec, [s, s], [t, t]) for s in (-1.0, 1.0) for t in (-1.0, 1.0)}
    assert len(vals) > 1


def prim_from_cons(u, bn, gamma):
    d = u[0]
    v = u[1:4] / d
    bt = u[5:7]
    p = (gamma - 1) * (u[4] - 0.5 * d * np.sum(v * v) - 0.5 * (bn * bn + np.sum(bt * bt)))
    return np.array([d, v[0], v[1], v[2], p, bt[0], bt[1]])


def test_hlld_single_star_flux_is_physical_flux_of_star_state(oracle):
    """In the single-star fan (S_L < 0 <= S*_L) HLLD returns F_L + S_L (U*_L - U_L).  The star state it
    implies carries the physical flux structure with its own total pressure p_T* (taken here from the
    normal-momentum component): F = (rho* u*, ., rho* u* v*_t - b_n B*_t, (E* + p_T*) u* - b_n (v*.B*),
    B*_t u* - b_n v*_t).  These are the jump conditions across S_L that define the single-star state."""
    rng = np.random.default_rng(21)
    tested = 0
    for _ in range(4000):
        wl, wr = rand_state(rng, 1.5), rand_state(rng, 1.5)
        bn = rng.uniform(1.0, 2.5) * rng.choice([-1, 1])
        f = oracle.riemann(1, wl, wr, bn, G)
        ul, fl = cons_def(wl, bn, G), flux_def(wl, bn, G)
        cl = oracle.fast_speed(wl[0], wl[4], bn, wl[5], wl[6], G)
        cr = oracle.fast_speed(wr[0], wr[4], bn, wr[5], wr[6], G)
        sl = min(wl[1], wr[1]) - max(cl, cr)
        ust = ul + (f - fl) / sl
        d = ust[0]
        un, vt, bt, E = ust[1] / d, ust[2:4] / d, ust[5:7], ust[4]
        # keep only cases that sit in the single-star fan: S*_L = u* - |bn|/sqrt(rho*) > 0 > S_L
        if not (sl < 0 and un - abs(bn) / math.sqrt(d) > 1e-3):
            continue
        pts = f[1] - d * un * un + bn * bn
        ref = np.array([d * un, f[1], d * un * vt[0] - bn * bt[0], d * un * vt[1] - bn * bt[1],
                        (E + pts) * un - bn * (un * bn + vt @ bt), bt[0] * un - bn * vt[0], bt[1] * un - bn * vt[1]])
        np.testing.assert_allclose(f, ref, rtol=0, atol=1e-12 * (1 + np.max(np.abs(ref))))
        tested += 1
    assert tested >= 20


@pytest.mark.parametrize("u0", [0.3, -0.25])
@pytest.mark.parametrize("bn", [0.8, -1.1])
def test_hlld_exact_for_alfven_contact_alfven_fan(oracle, u0, bn):
    """Riemann problem whose exact solution is a left rotational discontinuity, a contact with a density
    jump and a right rotational discontinuity (equal u_n and p throughout, |b_t| kept across each
    rotation).  HLLD resolves this fan exactly: the flux is the physical flux of the state next to the
    interface."""
    p = 0.6
    rl, rr = 1.4, 0.5
    b2 = np.array([0.5, -0.35])            # transverse field between the two rotations
    v2 = np.array([0.15, 0.05])            # transverse velocity between the two rotations
    rot = lambda b, th: np.array([math.cos(th) * b[0] - math.sin(th) * b[1], math.sin(th) * b[0] + math.cos(th) * b[1]])
    btl, btr = rot(b2, 0.9), rot(b2, -1.3)
    s = math.copysign(1.0, bn)
    vtl = v2 - s * (b2 - btl) / math.sqrt(rl)   # across the left-going rotation (speed u0 - c_A,L)
    vtr = v2 - s * (btr - b2) / math.sqrt(rr)   # across the right-going rotation (speed u0 + c_A,R)
    wl = np.array([rl, u0, vtl[0], vtl[1], p, btl[0], btl[1]])
    wr = np.array([rr, u0, vtr[0], vtr[1], p, btr[0], btr[1]])
    w2l = np.array([rl, u0, v2[0], v2[1], p, b2[0], b2[1]])
    w2r = np.array([rr, u0, v2[0], v2[1], p, b2[0], b2[1]])
    sl_a, sr_a = u0 - abs(bn) / math.sqrt(rl), u0 + abs(bn) / math.sqrt(rr)
    # check the construction against the jump conditions of the flux definition
    for (wa, wb, sp) in ((wl, w2l, sl_a), (w2l, w2r, u0), (w2r, wr, sr_a)):
        np.testing.assert_allclose(flux_def(wb, bn, G) - flux_def(wa, bn, G),
                                   sp * (cons_def(wb, bn, G) - cons_def(wa, bn, G)), atol=1e-14)
    if sl_a > 0:
        ref = wl
    elif u0 > 0:
        ref = w2l
    elif sr_a > 0:
        ref = w2r
    else:
        ref = wr
    f = oracle.riemann(1, wl, wr, bn, G)
    np.testing.assert_allclose(f, flux_def(ref, bn, G), rtol=0, atol=3e-14)
