"""Pins of the oracle's HLLE with Einfeldt's outer speeds (Roe-averaged fast speed, Sec. 3.2.2 names the
solver and Roe's linearisation) against what the mathematics fixes, without a GPU.

- equal states give the physical flux, and the same flux as HLLE with the states' own speeds
- gas dynamics (no field): the test's Roe averages u~, H~ satisfy Roe's property A(u~, H~) dU = dF for the
  Euler Jacobian (textbook), and the oracle's flux is the HLL flux with S_L = min(u_L - a_L, u~ - a~),
  S_R = max(u_R + a_R, u~ + a~)
- MHD, unequal densities and transverse fields: a Roe matrix of the 1D ideal-MHD flux is built here, row by
  row, from exact difference identities (no X, no closed-form speed in it); it satisfies Roe's property
  A dU = dF to round-off, and its extreme eigenvalues are the oracle's u~ -+ c~_f
- MHD, two states joined by one exact fast shock (Rankine-Hugoniot conditions solved here): Roe's property
  makes the shock speed an eigenvalue of every Roe matrix, so u~ -+ c~_f is the shock speed and Einfeldt's
  HLLE returns the exact upwind flux; X > 0 and rho_L != rho_R there
- with a field but equal densities and transverse fields the flux is the HLL flux with the fast speed of
  the averaged state, a~^2 = (gamma-1)(H~ - u~^2/2 - B^2/rho)
- the scheme: mirror symmetry and MeshBlock independence bitwise; density and pressure stay positive
  through the strong double rarefaction where a linearised solver loses positivity
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

G = 5.0 / 3.0


def cons(w, bn, g):
    rho, u, v, wz, p, b1, b2 = w
    e = p / (g - 1) + 0.5 * rho * (u * u + v * v + wz * wz) + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    return np.array([rho, rho * u, rho * v, rho * wz, e, b1, b2])


def hll(oracle, wl, wr, bn, g, sl, sr):
    fl, fr = oracle.riemann(0, wl, wl, bn, g), oracle.riemann(0, wr, wr, bn, g)  # physical fluxes
    ul, ur = cons(wl, bn, g), cons(wr, bn, g)
    bm, bp = min(sl, 0.0), max(sr, 0.0)
    return ((bp * fl - bm * fr) + bp * bm * (ur - ul)) / (bp - bm)


def fast(w, bn, g):
    rho, p = w[0], w[4]
    a2, ca2, ct2 = g * p / rho, bn * bn / rho, (w[5] ** 2 + w[6] ** 2) / rho
    return np.sqrt(0.5 * (a2 + ca2 + ct2 + np.sqrt((ca2 + ct2 - a2) ** 2 + 4 * a2 * ct2)))


def test_equal_states(oracle):
    rng = np.random.default_rng(1)
    for _ in range(100):
        w = np.array([rng.uniform(0.2, 3), *rng.uniform(-2, 2, 3), rng.uniform(0.05, 3), *rng.uniform(-2, 2, 2)])
        bn = rng.uniform(-2, 2)
        f = oracle.riemann(2, w, w, bn, G)
        np.testing.assert_allclose(f, oracle.riemann(0, w, w, bn, G), rtol=1e-14, atol=1e-14)


def euler_jacobian(u, h, g):
    """Jacobian dF_x/dU of the 3D Euler equations at velocity u = (u, v, w) and total enthalpy h."""
    ux, uy, uz = u
    q2 = ux * ux + uy * uy + uz * uz
    gm = g - 1
    return np.array([
        [0, 1, 0, 0, 0],
        [0.5 * gm * q2 - ux * ux, (3 - g) * ux, -gm * uy, -gm * uz, gm],
        [-ux * uy, uy, ux, 0, 0],
        [-ux * uz, uz, 0, ux, 0],
        [ux * (0.5 * gm * q2 - h), h - gm * ux * ux, -gm * ux * uy, -gm * ux * uz, g * ux]])


def test_gas_dynamics_einfeldt_speeds(oracle):
    rng = np.random.default_rng(2)
    g = 1.4
    for _ in range(200):
        wl = np.array([rng.uniform(0.1, 5), *rng.uniform(-3, 3, 3), rng.uniform(0.05, 5), 0.0, 0.0])
        wr = np.array([rng.uniform(0.1, 5), *rng.uniform(-3, 3, 3), rng.uniform(0.05, 5), 0.0, 0.0])
        sl_, sr_ = np.sqrt(wl[0]), np.sqrt(wr[0])
        ut = (sl_ * wl[1:4] + sr_ * wr[1:4]) / (sl_ + sr_)
        hl = (cons(wl, 0.0, g)[4] + wl[4]) / wl[0]
        hr = (cons(wr, 0.0, g)[4] + wr[4]) / wr[0]
        ht = (sl_ * hl + sr_ * hr) / (sl_ + sr_)
        # Roe's property pins these averages
        ul, ur = cons(wl, 0.0, g)[:5], cons(wr, 0.0, g)[:5]
        fl, fr = oracle.riemann(0, wl, wl, 0.0, g)[:5], oracle.riemann(0, wr, wr, 0.0, g)[:5]
        np.testing.assert_allclose(euler_jacobian(ut, ht, g) @ (ur - ul), fr - fl, rtol=1e-12, atol=1e-12)
        at = np.sqrt((g - 1) * (ht - 0.5 * ut @ ut))
        sl = min(wl[1] - np.sqrt(g * wl[4] / wl[0]), ut[0] - at)
        sr = max(wr[1] + np.sqrt(g * wr[4] / wr[0]), ut[0] + at)
        np.testing.assert_allclose(oracle.riemann(2, wl, wr, 0.0, g), hll(oracle, wl, wr, 0.0, g, sl, sr),
                                   rtol=1e-12, atol=1e-12)


def mhd_flux(w, bn, g):
    """Physical x-flux of 1D ideal MHD for the primitive state w = (rho, u, v, w, p, b_y, b_z)."""
    rho, u, v, wz, p, b1, b2 = w
    e = cons(w, bn, g)[4]
    pt = p + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    vb = u * bn + v * b1 + wz * b2
    return np.array([rho * u, rho * u * u + pt - bn * bn, rho * u * v - bn * b1, rho * u * wz - bn * b2,
                     (e + pt) * u - bn * vb, b1 * u - bn * v, b2 * u - bn * wz])


def roe_matrix(wl, wr, bn, g):
    """A Roe matrix of the 1D ideal-MHD flux in the conserved variables (rho, M, E, b_y, b_z), written row by
    row from exact identities for the difference of each flux term between the two states.  With s = sqrt(rho),
    rho~ = s_L s_R and sqrt(rho)-weighted averages v~ and H~ = (E + p_T)/rho:
      d(M_a M_b / rho) = v~_a dM_b + v~_b dM_a - v~_a v~_b d(rho)
      d(v_a)           = (dM_a - v~_a d(rho)) / rho~
      d(rho H v_n)     = H~ dM_n + v~_n d(rho H) - v~_n H~ d(rho),   d(rho H) = dE + d(p_T)
      d(b v_a)         = v~_a db + b* d(v_a)   with the cross-weighted b* = (s_R b_L + s_L b_R)/(s_L + s_R)
      d(|b_t|^2 / 2)   = b* . db_t + X d(rho),  X = |b_t,R - b_t,L|^2 / (2 (s_L + s_R)^2)
                         (the arithmetic mean of b_t minus b* is (s_R - s_L) db_t / (2 (s_L + s_R)), and
                         d(rho) = (s_R - s_L)(s_L + s_R))
      d(p_T)           = (gamma-1)(dE - v~ . dM + |v~|^2/2 d(rho)) - (gamma-2)(b* . db_t + X d(rho))
    Each identity is exact for any two states, so A dU = dF holds to round-off.  Writing the magnetic
    pressure through b* keeps one averaged transverse field in every row; X then sits in the density
    column.  (Through the arithmetic mean instead, A would be another Roe matrix with other eigenvalues
    away from shocks; every Roe matrix has the speed of a single shock joining the two states as an
    eigenvalue.)"""
    sl, sr = np.sqrt(wl[0]), np.sqrt(wr[0])
    rt = sl * sr
    v = (sl * wl[1:4] + sr * wr[1:4]) / (sl + sr)
    h = [(cons(w, bn, g)[4] + w[4] + 0.5 * (bn * bn + w[5] ** 2 + w[6] ** 2)) / w[0] for w in (wl, wr)]
    ht = (sl * h[0] + sr * h[1]) / (sl + sr)
    bstar = (sr * wl[5:7] + sl * wr[5:7]) / (sl + sr)
    db = wr[5:7] - wl[5:7]
    x = db @ db / (2 * (sl + sr) ** 2)
    dpt = np.zeros(7)
    dpt[0] = (g - 1) * 0.5 * v @ v - (g - 2) * x
    dpt[1:4] = -(g - 1) * v
    dpt[4] = g - 1
    dpt[5:7] = -(g - 2) * bstar
    dv = np.zeros((3, 7))
    for a in range(3):
        dv[a, 1 + a] = 1.0 / rt
        dv[a, 0] = -v[a] / rt
    A = np.zeros((7, 7))
    A[0, 1] = 1.0
    A[1] = dpt
    A[1, 1] += 2 * v[0]
    A[1, 0] -= v[0] * v[0]
    for c in range(2):
        A[2 + c, 2 + c] += v[0]
        A[2 + c, 1] += v[1 + c]
        A[2 + c, 0] -= v[0] * v[1 + c]
        A[2 + c, 5 + c] -= bn
    drh = dpt.copy()
    drh[4] += 1.0
    A[4] = v[0] * drh
    A[4, 1] += ht
    A[4, 0] -= v[0] * ht
    A[4] -= bn * bn * dv[0]
    for c in range(2):
        A[4] -= bn * bstar[c] * dv[1 + c]
        A[4, 5 + c] -= bn * v[1 + c]
        A[5 + c] = bstar[c] * dv[0] - bn * dv[1 + c]
        A[5 + c, 5 + c] += v[0]
    return A


def random_pair(rng):
    def one():
        return np.array([rng.uniform(0.2, 3), *rng.uniform(-2, 2, 3), rng.uniform(0.05, 3), *rng.uniform(-2, 2, 2)])
    return one(), one(), rng.uniform(-2, 2)


def test_mhd_roe_matrix_property_and_fast_eigenvalues(oracle):
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(1000):
        wl, wr, bn = random_pair(rng)
        A = roe_matrix(wl, wr, bn, G)
        du = cons(wr, bn, G) - cons(wl, bn, G)
        df = mhd_flux(wr, bn, G) - mhd_flux(wl, bn, G)
        np.testing.assert_allclose(A @ du, df, rtol=0, atol=1e-12 * (1 + np.abs(df).max()))
        lam = np.linalg.eigvals(A)
        assert np.abs(lam.imag).max() <= 1e-6 * np.abs(lam.real).max()
        lam = np.sort(lam.real)
        un, cf = oracle.roe_fast_speed(wl, wr, bn, G)
        err = max(abs(lam[-1] - (un + cf)), abs(lam[0] - (un - cf))) / cf
        worst = max(worst, err)
    print("Roe matrix: max relative gap of the extreme eigenvalues to u~ -+ c~_f: %.2e" % worst)
    assert worst <= 1e-10


def fast_shock(rho1, p1, bn, bt1, r, g):
    """Upstream (left, flowing in at u1 > 0) and downstream states of a fast shock at rest, compression r,
    from the Rankine-Hugoniot conditions: mass, transverse momentum, induction and normal momentum fix the
    downstream state for a given u1; the energy condition fixes u1 (root between the upstream fast speed and
    20 times it)."""
    from scipy.optimize import brentq

    def down(u1):
        m = rho1 * u1
        b2 = bt1 * r * (rho1 * u1 * u1 - bn * bn) / (rho1 * u1 * u1 - r * bn * bn)
        v2 = bn * (b2 - bt1) / m
        p2 = p1 + m * (u1 - u1 / r) + 0.5 * (bt1 * bt1 - b2 * b2)
        return (np.array([rho1, u1, 0.0, 0.0, p1, bt1, 0.0]), np.array([rho1 * r, u1 / r, v2, 0.0, p2, b2, 0.0]))

    def energy_jump(u1):
        wa, wb = down(u1)
        return mhd_flux(wb, bn, g)[4] - mhd_flux(wa, bn, g)[4]

    c1 = np.sqrt(fast(np.array([rho1, 0, 0, 0, p1, bt1, 0.0]), bn, g) ** 2)
    us = np.linspace(c1 * 1.0001, 20 * c1, 2000)
    f = [energy_jump(u) for u in us]
    for a in range(len(us) - 1):
        if f[a] * f[a + 1] < 0:
            u1 = brentq(energy_jump, us[a], us[a + 1], xtol=1e-15, rtol=1e-15)
            return down(u1)
    return None


def boost(w, bn, vx, vt, theta):
    """The state in a frame moving with (-vx, -vt): velocities shifted, the transverse plane rotated by theta."""
    c, s = np.cos(theta), np.sin(theta)
    rho, u, v, wz, p, b1, b2 = w
    vy, vz = c * v - s * wz + vt[0], s * v + c * wz + vt[1]
    by, bz = c * b1 - s * b2, s * b1 + c * b2
    return np.array([rho, u + vx, vy, vz, p, by, bz])


def test_exact_fast_shocks_move_at_the_roe_fast_speed(oracle):
    rng = np.random.default_rng(12)
    checked = 0
    for _ in range(60):
        rho1, p1 = rng.uniform(0.3, 2), rng.uniform(0.1, 2)
        bn, bt1 = rng.uniform(0.1, 1.5) * rng.choice([-1, 1]), rng.uniform(0.1, 1.5)
        r = rng.uniform(1.1, 3.6)
        pair = fast_shock(rho1, p1, bn, bt1, r, G)
        if pair is None:
            continue
        wa, wb = pair
        s = -rng.uniform(0.01, 0.4) * wb[1]    # the shock moves left, slower than the downstream flow
        vt, theta = rng.uniform(-1, 1, 2), rng.uniform(0, 2 * np.pi)
        wl, wr = boost(wa, bn, s, vt, theta), boost(wb, bn, s, vt, theta)
        du = cons(wr, bn, G) - cons(wl, bn, G)
        df = mhd_flux(wr, bn, G) - mhd_flux(wl, bn, G)
        scale = np.abs(mhd_flux(wr, bn, G)).max()
        assert np.abs(df - s * du).max() <= 1e-12 * scale        # Rankine-Hugoniot
        un, cf = oracle.roe_fast_speed(wl, wr, bn, G)
        assert abs((un - cf) - s) <= 1e-12 * cf
        # S_L = s exactly, so Einfeldt's HLLE returns the flux of the right (downstream) state
        np.testing.assert_allclose(oracle.riemann(2, wl, wr, bn, G), mhd_flux(wr, bn, G), rtol=0,
                                   atol=1e-12 * scale)
        # the mirror image: a right-facing shock moving right, upwind flux of the left state
        mir = np.array([1, -1, 1, 1, 1, 1, 1.0])
        ml, mr = wr * mir, wl * mir
        un, cf = oracle.roe_fast_speed(ml, mr, -bn, G)
        assert abs((un + cf) + s) <= 1e-12 * cf
        np.testing.assert_allclose(oracle.riemann(2, ml, mr, -bn, G), mhd_flux(ml, -bn, G), rtol=0,
                                   atol=1e-12 * scale)
        checked += 1
    assert checked >= 40


def test_mhd_equal_density_and_field(oracle):
    rng = np.random.default_rng(3)
    for _ in range(200):
        rho = rng.uniform(0.2, 3)
        bt = rng.uniform(-2, 2, 2)
        bn = rng.uniform(-2, 2)
        wl = np.array([rho, *rng.uniform(-2, 2, 3), rng.uniform(0.05, 3), *bt])
        wr = np.array([rho, *rng.uniform(-2, 2, 3), rng.uniform(0.05, 3), *bt])
        ut = 0.5 * (wl[1:4] + wr[1:4])
        h = [(cons(w, bn, G)[4] + w[4] + 0.5 * (bn * bn + bt @ bt)) / rho for w in (wl, wr)]
        ht = 0.5 * (h[0] + h[1])
        a2 = (G - 1) * (ht - 0.5 * ut @ ut - (bn * bn + bt @ bt) / rho)
        # the averaged state's fast speed (X = 0, Y = 1): sound speed a~, the common field
        wt = np.array([rho, *ut, a2 * rho / G, *bt])
        cft = fast(wt, bn, G)
        sl = min(wl[1] - fast(wl, bn, G), ut[0] - cft)
        sr = max(wr[1] + fast(wr, bn, G), ut[0] + cft)
        np.testing.assert_allclose(oracle.riemann(2, wl, wr, bn, G), hll(oracle, wl, wr, bn, G, sl, sr),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 2])
def test_hlle_roe_mirror_and_blocks(oracle, axis):
    p = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=71 + axis)
    ms = [oracle.Mesh.from_problem(p, riemann=oracle.HLLE_ROE, mb=mb) for mb in ((8, 8, 8), (16, 16, 16))]
    for _ in range(3):
        dt = ms[0].new_dt(0.3)
        for m in ms:
            m.step(dt)
    u, b1, b2, b3 = ms[0].get_cons()
    npa = 3 - axis
    for v in range(5):
        flipped = np.flip(u[v], axis=npa - 1)
        np.testing.assert_array_equal(u[v], -flipped if v == 1 + axis else flipped)
    assert all(np.array_equal(a, b) for a, b in zip(ms[0].get_cons(), ms[1].get_cons()))


def test_double_rarefaction_stays_positive(oracle):
    """Einfeldt's speeds bound the fan of two strong rarefactions (u = -+2, the '1-2-3' problem), so
    density and pressure stay positive without floors."""
    prob = inputs.shock_tube(128, axis=0, left=(1.0, 2.0, 0.0, 0.0, 0.4), right=(1.0, -2.0, 0.0, 0.0, 0.4),
                             gamma=1.4)
    m = oracle.Mesh.from_problem(prob, riemann=oracle.HLLE_ROE, mb=(32, 1, 1), dfloor=1e-300, pfloor=1e-300)
    m.run(0.1, cfl=0.4)
    u = m.get_cons()[0]
    rho = u[0]
    p = (1.4 - 1) * (u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / rho)
    print("double rarefaction: min rho %.3e, min p %.3e, floors %d" % (rho.min(), p.min(), m.floor_count()))
    assert rho.min() > 0 and p.min() > 0 and m.floor_count() == 0
