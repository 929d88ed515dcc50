"""Pins of the oracle's HLLE with Einfeldt's outer speeds (Roe-averaged fast speed, Sec. 3.2.2 names the
solver and Roe's linearisation) against what the mathematics fixes, without a GPU.

- equal states give the physical flux, and the same flux as HLLE with the states' own speeds
- gas dynamics (no field): the test's Roe averages u~, H~ satisfy Roe's property A(u~, H~) dU = dF for the
  Euler Jacobian (textbook), and the oracle's flux is the HLL flux with S_L = min(u_L - a_L, u~ - a~),
  S_R = max(u_R + a_R, u~ + a~)
- with a field but equal densities and transverse fields (X = 0, Y = 1 in the MHD Roe average) the flux
  is the HLL flux with the fast speed of the averaged state, a~^2 = (gamma-1)(H~ - u~^2/2 - B^2/rho)
- the scheme: mirror symmetry and MeshBlock independence bitwise; density and pressure stay positive
  through the strong double rarefaction where a linearised solver loses positivity
X and Y themselves are pinned only through those limits (parity partially pinned).
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
