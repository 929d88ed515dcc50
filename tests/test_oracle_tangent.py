"""Pins of the oracle's tangent-linear (dual numbers) of one VL2 cycle: it matches central finite
differences of the oracle's own cycle, is linear in the direction, and leaves the state untouched."""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs


def smooth_state(oracle, n=8, v0=(0.7, 0.4, 0.2)):
    prob = inputs.linear_wave(n, mb=n // 2, kind="fast", amp=1e-2, v0=v0)
    m = oracle.Mesh.from_problem(prob)
    geom = (prob.nx, prob.mb, prob.xmin, prob.xmax, prob.bc)
    return prob, geom, m.get_cons(), m.new_dt(0.3)


def direction(state, seed, scale):
    rng = np.random.default_rng(seed)
    u, b1, b2, b3 = state
    du = scale * rng.standard_normal(u.shape)
    # a divergence-free field direction keeps the periodic duplicates consistent: use zero for B here
    # except a uniform shift (exactly divergence free and periodic)
    db = [np.full_like(b, scale * rng.standard_normal()) for b in (b1, b2, b3)]
    return (du,) + tuple(db)


def test_tangent_linear_matches_central_differences(oracle):
    prob, geom, x, dt = smooth_state(oracle)
    d = direction(x, 1, 1.0)
    y, jd = oracle.tl_step(geom, dt, x, d, gamma=prob.gamma)
    y0 = oracle.step_cons(geom, dt, x, gamma=prob.gamma)
    for a, b in zip(y, y0):
        np.testing.assert_array_equal(a, b)  # the value part is the plain cycle
    h = 1e-7
    xp = tuple(a + h * t for a, t in zip(x, d))
    xm = tuple(a - h * t for a, t in zip(x, d))
    yp = oracle.step_cons(geom, dt, xp, gamma=prob.gamma)
    ym = oracle.step_cons(geom, dt, xm, gamma=prob.gamma)
    for a, b, j in zip(yp, ym, jd):
        fd = (a - b) / (2 * h)
        scale = np.max(np.abs(j)) + 1e-30
        assert np.max(np.abs(fd - j)) / scale <= 1e-6


def test_tangent_linear_is_linear(oracle):
    prob, geom, x, dt = smooth_state(oracle)
    d1, d2 = direction(x, 2, 1.0), direction(x, 3, 1.0)
    _, j1 = oracle.tl_step(geom, dt, x, d1, gamma=prob.gamma)
    _, j2 = oracle.tl_step(geom, dt, x, d2, gamma=prob.gamma)
    _, j12 = oracle.tl_step(geom, dt, x, tuple(2.0 * a - 3.0 * b for a, b in zip(d1, d2)), gamma=prob.gamma)
    for a, b, c in zip(j1, j2, j12):
        np.testing.assert_allclose(c, 2.0 * a - 3.0 * b, rtol=0, atol=1e-12 * (np.max(np.abs(c)) + 1e-30))


def riemann_states(n, seed):
    """Random interface states (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) and normal fields spanning the HLLD
    regions: slow and supersonic normal flow, weak and strong fields."""
    rng = np.random.default_rng(seed)
    wl = np.column_stack([rng.uniform(0.2, 5.0, n), rng.uniform(-4, 4, n), rng.uniform(-2, 2, (n, 2)),
                          rng.uniform(0.05, 5.0, n), rng.uniform(-2, 2, (n, 2))])
    wr = np.column_stack([rng.uniform(0.2, 5.0, n), rng.uniform(-4, 4, n), rng.uniform(-2, 2, (n, 2)),
                          rng.uniform(0.05, 5.0, n), rng.uniform(-2, 2, (n, 2))])
    bn = rng.uniform(-2, 2, n)
    return wl, wr, bn


@pytest.mark.parametrize("solver", [0, 1])
def test_riemann_jacobian_matches_central_differences(oracle, solver):
    """The oracle's dual-number Riemann Jacobian (used to check the GPU adjoint) against central
    differences of the oracle's own flux, column by column."""
    wl, wr, bn = riemann_states(200, 11 + solver)
    jac = oracle.riemann_jacobian(solver, wl, wr, bn, 5.0 / 3.0)
    h = 1e-6
    worst = 0.0
    for q in range(len(bn)):
        x = np.concatenate([wl[q], wr[q], [bn[q]]])
        for k in range(15):
            xp, xm = x.copy(), x.copy()
            xp[k] += h
            xm[k] -= h
            fp = oracle.riemann(solver, xp[:7], xp[7:14], xp[14], 5.0 / 3.0)
            fm = oracle.riemann(solver, xm[:7], xm[7:14], xm[14], 5.0 / 3.0)
            fd = (fp - fm) / (2 * h)
            scale = max(1.0, float(np.max(np.abs(jac[q]))))
            err = float(np.max(np.abs(fd - jac[q, :, k]))) / scale
            # a difference across a region switch (a wave speed through zero) is not a derivative: skip
            # the few columns where the two one-sided differences disagree
            f0 = oracle.riemann(solver, x[:7], x[7:14], x[14], 5.0 / 3.0)
            one_sided = np.max(np.abs((fp - f0) / h - (f0 - fm) / h)) / scale
            if one_sided > 1e-3:
                continue
            worst = max(worst, err)
    print("oracle Riemann Jacobian vs central differences (solver %d): worst %.2e" % (solver, worst))
    assert worst <= 1e-6
