"""Pins of the oracle's full VL2 step against what the paper and the mathematics fix (no GPU).

- second-order L1 convergence of linear waves (Sec. 3.3.1, eq. RMS-error)
- CT keeps div B at round-off (Sec. 2.1.1, 3.1)
- conservation of mass, momentum and energy on periodic meshes (finite-volume form, Sec. 3.1)
- mirror symmetry (Sec. 3.3.5) and identical results along x, y, z (Sec. 3.3.3), bitwise
- exact Riemann solution of Sod-type tubes (hydro, and with a normal field only)
- VL2 = DC predictor over dt/2 then PLM corrector over dt from u^n (Sec. 3.2.3)
- MeshBlock decomposition, thread count and shared-edge EMF copies do not change results
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from exact_riemann import sample
from paper_2005_06651_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
G = 5.0 / 3.0


def cell_b(b1, b2, b3):
    return (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:, :] + b2[:, :-1, :]),
            0.5 * (b3[1:] + b3[:-1]))


def rms_l1_error(state, ref):
    """eq. RMS-error: sqrt(sum_n (mean |U_n - U_n,exact|)^2) over rho, M (3), E, b_c (3)."""
    u, b1, b2, b3 = state
    u0, c1, c2, c3 = ref
    bc, bc0 = cell_b(b1, b2, b3), cell_b(c1, c2, c3)
    e = [np.mean(np.abs(u[v] - u0[v])) for v in range(5)] + [np.mean(np.abs(bc[d] - bc0[d])) for d in range(3)]
    return float(np.sqrt(np.sum(np.square(e))))


def wave_error(oracle, prob):
    m = oracle.Mesh.from_problem(prob)
    ref = m.get_cons()
    m.run(prob.meta["period"], cfl=0.3)
    assert m.floor_count() == 0
    return rms_l1_error(m.get_cons(), ref)


def test_wave_setup_matches_paper_speeds():
    """The wave-frame background b = (1, sqrt 2, 1/2), rho = 1, p = 1/gamma has c_f = 2 (Sec. 3.3.2)."""
    gold = json.load(open(os.path.join(HERE, "golden", "paper_setups.json")))
    s, _ = inputs.wave_eigen("fast", 1.0, np.zeros(3), 1.0 / G, np.array([1.0, math.sqrt(2.0), 0.5]), G)
    assert s == pytest.approx(gold["fast_wave_speed"]["value"], rel=1e-12)
    s, _ = inputs.wave_eigen("alfven", 1.0, np.zeros(3), 1.0 / G, np.array([1.0, math.sqrt(2.0), 0.5]), G)
    assert s == pytest.approx(1.0, rel=1e-12)


@pytest.mark.slow
def test_linear_alfven_wave_second_order_3d(oracle):
    """3D Alfven wave along the cube diagonal: L1 error slope between N = 32 and 64 in [1.8, 2.2]."""
    e32 = wave_error(oracle, inputs.linear_wave(32, mb=16, kind="alfven"))
    e64 = wave_error(oracle, inputs.linear_wave(64, mb=32, kind="alfven"))
    slope = math.log2(e32 / e64)
    assert 1.8 <= slope <= 2.2, (e32, e64, slope)


def _wave2d(kind, n, v0=(0.0, 0.0, 0.0)):
    """Same wave family inclined at 45 degrees in the x-y plane of an n x n x 2 periodic box."""
    p = inputs.linear_wave(n, kind=kind, v0=v0)
    # rebuild with k = 2 pi (1, 1, 0): reuse the generator on a box that is thin in z
    return _inclined(kind, (n, n, 2), (2 * math.pi, 2 * math.pi, 0.0), v0)


def _inclined(kind, nx, kvec, v0, amp=1e-6):
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 1.0, 2.0 / nx[0])
    kvec = np.array(kvec, float)
    kmag = np.linalg.norm(kvec)
    nhat = kvec / kmag
    t1 = np.array([nhat[1], -nhat[0], 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nhat, t1)
    bw = np.array([1.0, math.sqrt(2.0), 0.5])
    bw /= np.linalg.norm(bw)
    v0 = np.asarray(v0, float)
    vw = np.array([v0 @ nhat, v0 @ t1, v0 @ t2])
    speed, r = inputs.wave_eigen(kind, 1.0, vw, 1.0 / G, bw, G)
    x, y, z = inputs._cell_coords(nx, xmin, xmax)
    s = amp * np.sin(kvec[0] * x + kvec[1] * y)
    w = np.empty((5,) + x.shape)
    w[0] = 1 + r[0] * s
    vel = [vw[0] + r[1] * s, vw[1] + r[2] * s, vw[2] + r[3] * s]
    for d in range(3):
        w[1 + d] = vel[0] * nhat[d] + vel[1] * t1[d] + vel[2] * t2[d]
    w[4] = 1 / G + r[4] * s
    av = (-amp * r[6] / kmag) * t1 + (amp * r[5] / kmag) * t2
    (exx, exy, _), (eyx, eyy, _), (ezx, ezy, _) = inputs._edge_coords(nx, xmin, xmax)
    ax = av[0] * np.cos(kvec[0] * exx + kvec[1] * exy)
    ay = av[1] * np.cos(kvec[0] * eyx + kvec[1] * eyy)
    az = av[2] * np.cos(kvec[0] * ezx + kvec[1] * ezy)
    b1, b2, b3 = inputs.faces_from_potential(nx, xmin, xmax, ax, ay, az)
    bg = bw[0] * nhat + bw[1] * t1 + bw[2] * t2
    b1 += bg[0]
    b2 += bg[1]
    b3 += bg[2]
    return inputs.Problem("wave2d", nx, nx, xmin, xmax, G, w, b1, b2, b3,
                          meta={"period": (2 * math.pi / kmag) / abs(speed)})


@pytest.mark.parametrize("kind,v0", [("fast", (0, 0, 0)), ("slow", (0, 0, 0)), ("entropy", (1.0, 0.0, 0.0)),
                                     ("alfven", (0.7, 0.4, 0.2))])
def test_linear_waves_second_order_2d(oracle, kind, v0):
    e1 = wave_error(oracle, _inclined(kind, (32, 32, 2), (2 * math.pi, 2 * math.pi, 0.0), v0))
    e2 = wave_error(oracle, _inclined(kind, (64, 64, 2), (2 * math.pi, 2 * math.pi, 0.0), v0))
    slope = math.log2(e1 / e2)
    assert 1.8 <= slope <= 2.2, (kind, e1, e2, slope)


def _ot(oracle, n=32, mb=16, **kw):
    p = inputs.orszag_tang(n=n, mb=mb, seed=2005)
    return p, oracle.Mesh.from_problem(p, **kw)


def test_divb_and_conservation(oracle):
    p, m = _ot(oracle)
    assert m.divb_norm() <= 1e-13
    t0 = m.totals()
    scale = np.array([t0[0], t0[4], t0[4], t0[4], t0[4]])
    for s in range(6):
        m.step(m.new_dt(0.3))
        assert m.divb_norm() <= 1e-13
        t = m.totals()
        drift = np.abs(t[:5] - t0[:5]) / scale
        assert np.all(drift <= 1e-13 * (s + 1)), drift
        # the cell-centred field average is conserved too on a periodic mesh (sum of face values)
        assert np.all(np.abs(t[5:] - t0[5:]) <= 1e-13 * (s + 1) * max(1.0, np.max(np.abs(t0[5:]))))
    assert m.floor_count() == 0
    assert m.emf_mismatch_count() == 0


def test_block_decomposition_bitwise(oracle):
    """The same 32^3 state as one block, as 8 blocks of 16^3 and as 32 blocks of 8x16x8: identical bits."""
    outs = []
    for mb in [(32, 32, 32), (16, 16, 16), (8, 16, 8)]:
        p, m = _ot(oracle, n=32, mb=mb)
        for _ in range(3):
            m.step(0.004)
        outs.append(m.get_cons())
        assert m.emf_mismatch_count() == 0
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def test_thread_count_bitwise(tmp_path):
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from oracle import orc\nfrom paper_2005_06651_gb300 import inputs\n"
        "p = inputs.orszag_tang(n=32, mb=8, seed=2005); m = orc.Mesh.from_problem(p)\n"
        "[m.step(0.004) for _ in range(2)]\nu, b1, b2, b3 = m.get_cons()\n"
        "np.savez(sys.argv[1], u=u, b1=b1, b2=b2, b3=b3)\n" % (os.path.dirname(HERE), HERE))
    res = []
    for nt in ("1", "3"):
        f = str(tmp_path / ("t%s.npz" % nt))
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        subprocess.run([sys.executable, "-c", code, f], check=True, env=env)
        res.append(np.load(f))
    for k in ("u", "b1", "b2", "b3"):
        np.testing.assert_array_equal(res[0][k], res[1][k])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_bitwise(oracle, axis):
    p = inputs.mirror_symmetric(n=16, mb=8, axis=axis, seed=7 + axis)
    m = oracle.Mesh.from_problem(p)
    for _ in range(4):
        m.step(m.new_dt(0.3))
    u, b1, b2, b3 = m.get_cons()
    npa = 3 - axis  # numpy axis of u (var, z, y, x)
    for v in range(5):
        flipped = np.flip(u[v], axis=npa - 1)
        if v == 1 + axis:
            np.testing.assert_array_equal(u[v], -flipped)
        else:
            np.testing.assert_array_equal(u[v], flipped)
    for c, b in enumerate((b1, b2, b3)):
        flipped = np.flip(b, axis=2 - axis)
        np.testing.assert_array_equal(b, -flipped if c == axis else flipped)


def _tube_profile(oracle, axis, n, t_end, b_n=0.0, riemann=1):
    p = inputs.shock_tube(n=n, axis=axis, b_left=(b_n, 0, 0), b_right=(b_n, 0, 0))
    m = oracle.Mesh.from_problem(p, riemann=riemann)
    m.run(t_end, cfl=0.3)
    u, b1, b2, b3 = m.get_cons()
    return u, (b1, b2, b3), m


def test_axis_permutation_bitwise(oracle):
    """A tube along x, y or z gives the same numbers (Sec. 3.3.3), with the velocity components permuted."""
    outs = [_tube_profile(oracle, ax, 64, 0.05, b_n=0.0)[0] for ax in range(3)]
    for ax in range(3):
        u = outs[ax]
        prof = [u[0].reshape(-1), u[1 + ax].reshape(-1), u[4].reshape(-1)]
        ref = [outs[0][0].reshape(-1), outs[0][1].reshape(-1), outs[0][4].reshape(-1)]
        for a, b in zip(prof, ref):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("b_n", [0.0, 0.75])
@pytest.mark.parametrize("riemann", [1, 0])
def test_sod_tube_converges_to_exact_solution(oracle, b_n, riemann):
    """Sod's tube (gamma = 1.4) against the exact Euler solution; with only a normal field (b_n) the
    exact hydro solution still holds.  L1 density error shrinks under refinement at about first order
    (discontinuities) and is small at N = 512."""
    left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    t = 0.1
    errs = []
    for n in (128, 256, 512):
        p = inputs.shock_tube(n=n, axis=0, b_left=(b_n, 0, 0), b_right=(b_n, 0, 0))
        m = oracle.Mesh.from_problem(p, riemann=riemann)
        m.run(t, cfl=0.3)
        u = m.get_cons()[0]
        rho = u[0].reshape(-1)
        x = (np.arange(n) + 0.5) / n
        # Riemann problems at x = 3/4 (left | right) and x = 1/4 (right | left, mirrored)
        ex = np.where(x > 0.5, sample(left, right, 1.4, (x - 0.75) / t)[0],
                      sample(left, right, 1.4, (0.25 - x) / t)[0])
        errs.append(float(np.mean(np.abs(rho - ex))))
        assert m.floor_count() == 0
    assert errs[2] < 5e-3, errs
    assert errs[0] / errs[1] > 1.4 and errs[1] / errs[2] > 1.4, errs


def test_vl2_is_dc_half_step_then_plm_full_step(oracle):
    """One VL2 cycle equals, to round-off, the composition written from the coefficients the paper
    prints (golden fixture): u^(1/2) = u^n + (dt/2) L_DC(u^n) [RK1 with donor cell], then
    u^(n+1) = u^n + dt L_PLM(u^(1/2)) with L_PLM formed here from the oracle's PLM fluxes/EMFs."""
    gold = json.load(open(os.path.join(HERE, "golden", "paper_setups.json")))["rk2s_coefficients"]
    assert gold["VL2"]["gamma"] == [[0, 1], [0, 1]] and gold["VL2"]["beta"] == [0.5, 1]
    beta0, beta1 = gold["VL2"]["beta"]
    p = inputs.orszag_tang(n=16, mb=8, seed=11)
    dt = 0.01
    a = oracle.Mesh.from_problem(p)
    un = a.get_cons()
    a.step(dt)
    vl2 = a.get_cons()
    b = oracle.Mesh.from_problem(p, integrator=oracle.RK1)
    b.step(beta0 * dt)  # RK1: forward Euler with donor-cell fluxes
    fx, fy, fz = b.debug_fluxes(oracle.PLM)
    e1, e2, e3 = b.debug_emfs(oracle.PLM)
    h = np.array(p.dx)
    u0, c1, c2, c3 = un
    # flux component of each conserved variable in each sweep (cyclic sweep frames)
    comp = {0: [0, 0, 0], 1: [1, 3, 2], 2: [2, 1, 3], 3: [3, 2, 1], 4: [4, 4, 4]}
    out = np.empty_like(u0)
    for v in range(5):
        div = ((fx[comp[v][0]][:, :, 1:] - fx[comp[v][0]][:, :, :-1]) / h[0]
               + (fy[comp[v][1]][:, 1:, :] - fy[comp[v][1]][:, :-1, :]) / h[1]) \
            + (fz[comp[v][2]][1:] - fz[comp[v][2]][:-1]) / h[2]
        out[v] = u0[v] - beta1 * dt * div
    np.testing.assert_allclose(out, vl2[0], rtol=0, atol=1e-13)
    nb1 = c1 - beta1 * dt * ((e3[:, 1:, :] - e3[:, :-1, :]) / h[1] - (e2[1:, :, :] - e2[:-1, :, :]) / h[2])
    nb2 = c2 - beta1 * dt * ((e1[1:, :, :] - e1[:-1, :, :]) / h[2] - (e3[:, :, 1:] - e3[:, :, :-1]) / h[0])
    nb3 = c3 - beta1 * dt * ((e2[:, :, 1:] - e2[:, :, :-1]) / h[0] - (e1[:, 1:, :] - e1[:, :-1, :]) / h[1])
    np.testing.assert_allclose(nb1, vl2[1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(nb2, vl2[2], rtol=0, atol=1e-13)
    np.testing.assert_allclose(nb3, vl2[3], rtol=0, atol=1e-13)


def test_dt_closed_forms(oracle):
    """Uniform states: dt = C0 min_d dx_d / (|v_d| + c_f,d) with textbook fast speeds."""
    nx = (8, 6, 4)
    xmin, xmax = (0.0, 0.0, 0.0), (1.0, 0.9, 0.5)
    h = [(xmax[d] - xmin[d]) / nx[d] for d in range(3)]
    rho, p, v = 1.7, 0.9, (0.3, -0.6, 0.2)
    a = math.sqrt(G * p / rho)
    for bvec in [(0.0, 0.0, 0.0), (0.8, 0.0, 0.0), (0.0, 0.0, 1.1)]:
        w = np.empty((5, nx[2], nx[1], nx[0]))
        w[0], w[1], w[2], w[3], w[4] = rho, v[0], v[1], v[2], p
        b1, b2, b3 = inputs.uniform_faces(nx, bvec)
        m = oracle.Mesh(nx, (4, 3, 2), xmin, xmax, G)
        m.set_prims(w, b1, b2, b3)
        best = []
        for d in range(3):
            bn2 = bvec[d] ** 2
            bt2 = sum(bvec[e] ** 2 for e in range(3) if e != d)
            if bt2 == 0.0:
                cf = max(a, math.sqrt(bn2 / rho))
            elif bn2 == 0.0:
                cf = math.sqrt(a * a + bt2 / rho)
            else:
                raise AssertionError
            best.append(h[d] / (abs(v[d]) + cf))
        assert m.new_dt(0.3) == pytest.approx(0.3 * min(best), rel=1e-14)


def test_cons_prim_round_trip(oracle):
    p = inputs.orszag_tang(n=16, mb=8, seed=3)
    m = oracle.Mesh.from_problem(p)
    w = m.get_prims()
    np.testing.assert_allclose(w[:5], p.w, rtol=1e-14, atol=1e-14)
    bc = cell_b(p.b1, p.b2, p.b3)
    for d in range(3):
        np.testing.assert_array_equal(w[5 + d], bc[d])


def _plm_rhs(oracle, mesh, state, dx):
    """L(U) of a state: -div F and -curl E from the oracle's PLM fluxes and EMFs of that state."""
    mesh.set_cons(*state)
    fx, fy, fz = mesh.debug_fluxes(oracle.PLM)
    e1, e2, e3 = mesh.debug_emfs(oracle.PLM)
    comp = {0: [0, 0, 0], 1: [1, 3, 2], 2: [2, 1, 3], 3: [3, 2, 1], 4: [4, 4, 4]}
    lu = np.empty_like(state[0])
    for v in range(5):
        lu[v] = -(((fx[comp[v][0]][:, :, 1:] - fx[comp[v][0]][:, :, :-1]) / dx[0]
                   + (fy[comp[v][1]][:, 1:, :] - fy[comp[v][1]][:, :-1, :]) / dx[1])
                  + (fz[comp[v][2]][1:] - fz[comp[v][2]][:-1]) / dx[2])
    lb1 = -((e3[:, 1:, :] - e3[:, :-1, :]) / dx[1] - (e2[1:, :, :] - e2[:-1, :, :]) / dx[2])
    lb2 = -((e1[1:, :, :] - e1[:-1, :, :]) / dx[2] - (e3[:, :, 1:] - e3[:, :, :-1]) / dx[0])
    lb3 = -((e2[:, :, 1:] - e2[:, :, :-1]) / dx[0] - (e1[:, 1:, :] - e1[:, :-1, :]) / dx[1])
    return lu, lb1, lb2, lb3


@pytest.mark.parametrize("name", ["RK2", "RK3"])
def test_rk_cycle_is_the_printed_2s_stages(oracle, name):
    """One RK2 / RK3 cycle of the oracle equals, to round-off, eq. rk-2s composed here from the
    coefficients the paper prints (golden fixture): u1 = u0 (delta_0 = 1), then per stage
    u0 = gamma_s0 u0 + gamma_s1 u1 + beta_s dt L_PLM(u0), with L_PLM formed here from the oracle's PLM
    fluxes and EMFs of each stage's state."""
    gold = json.load(open(os.path.join(HERE, "golden", "paper_setups.json")))["rk2s_coefficients"][name]
    p = inputs.orszag_tang(n=16, mb=8, seed=11)
    dt = 0.005
    a = oracle.Mesh.from_problem(p, integrator=getattr(oracle, name))
    u0 = [np.array(x) for x in a.get_cons()]
    a.step(dt)
    ref = a.get_cons()
    helper = oracle.Mesh.from_problem(p)
    u1 = [x.copy() for x in u0]
    for (g0, g1), beta in zip(gold["gamma"], gold["beta"]):
        L = _plm_rhs(oracle, helper, u0, np.array(p.dx))
        u0 = [(g0 * x0 + g1 * x1) + beta * dt * lx for x0, x1, lx in zip(u0, u1, L)]
    for got, want in zip(ref, u0):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("integrator", ["RK2", "RK3"])
def test_rk_integrators_second_order_2d(oracle, integrator):
    """RK2 and RK3 with PLM fluxes on the inclined fast wave: L1 slope 48 -> 96 in [1.8, 2.2] (PLM limits
    the order to 2; observed 1.90 and 1.93 here, 1.97 and 1.99 at 64 -> 128, 1.80 and 1.84 at 32 -> 64)."""
    errs = []
    for n in (48, 96):
        prob = _inclined("fast", (n, n, 2), (2 * math.pi, 2 * math.pi, 0.0), (0.0, 0.0, 0.0))
        m = oracle.Mesh.from_problem(prob, integrator=getattr(oracle, integrator))
        ref = m.get_cons()
        m.run(prob.meta["period"], cfl=0.3)
        assert m.floor_count() == 0
        errs.append(rms_l1_error(m.get_cons(), ref))
    slope = math.log2(errs[0] / errs[1])
    print("%s + PLM fast wave: L1 %.3e -> %.3e, slope %.3f" % (integrator, errs[0], errs[1], slope))
    assert 1.8 <= slope <= 2.2, (integrator, errs, slope)


def test_blast_setup_and_pressure_floor(oracle):
    """The blast holds the stated internal energy inside r0 on a uniform field; in its low-beta ambient the
    pressure floor (reading 2) fires in the first donor-cell cycle, and each floored cell then holds
    p = pfloor up to the rounding of E, with mass untouched and div B still at round-off."""
    prob = inputs.blast(32, mb=16, r0=0.1, magnetized=True)
    dv = 1.0 / 32 ** 3
    inside = prob.w[4] > 1e-3
    assert int(inside.sum()) == prob.meta["cells_inside"] > 0
    assert np.sum(prob.w[4][inside]) / (G - 1.0) * dv == pytest.approx(1.0, rel=1e-13)
    assert np.all(prob.w[4][~inside] == 1e-3) and np.all(prob.w[0] == 1.0)
    assert np.all(prob.b1 == math.sqrt(3.0)) and np.all(prob.b2 == 1.0) and np.all(prob.b3 == 0.0)
    o = oracle.Mesh.from_problem(prob, riemann=oracle.HLLD, integrator=oracle.RK1)
    m0 = o.totals()[0]
    o.step(o.new_dt(0.3))
    assert o.floor_count() == 0
    o.new_dt(0.3)
    fired = o.floor_count()
    assert fired > 0
    u = o.get_cons()[0]
    w = o.get_prims()  # recomputes p = (gamma-1)(E - ke - me) from the rewritten E
    tol = 8 * np.finfo(float).eps * (G - 1.0) * u[4]  # a few ulps of E
    floored = np.abs(w[4] - 1e-12) <= tol
    assert int(floored.sum()) >= 1
    assert np.all(w[4] >= 1e-12 - tol)
    assert o.totals()[0] == pytest.approx(m0, rel=1e-14)
    assert o.divb_norm() <= 1e-13
