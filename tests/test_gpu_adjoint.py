"""Adjoint of the VL2 cycle on the GPU (vl2_step_vjp) and the checkpointed rollout gradient.

- dot-product test: <J dx, y> with J dx from the oracle's dual-number tangent-linear (CPU) equals
  <dx, J^T y> with J^T y from the GPU adjoint, to 1e-12 relative;
- central finite differences of the GPU cycle agree with J^T y along random directions (1e-6 relative);
- the gradient of a loss after many cycles (torch.autograd.Function with sqrt(N) checkpointing) agrees
  with central finite differences of the same rollout (same fixed steps) to 1e-6 relative.
Inputs are smooth waves advected by a background flow, so that no mass flux changes sign and limiter
switches are not crossed by the perturbations.
"""
import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

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


def smooth(n=12, mb=6, amp=1e-2, kind="fast"):
    return inputs.linear_wave(n, mb=mb, kind=kind, amp=amp, v0=(0.7, 0.4, 0.2))


def periodic_direction(state, rng, scale=1.0):
    """Random direction on the conserved state, with periodic duplicate faces equal (face N == face 0)."""
    u, b1, b2, b3 = state
    du = scale * rng.standard_normal(u.shape)
    d1 = scale * rng.standard_normal(b1.shape)
    d1[:, :, -1] = d1[:, :, 0]
    d2 = scale * rng.standard_normal(b2.shape)
    d2[:, -1, :] = d2[:, 0, :]
    d3 = scale * rng.standard_normal(b3.shape)
    d3[-1, :, :] = d3[0, :, :]
    return du, d1, d2, d3


def to_dev(arrs):
    import torch

    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)


def dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


def absdot(a, b):
    return sum(float(np.sum(np.abs(x * y))) for x, y in zip(a, b))


@pytest.mark.parametrize("riemann", [1, 0])
def test_dot_product_gpu_adjoint_vs_oracle_tangent_linear(vl2, oracle, riemann):
    prob = smooth()
    g = vl2.Mesh.from_problem(prob, adjoint=True, riemann=riemann)
    x = g.get_cons()
    dt = g.new_dt()
    rng = np.random.default_rng(7)
    dx = periodic_direction(x, rng)
    y = tuple(rng.standard_normal(a.shape) for a in x)
    geom = (prob.nx, prob.mb, prob.xmin, prob.xmax, prob.bc)
    _, jdx = oracle.tl_step(geom, dt, x, dx, gamma=prob.gamma, riemann=riemann)
    lhs = dot(jdx, y)
    jty = g.step_vjp(dt, to_dev(y))
    jty = tuple(t.cpu().numpy() for t in jty)
    rhs = dot(dx, jty)
    scale = absdot(jdx, y)
    print("dot-product test (riemann %d): <J dx, y> = %.15e, <dx, J^T y> = %.15e, rel %.2e"
          % (riemann, lhs, rhs, abs(lhs - rhs) / scale))
    assert abs(lhs - rhs) <= 1e-12 * scale


@pytest.mark.parametrize("layout", ["blocks_2x1x3", "outflow_xz", "outflow_all_2x2x2"])
def test_dot_product_uneven_blocks_and_outflow(vl2, oracle, layout):
    """Ghost-exchange transposes beyond the periodic cube of equal blocks: 2 x 1 x 3 blocks (a direction
    with one block wraps onto itself), outflow boundaries on x and z, and outflow everywhere."""
    P, O = vl2.PERIODIC, vl2.OUTFLOW
    mb, bc = {"blocks_2x1x3": ((6, 12, 4), (P,) * 6),
              "outflow_xz": ((6, 6, 6), (O, O, P, P, O, O)),
              "outflow_all_2x2x2": ((6, 6, 6), (O,) * 6)}[layout]
    prob = smooth()
    g = vl2.Mesh(prob.nx, mb, prob.xmin, prob.xmax, prob.gamma, bc=bc, adjoint=True)
    g.set_prims(prob.w, prob.b1, prob.b2, prob.b3)
    x = g.get_cons()
    dt = g.new_dt()
    rng = np.random.default_rng(17)
    dx = periodic_direction(x, rng)
    y = tuple(rng.standard_normal(a.shape) for a in x)
    geom = (prob.nx, mb, prob.xmin, prob.xmax, bc)
    _, jdx = oracle.tl_step(geom, dt, x, dx, gamma=prob.gamma, riemann=1)
    lhs = dot(jdx, y)
    rhs = dot(dx, [t.cpu().numpy() for t in g.step_vjp(dt, to_dev(y))])
    scale = absdot(jdx, y)
    print("dot-product test (%s): rel %.2e" % (layout, abs(lhs - rhs) / scale))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_adjoint_matches_central_differences_of_the_gpu_cycle(vl2):
    prob = smooth(n=12, mb=6)
    g = vl2.Mesh.from_problem(prob, adjoint=True)
    x = g.get_cons()
    dt = g.new_dt()
    rng = np.random.default_rng(11)
    y = tuple(rng.standard_normal(a.shape) for a in x)
    g.set_cons(*x)
    jty = tuple(t.cpu().numpy() for t in g.step_vjp(dt, to_dev(y)))
    for trial in range(3):
        d = periodic_direction(x, rng)
        h = 1e-6
        vals = []
        for sgn in (1.0, -1.0):
            g.set_cons(*[a + sgn * h * b for a, b in zip(x, d)])
            g.step(dt)
            vals.append(dot(g.get_cons(), y))
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = dot(jty, d)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (trial, fd, ad)


def smooth_direction(prob, rng):
    """Low-wavenumber velocity direction with random phases: a small step along it does not move a
    smooth flow across the limiter's switch, where the map is not differentiable."""
    import torch

    x, y, z = inputs._cell_coords(prob.nx, prob.xmin, prob.xmax)
    ph = rng.uniform(0, 2 * np.pi, size=(3, 3))
    d = np.stack([np.sin(2 * np.pi * x + ph[c, 0]) * np.cos(2 * np.pi * y + ph[c, 1]) *
                  np.sin(2 * np.pi * z + ph[c, 2]) for c in range(3)])
    return torch.from_numpy(np.ascontiguousarray(d)).cuda()


def rollout_fd_check(n, mb, nsteps, every, ndir, h):
    import torch

    from paper_2005_06651_gb300 import adjoint

    prob = inputs.linear_wave(n, mb=mb, kind="fast", amp=1e-2, v0=(0.7, 0.4, 0.2))
    runner = adjoint.Rollout(prob, nsteps=nsteps, checkpoint_every=every)
    rng = np.random.default_rng(5005)
    target = torch.from_numpy(prob.w[0] + 0.01 * rng.standard_normal(prob.w[0].shape)).cuda()
    dv = float(np.prod(prob.dx))
    v0 = torch.from_numpy(np.ascontiguousarray(prob.w[1:4])).cuda().requires_grad_(True)
    u = adjoint.rollout(v0, runner)
    loss = ((u[0] - target) ** 2).sum() * dv
    loss.backward()
    grad = v0.grad.detach().clone()
    runner.fixed_dts = list(runner.dts)  # finite differences at the same steps
    for trial in range(ndir):
        d = smooth_direction(prob, rng)
        vals = []
        for sgn in (1.0, -1.0):
            with torch.no_grad():
                uu = runner.run_forward(v0.detach() + sgn * h * d)
                vals.append(float(((uu[0] - target) ** 2).sum() * dv))
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = float((grad * d).sum())
        print("rollout %d^3, %d cycles, check %d: FD %.12e, adjoint %.12e, rel %.2e"
              % (n, nsteps, trial, fd, ad, abs(fd - ad) / abs(ad)))
        assert abs(fd - ad) <= 1e-6 * abs(ad)
    runner.mesh.close()


def test_rollout_gradient_matches_central_differences(vl2):
    rollout_fd_check(16, 8, nsteps=12, every=4, ndir=3, h=1e-7)


def test_rollout_gradient_64cubed_100_cycles(vl2):
    """The differentiation workload itself: 64^3 in 32^3 MeshBlocks, 100 cycles, checkpoint every 10.

    The step is smaller than at 16^3: the number of limiter switches that a step of size h moves across
    grows with h, with the cell count and with the number of cycles, and each adds an O(h) error to the
    difference quotient.  At this size h = 1e-7 leaves ~1e-5 of such error, and h = 1e-8 leaves ~3e-9,
    with the quotient's rounding error (~1e-8 at h = 1e-8) still far below the bound."""
    rollout_fd_check(64, 32, nsteps=100, every=10, ndir=2, h=1e-8)


def test_step_vjp_is_deterministic(vl2):
    """The adjoint gathers every sum in a fixed order (no atomics): two calls give identical bits."""
    prob = smooth(n=12, mb=6)
    g = vl2.Mesh.from_problem(prob, adjoint=True)
    dt = g.new_dt()
    rng = np.random.default_rng(3)
    y = to_dev(tuple(rng.standard_normal(a.shape) for a in g.get_cons()))
    first = [t.cpu().numpy() for t in g.step_vjp(dt, y)]
    second = [t.cpu().numpy() for t in g.step_vjp(dt, y)]
    for a, b in zip(first, second):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("ct_delta", [0.0, 1e-2])
def test_recorded_vjp_equals_step_vjp_bitwise(vl2, ct_delta):
    """vl2_step_record keeps what the cycle's adjoint reads; vl2_step_vjp_recorded from that tape gives the same
    bits as vl2_step_vjp at the cycle's starting state, the recorded cycle's state is vl2_step's, and the
    recorded adjoint leaves the mesh's state alone."""
    import torch

    prob = inputs.turbulence(n=16, mb=8, seed=21, mach=1.0, beta=10.0)
    g = vl2.Mesh.from_problem(prob, adjoint=True, ct_delta=ct_delta)
    dt = g.new_dt()
    x0 = g.get_cons()
    rng = np.random.default_rng(4)
    y = to_dev(tuple(rng.standard_normal(a.shape) for a in x0))
    ref = [t.cpu().numpy() for t in g.step_vjp(dt, y)]
    plain = vl2.Mesh.from_problem(prob, ct_delta=ct_delta)
    plain.step(dt)
    g.set_cons(*x0)
    tape = g.new_tape()
    g.step_record(dt, tape)
    for a, b in zip(g.get_cons(), plain.get_cons()):
        np.testing.assert_array_equal(a, b)
    after = g.get_cons()
    got = [t.cpu().numpy() for t in g.step_vjp_recorded(dt, tape, y)]
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(g.get_cons(), after):
        np.testing.assert_array_equal(a, b)
    torch.cuda.synchronize()


def test_rollout_gradient_with_and_without_tapes_bitwise(vl2):
    import torch

    from paper_2005_06651_gb300 import adjoint

    prob = inputs.turbulence(n=16, mb=8, seed=22, mach=1.0, beta=10.0)
    grads = []
    for record in (True, False):
        runner = adjoint.Rollout(prob, nsteps=9, checkpoint_every=3, record=record)
        v0 = torch.from_numpy(np.ascontiguousarray(prob.w[1:4])).cuda().requires_grad_(True)
        u = adjoint.rollout(v0, runner)
        (u[0] ** 2).sum().backward()
        grads.append(v0.grad.detach().cpu().numpy())
        runner.mesh.close()
    np.testing.assert_array_equal(grads[0], grads[1])


def test_rollout_gradient_independent_of_checkpoint_interval(vl2):
    """Recomputation from checkpoints replays the forward bit for bit and the adjoint is deterministic, so
    the gradient does not depend on the checkpoint interval, bit for bit."""
    import torch

    from paper_2005_06651_gb300 import adjoint

    prob = inputs.linear_wave(16, mb=8, kind="fast", amp=1e-2, v0=(0.7, 0.4, 0.2))
    grads = []
    for every in (1, 3, 7, 20):
        runner = adjoint.Rollout(prob, nsteps=7, checkpoint_every=every)
        v0 = torch.from_numpy(np.ascontiguousarray(prob.w[1:4])).cuda().requires_grad_(True)
        u = adjoint.rollout(v0, runner)
        (u[0] ** 2).sum().backward()
        grads.append(v0.grad.detach().cpu().numpy())
        runner.mesh.close()
    for g in grads[1:]:
        np.testing.assert_array_equal(g, grads[0])


def special_riemann_states():
    """Interfaces chosen to reach every branch of the one-sided HLLD: a tangential discontinuity at rest
    (v_n = 0 and equal total pressure on both sides, so S_M = 0 exactly and both sides are averaged),
    supersonic flow either way (outer states), b_n = 0, and no transverse field with b_n^2 > gamma p
    (the degenerate single-star case)."""
    g = 5.0 / 3.0
    rows = []
    base = np.array([1.3, 0.4, -0.2, 0.7, 0.9, 0.5, -0.3])
    rest_l = np.array([1.3, 0.0, -0.2, 0.7, 0.9, 0.5, -0.3])
    rest_r = np.array([0.7, 0.0, 0.4, -0.1, 0.9, -0.3, 0.5])  # same p and |b_t|: equal total pressure
    rows.append((rest_l, rest_r, 0.8))
    rows.append((rest_l, rest_r, -0.8))
    sup = base.copy()
    sup[1] = 9.0
    rows.append((sup, sup * np.array([1.1, 1, 1, 1, 0.9, 1, 1]), 0.3))
    sub = base.copy()
    sub[1] = -9.0
    rows.append((sub * np.array([0.9, 1, 1, 1, 1.1, 1, 1]), sub, 0.3))
    rows.append((base, base * np.array([1.2, -1, 1, 1, 0.8, 1, -1]), 0.0))
    deg = np.array([1.0, 0.1, 0.3, -0.2, 0.3 / g, 0.0, 0.0])
    rows.append((deg, deg * np.array([1.1, 1.3, 1, 1, 1.05, 1, 1]), 1.5))
    wl = np.array([r[0] for r in rows])
    wr = np.array([r[1] for r in rows])
    bn = np.array([r[2] for r in rows])
    return wl, wr, bn


@pytest.mark.parametrize("riemann", [1, 0])
def test_riemann_vjp_matches_oracle_jacobian(vl2, oracle, riemann):
    """The adjoint's reverse-mode Riemann derivative, interface by interface, against the oracle's
    dual-number Jacobian: lf . dF/dx for 4000 random interfaces spanning the fan's regions and the
    special cases above, relative to |lf| |J|."""
    import torch

    from test_oracle_tangent import riemann_states

    wl, wr, bn = riemann_states(4000, 2024 + riemann)
    sw, sr, sb = special_riemann_states()
    wl, wr, bn = np.vstack([wl, sw]), np.vstack([wr, sr]), np.concatenate([bn, sb])
    rng = np.random.default_rng(99)
    lf = rng.standard_normal((len(bn), 7))
    jac = oracle.riemann_jacobian(riemann, wl, wr, bn, 5.0 / 3.0)
    ref = np.einsum("qm,qmk->qk", lf, jac)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (wl, wr, bn, lf)]
    got = vl2.debug_riemann_vjp(riemann, *dev, 5.0 / 3.0).cpu().numpy()
    scale = np.abs(lf).sum(1) * np.abs(jac).max(axis=(1, 2)) + 1.0
    err = np.abs(got - ref).max(1) / scale
    print("Riemann VJP vs oracle Jacobian (riemann %d): max %.2e, special states %s"
          % (riemann, err.max(), np.array2string(err[-len(sb):], precision=1)))
    assert err.max() <= 1e-12
