"""Stream-ordered stepping: vl2_set_prims_async, vl2_step_cfl (the CFL step formed and read on the device),
vl2_last_dt, and the streamed loop built on them, against the synchronous calls.

vl2_step_cfl performs the arithmetic of vl2_new_dt followed by vl2_step (Sec. 2.1.7 and 3.2.3), and
vl2_set_prims_async that of vl2_set_prims, so the states agree bit for bit; the synchronous path is held to
the oracle by test_gpu_parity.py.
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


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_cfl_equals_new_dt_then_step_bitwise(vl2, precision):
    prob = inputs.orszag_tang(n=(32, 24, 16), mb=(16, 12, 8), seed=2005)
    prec = vl2.MIXED if precision == "mixed" else vl2.FP64
    a = vl2.Mesh.from_problem(prob, precision=prec)
    b = vl2.Mesh.from_problem(prob, precision=prec)
    for _ in range(5):
        dt = a.new_dt()
        a.step(dt)
        b.step_cfl()
        assert b.last_dt() == dt
    assert _same(a.get_cons(), b.get_cons())


def test_set_prims_async_equals_set_prims(vl2):
    import torch

    prob = inputs.turbulence(n=32, mb=16, seed=3003, mach=1.0, beta=1.0)
    ref = vl2.Mesh.from_problem(prob)
    dev_in = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (prob.w, prob.b1, prob.b2, prob.b3)]
    pinned = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (prob.w, prob.b1, prob.b2, prob.b3)]
    for src in (dev_in, pinned):
        m = vl2.Mesh(prob.nx, prob.mb, prob.xmin, prob.xmax, prob.gamma)
        m.set_prims_async(*src)
        assert _same(ref.get_cons(), m.get_cons())
        m.step_cfl()
        r2 = vl2.Mesh.from_problem(prob)
        r2.step(r2.new_dt())
        assert _same(r2.get_cons(), m.get_cons())


def test_async_periodic_check_reported_by_the_next_wait(vl2):
    prob = inputs.orszag_tang(n=16, mb=8, seed=2005)
    b1 = prob.b1.copy()
    b1[3, 5, -1] += 1e-3  # face N of a periodic mesh no longer equals face 0
    m = vl2.Mesh(prob.nx, prob.mb, prob.xmin, prob.xmax, prob.gamma)
    m.set_prims_async(prob.w, b1, prob.b2, prob.b3)  # host arrays: the call still does not check
    with pytest.raises(vl2.VL2Error) as e:
        m.new_dt()
    assert e.value.status == vl2.VL2_E_ARG
    m.set_prims(prob.w, prob.b1, prob.b2, prob.b3)  # reported once; a consistent state steps normally
    m.step(m.new_dt())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_streamed_steps_match_the_synchronous_loop(vl2, precision):
    """The streamed loop (copies on two streams, double-buffered staging) gives every step's result as the
    synchronous set_prims / new_dt / step / get_cons loop does."""
    import torch

    prob = inputs.orszag_tang(n=32, mb=16, seed=2005)
    prec = vl2.MIXED if precision == "mixed" else vl2.FP64
    ref = vl2.Mesh.from_problem(prob, precision=prec)
    ref.step(ref.new_dt())
    want = ref.get_cons()
    m = vl2.Mesh(prob.nx, prob.mb, prob.xmin, prob.xmax, prob.gamma, precision=prec,
                 stream=torch.cuda.Stream())
    host_in = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (prob.w, prob.b1, prob.b2, prob.b3)]
    host_out = [torch.empty(x.shape, dtype=torch.float64).pin_memory() for x in want]
    dt = m.streamed_steps(host_in, host_out, 4)
    assert dt > 0
    assert _same(want, [x.numpy() for x in host_out])
