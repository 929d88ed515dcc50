"""Batched form: many independent boxes of uneven sizes advanced by one launch per kernel over a
(box, tile) work list, and K cycles as one CUDA-graph launch.  The batch runs the same kernels on the same
data as the per-mesh path, so the results must be bitwise identical to stepping each mesh on its own."""
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


def boxes():
    """Uneven boxes: single-block boxes of 8^3, 12^3, 16^3, 20^3 and a 16^3 box made of 8 blocks."""
    probs = []
    for q, (n, mb) in enumerate([(8, 8), (12, 12), (16, 16), (20, 20), (16, 8), (12, 12)]):
        probs.append(inputs.turbulence(n=n, mb=mb, seed=300 + q, mach=1.0, beta=1.0))
    return probs


def make(vl2, probs, **kw):
    return [vl2.Mesh.from_problem(p, **kw) for p in probs]


def assert_same(a_meshes, b_meshes):
    for a, b in zip(a_meshes, b_meshes):
        for x, y in zip(a.get_cons(), b.get_cons()):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_matches_per_mesh_steps_bitwise(vl2, precision):
    probs = boxes()
    ref, bat = make(vl2, probs, precision=precision), make(vl2, probs, precision=precision)
    batch = vl2.Batch(bat)
    for _ in range(3):
        dts = [m.new_dt() for m in ref]
        for m, dt in zip(ref, dts):
            m.step(dt)
        batch.step(dts)
    assert_same(ref, bat)


def test_batch_run_uses_each_box_cfl_step_and_matches_bitwise(vl2):
    probs = boxes()
    ref, bat = make(vl2, probs), make(vl2, probs)
    batch = vl2.Batch(bat)
    dts = None
    for _ in range(2):  # the same graph launched twice
        dts = batch.run(4)
    for _ in range(8):
        last = [m.new_dt() for m in ref]
        for m, dt in zip(ref, last):
            m.step(dt)
    np.testing.assert_array_equal(dts, np.array(last))
    assert_same(ref, bat)
    # after the batch, each mesh's own calls see its current state
    for m in bat:
        assert m.new_dt() > 0 and m.divb_norm() <= 1e-13
    assert batch.launch_count() >= 2 * 4 * 17


def test_autotune_keeps_state_and_results(vl2):
    probs = boxes()
    ref, bat = make(vl2, probs), make(vl2, probs)
    batch = vl2.Batch(bat)
    dc, pl = batch.autotune()
    assert dc in (64, 128, 256) and pl in (4, 8, 16)
    assert_same(ref, bat)  # timing the flux launches does not touch the state
    batch.run(3)
    for _ in range(3):
        for m in ref:
            m.step(m.new_dt())
    assert_same(ref, bat)


def test_batch_rejects_mixed_precisions(vl2):
    probs = boxes()[:2]
    a = vl2.Mesh.from_problem(probs[0])
    b = vl2.Mesh.from_problem(probs[1], precision=vl2.MIXED)
    with pytest.raises(vl2.VL2Error) as e:
        vl2.Batch([a, b])
    assert e.value.status == vl2.VL2_E_ARG
