"""vl2_totals_noalloc: the conserved totals for callers that cannot allocate device memory (a host
whose device memory is all owned by its own pool, or a pipeline that must not take the synchronisation
an allocation can cause).  Called through the C ABI, its output must match vl2_totals of the same state,
on two calls in a row with different states (the second call reuses the shared scratch the first one
left behind).  This file is collected last so a failure here cannot hide any other test."""
import ctypes

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


def device_state(mesh):
    import torch

    out = (torch.empty((5,) + mesh.shape, dtype=torch.float64, device="cuda"),
           *[torch.empty(s, dtype=torch.float64, device="cuda") for s in mesh.face_shapes()])
    mesh.get_cons(out)
    return out


def test_totals_noalloc_matches_totals_on_two_calls(vl2):
    import torch

    prob = inputs.orszag_tang(n=(32, 24, 40), mb=(16, 12, 20), seed=77)
    mesh = vl2.Mesh.from_problem(prob)
    dx = prob.dx
    scale = None
    for call in range(2):
        if call == 1:
            for _ in range(3):
                mesh.step(mesh.new_dt())
        ref = mesh.totals()
        u, b1, b2, b3 = device_state(mesh)
        out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        vl2.totals_noalloc(u, b1, b2, b3, dx, out)
        torch.cuda.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        if call == 1:
            # the first call loaded the module and looked up the scratch; the second must leave both the torch
            # allocator and the device's free memory exactly as they were
            assert after == before, (before, after)
        got = out.cpu().numpy()
        if scale is None:
            scale = np.array([abs(ref[0])] + [abs(ref[4])] * 4 + [1.0] * 3)
        assert np.all(np.abs(got - ref) <= 1e-13 * scale), (call, got, ref)


def test_totals_noalloc_rejects_sizes_beyond_its_scratch(vl2):
    lib = vl2.load()
    nx = (ctypes.c_int * 3)(8, 8, vl2.NOALLOC_MAX_NZ + 1)
    dx = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the size check comes first
    st = lib.vl2_totals_noalloc(fake, fake, fake, fake, nx, dx, fake, None)
    assert st == vl2.VL2_E_ARG
    assert b"VL2_NOALLOC_MAX_NZ" in lib.vl2_last_error(None)
