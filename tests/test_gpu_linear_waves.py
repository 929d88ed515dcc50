"""Linear-wave convergence on the GPU (Sec. 3.3.1, eq. RMS-error): the 3D adiabatic MHD Alfven, slow and fast
waves of amplitude 1e-6 along the diagonal of the unit periodic cube (k = 2 pi (1, 1, 1), background rho = 1,
p = 1/gamma, |B| = 1 along (1, sqrt 2, 1/2) in the wave frame), one MeshBlock, VL2 + PLM + HLLD + CT, CFL 0.3,
one wave period (last step clipped), at N = 16, 32 and 64.

For each wave and N the GPU's L1 error (eq. RMS-error over rho, M, E and b_c) is compared with the oracle's,
both driven by the oracle's time-step sequence (the oracle runs in 16^3 MeshBlocks, which its block-
invariance pin makes bitwise the single-block result).  The L1 of a 1e-6 wave is ~1e-8 of the state, while
the two paths differ by rounding (~1e-16 of the state per cycle), so the L1 values cannot agree to much better
than 1e-16 / 1e-8 relative: the test asserts the bound that follows from the triangle inequality,
|L1_gpu - L1_oracle| <= RMS over variables of mean |U_gpu - U_oracle|, and a relative difference <= 1e-6.
The GPU's own slope log2(L1(32) / L1(64)) must lie in [1.8, 2.2] (second order, Sec. 3.3.1).  The slope
from 16 to 32 (about 9 cells per wavelength at N = 16) is pre-asymptotic, about 1.6 for all three waves in
the oracle, and is reported, not bounded."""
import math

import numpy as np
import pytest

from paper_2005_06651_gb300 import inputs

pytestmark = pytest.mark.gpu

WAVES = ("alfven", "slow", "fast")
SIZES = (16, 32, 64)


@pytest.fixture(scope="module")
def vl2():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_06651_gb300 import build, vl2 as mod

    build.build()
    mod.load()
    return mod


def cell_b(b1, b2, b3):
    return (0.5 * (b1[:, :, 1:] + b1[:, :, :-1]), 0.5 * (b2[:, 1:, :] + b2[:, :-1, :]), 0.5 * (b3[1:] + b3[:-1]))


def means(state, ref):
    """mean |U_n - ref_n| over rho, M (3), E, b_c (3)."""
    u, b1, b2, b3 = state
    u0, c1, c2, c3 = ref
    bc, bc0 = cell_b(b1, b2, b3), cell_b(c1, c2, c3)
    return np.array([np.mean(np.abs(u[v] - u0[v])) for v in range(5)] +
                    [np.mean(np.abs(bc[d] - bc0[d])) for d in range(3)])


def l1(state, ref):
    return float(np.sqrt(np.sum(np.square(means(state, ref)))))


@pytest.fixture(scope="module")
def results(vl2, oracle):
    out = {}
    for kind in WAVES:
        for n in SIZES:
            prob = inputs.linear_wave(n, kind=kind, amp=1e-6)
            g = vl2.Mesh.from_problem(prob)  # one MeshBlock of n^3, the configuration's layout
            o = oracle.Mesh.from_problem(prob, mb=(16, 16, 16))
            ref = o.get_cons()
            t, t_end, steps = 0.0, prob.meta["period"], 0
            while t < t_end:
                dt = o.new_dt(0.3)
                if t + dt > t_end:
                    dt = t_end - t
                g.step(dt)
                o.step(dt)
                t += dt
                steps += 1
            gs, os_ = g.get_cons(), o.get_cons()
            assert g.floor_count() == 0 and o.floor_count() == 0
            out[kind, n] = {"gpu": l1(gs, ref), "oracle": l1(os_, ref), "steps": steps,
                            "bound": float(np.sqrt(np.sum(np.square(means(gs, os_)))))}
    return out


@pytest.mark.parametrize("kind", WAVES)
@pytest.mark.parametrize("n", SIZES)
def test_gpu_l1_matches_the_oracle(results, kind, n):
    r = results[kind, n]
    rel = abs(r["gpu"] - r["oracle"]) / r["oracle"]
    print("%s wave N=%d (%d steps): L1 GPU %.6e, oracle %.6e, relative difference %.1e"
          % (kind, n, r["steps"], r["gpu"], r["oracle"], rel))
    assert abs(r["gpu"] - r["oracle"]) <= r["bound"] + 1e-300
    assert rel <= 1e-6


@pytest.mark.parametrize("kind", WAVES)
def test_gpu_second_order(results, kind):
    errs = [results[kind, n]["gpu"] for n in SIZES]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(SIZES) - 1)]
    print("%s wave: GPU L1 %s, slopes %s" % (kind, ["%.3e" % e for e in errs], ["%.3f" % s for s in slopes]))
    assert 1.8 <= slopes[-1] <= 2.2, slopes
