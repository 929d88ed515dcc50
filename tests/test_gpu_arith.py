"""The library's hand-written FP64 arithmetic against IEEE results, through vl2_debug_arith (C ABI).

The flux kernels replace the FP64 divide and square root by Newton-refined hardware seeds (rcp_nr,
rsqrt_nr, sqrt_nr: one cubically convergent step from rcp.approx / rsqrt.approx, the series form of
Markstein and of Muller et al.), and convert between float and double on the integer pipe (to_f32, to_f64).
Bounds checked here on about 10^6 inputs each, plus the ends of every domain:
- rcp_nr, sqrt_nr and the _any variants within 1 ulp of the correctly rounded 1/x and sqrt (numpy's IEEE
  division and square root on the host);
- rsqrt_nr and rroot_any within 1 ulp of the exact 1/sqrt(x) (exact rational arithmetic on a sample);
- inv_any over every finite non-zero input, including |x| >= 2^1021 (the end of rcp_nr's documented domain;
  above 2^1022 the reciprocal seed flushes and rcp_nr alone returns 0);
- to_f32 bitwise equal to IEEE round-to-nearest-even (numpy's conversion and CUDA's __double2float_rn) on
  random doubles, exact ties, the ends of the float range, zeros, infinities; to_f64 bitwise exact on random
  float bit patterns.
"""
from fractions import Fraction

import numpy as np
import pytest

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


def run(vl2, fn, x):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = vl2.debug_arith(fn, t)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def log_uniform(rng, n, e_lo, e_hi, signed=True):
    """Random normal doubles 2^e * m, e uniform in [e_lo, e_hi), m uniform in [1, 2)."""
    x = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(e_lo, e_hi, n))
    if signed:
        x *= rng.choice([-1.0, 1.0], n)
    return x


def ulp_gap(a, b):
    """Distance in units in the last place between doubles of the same sign (0 when bitwise equal)."""
    ia, ib = a.view(np.int64), b.view(np.int64)
    assert np.all(np.signbit(a) == np.signbit(b))
    return np.abs(ia - ib)


def edges(lo_exp, hi_exp):
    """The ends of a binade range: the first and last few doubles at 2^lo_exp and below 2^hi_exp."""
    lo = np.ldexp(1.0, lo_exp)
    hi = np.ldexp(1.0, hi_exp)
    out = [lo, np.nextafter(lo, np.inf), np.nextafter(np.nextafter(lo, np.inf), np.inf),
           np.nextafter(hi, 0.0), np.nextafter(np.nextafter(hi, 0.0), 0.0), 1.0, np.nextafter(1.0, 2.0),
           np.nextafter(1.0, 0.0), 2.0, 3.0, 0.1, 1e-300, 1e300]
    return np.array([v for v in out if lo <= v < hi])


def test_rcp_nr_within_one_ulp(vl2):
    rng = np.random.default_rng(1)
    x = np.concatenate([log_uniform(rng, 1_000_000, -1022, 1021), edges(-1022, 1021), -edges(-1022, 1021)])
    with np.errstate(over="ignore"):
        ref = 1.0 / x
    for fn in (vl2.AR_RCP_NR, vl2.AR_INV_ANY):
        gap = ulp_gap(run(vl2, fn, x), ref)
        print("fn %d: max ulp gap to IEEE 1/x over %d inputs: %d (%.3f%% not correctly rounded)"
              % (fn, x.size, gap.max(), 100.0 * np.mean(gap > 0)))
        assert gap.max() <= 1
    # CUDA's own division is the correctly rounded one
    assert np.array_equal(run(vl2, vl2.AR_IEEE_RCP, x), ref)


def test_inv_any_covers_the_whole_range(vl2):
    rng = np.random.default_rng(2)
    big = log_uniform(rng, 20000, 1021, 1024)
    tiny = np.concatenate([log_uniform(rng, 20000, -1074, -1022), np.array([5e-324, 1e-320, 2.2250738585072e-308])])
    x = np.concatenate([big, -big, tiny, -tiny, [np.finfo(np.float64).max, -np.finfo(np.float64).max]])
    with np.errstate(over="ignore", divide="ignore"):
        ref = 1.0 / x
    got = run(vl2, vl2.AR_INV_ANY, x)
    assert np.array_equal(got, ref)  # the IEEE division outside the Newton form's domain
    # rcp_nr alone flushes where 1/x is subnormal (documented): |x| > 2^1022
    above = big[np.abs(big) > np.ldexp(1.0, 1022)]
    assert np.all(run(vl2, vl2.AR_RCP_NR, above) == 0.0)


def test_sqrt_forms_within_one_ulp(vl2):
    rng = np.random.default_rng(3)
    x = np.concatenate([log_uniform(rng, 1_000_000, -1022, 1024, signed=False), edges(-1022, 1024)])
    ref = np.sqrt(x)
    for fn in (vl2.AR_SQRT_NR, vl2.AR_ROOT_ANY):
        gap = ulp_gap(run(vl2, fn, x), ref)
        print("fn %d: max ulp gap to IEEE sqrt: %d (%.3f%% not correctly rounded)" % (fn, gap.max(), 100.0 * np.mean(gap > 0)))
        assert gap.max() <= 1
    assert np.array_equal(run(vl2, vl2.AR_IEEE_SQRT, x), ref)
    # root_any over zeros and subnormals
    sub = np.concatenate([[0.0, 5e-324], log_uniform(rng, 20000, -1074, -1022, signed=False)])
    assert np.array_equal(run(vl2, vl2.AR_ROOT_ANY, sub), np.sqrt(sub))
    assert run(vl2, vl2.AR_SQRT_NR, np.array([0.0]))[0] == 0.0


def exact_rsqrt_ulps(x, y):
    """|y - 1/sqrt(x)| in ulps of the exact value, from exact rationals: with e = 1 - x y^2 (exact),
    y = (1/sqrt x) sqrt(1 - e), so the relative error is 1 - sqrt(1 - e) ~ e/2 + e^2/8."""
    out = np.empty(x.size)
    for n, (xv, yv) in enumerate(zip(x, y)):
        e = 1 - Fraction(xv) * Fraction(yv) * Fraction(yv)
        rel = abs(float(e) / 2 + float(e) ** 2 / 8)
        exact = float(yv) / np.sqrt(1.0 - float(e)) if abs(float(e)) < 0.5 else 1.0 / np.sqrt(xv)
        ulp = np.ldexp(1.0, int(np.floor(np.log2(exact))) - 52)
        out[n] = rel * exact / ulp
    return out


def test_rsqrt_forms_within_one_ulp(vl2):
    rng = np.random.default_rng(4)
    x = np.concatenate([log_uniform(rng, 1_000_000, -1022, 1024, signed=False), edges(-1022, 1024)])
    y = run(vl2, vl2.AR_RSQRT_NR, x)
    # every result within 2 ulps of CUDA's rsqrt (itself within 1 ulp), the exact check on a sample
    cuda = run(vl2, vl2.AR_CUDA_RSQRT, x)
    assert ulp_gap(y, cuda).max() <= 2
    pick = np.concatenate([rng.choice(x.size, 20000, replace=False), np.arange(x.size - 13, x.size)])
    u = exact_rsqrt_ulps(x[pick], y[pick])
    print("rsqrt_nr: max error %.3f ulp on %d inputs (exact rationals)" % (u.max(), pick.size))
    assert u.max() < 1.0
    ya = run(vl2, vl2.AR_RROOT_ANY, x[pick])
    assert np.array_equal(ya, y[pick])
    sub = log_uniform(rng, 2000, -1074, -1022, signed=False)
    with np.errstate(divide="ignore"):
        assert np.array_equal(run(vl2, vl2.AR_RROOT_ANY, sub), 1.0 / np.sqrt(sub))


def test_to_f32_rounds_to_nearest_even(vl2):
    rng = np.random.default_rng(5)
    f32 = np.finfo(np.float32)
    # random doubles across and beyond the float range
    a = log_uniform(rng, 600_000, -160, 140)
    # exact ties: a float plus half its ulp (round to even), and just either side of the tie
    fl = log_uniform(rng, 100_000, -126, 127).astype(np.float32).astype(np.float64)
    half = np.ldexp(1.0, np.frexp(fl)[1] - 25)
    ties = np.concatenate([fl + half, fl - half, np.nextafter(fl + half, np.inf), np.nextafter(fl + half, -np.inf)])
    ends = np.array([f32.max, np.nextafter(float(f32.max), np.inf), float(f32.max) + np.ldexp(1.0, 103),
                     float(f32.max) + np.ldexp(1.0, 104), float(f32.tiny), float(f32.tiny) * 0.5, 1.4e-45, 7e-46,
                     7.1e-46, 0.0, -0.0, np.inf, -np.inf, 1e300, -1e300, 1e-300])
    x = np.concatenate([a, ties, ends, -ends])
    with np.errstate(over="ignore", under="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    got = run(vl2, vl2.AR_TO_F32, x)
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))
    assert np.array_equal(run(vl2, vl2.AR_CUDA_D2F, x).view(np.int64), ref.view(np.int64))
    nan = run(vl2, vl2.AR_TO_F32, np.array([np.nan]))
    assert np.isnan(nan[0])


def test_to_f64_is_exact(vl2):
    rng = np.random.default_rng(6)
    bits = rng.integers(0, 1 << 32, 1_000_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[~np.isnan(f)]
    extra = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, np.finfo(np.float32).tiny, np.finfo(np.float32).max],
                     dtype=np.float32)
    f = np.concatenate([f, extra])
    x = f.astype(np.float64)
    got = run(vl2, vl2.AR_TO_F64, x)
    assert np.array_equal(got.view(np.int64), x.view(np.int64))
