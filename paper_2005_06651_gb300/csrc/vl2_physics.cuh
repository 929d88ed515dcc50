// Device physics of the VL2 MHD step (Stone et al. 2020, arXiv:2005.06651, Sec. 3.1-3.2).
// Interface states are 7-vectors in the sweep frame (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) with
// (n, t1, t2) = (x, y, z), (y, z, x), (z, x, y); fluxes use the same slots (mass, M_n, M_t1, M_t2,
// E, B_t1, B_t2).  Reciprocals are formed once and reused (FP64 ones by rcp_nr below, within about one
// ulp); FMA contraction is allowed.
#pragma once
#include <cuda_runtime.h>

namespace vl2 {

// ---- FP64 reciprocal and square root ------------------------------------------------------------
// The FP64 divide and square root are the costliest steps of the flux arithmetic on this part.  Here the
// PTX approximations rcp.approx.ftz.f64 and rsqrt.approx.ftz.f64 (relative error about 1e-6, measured)
// are refined by one cubically convergent Newton step (Newton's method on 1/r - b and on 1/y^2 - x, in the
// series form given by Markstein and in Muller et al., Handbook of Floating-Point Arithmetic):
//   r ~ 1/b,       e = 1 - b r:        1/b      = r (1 + e + e^2 + ...)
//   y ~ x^(-1/2),  h = 1 - x y^2:      x^(-1/2) = y (1 + h/2 + 3 h^2/8 + ...),  x^(1/2) = x y (1 + h/2 + ...)
// The remaining relative error is O(1e-18) plus the rounding of the last steps: within one ulp of the
// correctly rounded result, not always equal to it (bounded by a test against IEEE results).  Inputs are
// finite normal numbers (no denormals), and rcp_nr needs |b| < 2^1021 (its seed flushes to 0 where 1/b is
// near or below the smallest normal, and the result is then 0); sqrt_nr also takes +0 and returns +0.
// Other scalar types (float, dual numbers) use their own / and sqrt.
#ifndef VL2_VALUE_SAFE
__device__ __forceinline__ double rcp_nr(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  const double e = fma(-b, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double rsqrt_nr(double x) {  // x a positive normal number
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double h = fma(-(x * y), y, 1.0);
  return fma(y * h, fma(0.375, h, 0.5), y);
}
// sqrt(x) = s (1 - h)^(-1/2) with s = x y rounded and h = 1 - s y: the series is applied to s itself, so the
// rounding of s enters only through h (half of it survives) and the result is within one ulp.
__device__ __forceinline__ double sqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double s = x * y;
  const double h = fma(-s, y, 1.0);
  const double r = fma(s * h, fma(0.375, h, 0.5), s);
  return (__double_as_longlong(x) << 1) == 0 ? x : r;
}
#else
// Value-safe build (VL2_VALUE_SAFE, compiled with -fmad=false): the IEEE division and square root, each
// correctly rounded, and no contraction anywhere, so that every expression written symmetrically in its
// left and right operands gives bitwise mirror-symmetric results (Sec. 3.3.5 asks for value-safe arithmetic
// where symmetric solutions must stay symmetric).
__device__ __forceinline__ double rcp_nr(double b) { return 1.0 / b; }
__device__ __forceinline__ double rsqrt_nr(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ double sqrt_nr(double x) { return sqrt(x); }
#endif
// Products rounded on their own (never contracted into an FMA with a following add).  Used where two
// products cancel exactly for mirror-image states, so that the difference is exactly zero there (an FMA
// would leave the rounding error of one product): the contact speed S_M and the mass flux of a
// symmetry plane, whose sign decides the HLLD side and the CT upwind cell.
template <class R> __device__ __forceinline__ R mul_rn(R a, R b) { return a * b; }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }

template <class R> __device__ __forceinline__ R inv(R x) { return R(1) / x; }
template <> __device__ __forceinline__ double inv<double>(double x) { return rcp_nr(x); }
template <class R> __device__ __forceinline__ R root(R x) { return sqrt(x); }
template <> __device__ __forceinline__ double root<double>(double x) { return sqrt_nr(x); }
template <class R> __device__ __forceinline__ R rroot(R x) { return rsqrt(x); }
template <> __device__ __forceinline__ double rroot<double>(double x) { return rsqrt_nr(x); }
// The same for any input of the operation's domain: the Newton forms take normal numbers only, and the
// reciprocal seed (.ftz) flushes to 0 where it would be subnormal, which |x| close to or above 2^1022 can
// give; inputs outside [2^-1022, 2^1021) take the IEEE operation.
constexpr double DBL_NORMAL_MIN = 2.2250738585072014e-308;
constexpr double RCP_NR_MAX = 0x1p1021;  // rcp_nr is used on 2^-1022 <= |x| < 2^1021
template <class R> __device__ __forceinline__ R inv_any(R x) { return R(1) / x; }
template <> __device__ __forceinline__ double inv_any<double>(double x) {
  const double a = fabs(x);
  return (a >= DBL_NORMAL_MIN && a < RCP_NR_MAX) ? rcp_nr(x) : 1.0 / x;
}
template <class R> __device__ __forceinline__ R root_any(R x) { return sqrt(x); }
template <> __device__ __forceinline__ double root_any<double>(double x) {
  return x >= DBL_NORMAL_MIN ? sqrt_nr(x) : sqrt(x);
}
template <class R> __device__ __forceinline__ R rroot_any(R x) { return R(1) / sqrt(x); }
template <> __device__ __forceinline__ double rroot_any<double>(double x) {
  return x >= DBL_NORMAL_MIN ? rsqrt_nr(x) : 1.0 / sqrt(x);
}

// ---- float <-> double on the integer pipe ----------------------------------------------------------
// On this part a hardware conversion between float and double occupies the FP64 pipe like an FP64
// operation.  Both directions are written here on the IEEE 754 bit layouts (binary32: 8-bit exponent,
// bias 127; binary64: 11-bit exponent, bias 1023), which moves the work to the integer pipe.  Results
// equal the hardware conversion (round to nearest even for double -> float); zeros are handled here, and
// the rare cases outside the normal float range (denormal float inputs or results, overflow, inf, nan)
// fall back to the hardware conversion.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int mag = u & 0x7fffffffu;
  const unsigned int e = mag >> 23;
  if (e - 1u >= 254u) {  // exponent field 0 or 255
    if (mag == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));  // signed zero
    return (double)f;
  }
  const unsigned long long bits =
      ((unsigned long long)(u >> 31) << 63) | (((unsigned long long)mag << 29) + (896ULL << 52));
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = u & 0x7fffffffffffffffULL;
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  // double exponent field 897..1150 maps to the float exponents 1..254 (the rounding carry may reach 255 = inf)
  if (mag - (897ULL << 52) < (254ULL << 52)) {
    const unsigned long long r = mag + 0x0fffffffULL + ((mag >> 29) & 1ULL);  // nearest, ties to even
    return __uint_as_float(sign | (unsigned int)((r >> 29) - (896ULL << 23)));
  }
  if (mag == 0ULL) return __uint_as_float(sign);
  return (float)x;
}
__device__ __forceinline__ float to_f32(float x) { return x; }

// Fast magnetosonic speed along the normal (Sec. 2.1.7 uses |v| + C_f):
// C_f^2 = (a^2 + c_n^2 + c_t^2 + sqrt((a^2 - c_n^2)^2 + c_t^2 (c_t^2 + 2 a^2 + 2 c_n^2))) / 2,
// a^2 = gamma p / rho, c_n^2 = b_n^2 / rho, c_t^2 = |b_t|^2 / rho.
// C_f^2 from hid = 1 / (2 rho): the same form scaled by rho^2 inside the root (rho C_f^2 with gamma p, b_n^2,
// |b_t|^2), one 1/(2 rho) at the end
template <class R>
__device__ __forceinline__ R fast_speed2_h(R hid, R p, R bn2, R bt2, R gamma) {
  const R gp = gamma * p;
  const R df = gp - bn2;
  const R sn = gp + bn2;
  const R rad = df * df + bt2 * (bt2 + R(2) * sn);
  return ((sn + bt2) + root(rad)) * hid;
}
template <class R>
__device__ __forceinline__ R fast_speed2_r(R id, R p, R bn2, R bt2, R gamma) {  // C_f^2 from id = 1 / rho
  return fast_speed2_h(R(0.5) * id, p, bn2, bt2, gamma);
}
template <class R>
__device__ __forceinline__ R fast_speed_r(R id, R p, R bn2, R bt2, R gamma) {
  return root(fast_speed2_r(id, p, bn2, bt2, gamma));
}

// Conserved 7-vector and physical flux of one sweep-frame state (eq. cons, eq. total_energy), given
// |B|^2 = bb and the total pressure pt = p + bb/2 of the state.
template <class R>
__device__ __forceinline__ void phys_flux_bb(const R* w, R bn, R igm1, R bb, R pt, R* u, R* f) {
  const R d = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[5], b2 = w[6];
  const R e = p * igm1 + R(0.5) * d * ((vn * vn + v1 * v1) + v2 * v2) + R(0.5) * bb;
  const R vb = (vn * bn + v1 * b1) + v2 * b2;
  const R m = d * vn;
  u[0] = d; u[1] = m; u[2] = d * v1; u[3] = d * v2; u[4] = e; u[5] = b1; u[6] = b2;
  f[0] = m;
  f[1] = m * vn + pt - bn * bn;
  f[2] = m * v1 - bn * b1;
  f[3] = m * v2 - bn * b2;
  f[4] = (e + pt) * vn - bn * vb;
  f[5] = b1 * vn - bn * v1;
  f[6] = b2 * vn - bn * v2;
}
template <class R>
__device__ __forceinline__ void phys_flux(const R* w, R bn, R igm1, R* u, R* f) {
  const R bb = (bn * bn + w[5] * w[5]) + w[6] * w[6];
  phys_flux_bb(w, bn, igm1, bb, w[4] + R(0.5) * bb, u, f);
}

// ---- sign tests and orderings on the integer pipe --------------------------------------------
// The FP64 pipe is the bottleneck of the plain kernels, so comparisons of doubles are done on the IEEE
// bit patterns (integer compares) rather than with FP64 compare instructions.  They return exactly what
// the corresponding IEEE comparison returns (NaN aside).
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int dbits(float x) { return __float_as_int(x); }
// x > 0 (false for +0 and -0)
template <class R> __device__ __forceinline__ bool gt0(R x) { return dbits(x) > 0; }
// x >= 0 (true for -0)
template <class R> __device__ __forceinline__ bool ge0(R x) {
  const auto b = dbits(x);
  return b >= 0 || (b << 1) == 0;
}
// x < 0 (false for -0)
template <class R> __device__ __forceinline__ bool lt0(R x) { return !ge0(x); }
template <class R> __device__ __forceinline__ bool is0(R x) { return (dbits(x) << 1) == 0; }
// total-order key: a < b  <=>  key(a) < key(b) for all non-NaN a, b (-0 and +0 map to 0 and -1)
__device__ __forceinline__ long long okey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ int okey(float x) {
  const int b = dbits(x);
  return b ^ ((b >> 31) & 0x7fffffff);
}
// min / max with ties going to b (the values agree at a tie; the rule fixes which argument a derivative
// follows there)
template <class R> __device__ __forceinline__ R imin(R a, R b) { return okey(a) < okey(b) ? a : b; }
template <class R> __device__ __forceinline__ R imax(R a, R b) { return okey(a) > okey(b) ? a : b; }
template <class R> __device__ __forceinline__ bool igt(R a, R b) { return okey(a) > okey(b); }
// The two sweep-frame states are bitwise equal.  The flux of such a pair is the physical flux of the state
// (consistency of every Riemann solver; HLLE's and HLLD's own arithmetic give it up to rounding, with the
// same sign of the mass flux, exactly zero when v_n is), so both solvers form it directly: uniform regions
// at rest would otherwise take HLLD's S_M == 0 branch and evaluate both sides of the fan.
template <class R> __device__ __forceinline__ bool same_state(const R* a, const R* b) {
  auto x = dbits(a[0]) ^ dbits(b[0]);
#pragma unroll
  for (int n = 1; n < 7; ++n) x |= dbits(a[n]) ^ dbits(b[n]);
  return x == 0;
}

// HLLE flux; outer speeds are the extreme fast-wave speeds of the two states (Sec. 3.2.2 names the
// solver; the speed estimate is this library's reading).
template <class R>
__device__ __forceinline__ void flux_hlle(const R* wl, const R* wr, R bn, R gamma, R igm1, R* f, bool roe = false) {
  R ul[7], fl[7], ur[7], fr[7];
  phys_flux(wl, bn, igm1, ul, fl);
  if (same_state(wl, wr)) {
#pragma unroll
    for (int n = 0; n < 7; ++n) f[n] = fl[n];
    return;
  }
  phys_flux(wr, bn, igm1, ur, fr);
  const R bn2 = bn * bn;
  const R hlr = R(0.5) * inv(wl[0] * wr[0]);  // 1/(2 rho_L) and 1/(2 rho_R) from one reciprocal
  const R cl = root(fast_speed2_h(wr[0] * hlr, wl[4], bn2, wl[5] * wl[5] + wl[6] * wl[6], gamma));
  const R cr = root(fast_speed2_h(wl[0] * hlr, wr[4], bn2, wr[5] * wr[5] + wr[6] * wr[6], gamma));
  R sl = imin(wl[1] - cl, wr[1] - cr);
  R sr = imax(wl[1] + cl, wr[1] + cr);
  if (roe) {
    // Einfeldt's speeds: S_L = min(u_L - c_L, u~ - c~_f), S_R = max(u_R + c_R, u~ + c~_f), with c~_f the fast
    // eigenvalue (about u~) of the Roe matrix of the 1D MHD flux built from sqrt(rho) weights for u and
    // H = (E + p_T) / rho, cross weights for b_t and rho~ = sqrt(rho_L rho_R); its magnetic-pressure difference
    // adds X = |db_t|^2 / (2 (sqrt(rho_L) + sqrt(rho_R))^2) to the sound speed term:
    //   a~^2 = (gamma-1)(H~ - |u~|^2/2 - |b~|^2/rho~) - (gamma-2) X,  c~_t^2 = |b~_t|^2 / rho~
    const R sdl = root(wl[0]), sdr = root(wr[0]);
    const R iws = inv(sdl + sdr);
    const R irho = inv(sdl * sdr);
    const R un = (sdl * wl[1] + sdr * wr[1]) * iws;
    const R u1 = (sdl * wl[2] + sdr * wr[2]) * iws, u2 = (sdl * wl[3] + sdr * wr[3]) * iws;
    const R b1 = (sdr * wl[5] + sdl * wr[5]) * iws, b2 = (sdr * wl[6] + sdl * wr[6]) * iws;
    const R ptl = wl[4] + R(0.5) * ((bn2 + wl[5] * wl[5]) + wl[6] * wl[6]);
    const R ptr = wr[4] + R(0.5) * ((bn2 + wr[5] * wr[5]) + wr[6] * wr[6]);
    const R h = ((ul[4] + ptl) * inv(sdl) + (ur[4] + ptr) * inv(sdr)) * iws;
    const R d1 = wl[5] - wr[5], d2 = wl[6] - wr[6];
    const R x = R(0.5) * (d1 * d1 + d2 * d2) * (iws * iws);
    const R btsq = b1 * b1 + b2 * b2;
    const R usq = (un * un + u1 * u1) + u2 * u2;
    const R gm1 = gamma - R(1), gm2 = gamma - R(2);
    const R ca2 = bn2 * irho;
    R a2 = gm1 * ((h - R(0.5) * usq) - (bn2 + btsq) * irho) - gm2 * x;
    a2 = a2 > R(0) ? a2 : R(0);
    const R ct2 = btsq * irho;
    const R tdif = ca2 + ct2 - a2;
    const R cf = root_any(R(0.5) * ((a2 + ca2 + ct2) + root_any(tdif * tdif + R(4) * a2 * ct2)));
    sl = imin(wl[1] - cl, un - cf);
    sr = imax(wr[1] + cr, un + cf);
  }
  const R bm = ge0(sl) ? R(0) : sl;
  const R bp = gt0(sr) ? sr : R(0);
  const R iden = inv(bp - bm);
  const R bpm = bp * bm;
#pragma unroll
  for (int n = 0; n < 7; ++n) f[n] = ((mul_rn(bp, fl[n]) - mul_rn(bm, fr[n])) + bpm * (ur[n] - ul[n])) * iden;
}

// One side (L or R) of the HLLD fan: the state, its conserved vector and physical flux, and its
// single-star state.
template <class R>
struct HlldSide {
  R w[7];   // rho, v_n, v_t1, v_t2, p, b_t1, b_t2
  R u[7];   // conserved
  R f[7];   // physical flux
  R s;      // outer speed S_L or S_R
  R pt;     // total pressure
  R a;      // rho (S - v_n)
  R dst;    // rho*
  R vt[2];  // v_t*
  R bt[2];  // b_t*
  R est;    // E*
  R vbst;   // v* . B*
};

// Transverse velocity and field of the single-star state (degenerate case: unchanged).
template <class R>
__device__ __forceinline__ void hlld_star_vb(const R* w, R a, R s, R sm, R bn, R bn2, R ptst, R* vt, R* bt) {
  const R dd = a * (s - sm) - bn2;
  vt[0] = w[2];
  vt[1] = w[3];
  bt[0] = w[5];
  bt[1] = w[6];
  if (igt(fabs(dd), R(1e-8) * ptst)) {
    const R idd = inv(dd);
    const R tv = bn * (sm - w[1]) * idd;
    const R tb = (a * (s - w[1]) - bn2) * idd;
    vt[0] = w[2] - w[5] * tv;
    vt[1] = w[3] - w[6] * tv;
    bt[0] = w[5] * tb;
    bt[1] = w[6] * tb;
  }
}

// Flux of one side of the fan: outer state, single-star or double-star region.  `o` is the other
// side's raw state (used only in the double-star region).
template <class R>
__device__ __forceinline__ void hlld_side_flux(HlldSide<R>& S, const R* o_w, R o_s, R o_a, bool left, R sm,
                                               R bn, R bn2, R ptst, R* f) {
  const R isms = inv(S.s - sm);
  S.dst = S.a * isms;
  hlld_star_vb(S.w, S.a, S.s, sm, bn, bn2, ptst, S.vt, S.bt);
  const R vb = (S.w[1] * bn + S.w[2] * S.w[5]) + S.w[3] * S.w[6];
  S.vbst = (sm * bn + S.vt[0] * S.bt[0]) + S.vt[1] * S.bt[1];
  S.est = ((((S.s - S.w[1]) * S.u[4] - S.pt * S.w[1]) + ptst * sm) + bn * (vb - S.vbst)) * isms;
  const R rs = rroot(S.dst);
  const R abn = fabs(bn);
  const R sst = left ? sm - abn * rs : sm + abn * rs;
  // region: outer if the outer wave has not reached the interface, single star if the Alfven wave has not
  const bool outer = left ? ge0(S.s) : !gt0(S.s);
  const bool single = left ? ge0(sst) : !gt0(sst);
  R us[7];
  us[0] = S.dst;
  us[1] = S.dst * sm;
  us[2] = S.dst * S.vt[0];
  us[3] = S.dst * S.vt[1];
  us[4] = S.est;
  us[5] = S.bt[0];
  us[6] = S.bt[1];
#pragma unroll
  for (int n = 0; n < 7; ++n) f[n] = S.f[n];
  if (!outer) {
#pragma unroll
    for (int n = 0; n < 7; ++n) f[n] = f[n] + S.s * (us[n] - S.u[n]);
  }
  if (!outer && !single) {
    // double star: needs the other side's single-star density, velocity and field
    const R o_dst = o_a * inv(o_s - sm);
    R o_vt[2], o_bt[2];
    hlld_star_vb(o_w, o_a, o_s, sm, bn, bn2, ptst, o_vt, o_bt);
    const R sq = S.dst * rs;  // sqrt(rho*) of this side
    const R o_sq = root(o_dst);
    const R sql = left ? sq : o_sq, sqr = left ? o_sq : sq;
    const R* vtl = left ? S.vt : o_vt;
    const R* vtr = left ? o_vt : S.vt;
    const R* btl = left ? S.bt : o_bt;
    const R* btr = left ? o_bt : S.bt;
    const R sgn = ge0(bn) ? R(1) : R(-1);
    const R isq = inv(sql + sqr);
    const R vss1 = ((sql * vtl[0] + sqr * vtr[0]) + (btr[0] - btl[0]) * sgn) * isq;
    const R vss2 = ((sql * vtl[1] + sqr * vtr[1]) + (btr[1] - btl[1]) * sgn) * isq;
    const R bss1 = ((sql * btr[0] + sqr * btl[0]) + (sql * sqr) * (vtr[0] - vtl[0]) * sgn) * isq;
    const R bss2 = ((sql * btr[1] + sqr * btl[1]) + (sql * sqr) * (vtr[1] - vtl[1]) * sgn) * isq;
    const R vbss = (sm * bn + vss1 * bss1) + vss2 * bss2;
    // The density and the normal momentum rho* S_M do not change across the Alfven waves (U** and U* share
    // them), so the mass and normal-momentum fluxes stay the single-star ones; the other five components
    // take the jump sst (U** - U*).
    R uss[7];
    uss[2] = S.dst * vss1;
    uss[3] = S.dst * vss2;
    uss[4] = left ? S.est - sq * (S.vbst - vbss) * sgn : S.est + sq * (S.vbst - vbss) * sgn;
    uss[5] = bss1;
    uss[6] = bss2;
#pragma unroll
    for (int n = 2; n < 7; ++n) f[n] = f[n] + sst * (uss[n] - us[n]);
  }
}

// HLLD flux (Miyoshi & Kusano 2005; the paper names the solver in Sec. 3.2.2):
// outer speeds S_L = min(u_L,u_R) - max(c_L,c_R), S_R = max(u_L,u_R) + max(c_L,c_R); contact speed
// S_M and total pressure p_T* from the two-sided forms; single-star states (degenerate when
// |rho (S-u)(S-S_M) - b_n^2| <= 1e-8 p_T*); Alfven speeds S*_{L,R} = S_M -+ |b_n| / sqrt(rho*);
// double-star states with sign(0) = +1.  Selection: the sign of S_M picks the side, ties at an outer
// or Alfven speed of exactly zero take the outer state, S_M == 0 averages both sides.  Only the
// picked side's star state is formed (the other side's only in the double-star region).  Bitwise-equal
// states take the physical flux (same_state).
template <class R>
__device__ __forceinline__ void flux_hlld(const R* wl, const R* wr, R bn, R gamma, R igm1, R* f) {
  if (same_state(wl, wr)) {
    R u[7];
    phys_flux(wl, bn, igm1, u, f);
    return;
  }
  const R bn2 = bn * bn;
  const R btl2 = wl[5] * wl[5] + wl[6] * wl[6];
  const R btr2 = wr[5] * wr[5] + wr[6] * wr[6];
  // 1/(2 rho_L) and 1/(2 rho_R) from one reciprocal (the halving is exact, so rho_R (1/(2 rho_L rho_R)) is
  // bitwise (rho_R / (rho_L rho_R)) / 2)
  const R hlr = R(0.5) * inv(wl[0] * wr[0]);
  // max(C_f,L, C_f,R) = sqrt(max(C_f,L^2, C_f,R^2)): one square root for both sides
  const R cmax = root(imax(fast_speed2_h(wr[0] * hlr, wl[4], bn2, btl2, gamma),
                           fast_speed2_h(wl[0] * hlr, wr[4], bn2, btr2, gamma)));
  const R sl = imin(wl[1], wr[1]) - cmax;
  const R sr = imax(wl[1], wr[1]) + cmax;
  const R bbl = bn2 + btl2, bbr = bn2 + btr2;
  const R ptl = wl[4] + R(0.5) * bbl, ptr = wr[4] + R(0.5) * bbr;
  const R al = (sl - wl[1]) * wl[0], ar = (sr - wr[1]) * wr[0];
  const R iden = inv(ar - al);
  const R sm = ((mul_rn(ar, wr[1]) - mul_rn(al, wl[1])) + (ptl - ptr)) * iden;
  const R ptst = ((ar * ptl - al * ptr) + (ar * al) * (wr[1] - wl[1])) * iden;
  const bool left = ge0(sm);
  HlldSide<R> S;
#pragma unroll
  for (int n = 0; n < 7; ++n) S.w[n] = left ? wl[n] : wr[n];
  S.s = left ? sl : sr;
  S.pt = left ? ptl : ptr;
  S.a = left ? al : ar;
  phys_flux_bb(S.w, bn, igm1, left ? bbl : bbr, S.pt, S.u, S.f);
  const R* o_w = left ? wr : wl;
  hlld_side_flux(S, o_w, left ? sr : sl, left ? ar : al, left, sm, bn, bn2, ptst, f);
  if (is0(sm)) {  // both sides are valid at S_M == 0: average them (exact mirror symmetry)
    HlldSide<R> T;
#pragma unroll
    for (int n = 0; n < 7; ++n) T.w[n] = wr[n];
    T.s = sr;
    T.pt = ptr;
    T.a = ar;
    phys_flux_bb(T.w, bn, igm1, bbr, ptr, T.u, T.f);
    R g[7];
    hlld_side_flux(T, wl, sl, al, false, sm, bn, bn2, ptst, g);
#pragma unroll
    for (int n = 0; n < 7; ++n) f[n] = R(0.5) * (f[n] + g[n]);
  }
}

// Original van Leer limited slope on a uniform grid (Sec. 3.2.1).
template <class R>
__device__ __forceinline__ R vl_slope(R qm, R q0, R qp) {
  const R dl = q0 - qm, dr = qp - q0;
  const R pr = dl * dr;
  return gt0(pr) ? (R(2) * pr) / (dl + dr) : R(0);
}

// PLM values of one variable of a cell at its lower and upper faces from the cell (qc) and its two
// neighbours along the sweep (qm, qp), Sec. 3.2.1: q -+ delta/2 with the van Leer slope's half
// delta/2 = dl dr / (dl + dr) where dl dr > 0, else 0 (the slope's factor 2 and the 1/2 cancel exactly).
// The limiter denominator is inverted by the Newton reciprocal in FP64.  The fast build writes both face
// values as explicit fused multiply-adds, so that every kernel calling this (the forward sweeps and the
// adjoint's replay of them) rounds them alike whatever code surrounds it; the value-safe build (no
// contraction anywhere) multiplies and then adds.
template <class T>
__device__ __forceinline__ void plm_var_faces(T qm, T qc, T qp, T& lo, T& hi) {
  const T dl = qc - qm, dr = qp - qc;
  const bool pos = gt0(dl * dr);
  const T den = pos ? dl + dr : T(1);
  const T rc = sizeof(T) == 8 ? inv(den) : T(1) / den;
#ifdef VL2_VALUE_SAFE
  const T half = pos ? (dl * dr) * rc : T(0);
  lo = qc - half;
  hi = qc + half;
#else
  const T pr = pos ? dl * dr : T(0);
  lo = fma(-pr, rc, qc);
  hi = fma(pr, rc, qc);
#endif
}

// The same for the 7 sweep variables of one cell.
template <class T>
__device__ __forceinline__ void plm_cell_faces(const T* qm, const T* qc, const T* qp, T* lo, T* hi) {
#pragma unroll
  for (int n = 0; n < 7; ++n) plm_var_faces<T>(qm[n], qc[n], qp[n], lo[n], hi[n]);
}

// PPM (Sec. 3.2.1).  Face value: eq. ppm-uniform-weights, q_{i-1/2} = 7/12 (q_{i-1} + q_i) - 1/12 (q_{i-2} + q_{i+1});
// a face value outside the range of its two cells becomes (q_{i-1} + q_i)/2 - D2lim/6 with
// D2 = 3 (q_{i-1} + q_i - 2 q_{i-1/2}) limited by the neighbouring second differences (factor C = 1.25) when
// all share its sign, else 0 (Colella & Sekora 2008).  Cell: at an extremum the parabola's second
// derivative 6 (qL + qR - 2 q_i) is limited the same way against the second differences of the cells around
// and both edges move towards q_i by D2lim / D2; elsewhere an edge more than twice as far from q_i as the
// other is pulled in to twice that distance.  Second differences are (outer sum) - 2 middle, so mirrored
// inputs give mirrored results; comparisons run on the integer pipe.
template <class R> __device__ __forceinline__ int sgn3(R x) { return gt0(x) ? 1 : (lt0(x) ? -1 : 0); }
template <class R> __device__ __forceinline__ bool ige(R a, R b) { return okey(a) >= okey(b); }

template <class R>
__device__ __forceinline__ R ppm_face(R qm2, R qm1, R q0, R qp1) {
  const R C = R(1.25);
  R f = R(7.0 / 12.0) * (qm1 + q0) - R(1.0 / 12.0) * (qm2 + qp1);
  if (lt0((f - qm1) * (q0 - f))) {
    const R d2 = R(3) * ((qm1 + q0) - R(2) * f);
    const R d2l = (qm2 + q0) - R(2) * qm1;
    const R d2r = (qm1 + qp1) - R(2) * q0;
    const int s = sgn3(d2);
    R lim = R(0);
    if (s != 0 && sgn3(d2l) == s && sgn3(d2r) == s)
      lim = R(s) * imin(fabs(d2), imin(C * fabs(d2l), C * fabs(d2r)));
    f = R(0.5) * (qm1 + q0) - lim * R(1.0 / 6.0);
  }
  return f;
}

// The cell step: limits the edges (ql, qr) of cell i, given the face values, from q_{i-2} .. q_{i+2}.
template <class R>
__device__ __forceinline__ void ppm_cell(R qm2, R qm1, R q0, R qp1, R qp2, R& ql, R& qr) {
  const R C = R(1.25);
  if (!gt0((qr - q0) * (q0 - ql)) || !gt0((qp1 - q0) * (q0 - qm1))) {  // an extremum
    const R d2 = R(6) * ((ql + qr) - R(2) * q0);
    const R d2c = (qm1 + qp1) - R(2) * q0;
    const R d2l = (qm2 + q0) - R(2) * qm1;
    const R d2r = (q0 + qp2) - R(2) * qp1;
    const int s = sgn3(d2);
    if (s == 0) {
      ql = q0;
      qr = q0;
    } else {
      R lim = R(0);
      if (sgn3(d2c) == s && sgn3(d2l) == s && sgn3(d2r) == s)
        lim = R(s) * imin(fabs(d2), imin(C * fabs(d2c), imin(C * fabs(d2l), C * fabs(d2r))));
      const R r = lim * inv(d2);
      ql = q0 + r * (ql - q0);
      qr = q0 + r * (qr - q0);
    }
  } else {
    const R dl = ql - q0, dr = qr - q0;
    if (ige(fabs(dl), R(2) * fabs(dr))) ql = q0 - R(2) * dr;
    if (ige(fabs(dr), R(2) * fabs(dl))) qr = q0 - R(2) * dl;
  }
}

template <class R>
__device__ __forceinline__ void ppm_edges(R qm2, R qm1, R q0, R qp1, R qp2, R& ql, R& qr) {
  ql = ppm_face(qm2, qm1, q0, qp1);
  qr = ppm_face(qm1, q0, qp1, qp2);
  ppm_cell(qm2, qm1, q0, qp1, qp2, ql, qr);
}

// Characteristic PLM of one cell (Sec. 3.2.1: the limiter acts on C = L W).  q = (rho, v_n, v_t1, v_t2, p,
// b_t1, b_t2) of the cell and its two neighbours along the sweep, bn the cell's normal field.  The
// eigenvectors of the primitive system are those with the alpha/beta normalisation (finite where waves
// coincide; alpha evaluated without cancellation, exact at b_t = 0).  With it alpha_f^2 c_f^2 +
// alpha_s^2 c_s^2 = a^2, and the left eigenvectors take the closed form used below:
//   fast -+ : (0, -+C_f, +-Q_s beta, 0) / (2 a^2) + (alpha_f, A_s beta) / (2 rho a^2) on (v_n, v_t, p, b_t),
//   slow -+ : (0, -+C_s, -+Q_f beta, 0) / (2 a^2) + (alpha_s, -A_f beta) / (2 rho a^2),
//   Alfven -+: (v_t . beta_perp) / 2 +- s (b_t . beta_perp) / (2 sqrt(rho)), beta_perp = (-beta_2, beta_1),
//   entropy : d rho - dp / a^2.
// Each characteristic difference pair gets the van Leer half-slope c_l c_r / (c_l + c_r), the half-slopes
// are projected back with R, and each face value is kept within the range of the two cells sharing
// the face.  lo / hi: the values at the cell's lower / upper face.
template <class R>
struct CharSys {
  R rho, a2, af, as, b1, b2, sg, sr, Cf, Cs, Qf, Qs, Af, As, n2a, n2ra, hs;

  __device__ __forceinline__ void init(const R q0[7], R bn, R gamma) {
    rho = q0[0];
    const R irho = inv_any(rho);
    a2 = gamma * q0[4] * irho;
    const R ca2 = bn * bn * irho;
    const R btsq = q0[5] * q0[5] + q0[6] * q0[6];
    const R ct2 = btsq * irho;
    const R tdif = ca2 + ct2 - a2;
    const R root = root_any(tdif * tdif + R(4) * a2 * ct2);  // c_f^2 - c_s^2
    const R cf2 = R(0.5) * ((a2 + ca2 + ct2) + root);
    const R xs = a2 - ca2 + ct2;
    const R cf2_a2 = tdif >= R(0) ? R(0.5) * (tdif + root) : R(2) * a2 * ct2 * inv_any(root - tdif);
    const R cf2_ca2 = xs >= R(0) ? R(0.5) * (xs + root) : R(2) * ca2 * ct2 * inv_any(root - xs);
    const R icf2 = inv_any(cf2);
    af = R(1);
    as = R(0);
    if (root != R(0)) {
      const R ir = inv_any(root);
      af = root_any(a2 * cf2_ca2 * icf2 * ir);  // (a^2 - c_s^2) / (c_f^2 - c_s^2)
      as = root_any(cf2_a2 * ir);
    }
    const R a = root_any(a2), cf = root_any(cf2), cs = root_any(a2 * ca2 * icf2);
    b1 = R(0.70710678118654752440);
    b2 = R(0.70710678118654752440);
    if (btsq != R(0)) {
      const R ibt = rroot_any(btsq);
      b1 = q0[5] * ibt;
      b2 = q0[6] * ibt;
    }
    sg = bn >= R(0) ? R(1) : R(-1);
    sr = root_any(rho);
    const R isr = rroot_any(rho);
    Cf = cf * af;
    Cs = cs * as;
    Qf = sg * Cf;
    Qs = sg * Cs;
    Af = a * af * sr;
    As = a * as * sr;
    n2a = R(0.5) * inv_any(a2);
    n2ra = n2a * irho;
    hs = R(0.5) * sg * isr;
  }
  // c = L d, in the order of the eigenvalues v - c_f, v - c_a, v - c_s, v, v + c_s, v + c_a, v + c_f
  __device__ __forceinline__ void project(const R* d, R* c) const {
    const R vp = b1 * d[2] + b2 * d[3], va = b1 * d[3] - b2 * d[2];
    const R bp = b1 * d[5] + b2 * d[6], ba = b1 * d[6] - b2 * d[5];
    const R pf = n2ra * (af * d[4] + As * bp), ps = n2ra * (as * d[4] - Af * bp);
    const R uf = n2a * (Cf * d[1] - Qs * vp), us = n2a * (Cs * d[1] + Qf * vp);
    c[0] = pf - uf;
    c[1] = R(0.5) * va + hs * ba;
    c[2] = ps - us;
    c[3] = d[0] - R(2) * n2a * d[4];
    c[4] = ps + us;
    c[5] = R(0.5) * va - hs * ba;
    c[6] = pf + uf;
  }
  // d = R m
  __device__ __forceinline__ void back(const R* m, R* d) const {
    const R fsum = m[0] + m[6], ssum = m[2] + m[4];
    d[0] = rho * (af * fsum + as * ssum) + m[3];
    d[1] = Cf * (m[6] - m[0]) + Cs * (m[4] - m[2]);
    const R vp = Qs * (m[0] - m[6]) + Qf * (m[4] - m[2]), va = m[1] + m[5];
    d[2] = b1 * vp - b2 * va;
    d[3] = b2 * vp + b1 * va;
    d[4] = rho * a2 * (af * fsum + as * ssum);
    const R bp = As * fsum - Af * ssum, ba = sg * sr * (m[1] - m[5]);
    d[5] = b1 * bp - b2 * ba;
    d[6] = b2 * bp + b1 * ba;
  }
};

template <class R>
__device__ __forceinline__ R clamp_between(R x, R q1, R q2) {
  return fmin(fmax(x, fmin(q1, q2)), fmax(q1, q2));
}

template <class R>
__device__ __forceinline__ void char_plm_cell(const R qm[7], const R q0[7], const R qp[7], R bn, R gamma, R lo[7],
                                              R hi[7]) {
  CharSys<R> cs;
  cs.init(q0, bn, gamma);
  R m[7];
  {
    R dl[7], dr[7], cl[7], cr[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      dl[n] = q0[n] - qm[n];
      dr[n] = qp[n] - q0[n];
    }
    cs.project(dl, cl);
    cs.project(dr, cr);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      // where c_l c_r > 0 both are at least ~1e-162, so c_l + c_r is a normal number
      const bool pos = gt0(cl[k] * cr[k]);
      const R den = pos ? cl[k] + cr[k] : R(1);
      m[k] = pos ? (cl[k] * cr[k]) * inv(den) : R(0);
    }
  }
  R dh[7];  // half of the limited slope, back in primitives
  cs.back(m, dh);
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    lo[n] = clamp_between(q0[n] - dh[n], qm[n], q0[n]);
    hi[n] = clamp_between(q0[n] + dh[n], q0[n], qp[n]);
  }
}

// Characteristic PPM of one cell: the stencil differences q_j - q_0 (j = -2, -1, 1, 2) projected with the
// cell's L, the PPM edge steps on each characteristic field, both edges projected back with R, and each
// face value kept within the range of the two cells sharing the face.  qs[j][n] = stencil value j - 2.
template <class R>
__device__ __forceinline__ void char_ppm_cell(const R qs[5][7], R bn, R gamma, R lo[7], R hi[7]) {
  CharSys<R> cs;
  cs.init(qs[2], bn, gamma);
  R c[4][7];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    R d[7];
    const int s = j < 2 ? j : j + 1;
#pragma unroll
    for (int n = 0; n < 7; ++n) d[n] = qs[s][n] - qs[2][n];
    cs.project(d, c[j]);
  }
  R el[7], er[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) ppm_edges(c[0][k], c[1][k], R(0), c[2][k], c[3][k], el[k], er[k]);
  R dl[7], dr[7];
  cs.back(el, dl);
  cs.back(er, dr);
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    lo[n] = clamp_between(qs[2][n] + dl[n], qs[1][n], qs[2][n]);
    hi[n] = clamp_between(qs[2][n] + dr[n], qs[2][n], qs[3][n]);
  }
}

// Upwind CT corner EMF (Gardiner & Stone 2005) for an edge with transverse directions a, b:
// mean of the four face EMFs plus one quarter of the upwinded face-to-corner corrections.
// ea[0..1]: a-face EMFs at b-index -1, 0; eb[0..1]: b-face EMFs at a-index -1, 0;
// ec[0..3]: cell EMFs at (a-1,b-1), (a,b-1), (a-1,b), (a,b); ma, mb: the matching face mass fluxes.
//
// ct_pick: the upwind choice between two face-to-corner gradients lo = lo_a - lo_b (the lower cell's) and
// hi = hi_a - hi_b (the upper cell's) by the sign of the face mass flux m: lo where m > 0, hi where m < 0,
// their mean where m = 0.  In FP32 the operands are picked before the subtraction (one difference instead of
// two: the FP32 corner kernel measured 7% faster); in FP64 both differences are formed and the result
// picked (picking the 64-bit operands first measured 11% slower), with the same value either way.
template <class R>
__device__ __forceinline__ R ct_pick(R m, R lo_a, R lo_b, R hi_a, R hi_b) {
  if constexpr (sizeof(R) == 4) {
    if (is0(m)) return R(0.5) * ((lo_a - lo_b) + (hi_a - hi_b));
    const bool up = gt0(m);
    return (up ? lo_a : hi_a) - (up ? lo_b : hi_b);
  } else {
    const R lo = lo_a - lo_b, hi = hi_a - hi_b;
    return gt0(m) ? lo : (lt0(m) ? hi : R(0.5) * (lo + hi));
  }
}

// [option, not the paper's method] smoothed upwind weight: w = (1 + tanh(m / delta)) / 2 on the gradient of the
// cell the mass flux m comes from, 1 - w on the other.  Where |m| > 20 delta, 1 - |tanh(m / delta)| < 1e-17 is
// below half an ulp of 1 (2^-54), so tanh rounds to +-1 and w to exactly 1 or 0: the sign switch's pick,
// taken here without the tanh.  At m = 0, w = 1/2 is the switch's mean.
// Inside the band the weight is evaluated as (1 + tanh x) / 2 = 1 / (1 + exp(-2x)), x = m / delta: one
// exponential and a reciprocal (|x| <= 20 keeps exp(-2x) within [4e-18, 3e17]).
template <class R>
__device__ __forceinline__ R ct_weight(R m, R delta, R band) {
  if (fabs(m) > band) return m > R(0) ? R(1) : R(0);
  if (m == R(0)) return R(0.5);  // tanh(0) = 0; also where delta underflows to 0 in R
  return inv(R(1) + exp(R(-2) * (m / delta)));
}

template <class R>
__device__ __forceinline__ R ct_pick_w(R w, R lo, R hi) {
  return w == R(1) ? lo : (w == R(0) ? hi : w * lo + (R(1) - w) * hi);
}

// The corner EMF with upwind picks by sign (SMOOTH false: ma, mb are the face mass fluxes) or by the weights
// above (SMOOTH true: ma, mb are already the weights of those faces).
template <class R, bool SMOOTH = false>
__device__ __forceinline__ R ct_corner(const R* ea, const R* eb, const R* ec, const R* ma, const R* mb) {
  const R sum4 = (ea[0] + ea[1]) + (eb[0] + eb[1]);
  if constexpr (SMOOTH) {
    const R tlo = ct_pick_w(ma[0], eb[0] - ec[0], eb[1] - ec[1]);
    const R thi = ct_pick_w(ma[1], ec[2] - eb[0], ec[3] - eb[1]);
    const R slo = ct_pick_w(mb[0], ea[0] - ec[0], ea[1] - ec[2]);
    const R shi = ct_pick_w(mb[1], ec[1] - ea[0], ec[3] - ea[1]);
    return (R(0.25) * sum4 + R(0.25) * (tlo - thi)) + R(0.25) * (slo - shi);
  }
  const R tlo = ct_pick(ma[0], eb[0], ec[0], eb[1], ec[1]);
  const R thi = ct_pick(ma[1], ec[2], eb[0], ec[3], eb[1]);
  const R slo = ct_pick(mb[0], ea[0], ec[0], ea[1], ec[2]);
  const R shi = ct_pick(mb[1], ec[1], ea[0], ec[3], ea[1]);
  return (R(0.25) * sum4 + R(0.25) * (tlo - thi)) + R(0.25) * (slo - shi);
}

}  // namespace vl2
