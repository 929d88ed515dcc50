// Device physics of the VL2 MHD step (Stone et al. 2020, arXiv:2005.06651, Sec. 3.1-3.2).
// Interface states are 7-vectors in the sweep frame (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) with
// (n, t1, t2) = (x, y, z), (y, z, x), (z, x, y); fluxes use the same slots (mass, M_n, M_t1, M_t2,
// E, B_t1, B_t2).  Reciprocals are formed once and reused; FMA contraction is allowed.
#pragma once
#include <cuda_runtime.h>

namespace vl2 {

// Fast magnetosonic speed along the normal (Sec. 2.1.7 uses |v| + C_f):
// C_f^2 = (a^2 + c_n^2 + c_t^2 + sqrt((a^2 - c_n^2)^2 + c_t^2 (c_t^2 + 2 a^2 + 2 c_n^2))) / 2,
// a^2 = gamma p / rho, c_n^2 = b_n^2 / rho, c_t^2 = |b_t|^2 / rho.
template <class R>
__device__ __forceinline__ R fast_speed_r(R id, R p, R bn2, R bt2, R gamma) {
  const R asq = gamma * p * id;
  const R cn = bn2 * id;
  const R ct = bt2 * id;
  const R df = asq - cn;
  const R rad = df * df + ct * (ct + R(2) * (asq + cn));
  return sqrt(R(0.5) * ((asq + cn + ct) + sqrt(rad)));
}

// Conserved 7-vector and physical flux of one sweep-frame state (eq. cons, eq. total_energy).
template <class R>
__device__ __forceinline__ void phys_flux(const R* w, R bn, R igm1, R* u, R* f) {
  const R d = w[0], vn = w[1], v1 = w[2], v2 = w[3], p = w[4], b1 = w[5], b2 = w[6];
  const R bb = (bn * bn + b1 * b1) + b2 * b2;
  const R e = p * igm1 + R(0.5) * d * ((vn * vn + v1 * v1) + v2 * v2) + R(0.5) * bb;
  const R pt = p + R(0.5) * bb;
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

// HLLE flux; outer speeds are the extreme fast-wave speeds of the two states (Sec. 3.2.2 names the
// solver; the speed estimate is this library's reading).
template <class R>
__device__ __forceinline__ void flux_hlle(const R* wl, const R* wr, R bn, R gamma, R igm1, R* f) {
  R ul[7], fl[7], ur[7], fr[7];
  phys_flux(wl, bn, igm1, ul, fl);
  phys_flux(wr, bn, igm1, ur, fr);
  const R bn2 = bn * bn;
  const R cl = fast_speed_r(R(1) / wl[0], wl[4], bn2, wl[5] * wl[5] + wl[6] * wl[6], gamma);
  const R cr = fast_speed_r(R(1) / wr[0], wr[4], bn2, wr[5] * wr[5] + wr[6] * wr[6], gamma);
  const R sl = fmin(wl[1] - cl, wr[1] - cr);
  const R sr = fmax(wl[1] + cl, wr[1] + cr);
  const R bm = fmin(sl, R(0));
  const R bp = fmax(sr, R(0));
  const R iden = R(1) / (bp - bm);
  const R bpm = bp * bm;
#pragma unroll
  for (int n = 0; n < 7; ++n) f[n] = ((bp * fl[n] - bm * fr[n]) + bpm * (ur[n] - ul[n])) * iden;
}

// HLLD flux (Miyoshi & Kusano 2005; the paper names the solver in Sec. 3.2.2):
// outer speeds S_L = min(u_L,u_R) - max(c_L,c_R), S_R = max(u_L,u_R) + max(c_L,c_R); contact speed
// S_M and total pressure p_T* from the two-sided forms; single-star states (degenerate when
// |rho (S-u)(S-S_M) - b_n^2| <= 1e-8 p_T*); Alfven speeds S*_{L,R} = S_M -+ |b_n| / sqrt(rho*);
// double-star states with sign(0) = +1.  Selection: the sign of S_M picks the side, ties at an outer
// or Alfven speed of exactly zero take the outer state, S_M == 0 averages both sides.
template <class R>
__device__ __forceinline__ void flux_hlld(const R* wl, const R* wr, R bn, R gamma, R igm1, R* f) {
  R uo[2][7], fo[2][7];
  phys_flux(wl, bn, igm1, uo[0], fo[0]);
  phys_flux(wr, bn, igm1, uo[1], fo[1]);
  const R bn2 = bn * bn;
  const R idl = R(1) / wl[0], idr = R(1) / wr[0];
  const R btl2 = wl[5] * wl[5] + wl[6] * wl[6];
  const R btr2 = wr[5] * wr[5] + wr[6] * wr[6];
  const R cl = fast_speed_r(idl, wl[4], bn2, btl2, gamma);
  const R cr = fast_speed_r(idr, wr[4], bn2, btr2, gamma);
  const R cmax = fmax(cl, cr);
  const R s[2] = {fmin(wl[1], wr[1]) - cmax, fmax(wl[1], wr[1]) + cmax};
  const R pt[2] = {wl[4] + R(0.5) * (bn2 + btl2), wr[4] + R(0.5) * (bn2 + btr2)};
  const R a[2] = {(s[0] - wl[1]) * wl[0], (s[1] - wr[1]) * wr[0]};
  const R iden = R(1) / (a[1] - a[0]);
  const R sm = ((a[1] * wr[1] - a[0] * wl[1]) + (pt[0] - pt[1])) * iden;
  const R ptst = ((a[1] * pt[0] - a[0] * pt[1]) + (a[1] * a[0]) * (wr[1] - wl[1])) * iden;

  R us[2][7], vbst[2], dst[2], vst[2][2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const R* w = side ? wr : wl;
    const R sms = s[side] - sm;
    const R isms = R(1) / sms;
    const R dd = a[side] * sms - bn2;
    R vt1 = w[2], vt2 = w[3], bt1 = w[5], bt2 = w[6];
    if (fabs(dd) > R(1e-8) * ptst) {
      const R idd = R(1) / dd;
      const R tv = bn * (sm - w[1]) * idd;
      const R tb = (a[side] * (s[side] - w[1]) - bn2) * idd;
      vt1 = w[2] - w[5] * tv;
      vt2 = w[3] - w[6] * tv;
      bt1 = w[5] * tb;
      bt2 = w[6] * tb;
    }
    dst[side] = a[side] * isms;
    vst[side][0] = vt1;
    vst[side][1] = vt2;
    const R vb = (w[1] * bn + w[2] * w[5]) + w[3] * w[6];
    vbst[side] = (sm * bn + vt1 * bt1) + vt2 * bt2;
    us[side][0] = dst[side];
    us[side][1] = dst[side] * sm;
    us[side][2] = dst[side] * vt1;
    us[side][3] = dst[side] * vt2;
    us[side][4] = ((((s[side] - w[1]) * uo[side][4] - pt[side] * w[1]) + ptst * sm) + bn * (vb - vbst[side])) * isms;
    us[side][5] = bt1;
    us[side][6] = bt2;
  }
  const R rsl = rsqrt(dst[0]), rsr = rsqrt(dst[1]);
  const R sql = dst[0] * rsl, sqr = dst[1] * rsr;  // sqrt(rho*_L), sqrt(rho*_R)
  const R abn = fabs(bn);
  const R sst[2] = {sm - abn * rsl, sm + abn * rsr};
  const R sgn = (bn >= R(0)) ? R(1) : R(-1);
  const R isq = R(1) / (sql + sqr);
  const R vss1 = ((sql * vst[0][0] + sqr * vst[1][0]) + (us[1][5] - us[0][5]) * sgn) * isq;
  const R vss2 = ((sql * vst[0][1] + sqr * vst[1][1]) + (us[1][6] - us[0][6]) * sgn) * isq;
  const R bss1 = ((sql * us[1][5] + sqr * us[0][5]) + (sql * sqr) * (vst[1][0] - vst[0][0]) * sgn) * isq;
  const R bss2 = ((sql * us[1][6] + sqr * us[0][6]) + (sql * sqr) * (vst[1][1] - vst[0][1]) * sgn) * isq;
  const R vbss = (sm * bn + vss1 * bss1) + vss2 * bss2;

  // region on each side: 0 outer, 1 single star, 2 double star
  const int regl = (s[0] >= R(0)) ? 0 : ((sst[0] >= R(0)) ? 1 : 2);
  const int regr = (s[1] <= R(0)) ? 0 : ((sst[1] <= R(0)) ? 1 : 2);
  const bool use_l = sm >= R(0);
  const bool use_r = sm <= R(0);
  R fsum[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) fsum[n] = R(0);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (side == 0 ? !use_l : !use_r) continue;
    const int reg = side ? regr : regl;
    R fl[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) fl[n] = fo[side][n];
    if (reg >= 1) {
#pragma unroll
      for (int n = 0; n < 7; ++n) fl[n] = fl[n] + s[side] * (us[side][n] - uo[side][n]);
    }
    if (reg == 2) {
      R uss[7];
      uss[0] = dst[side];
      uss[1] = dst[side] * sm;
      uss[2] = dst[side] * vss1;
      uss[3] = dst[side] * vss2;
      uss[4] = side ? us[1][4] + sqr * (vbst[1] - vbss) * sgn : us[0][4] - sql * (vbst[0] - vbss) * sgn;
      uss[5] = bss1;
      uss[6] = bss2;
#pragma unroll
      for (int n = 0; n < 7; ++n) fl[n] = fl[n] + sst[side] * (uss[n] - us[side][n]);
    }
#pragma unroll
    for (int n = 0; n < 7; ++n) fsum[n] = fsum[n] + fl[n];
  }
  const R scale = (use_l && use_r) ? R(0.5) : R(1);
#pragma unroll
  for (int n = 0; n < 7; ++n) f[n] = fsum[n] * scale;
}

// Original van Leer limited slope on a uniform grid (Sec. 3.2.1).
template <class R>
__device__ __forceinline__ R vl_slope(R qm, R q0, R qp) {
  const R dl = q0 - qm, dr = qp - q0;
  const R pr = dl * dr;
  return (pr > R(0)) ? (R(2) * pr) / (dl + dr) : R(0);
}

// Upwind CT corner EMF (Gardiner & Stone 2005) for an edge with transverse directions a, b:
// mean of the four face EMFs plus one quarter of the upwinded face-to-corner corrections.
// ea[0..1]: a-face EMFs at b-index -1, 0; eb[0..1]: b-face EMFs at a-index -1, 0;
// ec[0..3]: cell EMFs at (a-1,b-1), (a,b-1), (a-1,b), (a,b); ma, mb: the matching face mass fluxes.
__device__ __forceinline__ double ct_pick(double m, double lo, double hi) {
  return (m > 0.0) ? lo : ((m < 0.0) ? hi : 0.5 * (lo + hi));
}

__device__ __forceinline__ double ct_corner(const double* ea, const double* eb, const double* ec,
                                            const double* ma, const double* mb) {
  const double sum4 = (ea[0] + ea[1]) + (eb[0] + eb[1]);
  const double tlo = ct_pick(ma[0], eb[0] - ec[0], eb[1] - ec[1]);
  const double thi = ct_pick(ma[1], ec[2] - eb[0], ec[3] - eb[1]);
  const double slo = ct_pick(mb[0], ea[0] - ec[0], ea[1] - ec[2]);
  const double shi = ct_pick(mb[1], ec[1] - ea[0], ec[3] - ea[1]);
  return (0.25 * sum4 + 0.25 * (tlo - thi)) + 0.25 * (slo - shi);
}

}  // namespace vl2
