// Reverse-mode derivatives (vector-Jacobian products) of the device Riemann fluxes in FP64:
//   given lam_F (7), return lam_F . dF/dw_L, lam_F . dF/dw_R and lam_F . dF/db_n
// for the flux functions of vl2_physics.cuh (HLLE and the one-sided HLLD, Sec. 3.2.2).  Each function
// first recomputes the forward values with the same arithmetic and branch decisions as the forward flux
// (so a region, degeneracy or upwind choice is the one the forward step took), then runs the chain rule
// backwards through the same statements.  Derivatives are those of the exact formulas: 1/rho is
// differentiated as 1/rho even where the forward forms it from a joint reciprocal, sqrt and the fast
// speed by their closed-form derivatives.  At a point where a branch switches, the derivative of the
// branch the forward took is returned (a piecewise-smooth map's one-sided derivative).
#pragma once
#include "vl2_physics.cuh"

namespace vl2 {

// ---- physical flux: u(w), f(w, b_n) -----------------------------------------------------------------
// gu, gf: adjoints of u and f; adds into gw[7] and gbn.
__device__ __forceinline__ void phys_flux_vjp(const double* w, double bn, double igm1, const double* gu,
                                              const double* gf, double* gw, double& gbn) {
  const double d = w[0], vn = w[1], v1 = w[2], v2 = w[3], b1 = w[5], b2 = w[6];
  const double bb = (bn * bn + b1 * b1) + b2 * b2;
  const double v2s = (vn * vn + v1 * v1) + v2 * v2;
  const double e = w[4] * igm1 + 0.5 * d * v2s + 0.5 * bb;
  const double pt = w[4] + 0.5 * bb;
  const double vb = (vn * bn + v1 * b1) + v2 * b2;
  const double m = d * vn;
  // f0 = m; f1 = m vn + pt - bn^2; f2 = m v1 - bn b1; f3 = m v2 - bn b2; f4 = (e + pt) vn - bn vb;
  // f5 = b1 vn - bn v1; f6 = b2 vn - bn v2;   u = (d, m, d v1, d v2, e, b1, b2)
  const double gm = gu[1] + gf[0] + gf[1] * vn + gf[2] * v1 + gf[3] * v2;
  const double ge = gu[4] + gf[4] * vn;
  const double gpt = gf[1] + gf[4] * vn;
  const double gvb = -gf[4] * bn;
  const double gbb = 0.5 * (ge + gpt);
  gw[0] += gu[0] + gm * vn + 0.5 * ge * v2s + gu[2] * v1 + gu[3] * v2;
  gw[1] += gf[1] * m + gf[4] * (e + pt) + gf[5] * b1 + gf[6] * b2 + gvb * bn + gm * d + ge * d * vn;
  gw[2] += gf[2] * m - gf[5] * bn + gvb * b1 + gu[2] * d + ge * d * v1;
  gw[3] += gf[3] * m - gf[6] * bn + gvb * b2 + gu[3] * d + ge * d * v2;
  gw[4] += ge * igm1 + gpt;
  gw[5] += gu[5] - gf[2] * bn + gf[5] * vn + gvb * v1 + 2.0 * gbb * b1;
  gw[6] += gu[6] - gf[3] * bn + gf[6] * vn + gvb * v2 + 2.0 * gbb * b2;
  gbn += -2.0 * bn * gf[1] - gf[2] * b1 - gf[3] * b2 - gf[4] * vb - gf[5] * v1 - gf[6] * v2 + gvb * vn +
         2.0 * gbb * bn;
}

// ---- fast magnetosonic speed c(id, p, bn2, bt2) (fast_speed_r) ----------------------------------------
// Adds the adjoints of id = 1/rho, p, b_n^2 and |b_t|^2.
__device__ __forceinline__ void fast_speed_vjp(double id, double p, double bn2, double bt2, double gamma, double gc,
                                               double& gid, double& gp, double& gbn2, double& gbt2) {
  const double asq = gamma * p * id, cn = bn2 * id, ct = bt2 * id;
  const double df = asq - cn;
  const double rad = df * df + ct * (ct + 2.0 * (asq + cn));
  const double R = sqrt_nr(rad);
  const double X = 0.5 * ((asq + cn + ct) + R);
  const double c = sqrt_nr(X);
  const double gX = gc * 0.5 * rcp_nr(c);
  const double gA = 0.5 * gX;
  // R = |df| where rad = 0 (no transverse field and a = c_n): its derivative is not defined; take 0
  const double gR = 0.5 * gX;
  const double grad = ((__double_as_longlong(R) << 1) == 0) ? 0.0 : gR * 0.5 * rcp_nr(R);
  const double gdf = grad * 2.0 * df;
  const double gct = grad * (2.0 * ct + 2.0 * (asq + cn)) + gA;
  const double gasq = grad * 2.0 * ct + gdf + gA;
  const double gcn = grad * 2.0 * ct - gdf + gA;
  gp += gasq * gamma * id;
  gid += gasq * gamma * p + gcn * bn2 + gct * bt2;
  gbn2 += gcn * id;
  gbt2 += gct * id;
}

// ---- HLLE ----------------------------------------------------------------------------------------------
__device__ __forceinline__ void flux_hlle_vjp(const double* wl, const double* wr, double bn, double gamma, double igm1,
                                              const double* lf, double* gwl, double* gwr, double& gbn) {
  double ul[7], fl[7], ur[7], fr[7];
  phys_flux(wl, bn, igm1, ul, fl);
  phys_flux(wr, bn, igm1, ur, fr);
  const double bn2 = bn * bn;
  const double btl2 = wl[5] * wl[5] + wl[6] * wl[6], btr2 = wr[5] * wr[5] + wr[6] * wr[6];
  const double ilr = rcp_nr(wl[0] * wr[0]);
  const double idl = wr[0] * ilr, idr = wl[0] * ilr;
  const double cl = fast_speed_r(idl, wl[4], bn2, btl2, gamma);
  const double cr = fast_speed_r(idr, wr[4], bn2, btr2, gamma);
  const double a0 = wl[1] - cl, a1 = wr[1] - cr, c0 = wl[1] + cl, c1 = wr[1] + cr;
  const bool sl_right = !(okey(a0) < okey(a1));  // imin(a0, a1) picked a1
  const bool sr_right = !(okey(c0) > okey(c1));  // imax(c0, c1) picked c1
  const double sl = sl_right ? a1 : a0, sr = sr_right ? c1 : c0;
  const bool bm_on = !ge0(sl), bp_on = gt0(sr);
  const double bm = bm_on ? sl : 0.0, bp = bp_on ? sr : 0.0;
  const double iden = rcp_nr(bp - bm);
  const double bpm = bp * bm;
  double giden = 0.0, gbp = 0.0, gbm = 0.0, gbpm = 0.0;
  double gul[7], gfl[7], gur[7], gfr[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const double N = (mul_rn(bp, fl[n]) - mul_rn(bm, fr[n])) + bpm * (ur[n] - ul[n]);
    giden += lf[n] * N;
    const double gN = lf[n] * iden;
    gfl[n] = gN * bp;
    gfr[n] = -gN * bm;
    gur[n] = gN * bpm;
    gul[n] = -gN * bpm;
    gbp += gN * fl[n];
    gbm -= gN * fr[n];
    gbpm += gN * (ur[n] - ul[n]);
  }
  gbp += gbpm * bm - giden * iden * iden;
  gbm += gbpm * bp + giden * iden * iden;
  const double gsl = bm_on ? gbm : 0.0, gsr = bp_on ? gbp : 0.0;
  double gcl = 0.0, gcr = 0.0;
  if (sl_right) {
    gwr[1] += gsl;
    gcr -= gsl;
  } else {
    gwl[1] += gsl;
    gcl -= gsl;
  }
  if (sr_right) {
    gwr[1] += gsr;
    gcr += gsr;
  } else {
    gwl[1] += gsr;
    gcl += gsr;
  }
  double gidl = 0.0, gidr = 0.0, gbn2 = 0.0, gbtl2 = 0.0, gbtr2 = 0.0;
  fast_speed_vjp(idl, wl[4], bn2, btl2, gamma, gcl, gidl, gwl[4], gbn2, gbtl2);
  fast_speed_vjp(idr, wr[4], bn2, btr2, gamma, gcr, gidr, gwr[4], gbn2, gbtr2);
  gwl[0] -= gidl * idl * idl;
  gwr[0] -= gidr * idr * idr;
  gwl[5] += 2.0 * wl[5] * gbtl2;
  gwl[6] += 2.0 * wl[6] * gbtl2;
  gwr[5] += 2.0 * wr[5] * gbtr2;
  gwr[6] += 2.0 * wr[6] * gbtr2;
  gbn += 2.0 * bn * gbn2;
  phys_flux_vjp(wl, bn, igm1, gul, gfl, gwl, gbn);
  phys_flux_vjp(wr, bn, igm1, gur, gfr, gwr, gbn);
}

// ---- HLLD ------------------------------------------------------------------------------------------------
// Single-star transverse velocity and field of one side (hlld_star_vb), with what its reverse needs.
struct StarFwd {
  bool nondeg;
  double idd, tv, tb, vt[2], bt[2];
};
__device__ __forceinline__ void hlld_star_fwd(const double* w, double a, double s, double sm, double bn, double bn2,
                                              double ptst, StarFwd& z) {
  const double dd = a * (s - sm) - bn2;
  z.nondeg = igt(fabs(dd), 1e-8 * ptst);
  z.vt[0] = w[2];
  z.vt[1] = w[3];
  z.bt[0] = w[5];
  z.bt[1] = w[6];
  z.idd = z.tv = z.tb = 0.0;
  if (z.nondeg) {
    z.idd = rcp_nr(dd);
    z.tv = bn * (sm - w[1]) * z.idd;
    z.tb = (a * (s - w[1]) - bn2) * z.idd;
    z.vt[0] = w[2] - w[5] * z.tv;
    z.vt[1] = w[3] - w[6] * z.tv;
    z.bt[0] = w[5] * z.tb;
    z.bt[1] = w[6] * z.tb;
  }
}
__device__ __forceinline__ void hlld_star_vjp(const double* w, double a, double s, double sm, double bn, double bn2,
                                              const StarFwd& z, const double* gvt, const double* gbt, double* gw,
                                              double& ga, double& gs, double& gsm, double& gbn, double& gbn2) {
  gw[2] += gvt[0];
  gw[3] += gvt[1];
  if (!z.nondeg) {
    gw[5] += gbt[0];
    gw[6] += gbt[1];
    return;
  }
  // vt = (w2 - w5 tv, w3 - w6 tv), bt = (w5 tb, w6 tb)
  gw[5] += gbt[0] * z.tb - gvt[0] * z.tv;
  gw[6] += gbt[1] * z.tb - gvt[1] * z.tv;
  const double gtv = -(gvt[0] * w[5] + gvt[1] * w[6]);
  const double gtb = gbt[0] * w[5] + gbt[1] * w[6];
  // tv = TV idd, TV = bn (sm - w1); tb = TB idd, TB = a (s - w1) - bn2; idd = 1/dd, dd = a (s - sm) - bn2
  const double TV = bn * (sm - w[1]);
  const double TB = a * (s - w[1]) - bn2;
  const double gTV = gtv * z.idd, gTB = gtb * z.idd;
  const double gdd = -(gtv * TV + gtb * TB) * z.idd * z.idd;
  gbn += gTV * (sm - w[1]);
  gsm += gTV * bn - gdd * a;
  gw[1] -= gTV * bn + gTB * a;
  ga += gTB * (s - w[1]) + gdd * (s - sm);
  gs += gTB * a + gdd * a;
  gbn2 -= gTB + gdd;
}

// Reverse of hlld_side_flux for one side: w, s, pt, a of the side; o_w, o_s, o_a of the other side (used in
// the double-star region).  gF is the adjoint of the side's flux.  Adds into the adjoints of all of them and
// of sm, ptst, bn and bn^2.
__device__ __forceinline__ void hlld_side_vjp(const double* w, double s, double pt, double a, const double* o_w,
                                              double o_s, double o_a, bool left, double sm, double bn, double bn2,
                                              double ptst, double igm1, const double* gF, double* gw, double& gs,
                                              double& gpt, double& ga, double* gow, double& gos, double& goa,
                                              double& gsm, double& gptst, double& gbn, double& gbn2) {
  // forward values
  double u[7], f[7];
  phys_flux(w, bn, igm1, u, f);
  const double X = s - sm;
  const double isms = rcp_nr(X);
  const double dst = a * isms;
  StarFwd z;
  hlld_star_fwd(w, a, s, sm, bn, bn2, ptst, z);
  const double vb = (w[1] * bn + w[2] * w[5]) + w[3] * w[6];
  const double vbst = (sm * bn + z.vt[0] * z.bt[0]) + z.vt[1] * z.bt[1];
  const double EN = (((s - w[1]) * u[4] - pt * w[1]) + ptst * sm) + bn * (vb - vbst);
  const double est = EN * isms;
  const double rs = rsqrt(dst);
  const double abn = fabs(bn);
  const double tau = left ? -1.0 : 1.0;  // sst = sm + tau |bn| / sqrt(rho*)
  const double sst = sm + tau * abn * rs;
  const bool outer = left ? ge0(s) : !gt0(s);
  const bool single = left ? ge0(sst) : !gt0(sst);
  const double us[7] = {dst, dst * sm, dst * z.vt[0], dst * z.vt[1], est, z.bt[0], z.bt[1]};
  // reverse
  double gu[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double gus[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double gdst = 0.0, gest = 0.0, grs = 0.0, gabn = 0.0, gvbst = 0.0;
  double gvt[2] = {0.0, 0.0}, gbt[2] = {0.0, 0.0};
  if (!outer && !single) {
    const double io = rcp_nr(o_s - sm);
    const double o_dst = o_a * io;
    StarFwd oz;
    hlld_star_fwd(o_w, o_a, o_s, sm, bn, bn2, ptst, oz);
    const double sq = dst * rs;
    const double o_sq = sqrt_nr(o_dst);
    const double sql = left ? sq : o_sq, sqr = left ? o_sq : sq;
    const double* vtl = left ? z.vt : oz.vt;
    const double* vtr = left ? oz.vt : z.vt;
    const double* btl = left ? z.bt : oz.bt;
    const double* btr = left ? oz.bt : z.bt;
    const double sgn = ge0(bn) ? 1.0 : -1.0;
    const double isq = rcp_nr(sql + sqr);
    double NV[2], NB[2], vss[2], bss[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      NV[k] = (sql * vtl[k] + sqr * vtr[k]) + (btr[k] - btl[k]) * sgn;
      NB[k] = (sql * btr[k] + sqr * btl[k]) + (sql * sqr) * (vtr[k] - vtl[k]) * sgn;
      vss[k] = NV[k] * isq;
      bss[k] = NB[k] * isq;
    }
    const double vbss = (sm * bn + vss[0] * bss[0]) + vss[1] * bss[1];
    const double sigma = left ? -1.0 : 1.0;  // uss[4] = est + sigma sq (vbst - vbss) sgn
    const double uss[7] = {dst, dst * sm, dst * vss[0], dst * vss[1], est + sigma * sq * (vbst - vbss) * sgn,
                           bss[0], bss[1]};
    // F += sst (uss - us)
    double gsst = 0.0, guss[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      gsst += gF[n] * (uss[n] - us[n]);
      guss[n] = gF[n] * sst;
      gus[n] -= gF[n] * sst;
    }
    gdst += guss[0] + guss[1] * sm + guss[2] * vss[0] + guss[3] * vss[1];
    gsm += guss[1] * dst;
    double gvss[2] = {guss[2] * dst, guss[3] * dst};
    double gbss[2] = {guss[5], guss[6]};
    gest += guss[4];
    double gsq = guss[4] * sigma * sgn * (vbst - vbss);
    gvbst += guss[4] * sigma * sgn * sq;
    const double gvbss = -guss[4] * sigma * sgn * sq;
    gsm += gvbss * bn;
    gbn += gvbss * sm;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      gvss[k] += gvbss * bss[k];
      gbss[k] += gvbss * vss[k];
    }
    double gisq = 0.0, gsql = 0.0, gsqr = 0.0;
    double gvtl[2] = {0.0, 0.0}, gvtr[2] = {0.0, 0.0}, gbtl[2] = {0.0, 0.0}, gbtr[2] = {0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double dv = vtr[k] - vtl[k];
      const double gNB = gbss[k] * isq;
      gisq += gbss[k] * NB[k];
      gsql += gNB * (btr[k] + sqr * dv * sgn);
      gsqr += gNB * (btl[k] + sql * dv * sgn);
      gbtr[k] += gNB * sql;
      gbtl[k] += gNB * sqr;
      gvtr[k] += gNB * sql * sqr * sgn;
      gvtl[k] -= gNB * sql * sqr * sgn;
      const double gNV = gvss[k] * isq;
      gisq += gvss[k] * NV[k];
      gsql += gNV * vtl[k];
      gsqr += gNV * vtr[k];
      gvtl[k] += gNV * sql;
      gvtr[k] += gNV * sqr;
      gbtr[k] += gNV * sgn;
      gbtl[k] -= gNV * sgn;
    }
    const double gQ = -gisq * isq * isq;
    gsql += gQ;
    gsqr += gQ;
    double gosq, govt[2], gobt[2];
    if (left) {
      gsq += gsql;
      gosq = gsqr;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        gvt[k] += gvtl[k];
        gbt[k] += gbtl[k];
        govt[k] = gvtr[k];
        gobt[k] = gbtr[k];
      }
    } else {
      gsq += gsqr;
      gosq = gsql;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        gvt[k] += gvtr[k];
        gbt[k] += gbtr[k];
        govt[k] = gvtl[k];
        gobt[k] = gbtl[k];
      }
    }
    gdst += gsq * 0.5 * rs;  // sq = sqrt(rho*)
    const double godst = gosq * 0.5 * rcp_nr(o_sq);
    hlld_star_vjp(o_w, o_a, o_s, sm, bn, bn2, oz, govt, gobt, gow, goa, gos, gsm, gbn, gbn2);
    // o_dst = o_a / (o_s - sm)
    goa += godst * io;
    const double goX = -godst * o_a * io * io;
    gos += goX;
    gsm -= goX;
    // sst = sm + tau |bn| rs
    gsm += gsst;
    gabn += tau * gsst * rs;
    grs += tau * gsst * abn;
  }
  if (!outer) {  // F += s (us - u)
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      gs += gF[n] * (us[n] - u[n]);
      gus[n] += gF[n] * s;
      gu[n] -= gF[n] * s;
    }
  }
  // us = (dst, dst sm, dst vt0, dst vt1, est, bt0, bt1)
  gdst += gus[0] + gus[1] * sm + gus[2] * z.vt[0] + gus[3] * z.vt[1];
  gsm += gus[1] * dst;
  gvt[0] += gus[2] * dst;
  gvt[1] += gus[3] * dst;
  gest += gus[4];
  gbt[0] += gus[5];
  gbt[1] += gus[6];
  gdst -= 0.5 * grs * rs * rs * rs;  // rs = dst^(-1/2)
  gbn += ge0(bn) ? gabn : -gabn;
  // est = EN isms, EN = (s - w1) u4 - pt w1 + ptst sm + bn (vb - vbst)
  const double gEN = gest * isms;
  double gisms = gest * EN;
  gs += gEN * u[4];
  gw[1] -= gEN * (u[4] + pt);
  gu[4] += gEN * (s - w[1]);
  gpt -= gEN * w[1];
  gptst += gEN * sm;
  gsm += gEN * ptst;
  gbn += gEN * (vb - vbst);
  const double gvb = gEN * bn;
  gvbst -= gEN * bn;
  // vbst = sm bn + vt . bt
  gsm += gvbst * bn;
  gbn += gvbst * sm;
  gvt[0] += gvbst * z.bt[0];
  gvt[1] += gvbst * z.bt[1];
  gbt[0] += gvbst * z.vt[0];
  gbt[1] += gvbst * z.vt[1];
  // vb = w1 bn + w2 w5 + w3 w6
  gw[1] += gvb * bn;
  gbn += gvb * w[1];
  gw[2] += gvb * w[5];
  gw[5] += gvb * w[2];
  gw[3] += gvb * w[6];
  gw[6] += gvb * w[3];
  hlld_star_vjp(w, a, s, sm, bn, bn2, z, gvt, gbt, gw, ga, gs, gsm, gbn, gbn2);
  // dst = a isms, isms = 1/(s - sm)
  ga += gdst * isms;
  gisms += gdst * a;
  const double gX = -gisms * isms * isms;
  gs += gX;
  gsm -= gX;
  phys_flux_vjp(w, bn, igm1, gu, gF, gw, gbn);
}

__device__ __forceinline__ void flux_hlld_vjp(const double* wl, const double* wr, double bn, double gamma, double igm1,
                                              const double* lf, double* gwl, double* gwr, double& gbn) {
  const double bn2 = bn * bn;
  const double btl2 = wl[5] * wl[5] + wl[6] * wl[6], btr2 = wr[5] * wr[5] + wr[6] * wr[6];
  const double ilr = rcp_nr(wl[0] * wr[0]);
  const double idl = wr[0] * ilr, idr = wl[0] * ilr;
  const double cl = fast_speed_r(idl, wl[4], bn2, btl2, gamma);
  const double cr = fast_speed_r(idr, wr[4], bn2, btr2, gamma);
  const bool c_right = !(okey(cl) > okey(cr));          // imax(cl, cr) picked cr
  const bool vmin_right = !(okey(wl[1]) < okey(wr[1]));  // imin(wl1, wr1) picked wr1
  const bool vmax_right = !(okey(wl[1]) > okey(wr[1]));  // imax(wl1, wr1) picked wr1
  const double cmax = c_right ? cr : cl;
  const double sl = (vmin_right ? wr[1] : wl[1]) - cmax;
  const double sr = (vmax_right ? wr[1] : wl[1]) + cmax;
  const double ptl = wl[4] + 0.5 * (bn2 + btl2), ptr = wr[4] + 0.5 * (bn2 + btr2);
  const double al = (sl - wl[1]) * wl[0], ar = (sr - wr[1]) * wr[0];
  const double iden = rcp_nr(ar - al);
  const double NM = (mul_rn(ar, wr[1]) - mul_rn(al, wl[1])) + (ptl - ptr);
  const double sm = NM * iden;
  const double dv = wr[1] - wl[1];
  const double NP = (ar * ptl - al * ptr) + (ar * al) * dv;
  const double ptst = NP * iden;
  double gsl = 0.0, gsr = 0.0, gptl = 0.0, gptr = 0.0, gal = 0.0, gar = 0.0, gsm = 0.0, gptst = 0.0, gbn2 = 0.0;
  if (is0(sm)) {  // the forward averages both sides
    double h[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) h[n] = 0.5 * lf[n];
    hlld_side_vjp(wl, sl, ptl, al, wr, sr, ar, true, sm, bn, bn2, ptst, igm1, h, gwl, gsl, gptl, gal, gwr, gsr, gar,
                  gsm, gptst, gbn, gbn2);
    hlld_side_vjp(wr, sr, ptr, ar, wl, sl, al, false, sm, bn, bn2, ptst, igm1, h, gwr, gsr, gptr, gar, gwl, gsl, gal,
                  gsm, gptst, gbn, gbn2);
  } else if (ge0(sm)) {
    hlld_side_vjp(wl, sl, ptl, al, wr, sr, ar, true, sm, bn, bn2, ptst, igm1, lf, gwl, gsl, gptl, gal, gwr, gsr, gar,
                  gsm, gptst, gbn, gbn2);
  } else {
    hlld_side_vjp(wr, sr, ptr, ar, wl, sl, al, false, sm, bn, bn2, ptst, igm1, lf, gwr, gsr, gptr, gar, gwl, gsl, gal,
                  gsm, gptst, gbn, gbn2);
  }
  // sm = NM / D, ptst = NP / D, D = ar - al
  const double gNM = gsm * iden, gNP = gptst * iden;
  const double gD = -(gsm * NM + gptst * NP) * iden * iden;
  gar += gNM * wr[1] + gNP * (ptl + al * dv) + gD;
  gal += -gNM * wl[1] + gNP * (ar * dv - ptr) - gD;
  gwr[1] += gNM * ar + gNP * ar * al;
  gwl[1] -= gNM * al + gNP * ar * al;
  gptl += gNM + gNP * ar;
  gptr -= gNM + gNP * al;
  // al = (sl - wl1) wl0, ar = (sr - wr1) wr0
  gsl += gal * wl[0];
  gwl[1] -= gal * wl[0];
  gwl[0] += gal * (sl - wl[1]);
  gsr += gar * wr[0];
  gwr[1] -= gar * wr[0];
  gwr[0] += gar * (sr - wr[1]);
  // pt = p + (bn^2 + |bt|^2) / 2
  double gbtl2 = 0.5 * gptl, gbtr2 = 0.5 * gptr;
  gwl[4] += gptl;
  gwr[4] += gptr;
  gbn2 += 0.5 * (gptl + gptr);
  // sl = vmin - cmax, sr = vmax + cmax
  if (vmin_right) gwr[1] += gsl; else gwl[1] += gsl;
  if (vmax_right) gwr[1] += gsr; else gwl[1] += gsr;
  const double gcmax = gsr - gsl;
  double gcl = c_right ? 0.0 : gcmax, gcr = c_right ? gcmax : 0.0;
  double gidl = 0.0, gidr = 0.0;
  fast_speed_vjp(idl, wl[4], bn2, btl2, gamma, gcl, gidl, gwl[4], gbn2, gbtl2);
  fast_speed_vjp(idr, wr[4], bn2, btr2, gamma, gcr, gidr, gwr[4], gbn2, gbtr2);
  gwl[0] -= gidl * idl * idl;
  gwr[0] -= gidr * idr * idr;
  gwl[5] += 2.0 * wl[5] * gbtl2;
  gwl[6] += 2.0 * wl[6] * gbtl2;
  gwr[5] += 2.0 * wr[5] * gbtr2;
  gwr[6] += 2.0 * wr[6] * gbtr2;
  gbn += 2.0 * bn * gbn2;
}

}  // namespace vl2
