// Reverse (adjoint) of one VL2 cycle in FP64: given the adjoint of the cycle's output state, the adjoint
// of its input state, with dt held fixed.  Written kernel by kernel in reverse order of the cycle
// (Sec. 3.2.3): update -> CT corner EMFs -> fluxes (PLM / donor cell + Riemann solver) -> cons->prim ->
// ghost exchange, for the corrector and then the predictor.  The linear steps (update, CT for the frozen
// upwind choices, ghost exchange, PLM limiter away from its switch) have hand-derived transposes; with the
// smoothed CT weight the corner is also differentiated in the face mass fluxes; the Riemann solvers have
// hand-written reverse-mode derivatives (vl2_riemann_vjp.cuh) that replay the forward flux's arithmetic
// and branch decisions.
#include "vl2_internal.h"
#include "vl2_physics.cuh"
#include "vl2_riemann_vjp.cuh"

namespace vl2 {

// The adjoint is written for two ghost layers (the API refuses adjoint meshes with another ng).
constexpr int NG = 2;

static inline unsigned grid_of(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

__device__ __forceinline__ void loc_of(const Geom& g, int b, int* loc) {
  loc[0] = b % g.nb[0];
  loc[1] = (b / g.nb[0]) % g.nb[1];
  loc[2] = b / (g.nb[0] * g.nb[1]);
}

__device__ __forceinline__ int flux_comp(int v, int d) {
  if (v == 0) return 0;
  if (v == 4) return 4;
  const int m = v - 1;
  return (m == d) ? 1 : ((m == (d + 1) % 3) ? 2 : 3);
}

// ------------------------------------------------------------------------------------------------
// Output adjoint (global layout) -> block layout: every cell, and each face on the copy the forward
// gather reads (the block where it is the lower face; face N from the last block).
// ------------------------------------------------------------------------------------------------
__global__ void k_adj_scatter_out(Geom g, double* lu, double* lb0, double* lb1, double* lb2, const double* gu,
                                  const double* gb1, const double* gb2, const double* gb3) {
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex, (rem / ex) % ey, rem / (ex * ey)};
  int loc[3];
  loc_of(g, b, loc);
  int gi[3];
  for (int q = 0; q < 3; ++q) gi[q] = loc[q] * g.mb[q] + li[q];
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const bool in[3] = {li[0] < g.mb[0], li[1] < g.mb[1], li[2] < g.mb[2]};
  const bool own[3] = {in[0] || gi[0] == NX, in[1] || gi[1] == NY, in[2] || gi[2] == NZ};
  const long long o = (long long)b * g.box + cell_off(g, li[2] + NG, li[1] + NG, li[0] + NG);
  if (own[0] && in[1] && in[2]) lb0[o] = gb1[((long long)gi[2] * NY + gi[1]) * (NX + 1) + gi[0]];
  if (own[1] && in[0] && in[2]) lb1[o] = gb2[((long long)gi[2] * (NY + 1) + gi[1]) * NX + gi[0]];
  if (own[2] && in[0] && in[1]) lb2[o] = gb3[((long long)gi[2] * NY + gi[1]) * NX + gi[0]];
  if (in[0] && in[1] && in[2]) {
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)gi[2] * NY + gi[1]) * NX + gi[0];
    const long long c = (long long)b * 5 * g.box + cell_off(g, li[2] + NG, li[1] + NG, li[0] + NG);
    for (int v = 0; v < 5; ++v) lu[c + (long long)v * g.box] = gu[v * n + gc];
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of the register update U_out = U_base + h L(F), B_out = B_base - h curl E: face adjoints of
// the fluxes (all 7 components written; the induction ones start at 0), edge adjoints of the EMFs, and,
// when the base is a different register, lam_base += lam_out on the active cells and faces.
// ------------------------------------------------------------------------------------------------
__global__ void k_adj_update(Geom g, const double* lu_out, const double* lbo0, const double* lbo1, const double* lbo2,
                             double* lu_base, double* lbb0, double* lbb1, double* lbb2, double* lf0, double* lf1,
                             double* lf2, double* le0, double* le1, double* le2, double h, int add_base) {
  const int ex = g.mb[0] + 2, ey = g.mb[1] + 2, ez = g.mb[2] + 2;  // nodes NG-1 .. NG+mb
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex + NG - 1, (rem / ex) % ey + NG - 1, rem / (ex * ey) + NG - 1};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const double* LBo[3] = {lbo0, lbo1, lbo2};
  double* LBb[3] = {lbb0, lbb1, lbb2};
  double* LF[3] = {lf0, lf1, lf2};
  double* LE[3] = {le0, le1, le2};
  const long long fb = (long long)b * g.box;
  const double* LU = lu_out + (long long)b * 5 * g.box;
  // faces of sweep d at node c: flux region ng..ng+mb along d, ng-1..ng+mb across
  for (int d = 0; d < 3; ++d) {
    bool ok = li[d] >= NG;
    for (int q = 0; q < 3; ++q) ok = ok && li[q] <= NG + g.mb[q];
    if (!ok) continue;
    double* F = LF[d] + (long long)b * 7 * g.box + c;
    for (int n = 0; n < 7; ++n) F[(long long)n * g.box] = 0.0;
    for (int v = 0; v < 5; ++v) {
      const double above = LU[(long long)v * g.box + c];
      const double below = LU[(long long)v * g.box + c - stride[d]];
      F[(long long)flux_comp(v, d) * g.box] = h * g.idx[d] * (above - below);
    }
  }
  // edges of family e at node c: ng..ng+mb-1 along e, ng..ng+mb across
  for (int e = 0; e < 3; ++e) {
    bool ok = li[e] >= NG && li[e] <= NG + g.mb[e] - 1;
    for (int q = 0; q < 3; ++q)
      if (q != e) ok = ok && li[q] >= NG && li[q] <= NG + g.mb[q];
    if (!ok) continue;
    const int f1 = (e + 1) % 3, f2 = (e + 2) % 3;
    // B_f1 uses E_e as its "bq" edge (curl_f1 = (E_e(+a) - E_e) idx_a - ..., a = f1+1 = e+2)
    const int a1 = (f1 + 1) % 3;
    // B_f2 uses E_e as its "a" edge (curl_f2 = ... - (E_e(+bq) - E_e) idx_bq, bq = f2+2 = e+1)
    const int bq2 = (f2 + 2) % 3;
    const double* B1 = LBo[f1] + fb;
    const double* B2 = LBo[f2] + fb;
    const double v = -h * g.idx[a1] * B1[c - stride[a1]] + h * g.idx[a1] * B1[c] + h * g.idx[bq2] * B2[c - stride[bq2]] -
                     h * g.idx[bq2] * B2[c];
    LE[e][fb + c] = v;
  }
  if (add_base) {
    bool cell = true;
    for (int q = 0; q < 3; ++q) cell = cell && li[q] >= NG && li[q] <= NG + g.mb[q] - 1;
    if (cell) {
      double* UB = lu_base + (long long)b * 5 * g.box + c;
      for (int v = 0; v < 5; ++v) UB[(long long)v * g.box] += LU[(long long)v * g.box + c];
    }
    for (int fd = 0; fd < 3; ++fd) {
      bool face = li[fd] >= NG && li[fd] <= NG + g.mb[fd];
      for (int q = 0; q < 3; ++q)
        if (q != fd) face = face && li[q] >= NG && li[q] <= NG + g.mb[q] - 1;
      if (face) LBb[fd][fb + c] += LBo[fd][fb + c];
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of the upwind-CT corner EMFs (linear in the face and cell EMFs for the upwind choices the
// forward step made from the signs of the face mass fluxes).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void pick_w(double m, double& w0, double& w1) {
  if (gt0(m)) {
    w0 = 1.0;
    w1 = 0.0;
  } else if (lt0(m)) {
    w0 = 0.0;
    w1 = 1.0;
  } else {
    w0 = w1 = 0.5;
  }
}

// Smoothed upwind weight of the forward corner, evaluated by the forward step's own ct_weight (so the adjoint
// linearises about the very weight the forward cycle used), and its derivative in the mass flux:
// w = 1 / (1 + exp(-2 m / delta)) gives dw/dm = 2 w (1 - w) / delta, which is 0 where the weight is flat at
// 0 or 1 (|m| > 20 delta).
__device__ __forceinline__ void smooth_w(double m, double delta, double& w, double& dw) {
  w = ct_weight<double>(m, delta, 20.0 * delta);
  dw = 2.0 * w * (1.0 - w) / delta;
}

__device__ __forceinline__ void pick_w(double m, double delta, double& w0, double& w1) {
  if (delta > 0.0) {
    double dw;
    smooth_w(m, delta, w0, dw);
    w1 = 1.0 - w0;
  } else {
    pick_w(m, w0, w1);
  }
}

// Upwind weights and adjoint coefficients of one corner EMF (family e, node c): the corner EMF is
//   E = cea0 ea(b-1) + cea1 ea(b) + ceb0 eb(a-1) + ceb1 eb(a) + cec0 ec(a-1,b-1) + cec1 ec(a,b-1)
//     + cec2 ec(a-1,b) + cec3 ec(a,b)
// with ea = -F_a[B_t1] and eb = +F_b[B_t2] (the face EMFs) and ec = -v x b (cell EMFs).
struct EdgeCoef {
  double cea0, cea1, ceb0, ceb1, cec0, cec1, cec2, cec3;
};
__device__ __forceinline__ EdgeCoef edge_coef(const double* Ma, const double* Mb, long long c, long long sa,
                                              long long sb, double delta) {
  double w0, w1, u0, u1, s0, s1, r0, r1;
  pick_w(Ma[c - sb], delta, w0, w1);  // tlo: gradient along b below the corner, by the a-face mass flux at b-1
  pick_w(Ma[c], delta, u0, u1);       // thi
  pick_w(Mb[c - sa], delta, s0, s1);  // slo: gradient along a, by the b-face mass flux at a-1
  pick_w(Mb[c], delta, r0, r1);       // shi
  EdgeCoef k;
  k.cea0 = 0.25 * (1.0 + s0 + r0);
  k.cea1 = 0.25 * (1.0 + s1 + r1);
  k.ceb0 = 0.25 * (1.0 + w0 + u0);
  k.ceb1 = 0.25 * (1.0 + w1 + u1);
  k.cec0 = -0.25 * (w0 + s0);
  k.cec1 = -0.25 * (w1 + r0);
  k.cec2 = -0.25 * (u0 + s1);
  k.cec3 = -0.25 * (u1 + r1);
  return k;
}

// corner EMFs of family e exist at nodes NG..NG+mb-1 along e and NG..NG+mb across
__device__ __forceinline__ bool edge_valid(const Geom& g, int e, const int* n) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 3; ++q) ok = ok && n[q] >= NG && n[q] <= NG + g.mb[q] - (q == e ? 1 : 0);
  return ok;
}

// Of the corner EMF of family e at node n + da s_a + db s_b, lam_E times dE/dw of one of its weights (slot 0:
// tlo by ma[0], 1: thi by ma[1], 2: slo by mb[0], 3: shi by mb[1]); each correction enters E as
// +-(1/4)(w lo + (1 - w) hi), so dE/dw = +-(1/4)(lo - hi).  Zero outside the corners that exist.
__device__ __forceinline__ double corner_dm(const Geom& g, const double* W, const double* const* M, long long e5off,
                                           long long e6off, const double* const* LE, const long long* stride,
                                           const int* li, int b, long long c, int e, int da, int db, int slot) {
  const int a = (e + 1) % 3, bq = (e + 2) % 3;
  int n[3] = {li[0], li[1], li[2]};
  n[a] += da;
  n[bq] += db;
  if (!edge_valid(g, e, n)) return 0.0;
  const long long sa = stride[a], sb = stride[bq];
  const long long cn = c + da * sa + db * sb;
  const double lam = LE[e][cn];
  if (lam == 0.0) return 0.0;
  const double* Wb = W + (long long)b * 8 * g.box;
  auto cell_emf = [&](long long q) {  // -(v x b_c) component e of cell q
    const double vx = Wb[g.box + q], vy = Wb[2 * g.box + q], vz = Wb[3 * g.box + q];
    const double ux = Wb[5 * g.box + q], uy = Wb[6 * g.box + q], uz = Wb[7 * g.box + q];
    return e == 0 ? vz * uy - vy * uz : (e == 1 ? vx * uz - vz * ux : vy * ux - vx * uy);
  };
  const double* Fa5 = M[a] + e5off;
  const double* Fb6 = M[bq] + e6off;
  double d;
  switch (slot) {
    case 0: d = (Fb6[cn - sa] - cell_emf(cn - sa - sb)) - (Fb6[cn] - cell_emf(cn - sb)); break;
    case 1: d = -((cell_emf(cn - sa) - Fb6[cn - sa]) - (cell_emf(cn) - Fb6[cn])); break;
    case 2: d = (-Fa5[cn - sb] - cell_emf(cn - sa - sb)) - (-Fa5[cn] - cell_emf(cn - sa)); break;
    default: d = -((cell_emf(cn - sb) + Fa5[cn - sb]) - (cell_emf(cn) + Fa5[cn])); break;
  }
  return 0.25 * lam * d;
}

// Transpose of the upwind CT (linear for the upwind choices the forward step made), as a gather: the
// thread of node n collects, in a fixed order, what the corner EMFs around it give to (i) the face-EMF
// components of the fluxes at n (F_d[B_t1] from family d+2 at n and n + s_(d+1); F_d[B_t2] from family
// d+1 at n and n + s_(d+2)) and (ii) the primitives of cell n through its three cell EMFs (each from the
// four edges of its family around the cell).  With the smoothed weight (delta > 0) the corners are also
// functions of the face mass fluxes: (iii) the mass-flux component of the fluxes at n collects
// dE/dm = +-(1/4) dw/dm (lo - hi) of the four corners that weigh by it, from the forward face EMFs (at
// e5off / e6off after each block's mass fluxes) and the cell EMFs -v x b of W.
template <bool SMOOTH>
__global__ void k_adj_ct(Geom g, const double* W, const double* m0, const double* m1, const double* m2, long long mstride,
                         long long e5off, long long e6off, double delta_in, const double* le0, const double* le1,
                         const double* le2, double* lf0, double* lf1, double* lf2, double* lw) {
  const double delta = SMOOTH ? delta_in : 0.0;
  const int ex = g.mb[0] + 2, ey = g.mb[1] + 2, ez = g.mb[2] + 2;  // nodes NG-1 .. NG+mb
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex + NG - 1, (rem / ex) % ey + NG - 1, rem / (ex * ey) + NG - 1};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const double* M[3] = {m0 + (long long)b * mstride, m1 + (long long)b * mstride, m2 + (long long)b * mstride};
  const double* LE[3] = {le0 + (long long)b * g.box, le1 + (long long)b * g.box, le2 + (long long)b * g.box};
  double* LF[3] = {lf0 + (long long)b * 7 * g.box, lf1 + (long long)b * 7 * g.box, lf2 + (long long)b * 7 * g.box};
  // edge family e at node c + s_p + s_q (p, q in {a, b} offsets given as 0/1): value lam * coefficient
  auto edge_term = [&](int e, int da, int db, int which) -> double {
    const int a = (e + 1) % 3, bq = (e + 2) % 3;
    int n[3] = {li[0], li[1], li[2]};
    n[a] += da;
    n[bq] += db;
    if (!edge_valid(g, e, n)) return 0.0;
    const long long cn = c + da * stride[a] + db * stride[bq];
    const double lam = LE[e][cn];
    if (lam == 0.0) return 0.0;
    const EdgeCoef k = edge_coef(M[a], M[bq], cn, stride[a], stride[bq], delta);
    switch (which) {
      case 0: return k.cea0 * lam;
      case 1: return k.cea1 * lam;
      case 2: return k.ceb0 * lam;
      case 3: return k.ceb1 * lam;
      case 4: return k.cec0 * lam;
      case 5: return k.cec1 * lam;
      case 6: return k.cec2 * lam;
      default: return k.cec3 * lam;
    }
  };
  // (i) face EMF components of the fluxes at node c, for faces in the flux region of each sweep
  for (int d = 0; d < 3; ++d) {
    bool face = li[d] >= NG;
    for (int q = 0; q < 3; ++q) face = face && li[q] <= NG + g.mb[q];
    if (!face) continue;
    const int e5 = (d + 2) % 3;  // family whose a-faces are d-faces: ea = -F_d[B_t1]
    const int e6 = (d + 1) % 3;  // family whose b-faces are d-faces: eb = +F_d[B_t2]
    const double g5 = -(edge_term(e5, 0, 0, 1) + edge_term(e5, 0, 1, 0));
    const double g6 = edge_term(e6, 0, 0, 3) + edge_term(e6, 1, 0, 2);
    LF[d][5 * g.box + c] += g5;
    LF[d][6 * g.box + c] += g6;
    if constexpr (SMOOTH) {
      double w, dw;
      smooth_w(M[d][c], delta, w, dw);
      if (dw != 0.0) {
        // slots of this face: ma[1] (thi) and ma[0] (tlo) of family e5 at n and n + s_(d+1); mb[1] (shi) and
        // mb[0] (slo) of family e6 at n and n + s_(d+2)
        const double gm = corner_dm(g, W, M, e5off, e6off, LE, stride, li, b, c, e5, 0, 0, 1) +
                          corner_dm(g, W, M, e5off, e6off, LE, stride, li, b, c, e5, 0, 1, 0) +
                          corner_dm(g, W, M, e5off, e6off, LE, stride, li, b, c, e6, 0, 0, 3) +
                          corner_dm(g, W, M, e5off, e6off, LE, stride, li, b, c, e6, 1, 0, 2);
        LF[d][c] += dw * gm;
      }
    }
  }
  // (ii) primitives of cell c through its cell EMFs (E = -v x b)
  const double* Wc = W + (long long)b * 8 * g.box + c;
  double* LW = lw + (long long)b * 8 * g.box + c;
  const long long box = g.box;
  double lam[3];
  for (int e = 0; e < 3; ++e)
    lam[e] = edge_term(e, 0, 0, 7) + edge_term(e, 1, 0, 6) + edge_term(e, 0, 1, 5) + edge_term(e, 1, 1, 4);
  if (lam[0] == 0.0 && lam[1] == 0.0 && lam[2] == 0.0) return;
  const double vx = Wc[box], vy = Wc[2 * box], vz = Wc[3 * box];
  const double bx = Wc[5 * box], by = Wc[6 * box], bz = Wc[7 * box];
  // E_x = vz by - vy bz, E_y = vx bz - vz bx, E_z = vy bx - vx by
  LW[1 * box] += lam[1] * bz - lam[2] * by;
  LW[2 * box] += lam[2] * bx - lam[0] * bz;
  LW[3 * box] += lam[0] * by - lam[1] * bx;
  LW[5 * box] += lam[2] * vy - lam[1] * vz;
  LW[6 * box] += lam[0] * vz - lam[2] * vx;
  LW[7 * box] += lam[1] * vx - lam[0] * vy;
}

// ------------------------------------------------------------------------------------------------
// Transpose of the face fluxes: lam_F . dF/d(w_L, w_R, b_n) by reverse mode (one value pass and one
// reverse pass per face), then through the reconstruction to the cells (PLM: van Leer slope derivatives;
// its switch at dl*dr = 0 is frozen).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void vl_slope_grad(double qm, double q0, double qp, double& dqm, double& dq0, double& dqp) {
  const double dl = q0 - qm, dr = qp - q0;
  if (gt0(dl * dr)) {
    const double s = dl + dr;
    const double s2 = s * s;  // > 0 here (dl and dr have the same sign)
    const double is2 = s2 >= 2.2250738585072014e-308 ? rcp_nr(s2) : 1.0 / s2;  // rcp_nr takes normal numbers
    const double gdl = 2.0 * dr * dr * is2;  // d delta / d dl
    const double gdr = 2.0 * dl * dl * is2;  // d delta / d dr
    dqm = -gdl;
    dq0 = gdl - gdr;
    dqp = gdr;
  } else {
    dqm = dq0 = dqp = 0.0;
  }
}

template <int DIR, int REC, int RS>
__global__ void __launch_bounds__(128) k_adj_flux(Geom g, const double* __restrict__ W, const double* __restrict__ Bn,
                                                  double* LF, double* LR, double* lbn) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  const int h = g.flux_halo;  // the faces of the forward flux kernels (transverse halo only with flux_halo)
  const int rx = g.mb[0] + (DIR == 0 ? 1 : 2 * h);
  const int ry = g.mb[1] + (DIR == 1 ? 1 : 2 * h);
  const int rz = g.mb[2] + (DIR == 2 ? 1 : 2 * h);
  const long long per = (long long)rx * ry * rz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % rx + (DIR == 0 ? NG : NG - h);
  rem /= rx;
  const int j = rem % ry + (DIR == 1 ? NG : NG - h);
  const int k = rem / ry + (DIR == 2 ? NG : NG - h);
  const long long c = cell_off(g, k, j, i);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  double* Fl = LF + (long long)b * 7 * g.box + c;
  double* Fr = LR + (long long)b * 7 * g.box + c;
  double lf[7];
  bool any = false;
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    lf[n] = Fl[(long long)n * g.box];
    any = any || lf[n] != 0.0;
  }
  if (!any) {  // this face passes nothing to its states
#pragma unroll
    for (int n = 0; n < 7; ++n) Fr[(long long)n * g.box] = 0.0;
    return;
  }
  const double* Wb = W + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  double wl[7], wr[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const double* p = Wb + (long long)var[n] * g.box + c;
    if (REC == REC_DC) {
      wl[n] = p[-sd];
      wr[n] = p[0];
    } else {  // the forward sweep's face values: the upper face of cell i-1, the lower face of cell i
      double unused;
      plm_var_faces<double>(p[-2 * sd], p[-sd], p[0], unused, wl[n]);
      plm_var_faces<double>(p[-sd], p[0], p[sd], wr[n], unused);
    }
  }
  const double bn = Bn[(long long)b * g.box + c];
  // adjoints of the 15 Riemann inputs: lam_x[k] = sum_n lf[n] dF_n/dx_k, by reverse mode
  double lx[15];
#pragma unroll
  for (int q = 0; q < 15; ++q) lx[q] = 0.0;
  if (RS == RS_HLLD)
    flux_hlld_vjp(wl, wr, bn, g.gamma, g.igm1, lf, lx, lx + 7, lx[14]);
  else
    flux_hlle_vjp(wl, wr, bn, g.gamma, g.igm1, lf, lx, lx + 7, lx[14]);
  lbn[(long long)b * g.box + c] += lx[14];
  // the face's left- and right-state adjoints, for the cells to collect (in place of the flux adjoint)
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    Fl[(long long)n * g.box] = lx[n];
    Fr[(long long)n * g.box] = lx[7 + n];
  }
}

// Transpose of the forward halo copy (k_flux_halo, meshes with flux_halo = 0): the faces just outside a
// block's transverse range are copies of its neighbours' faces, so the adjoints the CT transpose left on
// those copies (mass flux and the two transverse induction fluxes) belong to the owners.  As a gather: each
// owned d-face on a boundary row of a transverse direction t adds, in a fixed order (t = d+1 then d+2; the
// copy in the block below, then the one above), the adjoint of its copy in the neighbouring block along t.
// One thread per owned face; threads off every boundary row return at once.
__global__ void __launch_bounds__(256) k_adj_flux_halo(Geom g, double* lf0, double* lf1, double* lf2) {
  if (g.flux_halo) return;
  long long per[3], tot = 0;
  for (int d = 0; d < 3; ++d) {
    per[d] = (long long)(g.mb[0] + (d == 0)) * (g.mb[1] + (d == 1)) * (g.mb[2] + (d == 2));
    tot += per[d];
  }
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot * g.nblk) return;
  const int b = (int)(t / tot);
  long long r = t - (long long)b * tot;
  int d = 0;
  while (r >= per[d]) r -= per[d++];
  const int ex = g.mb[0] + (d == 0), ey = g.mb[1] + (d == 1);
  int li[3] = {(int)(r % ex) + NG, (int)((r / ex) % ey) + NG, (int)(r / ((long long)ex * ey)) + NG};
  double* LF = d == 0 ? lf0 : (d == 1 ? lf1 : lf2);
  const int loc[3] = {b % g.nb[0], (b / g.nb[0]) % g.nb[1], b / (g.nb[0] * g.nb[1])};
  const long long own = (long long)b * 7 * g.box + cell_off(g, li[2], li[1], li[0]);
  double acc[3] = {0.0, 0.0, 0.0};
  bool any = false;
  for (int k = 1; k <= 2; ++k) {
    const int tq = (d + k) % 3;
    for (int side = 0; side < 2; ++side) {
      // side 0: our lower row is copied into the upper halo of the block below; side 1: our upper row into
      // the lower halo of the block above
      if (li[tq] != (side ? NG + g.mb[tq] - 1 : NG)) continue;
      int nl[3] = {loc[0], loc[1], loc[2]};
      nl[tq] = (nl[tq] + (side ? 1 : g.nb[tq] - 1)) % g.nb[tq];
      const int bs = (nl[2] * g.nb[1] + nl[1]) * g.nb[0] + nl[0];
      int hi_[3] = {li[0], li[1], li[2]};
      hi_[tq] = side ? NG - 1 : NG + g.mb[tq];
      const long long o = (long long)bs * 7 * g.box + cell_off(g, hi_[2], hi_[1], hi_[0]);
      acc[0] += LF[o];
      acc[1] += LF[o + 5 * g.box];
      acc[2] += LF[o + 6 * g.box];
      any = true;
    }
  }
  if (!any) return;
  LF[own] += acc[0];
  LF[own + 5 * g.box] += acc[1];
  LF[own + 6 * g.box] += acc[2];
}

// The van Leer slopes' share of the face-state adjoints of one PLM sweep, formed once per slope: for the slope
// delta_j of cell j (on q_{j-1}, q_j, q_{j+1}), lam delta_j = a(j+1)/2 - r(j)/2 times its three partial
// derivatives, stored as the contributions PM (to q_{j-1}), P0 (to q_j) and PP (to q_{j+1}) that
// k_adj_flux_cells then gathers.  Only the slopes of cells next to a face of the flux region are formed.
template <int DIR>
__global__ void __launch_bounds__(128) k_adj_slopes(Geom g, const double* __restrict__ W,
                                                    const double* __restrict__ LA, const double* __restrict__ LR,
                                                    double* PM, double* P0, double* PP) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  // cells NG-1 .. NG+mb along the sweep; transversally the rows of the flux kernels' faces
  const int h = g.flux_halo;
  const int nx = g.mb[0] + (DIR == 0 ? 2 : 2 * h), ny = g.mb[1] + (DIR == 1 ? 2 : 2 * h),
            nz = g.mb[2] + (DIR == 2 ? 2 : 2 * h);
  const long long per = (long long)nx * ny * nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % nx + (DIR == 0 ? NG - 1 : NG - h), (rem / nx) % ny + (DIR == 1 ? NG - 1 : NG - h),
                     rem / (nx * ny) + (DIR == 2 ? NG - 1 : NG - h)};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  const int id = li[DIR];
  auto face_ok = [&](int f) { return f >= NG && f <= NG + g.mb[DIR]; };
  const bool lo = face_ok(id), hi = face_ok(id + 1);
  const long long fb = (long long)b * 7 * g.box + c;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  const double* Wb = W + (long long)b * 8 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const long long o = fb + (long long)n * g.box;
    double pm = 0.0, p0 = 0.0, pp = 0.0;
    if (lo || hi) {
      const double a1 = hi ? LA[o + sd] : 0.0;  // a(j+1)
      const double r0 = lo ? LR[o] : 0.0;       // r(j)
      const double ld = 0.5 * a1 - 0.5 * r0;
      const double* q = Wb + (long long)var[n] * g.box;
      double dm, d0, dp;
      vl_slope_grad(q[-sd], q[0], q[sd], dm, d0, dp);
      pm = ld * dm;
      p0 = ld * d0;
      pp = ld * dp;
    }
    PM[o] = pm;
    P0[o] = p0;
    PP[o] = pp;
  }
}

// The cells' share of the face-state adjoints of one sweep, gathered per cell in a fixed order.  With
// a(f), r(f) the adjoints of the left and right states of face f (between cells f-1 and f):
//   donor cell:  lam q_i += a(i+1) + r(i)
//   PLM:         w_L(f) = q_{f-1} + delta_{f-1}/2, w_R(f) = q_f - delta_f/2, so
//                lam delta_j = a(j+1)/2 - r(j)/2 and
//                lam q_i += a(i+1) + r(i) + sum_{j=i-1..i+1} lam delta_j d delta_j / d q_i.
// Faces outside the sweep's flux region contribute nothing.
template <int DIR, int REC>
__global__ void __launch_bounds__(128) k_adj_flux_cells(Geom g, const double* __restrict__ W,
                                                        const double* __restrict__ LA, const double* __restrict__ LR,
                                                        const double* __restrict__ PM, const double* __restrict__ P0,
                                                        const double* __restrict__ PP, double* lw) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int H = (REC == REC_DC) ? 1 : 2;  // cells NG-H .. NG+mb-1+H along the sweep
  const int h = g.flux_halo;                  // transversally the rows of the flux kernels' faces
  const int nx = g.mb[0] + (DIR == 0 ? 2 * H : 2 * h), ny = g.mb[1] + (DIR == 1 ? 2 * H : 2 * h),
            nz = g.mb[2] + (DIR == 2 ? 2 * H : 2 * h);
  const long long per = (long long)nx * ny * nz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % nx + (DIR == 0 ? NG - H : NG - h), (rem / nx) % ny + (DIR == 1 ? NG - H : NG - h),
                     rem / (nx * ny) + (DIR == 2 ? NG - H : NG - h)};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  const int id = li[DIR];
  auto face_ok = [&](int f) { return f >= NG && f <= NG + g.mb[DIR]; };
  const long long fb = (long long)b * 7 * g.box + c;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  double* LWb = lw + (long long)b * 8 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const long long o = fb + (long long)n * g.box;
    const double a1 = face_ok(id + 1) ? LA[o + sd] : 0.0;  // a(i+1)
    const double r0 = face_ok(id) ? LR[o] : 0.0;           // r(i)
    double lam = a1 + r0;
    if (REC == REC_PLM) {
      // the slopes of cells i-1, i, i+1 (each formed once, by k_adj_slopes), where next to the flux region
      if (face_ok(id) || face_ok(id - 1)) lam += PP[o - sd];   // slope of cell i-1: d/dq_i
      if (face_ok(id + 1) || face_ok(id)) lam += P0[o];        // slope of cell i
      if (face_ok(id + 2) || face_ok(id + 1)) lam += PM[o + sd];  // slope of cell i+1
    }
    LWb[(long long)var[n] * g.box] += lam;
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of cons->prim on every cell (no floor active): lam_U from lam_W, and the cell-centred field's
// adjoint split half and half onto the two faces of each direction, gathered per face (lower cell first).
// One thread per node 0 .. mb+2 NG of the box: the cell at the node (if any) and the three faces there.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double prim_field_adj(const Geom& g, const double* Wc, const double* Lc, int d) {
  // d p / d b_c,d = -(gamma-1) b_c,d, and lam_W carries the cell-centred field directly
  return Lc[(5 + d) * g.box] - g.gm1 * Lc[4 * g.box] * Wc[(5 + d) * g.box];
}

__global__ void k_adj_prim(Geom g, const double* W, const double* lw, double* lu, double* lb0, double* lb1, double* lb2) {
  const int ex = g.mb[0] + 2 * NG + 1, ey = g.mb[1] + 2 * NG + 1, ez = g.mb[2] + 2 * NG + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex, (rem / ex) % ey, rem / (ex * ey)};
  const int cmax[3] = {g.mb[0] + 2 * NG, g.mb[1] + 2 * NG, g.mb[2] + 2 * NG};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const double* Wb = W + (long long)b * 8 * g.box;
  const double* Lb = lw + (long long)b * 8 * g.box;
  const bool cell = li[0] < cmax[0] && li[1] < cmax[1] && li[2] < cmax[2];
  if (cell) {
    const double* Wc = Wb + c;
    const double* Lc = Lb + c;
    const double lrho = Lc[0], lvx = Lc[g.box], lvy = Lc[2 * g.box], lvz = Lc[3 * g.box], lp = Lc[4 * g.box];
    const double d = Wc[0], vx = Wc[g.box], vy = Wc[2 * g.box], vz = Wc[3 * g.box];
    const double id = 1.0 / d;
    const double gp = g.gm1 * lp;
    double* U = lu + (long long)b * 5 * g.box + c;
    U[0] += lrho - (lvx * vx + lvy * vy + lvz * vz) * id + gp * 0.5 * (vx * vx + vy * vy + vz * vz);
    U[g.box] += lvx * id - gp * vx;
    U[2 * g.box] += lvy * id - gp * vy;
    U[3 * g.box] += lvz * id - gp * vz;
    U[4 * g.box] += gp;
  }
  double* LB[3] = {lb0, lb1, lb2};
  for (int d = 0; d < 3; ++d) {
    bool face = li[d] <= cmax[d];
    for (int q = 0; q < 3; ++q)
      if (q != d) face = face && li[q] < cmax[q];
    if (!face) continue;
    double x = 0.0;
    if (li[d] >= 1) x += 0.5 * prim_field_adj(g, Wb + c - stride[d], Lb + c - stride[d], d);  // cell below
    if (li[d] < cmax[d]) x += 0.5 * prim_field_adj(g, Wb + c, Lb + c, d);                    // cell above
    LB[d][(long long)b * g.box + c] += x;
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of the ghost exchange.  The exchange copies into each ghost element the element whose index
// is given, direction by direction, by source_of (periodic wrap or outflow clamp).  For cells the copy map
// is a product of one-dimensional maps, one per direction, and its transpose is applied one direction at a
// time.  For the faces of direction fd the map along fd depends on the other two directions: a face on a
// block's upper surface (index NG+mb along fd, below global face N) is kept when the element is active in
// the other directions, but is copied from the next block's lower face when it is a ghost in one of them.
// The map is then the product (map along fd, with that rule) x (the other two, plain), the former applied
// last, so its transpose along fd comes first.  Pass p treats direction p for cells and direction fd + p
// for faces of direction fd: every element that is active along that direction (for the rule above)
// collects, in a fixed order, the adjoints of the elements that copy from it (same indices in the other
// directions), then those elements are cleared.  After the three passes every ghost adjoint sits in the
// active element it came from.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void source_of_adj(const Geom& g, int q, int gi, bool face, int& blk, int& loc) {
  const int N = g.N[q];
  int m = gi;
  const bool inside = (m >= 0 && m < N) || (face && m == N);
  if (!inside) {
    if (m < 0) {
      if (g.bc[2 * q] == BC_PERIODIC) {
        m %= N;
        if (m < 0) m += N;
      } else {
        m = 0;
      }
    } else {
      if (g.bc[2 * q + 1] == BC_PERIODIC)
        m %= N;
      else
        m = face ? N : N - 1;
    }
  }
  if (face && m == N) {
    blk = g.nb[q] - 1;
    loc = g.mb[q] + NG;
  } else {
    blk = m / g.mb[q];
    loc = m - blk * g.mb[q] + NG;
  }
}

// Element kinds: 0 = cell (5 conserved variables), 1 + fd = face of direction fd.
__device__ __forceinline__ int hi_index(const Geom& g, int kind, int q) {  // largest index along q
  return g.mb[q] + 2 * NG - ((kind == 1 + q) ? 0 : 1);
}
__device__ __forceinline__ int hi_active(const Geom& g, int kind, int q) {  // largest active index along q
  return NG + g.mb[q] - ((kind == 1 + q) ? 0 : 1);
}

// Is the element (kind, li) a ghost in a direction other than q?
__device__ __forceinline__ bool ghost_elsewhere(const Geom& g, int kind, const int* li, int q) {
  bool gh = false;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    if (r != q) gh = gh || li[r] < NG || li[r] > hi_active(g, kind, r);
  return gh;
}
// Is the element copied along q (a ghost along q, or an upper-surface face that the rule above moves)?
__device__ __forceinline__ bool moved_along(const Geom& g, int kind, const int* li, int q, int locq) {
  if (li[q] < NG || li[q] > hi_active(g, kind, q)) return true;
  return kind == 1 + q && li[q] == NG + g.mb[q] && locq < g.nb[q] - 1 && ghost_elsewhere(g, kind, li, q);
}

// Pass direction of element kind `kind` in pass PASS: cells and x-faces take PASS, y-faces PASS+1, z-faces
// PASS+2 (mod 3).
template <int PASS>
__device__ __forceinline__ int pass_dir(int kind) {
  return kind == 0 ? PASS : (kind - 1 + PASS) % 3;
}

// Compact thread spaces of one pass.  For each kind the pass touches only a few indices along its pass
// direction q (the gather: the NG+2 active indices nearest each end, the only ones a ghost copies from; the
// clear: the ghost indices and the upper surface), each over the full extents of the other two directions.
// A flat index within one block is split as kind, then slot s (the index along q), then the two other
// directions, the lower one fastest.  `slots` is the number of slots per kind.
struct PassElem {
  int kind, q, li[3];
};
template <int PASS>
__device__ __forceinline__ bool pass_elem(const Geom& g, long long r, int slots, PassElem& e) {
  const int ext[3] = {g.mb[0] + 2 * NG + 1, g.mb[1] + 2 * NG + 1, g.mb[2] + 2 * NG + 1};
  for (int kind = 0; kind < 4; ++kind) {
    const int q = pass_dir<PASS>(kind), r1 = q == 0 ? 1 : 0, r2 = q == 2 ? 1 : 2;
    const long long n = (long long)slots * ext[r1] * ext[r2];
    if (r >= n) {
      r -= n;
      continue;
    }
    e.kind = kind;
    e.q = q;
    e.li[r1] = (int)(r % ext[r1]);
    e.li[r2] = (int)((r / ext[r1]) % ext[r2]);
    e.li[q] = (int)(r / ((long long)ext[r1] * ext[r2]));  // the slot, mapped to an index by the caller
    return true;
  }
  return false;
}
// Threads per block of one pass: each direction's slots times its other two extents, for the four kinds
// (cells and x-faces both take direction `pass`).
inline long long pass_elems(const Geom& g, int slots, int pass) {
  const long long e0 = g.mb[0] + 2 * NG + 1, e1 = g.mb[1] + 2 * NG + 1, e2 = g.mb[2] + 2 * NG + 1;
  const long long a[3] = {e1 * e2, e0 * e2, e0 * e1};
  return (long long)slots * (a[0] + a[1] + a[2] + a[pass]);
}

// Gather of pass PASS: each target element (an active index along its pass direction q within NG + 1 of a
// block end: a neighbour's ghost layer, a periodic wrap or an outflow clamp reaches no further, and small
// blocks are near an end everywhere) collects, in a fixed order, the adjoints of the elements that copy from
// it.  PASS is a template parameter, so every direction index below is a compile-time constant and the small
// index arrays stay in registers.
template <int PASS>
__global__ void __launch_bounds__(256) k_adj_ghost_gather(Geom g, long long per, double* lu, double* lb0, double* lb1,
                                                          double* lb2) {
  constexpr int S = NG + 2;  // targets nearest each end
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  PassElem e;
  if (!pass_elem<PASS>(g, t - (long long)b * per, 2 * S, e)) return;
  const int kind = e.kind, q = e.q;
  int li[3] = {e.li[0], e.li[1], e.li[2]};
  const int ha = hi_active(g, kind, q);
  const int slot = li[q];
  if (slot < S) {
    li[q] = NG + slot;
    if (li[q] > ha) return;
  } else {
    li[q] = ha - (slot - S);
    if (li[q] < NG + S) return;  // already a lower target (short blocks)
  }
#pragma unroll
  for (int r = 0; r < 3; ++r)
    if (li[r] > hi_index(g, kind, r)) return;
  int loc[3];
  loc_of(g, b, loc);
  if (moved_along(g, kind, li, q, loc[q])) return;  // targets only
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const long long bstride[3] = {1LL, (long long)g.nb[0], (long long)g.nb[0] * g.nb[1]};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const bool face = (kind == 1 + q);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  bool got = false;
  auto take = [&](long long blk2, long long c2) {
    if (kind == 0) {
      const double* U2 = lu + blk2 * 5 * g.box + c2;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += U2[(long long)v * g.box];
    } else {
      acc[0] += (kind == 1 ? lb0 : (kind == 2 ? lb1 : lb2))[blk2 * g.box + c2];
    }
    got = true;
  };
  // an upper-surface face of the block below that is moved onto this lower face
  if (face && li[q] == NG && loc[q] >= 1 && ghost_elsewhere(g, kind, li, q))
    take((long long)b - bstride[q], c + (long long)g.mb[q] * stride[q]);
  // ghosts along q in this block and the blocks within reach along q (distinct, existing) that copy from
  // here: a ghost of block bq has global index up to bq mb + mb + NG, at most R = 1 + (NG + mb) / mb
  // blocks away (R <= 4 for mb >= 1)
  const int R = 1 + (NG + g.mb[q]) / g.mb[q];
  auto block_at = [&](int dl) -> int {  // block along q at offset dl (wrapped), or -1 beyond an outflow edge
    int bq = loc[q] + dl;
    if (bq < 0 || bq >= g.nb[q]) {
      if (g.bc[dl < 0 ? 2 * q : 2 * q + 1] != BC_PERIODIC) return -1;
      bq = ((bq % g.nb[q]) + g.nb[q]) % g.nb[q];
    }
    return bq;
  };
  for (int dl = -R; dl <= R; ++dl) {
    const int bq = block_at(dl);
    if (bq < 0) continue;
    bool dup = false;  // an earlier offset that wraps onto the same block
    for (int d2 = -R; d2 < dl; ++d2) dup = dup || block_at(d2) == bq;
    if (dup) continue;
    const int hi = hi_index(g, kind, q);
    // the ghosts along q only: indices 0 .. NG-1, then ha+1 .. hi (in that order)
    for (int gl = 0; gl <= hi; gl = (gl == NG - 1) ? ha + 1 : gl + 1) {
      int sblk, sloc;
      source_of_adj(g, q, bq * g.mb[q] + gl - NG, face, sblk, sloc);
      if (sblk != loc[q] || sloc != li[q]) continue;
      take((long long)b + (long long)(bq - loc[q]) * bstride[q], c + (long long)(gl - li[q]) * stride[q]);
    }
  }
  if (!got) return;
  if (kind == 0) {
    double* U = lu + (long long)b * 5 * g.box + c;
#pragma unroll
    for (int v = 0; v < 5; ++v) U[(long long)v * g.box] += acc[v];
  } else {
    (kind == 1 ? lb0 : (kind == 2 ? lb1 : lb2))[(long long)b * g.box + c] += acc[0];
  }
}

// Clear of pass PASS: the elements moved along their pass direction (its ghost indices 0 .. NG-1 and
// ha+1 .. hi, and the upper-surface faces the rule above moves, index ha) drop the adjoints just gathered.
template <int PASS>
__global__ void __launch_bounds__(256) k_adj_ghost_clear(Geom g, long long per, double* lu, double* lb0, double* lb1,
                                                         double* lb2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  PassElem e;
  if (!pass_elem<PASS>(g, t - (long long)b * per, 2 * NG + 1, e)) return;
  const int kind = e.kind, q = e.q;
  int li[3] = {e.li[0], e.li[1], e.li[2]};
  const int ha = hi_active(g, kind, q), hi = hi_index(g, kind, q);
  const int slot = li[q];
  li[q] = slot < NG ? slot : ha + (slot - NG);  // 0 .. NG-1, then ha .. ha+NG
  if (slot >= NG && li[q] > hi) return;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    if (li[r] > hi_index(g, kind, r)) return;
  int loc[3];
  loc_of(g, b, loc);
  if (!moved_along(g, kind, li, q, loc[q])) return;
  const long long c = cell_off(g, li[2], li[1], li[0]);
  if (kind == 0) {
    double* U = lu + (long long)b * 5 * g.box + c;
    for (int v = 0; v < 5; ++v) U[(long long)v * g.box] = 0.0;
  } else {
    (kind == 1 ? lb0 : (kind == 2 ? lb1 : lb2))[(long long)b * g.box + c] = 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// Block layout -> input adjoint (global layout), one thread per global element: cells one to one; a face
// sums its block copies in a fixed order (a face on the boundary between blocks k-1 and k has two: the
// upper face of block k-1, then the lower face of block k).  Writes every output element.
// ------------------------------------------------------------------------------------------------
__global__ void k_adj_gather_in(Geom g, const double* lu, const double* lb0, const double* lb1, const double* lb2,
                                double* gu, double* gb1, double* gb2, double* gb3) {
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long ex = NX + 1, ey = NY + 1, ez = NZ + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ex * ey * ez) return;
  const int gi[3] = {(int)(t % ex), (int)((t / ex) % ey), (int)(t / (ex * ey))};
  const int N[3] = {NX, NY, NZ};
  // block coordinate and local index of a global cell index along q
  auto cell_loc = [&](int q, int m, int& blk, int& l) {
    blk = m / g.mb[q];
    l = m - blk * g.mb[q] + NG;
  };
  const bool in[3] = {gi[0] < NX, gi[1] < NY, gi[2] < NZ};
  if (in[0] && in[1] && in[2]) {
    int bb[3], l[3];
    for (int q = 0; q < 3; ++q) cell_loc(q, gi[q], bb[q], l[q]);
    const long long blk = ((long long)bb[2] * g.nb[1] + bb[1]) * g.nb[0] + bb[0];
    const long long cu = blk * 5 * g.box + cell_off(g, l[2], l[1], l[0]);
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)gi[2] * NY + gi[1]) * NX + gi[0];
    for (int v = 0; v < 5; ++v) gu[v * n + gc] = lu[cu + (long long)v * g.box];
  }
  const double* LB[3] = {lb0, lb1, lb2};
  double* GB[3] = {gb1, gb2, gb3};
  for (int fd = 0; fd < 3; ++fd) {
    bool ok = true;
    for (int q = 0; q < 3; ++q)
      if (q != fd) ok = ok && in[q];
    if (!ok) continue;
    int bb[3], l[3];
    for (int q = 0; q < 3; ++q)
      if (q != fd) cell_loc(q, gi[q], bb[q], l[q]);
    double x = 0.0;
    const int m = gi[fd];
    // upper face of the block below (faces k*mb, 0 < k <= nb)
    if (m > 0 && m % g.mb[fd] == 0) {
      bb[fd] = m / g.mb[fd] - 1;
      l[fd] = NG + g.mb[fd];
      const long long blk = ((long long)bb[2] * g.nb[1] + bb[1]) * g.nb[0] + bb[0];
      x += LB[fd][blk * g.box + cell_off(g, l[2], l[1], l[0])];
    }
    // the face as a lower or interior face of its own block (all but global face N)
    if (m < N[fd]) {
      cell_loc(fd, m, bb[fd], l[fd]);
      const long long blk = ((long long)bb[2] * g.nb[1] + bb[1]) * g.nb[0] + bb[0];
      x += LB[fd][blk * g.box + cell_off(g, l[2], l[1], l[0])];
    }
    long long o;
    if (fd == 0)
      o = ((long long)gi[2] * NY + gi[1]) * (NX + 1) + gi[0];
    else if (fd == 1)
      o = ((long long)gi[2] * (NY + 1) + gi[1]) * NX + gi[0];
    else
      o = ((long long)gi[2] * NY + gi[1]) * NX + gi[0];
    GB[fd][o] = x;
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of prims -> conserved (the set-up map): from lam_U (global layout) and the primitives
// (rho, v, p) and cell field, lam_w = (lam_rho, lam_v, lam_p); the field part is not returned.
// ------------------------------------------------------------------------------------------------
__global__ void k_prims_vjp(long long n, double igm1, const double* w, const double* lam_u, double* lam_w) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double d = w[t], vx = w[n + t], vy = w[2 * n + t], vz = w[3 * n + t];
  const double l0 = lam_u[t], l1 = lam_u[n + t], l2 = lam_u[2 * n + t], l3 = lam_u[3 * n + t], l4 = lam_u[4 * n + t];
  // U = (rho, rho v, p/(gamma-1) + rho v^2/2 + |b_c|^2/2)
  lam_w[t] = l0 + l1 * vx + l2 * vy + l3 * vz + l4 * 0.5 * (vx * vx + vy * vy + vz * vz);
  lam_w[n + t] = d * (l1 + l4 * vx);
  lam_w[2 * n + t] = d * (l2 + l4 * vy);
  lam_w[3 * n + t] = d * (l3 + l4 * vz);
  lam_w[4 * n + t] = l4 * igm1;
}

// Pointwise Riemann VJP for n interfaces (rows of 7 / 15), for checking the adjoint's flux derivative.
__global__ void k_riemann_vjp_points(int rs, long long n, const double* wl, const double* wr, const double* bn,
                                     const double* lf, double gamma, double* out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double a[7], b[7], l[7], x[15];
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    a[m] = wl[7 * q + m];
    b[m] = wr[7 * q + m];
    l[m] = lf[7 * q + m];
  }
#pragma unroll
  for (int k = 0; k < 15; ++k) x[k] = 0.0;
  const double igm1 = 1.0 / (gamma - 1.0);
  if (rs == RS_HLLD)
    flux_hlld_vjp(a, b, bn[q], gamma, igm1, l, x, x + 7, x[14]);
  else
    flux_hlle_vjp(a, b, bn[q], gamma, igm1, l, x, x + 7, x[14]);
#pragma unroll
  for (int k = 0; k < 15; ++k) out[15 * q + k] = x[k];
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
constexpr int AT = 256;

static long long nodes_ext(const Geom& g) {
  return (long long)(g.mb[0] + 2) * (g.mb[1] + 2) * (g.mb[2] + 2) * g.nblk;
}
static long long nodes_act(const Geom& g) {
  return (long long)(g.mb[0] + 1) * (g.mb[1] + 1) * (g.mb[2] + 1) * g.nblk;
}

cudaError_t adj_scatter_out(const Geom& g, const AdjArrays& j, const double* gu, const double* gb1, const double* gb2,
                            const double* gb3, cudaStream_t st) {
  k_adj_scatter_out<<<grid_of(nodes_act(g), AT), AT, 0, st>>>(g, j.lu[0], j.lb[0][0], j.lb[0][1], j.lb[0][2], gu, gb1,
                                                              gb2, gb3);
  return cudaGetLastError();
}

cudaError_t adj_update(const Geom& g, const AdjArrays& j, int out_reg, int base_reg, double h, cudaStream_t st) {
  k_adj_update<<<grid_of(nodes_ext(g), AT), AT, 0, st>>>(
      g, j.lu[out_reg], j.lb[out_reg][0], j.lb[out_reg][1], j.lb[out_reg][2], j.lu[base_reg], j.lb[base_reg][0],
      j.lb[base_reg][1], j.lb[base_reg][2], j.lf[0], j.lf[1], j.lf[2], j.le[0], j.le[1], j.le[2], h,
      out_reg != base_reg ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t adj_ct(const Geom& g, const AdjArrays& j, const double* W, const double* const* mflux, long long mstride,
                   long long e5off, long long e6off, cudaStream_t st) {
  if (g.ct_delta > 0.0)
    k_adj_ct<true><<<grid_of(nodes_ext(g), AT), AT, 0, st>>>(g, W, mflux[0], mflux[1], mflux[2], mstride, e5off,
                                                             e6off, g.ct_delta, j.le[0], j.le[1], j.le[2], j.lf[0],
                                                             j.lf[1], j.lf[2], j.lw);
  else
    k_adj_ct<false><<<grid_of(nodes_ext(g), AT), AT, 0, st>>>(g, W, mflux[0], mflux[1], mflux[2], mstride, e5off,
                                                              e6off, 0.0, j.le[0], j.le[1], j.le[2], j.lf[0],
                                                              j.lf[1], j.lf[2], j.lw);
  return cudaGetLastError();
}

cudaError_t adj_flux_halo(const Geom& g, const AdjArrays& j, cudaStream_t st) {
  if (g.flux_halo) return cudaSuccess;
  long long n = 0;
  for (int d = 0; d < 3; ++d) n += (long long)(g.mb[0] + (d == 0)) * (g.mb[1] + (d == 1)) * (g.mb[2] + (d == 2));
  n *= g.nblk;
  k_adj_flux_halo<<<grid_of(n, 256), 256, 0, st>>>(g, j.lf[0], j.lf[1], j.lf[2]);
  return cudaGetLastError();
}

template <int DIR, int REC, int RS>
static cudaError_t adj_flux_one(const Geom& g, const AdjArrays& j, const double* W, const double* Bn, double* lbn,
                                cudaStream_t st) {
  long long n = g.nblk;
  for (int q = 0; q < 3; ++q) n *= g.mb[q] + (q == DIR ? 1 : 2 * g.flux_halo);
  k_adj_flux<DIR, REC, RS><<<grid_of(n, 128), 128, 0, st>>>(g, W, Bn, j.lf[DIR], j.lr, lbn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (REC == REC_PLM) {
    long long ns = g.nblk;
    for (int q = 0; q < 3; ++q) ns *= g.mb[q] + (q == DIR ? 2 : 2 * g.flux_halo);
    k_adj_slopes<DIR><<<grid_of(ns, 128), 128, 0, st>>>(g, W, j.lf[DIR], j.lr, j.ps[0], j.ps[1], j.ps[2]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  constexpr int H = (REC == REC_DC) ? 1 : 2;
  long long nc = g.nblk;
  for (int q = 0; q < 3; ++q) nc *= g.mb[q] + (q == DIR ? 2 * H : 2 * g.flux_halo);
  k_adj_flux_cells<DIR, REC><<<grid_of(nc, 128), 128, 0, st>>>(g, W, j.lf[DIR], j.lr, j.ps[0], j.ps[1], j.ps[2],
                                                              j.lw);
  return cudaGetLastError();
}

template <int REC, int RS>
static cudaError_t adj_flux_all(const Geom& g, const AdjArrays& j, const double* W, const double* const* Bn,
                                double* const* lbn, cudaStream_t st) {
  cudaError_t e = adj_flux_one<0, REC, RS>(g, j, W, Bn[0], lbn[0], st);
  if (e == cudaSuccess) e = adj_flux_one<1, REC, RS>(g, j, W, Bn[1], lbn[1], st);
  if (e == cudaSuccess) e = adj_flux_one<2, REC, RS>(g, j, W, Bn[2], lbn[2], st);
  return e;
}

cudaError_t adj_fluxes(const Geom& g, const AdjArrays& j, int recon, int riemann, const double* W,
                       const double* const* Bn, int lam_reg, cudaStream_t st) {
  double* const lbn[3] = {j.lb[lam_reg][0], j.lb[lam_reg][1], j.lb[lam_reg][2]};
  if (recon == REC_DC)
    return riemann == RS_HLLD ? adj_flux_all<REC_DC, RS_HLLD>(g, j, W, Bn, lbn, st)
                              : adj_flux_all<REC_DC, RS_HLLE>(g, j, W, Bn, lbn, st);
  return riemann == RS_HLLD ? adj_flux_all<REC_PLM, RS_HLLD>(g, j, W, Bn, lbn, st)
                            : adj_flux_all<REC_PLM, RS_HLLE>(g, j, W, Bn, lbn, st);
}

cudaError_t adj_prim(const Geom& g, const AdjArrays& j, const double* W, int lam_reg, cudaStream_t st) {
  // one thread per node 0 .. mb + 2 NG (cells and their faces)
  const long long n = (long long)(g.mb[0] + 2 * NG + 1) * (g.mb[1] + 2 * NG + 1) * (g.mb[2] + 2 * NG + 1) * g.nblk;
  k_adj_prim<<<grid_of(n, AT), AT, 0, st>>>(g, W, j.lw, j.lu[lam_reg], j.lb[lam_reg][0], j.lb[lam_reg][1],
                                            j.lb[lam_reg][2]);
  return cudaGetLastError();
}

cudaError_t adj_ghosts(const Geom& g, const AdjArrays& j, int lam_reg, cudaStream_t st) {
  double* U = j.lu[lam_reg];
  double* const* Bl = j.lb[lam_reg];
  for (int pass = 0; pass < 3; ++pass) {
    const long long pg = pass_elems(g, 2 * (NG + 2), pass), pc = pass_elems(g, 2 * NG + 1, pass);  // per block
    if (pass == 0) {
      k_adj_ghost_gather<0><<<grid_of(pg * g.nblk, AT), AT, 0, st>>>(g, pg, U, Bl[0], Bl[1], Bl[2]);
      k_adj_ghost_clear<0><<<grid_of(pc * g.nblk, AT), AT, 0, st>>>(g, pc, U, Bl[0], Bl[1], Bl[2]);
    } else if (pass == 1) {
      k_adj_ghost_gather<1><<<grid_of(pg * g.nblk, AT), AT, 0, st>>>(g, pg, U, Bl[0], Bl[1], Bl[2]);
      k_adj_ghost_clear<1><<<grid_of(pc * g.nblk, AT), AT, 0, st>>>(g, pc, U, Bl[0], Bl[1], Bl[2]);
    } else {
      k_adj_ghost_gather<2><<<grid_of(pg * g.nblk, AT), AT, 0, st>>>(g, pg, U, Bl[0], Bl[1], Bl[2]);
      k_adj_ghost_clear<2><<<grid_of(pc * g.nblk, AT), AT, 0, st>>>(g, pc, U, Bl[0], Bl[1], Bl[2]);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t adj_gather_in(const Geom& g, const AdjArrays& j, double* gu, double* gb1, double* gb2, double* gb3,
                          cudaStream_t st) {
  const long long n = (long long)(g.N[0] + 1) * (g.N[1] + 1) * (g.N[2] + 1);
  k_adj_gather_in<<<grid_of(n, AT), AT, 0, st>>>(g, j.lu[0], j.lb[0][0], j.lb[0][1], j.lb[0][2], gu, gb1,
                                                            gb2, gb3);
  return cudaGetLastError();
}

cudaError_t prims_vjp(long long ncell, double igm1, const double* w, const double* lam_u, double* lam_w, cudaStream_t st) {
  k_prims_vjp<<<grid_of(ncell, AT), AT, 0, st>>>(ncell, igm1, w, lam_u, lam_w);
  return cudaGetLastError();
}

cudaError_t riemann_vjp_points(int rs, long long n, const double* wl, const double* wr, const double* bn,
                               const double* lf, double gamma, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_riemann_vjp_points<<<grid_of(n, 128), 128, 0, st>>>(rs, n, wl, wr, bn, lf, gamma, out);
  return cudaGetLastError();
}

}  // namespace vl2
