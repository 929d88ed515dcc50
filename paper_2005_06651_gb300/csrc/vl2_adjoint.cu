// Reverse (adjoint) of one VL2 cycle in FP64: given the adjoint of the cycle's output state, the adjoint
// of its input state, with dt held fixed.  Written kernel by kernel in reverse order of the cycle
// (Sec. 3.2.3): update -> CT corner EMFs -> fluxes (PLM / donor cell + Riemann solver) -> cons->prim ->
// ghost exchange, for the corrector and then the predictor.  The linear steps (update, CT for the frozen
// upwind choices, ghost exchange, PLM limiter away from its switch) have hand-derived transposes; the
// Riemann solvers have hand-written reverse-mode derivatives (vl2_riemann_vjp.cuh) that replay the
// forward flux's arithmetic and branch decisions.
#include "vl2_internal.h"
#include "vl2_physics.cuh"
#include "vl2_riemann_vjp.cuh"

namespace vl2 {

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

__device__ __forceinline__ void cell_emf_adj(int e, const double* Wc, long long box, double lam, double* LWc) {
  const double vx = Wc[box], vy = Wc[2 * box], vz = Wc[3 * box];
  const double bx = Wc[5 * box], by = Wc[6 * box], bz = Wc[7 * box];
  if (e == 0) {  // vz by - vy bz
    atomicAdd(LWc + 3 * box, lam * by);
    atomicAdd(LWc + 6 * box, lam * vz);
    atomicAdd(LWc + 2 * box, -lam * bz);
    atomicAdd(LWc + 7 * box, -lam * vy);
  } else if (e == 1) {  // vx bz - vz bx
    atomicAdd(LWc + 1 * box, lam * bz);
    atomicAdd(LWc + 7 * box, lam * vx);
    atomicAdd(LWc + 3 * box, -lam * bx);
    atomicAdd(LWc + 5 * box, -lam * vz);
  } else {  // vy bx - vx by
    atomicAdd(LWc + 2 * box, lam * bx);
    atomicAdd(LWc + 5 * box, lam * vy);
    atomicAdd(LWc + 1 * box, -lam * by);
    atomicAdd(LWc + 6 * box, -lam * vx);
  }
}

__global__ void k_adj_ct(Geom g, const double* W, const double* m0, const double* m1, const double* m2, long long mstride,
                         const double* le0, const double* le1, const double* le2, double* lf0, double* lf1,
                         double* lf2, double* lw) {
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex + NG, (rem / ex) % ey + NG, rem / (ex * ey) + NG};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const double* M[3] = {m0, m1, m2};
  const double* LE[3] = {le0, le1, le2};
  double* LF[3] = {lf0, lf1, lf2};
  const double* Wb = W + (long long)b * 8 * g.box;
  double* LWb = lw + (long long)b * 8 * g.box;
  for (int e = 0; e < 3; ++e) {
    if (li[e] > NG + g.mb[e] - 1) continue;
    const double lam = LE[e][(long long)b * g.box + c];
    if (lam == 0.0) continue;
    const int a = (e + 1) % 3, bq = (e + 2) % 3;
    const long long sa = stride[a], sb = stride[bq];
    const double* Ma = M[a] + (long long)b * mstride;
    const double* Mb = M[bq] + (long long)b * mstride;
    double w0, w1, u0, u1, s0, s1, r0, r1;
    pick_w(Ma[c - sb], w0, w1);  // tlo: gradient along b below the corner, by the a-face mass flux at b-1
    pick_w(Ma[c], u0, u1);       // thi
    pick_w(Mb[c - sa], s0, s1);  // slo: gradient along a, by the b-face mass flux at a-1
    pick_w(Mb[c], r0, r1);       // shi
    const double cea0 = 0.25 * (1.0 + s0 + r0), cea1 = 0.25 * (1.0 + s1 + r1);
    const double ceb0 = 0.25 * (1.0 + w0 + u0), ceb1 = 0.25 * (1.0 + w1 + u1);
    const double cec0 = -0.25 * (w0 + s0), cec1 = -0.25 * (w1 + r0);
    const double cec2 = -0.25 * (u0 + s1), cec3 = -0.25 * (u1 + r1);
    double* Fa = LF[a] + (long long)b * 7 * g.box;
    double* Fb = LF[bq] + (long long)b * 7 * g.box;
    atomicAdd(Fa + 5 * g.box + c - sb, -cea0 * lam);  // ea = -F_a[B_t1]
    atomicAdd(Fa + 5 * g.box + c, -cea1 * lam);
    atomicAdd(Fb + 6 * g.box + c - sa, ceb0 * lam);  // eb = +F_b[B_t2]
    atomicAdd(Fb + 6 * g.box + c, ceb1 * lam);
    cell_emf_adj(e, Wb + c - sa - sb, g.box, cec0 * lam, LWb + c - sa - sb);
    cell_emf_adj(e, Wb + c - sb, g.box, cec1 * lam, LWb + c - sb);
    cell_emf_adj(e, Wb + c - sa, g.box, cec2 * lam, LWb + c - sa);
    cell_emf_adj(e, Wb + c, g.box, cec3 * lam, LWb + c);
  }
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
    const double is2 = 1.0 / (s * s);
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
                                                  const double* __restrict__ LF, double* lw, double* lbn) {
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  const int rx = g.mb[0] + (DIR == 0 ? 1 : 2);
  const int ry = g.mb[1] + (DIR == 1 ? 1 : 2);
  const int rz = g.mb[2] + (DIR == 2 ? 1 : 2);
  const long long per = (long long)rx * ry * rz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % rx + (DIR == 0 ? NG : NG - 1);
  rem /= rx;
  const int j = rem % ry + (DIR == 1 ? NG : NG - 1);
  const int k = rem / ry + (DIR == 2 ? NG : NG - 1);
  const long long c = cell_off(g, k, j, i);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  const double* Fl = LF + (long long)b * 7 * g.box + c;
  double lf[7];
  bool any = false;
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    lf[n] = Fl[(long long)n * g.box];
    any = any || lf[n] != 0.0;
  }
  if (!any) return;
  const double* Wb = W + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  double wl[7], wr[7], q[4][7];
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const double* p = Wb + (long long)var[n] * g.box + c;
    if (REC == REC_DC) {
      q[1][n] = p[-sd];
      q[2][n] = p[0];
      wl[n] = q[1][n];
      wr[n] = q[2][n];
    } else {
      q[0][n] = p[-2 * sd];
      q[1][n] = p[-sd];
      q[2][n] = p[0];
      q[3][n] = p[sd];
      wl[n] = q[1][n] + 0.5 * vl_slope(q[0][n], q[1][n], q[2][n]);
      wr[n] = q[2][n] - 0.5 * vl_slope(q[1][n], q[2][n], q[3][n]);
    }
  }
  const double bn = Bn[(long long)b * g.box + c];
  // adjoints of the 15 Riemann inputs: lam_x[k] = sum_n lf[n] dF_n/dx_k, by reverse mode
  double lx[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) lx[k] = 0.0;
  if (RS == RS_HLLD)
    flux_hlld_vjp(wl, wr, bn, g.gamma, g.igm1, lf, lx, lx + 7, lx[14]);
  else
    flux_hlle_vjp(wl, wr, bn, g.gamma, g.igm1, lf, lx, lx + 7, lx[14]);
  lbn[(long long)b * g.box + c] += lx[14];
  double* LWb = lw + (long long)b * 8 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    double* L = LWb + (long long)var[n] * g.box;
    if (REC == REC_DC) {
      atomicAdd(L - sd, lx[n]);
      atomicAdd(L, lx[7 + n]);
    } else {
      double gm, g0, gp, hm, h0, hp;
      vl_slope_grad(q[0][n], q[1][n], q[2][n], gm, g0, gp);  // w_L = q_{-1} + delta_{-1}/2
      vl_slope_grad(q[1][n], q[2][n], q[3][n], hm, h0, hp);  // w_R = q_0 - delta_0/2
      const double a = lx[n], r = lx[7 + n];
      atomicAdd(L - 2 * sd, 0.5 * gm * a);
      atomicAdd(L - sd, a * (1.0 + 0.5 * g0) - 0.5 * hm * r);
      atomicAdd(L, 0.5 * gp * a + r * (1.0 - 0.5 * h0));
      atomicAdd(L + sd, -0.5 * hp * r);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Transpose of cons->prim on every cell (no floor active): lam_U from lam_W, and the cell-centred field's
// adjoint split half and half onto the two faces of each direction.
// ------------------------------------------------------------------------------------------------
__global__ void k_adj_prim(Geom g, const double* W, const double* lw, double* lu, double* lb0, double* lb1, double* lb2) {
  const int ex = g.mb[0] + 2 * NG, ey = g.mb[1] + 2 * NG, ez = g.mb[2] + 2 * NG;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % ex;
  rem /= ex;
  const int j = rem % ey;
  const int k = rem / ey;
  const long long c = cell_off(g, k, j, i);
  const double* Wc = W + (long long)b * 8 * g.box + c;
  const double* Lc = lw + (long long)b * 8 * g.box + c;
  const double lrho = Lc[0], lvx = Lc[g.box], lvy = Lc[2 * g.box], lvz = Lc[3 * g.box], lp = Lc[4 * g.box];
  const double d = Wc[0], vx = Wc[g.box], vy = Wc[2 * g.box], vz = Wc[3 * g.box];
  const double bx = Wc[5 * g.box], by = Wc[6 * g.box], bz = Wc[7 * g.box];
  const double id = 1.0 / d;
  const double gp = g.gm1 * lp;
  double* U = lu + (long long)b * 5 * g.box + c;
  U[0] += lrho - (lvx * vx + lvy * vy + lvz * vz) * id + gp * 0.5 * (vx * vx + vy * vy + vz * vz);
  U[g.box] += lvx * id - gp * vx;
  U[2 * g.box] += lvy * id - gp * vy;
  U[3 * g.box] += lvz * id - gp * vz;
  U[4 * g.box] += gp;
  const double lbx = Lc[5 * g.box] - gp * bx, lby = Lc[6 * g.box] - gp * by, lbz = Lc[7 * g.box] - gp * bz;
  const long long fb = (long long)b * g.box + c;
  atomicAdd(lb0 + fb, 0.5 * lbx);
  atomicAdd(lb0 + fb + 1, 0.5 * lbx);
  atomicAdd(lb1 + fb, 0.5 * lby);
  atomicAdd(lb1 + fb + g.sx, 0.5 * lby);
  atomicAdd(lb2 + fb, 0.5 * lbz);
  atomicAdd(lb2 + fb + (long long)g.sx * g.sy, 0.5 * lbz);
}

// ------------------------------------------------------------------------------------------------
// Transpose of the ghost exchange: every ghost cell / ghost face adds its adjoint into the active element
// it was copied from, then is cleared.
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

__global__ void k_adj_ghosts(Geom g, double* lu, double* lb0, double* lb1, double* lb2) {
  const int ex = g.mb[0] + 2 * NG + 1, ey = g.mb[1] + 2 * NG + 1, ez = g.mb[2] + 2 * NG + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex, (rem / ex) % ey, rem / (ex * ey)};
  int loc[3];
  loc_of(g, b, loc);
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const int cmax[3] = {g.mb[0] + 2 * NG, g.mb[1] + 2 * NG, g.mb[2] + 2 * NG};
  if (li[0] < cmax[0] && li[1] < cmax[1] && li[2] < cmax[2]) {
    bool ghost = false;
    for (int q = 0; q < 3; ++q) ghost |= (li[q] < NG || li[q] >= NG + g.mb[q]);
    if (ghost) {
      int sb[3], sl[3];
      for (int q = 0; q < 3; ++q) source_of_adj(g, q, loc[q] * g.mb[q] + li[q] - NG, false, sb[q], sl[q]);
      const int src = (sb[2] * g.nb[1] + sb[1]) * g.nb[0] + sb[0];
      double* Ud = lu + (long long)b * 5 * g.box + c;
      double* Us = lu + (long long)src * 5 * g.box + cell_off(g, sl[2], sl[1], sl[0]);
      for (int v = 0; v < 5; ++v) {
        const double x = Ud[(long long)v * g.box];
        if (x != 0.0) atomicAdd(Us + (long long)v * g.box, x);
        Ud[(long long)v * g.box] = 0.0;
      }
    }
  }
  double* Bf[3] = {lb0, lb1, lb2};
  for (int fd = 0; fd < 3; ++fd) {
    bool valid = true, ghost = false;
    for (int q = 0; q < 3; ++q) {
      const int hi_valid = (q == fd) ? cmax[q] : cmax[q] - 1;
      const int hi_active = (q == fd) ? NG + g.mb[q] : NG + g.mb[q] - 1;
      valid &= li[q] <= hi_valid;
      ghost |= (li[q] < NG || li[q] > hi_active);
    }
    if (!valid || !ghost) continue;
    int sb[3], sl[3];
    for (int q = 0; q < 3; ++q) source_of_adj(g, q, loc[q] * g.mb[q] + li[q] - NG, q == fd, sb[q], sl[q]);
    const int src = (sb[2] * g.nb[1] + sb[1]) * g.nb[0] + sb[0];
    double* d = Bf[fd] + (long long)b * g.box + c;
    const double x = *d;
    if (x != 0.0) atomicAdd(Bf[fd] + (long long)src * g.box + cell_off(g, sl[2], sl[1], sl[0]), x);
    *d = 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// Block layout -> input adjoint (global layout): cells one to one; every active copy of a face adds into
// its global entry (interior block boundaries have two copies).  The outputs must be zero on entry.
// ------------------------------------------------------------------------------------------------
__global__ void k_adj_gather_in(Geom g, const double* lu, const double* lb0, const double* lb1, const double* lb2,
                                double* gu, double* gb1, double* gb2, double* gb3) {
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
  const long long o = (long long)b * g.box + cell_off(g, li[2] + NG, li[1] + NG, li[0] + NG);
  if (in[1] && in[2]) atomicAdd(gb1 + ((long long)gi[2] * NY + gi[1]) * (NX + 1) + gi[0], lb0[o]);
  if (in[0] && in[2]) atomicAdd(gb2 + ((long long)gi[2] * (NY + 1) + gi[1]) * NX + gi[0], lb1[o]);
  if (in[0] && in[1]) atomicAdd(gb3 + ((long long)gi[2] * NY + gi[1]) * NX + gi[0], lb2[o]);
  if (in[0] && in[1] && in[2]) {
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)gi[2] * NY + gi[1]) * NX + gi[0];
    const long long cu = (long long)b * 5 * g.box + cell_off(g, li[2] + NG, li[1] + NG, li[0] + NG);
    for (int v = 0; v < 5; ++v) gu[v * n + gc] = lu[cu + (long long)v * g.box];
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
                   cudaStream_t st) {
  k_adj_ct<<<grid_of(nodes_act(g), AT), AT, 0, st>>>(g, W, mflux[0], mflux[1], mflux[2], mstride, j.le[0], j.le[1],
                                                     j.le[2], j.lf[0], j.lf[1], j.lf[2], j.lw);
  return cudaGetLastError();
}

template <int DIR, int REC, int RS>
static cudaError_t adj_flux_one(const Geom& g, const AdjArrays& j, const double* W, const double* Bn, double* lbn,
                                cudaStream_t st) {
  long long n = g.nblk;
  for (int q = 0; q < 3; ++q) n *= g.mb[q] + (q == DIR ? 1 : 2);
  k_adj_flux<DIR, REC, RS><<<grid_of(n, 128), 128, 0, st>>>(g, W, Bn, j.lf[DIR], j.lw, lbn);
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
  const long long n = (long long)(g.mb[0] + 2 * NG) * (g.mb[1] + 2 * NG) * (g.mb[2] + 2 * NG) * g.nblk;
  k_adj_prim<<<grid_of(n, AT), AT, 0, st>>>(g, W, j.lw, j.lu[lam_reg], j.lb[lam_reg][0], j.lb[lam_reg][1],
                                            j.lb[lam_reg][2]);
  return cudaGetLastError();
}

cudaError_t adj_ghosts(const Geom& g, const AdjArrays& j, int lam_reg, cudaStream_t st) {
  const long long n = (long long)(g.mb[0] + 2 * NG + 1) * (g.mb[1] + 2 * NG + 1) * (g.mb[2] + 2 * NG + 1) * g.nblk;
  k_adj_ghosts<<<grid_of(n, AT), AT, 0, st>>>(g, j.lu[lam_reg], j.lb[lam_reg][0], j.lb[lam_reg][1], j.lb[lam_reg][2]);
  return cudaGetLastError();
}

cudaError_t adj_gather_in(const Geom& g, const AdjArrays& j, double* gu, double* gb1, double* gb2, double* gb3,
                          cudaStream_t st) {
  k_adj_gather_in<<<grid_of(nodes_act(g), AT), AT, 0, st>>>(g, j.lu[0], j.lb[0][0], j.lb[0][1], j.lb[0][2], gu, gb1,
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
