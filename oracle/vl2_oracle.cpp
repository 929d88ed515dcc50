/*
 * vl2_oracle.cpp -- plain, slow, FP64 CPU oracle of one VL2 cycle of adiabatic ideal MHD on a
 * uniform mesh of equal-size MeshBlocks (Stone, Tomida, White & Felker 2020, "The Athena++
 * Adaptive Mesh Refinement Framework", arXiv:2005.06651).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline / reference leg may load it; the product path never
 * calls it, and it shares no code, header or table with the CUDA sources.
 *
 * What it follows, step by step (sections / equations of the paper):
 *   - equations of ideal MHD, mu = 1, total energy E = e + rho v^2/2 + B^2/2     (Sec. 3.1, eq. cons,
 *     eq. total_energy), ideal-gas EOS P = (gamma-1) e                          (Sec. 3.1)
 *   - finite volumes: cell-averaged U, face-area-averaged B, edge EMFs (upwind CT) (Sec. 3.1, Sec. 2.1.1)
 *   - MeshBlocks of equal size with N_G = 2 ghost layers (3 for PPM), filled from the 26 neighbours
 *     (periodic wrap, or outflow = copy of the nearest active cell)              (Sec. 2.1, 2.1.1)
 *   - EMFs on edges shared by several MeshBlocks are averaged over the copies   (Sec. 2.1.1)
 *   - donor-cell and PLM reconstruction of primitives, original van Leer limiter (Sec. 3.2.1)
 *   - PPM reconstruction of primitives: fourth-order face values (eq. ppm-uniform-weights) and the
 *     smooth-extremum-preserving limiter the paper names (Colella & Sekora 2008, as extended by
 *     McCorquodale & Colella); N_G = 3                                          (Sec. 3.2.1, 2.1.1)
 *   - HLLE and HLLD approximate Riemann solvers                                 (Sec. 3.2.2)
 *   - 2S low-storage register scheme (eq. rk-2s) with the VL2 coefficients; the
 *     predictor uses donor-cell fluxes                                           (Sec. 3.2.3)
 *   - one global time step from |v| + C_f                                      (Sec. 2.1.7, 3.2.3)
 *   - passive scalars rho C_i, d(rho C_i)/dt + div(rho v C_i) = 0 (eq. passive_scalars), C_i reconstructed
 *     like the other primitives and carried by the Riemann mass flux from the upwind side   (Sec. 3.1)
 *   - options beside the paper's defaults: PLM and PPM on characteristic variables C = L W (Sec. 3.2.1;
 *     eigensystem derived from the primitive equations, L = R^-1 by elimination), HLLE with Einfeldt's
 *     Roe-averaged speeds (Sec. 3.2.2), and a smoothed upwind weight in the CT corner (tanh of the mass
 *     flux; the tangent-linear carries its derivative)
 *
 * The paper names HLLE / HLLD / upwind CT / VL2 but prints no formulas for them; the formulas here
 * are written from the published methods (HLLD: Miyoshi & Kusano 2005; upwind CT: Gardiner &
 * Stone 2005; VL2: Stone & Gardiner 2009).  Every point where the paper is silent is marked
 * [reading] below; the CUDA path takes the same reading.
 *
 * Every expression that combines a left and a right quantity is written so that it is exactly
 * (bitwise) mirror symmetric: swapping L and R and negating the normal components gives the
 * negated result in IEEE arithmetic.  Build with -ffp-contract=off (no FMA contraction), as the
 * paper requires for value-safe symmetric results (Sec. 3.3.5).
 *
 * Parity pins: every function here is pinned by a CPU test (consistency, exact contact / rotational
 * discontinuity, exact Sod solution, linear-wave convergence slope, CT identities, conservation,
 * mirror / axis symmetry).  The choice of the upwind cell in the CT corner EMF (gs05) is pinned only
 * through the convergence slope and the symmetry tests ("parity partially pinned").  Of the options,
 * Einfeldt's HLLE speed is pinned by a Roe matrix built independently from exact difference identities
 * (Roe's property, its extreme eigenvalues) and by exact fast shocks, whose speed it must reproduce; the
 * characteristic eigensystem is pinned by A R = R lam and L R = I, the smoothed weight by its limits,
 * its conditioning and its tangent against finite differences.
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace orc {

using std::fabs;
using std::sqrt;

enum { RS_HLLE = 0, RS_HLLD = 1, RS_HLLE_ROE = 2 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };
enum { REC_DC = 0, REC_PLM = 1, REC_PPM = 2, REC_PLM_CHAR = 3, REC_PPM_CHAR = 4 };
enum { INT_VL2 = 0, INT_RK1 = 1, INT_RK2 = 2, INT_RK3 = 3 };

/* Interface-state layout (normal n, transverse t1, t2 taken cyclically: x->(y,z), y->(z,x),
 * z->(x,y)), and flux layout (mass, normal momentum, two transverse momenta, energy, two transverse
 * field components). */
enum { IDN = 0, IVN = 1, IVT1 = 2, IVT2 = 3, IPR = 4, IBT1 = 5, IBT2 = 6, NW7 = 7 };

template <class T> static inline T vmin(T a, T b) { return (a < b) ? a : b; }
template <class T> static inline T vmax(T a, T b) { return (a > b) ? a : b; }

/* Operation-counting scalar: carries the FP64 value and counts every arithmetic operation applied to
 * it (add/sub, mul, div, sqrt, compare; sign changes and |x| are free).  Instantiating the pointwise
 * functions with it gives the algorithmic FP64 work of one face, used as the roofline's unit cost. */
struct OpCount {
  long long add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
static thread_local OpCount g_ops;
struct Flop {
  double v;
  Flop() : v(0.0) {}
  Flop(double x) : v(x) {}
};
static inline Flop operator+(Flop a, Flop b) { ++g_ops.add; return Flop(a.v + b.v); }
static inline Flop operator-(Flop a, Flop b) { ++g_ops.add; return Flop(a.v - b.v); }
static inline Flop operator*(Flop a, Flop b) { ++g_ops.mul; return Flop(a.v * b.v); }
static inline Flop operator/(Flop a, Flop b) { ++g_ops.div; return Flop(a.v / b.v); }
static inline Flop operator+(double a, Flop b) { return Flop(a) + b; }
static inline Flop operator-(double a, Flop b) { return Flop(a) - b; }
static inline Flop operator*(double a, Flop b) { return Flop(a) * b; }
static inline Flop operator/(double a, Flop b) { return Flop(a) / b; }
static inline Flop operator+(Flop a, double b) { return a + Flop(b); }
static inline Flop operator-(Flop a, double b) { return a - Flop(b); }
static inline Flop operator*(Flop a, double b) { return a * Flop(b); }
static inline Flop operator/(Flop a, double b) { return a / Flop(b); }
static inline Flop operator-(Flop a) { return Flop(-a.v); }
static inline bool operator<(Flop a, Flop b) { ++g_ops.cmp; return a.v < b.v; }
static inline bool operator>(Flop a, Flop b) { ++g_ops.cmp; return a.v > b.v; }
static inline bool operator<=(Flop a, Flop b) { ++g_ops.cmp; return a.v <= b.v; }
static inline bool operator>=(Flop a, Flop b) { ++g_ops.cmp; return a.v >= b.v; }
static inline bool operator==(Flop a, Flop b) { ++g_ops.cmp; return a.v == b.v; }
static inline bool operator<(Flop a, double b) { return a < Flop(b); }
static inline bool operator>(Flop a, double b) { return a > Flop(b); }
static inline bool operator<=(Flop a, double b) { return a <= Flop(b); }
static inline bool operator>=(Flop a, double b) { return a >= Flop(b); }
static inline Flop fabs(Flop a) { return Flop(std::fabs(a.v)); }
static inline Flop sqrt(Flop a) { ++g_ops.sqrt; return Flop(std::sqrt(a.v)); }

/* Dual number (value, tangent) for the tangent-linear of a cycle: every operation carries its exact
 * first-order derivative along one input direction (forward-mode differentiation).  Comparisons look at
 * the value only, so a branch (limiter, Riemann fan region, upwind choice) is frozen at the point. */
struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double t) : v(x), d(t) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static inline Dual operator+(double a, Dual b) { return Dual(a) + b; }
static inline Dual operator-(double a, Dual b) { return Dual(a) - b; }
static inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
static inline Dual operator/(double a, Dual b) { return Dual(a) / b; }
static inline Dual operator+(Dual a, double b) { return a + Dual(b); }
static inline Dual operator-(Dual a, double b) { return a - Dual(b); }
static inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
static inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
static inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
static inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
static inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
static inline bool operator==(Dual a, Dual b) { return a.v == b.v; }
static inline bool operator<(Dual a, double b) { return a.v < b; }
static inline bool operator>(Dual a, double b) { return a.v > b; }
static inline bool operator<=(Dual a, double b) { return a.v <= b; }
static inline bool operator>=(Dual a, double b) { return a.v >= b; }
static inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
static inline Dual sqrt(Dual a) {
  const double r = std::sqrt(a.v);
  return Dual(r, a.d / (2.0 * r));
}
static inline double tanh(double a) { return std::tanh(a); }
static inline Dual tanh(Dual a) {  // d tanh(x) / dx = 1 - tanh(x)^2
  const double t = std::tanh(a.v);
  return Dual(t, a.d * (1.0 - t * t));
}
template <class T> static inline T make_scalar(double v, double t);
template <> inline double make_scalar<double>(double v, double) { return v; }
template <> inline Dual make_scalar<Dual>(double v, double t) { return Dual(v, t); }

/* ---------------------------------------------------------------------------------------------
 * Pointwise physics
 * ------------------------------------------------------------------------------------------- */

/* Conserved state and physical flux of one 1D interface state (eq. cons with P* = P + B^2/2,
 * eq. total_energy, ideal EOS). */
template <class T>
static void physical_flux(const T w[NW7], T bn, double gamma, T u[NW7], T f[NW7]) {
  const T d = w[IDN], vn = w[IVN], vt1 = w[IVT1], vt2 = w[IVT2], p = w[IPR];
  const T bt1 = w[IBT1], bt2 = w[IBT2];
  const T b2 = (bn * bn + bt1 * bt1) + bt2 * bt2;
  const T v2 = (vn * vn + vt1 * vt1) + vt2 * vt2;
  const T e = p / (gamma - 1.0) + 0.5 * d * v2 + 0.5 * b2;
  const T pt = p + 0.5 * b2;
  const T vb = (vn * bn + vt1 * bt1) + vt2 * bt2;
  u[IDN] = d;
  u[IVN] = d * vn;
  u[IVT1] = d * vt1;
  u[IVT2] = d * vt2;
  u[IPR] = e;
  u[IBT1] = bt1;
  u[IBT2] = bt2;
  f[IDN] = d * vn;
  f[IVN] = d * vn * vn + pt - bn * bn;
  f[IVT1] = d * vn * vt1 - bn * bt1;
  f[IVT2] = d * vn * vt2 - bn * bt2;
  f[IPR] = (e + pt) * vn - bn * vb;
  f[IBT1] = bt1 * vn - bn * vt1;
  f[IBT2] = bt2 * vn - bn * vt2;
}

/* Fast magnetosonic speed along the normal, C_f^2 = (a^2 + b^2/rho + sqrt((a^2 + b^2/rho)^2 -
 * 4 a^2 b_n^2/rho)) / 2, with the radicand rewritten as (a^2 - c_n^2)^2 + c_t^2 (c_t^2 + 2 a^2 + 2 c_n^2)
 * (algebraically identical, never negative). */
template <class T>
static T fast_speed(T d, T p, T bn, T bt1, T bt2, double gamma) {
  const T asq = gamma * p / d;
  const T cnsq = bn * bn / d;
  const T ctsq = (bt1 * bt1 + bt2 * bt2) / d;
  const T diff = asq - cnsq;
  const T rad = diff * diff + ctsq * (ctsq + 2.0 * (asq + cnsq));
  const T cf2 = 0.5 * ((asq + cnsq + ctsq) + sqrt(rad));
  return sqrt(cf2);
}

/* HLLE flux [reading: the paper prints no formula; outer speeds are the extreme fast-wave speeds of
 * the two states, S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R)]. */
template <class T>
static void flux_hlle(const T wl[NW7], const T wr[NW7], T bn, double gamma, T f[NW7]) {
  T ul[NW7], ur[NW7], fl[NW7], fr[NW7];
  physical_flux(wl, bn, gamma, ul, fl);
  physical_flux(wr, bn, gamma, ur, fr);
  const T cl = fast_speed(wl[IDN], wl[IPR], bn, wl[IBT1], wl[IBT2], gamma);
  const T cr = fast_speed(wr[IDN], wr[IPR], bn, wr[IBT1], wr[IBT2], gamma);
  const T sl = vmin(wl[IVN] - cl, wr[IVN] - cr);
  const T sr = vmax(wl[IVN] + cl, wr[IVN] + cr);
  const T bm = vmin(sl, T(0.0));
  const T bp = vmax(sr, T(0.0));
  for (int n = 0; n < NW7; ++n)
    f[n] = ((bp * fl[n] - bm * fr[n]) + (bp * bm) * (ur[n] - ul[n])) / (bp - bm);
}

/* Fast speed of a Roe matrix of the 1D ideal-MHD flux, about the Roe-averaged normal velocity (the paper
 * names HLLE and Roe's linearisation, Sec. 3.2.2, without formulas) [reading].  The matrix is the one whose
 * rows are exact difference identities of the flux in the averages
 *   rho~ = sqrt(rho_L rho_R), u~ and H~ = (E + p_T) / rho weighted by sqrt(rho),
 *   b~_t = (sqrt(rho_R) b_t,L + sqrt(rho_L) b_t,R) / (sqrt(rho_L) + sqrt(rho_R))   (cross weights),
 * e.g. d(rho u v) = u~ d(rho v) + v~ d(rho u) - u~ v~ d(rho), d(b_t v_n) = v~_n db_t + b~_t dv_n,
 * dv_n = (d(rho v_n) - v~_n d(rho)) / rho~; the magnetic pressure differs as
 *   d(|b_t|^2 / 2) = b~_t . db_t + X d(rho),   X = |b_t,L - b_t,R|^2 / (2 (sqrt(rho_L) + sqrt(rho_R))^2).
 * Its fast eigenvalues are u~ -+ c~_f with
 *   a~^2 = (gamma - 1)(H~ - |u~|^2 / 2 - |b~|^2 / rho~) - (gamma - 2) X   (|b~|^2 = b_n^2 + |b~_t|^2),
 *   c~_a^2 = b_n^2 / rho~, c~_t^2 = |b~_t|^2 / rho~,
 *   c~_f^2 = (a~^2 + c~_a^2 + c~_t^2 + sqrt((c~_a^2 + c~_t^2 - a~^2)^2 + 4 a~^2 c~_t^2)) / 2.
 * a~^2 >= 0 holds in exact arithmetic (the sqrt(rho) average of |u|^2 is >= |u~|^2 and the field part of
 * H~ exceeds |b~|^2 / rho~ by 2 X); it is floored at 0 against rounding.  Pins: the matrix satisfies
 * Roe's property and has these eigenvalues (checked against an independently built matrix), and for two
 * states joined by one exact fast shock u~ -+ c~_f is the shock speed, as Roe's property requires. */
template <class T>
static void roe_fast_speed(const T wl[NW7], const T wr[NW7], T bn, double gamma, T* un_out, T* cf_out) {
  T ul[NW7], ur[NW7], fl[NW7], fr[NW7];
  physical_flux(wl, bn, gamma, ul, fl);
  physical_flux(wr, bn, gamma, ur, fr);
  const T sdl = sqrt(wl[IDN]), sdr = sqrt(wr[IDN]);
  const T wsum = sdl + sdr;
  const T rho = sdl * sdr;
  T v[3], bt[2];
  for (int k = 0; k < 3; ++k) v[k] = (sdl * wl[IVN + k] + sdr * wr[IVN + k]) / wsum;
  for (int k = 0; k < 2; ++k) bt[k] = (sdr * wl[IBT1 + k] + sdl * wr[IBT1 + k]) / wsum;
  const T ptl = wl[IPR] + 0.5 * ((bn * bn + wl[IBT1] * wl[IBT1]) + wl[IBT2] * wl[IBT2]);
  const T ptr = wr[IPR] + 0.5 * ((bn * bn + wr[IBT1] * wr[IBT1]) + wr[IBT2] * wr[IBT2]);
  const T h = ((ul[4] + ptl) / sdl + (ur[4] + ptr) / sdr) / wsum;
  const T x = 0.5 * ((wl[IBT1] - wr[IBT1]) * (wl[IBT1] - wr[IBT1]) + (wl[IBT2] - wr[IBT2]) * (wl[IBT2] - wr[IBT2])) /
              (wsum * wsum);
  const T btsq = bt[0] * bt[0] + bt[1] * bt[1];
  const T vsq = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
  const T ca2 = bn * bn / rho;
  T a2 = (gamma - 1.0) * ((h - 0.5 * vsq) - (bn * bn + btsq) / rho) - (gamma - 2.0) * x;
  if (a2 < 0.0) a2 = T(0.0);
  const T ct2 = btsq / rho;
  const T tdif = ca2 + ct2 - a2;
  *un_out = v[0];
  *cf_out = sqrt(0.5 * ((a2 + ca2 + ct2) + sqrt(tdif * tdif + 4.0 * a2 * ct2)));
}

/* HLLE flux with Einfeldt's outer speeds: S_L = min(u_L - c_L, u~ - c~_f), S_R = max(u_R + c_R, u~ + c~_f),
 * with u~ and c~_f from roe_fast_speed. */
template <class T>
static void flux_hlle_roe(const T wl[NW7], const T wr[NW7], T bn, double gamma, T f[NW7]) {
  T ul[NW7], ur[NW7], fl[NW7], fr[NW7];
  physical_flux(wl, bn, gamma, ul, fl);
  physical_flux(wr, bn, gamma, ur, fr);
  const T cl = fast_speed(wl[IDN], wl[IPR], bn, wl[IBT1], wl[IBT2], gamma);
  const T cr = fast_speed(wr[IDN], wr[IPR], bn, wr[IBT1], wr[IBT2], gamma);
  T un, cf;
  roe_fast_speed(wl, wr, bn, gamma, &un, &cf);
  const T sl = vmin(wl[IVN] - cl, un - cf);
  const T sr = vmax(wr[IVN] + cr, un + cf);
  const T bm = vmin(sl, T(0.0));
  const T bp = vmax(sr, T(0.0));
  for (int n = 0; n < NW7; ++n)
    f[n] = ((bp * fl[n] - bm * fr[n]) + (bp * bm) * (ur[n] - ul[n])) / (bp - bm);
}

/* HLLD flux (Miyoshi & Kusano 2005), written out in the order of that method:
 * outer speeds, contact speed S_M, total pressure p_T*, single-star states, Alfven speeds S*_L/R,
 * double-star states, flux selection.
 * [reading] S_L = min(u_L,u_R) - max(c_L,c_R), S_R = max(u_L,u_R) + max(c_L,c_R);
 * [reading] p_T* in its symmetric two-sided form;
 * [reading] degenerate single-star case when |rho(S-u)(S-S_M) - b_n^2| <= 1e-8 p_T*: transverse
 *           velocity and field unchanged;
 * [reading] sign(b_n) = +1 for b_n = 0 (the double-star fans then have zero width);
 * [reading] selection: the sign of S_M picks the side; on a side, ties at a wave speed of exactly 0
 *           go to the outer state (the added jump is multiplied by 0); at S_M == 0 exactly the two
 *           sides' double-star (or star) fluxes are averaged, which keeps the scheme exactly mirror
 *           symmetric. */
template <class T>
static void flux_hlld(const T wl[NW7], const T wr[NW7], T bn, double gamma, T f[NW7]) {
  T ul[NW7], ur[NW7], fl[NW7], fr[NW7];
  physical_flux(wl, bn, gamma, ul, fl);
  physical_flux(wr, bn, gamma, ur, fr);
  const T cl = fast_speed(wl[IDN], wl[IPR], bn, wl[IBT1], wl[IBT2], gamma);
  const T cr = fast_speed(wr[IDN], wr[IPR], bn, wr[IBT1], wr[IBT2], gamma);
  const T cmax = vmax(cl, cr);
  const T sl = vmin(wl[IVN], wr[IVN]) - cmax;
  const T sr = vmax(wl[IVN], wr[IVN]) + cmax;

  const T ptl = wl[IPR] + 0.5 * ((bn * bn + wl[IBT1] * wl[IBT1]) + wl[IBT2] * wl[IBT2]);
  const T ptr = wr[IPR] + 0.5 * ((bn * bn + wr[IBT1] * wr[IBT1]) + wr[IBT2] * wr[IBT2]);
  const T al = (sl - wl[IVN]) * wl[IDN];  // rho_L (S_L - u_L) < 0
  const T ar = (sr - wr[IVN]) * wr[IDN];  // rho_R (S_R - u_R) > 0
  const T den = ar - al;
  const T sm = ((ar * wr[IVN] - al * wl[IVN]) + (ptl - ptr)) / den;
  const T ptst = ((ar * ptl - al * ptr) + (ar * al) * (wr[IVN] - wl[IVN])) / den;

  /* single-star states */
  T us[2][NW7];
  T dst[2];
  const T* w[2] = {wl, wr};
  const T* uu[2] = {ul, ur};
  const T s[2] = {sl, sr};
  const T a[2] = {al, ar};
  const T pt[2] = {ptl, ptr};
  T vbst[2];
  T vtst[2][2], btst[2][2];
  for (int side = 0; side < 2; ++side) {
    const T* ws = w[side];
    const T sms = s[side] - sm;
    dst[side] = a[side] / sms;
    const T dd = a[side] * sms - bn * bn;
    if (fabs(dd) > 1.0e-8 * ptst) {
      const T tv = bn * (sm - ws[IVN]) / dd;
      const T tb = (a[side] * (s[side] - ws[IVN]) - bn * bn) / dd;
      vtst[side][0] = ws[IVT1] - ws[IBT1] * tv;
      vtst[side][1] = ws[IVT2] - ws[IBT2] * tv;
      btst[side][0] = ws[IBT1] * tb;
      btst[side][1] = ws[IBT2] * tb;
    } else {
      vtst[side][0] = ws[IVT1];
      vtst[side][1] = ws[IVT2];
      btst[side][0] = ws[IBT1];
      btst[side][1] = ws[IBT2];
    }
    const T vb = (ws[IVN] * bn + ws[IVT1] * ws[IBT1]) + ws[IVT2] * ws[IBT2];
    vbst[side] = (sm * bn + vtst[side][0] * btst[side][0]) + vtst[side][1] * btst[side][1];
    const T est = ((((s[side] - ws[IVN]) * uu[side][IPR] - pt[side] * ws[IVN]) + ptst * sm) +
                   bn * (vb - vbst[side])) /
                  sms;
    us[side][IDN] = dst[side];
    us[side][IVN] = dst[side] * sm;
    us[side][IVT1] = dst[side] * vtst[side][0];
    us[side][IVT2] = dst[side] * vtst[side][1];
    us[side][IPR] = est;
    us[side][IBT1] = btst[side][0];
    us[side][IBT2] = btst[side][1];
  }

  /* double-star states */
  const T sqdl = sqrt(dst[0]);
  const T sqdr = sqrt(dst[1]);
  const T abn = fabs(bn);
  const T sls = sm - abn / sqdl;
  const T srs = sm + abn / sqdr;
  const T sgn = (bn >= 0.0) ? T(1.0) : T(-1.0);
  const T sqsum = sqdl + sqdr;
  const T vt1ss = ((sqdl * vtst[0][0] + sqdr * vtst[1][0]) + (btst[1][0] - btst[0][0]) * sgn) / sqsum;
  const T vt2ss = ((sqdl * vtst[0][1] + sqdr * vtst[1][1]) + (btst[1][1] - btst[0][1]) * sgn) / sqsum;
  const T bt1ss =
      ((sqdl * btst[1][0] + sqdr * btst[0][0]) + (sqdl * sqdr) * (vtst[1][0] - vtst[0][0]) * sgn) / sqsum;
  const T bt2ss =
      ((sqdl * btst[1][1] + sqdr * btst[0][1]) + (sqdl * sqdr) * (vtst[1][1] - vtst[0][1]) * sgn) / sqsum;
  const T vbss = (sm * bn + vt1ss * bt1ss) + vt2ss * bt2ss;
  T uss[2][NW7];
  for (int side = 0; side < 2; ++side) {
    uss[side][IDN] = dst[side];
    uss[side][IVN] = dst[side] * sm;
    uss[side][IVT1] = dst[side] * vt1ss;
    uss[side][IVT2] = dst[side] * vt2ss;
    uss[side][IBT1] = bt1ss;
    uss[side][IBT2] = bt2ss;
  }
  uss[0][IPR] = us[0][IPR] - sqdl * (vbst[0] - vbss) * sgn;
  uss[1][IPR] = us[1][IPR] + sqdr * (vbst[1] - vbss) * sgn;

  /* flux selection: left-side pick and right-side pick */
  T fpl[NW7], fpr[NW7];
  for (int n = 0; n < NW7; ++n) {
    if (sl >= 0.0) {
      fpl[n] = fl[n];
    } else if (sls >= 0.0) {
      fpl[n] = fl[n] + sl * (us[0][n] - ul[n]);
    } else {
      fpl[n] = (fl[n] + sl * (us[0][n] - ul[n])) + sls * (uss[0][n] - us[0][n]);
    }
    if (sr <= 0.0) {
      fpr[n] = fr[n];
    } else if (srs <= 0.0) {
      fpr[n] = fr[n] + sr * (us[1][n] - ur[n]);
    } else {
      fpr[n] = (fr[n] + sr * (us[1][n] - ur[n])) + srs * (uss[1][n] - us[1][n]);
    }
  }
  for (int n = 0; n < NW7; ++n) {
    if (sm > 0.0)
      f[n] = fpl[n];
    else if (sm < 0.0)
      f[n] = fpr[n];
    else
      f[n] = 0.5 * (fpl[n] + fpr[n]);
  }
}

template <class T>
static void riemann(int solver, const T wl[NW7], const T wr[NW7], T bn, double gamma, T f[NW7]) {
  if (solver == RS_HLLE)
    flux_hlle(wl, wr, bn, gamma, f);
  else if (solver == RS_HLLE_ROE)
    flux_hlle_roe(wl, wr, bn, gamma, f);
  else
    flux_hlld(wl, wr, bn, gamma, f);
}

/* Piecewise-linear slope with the original van Leer (harmonic-mean) limiter on a uniform grid
 * (Sec. 3.2.1): delta = 2 dl dr / (dl + dr) if dl dr > 0, else 0. */
template <class T>
static T vanleer_slope(T qm, T q0, T qp) {
  const T dl = q0 - qm;
  const T dr = qp - q0;
  const T prod = dl * dr;
  if (prod > 0.0) return (2.0 * dl * dr) / (dl + dr);
  return T(0.0);
}

/* PPM edge values of one cell (Sec. 3.2.1) from the five cell values q[0..4] = q_{i-2} .. q_{i+2}:
 *   1. fourth-order face values, eq. ppm-uniform-weights:
 *        q_{i-1/2} = 7/12 (q_{i-1} + q_i) - 1/12 (q_{i-2} + q_{i+1});
 *   2. a face value outside the range of its two cells is replaced by
 *        (q_{i-1} + q_i)/2 - D2lim/6,   D2 = 3 (q_{i-1} - 2 q_{i-1/2} + q_i),
 *      D2lim = sign(D2) min(|D2|, C |D2L|, C |D2R|) when D2 and the neighbouring second differences
 *      D2L = q_{i-2} - 2 q_{i-1} + q_i, D2R = q_{i-1} - 2 q_i + q_{i+1} share its sign, else 0 (C = 1.25);
 *      with D2lim = D2 this returns the face value unchanged;
 *   3. the cell's parabola (edges qL, qR):
 *      - at an extremum ((qR - q_i)(q_i - qL) <= 0 or (q_{i+1} - q_i)(q_i - q_{i-1}) <= 0) its second
 *        derivative D2 = 6 (qL + qR - 2 q_i) is limited like step 2 against D2C = q_{i-1} - 2 q_i + q_{i+1},
 *        D2L and D2R of the cells around, and both edges move towards q_i by the factor D2lim / D2
 *        (to q_i when D2 = 0);
 *      - otherwise an edge whose distance from q_i exceeds twice the other edge's is pulled in to
 *        twice that distance on its side (the parabola stays monotone in the cell).
 * [reading] The paper prints step 1 and names the limiter; steps 2 and 3 follow Colella & Sekora
 * 2008.  McCorquodale & Colella's further test of third differences near smooth extrema is not
 * applied. */
// Second differences are written (outer sum) - 2 middle, so that mirrored inputs give bitwise mirrored
// results (as everywhere in this file).
template <class T> static inline T ppm_sign(T x) { return (x > 0.0) ? T(1.0) : ((x < 0.0) ? T(-1.0) : T(0.0)); }

template <class T>
static T ppm_face(T qm2, T qm1, T q0, T qp1) {
  const double C = 1.25;
  T f = (7.0 / 12.0) * (qm1 + q0) - (1.0 / 12.0) * (qm2 + qp1);
  if ((f - qm1) * (q0 - f) < 0.0) {
    const T d2 = 3.0 * ((qm1 + q0) - 2.0 * f);
    const T d2l = (qm2 + q0) - 2.0 * qm1;
    const T d2r = (qm1 + qp1) - 2.0 * q0;
    T lim = T(0.0);
    const T s = ppm_sign(d2);
    if (ppm_sign(d2l) == s && ppm_sign(d2r) == s && !(s == 0.0))
      lim = s * vmin(fabs(d2), vmin(C * fabs(d2l), C * fabs(d2r)));
    f = 0.5 * (qm1 + q0) - lim / 6.0;
  }
  return f;
}

/* Edges (ql, qr) of cell i from q[0..4] = q_{i-2} .. q_{i+2}.  A face between cells i-1 and i therefore
 * reads q_{i-3} .. q_{i+2}: three ghost layers. */
template <class T>
static void ppm_edges(const T q[5], T& ql, T& qr) {
  const double C = 1.25;
  const T qm2 = q[0], qm1 = q[1], q0 = q[2], qp1 = q[3], qp2 = q[4];
  ql = ppm_face(qm2, qm1, q0, qp1);
  qr = ppm_face(qm1, q0, qp1, qp2);
  if ((qr - q0) * (q0 - ql) <= 0.0 || (qp1 - q0) * (q0 - qm1) <= 0.0) {
    const T d2 = 6.0 * ((ql + qr) - 2.0 * q0);
    const T d2c = (qm1 + qp1) - 2.0 * q0;
    const T d2l = (qm2 + q0) - 2.0 * qm1;
    const T d2r = (q0 + qp2) - 2.0 * qp1;
    const T s = ppm_sign(d2);
    T lim = T(0.0);
    if (!(s == 0.0) && ppm_sign(d2c) == s && ppm_sign(d2l) == s && ppm_sign(d2r) == s)
      lim = s * vmin(fabs(d2), vmin(C * fabs(d2c), vmin(C * fabs(d2l), C * fabs(d2r))));
    if (s == 0.0) {
      ql = q0;
      qr = q0;
    } else {
      const T r = lim / d2;
      ql = q0 + r * (ql - q0);
      qr = q0 + r * (qr - q0);
    }
  } else {
    const T dl = ql - q0, dr = qr - q0;
    if (fabs(dl) >= 2.0 * fabs(dr)) ql = q0 - 2.0 * dr;
    if (fabs(dr) >= 2.0 * fabs(dl)) qr = q0 - 2.0 * dl;
  }
}

/* ---------------------------------------------------------------------------------------------
 * Characteristic reconstruction (Sec. 3.2.1): the limiter acts on C = L W, the rows of L being the
 * left eigenvectors of the primitive ideal-MHD system (the paper defers to Stone et al. 2008,
 * Appendix A).  Along the sweep normal n, with W = (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) and b_n held
 * fixed, the primitive equations read W_t + A W_n = 0 with
 *   A = [[v, rho,     0,     0,     0,       0,       0     ],
 *        [0, v,       0,     0,     1/rho,   b_t1/rho, b_t2/rho],
 *        [0, 0,       v,     0,     0,      -b_n/rho,  0     ],
 *        [0, 0,       0,     v,     0,       0,      -b_n/rho],
 *        [0, gamma p, 0,     0,     v,       0,       0     ],
 *        [0, b_t1,   -b_n,   0,     0,       v,       0     ],
 *        [0, b_t2,    0,    -b_n,   0,       0,       v     ]]   (v = v_n).
 * Its eigenvalues are v -+ c_f, v -+ c_a, v -+ c_s and v, with a^2 = gamma p / rho, c_a^2 = b_n^2 / rho,
 * c_t^2 = |b_t|^2 / rho, c_f^2 = (a^2 + c_a^2 + c_t^2 + sqrt((c_a^2 + c_t^2 - a^2)^2 + 4 a^2 c_t^2)) / 2
 * and c_s^2 = a^2 c_a^2 / c_f^2.  The right eigenvectors (columns of R, in the order of the
 * eigenvalues v - c_f, v - c_a, v - c_s, v, v + c_s, v + c_a, v + c_f) are written with the
 * normalisation that stays finite where waves coincide:
 *   beta = b_t / |b_t| (both components 1/sqrt(2) where b_t = 0), s = sign(b_n) (+1 at 0),
 *   alpha_f^2 = (a^2 - c_s^2) / (c_f^2 - c_s^2), alpha_s^2 = (c_f^2 - a^2) / (c_f^2 - c_s^2) (both in
 *   [0, 1], summing to 1), taken as (1, 0) where c_f = c_s,
 *   C_f = c_f alpha_f, C_s = c_s alpha_s, Q_f = s C_f, Q_s = s C_s,
 *   A_f = a alpha_f sqrt(rho), A_s = a alpha_s sqrt(rho):
 *   fast  v -+ c_f: (rho alpha_f, -+C_f, +-Q_s beta, rho a^2 alpha_f,  A_s beta)
 *   Alfven v -+ c_a: (0, 0, (-beta_2, beta_1), 0, -+s sqrt(rho) (beta_2, -beta_1))
 *   slow  v -+ c_s: (rho alpha_s, -+C_s, -+Q_f beta, rho a^2 alpha_s, -A_f beta)
 *   entropy v:      (1, 0, 0, 0, 0, 0, 0).
 * (Derived from A: for a magnetosonic speed c, d rho = rho dv_n / c, dp = rho a^2 dv_n / c,
 * db_t = b_t c dv_n / (c^2 - c_a^2), dv_t = -b_n db_t / (rho c); the normalisation follows from
 * (c^2 - a^2)(c^2 - c_a^2) = c_t^2 c^2.)  L is R^-1, formed here by Gauss-Jordan elimination. */
template <class T>
static void mhd_eigensystem(const T w[NW7], T bn, double gamma, T R[NW7][NW7], T lam[NW7]) {
  const T rho = w[IDN], v = w[IVN], p = w[IPR], bt1 = w[IBT1], bt2 = w[IBT2];
  const T a2 = gamma * p / rho;
  const T ca2 = bn * bn / rho;
  const T bt2sum = bt1 * bt1 + bt2 * bt2;
  const T ct2 = bt2sum / rho;
  const T tdif = ca2 + ct2 - a2;
  const T root = sqrt(tdif * tdif + 4.0 * a2 * ct2);  // c_f^2 - c_s^2
  const T cf2 = 0.5 * ((a2 + ca2 + ct2) + root);
  const T cs2 = a2 * ca2 / cf2;
  /* c_f^2 - a^2 = (tdif + root)/2 and c_f^2 - c_a^2 = (X + root)/2 with X = a^2 - c_a^2 + c_t^2, each
   * written without cancellation where its first term is negative ((root + x)(root - x) = 4 a^2 c_t^2,
   * resp. 4 c_a^2 c_t^2); a^2 - c_s^2 = a^2 (c_f^2 - c_a^2) / c_f^2.  The normalisation is then exact
   * where waves coincide (b_t = 0) and accurate near it. */
  const T X = a2 - ca2 + ct2;
  const T cf2_a2 = (tdif >= 0.0) ? 0.5 * (tdif + root) : 2.0 * a2 * ct2 / (root - tdif);
  const T cf2_ca2 = (X >= 0.0) ? 0.5 * (X + root) : 2.0 * ca2 * ct2 / (root - X);
  const T a2_cs2 = a2 * cf2_ca2 / cf2;
  const T a = sqrt(a2), ca = sqrt(ca2), cf = sqrt(cf2), cs = sqrt(cs2);
  T b1, b2;
  if (bt2sum == 0.0) {
    b1 = T(std::sqrt(0.5));
    b2 = T(std::sqrt(0.5));
  } else {
    const T bt = sqrt(bt2sum);
    b1 = bt1 / bt;
    b2 = bt2 / bt;
  }
  T af, as;
  if (root == 0.0) {  // c_f = c_s = a
    af = T(1.0);
    as = T(0.0);
  } else {
    af = sqrt(a2_cs2 / root);
    as = sqrt(cf2_a2 / root);
  }
  const double sg = (bn >= 0.0) ? 1.0 : -1.0;
  const T sr = sqrt(rho);
  const T Cf = cf * af, Cs = cs * as, Qf = sg * Cf, Qs = sg * Cs, Af = a * af * sr, As = a * as * sr;
  const T cols[NW7][NW7] = {
      {rho * af, -Cf, Qs * b1, Qs * b2, rho * a2 * af, As * b1, As * b2},       // v - c_f
      {T(0.0), T(0.0), -b2, b1, T(0.0), -sg * sr * b2, sg * sr * b1},           // v - c_a
      {rho * as, -Cs, -Qf * b1, -Qf * b2, rho * a2 * as, -Af * b1, -Af * b2},   // v - c_s
      {T(1.0), T(0.0), T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)},                 // v
      {rho * as, Cs, Qf * b1, Qf * b2, rho * a2 * as, -Af * b1, -Af * b2},      // v + c_s
      {T(0.0), T(0.0), -b2, b1, T(0.0), sg * sr * b2, -sg * sr * b1},           // v + c_a
      {rho * af, Cf, -Qs * b1, -Qs * b2, rho * a2 * af, As * b1, As * b2}};     // v + c_f
  for (int k = 0; k < NW7; ++k)
    for (int r = 0; r < NW7; ++r) R[r][k] = cols[k][r];
  const T sp[NW7] = {-cf, -ca, -cs, T(0.0), cs, ca, cf};
  for (int k = 0; k < NW7; ++k) lam[k] = v + sp[k];
}

/* Inverse of a 7 x 7 matrix by Gauss-Jordan elimination with partial pivoting. */
template <class T>
static void invert7(const T M[NW7][NW7], T Minv[NW7][NW7]) {
  T A[NW7][2 * NW7];
  for (int r = 0; r < NW7; ++r)
    for (int c = 0; c < NW7; ++c) {
      A[r][c] = M[r][c];
      A[r][NW7 + c] = T(r == c ? 1.0 : 0.0);
    }
  for (int c = 0; c < NW7; ++c) {
    int piv = c;
    for (int r = c + 1; r < NW7; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c)
      for (int q = 0; q < 2 * NW7; ++q) {
        const T t = A[c][q];
        A[c][q] = A[piv][q];
        A[piv][q] = t;
      }
    const T d = A[c][c];
    for (int q = 0; q < 2 * NW7; ++q) A[c][q] = A[c][q] / d;
    for (int r = 0; r < NW7; ++r) {
      if (r == c) continue;
      const T f = A[r][c];
      for (int q = 0; q < 2 * NW7; ++q) A[r][q] = A[r][q] - f * A[c][q];
    }
  }
  for (int r = 0; r < NW7; ++r)
    for (int c = 0; c < NW7; ++c) Minv[r][c] = A[r][NW7 + c];
}

/* Limited slope of the characteristic reconstruction for the cell with primitives q0 and normal field
 * bn between neighbours qm, qp [reading: the paper names the projection but prints its steps only by
 * reference]: C differences L (q0 - qm) and L (qp - q0) with L evaluated in the cell, the original van
 * Leer limiter on each characteristic field, and the limited slope projected back with R. */
template <class T>
static void char_slope(const T qm[NW7], const T q0[NW7], const T qp[NW7], T bn, double gamma, T dw[NW7]) {
  T R[NW7][NW7], L[NW7][NW7], lam[NW7];
  mhd_eigensystem(q0, bn, gamma, R, lam);
  invert7(R, L);
  T cm[NW7];
  for (int k = 0; k < NW7; ++k) {
    T cl = T(0.0), cr = T(0.0);
    for (int v = 0; v < NW7; ++v) {
      cl = cl + L[k][v] * (q0[v] - qm[v]);
      cr = cr + L[k][v] * (qp[v] - q0[v]);
    }
    cm[k] = vanleer_slope(-cl, T(0.0), cr);  // differences cl, cr
  }
  for (int v = 0; v < NW7; ++v) {
    T acc = T(0.0);
    for (int k = 0; k < NW7; ++k) acc = acc + R[v][k] * cm[k];
    dw[v] = acc;
  }
}

/* PPM edge values of the cell q[2] on characteristic variables [reading, as for char_slope]: the
 * differences q[j] - q[2] of the five-cell stencil projected with L of the cell, the PPM edge steps
 * (ppm_edges) on each characteristic field, and the two edges projected back with R.  ql / qr: the
 * primitive values at the cell's lower / upper face (before the range clamp). */
template <class T>
static void char_ppm_edges(const T q[5][NW7], T bn, double gamma, T ql[NW7], T qr[NW7]) {
  T R[NW7][NW7], L[NW7][NW7], lam[NW7];
  mhd_eigensystem(q[2], bn, gamma, R, lam);
  invert7(R, L);
  T cl[NW7], cr[NW7];
  for (int k = 0; k < NW7; ++k) {
    T c[5];
    for (int j = 0; j < 5; ++j) {
      T acc = T(0.0);
      for (int v = 0; v < NW7; ++v) acc = acc + L[k][v] * (q[j][v] - q[2][v]);
      c[j] = (j == 2) ? T(0.0) : acc;
    }
    ppm_edges(c, cl[k], cr[k]);
  }
  for (int v = 0; v < NW7; ++v) {
    T al = T(0.0), ar = T(0.0);
    for (int k = 0; k < NW7; ++k) {
      al = al + R[v][k] * cl[k];
      ar = ar + R[v][k] * cr[k];
    }
    ql[v] = q[2][v] + al;
    qr[v] = q[2][v] + ar;
  }
}

/* A primitive face value from the characteristic reconstruction, kept within the range of the two
 * cells sharing the face [reading: projecting back can leave that range, and density and pressure
 * must stay positive]. */
template <class T>
static T clamp_between(T x, T q1, T q2) {
  const T lo = vmin(q1, q2), hi = vmax(q1, q2);
  return vmin(vmax(x, lo), hi);
}

/* Upwind constrained-transport corner EMF (Gardiner & Stone 2005), for an edge whose two
 * transverse directions are "a" (first) and "b" (second), e.g. E_z at (i-1/2, j-1/2) with a = x,
 * b = y.  The corner value is the mean of the four face values plus one quarter of each of the two
 * upwinded second-difference corrections, obtained by integrating from each face centre to the
 * corner with the gradient taken in the upwind cell (sign of the face mass flux; mean of both cells
 * when the mass flux is exactly zero).
 *   ea[0], ea[1]: a-face EMFs at b-index j-1, j         (x-faces (i-1/2, j-1), (i-1/2, j))
 *   eb[0], eb[1]: b-face EMFs at a-index i-1, i         (y-faces (i-1, j-1/2), (i, j-1/2))
 *   ec[0..3]: cell-centre EMFs at (i-1,j-1), (i,j-1), (i-1,j), (i,j)
 *   ma[0], ma[1]: a-face mass fluxes at j-1, j;  mb[0], mb[1]: b-face mass fluxes at i-1, i. */
/* [option, not the paper's method] Smoothed upwind weight for the corner corrections: the gradient of
 * the cell on the side the mass flux m comes from gets the weight w = (1 + tanh(m / delta)) / 2, the
 * other cell's 1 - w.  w is 1/2 at m = 0 (the mean above) and tends to the upwind choice for
 * |m| >> delta; written w lo + (1 - w) hi, it equals the sharp choice bitwise where tanh saturates and
 * at m = 0.  delta = 0 is the sign switch itself.  For dual numbers the weight carries the tangent of m
 * (dw/dm = (1 - tanh^2) / (2 delta)): the smoothed corner is differentiable in the mass flux, the switch
 * is not. */
template <class T>
static T ct_smooth_pick(const T& m, double delta, const T& lo, const T& hi) {
  const T w = 0.5 * (1.0 + tanh(m / delta));
  return w * lo + (1.0 - w) * hi;
}

template <class T>
static T ct_corner(const T ea[2], const T eb[2], const T ec[4], const T ma[2], const T mb[2], double delta = 0.0) {
  const T sum4 = (ea[0] + ea[1]) + (eb[0] + eb[1]);
  if (delta > 0.0) {
    const T tlo = ct_smooth_pick(ma[0], delta, eb[0] - ec[0], eb[1] - ec[1]);
    const T thi = ct_smooth_pick(ma[1], delta, ec[2] - eb[0], ec[3] - eb[1]);
    const T slo = ct_smooth_pick(mb[0], delta, ea[0] - ec[0], ea[1] - ec[2]);
    const T shi = ct_smooth_pick(mb[1], delta, ec[1] - ea[0], ec[3] - ea[1]);
    return (0.25 * sum4 + 0.25 * (tlo - thi)) + 0.25 * (slo - shi);
  }
  /* gradient along b between the corner and the a-face below it, in the cell chosen by ma[0] */
  const T dlo_m = eb[0] - ec[0];  // cell i-1
  const T dlo_p = eb[1] - ec[1];  // cell i
  T tlo;
  if (ma[0] > 0.0)
    tlo = dlo_m;
  else if (ma[0] < 0.0)
    tlo = dlo_p;
  else
    tlo = 0.5 * (dlo_m + dlo_p);
  const T dhi_m = ec[2] - eb[0];
  const T dhi_p = ec[3] - eb[1];
  T thi;
  if (ma[1] > 0.0)
    thi = dhi_m;
  else if (ma[1] < 0.0)
    thi = dhi_p;
  else
    thi = 0.5 * (dhi_m + dhi_p);
  /* gradient along a between the corner and the b-face, in the cell chosen by the b-face mass flux */
  const T slo_m = ea[0] - ec[0];  // row j-1
  const T slo_p = ea[1] - ec[2];  // row j
  T slo;
  if (mb[0] > 0.0)
    slo = slo_m;
  else if (mb[0] < 0.0)
    slo = slo_p;
  else
    slo = 0.5 * (slo_m + slo_p);
  const T shi_m = ec[1] - ea[0];
  const T shi_p = ec[3] - ea[1];
  T shi;
  if (mb[1] > 0.0)
    shi = shi_m;
  else if (mb[1] < 0.0)
    shi = shi_p;
  else
    shi = 0.5 * (shi_m + shi_p);
  return (0.25 * sum4 + 0.25 * (tlo - thi)) + 0.25 * (slo - shi);
}

/* ---------------------------------------------------------------------------------------------
 * Mesh of equal-size MeshBlocks (Sec. 2.1)
 * ------------------------------------------------------------------------------------------- */

struct Params {
  int nx[3];  // global active cells
  int mb[3];  // MeshBlock active cells
  double xmin[3], xmax[3];
  double gamma;
  int riemann;
  int bc[6];  // x-, x+, y-, y+, z-, z+
  double dfloor, pfloor;
  int integrator;
  int recon;  // reconstruction of the higher-order stages: REC_PLM, REC_PPM, REC_PLM_CHAR or REC_PPM_CHAR
  int ng;     // ghost layers: 2 (DC, PLM) or 3 (PPM)
  int nscal;  // passive scalars (eq. passive_scalars)
  double ct_delta;  // smoothed CT upwind weight width (0: the paper's sign switch)
};

/* dense 3D array (k, j, i), i fastest */
template <class T> struct Arr3 {
  int n0 = 0, n1 = 0, n2 = 0;  // sizes in i, j, k
  std::vector<T> v;
  void init(int ni, int nj, int nk) {
    n0 = ni;
    n1 = nj;
    n2 = nk;
    v.assign((size_t)ni * nj * nk, T(0.0));
  }
  T& operator()(int k, int j, int i) { return v[((size_t)k * n1 + j) * n0 + i]; }
  const T& operator()(int k, int j, int i) const { return v[((size_t)k * n1 + j) * n0 + i]; }
};


template <class T> struct Block {
  int loc[3];
  Arr3<T> u[2][5];  // two registers of the cell-centred conserved variables (eq. rk-2s)
  Arr3<T> b[2][3];  // two registers of the face-centred field: b[.][0] on x-faces, ...
  Arr3<T> w[8];     // rho, vx, vy, vz, p, bcx, bcy, bcz
  Arr3<T> flx[3][NW7];  // fluxes on faces of direction d (component layout of the sweep)
  Arr3<T> emf[3];   // E1 on (j-1/2,k-1/2), E2 on (k-1/2,i-1/2), E3 on (i-1/2,j-1/2)
  std::vector<Arr3<T>> s[2];   // two registers of the passive-scalar masses rho C_i
  std::vector<Arr3<T>> cs;     // concentrations C_i (primitive)
  std::vector<Arr3<T>> fs[3];  // scalar fluxes on faces of direction d
  Arr3<T> acc[3];              // forcing acceleration a at the active cells (allocated when forcing is set)
};

template <class T> struct Mesh {
  Params P;
  int NG = 2;    // ghost layers (Sec. 2.1.1): 2 for second order, 3 for PPM
  int n[3];      // block active cells
  int nb[3];     // blocks per dim
  int c[3];      // cells with ghosts per dim
  double dx[3];
  std::vector<Block<T>> blk;
  long floor_events = 0;
  long emf_mismatch = 0;
  bool forced = false;  // a forcing acceleration field is set (source terms in every stage)

  int bid(int bx, int by, int bz) const { return (bz * nb[1] + by) * nb[0] + bx; }

  void init(const Params& p) {
    P = p;
    NG = p.ng;
    for (int d = 0; d < 3; ++d) {
      n[d] = p.mb[d];
      nb[d] = p.nx[d] / p.mb[d];
      c[d] = n[d] + 2 * NG;
      dx[d] = (p.xmax[d] - p.xmin[d]) / p.nx[d];
    }
    blk.resize((size_t)nb[0] * nb[1] * nb[2]);
    for (int bz = 0; bz < nb[2]; ++bz)
      for (int by = 0; by < nb[1]; ++by)
        for (int bx = 0; bx < nb[0]; ++bx) {
          Block<T>& B = blk[bid(bx, by, bz)];
          B.loc[0] = bx;
          B.loc[1] = by;
          B.loc[2] = bz;
          for (int r = 0; r < 2; ++r) {
            for (int v = 0; v < 5; ++v) B.u[r][v].init(c[0], c[1], c[2]);
            B.b[r][0].init(c[0] + 1, c[1], c[2]);
            B.b[r][1].init(c[0], c[1] + 1, c[2]);
            B.b[r][2].init(c[0], c[1], c[2] + 1);
          }
          for (int v = 0; v < 8; ++v) B.w[v].init(c[0], c[1], c[2]);
          for (int v = 0; v < NW7; ++v) {
            B.flx[0][v].init(c[0] + 1, c[1], c[2]);
            B.flx[1][v].init(c[0], c[1] + 1, c[2]);
            B.flx[2][v].init(c[0], c[1], c[2] + 1);
          }
          B.emf[0].init(c[0], c[1] + 1, c[2] + 1);
          B.emf[1].init(c[0] + 1, c[1], c[2] + 1);
          B.emf[2].init(c[0] + 1, c[1] + 1, c[2]);
          for (int r = 0; r < 2; ++r) {
            B.s[r].resize(p.nscal);
            for (auto& A : B.s[r]) A.init(c[0], c[1], c[2]);
          }
          B.cs.resize(p.nscal);
          for (auto& A : B.cs) A.init(c[0], c[1], c[2]);
          for (int d = 0; d < 3; ++d) {
            B.fs[d].resize(p.nscal);
            for (auto& A : B.fs[d]) A.init(c[0] + (d == 0), c[1] + (d == 1), c[2] + (d == 2));
          }
        }
  }

  /* Map a global index along dimension d that may lie outside [0, N) onto the cell (or face, when
   * `face` is set: valid range [0, N]) whose data fills it (Sec. 2.1.1): periodic wrap, or outflow =
   * nearest active cell / the boundary face. */
  int map_index(int d, int g, bool face) const {
    const int N = P.nx[d];
    if (g >= 0 && g < N) return g;
    if (face && g == N) return N;  // upper boundary face is an active face of the last block
    const bool lo = g < 0;
    const int bc = P.bc[2 * d + (lo ? 0 : 1)];
    if (bc == BC_PERIODIC) {
      int r = g % N;
      if (r < 0) r += N;
      return r;
    }
    if (face) return lo ? 0 : N;
    return lo ? 0 : N - 1;
  }

  /* Block and local index holding global cell (or face) index g along dimension d.  A face on the
   * boundary between two blocks is read from the block where it is the lower face; face N from the
   * last block's upper face. */
  void owner(int d, int g, bool face, int& b, int& l) const {
    if (face && g == P.nx[d]) {
      b = nb[d] - 1;
      l = n[d] + NG;
      return;
    }
    b = g / n[d];
    l = g - b * n[d] + NG;
  }

  /* Ghost exchange for one register (Sec. 2.1.1): cell-centred U and face-centred B, depth N_G,
   * 26 neighbours.  Faces on a block's own surface are active and are not overwritten. */
  void fill_ghosts(int r) {
#pragma omp parallel for schedule(static)
    for (size_t ib = 0; ib < blk.size(); ++ib) {
      Block<T>& B = blk[ib];
      for (int k = 0; k < c[2]; ++k)
        for (int j = 0; j < c[1]; ++j)
          for (int i = 0; i < c[0]; ++i) {
            const int li[3] = {i, j, k};
            bool ghost = false;
            for (int d = 0; d < 3; ++d)
              if (li[d] < NG || li[d] >= n[d] + NG) ghost = true;
            if (!ghost) continue;
            int sb[3], sl[3];
            for (int d = 0; d < 3; ++d) {
              const int g = map_index(d, B.loc[d] * n[d] + li[d] - NG, false);
              owner(d, g, false, sb[d], sl[d]);
            }
            const Block<T>& S = blk[bid(sb[0], sb[1], sb[2])];
            for (int v = 0; v < 5; ++v) B.u[r][v](k, j, i) = S.u[r][v](sl[2], sl[1], sl[0]);
            for (int q = 0; q < P.nscal; ++q) B.s[r][q](k, j, i) = S.s[r][q](sl[2], sl[1], sl[0]);
          }
      for (int fd = 0; fd < 3; ++fd) {
        Arr3<T>& A = B.b[r][fd];
        for (int k = 0; k < A.n2; ++k)
          for (int j = 0; j < A.n1; ++j)
            for (int i = 0; i < A.n0; ++i) {
              const int li[3] = {i, j, k};
              bool ghost = false;
              for (int d = 0; d < 3; ++d) {
                const int hi = (d == fd) ? n[d] + NG : n[d] + NG - 1;
                if (li[d] < NG || li[d] > hi) ghost = true;
              }
              if (!ghost) continue;
              int sb[3], sl[3];
              for (int d = 0; d < 3; ++d) {
                const bool face = (d == fd);
                const int g = map_index(d, B.loc[d] * n[d] + li[d] - NG, face);
                owner(d, g, face, sb[d], sl[d]);
              }
              A(k, j, i) = blk[bid(sb[0], sb[1], sb[2])].b[r][fd](sl[2], sl[1], sl[0]);
            }
      }
    }
  }

  /* cons -> prim for every cell of every block, ghosts included (Sec. 3.1):
   * b_c = mean of the two face values [reading: uniform-grid face average], v = M / rho,
   * p = (gamma-1)(E - |M|^2/(2 rho) - |b_c|^2/2).  [reading] Floors: rho < dfloor -> dfloor and
   * p < pfloor -> pfloor; an active cell whose floor fires has U rewritten to match, and the
   * event is counted. */
  void cons_to_prim(int r) {
    const double gm1 = P.gamma - 1.0;
    long fired_total = 0;
#pragma omp parallel for schedule(static) reduction(+ : fired_total)
    for (size_t ib = 0; ib < blk.size(); ++ib) {
      Block<T>& B = blk[ib];
      for (int k = 0; k < c[2]; ++k)
        for (int j = 0; j < c[1]; ++j)
          for (int i = 0; i < c[0]; ++i) {
            const T bcx = 0.5 * (B.b[r][0](k, j, i) + B.b[r][0](k, j, i + 1));
            const T bcy = 0.5 * (B.b[r][1](k, j, i) + B.b[r][1](k, j + 1, i));
            const T bcz = 0.5 * (B.b[r][2](k, j, i) + B.b[r][2](k + 1, j, i));
            T d = B.u[r][0](k, j, i);
            const T m1 = B.u[r][1](k, j, i), m2 = B.u[r][2](k, j, i), m3 = B.u[r][3](k, j, i);
            T e = B.u[r][4](k, j, i);
            const bool active = i >= NG && i < n[0] + NG && j >= NG && j < n[1] + NG && k >= NG &&
                                k < n[2] + NG;
            bool fired = false;
            if (d < P.dfloor) {
              d = T(P.dfloor);
              fired = true;
            }
            const T vx = m1 / d, vy = m2 / d, vz = m3 / d;
            const T ke = 0.5 * ((m1 * m1 + m2 * m2) + m3 * m3) / d;
            const T me = 0.5 * ((bcx * bcx + bcy * bcy) + bcz * bcz);
            T p = gm1 * (e - ke - me);
            if (p < P.pfloor) {
              p = T(P.pfloor);
              e = p / gm1 + ke + me;
              fired = true;
            }
            if (fired && active) {
              ++fired_total;
              B.u[r][0](k, j, i) = d;
              B.u[r][4](k, j, i) = e;
            }
            B.w[0](k, j, i) = d;
            B.w[1](k, j, i) = vx;
            B.w[2](k, j, i) = vy;
            B.w[3](k, j, i) = vz;
            B.w[4](k, j, i) = p;
            B.w[5](k, j, i) = bcx;
            B.w[6](k, j, i) = bcy;
            B.w[7](k, j, i) = bcz;
            for (int q = 0; q < P.nscal; ++q) B.cs[q](k, j, i) = B.s[r][q](k, j, i) / d;
          }
    }
    floor_events += fired_total;
  }

  /* 7-component interface state of cell (k,j,i) for a sweep in direction d: (rho, v_n, v_t1, v_t2,
   * p, b_t1, b_t2) with (n, t1, t2) = (d, d+1, d+2) mod 3. */
  void cell_state(const Block<T>& B, int d, int k, int j, int i, T q[NW7]) const {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    q[IDN] = B.w[0](k, j, i);
    q[IVN] = B.w[1 + d](k, j, i);
    q[IVT1] = B.w[1 + t1](k, j, i);
    q[IVT2] = B.w[1 + t2](k, j, i);
    q[IPR] = B.w[4](k, j, i);
    q[IBT1] = B.w[5 + t1](k, j, i);
    q[IBT2] = B.w[5 + t2](k, j, i);
  }

  /* Fluxes on every face a block needs: faces of direction d from the block's lower to its upper
   * surface, over the active cells plus one ghost layer in the two transverse directions (these
   * feed the corner EMFs on the block surface).  Donor cell: W_L = W_{i-1}, W_R = W_i; PLM: face
   * values of the van Leer limited linear profiles; PPM: the right edge of cell i-1 and the left edge
   * of cell i (Sec. 3.2.1). */
  void compute_fluxes(Block<T>& B, int recon) {
    for (int d = 0; d < 3; ++d) {
      int lo[3], hi[3];
      for (int e = 0; e < 3; ++e) {
        lo[e] = (e == d) ? NG : NG - 1;
        hi[e] = (e == d) ? n[e] + NG : n[e] + NG;  // inclusive
      }
      const int sh[3] = {d == 0, d == 1, d == 2};
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            T qm2[NW7], qm1[NW7], q0[NW7], qp1[NW7];
            cell_state(B, d, k - sh[2], j - sh[1], i - sh[0], qm1);
            cell_state(B, d, k, j, i, q0);
            T wl[NW7], wr[NW7];
            if (recon == REC_DC) {
              for (int v = 0; v < NW7; ++v) {
                wl[v] = qm1[v];
                wr[v] = q0[v];
              }
            } else if (recon == REC_PPM) {
              T qs[6][NW7];  // q_{i-3} .. q_{i+2} along d
              for (int o = -3; o <= 2; ++o)
                cell_state(B, d, k + o * sh[2], j + o * sh[1], i + o * sh[0], qs[o + 3]);
              for (int v = 0; v < NW7; ++v) {
                const T lo5[5] = {qs[0][v], qs[1][v], qs[2][v], qs[3][v], qs[4][v]};
                const T hi5[5] = {qs[1][v], qs[2][v], qs[3][v], qs[4][v], qs[5][v]};
                T ql, qr;
                ppm_edges(lo5, ql, qr);  // cell i-1
                wl[v] = qr;
                ppm_edges(hi5, ql, qr);  // cell i
                wr[v] = ql;
              }
            } else if (recon == REC_PPM_CHAR) {
              T qs[6][NW7];  // q_{i-3} .. q_{i+2} along d
              for (int o = -3; o <= 2; ++o)
                cell_state(B, d, k + o * sh[2], j + o * sh[1], i + o * sh[0], qs[o + 3]);
              T a[NW7], b2[NW7];
              char_ppm_edges(&qs[0], B.w[5 + d](k - sh[2], j - sh[1], i - sh[0]), P.gamma, a, b2);  // cell i-1
              for (int v = 0; v < NW7; ++v) wl[v] = clamp_between(b2[v], qs[2][v], qs[3][v]);
              char_ppm_edges(&qs[1], B.w[5 + d](k, j, i), P.gamma, a, b2);  // cell i
              for (int v = 0; v < NW7; ++v) wr[v] = clamp_between(a[v], qs[2][v], qs[3][v]);
            } else if (recon == REC_PLM_CHAR) {
              cell_state(B, d, k - 2 * sh[2], j - 2 * sh[1], i - 2 * sh[0], qm2);
              cell_state(B, d, k + sh[2], j + sh[1], i + sh[0], qp1);
              T dlm[NW7], dl0[NW7];
              char_slope(qm2, qm1, q0, B.w[5 + d](k - sh[2], j - sh[1], i - sh[0]), P.gamma, dlm);
              char_slope(qm1, q0, qp1, B.w[5 + d](k, j, i), P.gamma, dl0);
              for (int v = 0; v < NW7; ++v) {
                wl[v] = clamp_between(qm1[v] + 0.5 * dlm[v], qm1[v], q0[v]);
                wr[v] = clamp_between(q0[v] - 0.5 * dl0[v], qm1[v], q0[v]);
              }
            } else {
              cell_state(B, d, k - 2 * sh[2], j - 2 * sh[1], i - 2 * sh[0], qm2);
              cell_state(B, d, k + sh[2], j + sh[1], i + sh[0], qp1);
              for (int v = 0; v < NW7; ++v) {
                const T dlm = vanleer_slope(qm2[v], qm1[v], q0[v]);
                const T dl0 = vanleer_slope(qm1[v], q0[v], qp1[v]);
                wl[v] = qm1[v] + 0.5 * dlm;
                wr[v] = q0[v] - 0.5 * dl0;
              }
            }
            T f[NW7];
            riemann(P.riemann, wl, wr, B.b[0][d](k, j, i), P.gamma, f);
            for (int v = 0; v < NW7; ++v) B.flx[d][v](k, j, i) = f[v];
            /* passive scalars: C reconstructed like the primitives, carried by the mass flux from the
             * upwind side, F = F_rho C_L if F_rho >= 0, else F_rho C_R  [reading] */
            for (int q = 0; q < P.nscal; ++q) {
              const Arr3<T>& C = B.cs[q];
              auto at = [&](int o) { return C(k + o * sh[2], j + o * sh[1], i + o * sh[0]); };
              T cl, cr;
              if (recon == REC_DC) {
                cl = at(-1);
                cr = at(0);
              } else if (recon == REC_PPM || recon == REC_PPM_CHAR) {
                const T lo5[5] = {at(-3), at(-2), at(-1), at(0), at(1)};
                const T hi5[5] = {at(-2), at(-1), at(0), at(1), at(2)};
                T a, b2;
                ppm_edges(lo5, a, b2);
                cl = b2;
                ppm_edges(hi5, a, b2);
                cr = a;
              } else {
                cl = at(-1) + 0.5 * vanleer_slope(at(-2), at(-1), at(0));
                cr = at(0) - 0.5 * vanleer_slope(at(-1), at(0), at(1));
              }
              B.fs[d][q](k, j, i) = (f[IDN] >= 0.0) ? f[IDN] * cl : f[IDN] * cr;
            }
          }
    }
  }

  /* cell-centre EMF component e (0: E1, 1: E2, 2: E3) from E = -v x b_c */
  T cell_emf(const Block<T>& B, int e, int k, int j, int i) const {
    const T vx = B.w[1](k, j, i), vy = B.w[2](k, j, i), vz = B.w[3](k, j, i);
    const T bx = B.w[5](k, j, i), by = B.w[6](k, j, i), bz = B.w[7](k, j, i);
    if (e == 0) return vz * by - vy * bz;
    if (e == 1) return vx * bz - vz * bx;
    return vy * bx - vx * by;
  }

  /* Corner EMFs on every edge of the block's active region (Sec. 2.1.1 / upwind CT).  Edge
   * direction e, first transverse direction a = e+1, second b = e+2.  The face EMF of the same
   * component is -F_a[b_t1] on a-faces and +F_b[b_t2] on b-faces (E = -v x B). */
  void compute_emfs(Block<T>& B) {
    for (int e = 0; e < 3; ++e) {
      const int a = (e + 1) % 3, b = (e + 2) % 3;
      int lo[3], hi[3];
      for (int q = 0; q < 3; ++q) {
        lo[q] = NG;
        hi[q] = (q == e) ? n[q] + NG - 1 : n[q] + NG;
      }
      int sa[3] = {0, 0, 0}, sb[3] = {0, 0, 0};
      sa[a] = 1;
      sb[b] = 1;
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            /* edge at (a-1/2, b-1/2) of cell (k,j,i) */
            const int km_b = k - sb[2], jm_b = j - sb[1], im_b = i - sb[0];  // one step down in b
            const int km_a = k - sa[2], jm_a = j - sa[1], im_a = i - sa[0];  // one step down in a
            const int kmm = k - sa[2] - sb[2], jmm = j - sa[1] - sb[1], imm = i - sa[0] - sb[0];
            T ea[2], eb[2], ec[4], ma[2], mb[2];
            ea[0] = -B.flx[a][IBT1](km_b, jm_b, im_b);
            ea[1] = -B.flx[a][IBT1](k, j, i);
            eb[0] = B.flx[b][IBT2](km_a, jm_a, im_a);
            eb[1] = B.flx[b][IBT2](k, j, i);
            ma[0] = B.flx[a][IDN](km_b, jm_b, im_b);
            ma[1] = B.flx[a][IDN](k, j, i);
            mb[0] = B.flx[b][IDN](km_a, jm_a, im_a);
            mb[1] = B.flx[b][IDN](k, j, i);
            ec[0] = cell_emf(B, e, kmm, jmm, imm);    // (a-1, b-1)
            ec[1] = cell_emf(B, e, km_b, jm_b, im_b); // (a,   b-1)
            ec[2] = cell_emf(B, e, km_a, jm_a, im_a); // (a-1, b)
            ec[3] = cell_emf(B, e, k, j, i);          // (a,   b)
            B.emf[e](k, j, i) = ct_corner(ea, eb, ec, ma, mb, P.ct_delta);
          }
    }
  }

  /* Fluxes then corner EMFs of every block; blocks are independent (each owns its arrays). */
  void all_fluxes_and_emfs(int recon) {
#pragma omp parallel for schedule(static)
    for (size_t ib = 0; ib < blk.size(); ++ib) {
      compute_fluxes(blk[ib], recon);
      compute_emfs(blk[ib]);
    }
  }

  /* Shared-edge EMF averaging (Sec. 2.1.1): every edge held by more than one MeshBlock (or twice by
   * one block through periodic wrap) gets the mean of all its copies, formed as
   * first + sum(copy - first) / count so that equal copies average to themselves exactly.  Copies
   * that differ from the first are counted. */
  void average_shared_emfs() {
    for (int e = 0; e < 3; ++e) {
      int gdim[3];
      for (int q = 0; q < 3; ++q) gdim[q] = (q == e) ? P.nx[q] : P.nx[q] + 1;
      const size_t ng = (size_t)gdim[0] * gdim[1] * gdim[2];
      std::vector<T> ref(ng, T(0.0)), acc(ng, T(0.0));
      std::vector<int> cnt(ng, 0);
      for (int pass = 0; pass < 2; ++pass)
        for (auto& B : blk) {
          Arr3<T>& A = B.emf[e];
          for (int k = NG; k <= ((e == 2) ? n[2] + NG - 1 : n[2] + NG); ++k)
            for (int j = NG; j <= ((e == 1) ? n[1] + NG - 1 : n[1] + NG); ++j)
              for (int i = NG; i <= ((e == 0) ? n[0] + NG - 1 : n[0] + NG); ++i) {
                const int li[3] = {i, j, k};
                int g[3];
                for (int q = 0; q < 3; ++q) {
                  g[q] = B.loc[q] * n[q] + li[q] - NG;
                  if (q != e && g[q] == P.nx[q] && P.bc[2 * q + 1] == BC_PERIODIC) g[q] = 0;
                }
                const size_t gi = ((size_t)g[2] * gdim[1] + g[1]) * gdim[0] + g[0];
                if (pass == 0) {
                  if (cnt[gi] == 0) {
                    ref[gi] = A(k, j, i);
                  } else {
                    if (!(A(k, j, i) == ref[gi])) ++emf_mismatch;
                    acc[gi] = acc[gi] + (A(k, j, i) - ref[gi]);
                  }
                  ++cnt[gi];
                } else if (cnt[gi] > 1) {
                  A(k, j, i) = ref[gi] + acc[gi] / (double)cnt[gi];
                }
              }
        }
    }
  }

  /* 2S register update of one stage (eq. rk-2s):
   *   u1 <- u1 + delta_s u0 ;  u0 <- g0 u0 + g1 u1 + beta dt L(u0)
   * with L = -div F for the cell-centred variables and L = -curl E for the face field.
   * [reading: forcing] With a forcing acceleration a(x) set, L of the cell-centred variables also holds the
   * source terms of a body force on the stage state u0: rho a in the momentum and M . a in the energy
   * (the work of the force), L = -div F + S(u0).  The paper defines no forcing; this is the body-force form
   * of the momentum and energy equations, added in every stage like the flux divergence. */
  void register_update(double delta, double g0, double g1, double beta, double dt) {
#pragma omp parallel for schedule(static)
    for (size_t ib = 0; ib < blk.size(); ++ib) {
      Block<T>& B = blk[ib];
      for (int v = 0; v < 5; ++v)
        for (int k = NG; k < n[2] + NG; ++k)
          for (int j = NG; j < n[1] + NG; ++j)
            for (int i = NG; i < n[0] + NG; ++i) B.u[1][v](k, j, i) = B.u[1][v](k, j, i) + delta * B.u[0][v](k, j, i);
      for (int fd = 0; fd < 3; ++fd) {
        Arr3<T>& A1 = B.b[1][fd];
        Arr3<T>& A0 = B.b[0][fd];
        for (int k = NG; k <= n[2] + NG - (fd == 2 ? 0 : 1); ++k)
          for (int j = NG; j <= n[1] + NG - (fd == 1 ? 0 : 1); ++j)
            for (int i = NG; i <= n[0] + NG - (fd == 0 ? 0 : 1); ++i) A1(k, j, i) = A1(k, j, i) + delta * A0(k, j, i);
      }
      for (int q = 0; q < P.nscal; ++q)
        for (int k = NG; k < n[2] + NG; ++k)
          for (int j = NG; j < n[1] + NG; ++j)
            for (int i = NG; i < n[0] + NG; ++i) B.s[1][q](k, j, i) = B.s[1][q](k, j, i) + delta * B.s[0][q](k, j, i);
      const double h = beta * dt;
      /* passive scalars, with the association of the conserved variables below */
      for (int q = 0; q < P.nscal; ++q)
        for (int k = NG; k < n[2] + NG; ++k)
          for (int j = NG; j < n[1] + NG; ++j)
            for (int i = NG; i < n[0] + NG; ++i) {
              T dfl[3];
              for (int d = 0; d < 3; ++d) {
                const int ip = i + (d == 0), jp = j + (d == 1), kp = k + (d == 2);
                dfl[d] = (B.fs[d][q](kp, jp, ip) - B.fs[d][q](k, j, i)) / dx[d];
              }
              const T L = -((dfl[0] + dfl[1]) + dfl[2]);
              B.s[0][q](k, j, i) = (g0 * B.s[0][q](k, j, i) + g1 * B.s[1][q](k, j, i)) + h * L;
            }
      /* cell-centred: conserved variable v <- flux component (rho, M_n..., E) */
      for (int k = NG; k < n[2] + NG; ++k)
        for (int j = NG; j < n[1] + NG; ++j)
          for (int i = NG; i < n[0] + NG; ++i) {
            /* body-force source of the stage state (before u0 is overwritten below) */
            T src[5] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
            if (forced) {
              const T rho = B.u[0][0](k, j, i);
              const T ax = B.acc[0](k, j, i), ay = B.acc[1](k, j, i), az = B.acc[2](k, j, i);
              src[1] = rho * ax;
              src[2] = rho * ay;
              src[3] = rho * az;
              src[4] = (B.u[0][1](k, j, i) * ax + B.u[0][2](k, j, i) * ay) + B.u[0][3](k, j, i) * az;
            }
            for (int v = 0; v < 5; ++v) {
              T dfl[3];
              for (int d = 0; d < 3; ++d) {
                /* flux component carrying conserved variable v in a sweep along d */
                int comp;
                if (v == 0)
                  comp = IDN;
                else if (v == 4)
                  comp = IPR;
                else {
                  const int mdir = v - 1;  // momentum component x/y/z
                  if (mdir == d)
                    comp = IVN;
                  else if (mdir == (d + 1) % 3)
                    comp = IVT1;
                  else
                    comp = IVT2;
                }
                const int ip = i + (d == 0), jp = j + (d == 1), kp = k + (d == 2);
                dfl[d] = (B.flx[d][comp](kp, jp, ip) - B.flx[d][comp](k, j, i)) / dx[d];
              }
              const T L = forced ? -((dfl[0] + dfl[1]) + dfl[2]) + src[v] : -((dfl[0] + dfl[1]) + dfl[2]);
              B.u[0][v](k, j, i) = (g0 * B.u[0][v](k, j, i) + g1 * B.u[1][v](k, j, i)) + h * L;
            }
          }
      /* face field: B1 on x-faces uses E3 (along y) and E2 (along z), cyclically */
      for (int fd = 0; fd < 3; ++fd) {
        const int a = (fd + 1) % 3, b = (fd + 2) % 3;  // B_fd: -[(dE_b/d a) - (dE_a/d b)]
        Arr3<T>& A0 = B.b[0][fd];
        Arr3<T>& A1 = B.b[1][fd];
        for (int k = NG; k <= n[2] + NG - (fd == 2 ? 0 : 1); ++k)
          for (int j = NG; j <= n[1] + NG - (fd == 1 ? 0 : 1); ++j)
            for (int i = NG; i <= n[0] + NG - (fd == 0 ? 0 : 1); ++i) {
              const int ia = i + (a == 0), ja = j + (a == 1), ka = k + (a == 2);
              const int ib = i + (b == 0), jb = j + (b == 1), kb = k + (b == 2);
              const T curl = (B.emf[b](ka, ja, ia) - B.emf[b](k, j, i)) / dx[a] -
                             (B.emf[a](kb, jb, ib) - B.emf[a](k, j, i)) / dx[b];
              const T L = -curl;
              A0(k, j, i) = (g0 * A0(k, j, i) + g1 * A1(k, j, i)) + h * L;
            }
      }
    }
  }

  /* One cycle of a 2S integrator (eq. rk-2s, Sec. 3.2.3).  VL2: gamma_0 = {0,1}, beta_0 = 1/2 with
   * donor-cell fluxes in the predictor; gamma_1 = {0,1}, beta_1 = 1 with PLM fluxes. */
  void step(double dt) {
    struct Stage { double delta, g0, g1, beta; int recon; };
    std::vector<Stage> st;
    switch (P.integrator) {
      case INT_RK1: st = {{1.0, 0.0, 1.0, 1.0, REC_DC}}; break;
      case INT_RK2: st = {{1.0, 0.0, 1.0, 1.0, P.recon}, {0.0, 0.5, 0.5, 0.5, P.recon}}; break;
      case INT_RK3:
        st = {{1.0, 0.0, 1.0, 1.0, P.recon}, {0.0, 0.25, 0.75, 0.25, P.recon}, {0.0, 2.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, P.recon}};
        break;
      default: st = {{1.0, 0.0, 1.0, 0.5, REC_DC}, {0.0, 0.0, 1.0, 1.0, P.recon}}; break;
    }
    /* u1 <- 0 at the start of every cycle */
    for (auto& B : blk) {
      for (int v = 0; v < 5; ++v) std::fill(B.u[1][v].v.begin(), B.u[1][v].v.end(), T(0.0));
      for (int fd = 0; fd < 3; ++fd) std::fill(B.b[1][fd].v.begin(), B.b[1][fd].v.end(), T(0.0));
      for (auto& A : B.s[1]) std::fill(A.v.begin(), A.v.end(), T(0.0));
    }
    for (const Stage& s : st) {
      cons_to_prim(0);
      all_fluxes_and_emfs(s.recon);
      average_shared_emfs();
      register_update(s.delta, s.g0, s.g1, s.beta, dt);
      fill_ghosts(0);
    }
  }

  /* Fluxes and EMFs of the current state for one reconstruction, without updating (debug view). */
  void stage_terms(int recon) {
    cons_to_prim(0);
    all_fluxes_and_emfs(recon);
    average_shared_emfs();
  }

  /* Time step (Sec. 2.1.7, Sec. 3.2.3): dt = C0 min over active cells and directions of
   * dx_d / (|v_d| + C_f,d).  [reading] per-direction fast speed with b_c,d as the normal field. */
  double new_dt(double cfl) {
    cons_to_prim(0);
    double best = 1e300;
    for (auto& B : blk)
      for (int k = NG; k < n[2] + NG; ++k)
        for (int j = NG; j < n[1] + NG; ++j)
          for (int i = NG; i < n[0] + NG; ++i)
            for (int d = 0; d < 3; ++d) {
              const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
              const T cf = fast_speed(B.w[0](k, j, i), B.w[4](k, j, i), B.w[5 + d](k, j, i), B.w[5 + t1](k, j, i),
                                      B.w[5 + t2](k, j, i), P.gamma);
              const T dtd = dx[d] / (fabs(B.w[1 + d](k, j, i)) + cf);
              const double v = value_of(dtd);
              if (v < best) best = v;
            }
    return cfl * best;
  }

  static double value_of(double x) { return x; }
  static double value_of(Dual x) { return x.v; }
};

/* ---------------------------------------------------------------------------------------------
 * Global-array I/O (active region, [var][k][j][i])
 * ------------------------------------------------------------------------------------------- */

template <class T>
static void set_prims(Mesh<T>& M, const double* w, const double* b1, const double* b2, const double* b3) {
  const int NG = M.NG;
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (auto& B : M.blk) {
    const int o[3] = {B.loc[0] * M.n[0], B.loc[1] * M.n[1], B.loc[2] * M.n[2]};
    for (int k = 0; k <= M.n[2]; ++k)
      for (int j = 0; j <= M.n[1]; ++j)
        for (int i = 0; i <= M.n[0]; ++i) {
          const int gi = o[0] + i, gj = o[1] + j, gk = o[2] + k;
          if (j < M.n[1] && k < M.n[2])
            B.b[0][0](k + NG, j + NG, i + NG) = b1[((size_t)gk * NY + gj) * (NX + 1) + gi];
          if (i < M.n[0] && k < M.n[2])
            B.b[0][1](k + NG, j + NG, i + NG) = b2[((size_t)gk * (NY + 1) + gj) * NX + gi];
          if (i < M.n[0] && j < M.n[1])
            B.b[0][2](k + NG, j + NG, i + NG) = b3[((size_t)gk * NY + gj) * NX + gi];
        }
  }
  const double gm1 = M.P.gamma - 1.0;
  for (auto& B : M.blk) {
    const int o[3] = {B.loc[0] * M.n[0], B.loc[1] * M.n[1], B.loc[2] * M.n[2]};
    for (int k = 0; k < M.n[2]; ++k)
      for (int j = 0; j < M.n[1]; ++j)
        for (int i = 0; i < M.n[0]; ++i) {
          const size_t g = ((size_t)(o[2] + k) * NY + (o[1] + j)) * NX + (o[0] + i);
          const T d = w[0 * ncell + g], vx = w[1 * ncell + g], vy = w[2 * ncell + g], vz = w[3 * ncell + g];
          const T p = w[4 * ncell + g];
          const int K = k + NG, J = j + NG, I = i + NG;
          const T bcx = 0.5 * (B.b[0][0](K, J, I) + B.b[0][0](K, J, I + 1));
          const T bcy = 0.5 * (B.b[0][1](K, J, I) + B.b[0][1](K, J + 1, I));
          const T bcz = 0.5 * (B.b[0][2](K, J, I) + B.b[0][2](K + 1, J, I));
          B.u[0][0](K, J, I) = d;
          B.u[0][1](K, J, I) = d * vx;
          B.u[0][2](K, J, I) = d * vy;
          B.u[0][3](K, J, I) = d * vz;
          B.u[0][4](K, J, I) = p / gm1 + 0.5 * d * ((vx * vx + vy * vy) + vz * vz) + 0.5 * ((bcx * bcx + bcy * bcy) + bcz * bcz);
        }
  }
  M.fill_ghosts(0);
}

template <class T>
static void get_cons(const Mesh<T>& M, double* u, double* b1, double* b2, double* b3) {
  const int NG = M.NG;
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (const auto& B : M.blk) {
    const int o[3] = {B.loc[0] * M.n[0], B.loc[1] * M.n[1], B.loc[2] * M.n[2]};
    for (int k = 0; k <= M.n[2]; ++k)
      for (int j = 0; j <= M.n[1]; ++j)
        for (int i = 0; i <= M.n[0]; ++i) {
          const int gi = o[0] + i, gj = o[1] + j, gk = o[2] + k;
          const int K = k + NG, J = j + NG, I = i + NG;
          const bool own_i = (i < M.n[0]) || (gi == NX);
          const bool own_j = (j < M.n[1]) || (gj == NY);
          const bool own_k = (k < M.n[2]) || (gk == NZ);
          if (u && i < M.n[0] && j < M.n[1] && k < M.n[2]) {
            const size_t g = ((size_t)gk * NY + gj) * NX + gi;
            for (int v = 0; v < 5; ++v) u[v * ncell + g] = Mesh<T>::value_of(B.u[0][v](K, J, I));
          }
          if (b1 && own_i && j < M.n[1] && k < M.n[2])
            b1[((size_t)gk * NY + gj) * (NX + 1) + gi] = Mesh<T>::value_of(B.b[0][0](K, J, I));
          if (b2 && own_j && i < M.n[0] && k < M.n[2])
            b2[((size_t)gk * (NY + 1) + gj) * NX + gi] = Mesh<T>::value_of(B.b[0][1](K, J, I));
          if (b3 && own_k && i < M.n[0] && j < M.n[1])
            b3[((size_t)gk * NY + gj) * NX + gi] = Mesh<T>::value_of(B.b[0][2](K, J, I));
        }
  }
}

/* Set the conserved state directly from global arrays (active region), then exchange ghosts. */
template <class T>
static void set_cons(Mesh<T>& M, const double* u, const double* du, const double* b1, const double* db1,
                     const double* b2, const double* db2, const double* b3, const double* db3) {
  const int NG = M.NG;
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (auto& B : M.blk) {
    const int o[3] = {B.loc[0] * M.n[0], B.loc[1] * M.n[1], B.loc[2] * M.n[2]};
    for (int k = 0; k <= M.n[2]; ++k)
      for (int j = 0; j <= M.n[1]; ++j)
        for (int i = 0; i <= M.n[0]; ++i) {
          const int gi = o[0] + i, gj = o[1] + j, gk = o[2] + k;
          const int K = k + NG, J = j + NG, I = i + NG;
          if (j < M.n[1] && k < M.n[2]) {
            const size_t f = ((size_t)gk * NY + gj) * (NX + 1) + gi;
            B.b[0][0](K, J, I) = make_scalar<T>(b1[f], db1 ? db1[f] : 0.0);
          }
          if (i < M.n[0] && k < M.n[2]) {
            const size_t f = ((size_t)gk * (NY + 1) + gj) * NX + gi;
            B.b[0][1](K, J, I) = make_scalar<T>(b2[f], db2 ? db2[f] : 0.0);
          }
          if (i < M.n[0] && j < M.n[1]) {
            const size_t f = ((size_t)gk * NY + gj) * NX + gi;
            B.b[0][2](K, J, I) = make_scalar<T>(b3[f], db3 ? db3[f] : 0.0);
          }
          if (i < M.n[0] && j < M.n[1] && k < M.n[2]) {
            const size_t g = ((size_t)gk * NY + gj) * NX + gi;
            for (int v = 0; v < 5; ++v)
              B.u[0][v](K, J, I) = make_scalar<T>(u[v * ncell + g], du ? du[v * ncell + g] : 0.0);
          }
        }
  }
  M.fill_ghosts(0);
}

/* Tangent parts of the conserved state (global layout), the counterpart of get_cons. */
static void get_tangent(const Mesh<Dual>& M, double* du, double* db1, double* db2, double* db3) {
  const int NG = M.NG;
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (const auto& B : M.blk) {
    const int o[3] = {B.loc[0] * M.n[0], B.loc[1] * M.n[1], B.loc[2] * M.n[2]};
    for (int k = 0; k <= M.n[2]; ++k)
      for (int j = 0; j <= M.n[1]; ++j)
        for (int i = 0; i <= M.n[0]; ++i) {
          const int gi = o[0] + i, gj = o[1] + j, gk = o[2] + k;
          const int K = k + NG, J = j + NG, I = i + NG;
          const bool own_i = (i < M.n[0]) || (gi == NX);
          const bool own_j = (j < M.n[1]) || (gj == NY);
          const bool own_k = (k < M.n[2]) || (gk == NZ);
          if (i < M.n[0] && j < M.n[1] && k < M.n[2]) {
            const size_t g = ((size_t)gk * NY + gj) * NX + gi;
            for (int v = 0; v < 5; ++v) du[v * ncell + g] = B.u[0][v](K, J, I).d;
          }
          if (own_i && j < M.n[1] && k < M.n[2]) db1[((size_t)gk * NY + gj) * (NX + 1) + gi] = B.b[0][0](K, J, I).d;
          if (own_j && i < M.n[0] && k < M.n[2]) db2[((size_t)gk * (NY + 1) + gj) * NX + gi] = B.b[0][1](K, J, I).d;
          if (own_k && i < M.n[0] && j < M.n[1]) db3[((size_t)gk * NY + gj) * NX + gi] = B.b[0][2](K, J, I).d;
        }
  }
}

}  // namespace orc

/* =============================================================================================
 * C interface (ctypes)
 * =========================================================================================== */
using orc::Mesh;

extern "C" {

void* orc_mesh_new(const int* nx, const int* mb, const double* xmin, const double* xmax, double gamma,
                   int riemann, const int* bc, double dfloor, double pfloor, int integrator, int recon, int ng,
                   int nscal, double ct_delta) {
  orc::Params p;
  if (!(ct_delta >= 0.0) || !std::isfinite(ct_delta)) return nullptr;
  p.ct_delta = ct_delta;
  if (recon < orc::REC_PLM || recon > orc::REC_PPM_CHAR) return nullptr;
  if (nscal < 0 || nscal > 16) return nullptr;
  p.nscal = nscal;
  if (ng < 2 || ((recon == orc::REC_PPM || recon == orc::REC_PPM_CHAR) && ng < 3)) return nullptr;
  p.recon = recon;
  p.ng = ng;
  for (int d = 0; d < 3; ++d) {
    if (nx[d] <= 0 || mb[d] <= 0 || nx[d] % mb[d] != 0) return nullptr;
    p.nx[d] = nx[d];
    p.mb[d] = mb[d];
    p.xmin[d] = xmin[d];
    p.xmax[d] = xmax[d];
  }
  for (int f = 0; f < 6; ++f) p.bc[f] = bc[f];
  p.gamma = gamma;
  if (riemann < orc::RS_HLLE || riemann > orc::RS_HLLE_ROE) return nullptr;
  p.riemann = riemann;
  p.dfloor = dfloor;
  p.pfloor = pfloor;
  p.integrator = integrator;
  Mesh<double>* M = new Mesh<double>();
  M->init(p);
  return M;
}

void orc_mesh_free(void* m) { delete static_cast<Mesh<double>*>(m); }

void orc_set_prims(void* m, const double* w, const double* b1, const double* b2, const double* b3) {
  orc::set_prims(*static_cast<Mesh<double>*>(m), w, b1, b2, b3);
}

void orc_get_cons(void* m, double* u, double* b1, double* b2, double* b3) {
  orc::get_cons(*static_cast<Mesh<double>*>(m), u, b1, b2, b3);
}

/* Set the conserved state (global arrays, active region) and exchange ghosts. */
void orc_set_cons(void* m, const double* u, const double* b1, const double* b2, const double* b3) {
  orc::set_cons(*static_cast<Mesh<double>*>(m), u, nullptr, b1, nullptr, b2, nullptr, b3, nullptr);
}

/* cons -> prim of the current state on the active region: w[8][nz][ny][nx] (rho, v, p, b_c) */
/* Passive scalars from concentrations c[q][NZ][NY][NX]: rho C_q = rho c_q on the active cells (rho from the
 * current state, so set the state first), then the ghost exchange. */
void orc_set_scalars(void* m, const double* c) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (auto& B : M.blk)
    for (int q = 0; q < M.P.nscal; ++q)
      for (int k = 0; k < M.n[2]; ++k)
        for (int j = 0; j < M.n[1]; ++j)
          for (int i = 0; i < M.n[0]; ++i) {
            const size_t g = ((size_t)(B.loc[2] * M.n[2] + k) * NY + (B.loc[1] * M.n[1] + j)) * NX + (B.loc[0] * M.n[0] + i);
            const int K = k + M.NG, J = j + M.NG, I = i + M.NG;
            B.s[0][q](K, J, I) = B.u[0][0](K, J, I) * c[q * ncell + g];
          }
  M.fill_ghosts(0);
}

/* Forcing acceleration a[3][NZ][NY][NX] at the cell centres ([reading: forcing], see register_update);
 * NULL removes it. */
void orc_set_forcing(void* m, const double* a) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  M.forced = a != nullptr;
  if (!a) return;
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (auto& B : M.blk)
    for (int d = 0; d < 3; ++d) {
      B.acc[d].init(M.c[0], M.c[1], M.c[2]);
      for (int k = 0; k < M.n[2]; ++k)
        for (int j = 0; j < M.n[1]; ++j)
          for (int i = 0; i < M.n[0]; ++i) {
            const size_t g = ((size_t)(B.loc[2] * M.n[2] + k) * NY + (B.loc[1] * M.n[1] + j)) * NX + (B.loc[0] * M.n[0] + i);
            B.acc[d](k + M.NG, j + M.NG, i + M.NG) = a[d * ncell + g];
          }
    }
}

/* Scalar masses rho C_q of the active cells, out[q][NZ][NY][NX]. */
void orc_get_scalars(void* m, double* out) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (const auto& B : M.blk)
    for (int q = 0; q < M.P.nscal; ++q)
      for (int k = 0; k < M.n[2]; ++k)
        for (int j = 0; j < M.n[1]; ++j)
          for (int i = 0; i < M.n[0]; ++i) {
            const size_t g = ((size_t)(B.loc[2] * M.n[2] + k) * NY + (B.loc[1] * M.n[1] + j)) * NX + (B.loc[0] * M.n[0] + i);
            out[q * ncell + g] = B.s[0][q](k + M.NG, j + M.NG, i + M.NG);
          }
}

void orc_get_prims(void* m, double* w) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  M.cons_to_prim(0);
  const int NX = M.P.nx[0], NY = M.P.nx[1], NZ = M.P.nx[2];
  const size_t ncell = (size_t)NX * NY * NZ;
  for (const auto& B : M.blk)
    for (int k = 0; k < M.n[2]; ++k)
      for (int j = 0; j < M.n[1]; ++j)
        for (int i = 0; i < M.n[0]; ++i) {
          const size_t g = ((size_t)(B.loc[2] * M.n[2] + k) * NY + (B.loc[1] * M.n[1] + j)) * NX + (B.loc[0] * M.n[0] + i);
          for (int v = 0; v < 8; ++v) w[v * ncell + g] = B.w[v](k + M.NG, j + M.NG, i + M.NG);
        }
}

void orc_fill_ghosts(void* m) { static_cast<Mesh<double>*>(m)->fill_ghosts(0); }

void orc_step(void* m, double dt) { static_cast<Mesh<double>*>(m)->step(dt); }

double orc_new_dt(void* m, double cfl) { return static_cast<Mesh<double>*>(m)->new_dt(cfl); }

long orc_floor_count(void* m) { return static_cast<Mesh<double>*>(m)->floor_events; }

long orc_emf_mismatch_count(void* m) { return static_cast<Mesh<double>*>(m)->emf_mismatch; }

/* Fluxes of the current state on the global face grids: fx[7][NZ][NY][NX+1], fy[7][NZ][NY+1][NX],
 * fz[7][NZ+1][NY][NX]; component layout of each sweep (mass, M_n, M_t1, M_t2, E, B_t1, B_t2). */
void orc_debug_fluxes(void* m, int recon, double* fx, double* fy, double* fz) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  M.stage_terms(recon);
  const int N[3] = {M.P.nx[0], M.P.nx[1], M.P.nx[2]};
  double* out[3] = {fx, fy, fz};
  for (int d = 0; d < 3; ++d) {
    int gd[3] = {N[0], N[1], N[2]};
    gd[d] += 1;
    const size_t nf = (size_t)gd[0] * gd[1] * gd[2];
    for (const auto& B : M.blk)
      for (int k = 0; k < M.n[2] + (d == 2); ++k)
        for (int j = 0; j < M.n[1] + (d == 1); ++j)
          for (int i = 0; i < M.n[0] + (d == 0); ++i) {
            const int g[3] = {B.loc[0] * M.n[0] + i, B.loc[1] * M.n[1] + j, B.loc[2] * M.n[2] + k};
            const int li[3] = {i, j, k};
            if (li[d] == M.n[d] && g[d] != N[d]) continue;  // taken from the upper neighbour
            const size_t gi = ((size_t)g[2] * gd[1] + g[1]) * gd[0] + g[0];
            for (int v = 0; v < orc::NW7; ++v) out[d][v * nf + gi] = B.flx[d][v](k + M.NG, j + M.NG, i + M.NG);
          }
  }
}

/* Corner EMFs of the current state: e1[NZ+1][NY+1][NX], e2[NZ+1][NY][NX+1], e3[NZ][NY+1][NX+1]. */
void orc_debug_emfs(void* m, int recon, double* e1, double* e2, double* e3) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  M.stage_terms(recon);
  const int N[3] = {M.P.nx[0], M.P.nx[1], M.P.nx[2]};
  double* out[3] = {e1, e2, e3};
  for (int e = 0; e < 3; ++e) {
    int gd[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
    gd[e] -= 1;
    for (const auto& B : M.blk)
      for (int k = 0; k < M.n[2] + (e != 2); ++k)
        for (int j = 0; j < M.n[1] + (e != 1); ++j)
          for (int i = 0; i < M.n[0] + (e != 0); ++i) {
            const int g[3] = {B.loc[0] * M.n[0] + i, B.loc[1] * M.n[1] + j, B.loc[2] * M.n[2] + k};
            const int li[3] = {i, j, k};
            bool skip = false;
            for (int q = 0; q < 3; ++q)
              if (q != e && li[q] == M.n[q] && g[q] != N[q]) skip = true;
            if (skip) continue;
            const size_t gi = ((size_t)g[2] * gd[1] + g[1]) * gd[0] + g[0];
            out[e][gi] = B.emf[e](k + M.NG, j + M.NG, i + M.NG);
          }
  }
}

/* max over active cells of |div_h B| * min(dx) / max(rms |b_c|, 1e-300)  [reading] */
double orc_divb_norm(void* m) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  double mx = 0.0, s2 = 0.0;
  size_t cnt = 0;
  const int G = M.NG;
  for (const auto& B : M.blk)
    for (int k = G; k < M.n[2] + G; ++k)
      for (int j = G; j < M.n[1] + G; ++j)
        for (int i = G; i < M.n[0] + G; ++i) {
          const double dv = (B.b[0][0](k, j, i + 1) - B.b[0][0](k, j, i)) / M.dx[0] +
                            (B.b[0][1](k, j + 1, i) - B.b[0][1](k, j, i)) / M.dx[1] +
                            (B.b[0][2](k + 1, j, i) - B.b[0][2](k, j, i)) / M.dx[2];
          mx = std::fmax(mx, std::fabs(dv));
          const double bx = 0.5 * (B.b[0][0](k, j, i) + B.b[0][0](k, j, i + 1));
          const double by = 0.5 * (B.b[0][1](k, j, i) + B.b[0][1](k, j + 1, i));
          const double bz = 0.5 * (B.b[0][2](k, j, i) + B.b[0][2](k + 1, j, i));
          s2 += bx * bx + by * by + bz * bz;
          ++cnt;
        }
  const double hmin = std::fmin(M.dx[0], std::fmin(M.dx[1], M.dx[2]));
  const double rms = std::sqrt(s2 / (double)cnt);
  return mx * hmin / std::fmax(rms, 1e-300);
}

/* Volume integrals of rho, M1..3, E, b_c1..3 over the active region, Neumaier-compensated. */
void orc_totals(void* m, double* out) {
  Mesh<double>& M = *static_cast<Mesh<double>*>(m);
  const double dv = M.dx[0] * M.dx[1] * M.dx[2];
  double s[8] = {0}, cmp[8] = {0};
  const int G = M.NG;
  for (const auto& B : M.blk)
    for (int k = G; k < M.n[2] + G; ++k)
      for (int j = G; j < M.n[1] + G; ++j)
        for (int i = G; i < M.n[0] + G; ++i) {
          double x[8];
          for (int v = 0; v < 5; ++v) x[v] = B.u[0][v](k, j, i);
          x[5] = 0.5 * (B.b[0][0](k, j, i) + B.b[0][0](k, j, i + 1));
          x[6] = 0.5 * (B.b[0][1](k, j, i) + B.b[0][1](k, j + 1, i));
          x[7] = 0.5 * (B.b[0][2](k, j, i) + B.b[0][2](k + 1, j, i));
          for (int v = 0; v < 8; ++v) {
            const double y = x[v] * dv;
            const double t = s[v] + y;
            if (std::fabs(s[v]) >= std::fabs(y))
              cmp[v] += (s[v] - t) + y;
            else
              cmp[v] += (y - t) + s[v];
            s[v] = t;
          }
        }
  for (int v = 0; v < 8; ++v) out[v] = s[v] + cmp[v];
}

/* Tangent-linear of one VL2 cycle with a fixed dt, by dual numbers: from the conserved state (u, b1..3)
 * and a direction (du, db1..3), all in the global layout, return the new state and J*direction. */
void orc_tl_step(const int* nx, const int* mb, const double* xmin, const double* xmax, double gamma, int riemann,
                 const int* bc, double dt, double ct_delta, const double* u, const double* b1, const double* b2,
                 const double* b3,
                 const double* du, const double* db1, const double* db2, const double* db3, double* u_out,
                 double* b1_out, double* b2_out, double* b3_out, double* du_out, double* db1_out, double* db2_out,
                 double* db3_out) {
  orc::Params p;
  for (int d = 0; d < 3; ++d) {
    p.nx[d] = nx[d];
    p.mb[d] = mb[d];
    p.xmin[d] = xmin[d];
    p.xmax[d] = xmax[d];
  }
  for (int f = 0; f < 6; ++f) p.bc[f] = bc[f];
  p.gamma = gamma;
  p.riemann = riemann;
  p.dfloor = 1e-12;
  p.pfloor = 1e-12;
  p.integrator = orc::INT_VL2;
  p.recon = orc::REC_PLM;
  p.ng = 2;
  p.nscal = 0;
  p.ct_delta = ct_delta;
  orc::Mesh<orc::Dual> M;
  M.init(p);
  orc::set_cons(M, u, du, b1, db1, b2, db2, b3, db3);
  M.step(dt);
  orc::get_cons(M, u_out, b1_out, b2_out, b3_out);
  orc::get_tangent(M, du_out, db1_out, db2_out, db3_out);
}

/* Plain (value) cycle from a conserved state, same entry form as orc_tl_step (no tangent). */
void orc_step_cons(const int* nx, const int* mb, const double* xmin, const double* xmax, double gamma, int riemann,
                   const int* bc, double dt, double ct_delta, const double* u, const double* b1, const double* b2,
                 const double* b3,
                   double* u_out, double* b1_out, double* b2_out, double* b3_out) {
  orc::Params p;
  for (int d = 0; d < 3; ++d) {
    p.nx[d] = nx[d];
    p.mb[d] = mb[d];
    p.xmin[d] = xmin[d];
    p.xmax[d] = xmax[d];
  }
  for (int f = 0; f < 6; ++f) p.bc[f] = bc[f];
  p.gamma = gamma;
  p.riemann = riemann;
  p.dfloor = 1e-12;
  p.pfloor = 1e-12;
  p.integrator = orc::INT_VL2;
  p.recon = orc::REC_PLM;
  p.ng = 2;
  p.nscal = 0;
  p.ct_delta = ct_delta;
  orc::Mesh<double> M;
  M.init(p);
  orc::set_cons(M, u, nullptr, b1, nullptr, b2, nullptr, b3, nullptr);
  M.step(dt);
  orc::get_cons(M, u_out, b1_out, b2_out, b3_out);
}

/* ---- pointwise entry points for the unit pins ---- */
void orc_riemann(int solver, const double* wl, const double* wr, double bn, double gamma, double* f) {
  orc::riemann<double>(solver, wl, wr, bn, gamma, f);
}

/* Jacobians of the Riemann flux for n interfaces: jac[q][n][k] = dF_n / dx_k with x = (w_L[0..6], w_R[0..6],
   b_n), one dual-number evaluation per column (test infrastructure for the adjoint). */
void orc_riemann_jacobian(int solver, long long n, const double* wl, const double* wr, const double* bn, double gamma,
                          double* jac) {
  for (long long q = 0; q < n; ++q) {
    for (int k = 0; k < 15; ++k) {
      orc::Dual dl[orc::NW7], dr[orc::NW7], f[orc::NW7];
      for (int m = 0; m < orc::NW7; ++m) {
        dl[m] = orc::Dual(wl[7 * q + m], k == m ? 1.0 : 0.0);
        dr[m] = orc::Dual(wr[7 * q + m], k == 7 + m ? 1.0 : 0.0);
      }
      const orc::Dual b(bn[q], k == 14 ? 1.0 : 0.0);
      orc::riemann<orc::Dual>(solver, dl, dr, b, gamma, f);
      for (int m = 0; m < orc::NW7; ++m) jac[(q * 7 + m) * 15 + k] = f[m].d;
    }
  }
}

void orc_physical_flux(const double* w, double bn, double gamma, double* u, double* f) {
  orc::physical_flux<double>(w, bn, gamma, u, f);
}

double orc_fast_speed(double d, double p, double bn, double bt1, double bt2, double gamma) {
  return orc::fast_speed<double>(d, p, bn, bt1, bt2, gamma);
}

void orc_roe_fast_speed(const double* wl, const double* wr, double bn, double gamma, double* out) {
  orc::roe_fast_speed<double>(wl, wr, bn, gamma, &out[0], &out[1]);
}

double orc_vanleer_slope(double qm, double q0, double qp) { return orc::vanleer_slope<double>(qm, q0, qp); }

/* PPM edges of one cell from q[0..4] = q_{i-2} .. q_{i+2}: out[0] = left edge, out[1] = right edge. */
void orc_ppm_edges(const double* q, double* out) { orc::ppm_edges<double>(q, out[0], out[1]); }
/* R (row-major 7 x 7, columns the right eigenvectors), its inverse L and the eigenvalues of the primitive
 * MHD system at the state w = (rho, v_n, v_t1, v_t2, p, b_t1, b_t2) with normal field bn. */
void orc_mhd_eigensystem(const double* w, double bn, double gamma, double* R, double* L, double* lam) {
  double Rm[orc::NW7][orc::NW7], Lm[orc::NW7][orc::NW7];
  orc::mhd_eigensystem<double>(w, bn, gamma, Rm, lam);
  orc::invert7<double>(Rm, Lm);
  for (int r = 0; r < orc::NW7; ++r)
    for (int c = 0; c < orc::NW7; ++c) {
      R[r * orc::NW7 + c] = Rm[r][c];
      L[r * orc::NW7 + c] = Lm[r][c];
    }
}
/* Characteristic PPM edges (lower, upper) of the middle cell of the five states q[5][7]. */
void orc_char_ppm_edges(const double* q, double bn, double gamma, double* out) {
  double qs[5][orc::NW7], ql[orc::NW7], qr[orc::NW7];
  for (int j = 0; j < 5; ++j)
    for (int v = 0; v < orc::NW7; ++v) qs[j][v] = q[j * orc::NW7 + v];
  orc::char_ppm_edges<double>(qs, bn, gamma, ql, qr);
  for (int v = 0; v < orc::NW7; ++v) {
    out[2 * v] = ql[v];
    out[2 * v + 1] = qr[v];
  }
}
/* Limited slope of the characteristic reconstruction of the middle cell of q = (qm, q0, qp), 7 each. */
void orc_char_slope(const double* q, double bn, double gamma, double* dw) {
  orc::char_slope<double>(q, q + orc::NW7, q + 2 * orc::NW7, bn, gamma, dw);
}

/* PPM fourth-order face value between q[1] and q[2] from q[0..3], limited (step 2). */
double orc_ppm_face(const double* q) { return orc::ppm_face<double>(q[0], q[1], q[2], q[3]); }

/* FP64 operations of one face flux for the given reconstruction and solver, counted with the
 * operation-counting scalar.  q: the 7-component sweep-frame states of cells i-2, i-1, i, i+1
 * ([4][7]); out: add/sub, mul, div, sqrt, compare counts. */
void orc_count_face_ops(int recon, int solver, const double* q, double bn, double gamma, long long* out) {
  using orc::Flop;
  orc::g_ops = orc::OpCount();
  Flop wl[7], wr[7], f[7];
  for (int n = 0; n < 7; ++n) {
    if (recon == orc::REC_DC) {
      wl[n] = Flop(q[7 + n]);
      wr[n] = Flop(q[14 + n]);
    } else {
      const Flop dlm = orc::vanleer_slope(Flop(q[n]), Flop(q[7 + n]), Flop(q[14 + n]));
      const Flop dl0 = orc::vanleer_slope(Flop(q[7 + n]), Flop(q[14 + n]), Flop(q[21 + n]));
      wl[n] = Flop(q[7 + n]) + 0.5 * dlm;
      wr[n] = Flop(q[14 + n]) - 0.5 * dl0;
    }
  }
  orc::riemann<Flop>(solver, wl, wr, Flop(bn), gamma, f);
  out[0] = orc::g_ops.add;
  out[1] = orc::g_ops.mul;
  out[2] = orc::g_ops.div;
  out[3] = orc::g_ops.sqrt;
  out[4] = orc::g_ops.cmp;
}

double orc_ct_corner(const double* ea, const double* eb, const double* ec, const double* ma, const double* mb) {
  return orc::ct_corner<double>(ea, eb, ec, ma, mb);
}

}  // extern "C"
