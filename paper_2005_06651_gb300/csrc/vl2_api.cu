// C ABI of the GB300 VL2 MHD library (declarations and contracts in include/vl2mhd.h).
// Host orchestration only: argument checks, workspace carving, the kernel sequence of a VL2 cycle
// (Sec. 3.2.3) and the copies of global-array I/O.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vl2_internal.h"
#include "vl2mhd.h"

using vl2::Arrays;
using vl2::Geom;

struct vl2_mesh {
  vl2_params p;
  Geom g;
  Arrays a;
  cudaStream_t st = nullptr;
  std::vector<int> loc, nbr;
  bool initialized = false;
  bool w_valid = false;     // primitives of register 0 are current on every cell
  bool dt_pending = false;  // scal[SC_MAXRATE] holds the CFL rate of register 0
  unsigned long long floors_seen = 0;
  double* dres = nullptr;   // device result slots of the reductions
  double* ddt = nullptr;    // device slot of the step vl2_step_cfl formed (dres[15])
  std::string err;
  // kernel timing (vl2_profile) and launch counting
  bool prof = false;
  struct Rec {
    int kind;
    long long units;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
  double acc_ms[VL2_K_COUNT] = {0};
  long long acc_n[VL2_K_COUNT] = {0}, acc_units[VL2_K_COUNT] = {0};
  long long launches = 0;
  vl2::FluxShape fs;
  vl2::AdjArrays adj{};
  bool has_adj = false;
  double* acc_store = nullptr;  // reserved forcing array (params.forcing); a.acc points here once set
  vl2::MeshView view() const { return vl2::MeshView{g, a}; }
  int max_mb() const { return std::max(g.mb[0], std::max(g.mb[1], g.mb[2])); }
  // reconstruction of the higher-order stages (params.recon, 0 meaning PLM)
  int rec() const { return (p.recon >= VL2_PPM && p.recon <= VL2_PPM_CHAR) ? p.recon : VL2_PLM; }
  ~vl2_mesh() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

namespace {

thread_local std::string g_err;

vl2_status fail(vl2_mesh* m, vl2_status s, const std::string& msg) {
  if (m)
    m->err = msg;
  else
    g_err = msg;
  return s;
}

vl2_status cuda_fail(vl2_mesh* m, cudaError_t e, const char* where) {
  return fail(m, VL2_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define VL2_CHECK(m, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((m), e_, #call); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

long long ncells(const Geom& g) { return (long long)g.N[0] * g.N[1] * g.N[2]; }

long long nfaces_total(const Geom& g) {
  const long long X = g.N[0], Y = g.N[1], Z = g.N[2];
  return (X + 1) * Y * Z + X * (Y + 1) * Z + X * Y * (Z + 1);
}

long long max_face_grid(const Geom& g) {
  const long long X = g.N[0], Y = g.N[1], Z = g.N[2];
  long long m = (X + 1) * Y * Z;
  m = std::max(m, X * (Y + 1) * Z);
  m = std::max(m, X * Y * (Z + 1));
  return m;
}

long long max_edge_grid(const Geom& g) {
  const long long X = g.N[0], Y = g.N[1], Z = g.N[2];
  long long m = X * (Y + 1) * (Z + 1);
  m = std::max(m, (X + 1) * Y * (Z + 1));
  m = std::max(m, (X + 1) * (Y + 1) * Z);
  return m;
}

constexpr int RED_CTAS = 608;  // 4 per SM on a 152-SM GB300

vl2_status make_geom(const vl2_params* p, Geom& g, std::string& msg) {
  if (!p) {
    msg = "params is NULL";
    return VL2_E_ARG;
  }
  for (int d = 0; d < 3; ++d) {
    if (p->nx[d] <= 0 || p->mb[d] <= 0 || p->nx[d] % p->mb[d] != 0) {
      msg = "nx must be positive multiples of mb in every direction";
      return VL2_E_ARG;
    }
    if (!(p->xmax[d] > p->xmin[d])) {
      msg = "xmax must exceed xmin";
      return VL2_E_ARG;
    }
  }
  if (p->ng != 2 && p->ng != 3) {
    msg = "ng must be 2 or 3";
    return VL2_E_ARG;
  }
  if (p->recon < 0 || p->recon > VL2_PPM_CHAR) {
    msg = "recon must be VL2_PLM (or 0), VL2_PPM, VL2_PLM_CHAR or VL2_PPM_CHAR";
    return VL2_E_ARG;
  }
  if ((p->recon == VL2_PPM || p->recon == VL2_PPM_CHAR) && p->ng < 3) {
    msg = "PPM needs ng = 3 (a face reads three cells on each side)";
    return VL2_E_ARG;
  }
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->dfloor >= DBL_MIN) || !(p->pfloor >= DBL_MIN) ||
      !std::isfinite(p->dfloor) || !std::isfinite(p->pfloor)) {
    msg = "gamma > 1, cfl > 0 and floors that are positive normal numbers are required";
    return VL2_E_ARG;
  }
  if (p->riemann != VL2_HLLD && p->riemann != VL2_HLLE && p->riemann != VL2_HLLE_ROE) {
    msg = "riemann must be VL2_HLLD, VL2_HLLE or VL2_HLLE_ROE";
    return VL2_E_ARG;
  }
  if (p->precision != VL2_FP64 && p->precision != VL2_MIXED) {
    msg = "precision must be VL2_FP64 or VL2_MIXED";
    return VL2_E_ARG;
  }
  if (p->adjoint != 0 && (p->adjoint != 1 || p->precision != VL2_FP64)) {
    msg = "adjoint must be 0 or 1, and 1 needs VL2_FP64";
    return VL2_E_ARG;
  }
  if (p->integrator < VL2_INT_VL2 || p->integrator > VL2_INT_RK3) {
    msg = "integrator must be VL2_INT_VL2, VL2_INT_RK1, VL2_INT_RK2 or VL2_INT_RK3";
    return VL2_E_ARG;
  }
  if (p->adjoint && p->integrator != VL2_INT_VL2) {
    msg = "the adjoint (params.adjoint = 1) is written for the VL2 integrator";
    return VL2_E_ARG;
  }
  if (p->adjoint && p->riemann == VL2_HLLE_ROE) {
    msg = "the adjoint (params.adjoint = 1) is written for VL2_HLLD and VL2_HLLE";
    return VL2_E_ARG;
  }
  if (p->adjoint && (p->ng != 2 || (p->recon != 0 && p->recon != VL2_PLM))) {
    msg = "the adjoint (params.adjoint = 1) is written for PLM with ng = 2";
    return VL2_E_ARG;
  }
  if (p->nscalars < 0 || p->nscalars > VL2_MAX_SCALARS || (p->adjoint && p->nscalars)) {
    msg = "nscalars must be 0 .. VL2_MAX_SCALARS (and 0 with the adjoint)";
    return VL2_E_ARG;
  }
  if ((p->forcing != 0 && p->forcing != 1) || (p->forcing && p->adjoint)) {
    msg = "forcing must be 0 or 1 (and 0 with the adjoint)";
    return VL2_E_ARG;
  }
  if (!(p->ct_delta >= 0.0) || !std::isfinite(p->ct_delta)) {
    msg = "ct_delta must be finite and >= 0";
    return VL2_E_ARG;
  }
  for (int d = 0; d < 3; ++d) {
    const int lo = p->bc[2 * d], hi = p->bc[2 * d + 1];
    if ((lo != VL2_PERIODIC && lo != VL2_OUTFLOW) || (hi != VL2_PERIODIC && hi != VL2_OUTFLOW) ||
        ((lo == VL2_PERIODIC) != (hi == VL2_PERIODIC))) {
      msg = "bc must be periodic on both faces of a direction or outflow";
      return VL2_E_ARG;
    }
  }
  std::memset(&g, 0, sizeof(g));
  long long nblk = 1;
  for (int d = 0; d < 3; ++d) {
    g.N[d] = p->nx[d];
    g.mb[d] = p->mb[d];
    g.nb[d] = p->nx[d] / p->mb[d];
    nblk *= g.nb[d];
    g.dx[d] = (p->xmax[d] - p->xmin[d]) / p->nx[d];
    g.idx[d] = 1.0 / g.dx[d];
  }
  if (nblk > (1LL << 30)) {
    msg = "too many MeshBlocks";
    return VL2_E_ARG;
  }
  g.nblk = (int)nblk;
  g.ng = p->ng;
  g.ns = p->nscalars;
  g.ct_delta = p->ct_delta;
  g.hlle_roe = p->riemann == VL2_HLLE_ROE ? 1 : 0;
  g.sx = ((p->mb[0] + 2 * g.ng + 1) + 3) & ~3;
  g.sy = p->mb[1] + 2 * g.ng + 1;
  g.sz = p->mb[2] + 2 * g.ng + 1;
  g.box = (long long)g.sx * g.sy * g.sz;
  if (g.box * 8 > (1LL << 31)) {
    msg = "MeshBlock too large";
    return VL2_E_ARG;
  }
  for (int f = 0; f < 6; ++f) g.bc[f] = p->bc[f];
  g.flux_halo = 0;
  for (int f = 0; f < 6; ++f) g.flux_halo |= p->bc[f] != VL2_PERIODIC;
  g.gamma = p->gamma;
  g.gm1 = p->gamma - 1.0;
  g.igm1 = 1.0 / (p->gamma - 1.0);
  g.gamma_f = (float)g.gamma;
  g.igm1_f = (float)g.igm1;
  for (int d = 0; d < 3; ++d) g.idx_f[d] = (float)g.idx[d];
  g.dfloor = p->dfloor;
  g.pfloor = p->pfloor;
  return VL2_OK;
}

struct Plan {
  size_t off_u[2], off_b[2][3], off_w, off_f[3], off_e[3], off_ec, off_stage, off_red, off_scal, total;
  size_t off_s[2], off_cs, off_fsc[3];  // passive scalars (empty when ns = 0)
  size_t off_acc;                       // forcing acceleration (empty without params.forcing)
  size_t off_tmw;                       // tensor maps of w for the TMA-staged PLM sweeps (vl2::TMA_MAPS x 128 B)
  size_t stage_elems;
  size_t off_adj;  // start of the adjoint arrays (59 FP64 arrays per block, 65 with ct_delta) when requested
};
constexpr int ADJ_ARRAYS = 10 + 6 + 8 + 21 + 7 + 3 + 8 + 3;
constexpr int ADJ_ARRAYS_SMOOTH_CT = 6;  // the predictor's face EMFs, kept for the smoothed weight's derivative

Plan make_plan(const Geom& g, int precision, int adjoint, int forcing) {
  Plan pl;
  size_t o = 0;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  const size_t sper = (size_t)g.nblk * g.box * (precision == VL2_MIXED ? sizeof(float) : sizeof(double));
  for (int r = 0; r < 2; ++r) {
    pl.off_u[r] = o;
    o = align256(o + 5 * per);
    for (int d = 0; d < 3; ++d) {
      pl.off_b[r][d] = o;
      o = align256(o + per);
    }
  }
  pl.off_w = o;
  o = align256(o + 8 * sper);
  for (int d = 0; d < 3; ++d) {
    pl.off_f[d] = o;
    o = align256(o + 7 * sper);
  }
  for (int d = 0; d < 3; ++d) {
    pl.off_e[d] = o;
    o = align256(o + sper);
  }
  pl.off_ec = o;
  o = align256(o + 3 * sper);
  const size_t sc = (size_t)g.ns * per;
  for (int r = 0; r < 2; ++r) {
    pl.off_s[r] = o;
    o = align256(o + sc);
  }
  pl.off_cs = o;
  o = align256(o + sc);
  for (int d = 0; d < 3; ++d) {
    pl.off_fsc[d] = o;
    o = align256(o + sc);
  }
  pl.off_acc = o;
  if (forcing) o = align256(o + 3 * per);
  pl.off_tmw = o;
  o = align256(o + (size_t)vl2::TMA_MAPS * 128);
  const long long nc = ncells(g);
  long long st = 5 * nc + nfaces_total(g);
  st = std::max(st, (long long)g.ns * nc);
  st = std::max(st, 8 * nc);
  st = std::max(st, 7 * max_face_grid(g));
  st = std::max(st, max_edge_grid(g));
  pl.stage_elems = (size_t)st;
  pl.off_stage = o;
  o = align256(o + (size_t)st * sizeof(double));
  pl.off_red = o;
  o = align256(o + (size_t)RED_CTAS * 8 * sizeof(double));
  pl.off_scal = o;
  o = align256(o + vl2::SC_COUNT * sizeof(unsigned long long) + 16 * sizeof(double));
  pl.off_adj = o;
  if (adjoint) o = align256(o + (size_t)(ADJ_ARRAYS + (g.ct_delta > 0.0 ? ADJ_ARRAYS_SMOOTH_CT : 0)) * per);
  pl.total = o;
  return pl;
}

vl2_status sync(vl2_mesh* m) {
  VL2_CHECK(m, cudaStreamSynchronize(m->st));
  return VL2_OK;
}

vl2_status copy_in(vl2_mesh* m, double* dst, const double* src, size_t n, int where) {
  VL2_CHECK(m, cudaMemcpyAsync(dst, src, n * sizeof(double),
                               where == VL2_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, m->st));
  return VL2_OK;
}

vl2_status copy_out(vl2_mesh* m, double* dst, const double* src, size_t n) {
  VL2_CHECK(m, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  return VL2_OK;
}


bool bad_where(int where) { return where != VL2_HOST && where != VL2_DEVICE; }

cudaEvent_t pool_event(vl2_mesh* m) {
  if (m->pool_used == m->pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    m->pool.push_back(e);
  }
  return m->pool[m->pool_used++];
}

// Enqueue one kernel launch: counts it and, when profiling is on, brackets it with events.
template <class Fn>
cudaError_t timed(vl2_mesh* m, int kind, long long units, Fn&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (m->prof) {
    a = pool_event(m);
    b = pool_event(m);
    if (a) cudaEventRecord(a, m->st);
  }
  cudaError_t e = fn();
  ++m->launches;
  if (m->prof && a && b && e == cudaSuccess) {
    cudaEventRecord(b, m->st);
    m->recs.push_back({kind, units, a, b});
  }
  return e;
}

long long cells_all(const Geom& g) {
  return (long long)g.nblk * (g.mb[0] + 2 * g.ng) * (g.mb[1] + 2 * g.ng) * (g.mb[2] + 2 * g.ng);
}
long long nodes(const Geom& g) { return (long long)g.nblk * (g.mb[0] + 1) * (g.mb[1] + 1) * (g.mb[2] + 1); }
long long ghost_elems(const Geom& g) {
  return (long long)g.nblk * (g.mb[0] + 2 * g.ng + 1) * (g.mb[1] + 2 * g.ng + 1) * (g.mb[2] + 2 * g.ng + 1);
}
long long flux_faces(const Geom& g, int d) {
  long long n = g.nblk;
  for (int q = 0; q < 3; ++q) n *= g.mb[q] + (q == d ? 1 : 2 * g.flux_halo);
  return n;
}
long long halo_faces(const Geom& g) {
  if (g.flux_halo) return 0;
  long long n = 0;
  for (int d = 0; d < 3; ++d) n += 2LL * (g.mb[d] + 1) * (g.mb[(d + 1) % 3] + g.mb[(d + 2) % 3]);
  return n * g.nblk;
}

cudaError_t k_prim(vl2_mesh* m, int reg, bool dt) {
  return timed(m, VL2_K_PRIM, cells_all(m->g),
               [&] { return vl2::launch_prim(m->view(), nullptr, reg, true, dt, m->st); });
}
cudaError_t k_ghosts(vl2_mesh* m, int reg) {
  return timed(m, VL2_K_GHOSTS, ghost_elems(m->g), [&] { return vl2::launch_ghosts(m->view(), nullptr, reg, m->st); });
}
cudaError_t k_fluxes(vl2_mesh* m, int reg, int recon) {
  for (int d = 0; d < 3; ++d) {
    const int kind = recon == VL2_DC ? VL2_K_FLUX_DC
                                     : ((recon == VL2_PPM || recon == VL2_PPM_CHAR) ? VL2_K_FLUX_PPM : VL2_K_FLUX_PLM);
    cudaError_t e = timed(m, kind, flux_faces(m->g, d), [&] {
      return vl2::launch_flux(m->view(), nullptr, reg, recon, m->p.riemann, d, m->fs, m->max_mb(), m->st);
    });
    if (e != cudaSuccess) return e;
  }
  if (m->g.flux_halo) return cudaSuccess;
  return timed(m, VL2_K_FLUX_HALO, halo_faces(m->g), [&] { return vl2::launch_flux_halo(m->view(), nullptr, m->st); });
}
cudaError_t k_scalar_fluxes(vl2_mesh* m, int recon) {
  if (!m->g.ns) return cudaSuccess;
  for (int d = 0; d < 3; ++d) {
    cudaError_t e = timed(m, VL2_K_SCALARS, flux_faces(m->g, d),
                          [&] { return vl2::launch_scalar_fluxes(m->view(), recon, d, m->st); });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t k_scalar_update(vl2_mesh* m, int base, int out, double h, double g_base = 1.0, double g_other = 0.0) {
  if (!m->g.ns) return cudaSuccess;
  return timed(m, VL2_K_SCALARS, nodes(m->g),
               [&] { return vl2::launch_scalar_update(m->view(), base, out, h, g_base, g_other, m->st); });
}
cudaError_t k_emfs(vl2_mesh* m) {
  return timed(m, VL2_K_EMF, nodes(m->g), [&] { return vl2::launch_emfs(m->view(), nullptr, m->st); });
}
cudaError_t k_update(vl2_mesh* m, int base, int out, double h, double g_base = 1.0, double g_other = 0.0,
                     int stage = -1) {
  return timed(m, VL2_K_UPDATE, nodes(m->g), [&] {
    return vl2::launch_update(m->view(), nullptr, base, out, h, nullptr, 0.0, m->st, g_base, g_other, stage);
  });
}
// the plain update with h = beta * dt[0] read on the device (vl2_step_cfl)
cudaError_t k_update_ddt(vl2_mesh* m, int base, int out, double beta, int stage = -1) {
  return timed(m, VL2_K_UPDATE, nodes(m->g), [&] {
    return vl2::launch_update(m->view(), nullptr, base, out, 0.0, m->ddt, beta, m->st, 1.0, 0.0, stage);
  });
}

vl2_status ensure_prims(vl2_mesh* m) {
  if (!m->w_valid) {
    VL2_CHECK(m, k_prim(m, 0, false));
    m->w_valid = true;
  }
  return VL2_OK;
}

}  // namespace

namespace vl2 {
void record_error(const char* msg) { g_err = msg; }
}  // namespace vl2

extern "C" {

vl2_status vl2_workspace_bytes(const vl2_params* params, size_t* bytes) {
  Geom g;
  std::string msg;
  vl2_status s = make_geom(params, g, msg);
  if (s != VL2_OK) return fail(nullptr, s, msg);
  if (!bytes) return fail(nullptr, VL2_E_ARG, "bytes is NULL");
  *bytes = make_plan(g, params->precision, params->adjoint, params->forcing).total;
  return VL2_OK;
}

vl2_status vl2_mesh_create(const vl2_params* params, void* workspace, size_t bytes, vl2_mesh** out) {
  if (!out) return fail(nullptr, VL2_E_ARG, "out is NULL");
  *out = nullptr;
  Geom g;
  std::string msg;
  vl2_status s = make_geom(params, g, msg);
  if (s != VL2_OK) return fail(nullptr, s, msg);
  if (!workspace || ((uintptr_t)workspace & 255u)) return fail(nullptr, VL2_E_ARG, "workspace must be 256-byte aligned");
  const Plan pl = make_plan(g, params->precision, params->adjoint, params->forcing);
  if (bytes < pl.total) return fail(nullptr, VL2_E_NOMEM, "workspace smaller than vl2_workspace_bytes()");
  vl2_mesh* m = new (std::nothrow) vl2_mesh();
  if (!m) return fail(nullptr, VL2_E_ARG, "host allocation failed");
  m->p = *params;
  m->g = g;
  m->st = (cudaStream_t)params->stream;
  char* base = (char*)workspace;
  for (int r = 0; r < 2; ++r) {
    m->a.u[r] = (double*)(base + pl.off_u[r]);
    for (int d = 0; d < 3; ++d) m->a.b[r][d] = (double*)(base + pl.off_b[r][d]);
  }
  m->a.w = base + pl.off_w;
  for (int d = 0; d < 3; ++d) {
    m->a.f[d] = base + pl.off_f[d];
    m->a.e[d] = base + pl.off_e[d];
  }
  m->a.ec = base + pl.off_ec;
  m->a.mixed = params->precision == VL2_MIXED ? 1 : 0;
  for (int r = 0; r < 2; ++r) m->a.s[r] = g.ns ? (double*)(base + pl.off_s[r]) : nullptr;
  m->a.cs = g.ns ? (double*)(base + pl.off_cs) : nullptr;
  m->acc_store = params->forcing ? (double*)(base + pl.off_acc) : nullptr;
  m->a.acc = nullptr;
  for (int d = 0; d < 3; ++d) m->a.fsc[d] = g.ns ? (double*)(base + pl.off_fsc[d]) : nullptr;
  if (params->adjoint) {
    const size_t per = (size_t)g.nblk * g.box;
    double* q = (double*)(base + pl.off_adj);
    auto take = [&](size_t nvar) {
      double* r = q;
      q += nvar * per;
      return r;
    };
    for (int r = 0; r < 2; ++r) {
      m->adj.lu[r] = take(5);
      for (int d = 0; d < 3; ++d) m->adj.lb[r][d] = take(1);
    }
    m->adj.lw = take(8);
    for (int d = 0; d < 3; ++d) m->adj.lf[d] = take(7);
    m->adj.lr = take(7);
    for (int d = 0; d < 3; ++d) m->adj.le[d] = take(1);
    m->adj.w0 = take(8);
    for (int d = 0; d < 3; ++d) m->adj.m1[d] = take(g.ct_delta > 0.0 ? 3 : 1);
    for (int d = 0; d < 3; ++d) m->adj.ps[d] = static_cast<double*>(m->a.f[d]);  // FP64: the adjoint needs VL2_FP64
    m->has_adj = true;
  }
  m->a.stage = (double*)(base + pl.off_stage);
  m->a.stage_elems = pl.stage_elems;
  m->a.red = (double*)(base + pl.off_red);
  m->a.red_ctas = RED_CTAS;
  m->a.scal = (unsigned long long*)(base + pl.off_scal);
  m->dres = (double*)(m->a.scal + vl2::SC_COUNT);
  m->ddt = m->dres + 15;
  // block table and 26-neighbour table (x fastest block order)
  m->loc.resize((size_t)g.nblk * 3);
  m->nbr.resize((size_t)g.nblk * 27);
  for (int b = 0; b < g.nblk; ++b) {
    const int l[3] = {b % g.nb[0], (b / g.nb[0]) % g.nb[1], b / (g.nb[0] * g.nb[1])};
    for (int d = 0; d < 3; ++d) m->loc[3 * b + d] = l[d];
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int dd[3] = {di, dj, dk};
          int q[3];
          bool ok = true;
          for (int d = 0; d < 3; ++d) {
            q[d] = l[d] + dd[d];
            if (q[d] < 0 || q[d] >= g.nb[d]) {
              if (g.bc[2 * d] == vl2::BC_PERIODIC)
                q[d] = (q[d] + g.nb[d]) % g.nb[d];
              else
                ok = false;
            }
          }
          m->nbr[(size_t)b * 27 + (dk + 1) * 9 + (dj + 1) * 3 + (di + 1)] =
              ok ? (q[2] * g.nb[1] + q[1]) * g.nb[0] + q[0] : -1;
        }
  }
  // tensor maps of the primitives for the TMA-staged PLM sweeps (host-encoded once: w never moves)
  alignas(128) unsigned char maps[vl2::TMA_MAPS * 128];
  const char* why = nullptr;
  const bool have_maps = vl2::encode_w_maps(g, m->a.w, m->a.mixed ? 4 : 8, maps, &why);
  m->a.tmw = have_maps ? base + pl.off_tmw : nullptr;
  m->fs.plm_tma = 0;  // the line-tile PLM kernel measured faster on GB300 in both precisions
  cudaError_t e = vl2::prepare_kernel_attributes();
  if (e == cudaSuccess) e = cudaMemsetAsync(workspace, 0, pl.total, m->st);
  if (e == cudaSuccess && have_maps) e = cudaMemcpyAsync(base + pl.off_tmw, maps, sizeof(maps), cudaMemcpyHostToDevice, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) {
    delete m;
    return fail(nullptr, VL2_E_CUDA, std::string("workspace clear: ") + cudaGetErrorString(e));
  }
  vl2::prime_flux_tma(m->view(), m->rec(), m->p.riemann == VL2_HLLD ? vl2::RS_HLLD : vl2::RS_HLLE, m->fs, m->max_mb(),
                      m->st);
  *out = m;
  return VL2_OK;
}

vl2_status vl2_mesh_destroy(vl2_mesh* mesh) {
  delete mesh;
  return VL2_OK;
}

vl2_status vl2_block_layout(const vl2_mesh* mesh, vl2_layout* out) {
  if (!mesh || !out) return fail(nullptr, VL2_E_ARG, "NULL argument");
  out->nblocks = mesh->g.nblk;
  for (int d = 0; d < 3; ++d) {
    out->nb[d] = mesh->g.nb[d];
    out->mb[d] = mesh->g.mb[d];
  }
  out->ng = mesh->g.ng;
  out->sx = mesh->g.sx;
  out->sy = mesh->g.sy;
  out->sz = mesh->g.sz;
  out->block_stride_vars = mesh->g.box;
  out->block_loc = mesh->loc.data();
  out->neighbor = mesh->nbr.data();
  out->u = mesh->a.u[0];
  for (int d = 0; d < 3; ++d) out->b[d] = mesh->a.b[0][d];
  return VL2_OK;
}

vl2_status vl2_set_prims(vl2_mesh* m, const double* w, const double* b1, const double* b2, const double* b3,
                         int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!w || !b1 || !b2 || !b3 || bad_where(where)) return fail(m, VL2_E_ARG, "NULL input or bad where");
  const Geom& g = m->g;
  const long long nc = ncells(g);
  const long long n1 = (long long)(g.N[0] + 1) * g.N[1] * g.N[2];
  const long long n2 = (long long)g.N[0] * (g.N[1] + 1) * g.N[2];
  const long long n3 = (long long)g.N[0] * g.N[1] * (g.N[2] + 1);
  const double *dw = w, *d1 = b1, *d2 = b2, *d3 = b3;
  if (where == VL2_HOST) {
    double* s = m->a.stage;
    vl2_status st;
    if ((st = copy_in(m, s, w, 5 * nc, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc, b1, n1, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1, b2, n2, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1 + n2, b3, n3, where)) != VL2_OK) return st;
    dw = s;
    d1 = s + 5 * nc;
    d2 = d1 + n1;
    d3 = d2 + n2;
  }
  VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MISMATCH, 0, sizeof(unsigned long long), m->st));
  VL2_CHECK(m, vl2::launch_check_periodic(g, d1, d2, d3, m->a.scal + vl2::SC_MISMATCH, m->st));
  ++m->launches;
  unsigned long long mism = 0;
  VL2_CHECK(m, cudaMemcpyAsync(&mism, m->a.scal + vl2::SC_MISMATCH, sizeof(mism), cudaMemcpyDeviceToHost, m->st));
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  if (mism) return fail(m, VL2_E_ARG, "periodic duplicate faces (face N and face 0) differ");
  VL2_CHECK(m, vl2::launch_scatter_prims(g, m->a, dw, d1, d2, d3, m->st));
  ++m->launches;
  VL2_CHECK(m, k_ghosts(m, 0));
  m->initialized = true;
  m->w_valid = false;
  m->dt_pending = false;
  return sync(m);
}

vl2_status vl2_set_prims_async(vl2_mesh* m, const double* w, const double* b1, const double* b2, const double* b3,
                               int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!w || !b1 || !b2 || !b3 || bad_where(where)) return fail(m, VL2_E_ARG, "NULL input or bad where");
  const Geom& g = m->g;
  const long long nc = ncells(g);
  const long long n1 = (long long)(g.N[0] + 1) * g.N[1] * g.N[2];
  const long long n2 = (long long)g.N[0] * (g.N[1] + 1) * g.N[2];
  const long long n3 = (long long)g.N[0] * g.N[1] * (g.N[2] + 1);
  const double *dw = w, *d1 = b1, *d2 = b2, *d3 = b3;
  if (where == VL2_HOST) {
    double* s = m->a.stage;
    vl2_status st;
    if ((st = copy_in(m, s, w, 5 * nc, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc, b1, n1, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1, b2, n2, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1 + n2, b3, n3, where)) != VL2_OK) return st;
    dw = s;
    d1 = s + 5 * nc;
    d2 = d1 + n1;
    d3 = d2 + n2;
  }
  // the periodic-face check raises a sticky device flag, reported by the next vl2_new_dt or vl2_last_dt
  VL2_CHECK(m, vl2::launch_check_periodic(g, d1, d2, d3, m->a.scal + vl2::SC_MISMATCH_ASYNC, m->st));
  ++m->launches;
  VL2_CHECK(m, vl2::launch_scatter_prims(g, m->a, dw, d1, d2, d3, m->st));
  ++m->launches;
  VL2_CHECK(m, k_ghosts(m, 0));
  m->initialized = true;
  m->w_valid = false;
  m->dt_pending = false;
  return VL2_OK;
}

vl2_status vl2_set_scalars(vl2_mesh* m, const double* c, int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!c || bad_where(where)) return fail(m, VL2_E_ARG, "NULL input or bad where");
  if (!m->initialized) return fail(m, VL2_E_STATE, "set the state (vl2_set_prims / vl2_set_cons) first");
  if (!m->g.ns) return fail(m, VL2_E_ARG, "the mesh has no passive scalars");
  const long long n = (long long)m->g.ns * ncells(m->g);
  const double* dc = c;
  if (where == VL2_HOST) {
    vl2_status st;
    if ((st = copy_in(m, m->a.stage, c, n, where)) != VL2_OK) return st;
    dc = m->a.stage;
  }
  VL2_CHECK(m, vl2::launch_scatter_scalars(m->g, m->a, dc, m->st));
  ++m->launches;
  VL2_CHECK(m, k_ghosts(m, 0));
  m->w_valid = false;
  m->dt_pending = false;
  return sync(m);
}

vl2_status vl2_set_forcing(vl2_mesh* m, const double* a, int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (bad_where(where)) return fail(m, VL2_E_ARG, "bad where");
  if (!m->acc_store) return fail(m, VL2_E_STATE, "the mesh was created without params.forcing");
  if (!a) {
    m->a.acc = nullptr;
    return VL2_OK;
  }
  const double* da = a;
  if (where == VL2_HOST) {
    vl2_status st;
    if ((st = copy_in(m, m->a.stage, a, 3 * (size_t)ncells(m->g), where)) != VL2_OK) return st;
    da = m->a.stage;
  }
  VL2_CHECK(m, vl2::launch_scatter_forcing(m->g, m->acc_store, da, m->st));
  ++m->launches;
  m->a.acc = m->acc_store;
  return sync(m);
}

vl2_status vl2_get_scalars(vl2_mesh* m, double* out, int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!out || bad_where(where)) return fail(m, VL2_E_ARG, "NULL output or bad where");
  if (!m->g.ns) return fail(m, VL2_E_ARG, "the mesh has no passive scalars");
  const long long n = (long long)m->g.ns * ncells(m->g);
  if (where == VL2_DEVICE) {
    VL2_CHECK(m, vl2::launch_gather_scalars(m->g, m->a, out, m->st));
    ++m->launches;
    return VL2_OK;
  }
  VL2_CHECK(m, vl2::launch_gather_scalars(m->g, m->a, m->a.stage, m->st));
  ++m->launches;
  vl2_status st = copy_out(m, out, m->a.stage, n);
  if (st != VL2_OK) return st;
  return sync(m);
}

vl2_status vl2_set_cons(vl2_mesh* m, const double* u, const double* b1, const double* b2, const double* b3, int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!u || !b1 || !b2 || !b3 || bad_where(where)) return fail(m, VL2_E_ARG, "NULL input or bad where");
  const Geom& g = m->g;
  const long long nc = ncells(g);
  const long long n1 = (long long)(g.N[0] + 1) * g.N[1] * g.N[2];
  const long long n2 = (long long)g.N[0] * (g.N[1] + 1) * g.N[2];
  const long long n3 = (long long)g.N[0] * g.N[1] * (g.N[2] + 1);
  const double *du = u, *d1 = b1, *d2 = b2, *d3 = b3;
  if (where == VL2_HOST) {
    double* s = m->a.stage;
    vl2_status st;
    if ((st = copy_in(m, s, u, 5 * nc, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc, b1, n1, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1, b2, n2, where)) != VL2_OK) return st;
    if ((st = copy_in(m, s + 5 * nc + n1 + n2, b3, n3, where)) != VL2_OK) return st;
    du = s;
    d1 = s + 5 * nc;
    d2 = d1 + n1;
    d3 = d2 + n2;
  }
  VL2_CHECK(m, vl2::launch_scatter_cons(g, m->a, du, d1, d2, d3, m->st));
  ++m->launches;
  VL2_CHECK(m, k_ghosts(m, 0));
  m->initialized = true;
  m->w_valid = false;
  m->dt_pending = false;
  if (where == VL2_HOST) return sync(m);
  return VL2_OK;
}

}  // extern "C"

namespace {

// What the reverse sweep of one VL2 cycle reads: both stages' primitives (all cells), face mass fluxes (with
// the smoothed CT weight also their face EMFs F[B_t1], F[B_t2]; `mstride` between blocks, the EMF components
// at +box and +2 box) and the face fields of both stages.
struct CycleInputs {
  const double* w0;      // predictor primitives W(U^n): [nblk][8][box]
  const double* w1;      // corrector primitives W(U^{n+1/2})
  const double* m1[3];   // predictor face mass fluxes (per sweep direction)
  const double* m2[3];   // corrector face mass fluxes
  long long m1_stride, m2_stride, m2_e5, m2_e6;
  const double* b0[3];   // face fields of U^n
  const double* b1[3];   // face fields of U^{n+1/2}
};

// Reverse sweep of one VL2 cycle from its recorded inputs: the transposes of the corrector, then of the
// predictor, each as update, upwind-CT EMFs, Riemann fluxes (with PLM), cons->prim, ghost exchange.
vl2_status vjp_reverse(vl2_mesh* m, double dt, const CycleInputs& in, const double* lam_u, const double* lam_b1,
                       const double* lam_b2, const double* lam_b3, double* out_u, double* out_b1, double* out_b2,
                       double* out_b3) {
  const Geom& g = m->g;
  const vl2::AdjArrays& j = m->adj;
  cudaStream_t st = m->st;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  for (int r = 0; r < 2; ++r) {
    VL2_CHECK(m, cudaMemsetAsync(j.lu[r], 0, 5 * per, st));
    for (int d = 0; d < 3; ++d) VL2_CHECK(m, cudaMemsetAsync(j.lb[r][d], 0, per, st));
  }
  VL2_CHECK(m, cudaMemsetAsync(j.lw, 0, 8 * per, st));
  VL2_CHECK(m, vl2::adj_scatter_out(g, j, lam_u, lam_b1, lam_b2, lam_b3, st));
  // corrector: U0 <- U0 + dt L_PLM(U1)
  VL2_CHECK(m, vl2::adj_update(g, j, 0, 0, dt, st));
  VL2_CHECK(m, vl2::adj_ct(g, j, in.w1, in.m2, in.m2_stride, in.m2_e5, in.m2_e6, st));
  VL2_CHECK(m, vl2::adj_flux_halo(g, j, st));
  VL2_CHECK(m, vl2::adj_fluxes(g, j, vl2::REC_PLM, m->p.riemann, in.w1, in.b1, 1, st));
  VL2_CHECK(m, vl2::adj_prim(g, j, in.w1, 1, st));
  VL2_CHECK(m, vl2::adj_ghosts(g, j, 1, st));
  // predictor: U1 = U0 + dt/2 L_DC(U0)
  VL2_CHECK(m, cudaMemsetAsync(j.lw, 0, 8 * per, st));
  VL2_CHECK(m, vl2::adj_update(g, j, 1, 0, 0.5 * dt, st));
  VL2_CHECK(m, vl2::adj_ct(g, j, in.w0, in.m1, in.m1_stride, g.box, 2 * g.box, st));
  VL2_CHECK(m, vl2::adj_flux_halo(g, j, st));
  VL2_CHECK(m, vl2::adj_fluxes(g, j, vl2::REC_DC, m->p.riemann, in.w0, in.b0, 0, st));
  VL2_CHECK(m, vl2::adj_prim(g, j, in.w0, 0, st));
  VL2_CHECK(m, vl2::adj_ghosts(g, j, 0, st));
  VL2_CHECK(m, vl2::adj_gather_in(g, j, out_u, out_b1, out_b2, out_b3, st));
  // scatter, 2 x (update, CT, halo transpose, 3 x 2 flux (+3 slope passes for PLM), prim, 3 x 2 ghost passes),
  // gather
  m->launches += 32 + 3 + (g.flux_halo ? 0 : 2);
  return VL2_OK;
}

vl2_status vjp_args(vl2_mesh* m, double dt, const void* a, const void* b, const void* c, const void* d,
                    const void* e, const void* f, const void* g, const void* h) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!a || !b || !c || !d || !e || !f || !g || !h) return fail(m, VL2_E_ARG, "NULL argument");
  if (!m->has_adj) return fail(m, VL2_E_STATE, "mesh was created without params.adjoint");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(m, VL2_E_ARG, "dt must be finite and positive");
  return VL2_OK;
}

// Tape of one recorded cycle, carved from the caller's buffer (doubles, each part 256-byte aligned).
struct Tape {
  double *w0, *w1, *b0[3], *b1[3], *m1[3], *m2[3];
  long long mk;  // components kept per face: 1 (mass flux), 3 with the smoothed CT weight (+ two face EMFs)
  size_t bytes;
};
Tape carve_tape(const vl2_mesh* m, void* base) {
  const Geom& g = m->g;
  Tape t;
  t.mk = g.ct_delta > 0.0 ? 3 : 1;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  size_t o = 0;
  char* p = static_cast<char*>(base);
  auto take = [&](size_t nvar) {
    double* r = p ? reinterpret_cast<double*>(p + o) : nullptr;
    o = align256(o + nvar * per);
    return r;
  };
  t.w0 = take(8);
  t.w1 = take(8);
  for (int d = 0; d < 3; ++d) t.b0[d] = take(1);
  for (int d = 0; d < 3; ++d) t.b1[d] = take(1);
  for (int d = 0; d < 3; ++d) t.m1[d] = take(t.mk);
  for (int d = 0; d < 3; ++d) t.m2[d] = take(t.mk);
  t.bytes = o;
  return t;
}

// the face mass fluxes (and with the smoothed CT weight the two face EMFs) of the current flux arrays
vl2_status keep_mass_fluxes(vl2_mesh* m, double* const* dst, long long mk) {
  const Geom& g = m->g;
  for (int d = 0; d < 3; ++d) {
    VL2_CHECK(m, cudaMemcpy2DAsync(dst[d], mk * g.box * sizeof(double), m->a.f[d], 7 * g.box * sizeof(double),
                                   g.box * sizeof(double), g.nblk, cudaMemcpyDeviceToDevice, m->st));
    if (mk == 3)
      VL2_CHECK(m, cudaMemcpy2DAsync(dst[d] + g.box, mk * g.box * sizeof(double),
                                     static_cast<const double*>(m->a.f[d]) + 5 * g.box, 7 * g.box * sizeof(double),
                                     2 * g.box * sizeof(double), g.nblk, cudaMemcpyDeviceToDevice, m->st));
  }
  return VL2_OK;
}

}  // namespace

extern "C" {

vl2_status vl2_step_vjp(vl2_mesh* m, double dt, const double* lam_u, const double* lam_b1, const double* lam_b2,
                        const double* lam_b3, double* out_u, double* out_b1, double* out_b2, double* out_b3) {
  vl2_status s = vjp_args(m, dt, lam_u, lam_b1, lam_b2, lam_b3, out_u, out_b1, out_b2, out_b3);
  if (s != VL2_OK) return s;
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims/vl2_set_cons has not been called");
  const Geom& g = m->g;
  const vl2::AdjArrays& j = m->adj;
  cudaStream_t st = m->st;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  // forward recompute of the cycle's intermediates from x (register 0 is not written)
  VL2_CHECK(m, k_prim(m, 0, false));
  VL2_CHECK(m, cudaMemcpyAsync(j.w0, m->a.w, 8 * per, cudaMemcpyDeviceToDevice, st));
  VL2_CHECK(m, k_fluxes(m, 0, VL2_DC));
  // the predictor's mass fluxes (its upwind choices), and with the smoothed CT weight its face EMFs
  const long long mk = g.ct_delta > 0.0 ? 3 : 1;
  s = keep_mass_fluxes(m, j.m1, mk);
  if (s != VL2_OK) return s;
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update(m, 0, 1, 0.5 * dt));
  VL2_CHECK(m, k_ghosts(m, 1));
  VL2_CHECK(m, k_prim(m, 1, false));
  VL2_CHECK(m, k_fluxes(m, 1, VL2_PLM));
  m->w_valid = false;
  m->dt_pending = false;
  CycleInputs in;
  in.w0 = j.w0;
  in.w1 = static_cast<const double*>(m->a.w);
  for (int d = 0; d < 3; ++d) {
    in.m1[d] = j.m1[d];
    in.m2[d] = static_cast<const double*>(m->a.f[d]);
    in.b0[d] = m->a.b[0][d];
    in.b1[d] = m->a.b[1][d];
  }
  in.m1_stride = mk * g.box;
  in.m2_stride = 7 * g.box;
  in.m2_e5 = 5 * g.box;
  in.m2_e6 = 6 * g.box;
  return vjp_reverse(m, dt, in, lam_u, lam_b1, lam_b2, lam_b3, out_u, out_b1, out_b2, out_b3);
}

vl2_status vl2_tape_bytes(const vl2_mesh* m, size_t* bytes) {
  if (!m || !bytes) return fail(nullptr, VL2_E_ARG, "NULL argument");
  if (!m->has_adj) return fail(nullptr, VL2_E_STATE, "mesh was created without params.adjoint");
  *bytes = carve_tape(m, nullptr).bytes;
  return VL2_OK;
}

vl2_status vl2_step_record(vl2_mesh* m, double dt, void* tape) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!tape || ((uintptr_t)tape & 255u)) return fail(m, VL2_E_ARG, "tape must be non-NULL and 256-byte aligned");
  if (!m->has_adj) return fail(m, VL2_E_STATE, "mesh was created without params.adjoint");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims/vl2_set_cons has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(m, VL2_E_ARG, "dt must be finite and positive");
  const Geom& g = m->g;
  const Tape t = carve_tape(m, tape);
  cudaStream_t st = m->st;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  vl2_status s = ensure_prims(m);
  if (s != VL2_OK) return s;
  // The VL2 cycle of vl2_step, keeping what its adjoint reads.  The predictor writes its face field, and
  // cons->prim the corrector's primitives, straight into the tape: the mesh's own register-1 field and
  // primitive arrays are next needed by the following cycle, so for this one the mesh points at the tape
  // (restored on every exit).  The TMA-staged sweeps' tensor maps describe the mesh's own primitive array,
  // so with them the primitives are copied instead.
  struct Redirect {
    vl2_mesh* m;
    void* w;
    double* b1[3];
    void restore() {
      m->a.w = w;
      for (int d = 0; d < 3; ++d) m->a.b[1][d] = b1[d];
    }
    ~Redirect() { restore(); }
  } keep{m, m->a.w, {m->a.b[1][0], m->a.b[1][1], m->a.b[1][2]}};
  const bool w_direct = !vl2::flux_tma_applies(m->view(), vl2::REC_PLM, m->fs, m->max_mb());
  VL2_CHECK(m, cudaMemcpyAsync(t.w0, m->a.w, 8 * per, cudaMemcpyDeviceToDevice, st));
  for (int d = 0; d < 3; ++d) VL2_CHECK(m, cudaMemcpyAsync(t.b0[d], m->a.b[0][d], per, cudaMemcpyDeviceToDevice, st));
  VL2_CHECK(m, k_fluxes(m, 0, VL2_DC));
  if ((s = keep_mass_fluxes(m, t.m1, t.mk)) != VL2_OK) return s;
  VL2_CHECK(m, k_emfs(m));
  for (int d = 0; d < 3; ++d) m->a.b[1][d] = t.b1[d];
  VL2_CHECK(m, k_update(m, 0, 1, 0.5 * dt));
  VL2_CHECK(m, k_ghosts(m, 1));
  if (w_direct) m->a.w = t.w1;
  VL2_CHECK(m, k_prim(m, 1, false));
  if (!w_direct) VL2_CHECK(m, cudaMemcpyAsync(t.w1, m->a.w, 8 * per, cudaMemcpyDeviceToDevice, st));
  VL2_CHECK(m, k_fluxes(m, 1, VL2_PLM));
  if ((s = keep_mass_fluxes(m, t.m2, t.mk)) != VL2_OK) return s;
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update(m, 0, 0, dt, 1.0, 0.0, 1));
  keep.restore();  // the mesh's own arrays again
  VL2_CHECK(m, k_ghosts(m, 0));
  VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), st));
  VL2_CHECK(m, k_prim(m, 0, true));
  m->w_valid = true;
  m->dt_pending = true;
  return VL2_OK;
}

vl2_status vl2_step_vjp_recorded(vl2_mesh* m, double dt, const void* tape, const double* lam_u, const double* lam_b1,
                                 const double* lam_b2, const double* lam_b3, double* out_u, double* out_b1,
                                 double* out_b2, double* out_b3) {
  vl2_status s = vjp_args(m, dt, lam_u, lam_b1, lam_b2, lam_b3, out_u, out_b1, out_b2, out_b3);
  if (s != VL2_OK) return s;
  if (!tape || ((uintptr_t)tape & 255u)) return fail(m, VL2_E_ARG, "tape must be non-NULL and 256-byte aligned");
  const Geom& g = m->g;
  const Tape t = carve_tape(m, const_cast<void*>(tape));
  CycleInputs in;
  in.w0 = t.w0;
  in.w1 = t.w1;
  for (int d = 0; d < 3; ++d) {
    in.m1[d] = t.m1[d];
    in.m2[d] = t.m2[d];
    in.b0[d] = t.b0[d];
    in.b1[d] = t.b1[d];
  }
  in.m1_stride = in.m2_stride = t.mk * g.box;
  in.m2_e5 = g.box;
  in.m2_e6 = 2 * g.box;
  return vjp_reverse(m, dt, in, lam_u, lam_b1, lam_b2, lam_b3, out_u, out_b1, out_b2, out_b3);
}

vl2_status vl2_debug_riemann_vjp(int riemann, long long n, const double* wl, const double* wr, const double* bn,
                                 const double* lf, double gamma, double* out, void* stream) {
  if (n < 0 || (n > 0 && (!wl || !wr || !bn || !lf || !out))) return fail(nullptr, VL2_E_ARG, "bad pointer or n < 0");
  if (riemann != VL2_HLLD && riemann != VL2_HLLE) return fail(nullptr, VL2_E_ARG, "riemann must be VL2_HLLD or VL2_HLLE");
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(nullptr, VL2_E_ARG, "gamma must be > 1");
  const cudaError_t e = vl2::riemann_vjp_points(riemann == VL2_HLLD ? vl2::RS_HLLD : vl2::RS_HLLE, n, wl, wr, bn, lf,
                                                gamma, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(nullptr, VL2_E_CUDA, cudaGetErrorString(e));
  return VL2_OK;
}

vl2_status vl2_prims_vjp(vl2_mesh* m, const double* w, const double* lam_u, double* lam_w) {
  if (!m || !w || !lam_u || !lam_w) return fail(m, VL2_E_ARG, "NULL argument");
  VL2_CHECK(m, vl2::prims_vjp(ncells(m->g), m->g.igm1, w, lam_u, lam_w, m->st));
  ++m->launches;
  return VL2_OK;
}

vl2_status vl2_fill_ghosts(vl2_mesh* m) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  VL2_CHECK(m, k_ghosts(m, 0));
  m->w_valid = false;
  m->dt_pending = false;
  return VL2_OK;
}

namespace {
// One cycle of RK1 / RK2 / RK3 in the 2S form (Sec. 3.2.3, eq. rk-2s): u^(0) = U^n in register 0,
// u^(1) in register 1.  u^(1) = 0 + delta_0 u^(0) = U^n before the first stage (delta_s = 0 after it);
// each stage s then forms the fluxes of u^(0) (donor cell for RK1, PLM otherwise) and updates
// u^(0) = gamma_s0 u^(0) + gamma_s1 u^(1) + beta_s dt L(u^(0)) in place, followed by the ghost exchange and
// cons->prim (the last one with the CFL reduction).
struct RkStage {
  double g0, g1, beta;
};
vl2_status step_rk(vl2_mesh* m, double dt) {
  static const RkStage rk1[1] = {{0.0, 1.0, 1.0}};
  static const RkStage rk2[2] = {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}};
  static const RkStage rk3[3] = {{0.0, 1.0, 1.0}, {0.25, 0.75, 0.25}, {2.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0}};
  const RkStage* st = m->p.integrator == VL2_INT_RK1 ? rk1 : (m->p.integrator == VL2_INT_RK2 ? rk2 : rk3);
  const int ns = m->p.integrator == VL2_INT_RK1 ? 1 : (m->p.integrator == VL2_INT_RK2 ? 2 : 3);
  const int recon = m->p.integrator == VL2_INT_RK1 ? VL2_DC : m->rec();
  const Geom& g = m->g;
  const size_t per = (size_t)g.nblk * g.box * sizeof(double);
  // u^(1) = U^n (every element, so that register 1 is a complete copy)
  VL2_CHECK(m, cudaMemcpyAsync(m->a.u[1], m->a.u[0], 5 * per, cudaMemcpyDeviceToDevice, m->st));
  for (int d = 0; d < 3; ++d)
    VL2_CHECK(m, cudaMemcpyAsync(m->a.b[1][d], m->a.b[0][d], per, cudaMemcpyDeviceToDevice, m->st));
  if (g.ns)
    VL2_CHECK(m, cudaMemcpyAsync(m->a.s[1], m->a.s[0], g.ns * per, cudaMemcpyDeviceToDevice, m->st));
  for (int k = 0; k < ns; ++k) {
    if (k > 0) VL2_CHECK(m, k_prim(m, 0, false));
    VL2_CHECK(m, k_fluxes(m, 0, recon));
    VL2_CHECK(m, k_scalar_fluxes(m, recon));
    VL2_CHECK(m, k_emfs(m));
    VL2_CHECK(m, k_update(m, 0, 0, st[k].beta * dt, st[k].g0, st[k].g1));
    VL2_CHECK(m, k_scalar_update(m, 0, 0, st[k].beta * dt, st[k].g0, st[k].g1));
    VL2_CHECK(m, k_ghosts(m, 0));
  }
  VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), m->st));
  VL2_CHECK(m, k_prim(m, 0, true));
  m->w_valid = true;
  m->dt_pending = true;
  return VL2_OK;
}
}  // namespace

vl2_status vl2_step(vl2_mesh* m, double dt) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims has not been called");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(m, VL2_E_ARG, "dt must be finite and positive");
  vl2_status s = ensure_prims(m);
  if (s != VL2_OK) return s;
  if (m->p.integrator != VL2_INT_VL2) return step_rk(m, dt);
  // predictor: U* = U^n + (dt/2) L_DC(U^n) into register 1 (Sec. 3.2.3, VL2)
  VL2_CHECK(m, k_fluxes(m, 0, VL2_DC));
  VL2_CHECK(m, k_scalar_fluxes(m, VL2_DC));
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update(m, 0, 1, 0.5 * dt));
  VL2_CHECK(m, k_scalar_update(m, 0, 1, 0.5 * dt));
  VL2_CHECK(m, k_ghosts(m, 1));
  VL2_CHECK(m, k_prim(m, 1, false));
  // corrector: U^{n+1} = U^n + dt L_PLM(U*) (or L_PPM) in place in register 0
  VL2_CHECK(m, k_fluxes(m, 1, m->rec()));
  VL2_CHECK(m, k_scalar_fluxes(m, m->rec()));
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update(m, 0, 0, dt, 1.0, 0.0, 1));  // the fluxes (and forcing sources) come from register 1
  VL2_CHECK(m, k_scalar_update(m, 0, 0, dt));
  VL2_CHECK(m, k_ghosts(m, 0));
  // primitives of U^{n+1} for the next cycle, with the CFL reduction fused in
  VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), m->st));
  VL2_CHECK(m, k_prim(m, 0, true));
  m->w_valid = true;
  m->dt_pending = true;
  return VL2_OK;
}

vl2_status vl2_step_cfl(vl2_mesh* m) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims has not been called");
  if (m->p.integrator != VL2_INT_VL2 || m->g.ns)
    return fail(m, VL2_E_STATE, "vl2_step_cfl runs the VL2 integrator without passive scalars");
  if (!m->dt_pending) {  // the CFL rate of the current state (vl2_step leaves it behind)
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), m->st));
    VL2_CHECK(m, k_prim(m, 0, true));
    m->w_valid = true;
  }
  VL2_CHECK(m, vl2::launch_mesh_dt(m->a.scal, m->p.cfl, m->ddt, m->st));
  ++m->launches;
  // the cycle of vl2_step with h = beta dt read on the device
  VL2_CHECK(m, k_fluxes(m, 0, VL2_DC));
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update_ddt(m, 0, 1, 0.5));
  VL2_CHECK(m, k_ghosts(m, 1));
  VL2_CHECK(m, k_prim(m, 1, false));
  VL2_CHECK(m, k_fluxes(m, 1, m->rec()));
  VL2_CHECK(m, k_emfs(m));
  VL2_CHECK(m, k_update_ddt(m, 0, 0, 1.0, 1));
  VL2_CHECK(m, k_ghosts(m, 0));
  VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), m->st));
  VL2_CHECK(m, k_prim(m, 0, true));
  m->w_valid = true;
  m->dt_pending = true;
  return VL2_OK;
}

vl2_status vl2_last_dt(vl2_mesh* m, double* dt_out) {
  if (!m || !dt_out) return fail(m, VL2_E_ARG, "NULL argument");
  double dt = 0.0;
  unsigned long long sc[5];
  VL2_CHECK(m, cudaMemcpyAsync(&dt, m->ddt, sizeof(dt), cudaMemcpyDeviceToHost, m->st));
  VL2_CHECK(m, cudaMemcpyAsync(sc, m->a.scal, sizeof(sc), cudaMemcpyDeviceToHost, m->st));
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  *dt_out = dt;
  if (sc[vl2::SC_MISMATCH_ASYNC]) {
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MISMATCH_ASYNC, 0, sizeof(unsigned long long), m->st));
    return fail(m, VL2_E_ARG, "periodic duplicate faces (face N and face 0) differed in vl2_set_prims_async");
  }
  if (sc[vl2::SC_TIMEOUT]) {
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_TIMEOUT, 0, sizeof(unsigned long long), m->st));
    return fail(m, VL2_E_TIMEOUT, "a TMA tile copy did not land within its bounded wait; the step is incomplete");
  }
  const unsigned long long floors = sc[vl2::SC_FLOORS];
  const bool fired = floors > m->floors_seen;
  m->floors_seen = floors;
  if (!std::isfinite(dt) || !(dt > 0.0)) return fail(m, VL2_E_NONPHYS, "time step is not finite and positive");
  if (fired) return fail(m, VL2_E_NONPHYS, "a density or pressure floor fired");
  return VL2_OK;
}

vl2_status vl2_new_dt(vl2_mesh* m, double* dt_out) {
  if (!m || !dt_out) return fail(m, VL2_E_ARG, "NULL argument");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims has not been called");
  if (!m->dt_pending) {
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MAXRATE, 0, sizeof(unsigned long long), m->st));
    VL2_CHECK(m, k_prim(m, 0, true));
    m->w_valid = true;
    m->dt_pending = true;
  }
  unsigned long long sc[5];
  VL2_CHECK(m, cudaMemcpyAsync(sc, m->a.scal, sizeof(sc), cudaMemcpyDeviceToHost, m->st));
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  if (sc[vl2::SC_MISMATCH_ASYNC]) {
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_MISMATCH_ASYNC, 0, sizeof(unsigned long long), m->st));
    return fail(m, VL2_E_ARG, "periodic duplicate faces (face N and face 0) differed in vl2_set_prims_async");
  }
  if (sc[vl2::SC_TIMEOUT]) {
    VL2_CHECK(m, cudaMemsetAsync(m->a.scal + vl2::SC_TIMEOUT, 0, sizeof(unsigned long long), m->st));
    return fail(m, VL2_E_TIMEOUT, "a TMA tile copy did not land within its bounded wait; the step is incomplete");
  }
  double rate;
  std::memcpy(&rate, &sc[vl2::SC_MAXRATE], sizeof(rate));
  const double dt = m->p.cfl / rate;
  *dt_out = dt;
  const unsigned long long floors = sc[vl2::SC_FLOORS];
  const bool fired = floors > m->floors_seen;
  m->floors_seen = floors;
  if (!std::isfinite(dt) || !(dt > 0.0)) return fail(m, VL2_E_NONPHYS, "time step is not finite and positive");
  if (fired) return fail(m, VL2_E_NONPHYS, "a density or pressure floor fired");
  return VL2_OK;
}

vl2_status vl2_get_cons(vl2_mesh* m, double* u, double* b1, double* b2, double* b3, int where) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (bad_where(where)) return fail(m, VL2_E_ARG, "bad where");
  const Geom& g = m->g;
  if (where == VL2_DEVICE) {
    VL2_CHECK(m, vl2::launch_gather_cons(g, m->a, u, b1, b2, b3, m->st));
    ++m->launches;
    return VL2_OK;
  }
  const long long nc = ncells(g);
  const long long n1 = (long long)(g.N[0] + 1) * g.N[1] * g.N[2];
  const long long n2 = (long long)g.N[0] * (g.N[1] + 1) * g.N[2];
  const long long n3 = (long long)g.N[0] * g.N[1] * (g.N[2] + 1);
  double* s = m->a.stage;
  double *su = u ? s : nullptr, *s1 = b1 ? s + 5 * nc : nullptr, *s2 = b2 ? s + 5 * nc + n1 : nullptr,
         *s3 = b3 ? s + 5 * nc + n1 + n2 : nullptr;
  VL2_CHECK(m, vl2::launch_gather_cons(g, m->a, su, s1, s2, s3, m->st));
  ++m->launches;
  vl2_status st;
  if (u && (st = copy_out(m, u, su, 5 * nc)) != VL2_OK) return st;
  if (b1 && (st = copy_out(m, b1, s1, n1)) != VL2_OK) return st;
  if (b2 && (st = copy_out(m, b2, s2, n2)) != VL2_OK) return st;
  if (b3 && (st = copy_out(m, b3, s3, n3)) != VL2_OK) return st;
  return sync(m);
}

vl2_status vl2_get_prims(vl2_mesh* m, double* w, int where) {
  if (!m || !w) return fail(m, VL2_E_ARG, "NULL argument");
  if (bad_where(where)) return fail(m, VL2_E_ARG, "bad where");
  vl2_status s = ensure_prims(m);
  if (s != VL2_OK) return s;
  const long long nc = ncells(m->g);
  double* dst = where == VL2_DEVICE ? w : m->a.stage;
  VL2_CHECK(m, vl2::launch_gather_prims(m->g, m->a, dst, m->st));
  ++m->launches;
  if (where == VL2_DEVICE) return VL2_OK;
  if ((s = copy_out(m, w, dst, 8 * nc)) != VL2_OK) return s;
  return sync(m);
}

vl2_status vl2_divb_norm(vl2_mesh* m, double* out) {
  if (!m || !out) return fail(m, VL2_E_ARG, "NULL argument");
  VL2_CHECK(m, vl2::launch_divb(m->g, m->a, m->dres, m->st));
  double r[2];
  VL2_CHECK(m, cudaMemcpyAsync(r, m->dres, sizeof(r), cudaMemcpyDeviceToHost, m->st));
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  const Geom& g = m->g;
  const double hmin = std::fmin(g.dx[0], std::fmin(g.dx[1], g.dx[2]));
  const double rms = std::sqrt(r[1] / (double)ncells(g));
  *out = r[0] * hmin / std::fmax(rms, 1e-300);
  return VL2_OK;
}

vl2_status vl2_totals(vl2_mesh* m, double out[8]) {
  if (!m || !out) return fail(m, VL2_E_ARG, "NULL argument");
  VL2_CHECK(m, vl2::launch_totals(m->g, m->a, m->dres, m->st));
  VL2_CHECK(m, cudaMemcpyAsync(out, m->dres, 8 * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  return sync(m);
}

vl2_status vl2_floor_count(vl2_mesh* m, long long* out) {
  if (!m || !out) return fail(m, VL2_E_ARG, "NULL argument");
  unsigned long long v = 0;
  VL2_CHECK(m, cudaMemcpyAsync(&v, m->a.scal + vl2::SC_FLOORS, sizeof(v), cudaMemcpyDeviceToHost, m->st));
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  *out = (long long)v;
  return VL2_OK;
}

static vl2_status gather_out(vl2_mesh* m, int kind, int dir, double* out, long long n, int where) {
  double* dst = where == VL2_DEVICE ? out : m->a.stage;
  if (kind == 0)
    VL2_CHECK(m, vl2::launch_gather_fluxes(m->g, m->a, dir, dst, m->st));
  else
    VL2_CHECK(m, vl2::launch_gather_emfs(m->g, m->a, dir, dst, m->st));
  if (where == VL2_DEVICE) return VL2_OK;
  vl2_status s = copy_out(m, out, dst, (size_t)n);
  if (s != VL2_OK) return s;
  return sync(m);  // the staging buffer is reused by the next direction
}

vl2_status vl2_debug_fluxes(vl2_mesh* m, int recon, double* fx, double* fy, double* fz, int where) {
  if (!m || !fx || !fy || !fz) return fail(m, VL2_E_ARG, "NULL argument");
  if (bad_where(where) || (recon != VL2_DC && recon != VL2_PLM && recon != VL2_PLM_CHAR &&
                              !((recon == VL2_PPM || recon == VL2_PPM_CHAR) && m->g.ng >= 3)))
    return fail(m, VL2_E_ARG, "bad where or recon (PPM needs ng = 3)");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims has not been called");
  vl2_status s = ensure_prims(m);
  if (s != VL2_OK) return s;
  VL2_CHECK(m, k_fluxes(m, 0, recon));
  const Geom& g = m->g;
  double* outs[3] = {fx, fy, fz};
  for (int d = 0; d < 3; ++d) {
    long long gd[3] = {g.N[0], g.N[1], g.N[2]};
    gd[d] += 1;
    if ((s = gather_out(m, 0, d, outs[d], 7 * gd[0] * gd[1] * gd[2], where)) != VL2_OK) return s;
  }
  return VL2_OK;
}

vl2_status vl2_debug_emfs(vl2_mesh* m, int recon, double* e1, double* e2, double* e3, int where) {
  if (!m || !e1 || !e2 || !e3) return fail(m, VL2_E_ARG, "NULL argument");
  if (bad_where(where) || (recon != VL2_DC && recon != VL2_PLM && recon != VL2_PLM_CHAR &&
                              !((recon == VL2_PPM || recon == VL2_PPM_CHAR) && m->g.ng >= 3)))
    return fail(m, VL2_E_ARG, "bad where or recon (PPM needs ng = 3)");
  if (!m->initialized) return fail(m, VL2_E_STATE, "vl2_set_prims has not been called");
  vl2_status s = ensure_prims(m);
  if (s != VL2_OK) return s;
  VL2_CHECK(m, k_fluxes(m, 0, recon));
  VL2_CHECK(m, k_emfs(m));
  const Geom& g = m->g;
  double* outs[3] = {e1, e2, e3};
  for (int e = 0; e < 3; ++e) {
    long long gd[3] = {g.N[0] + 1, g.N[1] + 1, g.N[2] + 1};
    gd[e] -= 1;
    if ((s = gather_out(m, 1, e, outs[e], gd[0] * gd[1] * gd[2], where)) != VL2_OK) return s;
  }
  return VL2_OK;
}

vl2_status vl2_profile(vl2_mesh* m, int enable) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  m->prof = enable != 0;
  return VL2_OK;
}

vl2_status vl2_profile_read(vl2_mesh* m, int kind, double* ms, long long* launches, long long* units) {
  if (!m || !ms || !launches || !units) return fail(m, VL2_E_ARG, "NULL argument");
  if (kind < 0 || kind >= VL2_K_COUNT) return fail(m, VL2_E_ARG, "bad kernel kind");
  vl2_status s = sync(m);
  if (s != VL2_OK) return s;
  for (const auto& r : m->recs) {
    float t = 0.f;
    VL2_CHECK(m, cudaEventElapsedTime(&t, r.a, r.b));
    m->acc_ms[r.kind] += t;
    m->acc_n[r.kind] += 1;
    m->acc_units[r.kind] += r.units;
  }
  m->recs.clear();
  m->pool_used = 0;
  *ms = m->acc_ms[kind];
  *launches = m->acc_n[kind];
  *units = m->acc_units[kind];
  m->acc_ms[kind] = 0.0;
  m->acc_n[kind] = m->acc_units[kind] = 0;
  return VL2_OK;
}

vl2_status vl2_launch_count(const vl2_mesh* m, long long* n) {
  if (!m || !n) return fail(nullptr, VL2_E_ARG, "NULL argument");
  *n = m->launches;
  return VL2_OK;
}

vl2_status vl2_set_flux_shape(vl2_mesh* m, int dc_threads, int plm_lines, int tma) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if ((dc_threads != 64 && dc_threads != 128 && dc_threads != 256) ||
      (plm_lines != 4 && plm_lines != 8 && plm_lines != 16) || (tma != 0 && tma != 1))
    return fail(m, VL2_E_ARG, "dc_threads must be 64, 128 or 256, plm_lines 4, 8 or 16, tma 0 or 1");
  m->fs.dc_threads = dc_threads;
  m->fs.plm_lines = plm_lines;
  m->fs.plm_tma = tma;
  vl2::prime_flux_tma(m->view(), m->rec(), m->p.riemann == VL2_HLLD ? vl2::RS_HLLD : vl2::RS_HLLE, m->fs, m->max_mb(), m->st);
  return VL2_OK;
}

vl2_status vl2_get_flux_shape(const vl2_mesh* m, int* dc_threads, int* plm_lines, int* tma, int* tma_active) {
  if (!m) return fail(nullptr, VL2_E_ARG, "mesh is NULL");
  if (dc_threads) *dc_threads = m->fs.dc_threads;
  if (plm_lines) *plm_lines = m->fs.plm_lines;
  if (tma) *tma = m->fs.plm_tma;
  if (tma_active) *tma_active = vl2::flux_tma_applies(m->view(), vl2::REC_PLM, m->fs, m->max_mb()) && m->rec() == VL2_PLM;
  return VL2_OK;
}

const char* vl2_last_error(const vl2_mesh* mesh) { return mesh ? mesh->err.c_str() : g_err.c_str(); }

}  // extern "C"

/* =============================================================================================
 * Batched form: many independent meshes (boxes) advanced by one launch per kernel over a (box, tile)
 * work list; per-box CFL time steps stay on the device; K cycles are captured in one CUDA graph.
 * =========================================================================================== */
struct vl2_batch {
  enum { W_PRIM, W_GHOSTS, W_NODES, W_DC, W_PLM = W_DC + 3, W_HALO = W_PLM + 3, W_COUNT = W_HALO + 1 };
  std::vector<vl2_mesh*> meshes;
  int n = 0;
  cudaStream_t st = nullptr;
  vl2::MeshView* dviews = nullptr;
  double* ddt = nullptr;
  double* dcfl = nullptr;
  vl2::WorkItem* dwork[W_COUNT] = {nullptr};
  size_t cap[W_COUNT] = {0};
  int nwork[W_COUNT] = {0};
  vl2::FluxShape fs;
  int max_mb = 1;
  int riemann = VL2_HLLD;
  int recon = VL2_PLM;  // reconstruction of the corrector
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_steps = 0;
  long long launches = 0;
  // Graphs are captured and launched on a stream of the batch's own (the meshes' stream may be the legacy
  // default stream, which cannot be captured), ordered against the meshes' stream with two events.
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaStream_t cur = nullptr;  // stream the kernels of the current call go to
  std::string err;
  ~vl2_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace {

const int kDcCandidates[3] = {64, 128, 256};
const int kPlmCandidates[3] = {4, 8, 16};

vl2_status bfail(vl2_batch* b, vl2_status s, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_err = msg;
  return s;
}

#define VL2_BCHECK(b, call)                                                                              \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return bfail((b), VL2_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// tiles of kernel type w for one mesh under flux shape fs
long long batch_tiles(const vl2_mesh* m, int w, const vl2::FluxShape& fs, int max_mb) {
  const vl2::Geom& g = m->g;
  if (w == vl2_batch::W_PRIM) return vl2::tiles_prim(g);
  if (w == vl2_batch::W_GHOSTS) return vl2::tiles_ghosts(g);
  if (w == vl2_batch::W_NODES) return vl2::tiles_nodes(g);
  if (w == vl2_batch::W_HALO) return vl2::tiles_flux_halo(g);
  if (w < vl2_batch::W_PLM) return vl2::tiles_flux_dc(g, w - vl2_batch::W_DC, fs);
  const int d = w - vl2_batch::W_PLM;
  if (fs.plm_tma) return vl2::tiles_flux_tma(g, d, fs.plm_lines);  // set only where every mesh qualifies
  vl2::FluxShape f2 = fs;
  f2.plm_lines = vl2::plm_lines_for(g, d, fs, max_mb, m->rec());
  return vl2::tiles_flux_plm(g, d, f2);
}

// capacity of each work list: the most tiles any candidate launch shape produces
size_t batch_capacity(const std::vector<vl2_mesh*>& ms, int w, int max_mb) {
  size_t best = 0;
  for (int dc : kDcCandidates)
    for (int pl : kPlmCandidates)
      for (int tma = 0; tma < 2; ++tma) {
        vl2::FluxShape fs;
        fs.dc_threads = dc;
        fs.plm_lines = pl;
        fs.plm_tma = tma;
        size_t tot = 0;
        for (const vl2_mesh* m : ms) tot += (size_t)batch_tiles(m, w, fs, max_mb);
        best = std::max(best, tot);
      }
  return best;
}

// the TMA-staged PLM sweeps serve a batch only when every mesh of it qualifies under fs
bool batch_tma_ok(const vl2_batch* B, const vl2::FluxShape& fs) {
  for (const vl2_mesh* m : B->meshes)
    if (!vl2::flux_tma_applies(m->view(), B->recon, fs, B->max_mb)) return false;
  return true;
}

vl2_status batch_check(vl2_mesh* const* meshes, int n, std::string& msg) {
  if (!meshes || n <= 0) {
    msg = "meshes is NULL or n <= 0";
    return VL2_E_ARG;
  }
  for (int q = 0; q < n; ++q) {
    if (!meshes[q]) {
      msg = "NULL mesh in the batch";
      return VL2_E_ARG;
    }
    if (meshes[q]->p.integrator != VL2_INT_VL2 || meshes[q]->g.ns != 0) {
      msg = "the batched form runs the VL2 integrator without passive scalars";
      return VL2_E_ARG;
    }
    // one launch serves every mesh: the kernel variants (solver, precision, reconstruction, smoothed CT
    // or not) are chosen once, so the meshes must agree on them; the smoothed weight's delta is read per
    // mesh, but is required equal too so that a batch is one configuration
    if (meshes[q]->p.riemann != meshes[0]->p.riemann || meshes[q]->p.precision != meshes[0]->p.precision ||
        meshes[q]->rec() != meshes[0]->rec() || meshes[q]->g.ct_delta != meshes[0]->g.ct_delta) {
      msg = "all meshes of a batch need the same Riemann solver, precision, reconstruction and ct_delta";
      return VL2_E_ARG;
    }
  }
  return VL2_OK;
}

struct BatchPlan {
  size_t off_views, off_dt, off_cfl, off_work[vl2_batch::W_COUNT], total;
  size_t cap[vl2_batch::W_COUNT];
};

BatchPlan batch_plan(const std::vector<vl2_mesh*>& ms, int max_mb) {
  BatchPlan pl;
  size_t o = 0;
  pl.off_views = o;
  o = align256(o + ms.size() * sizeof(vl2::MeshView));
  pl.off_dt = o;
  o = align256(o + ms.size() * sizeof(double));
  pl.off_cfl = o;
  o = align256(o + ms.size() * sizeof(double));
  for (int w = 0; w < vl2_batch::W_COUNT; ++w) {
    pl.cap[w] = batch_capacity(ms, w, max_mb);
    pl.off_work[w] = o;
    o = align256(o + pl.cap[w] * sizeof(vl2::WorkItem));
  }
  pl.total = o;
  return pl;
}

// (re)build the work lists for the batch's flux shape and upload them
vl2_status batch_lists(vl2_batch* B) {
  for (int w = 0; w < vl2_batch::W_COUNT; ++w) {
    std::vector<vl2::WorkItem> list;
    for (int q = 0; q < B->n; ++q) {
      const long long t = batch_tiles(B->meshes[q], w, B->fs, B->max_mb);
      for (long long i = 0; i < t; ++i) list.push_back(vl2::WorkItem{q, (int)i});
    }
    if (list.size() > B->cap[w] || list.size() > (size_t)INT32_MAX) return bfail(B, VL2_E_ARG, "work list overflow");
    B->nwork[w] = (int)list.size();
    VL2_BCHECK(B, cudaMemcpyAsync(B->dwork[w], list.data(), list.size() * sizeof(vl2::WorkItem),
                                  cudaMemcpyHostToDevice, B->st));
  }
  VL2_BCHECK(B, cudaStreamSynchronize(B->st));
  return VL2_OK;
}

vl2::Dispatch disp(const vl2_batch* B, int w) {
  vl2::Dispatch d;
  d.views = B->dviews;
  d.work = B->dwork[w];
  d.nwork = B->nwork[w];
  return d;
}

// enqueue the flux launches of one reconstruction for every box
cudaError_t batch_fluxes(vl2_batch* B, int reg, int recon) {
  const vl2::MeshView v0 = B->meshes[0]->view();
  for (int d = 0; d < 3; ++d) {
    const vl2::Dispatch dd = disp(B, (recon == VL2_DC ? vl2_batch::W_DC : vl2_batch::W_PLM) + d);
    cudaError_t e = vl2::launch_flux(v0, &dd, reg, recon, B->riemann, d, B->fs, B->max_mb, B->cur);
    ++B->launches;
    if (e != cudaSuccess) return e;
  }
  const vl2::Dispatch dh = disp(B, vl2_batch::W_HALO);
  if (dh.nwork == 0) return cudaSuccess;
  ++B->launches;
  return vl2::launch_flux_halo(v0, &dh, B->cur);
}

// one VL2 cycle of every box; h = beta * dt[box] with dt in device memory.  With device_dt the cycle
// first turns each box's reduced CFL rate into its dt (Sec. 2.1.7 per box), else it only resets the rates.
cudaError_t batch_cycle(vl2_batch* B, bool device_dt) {
  const vl2::MeshView v0 = B->meshes[0]->view();
  cudaError_t e;
  const vl2::Dispatch dp = disp(B, vl2_batch::W_PRIM), dg = disp(B, vl2_batch::W_GHOSTS),
                      dn = disp(B, vl2_batch::W_NODES);
  if ((e = vl2::launch_batch_dt(B->dviews, B->n, device_dt ? B->dcfl : nullptr, B->ddt, B->cur)) != cudaSuccess) return e;
  if ((e = batch_fluxes(B, 0, VL2_DC)) != cudaSuccess) return e;
  if ((e = vl2::launch_emfs(v0, &dn, B->cur)) != cudaSuccess) return e;
  if ((e = vl2::launch_update(v0, &dn, 0, 1, 0.0, B->ddt, 0.5, B->cur)) != cudaSuccess) return e;
  if ((e = vl2::launch_ghosts(v0, &dg, 1, B->cur)) != cudaSuccess) return e;
  if ((e = vl2::launch_prim(v0, &dp, 1, true, false, B->cur)) != cudaSuccess) return e;
  if ((e = batch_fluxes(B, 1, B->recon)) != cudaSuccess) return e;
  if ((e = vl2::launch_emfs(v0, &dn, B->cur)) != cudaSuccess) return e;
  if ((e = vl2::launch_update(v0, &dn, 0, 0, 0.0, B->ddt, 1.0, B->cur, 1.0, 0.0, 1)) != cudaSuccess) return e;
  if ((e = vl2::launch_ghosts(v0, &dg, 0, B->cur)) != cudaSuccess) return e;
  if ((e = vl2::launch_prim(v0, &dp, 0, true, true, B->cur)) != cudaSuccess) return e;
  B->launches += 11;  // plus the 6 flux launches (and 2 halo copies) counted in batch_fluxes
  return cudaSuccess;
}

// make sure every box has current primitives and a reduced CFL rate
vl2_status batch_ready(vl2_batch* B) {
  bool all = true;
  for (vl2_mesh* m : B->meshes) {
    if (!m->initialized) return bfail(B, VL2_E_STATE, "a mesh of the batch has no state (vl2_set_prims)");
    all = all && m->w_valid && m->dt_pending;
  }
  if (!all) {
    const vl2::MeshView v0 = B->meshes[0]->view();
    const vl2::Dispatch dp = disp(B, vl2_batch::W_PRIM);
    VL2_BCHECK(B, vl2::launch_batch_dt(B->dviews, B->n, nullptr, B->ddt, B->cur));
    VL2_BCHECK(B, vl2::launch_prim(v0, &dp, 0, true, true, B->cur));
    B->launches += 2;
    for (vl2_mesh* m : B->meshes) m->w_valid = m->dt_pending = true;
  }
  return VL2_OK;
}

void batch_mark(vl2_batch* B) {
  for (vl2_mesh* m : B->meshes) m->w_valid = m->dt_pending = true;
}

}  // namespace

extern "C" {

vl2_status vl2_batch_workspace_bytes(vl2_mesh* const* meshes, int n, size_t* bytes) {
  std::string msg;
  vl2_status s = batch_check(meshes, n, msg);
  if (s != VL2_OK) return bfail(nullptr, s, msg);
  if (!bytes) return bfail(nullptr, VL2_E_ARG, "bytes is NULL");
  std::vector<vl2_mesh*> ms(meshes, meshes + n);
  int max_mb = 1;
  for (vl2_mesh* m : ms) max_mb = std::max(max_mb, m->max_mb());
  *bytes = batch_plan(ms, max_mb).total;
  return VL2_OK;
}

vl2_status vl2_batch_create(vl2_mesh* const* meshes, int n, void* workspace, size_t bytes, vl2_batch** out) {
  if (!out) return bfail(nullptr, VL2_E_ARG, "out is NULL");
  *out = nullptr;
  std::string msg;
  vl2_status s = batch_check(meshes, n, msg);
  if (s != VL2_OK) return bfail(nullptr, s, msg);
  if (!workspace || ((uintptr_t)workspace & 255u)) return bfail(nullptr, VL2_E_ARG, "workspace must be 256-byte aligned");
  vl2_batch* B = new (std::nothrow) vl2_batch();
  if (!B) return bfail(nullptr, VL2_E_ARG, "host allocation failed");
  B->meshes.assign(meshes, meshes + n);
  B->n = n;
  B->st = meshes[0]->st;
  B->cur = B->st;
  if (cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete B;
    return bfail(nullptr, VL2_E_CUDA, "batch stream/event creation failed");
  }
  B->riemann = meshes[0]->p.riemann;
  B->recon = meshes[0]->rec();
  for (vl2_mesh* m : B->meshes) B->max_mb = std::max(B->max_mb, m->max_mb());
  // launch shapes of the first mesh (the PLM kernel its meshes take alone), where they serve every mesh
  B->fs = meshes[0]->fs;
  if (B->fs.plm_tma && !batch_tma_ok(B, B->fs)) B->fs.plm_tma = 0;
  vl2::prime_flux_tma(meshes[0]->view(), B->recon, B->riemann == VL2_HLLD ? vl2::RS_HLLD : vl2::RS_HLLE, B->fs,
                      B->max_mb, B->st);
  const BatchPlan pl = batch_plan(B->meshes, B->max_mb);
  if (bytes < pl.total) {
    delete B;
    return bfail(nullptr, VL2_E_NOMEM, "workspace smaller than vl2_batch_workspace_bytes()");
  }
  char* base = (char*)workspace;
  B->dviews = (vl2::MeshView*)(base + pl.off_views);
  B->ddt = (double*)(base + pl.off_dt);
  B->dcfl = (double*)(base + pl.off_cfl);
  for (int w = 0; w < vl2_batch::W_COUNT; ++w) {
    B->dwork[w] = (vl2::WorkItem*)(base + pl.off_work[w]);
    B->cap[w] = pl.cap[w];
  }
  std::vector<vl2::MeshView> views;
  std::vector<double> cfl;
  for (vl2_mesh* m : B->meshes) {
    views.push_back(m->view());
    cfl.push_back(m->p.cfl);
  }
  cudaError_t e = cudaMemcpyAsync(B->dviews, views.data(), views.size() * sizeof(vl2::MeshView),
                                  cudaMemcpyHostToDevice, B->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->dcfl, cfl.data(), cfl.size() * sizeof(double), cudaMemcpyHostToDevice, B->st);
  if (e != cudaSuccess) {
    delete B;
    return bfail(nullptr, VL2_E_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  }
  if ((s = batch_lists(B)) != VL2_OK) {
    g_err = B->err;
    delete B;
    return s;
  }
  *out = B;
  return VL2_OK;
}

vl2_status vl2_batch_destroy(vl2_batch* batch) {
  delete batch;
  return VL2_OK;
}

vl2_status vl2_batch_autotune(vl2_batch* B, int* dc_threads, int* plm_lines) {
  if (!B) return bfail(nullptr, VL2_E_ARG, "batch is NULL");
  B->cur = B->st;
  vl2_status s = batch_ready(B);
  if (s != VL2_OK) return s;
  cudaEvent_t e0, e1;
  VL2_BCHECK(B, cudaEventCreate(&e0));
  VL2_BCHECK(B, cudaEventCreate(&e1));
  float best = 1e30f;
  vl2::FluxShape best_fs = B->fs;
  std::vector<vl2::FluxShape> cands;
  for (int dc : kDcCandidates)
    for (int pl : kPlmCandidates)
      for (int tma = 0; tma < 2; ++tma) {
        vl2::FluxShape fs;
        fs.dc_threads = dc;
        fs.plm_lines = pl;
        fs.plm_tma = tma;
        if (!tma || batch_tma_ok(B, fs)) cands.push_back(fs);
      }
  for (const vl2::FluxShape& fs : cands) {
    B->fs = fs;
    if ((s = batch_lists(B)) != VL2_OK) break;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {  // the flux launches only write flux scratch: the state is untouched
      VL2_BCHECK(B, cudaEventRecord(e0, B->st));
      VL2_BCHECK(B, batch_fluxes(B, 0, VL2_DC));
      VL2_BCHECK(B, batch_fluxes(B, 0, B->recon));
      VL2_BCHECK(B, cudaEventRecord(e1, B->st));
      VL2_BCHECK(B, cudaEventSynchronize(e1));
      float ms = 0.f;
      VL2_BCHECK(B, cudaEventElapsedTime(&ms, e0, e1));
      tmin = std::min(tmin, ms);
    }
    if (tmin < best) {
      best = tmin;
      best_fs = B->fs;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != VL2_OK) return s;
  B->fs = best_fs;
  if ((s = batch_lists(B)) != VL2_OK) return s;
  if (B->exec) {  // the captured graph used the old launch shapes
    cudaGraphExecDestroy(B->exec);
    cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->graph_steps = 0;
  }
  if (dc_threads) *dc_threads = B->fs.dc_threads;
  if (plm_lines) *plm_lines = B->fs.plm_lines;
  return VL2_OK;
}

vl2_status vl2_batch_step(vl2_batch* B, const double* dt, int where) {
  if (!B || !dt || bad_where(where)) return bfail(B, VL2_E_ARG, "NULL argument or bad where");
  B->cur = B->st;
  if (where == VL2_HOST)
    for (int q = 0; q < B->n; ++q)
      if (!(dt[q] > 0.0) || !std::isfinite(dt[q])) return bfail(B, VL2_E_ARG, "dt must be finite and positive");
  vl2_status s = batch_ready(B);
  if (s != VL2_OK) return s;
  VL2_BCHECK(B, cudaMemcpyAsync(B->ddt, dt, B->n * sizeof(double),
                                where == VL2_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, B->st));
  VL2_BCHECK(B, batch_cycle(B, false));
  batch_mark(B);
  if (where == VL2_HOST) VL2_BCHECK(B, cudaStreamSynchronize(B->st));  // the caller may reuse dt
  return VL2_OK;
}

vl2_status vl2_batch_run(vl2_batch* B, int nsteps, double* dt_last) {
  if (!B || nsteps <= 0) return bfail(B, VL2_E_ARG, "NULL batch or nsteps <= 0");
  B->cur = B->st;
  vl2_status s = batch_ready(B);
  if (s != VL2_OK) return s;
  VL2_BCHECK(B, cudaEventRecord(B->ev_in, B->st));
  VL2_BCHECK(B, cudaStreamWaitEvent(B->cap_stream, B->ev_in, 0));
  if (!B->exec || B->graph_steps != nsteps) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      cudaGraphDestroy(B->graph);
      B->exec = nullptr;
      B->graph = nullptr;
    }
    B->cur = B->cap_stream;
    VL2_BCHECK(B, cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const long long l0 = B->launches;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = batch_cycle(B, true);
    B->launches = l0;  // counted when the graph runs
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(B->cap_stream, &graph);
    B->cur = B->st;
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(B, VL2_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    B->graph = graph;
    VL2_BCHECK(B, cudaGraphInstantiate(&B->exec, B->graph, 0));
    B->graph_steps = nsteps;
  }
  VL2_BCHECK(B, cudaGraphLaunch(B->exec, B->cap_stream));
  VL2_BCHECK(B, cudaEventRecord(B->ev_out, B->cap_stream));
  VL2_BCHECK(B, cudaStreamWaitEvent(B->st, B->ev_out, 0));
  B->launches += 17LL * nsteps;
  batch_mark(B);
  if (dt_last) {
    VL2_BCHECK(B, cudaMemcpyAsync(dt_last, B->ddt, B->n * sizeof(double), cudaMemcpyDeviceToHost, B->st));
    VL2_BCHECK(B, cudaStreamSynchronize(B->st));
  }
  return VL2_OK;
}

vl2_status vl2_batch_flux_shape(const vl2_batch* B, int* dc_threads, int* plm_lines, int* tma) {
  if (!B) return bfail(nullptr, VL2_E_ARG, "batch is NULL");
  if (dc_threads) *dc_threads = B->fs.dc_threads;
  if (plm_lines) *plm_lines = B->fs.plm_lines;
  if (tma) *tma = B->fs.plm_tma;
  return VL2_OK;
}

vl2_status vl2_batch_set_flux_shape(vl2_batch* B, int dc_threads, int plm_lines, int tma) {
  if (!B) return bfail(nullptr, VL2_E_ARG, "batch is NULL");
  if ((dc_threads != 64 && dc_threads != 128 && dc_threads != 256) ||
      (plm_lines != 4 && plm_lines != 8 && plm_lines != 16) || (tma != 0 && tma != 1))
    return bfail(B, VL2_E_ARG, "dc_threads must be 64, 128 or 256, plm_lines 4, 8 or 16, tma 0 or 1");
  vl2::FluxShape fs;
  fs.dc_threads = dc_threads;
  fs.plm_lines = plm_lines;
  fs.plm_tma = tma;
  if (tma && !batch_tma_ok(B, fs)) return bfail(B, VL2_E_ARG, "the TMA-staged PLM kernel does not serve every mesh");
  B->fs = fs;
  vl2::prime_flux_tma(B->meshes[0]->view(), B->recon, B->riemann == VL2_HLLD ? vl2::RS_HLLD : vl2::RS_HLLE, fs,
                      B->max_mb, B->st);
  vl2_status s = batch_lists(B);
  if (s != VL2_OK) return s;
  if (B->exec) {  // the captured graph used the old launch shapes
    cudaGraphExecDestroy(B->exec);
    cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->graph_steps = 0;
  }
  return VL2_OK;
}

vl2_status vl2_batch_launch_count(const vl2_batch* B, long long* n) {
  if (!B || !n) return bfail(nullptr, VL2_E_ARG, "NULL argument");
  *n = B->launches;
  return VL2_OK;
}

const char* vl2_batch_last_error(const vl2_batch* B) { return B ? B->err.c_str() : g_err.c_str(); }

}  // extern "C"
