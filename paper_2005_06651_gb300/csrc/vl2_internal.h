// Internal geometry and kernel-launcher declarations of the GB300 VL2 MHD library.
// Host and device code both include this file; it holds no physics.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vl2 {

constexpr int NG = 2;  // ghost layers for second-order MHD (Sec. 2.1.1)

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };
enum { REC_DC = 0, REC_PLM = 1 };
enum { RS_HLLE = 0, RS_HLLD = 1 };

// Mesh geometry passed by value to every kernel.
struct Geom {
  int nblk;            // number of MeshBlocks
  int nb[3];           // blocks per direction
  int mb[3];           // active cells per block
  int sx, sy, sz;      // padded per-block box extents (cells incl. ghosts + 1 face, x row padded)
  long long box;       // sx * sy * sz elements per block per variable
  int N[3];            // global active cells
  int bc[6];           // x-, x+, y-, y+, z-, z+
  double idx[3];       // 1 / dx_d
  double dx[3];
  double gamma, gm1, igm1;
  double dfloor, pfloor;
};

__host__ __device__ inline long long cell_off(const Geom& g, int k, int j, int i) {
  return ((long long)k * g.sy + j) * g.sx + i;
}

// Device arrays of one mesh (all inside the caller's workspace).
struct Arrays {
  double* u[2];      // conserved registers: [nblk][5][box] (FP64 in every precision)
  double* b[2][3];   // face-field registers: [nblk][box] per direction (FP64)
  // Stage scratch; element type double (FP64 form) or float (mixed form: FP32 reconstruction, fluxes, EMFs)
  void* w;           // primitives rho, vx, vy, vz, p, bcx, bcy, bcz: [nblk][8][box]
  void* f[3];        // fluxes per sweep direction: [nblk][7][box]
  void* e[3];        // corner EMFs E1, E2, E3: [nblk][box]
  int mixed;         // 1: scratch is float
  double* stage;     // staging for global-array I/O
  size_t stage_elems;
  double* red;       // reduction partials
  int red_ctas;
  unsigned long long* scal;  // device scalars (see SC_*)
};

enum { SC_MAXRATE = 0, SC_FLOORS = 1, SC_MISMATCH = 2, SC_COUNT = 8 };

// ---- launchers (vl2_kernels.cu / vl2_flux.cu); all enqueue on `st` ----
cudaError_t launch_prim(const Geom& g, const Arrays& a, int reg, bool all_cells, bool want_dt, cudaStream_t st);
cudaError_t launch_ghosts(const Geom& g, const Arrays& a, int reg, cudaStream_t st);
cudaError_t launch_flux(const Geom& g, const Arrays& a, int reg, int recon, int riemann, int dir, cudaStream_t st);
cudaError_t launch_emfs(const Geom& g, const Arrays& a, cudaStream_t st);
cudaError_t launch_update(const Geom& g, const Arrays& a, int base_reg, int out_reg, double h, cudaStream_t st);
cudaError_t launch_scatter_prims(const Geom& g, const Arrays& a, const double* w, const double* b1,
                                 const double* b2, const double* b3, cudaStream_t st);
cudaError_t launch_check_periodic(const Geom& g, const double* b1, const double* b2, const double* b3,
                                  unsigned long long* count, cudaStream_t st);
cudaError_t launch_gather_cons(const Geom& g, const Arrays& a, double* u, double* b1, double* b2, double* b3,
                               cudaStream_t st);
cudaError_t launch_gather_prims(const Geom& g, const Arrays& a, double* w, cudaStream_t st);
cudaError_t launch_gather_fluxes(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st);
cudaError_t launch_gather_emfs(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st);
cudaError_t launch_divb(const Geom& g, const Arrays& a, double* result2, cudaStream_t st);
cudaError_t launch_totals(const Geom& g, const Arrays& a, double* result8, cudaStream_t st);

// Sets the message vl2_last_error(NULL) returns (entry points that have no mesh).
void record_error(const char* msg);

}  // namespace vl2
