// Internal geometry and kernel-launcher declarations of the GB300 VL2 MHD library.
// Host and device code both include this file; it holds no physics.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vl2 {


enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };
enum { REC_DC = 0, REC_PLM = 1, REC_PPM = 2, REC_PLM_CHAR = 3, REC_PPM_CHAR = 4 };
enum { RS_HLLE = 0, RS_HLLD = 1 };

// Mesh geometry passed by value to every kernel.
struct Geom {
  int nblk;            // number of MeshBlocks
  int nb[3];           // blocks per direction
  int mb[3];           // active cells per block
  int ng;              // ghost layers (Sec. 2.1.1): 2, or 3 for PPM
  int ns;              // passive scalars (eq. passive_scalars)
  int sx, sy, sz;      // padded per-block box extents (cells incl. ghosts + 1 face, x row padded)
  long long box;       // sx * sy * sz elements per block per variable
  int N[3];            // global active cells
  int bc[6];           // x-, x+, y-, y+, z-, z+
  double idx[3];       // 1 / dx_d
  double dx[3];
  double gamma, gm1, igm1;
  // the same in FP32 (rounded to nearest on the host), for FP32 stage arithmetic: a conversion in a kernel
  // would occupy the FP64 pipe once per thread
  float gamma_f, igm1_f, idx_f[3];
  int hlle_roe;  // 1: the HLLE solver takes Einfeldt's Roe-averaged outer speeds
  double dfloor, pfloor;
  double ct_delta;     // smoothed CT upwind weight width (0: the sign switch)
  // Faces one cell outside a block's transverse range feed the CT corners on the block surface.  1: the flux
  // kernels compute them from the block's ghost cells (a mesh with an outflow boundary, where such a face
  // can lie outside the mesh); 0: every block computes only its own transverse range, and k_flux_halo copies
  // those faces' mass flux and transverse induction fluxes from the neighbouring block that owns them
  // (periodic meshes), so each face flux is computed once per block surface.
  int flux_halo;
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
  void* ec;          // cell EMFs -(v x b_c), components 1, 2, 3, written by cons->prim: [nblk][3][box]
  int mixed;         // 1: scratch is float
  double* stage;     // staging for global-array I/O
  size_t stage_elems;
  double* red;       // reduction partials
  int red_ctas;
  unsigned long long* scal;  // device scalars (see SC_*)
  // passive scalars (FP64 in every precision; null when ns = 0)
  double* s[2];      // registers of the scalar masses rho C: [nblk][ns][box]
  double* cs;        // concentrations C, written by cons->prim: [nblk][ns][box]
  double* fsc[3];    // scalar fluxes per sweep direction: [nblk][ns][box]
  // forcing acceleration at the cell centres, FP64: [nblk][3][box] (active cells); null when no forcing is set
  double* acc;
  // TMA_MAPS tensor maps (CUtensorMap, 128 bytes each) describing w for the TMA-staged PLM sweeps, one per
  // sweep direction and tile height (tma_map_index); null when that path is not available for this mesh
  const void* tmw;
};

// Device scalars: CFL rate bits, floor count, periodic-check mismatches, and a flag set by a kernel whose
// bounded wait for a TMA tile expired (it skips its work and returns).
// SC_MISMATCH_ASYNC: the periodic-face check of a stream-ordered vl2_set_prims_async, sticky until a
// synchronising call reports it.
enum { SC_MAXRATE = 0, SC_FLOORS = 1, SC_MISMATCH = 2, SC_TIMEOUT = 3, SC_MISMATCH_ASYNC = 4, SC_COUNT = 8 };

// A mesh as the kernels see it (copied to device memory for batched launches).
struct MeshView {
  Geom g;
  Arrays a;
};

// One CTA of a batched launch: which mesh (box) and which tile of that mesh's work.
struct WorkItem {
  int box;
  int tile;
};

// How a launch is scheduled: one mesh (views == nullptr: tile = blockIdx.x), or many meshes through a
// work list of (box, tile) entries, one per CTA.
struct Dispatch {
  const MeshView* views = nullptr;  // device array, one per box
  const WorkItem* work = nullptr;   // device array, nwork entries
  int nwork = 0;
};

#ifdef __CUDACC__
// Resolve the mesh and tile of work item `item` (single mesh: the launch argument, tile = item; batch: the
// item's entry of the work list) and stage the mesh view in shared memory.  Every thread of the CTA must
// call it.  The view is copied as 8-byte words, one per thread of the first 64 (every launch that calls
// this has at least 64 threads per CTA), so that the barrier behind it waits for one round of loads rather
// than for one thread's serial copy of the whole view.
static_assert(sizeof(MeshView) % 8 == 0, "the mesh view is staged in 8-byte words");
static_assert(sizeof(MeshView) <= 64 * 8, "the mesh view is staged by the first 64 threads (every CTA has >= 64)");
__device__ __forceinline__ const MeshView& stage_view_item(MeshView& sv, const MeshView& single,
                                                           const MeshView* views, const WorkItem* work, int item,
                                                           int& tile, int* box = nullptr) {
  const MeshView* src = &single;
  if (work) {
    const WorkItem w = work[item];
    tile = w.tile;
    if (box) *box = w.box;
    src = views + w.box;
  } else {
    tile = item;
    if (box) *box = 0;
  }
  constexpr unsigned NW = (unsigned)(sizeof(MeshView) / 8);
  if (threadIdx.x < NW)
    reinterpret_cast<unsigned long long*>(&sv)[threadIdx.x] =
        reinterpret_cast<const unsigned long long*>(src)[threadIdx.x];
  __syncthreads();
  return sv;
}
// The same for the CTA's own item, blockIdx.x (one work item per CTA).
__device__ __forceinline__ const MeshView& stage_view(MeshView& sv, const MeshView& single, const MeshView* views,
                                                      const WorkItem* work, int& tile, int* box = nullptr) {
  return stage_view_item(sv, single, views, work, (int)blockIdx.x, tile, box);
}
#endif

// Threads per CTA of the per-element kernels, and the tunable flux launch shapes.
constexpr int THREADS = 256;
struct FluxShape {
  int dc_threads = 128;  // CTA size of the donor-cell flux kernel
  int plm_lines = 16;    // lines of faces per CTA of the PLM flux kernel (0: largest that fits)
  int plm_tma = 0;       // 1: PLM sweeps take the persistent TMA-staged kernel (tile height plm_lines: 4, 8, 16)
};

// ---- TMA-staged PLM sweeps (k_flux_tma).  A tile is plm_lines lines of faces along the sweep direction,
// adjacent along the faster transverse direction; its primitives arrive as one 4D box (x, y, z, variable)
// of w: the mb+4 cells ng-2 .. ng+mb+1 along the sweep, the tile's lines across it, all 8 variables. ----
constexpr int TMA_MAPS = 9;  // 3 sweep directions x tile heights 4, 8, 16
__host__ __device__ inline int tma_map_index(int dir, int lines) { return 3 * dir + (lines == 4 ? 0 : (lines == 8 ? 1 : 2)); }
// Box extents (x, y, z, variable) of a tile's primitives and the x offset of its first line inside the box.
// The box's first x coordinate is a multiple of 16 bytes (TMA): the sweep along x starts at cell ng-2 = 0,
// the others at the tile's first line rounded down, which needs xoff extra columns.
__host__ __device__ inline void tma_w_box(const Geom& g, int dir, int lines, int esize, int box[4], int* xoff) {
  const int q = 16 / esize;
  const int o = (g.ng - g.flux_halo) % q;
  *xoff = dir == 0 ? 0 : o;
  box[0] = dir == 0 ? (g.mb[0] + 4 + q - 1) / q * q : (o + lines + q - 1) / q * q;
  box[1] = dir == 1 ? g.mb[1] + 4 : (dir == 0 ? lines : 1);
  box[2] = dir == 2 ? g.mb[2] + 4 : 1;
  box[3] = 8;
}

// Work units of each kernel for one mesh (used to size single launches and to build work lists).
long long tiles_prim(const Geom& g);
long long tiles_ghosts(const Geom& g);
long long tiles_nodes(const Geom& g);  // EMF and update
long long tiles_flux_dc(const Geom& g, int dir, const FluxShape& fs);
long long tiles_flux_plm(const Geom& g, int dir, const FluxShape& fs);
long long tiles_flux_halo(const Geom& g);  // 0 when g.flux_halo
int plm_lines_for(const Geom& g, int dir, const FluxShape& fs, int max_mb, int recon);
// true when the PLM sweeps of this mesh (or batch: v is its first mesh, and every mesh qualifies) run as
// k_flux_tma under fs; tiles of one direction for that kernel
bool flux_tma_applies(const MeshView& v, int recon, const FluxShape& fs, int max_mb);
long long tiles_flux_tma(const Geom& g, int dir, int lines);
// Look up (outside any graph capture) the occupancy the TMA-staged launches of this shape will use.
void prime_flux_tma(const MeshView& v, int recon, int riemann, const FluxShape& fs, int max_mb, cudaStream_t st);
// Encode the TMA_MAPS tensor maps of the primitives w (device, 256-byte aligned; float or double elements)
// into maps (host memory, 128-byte aligned, TMA_MAPS * 128 bytes).  Returns false, with a message, when
// the driver cannot encode them (the mesh then keeps the line-tile kernel).
bool encode_w_maps(const Geom& g, const void* w, int esize, void* maps, const char** why);

// ---- launchers (vl2_kernels.cu / vl2_flux.cu); all enqueue on `st`.  d == nullptr: the single mesh v.
// For batched launches v only selects the precision; dtbox (per-box dt, device) and beta give h. ----
cudaError_t launch_prim(const MeshView& v, const Dispatch* d, int reg, bool all_cells, bool want_dt, cudaStream_t st);
cudaError_t launch_ghosts(const MeshView& v, const Dispatch* d, int reg, cudaStream_t st);
cudaError_t launch_mesh_dt(const unsigned long long* scal, double cfl, double* dt, cudaStream_t st);
cudaError_t launch_flux(const MeshView& v, const Dispatch* d, int reg, int recon, int riemann, int dir,
                        const FluxShape& fs, int max_mb, cudaStream_t st);
// copy the halo faces' mass flux and transverse induction fluxes from their owning blocks (meshes with
// flux_halo = 0; a no-op launch-free call when no mesh of the launch needs it)
cudaError_t launch_flux_halo(const MeshView& v, const Dispatch* d, cudaStream_t st);
cudaError_t launch_emfs(const MeshView& v, const Dispatch* d, cudaStream_t st);
// stage_reg: the register the stage's fluxes were formed from (its state carries the forcing source terms;
// -1: base_reg)
cudaError_t launch_update(const MeshView& v, const Dispatch* d, int base_reg, int out_reg, double h,
                          const double* dtbox, double beta, cudaStream_t st, double g_base = 1.0, double g_other = 0.0,
                          int stage_reg = -1);
cudaError_t launch_scatter_forcing(const Geom& g, double* acc, const double* a, cudaStream_t st);
// per-box dt from the CFL rates the last prim reduced: dt[box] = cfl / rate, rate reset to 0
cudaError_t launch_batch_dt(const MeshView* views, int nbox, const double* cfl, double* dt, cudaStream_t st);
cudaError_t prepare_kernel_attributes();
cudaError_t launch_scatter_prims(const Geom& g, const Arrays& a, const double* w, const double* b1,
                                 const double* b2, const double* b3, cudaStream_t st);
cudaError_t launch_check_periodic(const Geom& g, const double* b1, const double* b2, const double* b3,
                                  unsigned long long* count, cudaStream_t st);
cudaError_t launch_gather_cons(const Geom& g, const Arrays& a, double* u, double* b1, double* b2, double* b3,
                               cudaStream_t st);
cudaError_t launch_gather_prims(const Geom& g, const Arrays& a, double* w, cudaStream_t st);
// passive scalars: fluxes of one sweep direction for one reconstruction (the stage's mass fluxes must be
// in a.f[dir]), the register update, and the global-array I/O (concentrations in, masses out)
cudaError_t launch_scalar_fluxes(const MeshView& v, int recon, int dir, cudaStream_t st);
cudaError_t launch_scalar_update(const MeshView& v, int base_reg, int out_reg, double h, double g_base,
                                 double g_other, cudaStream_t st);
cudaError_t launch_scatter_scalars(const Geom& g, const Arrays& a, const double* c, cudaStream_t st);
cudaError_t launch_gather_scalars(const Geom& g, const Arrays& a, double* out, cudaStream_t st);
cudaError_t launch_gather_fluxes(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st);
cudaError_t launch_gather_emfs(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st);
cudaError_t launch_divb(const Geom& g, const Arrays& a, double* result2, cudaStream_t st);
cudaError_t launch_totals(const Geom& g, const Arrays& a, double* result8, cudaStream_t st);

// Adjoint (reverse) arrays of one mesh, FP64, block layout like the forward arrays.
struct AdjArrays {
  double* lu[2];     // adjoints of the two conserved registers: [nblk][5][box]
  double* lb[2][3];  // adjoints of the two face-field registers
  double* lw;        // adjoint of the primitives: [nblk][8][box]
  double* lf[3];     // adjoints of the face fluxes: [nblk][7][box]; then the left-state adjoints of the faces
  double* lr;        // right-state adjoints of the faces of the sweep being transposed: [nblk][7][box]
  double* le[3];     // adjoints of the corner EMFs
  double* w0;        // predictor primitives kept from the forward recompute: [nblk][8][box]
  double* m1[3];     // predictor face mass fluxes (upwind choices of its CT): [nblk][box]; with the smoothed CT
                     // weight also its face EMFs F[B_t1], F[B_t2]: [nblk][3][box]
  // the PLM slopes' contributions of one sweep [nblk][7][box] x 3 (to the cells below, at and above the
  // slope's cell).  They live in the forward flux arrays, free while the reverse sweep transposes fluxes
  // (its CT transpose, the last reader of a corrector mass flux, has run by then).
  double* ps[3];
};

cudaError_t adj_scatter_out(const Geom& g, const AdjArrays& j, const double* gu, const double* gb1, const double* gb2,
                            const double* gb3, cudaStream_t st);
cudaError_t adj_update(const Geom& g, const AdjArrays& j, int out_reg, int base_reg, double h, cudaStream_t st);
cudaError_t adj_ct(const Geom& g, const AdjArrays& j, const double* W, const double* const* mflux, long long mstride,
                   long long e5off, long long e6off, cudaStream_t st);
// transpose of the forward halo copy (no-op when g.flux_halo): owner faces collect their copies' adjoints
cudaError_t adj_flux_halo(const Geom& g, const AdjArrays& j, cudaStream_t st);
cudaError_t adj_fluxes(const Geom& g, const AdjArrays& j, int recon, int riemann, const double* W,
                       const double* const* Bn, int lam_reg, cudaStream_t st);
cudaError_t adj_prim(const Geom& g, const AdjArrays& j, const double* W, int lam_reg, cudaStream_t st);
cudaError_t adj_ghosts(const Geom& g, const AdjArrays& j, int lam_reg, cudaStream_t st);
cudaError_t adj_gather_in(const Geom& g, const AdjArrays& j, double* gu, double* gb1, double* gb2, double* gb3,
                          cudaStream_t st);
cudaError_t prims_vjp(long long ncell, double igm1, const double* w, const double* lam_u, double* lam_w, cudaStream_t st);
cudaError_t riemann_vjp_points(int rs, long long n, const double* wl, const double* wr, const double* bn,
                               const double* lf, double gamma, double* out, cudaStream_t st);
cudaError_t launch_scatter_cons(const Geom& g, const Arrays& a, const double* u, const double* b1, const double* b2,
                                const double* b3, cudaStream_t st);

// Sets the message vl2_last_error(NULL) returns (entry points that have no mesh).
void record_error(const char* msg);

}  // namespace vl2
