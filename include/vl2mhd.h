/*
 * vl2mhd.h -- C ABI of the GB300 (sm_103a) VL2 ideal-MHD stepper.
 *
 * The library advances 3D adiabatic ideal MHD (Stone et al. 2020, arXiv:2005.06651, Sec. 3.1,
 * eq. cons with mu = 1, ideal-gas EOS) on a uniform Cartesian mesh of equal-size MeshBlocks
 * (Sec. 2.1) held on one GPU, with the VL2 predictor-corrector (Sec. 3.2.3, eq. rk-2s: donor-cell
 * predictor over dt/2, PLM corrector over dt), PLM reconstruction of primitives with the van Leer
 * limiter (Sec. 3.2.1), HLLD or HLLE fluxes (Sec. 3.2.2), upwind constrained transport of the
 * face-centred field (Sec. 3.1, Sec. 2.1.1), ghost exchange between blocks (Sec. 2.1.1) and the
 * global CFL time step (Sec. 2.1.7).  Options: the RK1 / RK2 / RK3 integrators of the same 2S family
 * (Sec. 3.2.3), PPM reconstruction with three ghost layers (Sec. 3.2.1), passive scalars (eq.
 * passive_scalars), an FP32-flux mixed precision, a batched form for many independent meshes, and
 * the adjoint of the VL2 cycle.
 *
 * Conventions shared by every call
 *  - Every call returns a vl2_status; 0 (VL2_OK) is success.  Nothing throws across the ABI.
 *    vl2_last_error() returns a short message for the last failing call on a mesh.
 *  - All device work of a mesh is issued on the stream given in vl2_params.stream (a cudaStream_t
 *    passed as void*; NULL selects the legacy default stream).  Calls on one mesh are not
 *    re-entrant: do not call into the same mesh from two host threads at once.
 *  - The caller owns the device workspace (vl2_workspace_bytes / vl2_mesh_create) and every buffer
 *    it passes.  Caller buffers are only read or written during the call; `where` says whether a
 *    pointer is host memory (VL2_HOST, pinned or pageable) or device memory (VL2_DEVICE).  Calls
 *    that read back to host memory return after the data has arrived; calls with device buffers
 *    only enqueue on the mesh's stream.
 *  - Global arrays cover the active (non-ghost) cells of the whole mesh in C order, x fastest:
 *      cell arrays  [var][NZ][NY][NX]
 *      b1 (B_x)     [NZ][NY][NX+1]   face i is the lower x-face of cell i
 *      b2 (B_y)     [NZ][NY+1][NX]
 *      b3 (B_z)     [NZ+1][NY][NX]
 *    In a periodic direction the last face row duplicates the first (face N == face 0).
 */
#ifndef VL2MHD_H
#define VL2MHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vl2_status {
  VL2_OK = 0,
  VL2_E_ARG = 1,      /* invalid argument (null pointer, bad size, inconsistent parameters) */
  VL2_E_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
  VL2_E_NONPHYS = 3,  /* a density or pressure floor fired (value floored and counted), or dt not finite */
  VL2_E_TIMEOUT = 4,  /* a bounded device-side wait expired: the TMA-staged PLM sweeps wait (with a limit of
                         about a quarter second) for each tile's bulk copy; if one never lands the CTA skips
                         its tiles, the step's fluxes are incomplete, and the next vl2_new_dt returns this */
  VL2_E_STATE = 5,    /* call not valid in the mesh's current state */
  VL2_E_NOMEM = 6     /* workspace smaller than vl2_workspace_bytes() */
} vl2_status;

/* Riemann solver, Sec. 3.2.2.  VL2_HLLE bounds the fan by the two states' fast speeds; VL2_HLLE_ROE takes
 * Einfeldt's speeds min(u_L - c_L, u~ - c~_f), max(u_R + c_R, u~ + c~_f) with the MHD Roe average ~. */
enum { VL2_HLLE = 0, VL2_HLLD = 1, VL2_HLLE_ROE = 2 };
enum { VL2_PERIODIC = 0, VL2_OUTFLOW = 1 };/* per-face boundary condition */
enum { VL2_FP64 = 0, VL2_MIXED = 1 };      /* arithmetic of reconstruction, fluxes and EMFs */
enum { VL2_HOST = 0, VL2_DEVICE = 1 };     /* where a caller buffer lives */
/* reconstruction, Sec. 3.2.1 (PPM: eq. ppm-uniform-weights; PLM_CHAR / PPM_CHAR: PLM / PPM on the
 * characteristic variables C = L W of the primitive MHD system, each face value then kept within its two
 * cells' range) */
enum { VL2_DC = 0, VL2_PLM = 1, VL2_PPM = 2, VL2_PLM_CHAR = 3, VL2_PPM_CHAR = 4 };
/* time integrators of the 2S family (Sec. 3.2.3, eq. rk-2s and the coefficient list after it):
 * VL2 (default): donor-cell predictor with beta = 1/2, PLM corrector with beta = 1;
 * RK1: forward Euler with donor-cell fluxes; RK2 (SSPRK(2,2)) and RK3 (SSPRK(3,3)): PLM in every stage. */
enum { VL2_INT_VL2 = 0, VL2_INT_RK1 = 1, VL2_INT_RK2 = 2, VL2_INT_RK3 = 3 };

typedef struct vl2_params {
  int nx[3];          /* global active cells (x, y, z); each a multiple of mb[d] */
  int mb[3];          /* MeshBlock active cells (x, y, z), Sec. 2.1: equal for every block */
  int ng;             /* ghost layers (Sec. 2.1.1): 2 for DC / PLM, 3 for PPM (3 also allowed with PLM, same
                         results); the adjoint needs 2 */
  double xmin[3], xmax[3]; /* domain bounds; cells are uniform, dx_d = (xmax-xmin)/nx */
  double gamma;       /* adiabatic index of the ideal-gas EOS, P = (gamma-1) e (Sec. 3.1) */
  double cfl;         /* Courant number C0 of vl2_new_dt; <= 1/2 for VL2 in 3D (Sec. 3.2.3) */
  int riemann;        /* VL2_HLLD, VL2_HLLE or VL2_HLLE_ROE (not with adjoint) */
  int precision;      /* VL2_FP64: all arithmetic in FP64.  VL2_MIXED: reconstruction, Riemann fluxes and
                         CT EMFs in FP32 (FP32 scratch), while U and B stay FP64, cons->prim (pressure
                         recovery) is FP64, and the flux divergence / EMF curl are accumulated in FP64 */
  int bc[6];          /* boundary of faces x-, x+, y-, y+, z-, z+: VL2_PERIODIC or VL2_OUTFLOW;
                         periodic must be set on both faces of a direction */
  double dfloor, pfloor; /* density / pressure floors of cons->prim (positive normal numbers, >= DBL_MIN) */
  void* stream;       /* cudaStream_t for all device work of this mesh (may be NULL) */
  int adjoint;        /* 1: also reserve the arrays of vl2_step_vjp (VL2_FP64 only); 0: forward only */
  int integrator;     /* VL2_INT_VL2 (0, the default for a zero-initialised struct), VL2_INT_RK1, _RK2, _RK3 */
  int recon;          /* reconstruction of the higher-order stages (the VL2 corrector, every RK2 / RK3 stage):
                         VL2_PLM (also 0), VL2_PPM (needs ng = 3), VL2_PLM_CHAR or VL2_PPM_CHAR (needs
                         ng = 3); the adjoint takes VL2_PLM only.  The VL2 predictor and RK1 always use
                         donor cell (Sec. 3.2.3). */
  int nscalars;       /* passive scalars rho C_i, d(rho C_i)/dt + div(rho v C_i) = 0 (eq. passive_scalars):
                         0 .. VL2_MAX_SCALARS; 0 with adjoint; not in a batch */
  double ct_delta;    /* 0 (the default): the upwind CT corner picks the cell by the sign of the face mass flux,
                         the mean at zero (Sec. 3.1, gs05).  > 0: an option beside the paper's method, the
                         weight (1 + tanh(m / ct_delta)) / 2 on the upwind-side gradient, in mass-flux units;
                         it equals the sign switch where tanh saturates and at m = 0, and makes the corner a
                         smooth function of m (with adjoint, vl2_step_vjp then carries dw/dm).  Finite;
                         the meshes of a batch share one value. */
  int forcing;        /* 1: reserve the acceleration array of vl2_set_forcing (a body force; not with adjoint);
                         0 (the default): no forcing */
} vl2_params;

#define VL2_MAX_SCALARS 16

typedef struct vl2_mesh vl2_mesh;

/* Block layout of the mesh's device arrays (Sec. 2.1).  Pointers are owned by the mesh and stay valid
 * until vl2_mesh_destroy.  Block id b has logical position (bx, by, bz) = block_loc[3b..3b+2], x
 * fastest.  Element (var v, cell k, j, i) of block b in a cell array starts at
 *   base + (b * nvar + v) * block_stride_vars + (k * sy + j) * sx + i
 * with local indices including the ng ghost layers (active cells are ng .. ng+mb-1).  Face arrays
 * use the same strides, with one extra face along their own direction. */
typedef struct vl2_layout {
  int nblocks;
  int nb[3];            /* blocks per direction */
  int mb[3];            /* active cells per block */
  int ng;               /* ghost layers */
  int sx, sy, sz;       /* padded box extents (elements) in x, y, z */
  long long block_stride_vars; /* sx * sy * sz */
  const int* block_loc; /* host, [nblocks][3] */
  const int* neighbor;  /* host, [nblocks][27]: block id of neighbour (di,dj,dk) in {-1,0,1}^3 at
                           index (dk+1)*9 + (dj+1)*3 + (di+1), or -1 beyond an outflow boundary */
  double* u;            /* device, conserved variables rho, M1, M2, M3, E (nvar 5) of the current state */
  double* b[3];         /* device, face fields B1, B2, B3 (nvar 1 each) of the current state */
} vl2_layout;

/* Bytes of device workspace a mesh with these parameters needs (registers, primitives, fluxes,
 * EMFs, staging for global-array I/O, reduction scratch).  Errors: VL2_E_ARG for invalid
 * parameters (same checks as vl2_mesh_create). */
vl2_status vl2_workspace_bytes(const vl2_params* params, size_t* bytes);

/* Create a mesh of nx/mb MeshBlocks (Sec. 2.1) inside the caller's device workspace (at least
 * vl2_workspace_bytes(), 256-byte aligned; the caller keeps it alive until vl2_mesh_destroy and
 * frees it afterwards).  The state is zero until vl2_set_prims.  Errors: VL2_E_ARG (bad parameters,
 * misaligned workspace), VL2_E_NOMEM (workspace too small), VL2_E_CUDA. */
vl2_status vl2_mesh_create(const vl2_params* params, void* workspace, size_t bytes, vl2_mesh** out);

/* Release the host-side mesh object (the device workspace stays the caller's).  NULL is accepted. */
vl2_status vl2_mesh_destroy(vl2_mesh* mesh);

/* Describe the block layout (see vl2_layout).  Errors: VL2_E_ARG. */
vl2_status vl2_block_layout(const vl2_mesh* mesh, vl2_layout* out);

/* Set the state from primitives: w = [5][NZ][NY][NX] (rho, vx, vy, vz, p) at cell centres and the
 * face fields b1, b2, b3 (global layout above).  U = (rho, rho v, E) with E = p/(gamma-1) +
 * rho v^2/2 + |b_c|^2/2, b_c the mean of the two face values (Sec. 3.1, eq. total_energy); ghosts are
 * then exchanged (Sec. 2.1.1).  Errors: VL2_E_ARG (null pointer, periodic face duplicates that
 * differ), VL2_E_CUDA. */
vl2_status vl2_set_prims(vl2_mesh* mesh, const double* w, const double* b1, const double* b2,
                         const double* b3, int where);

/* Set the state from conserved variables directly: u = [5][NZ][NY][NX] (rho, M1, M2, M3, E) and the face
 * fields (global layout); ghosts are then exchanged.  Used to restore checkpoints.  Errors: VL2_E_ARG,
 * VL2_E_CUDA. */
vl2_status vl2_set_cons(vl2_mesh* mesh, const double* u, const double* b1, const double* b2, const double* b3,
                        int where);

/* Ghost exchange of the current state (Sec. 2.1.1): cell-centred U and face fields copied, depth
 * ng, from the 26 neighbours (periodic wrap; outflow copies the nearest active cell / boundary face).
 * Faces on a block's own surface are active and are not overwritten.  Errors: VL2_E_CUDA. */
vl2_status vl2_fill_ghosts(vl2_mesh* mesh);

/* One cycle with step dt (Sec. 3.2.3) of the mesh's integrator.  VL2: predictor U* = U^n + (dt/2) L_DC(U^n),
 * corrector U^{n+1} = U^n + dt L_PLM(U*), where L = -div F for U and -curl E (upwind CT corner EMFs) for
 * the face field.  RK1/RK2/RK3: eq. rk-2s with u^(0) = U^n, u^(1) = 0, then per stage s
 * u^(1) += delta_s u^(0), u^(0) = gamma_s0 u^(0) + gamma_s1 u^(1) + beta_s dt L(u^(0)), with the
 * coefficients the paper lists.  cons->prim and ghost exchange follow every stage.  Ghosts are valid on
 * return.  dt must be finite and > 0.  Work is only enqueued.  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_step(vl2_mesh* mesh, double dt);

/* CFL time step of the current state (Sec. 2.1.7, 3.2.3): dt = cfl * min over active cells and
 * directions d of dx_d / (|v_d| + C_f,d), C_f,d the fast speed with b_c,d as normal field.  Blocks on
 * the device; also reports floor events seen since the previous call: returns VL2_E_NONPHYS (with
 * *dt_out still set) when a density/pressure floor fired or dt is not finite, and VL2_E_ARG when a
 * vl2_set_prims_async since the previous report met periodic face duplicates that differ.  Errors:
 * VL2_E_ARG, VL2_E_CUDA, VL2_E_NONPHYS, VL2_E_TIMEOUT. */
vl2_status vl2_new_dt(vl2_mesh* mesh, double* dt_out);

/* Stream-ordered stepping, for callers that overlap host<->device copies with the cycles (no call below
 * waits for the device):
 * vl2_set_prims_async: vl2_set_prims without its two waits.  Host inputs must be page-locked for the copy to
 * be asynchronous; the staging area they pass through is shared with the host forms of the get calls.  The
 * periodic-face check raises a device flag that the next vl2_new_dt or vl2_last_dt reports (VL2_E_ARG).
 * vl2_step_cfl: one VL2 cycle whose step dt = cfl * min dx_d / (|v_d| + C_f,d) (as vl2_new_dt) is formed and
 * read on the device; the same arithmetic as vl2_new_dt followed by vl2_step, so the same bits.  VL2
 * integrator without passive scalars.  Errors: VL2_E_ARG, VL2_E_STATE, VL2_E_CUDA.
 * vl2_last_dt: waits, returns the step the last vl2_step_cfl used, and reports as vl2_new_dt does (floors,
 * a non-finite step, the asynchronous periodic check, an expired TMA wait). */
vl2_status vl2_set_prims_async(vl2_mesh* mesh, const double* w, const double* b1, const double* b2,
                               const double* b3, int where);
vl2_status vl2_step_cfl(vl2_mesh* mesh);
vl2_status vl2_last_dt(vl2_mesh* mesh, double* dt_out);

/* Copy out the conserved state: u = [5][NZ][NY][NX] (rho, M1, M2, M3, E) and the face fields (any of
 * the four pointers may be NULL to skip it).  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_get_cons(vl2_mesh* mesh, double* u, double* b1, double* b2, double* b3, int where);

/* Primitives of the current state on the active cells: w = [8][NZ][NY][NX] (rho, vx, vy, vz, p,
 * b_c1, b_c2, b_c3), with the floors of the cons->prim step applied (Sec. 3.1).  Errors as above. */
vl2_status vl2_get_prims(vl2_mesh* mesh, double* w, int where);

/* Discrete divergence diagnostic (Sec. 2.1.1: CT keeps div B at round-off):
 * *out = max over active cells of |div_h B| * min(dx) / max(rms |b_c|, 1e-300).  Blocks.
 * Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_divb_norm(vl2_mesh* mesh, double* out);

/* Volume integrals over the active cells: out[0..7] = sum(rho, M1, M2, M3, E, b_c1, b_c2, b_c3) dV,
 * FP64 with a fixed reduction order (deterministic).  Blocks.  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_totals(vl2_mesh* mesh, double out[8]);

/* Total number of cons->prim floor events on active cells since creation.  Blocks. */
vl2_status vl2_floor_count(vl2_mesh* mesh, long long* out);

/* Passive scalars (eq. passive_scalars).  vl2_set_scalars takes concentrations c[nscalars][NZ][NY][NX]
 * (C_i, the primitive form) and sets rho C_i = rho c_i on the active cells from the current density, so the
 * state must be set first; ghosts are exchanged.  vl2_get_scalars returns the scalar masses rho C_i in the
 * same layout.  Each scalar's flux is the Riemann mass flux times the upwind side's concentration,
 * reconstructed like the primitives of the stage.  Errors: VL2_E_ARG (no scalars, NULL, bad where),
 * VL2_E_STATE (state not set), VL2_E_CUDA. */
vl2_status vl2_set_scalars(vl2_mesh* mesh, const double* c, int where);
vl2_status vl2_get_scalars(vl2_mesh* mesh, double* out, int where);

/* Forcing (the paper defines none; this library's reading): a fixed body acceleration a(x) at the cell
 * centres, a = [3][NZ][NY][NX] (global cell layout).  Every stage of every integrator then adds the source
 * terms of the stage's state to L: rho a to the momentum and M . a (the force's work) to the energy, in the
 * same update as the flux divergence.  NULL removes the forcing.  Needs a mesh created with
 * params.forcing = 1; a batch reads each mesh's forcing as it was when the batch was created.
 * Errors: VL2_E_ARG (bad where), VL2_E_STATE (params.forcing was 0), VL2_E_CUDA. */
vl2_status vl2_set_forcing(vl2_mesh* mesh, const double* a, int where);

/* Inspection of one stage's terms for the current state (Sec. 3.2.1-3.2.2, 3.1), without updating
 * it: face fluxes of the given reconstruction (VL2_DC, VL2_PLM, or VL2_PPM on a mesh with ng = 3) on the
 * global face grids fx[7][NZ][NY][NX+1],
 * fy[7][NZ][NY+1][NX], fz[7][NZ+1][NY][NX], components in the sweep frame (mass, M_n, M_t1, M_t2,
 * E, B_t1, B_t2) with (n, t1, t2) = (x, y, z), (y, z, x), (z, x, y).  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_debug_fluxes(vl2_mesh* mesh, int recon, double* fx, double* fy, double* fz, int where);

/* Corner EMFs (upwind CT) of the current state for the given reconstruction on the global edge
 * grids e1[NZ+1][NY+1][NX] (E_x), e2[NZ+1][NY][NX+1] (E_y), e3[NZ][NY+1][NX+1] (E_z). */
vl2_status vl2_debug_emfs(vl2_mesh* mesh, int recon, double* e1, double* e2, double* e3, int where);

/* Adjoint of one VL2 cycle (Sec. 3.2.3) with dt held fixed: for the mesh's current state x and the
 * adjoint lam_out of the cycle's output (u [5][NZ][NY][NX] and face fields b1..b3, global layout, device),
 * writes lam_in = J(x)^T lam_out (same layout, device) where J is the Jacobian of the cycle.  The
 * cycle's forward intermediates are recomputed from x, which is left unchanged.  Reverse order: update,
 * upwind-CT EMFs (upwind choices frozen at x; with params.ct_delta > 0 the smoothed weights and their
 * derivative in the face mass fluxes), Riemann fluxes (reverse-mode derivative replaying the
 * forward flux's arithmetic and branches), PLM (limiter switch frozen), cons->prim, ghost exchange;
 * corrector first, then the predictor.  Face entries follow the global layout: the adjoint of face N of a
 * periodic direction is kept apart from face 0 (they are separate array entries).  Needs a mesh created
 * with params.adjoint = 1 and VL2_FP64, and no active floors.  Errors: VL2_E_ARG, VL2_E_STATE,
 * VL2_E_CUDA. */
vl2_status vl2_step_vjp(vl2_mesh* mesh, double dt, const double* lam_u, const double* lam_b1, const double* lam_b2,
                        const double* lam_b3, double* out_u, double* out_b1, double* out_b2, double* out_b3);

/* Bytes of device memory that one cycle recorded by vl2_step_record keeps (a "tape"): the predictor's and
 * corrector's primitives on every cell, their face mass fluxes (with params.ct_delta > 0 also the two face
 * EMFs of each face), and the face fields of both stages.  Needs a mesh created with params.adjoint = 1.
 * Errors: VL2_E_ARG, VL2_E_STATE. */
vl2_status vl2_tape_bytes(const vl2_mesh* mesh, size_t* bytes);

/* One VL2 cycle (Sec. 3.2.3), exactly as vl2_step, that also writes into `tape` (caller-owned device memory
 * of vl2_tape_bytes, 256-byte aligned) everything the cycle's adjoint reads.  A checkpointed rollout
 * replays a segment with it and then runs vl2_step_vjp_recorded backwards over the tapes, instead of
 * letting vl2_step_vjp recompute every cycle a second time.  Work is only enqueued.  Errors: VL2_E_ARG
 * (dt, tape), VL2_E_STATE (no adjoint arrays, no state), VL2_E_CUDA. */
vl2_status vl2_step_record(vl2_mesh* mesh, double dt, void* tape);

/* The adjoint of a cycle recorded by vl2_step_record with the same dt, read from its tape alone: the
 * same lam_in = J(x)^T lam_out as vl2_step_vjp at that cycle's starting state x (bitwise), without
 * recomputing the cycle.  The mesh's state is neither read nor changed.  Arguments and layouts as
 * vl2_step_vjp.  Errors: VL2_E_ARG, VL2_E_STATE, VL2_E_CUDA. */
vl2_status vl2_step_vjp_recorded(vl2_mesh* mesh, double dt, const void* tape, const double* lam_u,
                                 const double* lam_b1, const double* lam_b2, const double* lam_b3, double* out_u,
                                 double* out_b1, double* out_b2, double* out_b3);

/* Pointwise reverse-mode derivative of the Riemann flux (Sec. 3.2.2) used by vl2_step_vjp, for checking it
 * against an independent Jacobian: for n interfaces q with sweep-frame states wl[q][7], wr[q][7]
 * (rho, v_n, v_t1, v_t2, p, b_t1, b_t2), normal field bn[q] and flux adjoint lf[q][7] (mass, M_n, M_t1,
 * M_t2, E, B_t1, B_t2), writes out[q][k] = sum_m lf[q][m] dF_m/dx_k with x = (wl[0..6], wr[0..6], bn).
 * riemann: VL2_HLLD or VL2_HLLE; gamma > 1.  All arrays are device memory owned by the caller, row-major
 * as shown; the work is enqueued on `stream` (cudaStream_t, may be NULL) and the call does not wait.
 * Errors: VL2_E_ARG (NULL pointer, n < 0, bad riemann or gamma), VL2_E_CUDA. */
vl2_status vl2_debug_riemann_vjp(int riemann, long long n, const double* wl, const double* wr, const double* bn,
                                 const double* lf, double gamma, double* out, void* stream);

/* Adjoint of the set-up map prims -> conserved (eq. total_energy) with the field held fixed: from the
 * primitives w = [5][N] (rho, v, p; device, global layout) and lam_u = [5][N] (device), writes
 * lam_w = [5][N] (device).  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_prims_vjp(vl2_mesh* mesh, const double* w, const double* lam_u, double* lam_w);

/* Measurement aid (the paper has no counterpart): enqueue on `stream` one launch of `ctas` CTAs of
 * `threads` threads (32..256, a multiple of 32), each thread running 16 independent chains of `iters`
 * FP64 fused multiply-adds: 2 * 16 * iters * ctas * threads FP64 operations, with no memory traffic.
 * The caller times it (CUDA events on the same stream) to measure the FP64 peak that the roofline of the
 * FP64-bound kernels is stated against.  out: one device double, written only if the chains reach a
 * value they never reach (it keeps the arithmetic live).  Errors: VL2_E_ARG, VL2_E_CUDA. */
vl2_status vl2_debug_fp64_peak(long long iters, int ctas, int threads, double* out, void* stream);

/* Functions of vl2_debug_arith: this library's FP64 forms (Newton-refined reciprocal, reciprocal square
 * root and square root, and the variants that take any non-negative or non-zero input), its integer-pipe
 * conversions (double -> float rounded to nearest even, float -> double), and CUDA's own operations for
 * comparison (IEEE 1/x and sqrt, CUDA rsqrt, __double2float_rn). */
enum {
  VL2_AR_RCP_NR = 0, VL2_AR_RSQRT_NR = 1, VL2_AR_SQRT_NR = 2, VL2_AR_INV_ANY = 3, VL2_AR_ROOT_ANY = 4,
  VL2_AR_RROOT_ANY = 5, VL2_AR_TO_F32 = 6, VL2_AR_TO_F64 = 7, VL2_AR_IEEE_RCP = 8, VL2_AR_IEEE_SQRT = 9,
  VL2_AR_CUDA_RSQRT = 10, VL2_AR_CUDA_D2F = 11, VL2_AR_COUNT = 12
};

/* Test aid (the paper has no counterpart): out[i] = fn(x[i]) for i < n on the device, x and out device arrays
 * of n doubles owned by the caller; float results are returned widened exactly to double, and
 * VL2_AR_TO_F64 takes inputs that are floats (it converts (float)x[i]).  Domains of the Newton forms:
 * VL2_AR_RCP_NR needs 2^-1022 <= |x| < 2^1021 (near 2^1022 and above, the hardware seed flushes and
 * the result is 0); VL2_AR_RSQRT_NR and VL2_AR_SQRT_NR need normal x > 0 (SQRT_NR also takes +0); the _ANY variants
 * take every finite input of their domain.  Enqueued on `stream`; the call does not wait.
 * Errors: VL2_E_ARG (fn out of range, n < 0, NULL array), VL2_E_CUDA. */
vl2_status vl2_debug_arith(int fn, long long n, const double* x, double* out, void* stream);

/* Test aid for the bounded waits (the paper has no counterpart): one thread waits, with the wait the
 * TMA-staged kernels use, at most `polls` times (each a try-wait and a 256 ns sleep) on an mbarrier phase
 * that nothing completes, then writes out[0] = 1 (device int owned by the caller) when it gave up, which is
 * the expected outcome; the kernel then returns and the context stays usable.  Enqueued on `stream`.
 * Errors: VL2_E_ARG (out NULL, polls outside 1 .. 2^20), VL2_E_CUDA. */
vl2_status vl2_debug_wait_timeout(int polls, int* out, void* stream);

/* Kernel kinds of vl2_profile_read. */
enum {
  VL2_K_PRIM = 0,     /* cons -> prim on every cell (with the fused CFL reduction after a cycle) */
  VL2_K_GHOSTS = 1,   /* ghost exchange of U and the face field */
  VL2_K_FLUX_DC = 2,  /* donor-cell + Riemann fluxes of one sweep direction (units: faces) */
  VL2_K_FLUX_PLM = 3, /* PLM + Riemann fluxes of one sweep direction (units: faces) */
  VL2_K_EMF = 4,      /* upwind CT corner EMFs (units: corner nodes) */
  VL2_K_UPDATE = 5,   /* register update of U and the face field (units: nodes) */
  VL2_K_FLUX_PPM = 6, /* PPM + Riemann fluxes of one sweep direction (units: faces) */
  VL2_K_SCALARS = 7,  /* passive-scalar fluxes and updates */
  VL2_K_FLUX_HALO = 8, /* copy of the faces just outside each block's transverse range (mass flux and transverse
                          induction fluxes, for the CT corners) from the neighbouring block that computed them,
                          on fully periodic meshes (units: faces) */
  VL2_K_COUNT = 9
};

/* Per-kernel timing, the measuring side of the paper's zone-cycles-per-second benchmarks (Sec. 3.4.1).
 * vl2_profile(mesh, 1) brackets every later kernel launch of the mesh with CUDA events on its stream;
 * vl2_profile_read() waits for the stream, then returns and resets the accumulated device time (ms),
 * the launch count and the work units (cells, faces or nodes) of one kernel kind.  Events are owned
 * by the mesh.  Errors: VL2_E_ARG (NULL, bad kind), VL2_E_CUDA. */
vl2_status vl2_profile(vl2_mesh* mesh, int enable);
vl2_status vl2_profile_read(vl2_mesh* mesh, int kind, double* ms, long long* launches, long long* units);

/* Number of CUDA kernels this mesh has launched since creation (every launch, profiled or not). */
vl2_status vl2_launch_count(const vl2_mesh* mesh, long long* n);

/* Launch shapes of this mesh's face-flux kernels (Sec. 3.2.1-3.2.2 sweeps); they change no result bit.
 * dc_threads: CTA size of the donor-cell predictor sweeps, 64, 128 or 256.  plm_lines: lines of faces per
 * tile of the PLM corrector sweeps, 4, 8 or 16.  tma: 0 takes the line-tile PLM kernel (one CTA per tile,
 * primitives loaded by each thread); 1 takes the persistent PLM kernel, whose CTAs (as many as fit on the
 * GPU) walk the tiles and stage each tile's primitives (the mb+4 cells along the sweep, the tile's lines,
 * all 8 variables) in shared memory with one TMA bulk tensor copy, the next tile's copy in flight while the
 * current one is solved.  tma = 1 needs the tensor maps vl2_mesh_create encodes for meshes with two ghost
 * layers, and a tile that fits in shared memory; elsewhere, and for other reconstructions, the line-tile
 * kernel runs.  A new mesh starts with (128, 16, 0): on GB300 the line-tile kernel measured faster in both
 * precisions.  Errors: VL2_E_ARG (NULL mesh, values outside the sets). */
vl2_status vl2_set_flux_shape(vl2_mesh* mesh, int dc_threads, int plm_lines, int tma);

/* The launch shapes set above; tma_active (may be NULL) receives 1 when the PLM sweeps actually take the
 * TMA-staged kernel with these shapes.  Outputs may be NULL.  Errors: VL2_E_ARG. */
vl2_status vl2_get_flux_shape(const vl2_mesh* mesh, int* dc_threads, int* plm_lines, int* tma, int* tma_active);

/* ---- Batched form ----------------------------------------------------------------------------
 * Many independent meshes ("boxes", any sizes; the paper advances each MeshBlock independently between
 * exchanges, Sec. 2.1, 2.6) advanced together: each kernel of the VL2 cycle is one launch over a
 * (box, tile) work list that covers every box; each box keeps its own CFL time step (Sec. 2.1.7) on the
 * device; vl2_batch_run captures K cycles in one CUDA graph and launches it once.
 * The batch refers to the meshes' own device arrays (no copy): results are read back with the mesh calls
 * (vl2_get_cons, vl2_new_dt, ...).  All meshes need the VL2 integrator, no passive scalars, and the same
 * Riemann solver, precision, reconstruction and ct_delta; they must not be stepped through their own
 * calls while a batch call runs; the batch uses the first mesh's stream.
 * The caller owns the batch workspace (vl2_batch_workspace_bytes, 256-byte aligned) and the meshes; the
 * batch must be destroyed before its meshes. */
typedef struct vl2_batch vl2_batch;

/* Bytes of device workspace for a batch of these meshes (mesh views, per-box dt, work lists).
 * Errors: VL2_E_ARG (NULL, n <= 0, meshes that do not share the options above). */
vl2_status vl2_batch_workspace_bytes(vl2_mesh* const* meshes, int n, size_t* bytes);

/* Create the batch (builds and uploads its work lists).  It starts with the first mesh's flux launch shapes
 * (vl2_set_flux_shape), the TMA-staged PLM kernel only where it serves every mesh, so that by default each
 * box advances with the kernels it takes alone.  Errors: VL2_E_ARG, VL2_E_NOMEM, VL2_E_CUDA. */
vl2_status vl2_batch_create(vl2_mesh* const* meshes, int n, void* workspace, size_t bytes, vl2_batch** out);

vl2_status vl2_batch_destroy(vl2_batch* batch);

/* Pick the launch shapes of the flux kernels by timing them on the batch's current state (donor-cell CTA
 * size in {64, 128, 256}, PLM lines per CTA in {4, 8, 16}, and the PLM kernel: line tiles or persistent
 * TMA-staged tiles, see vl2_set_flux_shape); the state is not changed.  Outputs may be NULL.  Blocks.
 * Errors: VL2_E_STATE, VL2_E_CUDA. */
vl2_status vl2_batch_autotune(vl2_batch* batch, int* dc_threads, int* plm_lines);

/* The batch's current flux launch shapes (as vl2_get_flux_shape).  Outputs may be NULL.  Errors: VL2_E_ARG. */
vl2_status vl2_batch_flux_shape(const vl2_batch* batch, int* dc_threads, int* plm_lines, int* tma);

/* Set the batch's flux launch shapes (values as vl2_set_flux_shape) and rebuild its work lists; a captured
 * graph is dropped.  Errors: VL2_E_ARG (values outside the sets, or tma = 1 where the TMA-staged kernel does
 * not serve every mesh of the batch), VL2_E_CUDA. */
vl2_status vl2_batch_set_flux_shape(vl2_batch* batch, int dc_threads, int plm_lines, int tma);

/* One VL2 cycle of every box with the given per-box steps dt[n] (host or device, see `where`); the same
 * arithmetic as vl2_step on each mesh.  Errors: VL2_E_ARG (dt not finite and positive), VL2_E_STATE,
 * VL2_E_CUDA. */
vl2_status vl2_batch_step(vl2_batch* batch, const double* dt, int where);

/* nsteps VL2 cycles of every box, each with the box's own CFL step dt = cfl * (min over its active cells
 * of dx_d / (|v_d| + C_f,d)) formed on the device, as one CUDA-graph launch (captured on the first call
 * with this nsteps, then reused).  dt_last (host, n doubles, may be NULL) receives the last steps used;
 * with dt_last NULL the call only enqueues.  Errors: VL2_E_ARG, VL2_E_STATE, VL2_E_CUDA. */
vl2_status vl2_batch_run(vl2_batch* batch, int nsteps, double* dt_last);

/* Kernels launched by this batch since creation (a graph launch counts its kernels). */
vl2_status vl2_batch_launch_count(const vl2_batch* batch, long long* n);

/* Message of the last failing batch call (or of the last failing call with no batch, if NULL). */
const char* vl2_batch_last_error(const vl2_batch* batch);

/* Largest nz that vl2_totals_noalloc accepts: its fixed scratch holds one row of partial sums per
 * z-plane (VL2_NOALLOC_MAX_NZ x 8 doubles = 256 KiB per device). */
#define VL2_NOALLOC_MAX_NZ 4096

/* vl2_totals without any device allocation, for callers that cannot call cudaMalloc (a host that has
 * given all device memory to its own pool and forbids further allocations, or a pipeline that must not
 * take the device-wide synchronisation an allocation or free can cause).  The paper has no
 * counterpart: it is a deployment aid.
 * Inputs: a state in the global layout as device arrays u [5][NZ][NY][NX] (rho, M1, M2, M3, E) and the
 * face fields b1, b2, b3; nx = (NX, NY, NZ); dx = cell widths.  Output: out, a device array of 8 doubles,
 * receives the volume integrals of rho, M1, M2, M3, E, b_c1, b_c2, b_c3 (b_c the mean of the two face
 * values), with a fixed summation order.  Work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream) and the call returns without waiting.
 * Memory: the partial sums go to a file-scope device array that this library reserves on every GPU that
 * loads it, until the process exits; nothing is allocated or freed.  The first call on a device looks up
 * that array's device address with the device current, so make that first call before any stream
 * capture begins.  The address is kept for the life of the process: a device reset (cudaDeviceReset, or
 * any teardown of the device's primary context) leaves it stale, so do not call this entry point on a
 * device after resetting it.  All calls share the array: calls whose work overlaps on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Every slot a call reads it first writes, so
 * no clearing is needed between calls.
 * Errors: VL2_E_ARG (NULL pointer, non-positive size, nz > VL2_NOALLOC_MAX_NZ), VL2_E_CUDA; the message
 * is available from vl2_last_error(NULL). */
vl2_status vl2_totals_noalloc(const double* u, const double* b1, const double* b2, const double* b3,
                              const int nx[3], const double dx[3], double* out, void* stream);

/* Message of the last failing call on `mesh` (or of the last failing call with no mesh, if NULL).
 * The string is owned by the library. */
const char* vl2_last_error(const vl2_mesh* mesh);

#ifdef __cplusplus
}
#endif

#endif /* VL2MHD_H */
