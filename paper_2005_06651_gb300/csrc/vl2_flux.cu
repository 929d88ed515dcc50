// Face-flux kernels of the VL2 MHD step: reconstruction (donor cell, or PLM with the van Leer limiter,
// Sec. 3.2.1) and the HLLD / HLLE Riemann fluxes (Sec. 3.2.2) on every face a MeshBlock needs.  Each
// kernel runs either on one mesh (tile = blockIdx.x) or on a batch of meshes through a (box, tile)
// work list; the mesh view is staged in shared memory once per CTA.
#include "vl2_internal.h"
#include "vl2_physics.cuh"
#include "vl2_tma.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

namespace vl2 {

// Per-mesh constants in the stage's precision: the FP32 forms take the mesh's precomputed FP32 copies instead of
// converting per thread.  (The FP64 face field keeps the hardware conversion: narrowing it on the integer pipe
// measured slower in the FP32 sweeps, whose busiest pipe is the integer one.)
template <class T> __device__ __forceinline__ T stage_gamma(const Geom& g);
template <> __device__ __forceinline__ double stage_gamma<double>(const Geom& g) { return g.gamma; }
template <> __device__ __forceinline__ float stage_gamma<float>(const Geom& g) { return g.gamma_f; }
template <class T> __device__ __forceinline__ T stage_igm1(const Geom& g);
template <> __device__ __forceinline__ double stage_igm1<double>(const Geom& g) { return g.igm1; }
template <> __device__ __forceinline__ float stage_igm1<float>(const Geom& g) { return g.igm1_f; }

// ------------------------------------------------------------------------------------------------
// Predictor fluxes, one thread per face.  Faces of direction DIR cover the block's active faces along
// DIR (ng .. ng+mb) and its active cells transversally (ng .. ng+mb-1); with g.flux_halo also one ghost
// layer transversally (ng-1 .. ng+mb), whose faces feed the corner EMFs on the block surface (otherwise
// k_flux_halo copies those from the neighbouring blocks).
// ------------------------------------------------------------------------------------------------
template <int DIR, int REC, int RS, class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_flux(MeshView single, const MeshView* views, const WorkItem* work, int reg) {
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, views, work, tile);
  const Geom& g = V.g;
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  const int h = g.flux_halo;
  const int rx = g.mb[0] + (DIR == 0 ? 1 : 2 * h);
  const int ry = g.mb[1] + (DIR == 1 ? 1 : 2 * h);
  const int rz = g.mb[2] + (DIR == 2 ? 1 : 2 * h);
  const long long per = (long long)rx * ry * rz;
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % rx + (DIR == 0 ? g.ng : g.ng - h);
  rem /= rx;
  const int j = rem % ry + (DIR == 1 ? g.ng : g.ng - h);
  const int k = rem / ry + (DIR == 2 ? g.ng : g.ng - h);
  const long long c = cell_off(g, k, j, i);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  const T* Wb = static_cast<const T*>(V.a.w) + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  T wl[7], wr[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const T* q = Wb + (long long)var[n] * g.box + c;
    if (REC == REC_DC) {
      wl[n] = q[-sd];
      wr[n] = q[0];
    } else {
      const T qm2 = q[-2 * sd], qm1 = q[-sd], q0 = q[0], qp1 = q[sd];
      wl[n] = qm1 + T(0.5) * vl_slope(qm2, qm1, q0);
      wr[n] = q0 - T(0.5) * vl_slope(qm1, q0, qp1);
    }
  }
  const T bn = (T)V.a.b[reg][DIR][(long long)b * g.box + c];
  T f[7];
  if (RS == RS_HLLD)
    flux_hlld<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), f);
  else
    flux_hlle<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), f, g.hlle_roe != 0);
  T* Fb = static_cast<T*>(V.a.f[DIR]) + (long long)b * 7 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = f[n];
}

// ------------------------------------------------------------------------------------------------
// Corrector fluxes with each cell's reconstruction formed once (Sec. 3.2.1).  A CTA takes P lines of faces
// along DIR: phase A reconstructs the mb+2 cells of each line (ng-1 .. ng+mb) into shared memory (the
// cell's values at its lower and upper faces, 7 variables), phase B solves the mb+1 Riemann problems of each
// line from shared memory.  PLM: q -+ delta/2, each limiter denominator inverted by the Newton reciprocal
// (sharing one reciprocal among the 7 variables of a cell through their products measured no faster and
// needed a range fallback).  PPM (ng = 3): phase A first
// forms the mb+3 limited face values of each line once (a face is shared by the cells on its two sides)
// into shared memory behind the edge arrays, then limits each cell's parabola from its two faces.
// ------------------------------------------------------------------------------------------------
template <int DIR>
struct LineMap {
  // transverse directions ordered so that the fastest-varying memory index comes first
  static constexpr int TA = (DIR == 0) ? 1 : 0;
  static constexpr int TB = (DIR == 2) ? 1 : 2;
};

template <int DIR, int RS, class T, int REC>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_flux_plm(MeshView single, const MeshView* views, const WorkItem* work,
                                                     int reg, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  __shared__ MeshView sv;
  int tile_all;
  const MeshView& V = stage_view(sv, single, views, work, tile_all);
  const Geom& g = V.g;
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int TA = LineMap<DIR>::TA, TB = LineMap<DIR>::TB;
  const int L = g.mb[DIR] + 2;   // reconstructed cells per line
  const int NF = g.mb[DIR] + 1;  // faces per line
  const int h = g.flux_halo;     // lines of the transverse halo too (see k_flux)
  const int na = g.mb[TA] + 2 * h, nb = g.mb[TB] + 2 * h;
  const int nlines = na * nb;
  const int tiles = (nlines + P - 1) / P;
  const int b = tile_all / tiles;
  const int tile = tile_all - b * tiles;
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const long long sd = stride[DIR];
  const T* Wb = static_cast<const T*>(V.a.w) + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  // shared layout: the fastest thread index is contiguous
  auto sidx = [&](int v, int side, int p, int c) -> int {
    return (DIR == 0) ? (((v * 2 + side) * P + p) * L + c) : (((v * 2 + side) * L + c) * P + p);
  };
  if constexpr (REC == REC_PPM) {
    // phase A1: the limited face values 0 .. L of every line; face f is the lower face of cell ng-1+f
    T* fsm = smem + (size_t)14 * P * L;
    auto fidx = [&](int v, int p, int f) -> int {
      return (DIR == 0) ? ((v * P + p) * (L + 1) + f) : ((v * (L + 1) + f) * P + p);
    };
    for (int t = threadIdx.x; t < P * (L + 1); t += blockDim.x) {
      const int p = (DIR == 0) ? t / (L + 1) : t % P;
      const int f = (DIR == 0) ? t % (L + 1) : t / P;
      const int line = tile * P + p;
      if (line >= nlines) continue;
      int li[3];
      li[DIR] = g.ng - 1 + f;
      li[TA] = g.ng - h + line % na;
      li[TB] = g.ng - h + line / na;
      const long long o = cell_off(g, li[2], li[1], li[0]);
#pragma unroll
      for (int n = 0; n < 7; ++n) {
        const T* q = Wb + (long long)var[n] * g.box + o;
        fsm[fidx(n, p, f)] = ppm_face(q[-2 * sd], q[-sd], q[0], q[sd]);
      }
    }
    __syncthreads();
    // phase A2: each cell's edges from its two faces
    for (int t = threadIdx.x; t < P * L; t += blockDim.x) {
      const int p = (DIR == 0) ? t / L : t % P;
      const int c = (DIR == 0) ? t % L : t / P;
      const int line = tile * P + p;
      if (line >= nlines) continue;
      int li[3];
      li[DIR] = g.ng - 1 + c;
      li[TA] = g.ng - h + line % na;
      li[TB] = g.ng - h + line / na;
      const long long o = cell_off(g, li[2], li[1], li[0]);
#pragma unroll
      for (int n = 0; n < 7; ++n) {
        const T* q = Wb + (long long)var[n] * g.box + o;
        T ql = fsm[fidx(n, p, c)], qr = fsm[fidx(n, p, c + 1)];
        ppm_cell(q[-2 * sd], q[-sd], q[0], q[sd], q[2 * sd], ql, qr);
        smem[sidx(n, 0, p, c)] = ql;
        smem[sidx(n, 1, p, c)] = qr;
      }
    }
  }
  // phase A'': characteristic PPM of each cell from its five-cell stencil
  for (int t = threadIdx.x; REC == REC_PPM_CHAR && t < P * L; t += blockDim.x) {
    const int p = (DIR == 0) ? t / L : t % P;
    const int c = (DIR == 0) ? t % L : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = g.ng - 1 + c;
    li[TA] = g.ng - h + line % na;
    li[TB] = g.ng - h + line / na;
    const long long o = cell_off(g, li[2], li[1], li[0]);
    T qs[5][7], lo[7], hi[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const T* q = Wb + (long long)var[n] * g.box + o;
#pragma unroll
      for (int j = 0; j < 5; ++j) qs[j][n] = q[(j - 2) * sd];
    }
    char_ppm_cell<T>(qs, Wb[(long long)(5 + DIR) * g.box + o], stage_gamma<T>(g), lo, hi);
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      smem[sidx(n, 0, p, c)] = lo[n];
      smem[sidx(n, 1, p, c)] = hi[n];
    }
  }
  // phase A': reconstruct cells on characteristic variables (its face values, clamped to the neighbours)
  for (int t = threadIdx.x; REC == REC_PLM_CHAR && t < P * L; t += blockDim.x) {
    const int p = (DIR == 0) ? t / L : t % P;
    const int c = (DIR == 0) ? t % L : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = g.ng - 1 + c;
    li[TA] = g.ng - h + line % na;
    li[TB] = g.ng - h + line / na;
    const long long o = cell_off(g, li[2], li[1], li[0]);
    T qm[7], q0[7], qp[7], lo[7], hi[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const T* q = Wb + (long long)var[n] * g.box + o;
      qm[n] = q[-sd];
      q0[n] = q[0];
      qp[n] = q[sd];
    }
    char_plm_cell<T>(qm, q0, qp, Wb[(long long)(5 + DIR) * g.box + o], stage_gamma<T>(g), lo, hi);
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      smem[sidx(n, 0, p, c)] = lo[n];
      smem[sidx(n, 1, p, c)] = hi[n];
    }
  }
  // phase A: reconstruct cells (PLM)
  for (int t = threadIdx.x; REC == REC_PLM && t < P * L; t += blockDim.x) {
    const int p = (DIR == 0) ? t / L : t % P;
    const int c = (DIR == 0) ? t % L : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = g.ng - 1 + c;
    li[TA] = g.ng - h + line % na;
    li[TB] = g.ng - h + line / na;
    const long long o = cell_off(g, li[2], li[1], li[0]);
    T qm[7], qc[7], qp[7], lo[7], hi[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const T* q = Wb + (long long)var[n] * g.box + o;
      qm[n] = q[-sd];
      qc[n] = q[0];
      qp[n] = q[sd];
    }
    plm_cell_faces<T>(qm, qc, qp, lo, hi);
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      smem[sidx(n, 0, p, c)] = lo[n];  // value at the cell's lower face
      smem[sidx(n, 1, p, c)] = hi[n];  // value at the cell's upper face
    }
  }
  __syncthreads();
  // phase B: Riemann problems of the faces ng .. ng+mb of every line
  const double* Bn = V.a.b[reg][DIR];
  for (int t = threadIdx.x; t < P * NF; t += blockDim.x) {
    const int p = (DIR == 0) ? t / NF : t % P;
    const int f = (DIR == 0) ? t % NF : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = g.ng + f;
    li[TA] = g.ng - h + line % na;
    li[TB] = g.ng - h + line / na;
    const long long o = cell_off(g, li[2], li[1], li[0]);
    T wl[7], wr[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      wl[n] = smem[sidx(n, 1, p, f)];      // upper-face value of cell ng-1+f
      wr[n] = smem[sidx(n, 0, p, f + 1)];  // lower-face value of cell ng+f
    }
    const T bn = (T)Bn[(long long)b * g.box + o];
    T fl[7];
    if (RS == RS_HLLD)
      flux_hlld<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), fl);
    else
      flux_hlle<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), fl, g.hlle_roe != 0);
    T* Fb = static_cast<T*>(V.a.f[DIR]) + (long long)b * 7 * g.box + o;
#pragma unroll
    for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = fl[n];
  }
}

// ------------------------------------------------------------------------------------------------
// Corrector fluxes (PLM, Sec. 3.2.1, and the Riemann fluxes of Sec. 3.2.2) by persistent CTAs whose
// primitive tiles are staged in shared memory by TMA.  A tile is P lines of faces along DIR, adjacent along
// the faster transverse direction TA, in one TB row of one block; its primitives are one 4D box of w (see
// tma_w_box), loaded by a single bulk tensor copy that completes on an mbarrier.  Each CTA walks the work
// items blockIdx.x, blockIdx.x + gridDim.x, ... and copies the next item's box into the second of two buffers
// while it reconstructs and solves the current one, so the loads of w overlap the arithmetic.  Per tile the
// arithmetic is that of k_flux_plm (REC_PLM): phase A limits each cell's slope once into shared memory,
// phase B solves the faces, with the same operations in the same order, so both kernels give the same bits.
// A bounded wait that expires sets scal[SC_TIMEOUT] and the CTA returns after its copies have landed.
// ------------------------------------------------------------------------------------------------
constexpr int TMA_WAIT_POLLS = 1 << 20;  // polls of an mbarrier (each with a 256 ns sleep) before giving up

template <int DIR, int RS, class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2)
    k_flux_tma(MeshView single, const MeshView* views, const WorkItem* work, int nitems, int reg, int P, int wcap) {
  extern __shared__ __align__(128) unsigned char tile_smem[];  // its own name: the line kernel's is 16-aligned
  __shared__ MeshView sv;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int landed;
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int TA = LineMap<DIR>::TA, TB = LineMap<DIR>::TB;
  T* rec = reinterpret_cast<T*>(tile_smem + 2 * (size_t)wcap);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  // thread 0: start the copy of item i's box into buffer k
  auto issue = [&](int i, int k) {
    const MeshView* mv = &single;
    int tile = i;
    if (work) {
      const WorkItem w = work[i];
      mv = views + w.box;
      tile = w.tile;
    }
    const Geom& g = mv->g;
    const int h = g.flux_halo;
    const int na = g.mb[TA] + 2 * h, nbl = g.mb[TB] + 2 * h;
    const int tpr = (na + P - 1) / P;
    const int b = tile / (nbl * tpr);
    const int r = tile - b * (nbl * tpr);
    const int tb = r / tpr, ta0 = (r - tb * tpr) * P;
    int box[4], xoff;
    tma_w_box(g, DIR, P, (int)sizeof(T), box, &xoff);
    int c[4];
    c[DIR] = g.ng - 2;
    c[TA] = g.ng - h + ta0 - xoff;
    c[TB] = g.ng - h + tb;
    c[3] = 8 * b;
    const uint32_t bytes = (uint32_t)(box[0] * box[1] * box[2] * box[3]) * (uint32_t)sizeof(T);
    fence_proxy_async_smem();  // the CTA's reads of this buffer (previous item) come before the copy's writes
    mbar_arrive_expect_tx(&bar[k], bytes);
    tma_load_4d(tile_smem + (size_t)k * wcap, static_cast<const unsigned char*>(mv->a.tmw) + 128 * tma_map_index(DIR, P),
                c[0], c[1], c[2], c[3], &bar[k]);
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < nitems) issue((int)blockIdx.x, 0);
  int k = 0;
  for (int item = (int)blockIdx.x; item < nitems; item += (int)gridDim.x, ++k) {
    const int buf = k & 1;
    const uint32_t parity = (uint32_t)((k >> 1) & 1);
    const bool more = item + (int)gridDim.x < nitems;
    if (threadIdx.x == 0 && more) issue(item + (int)gridDim.x, buf ^ 1);
    int tile;
    const MeshView& V = stage_view_item(sv, single, views, work, item, tile);
    const Geom& g = V.g;
    if (threadIdx.x == 0) landed = mbar_wait_bounded(&bar[buf], parity, TMA_WAIT_POLLS) ? 1 : 0;
    __syncthreads();
    if (!landed) {
      if (threadIdx.x == 0) {
        atomicOr(V.a.scal + SC_TIMEOUT, 1ULL);
        mbar_wait_bounded(&bar[buf], parity, TMA_WAIT_POLLS);  // let this CTA's copies land before it exits
        if (more) mbar_wait_bounded(&bar[buf ^ 1], (uint32_t)(((k + 1) >> 1) & 1), TMA_WAIT_POLLS);
      }
      return;
    }
    mbar_wait_bounded(&bar[buf], parity, TMA_WAIT_POLLS);  // completed: each thread observes the copied bytes
    const int h = g.flux_halo;
    const int na = g.mb[TA] + 2 * h, nbl = g.mb[TB] + 2 * h;
    const int tpr = (na + P - 1) / P;
    const int b = tile / (nbl * tpr);
    const int r = tile - b * (nbl * tpr);
    const int tb = r / tpr, ta0 = (r - tb * tpr) * P;
    const int L = g.mb[DIR] + 2;   // reconstructed cells per line
    const int NF = g.mb[DIR] + 1;  // faces per line
    const int L4 = g.mb[DIR] + 4;  // cells of the box along DIR
    int box[4], xoff;
    tma_w_box(g, DIR, P, (int)sizeof(T), box, &xoff);
    const T* Ws = reinterpret_cast<const T*>(tile_smem + (size_t)buf * wcap);
    // box element of variable v, DIR index a (0 = cell ng-2), line p
    auto widx = [&](int v, int a, int p) -> int {
      return (DIR == 0) ? (v * P + p) * box[0] + a : (v * L4 + a) * box[0] + xoff + p;
    };
    auto sidx = [&](int v, int side, int p, int c) -> int {
      return (DIR == 0) ? (((v * 2 + side) * P + p) * L + c) : (((v * 2 + side) * L + c) * P + p);
    };
    const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
    // phase A: the lower- and upper-face values of the cells ng-1 .. ng+mb of every line
    for (int t = threadIdx.x; t < P * L; t += blockDim.x) {
      const int p = (DIR == 0) ? t / L : t % P;
      const int c = (DIR == 0) ? t % L : t / P;
      if (ta0 + p >= na) continue;
      T qm[7], qc[7], qp[7], lo[7], hi[7];
#pragma unroll
      for (int n = 0; n < 7; ++n) {
        qm[n] = Ws[widx(var[n], c, p)];
        qc[n] = Ws[widx(var[n], c + 1, p)];
        qp[n] = Ws[widx(var[n], c + 2, p)];
      }
      plm_cell_faces<T>(qm, qc, qp, lo, hi);
#pragma unroll
      for (int n = 0; n < 7; ++n) {
        rec[sidx(n, 0, p, c)] = lo[n];
        rec[sidx(n, 1, p, c)] = hi[n];
      }
    }
    __syncthreads();
    // phase B: Riemann problems of the faces ng .. ng+mb of every line
    const double* Bn = V.a.b[reg][DIR];
    for (int t = threadIdx.x; t < P * NF; t += blockDim.x) {
      const int p = (DIR == 0) ? t / NF : t % P;
      const int f = (DIR == 0) ? t % NF : t / P;
      if (ta0 + p >= na) continue;
      int li[3];
      li[DIR] = g.ng + f;
      li[TA] = g.ng - h + ta0 + p;
      li[TB] = g.ng - h + tb;
      const long long o = cell_off(g, li[2], li[1], li[0]);
      T wl[7], wr[7];
#pragma unroll
      for (int n = 0; n < 7; ++n) {
        wl[n] = rec[sidx(n, 1, p, f)];
        wr[n] = rec[sidx(n, 0, p, f + 1)];
      }
      const T bn = (T)Bn[(long long)b * g.box + o];
      T fl[7];
      if (RS == RS_HLLD)
        flux_hlld<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), fl);
      else
        flux_hlle<T>(wl, wr, bn, stage_gamma<T>(g), stage_igm1<T>(g), fl, g.hlle_roe != 0);
      T* Fb = static_cast<T*>(V.a.f[DIR]) + (long long)b * 7 * g.box + o;
#pragma unroll
      for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = fl[n];
    }
    __syncthreads();  // the view, the reconstruction and this buffer are rewritten by the next item
  }
}

// ------------------------------------------------------------------------------------------------
// Halo faces for the CT corners on a block's surface (meshes with flux_halo = 0).  The corners of edge
// family e read the a-faces one cell outside the block along b and the b-faces one cell outside along a
// (a, b the directions transverse to e): the mass flux (upwind choice) and the transverse induction fluxes
// (face EMFs).  Those faces lie in the neighbouring block's own transverse range, where the same arithmetic
// on the same cells computed them, so they are copied: components 0, 5 and 6 of the d-faces at normal
// index ng .. ng+mb_d on the four sides t = ng-1 / ng+mb of each transverse direction t (the other transverse
// index over the active range; the corner lines outside both are not read).  One thread per face, with the
// lower of the two free dimensions (memory order) fastest.
// ------------------------------------------------------------------------------------------------
__host__ __device__ inline long long halo_side_faces(const Geom& g, int d, int t) {
  const int o = 3 - d - t;  // the other transverse direction
  return (long long)(g.mb[d] + 1) * g.mb[o];
}
__host__ __device__ inline long long halo_faces_per_block(const Geom& g) {
  long long n = 0;
  for (int d = 0; d < 3; ++d) n += 2 * (halo_side_faces(g, d, (d + 1) % 3) + halo_side_faces(g, d, (d + 2) % 3));
  return n;
}

template <class T>
__global__ void __launch_bounds__(256) k_flux_halo(MeshView single, const MeshView* views, const WorkItem* work) {
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, views, work, tile);
  const Geom& g = V.g;
  if (g.flux_halo) return;
  const long long per = halo_faces_per_block(g);
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  long long r = t - (long long)b * per;
  // which direction d, transverse side direction s, and lower / upper side
  int d = 0, s = 0, hi = 0;
  for (d = 0; d < 3; ++d) {
    const int s1 = (d + 1) % 3, s2 = (d + 2) % 3;
    const long long n1 = halo_side_faces(g, d, s1), n2 = halo_side_faces(g, d, s2);
    if (r < 2 * n1) {
      s = s1;
      hi = (int)(r / n1);
      r -= hi * n1;
      break;
    }
    r -= 2 * n1;
    if (r < 2 * n2) {
      s = s2;
      hi = (int)(r / n2);
      r -= hi * n2;
      break;
    }
    r -= 2 * n2;
  }
  const int o = 3 - d - s;
  const int f0 = d < o ? d : o;  // the lower free dimension, fastest (the other one is f1 = d + o - f0)
  const int e0 = g.mb[f0] + (f0 == d ? 1 : 0);
  const int a0 = g.ng + (int)(r % e0), a1 = g.ng + (int)(r / e0);  // along f0 and f1
  const int ls = hi ? g.ng + g.mb[s] : g.ng - 1;
  const int ss = hi ? g.ng : g.ng + g.mb[s] - 1;  // the same face in the neighbouring block's own range
  // per-coordinate selects instead of arrays indexed by d, s (which would live in local memory)
  auto pick = [&](int q, int side) { return q == s ? side : (q == f0 ? a0 : a1); };
  // neighbouring block along s (periodic wrap; every neighbour exists on a fully periodic mesh)
  int l0 = b % g.nb[0], l1 = (b / g.nb[0]) % g.nb[1], l2 = b / (g.nb[0] * g.nb[1]);
  const int step = hi ? 1 : g.nb[s] - 1;
  if (s == 0) l0 = (l0 + step) % g.nb[0];
  if (s == 1) l1 = (l1 + step) % g.nb[1];
  if (s == 2) l2 = (l2 + step) % g.nb[2];
  const int bs = (l2 * g.nb[1] + l1) * g.nb[0] + l0;
  T* F = static_cast<T*>(V.a.f[d]);
  const long long dst = (long long)b * 7 * g.box + cell_off(g, pick(2, ls), pick(1, ls), pick(0, ls));
  const long long src = (long long)bs * 7 * g.box + cell_off(g, pick(2, ss), pick(1, ss), pick(0, ss));
  // the sources are faces of the neighbour's own range, which this launch does not write: three loads, then
  // three stores
  const T m = F[src], e1 = F[src + 5 * g.box], e2 = F[src + 6 * g.box];
  F[dst] = m;
  F[dst + 5 * g.box] = e1;
  F[dst + 6 * g.box] = e2;
}

long long tiles_flux_halo(const Geom& g) {
  if (g.flux_halo) return 0;
  return (halo_faces_per_block(g) * g.nblk + 255) / 256;
}

cudaError_t launch_flux_halo(const MeshView& v, const Dispatch* d, cudaStream_t st) {
  const long long grid = d ? d->nwork : tiles_flux_halo(v.g);
  if (grid <= 0) return cudaSuccess;
  const MeshView* vs = d ? d->views : nullptr;
  const WorkItem* wk = d ? d->work : nullptr;
  if (v.a.mixed)
    k_flux_halo<float><<<(unsigned)grid, 256, 0, st>>>(v, vs, wk);
  else
    k_flux_halo<double><<<(unsigned)grid, 256, 0, st>>>(v, vs, wk);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// launch shapes and launchers
// ------------------------------------------------------------------------------------------------
constexpr size_t PLM_SMEM_MAX = 112 * 1024;  // shared bytes one CTA may take (two fit in an SM)

static int lines_ta(const Geom& g, int dir) { return g.mb[dir == 0 ? 1 : 0] + 2 * g.flux_halo; }
static int lines_tb(const Geom& g, int dir) { return g.mb[dir == 2 ? 1 : 2] + 2 * g.flux_halo; }

// Lines per CTA: the requested count, reduced until a CTA's shared memory fits (max_mb = the longest
// line of any mesh sharing the launch).
// PPM adds the line's mb+3 face values of 7 variables.
static size_t line_bytes(int max_mb, int recon, size_t elem) {
  return ((size_t)(max_mb + 2) * 14 + (recon == REC_PPM ? (size_t)(max_mb + 3) * 7 : 0)) * elem;
}

int plm_lines_for(const Geom& g, int dir, const FluxShape& fs, int max_mb, int recon) {
  (void)g;
  (void)dir;
  const size_t per_line = line_bytes(max_mb, recon, sizeof(double));
  int P = fs.plm_lines > 0 ? fs.plm_lines : 16;
  while (P > 1 && (size_t)P * per_line > PLM_SMEM_MAX) --P;
  return P;
}

long long tiles_flux_dc(const Geom& g, int dir, const FluxShape& fs) {
  long long n = g.nblk;
  for (int q = 0; q < 3; ++q) n *= g.mb[q] + (q == dir ? 1 : 2 * g.flux_halo);
  return (n + fs.dc_threads - 1) / fs.dc_threads;
}

long long tiles_flux_plm(const Geom& g, int dir, const FluxShape& fs) {
  const int P = fs.plm_lines;
  const long long nlines = (long long)lines_ta(g, dir) * lines_tb(g, dir);
  return (long long)g.nblk * ((nlines + P - 1) / P);
}

// ---- the TMA-staged PLM path ----
static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// bytes of one primitive buffer of k_flux_tma (largest box of any mesh of the launch), a multiple of 128
static size_t tma_buf_bytes(int dir, int lines, int max_mb, int esize) {
  const int q = 16 / esize;
  const size_t elems = dir == 0 ? (size_t)((max_mb + 4 + q - 1) / q * q) * lines : (size_t)(lines + q) * (max_mb + 4);
  return (elems * 8 * esize + 127) / 128 * 128;
}
static size_t tma_smem(int dir, int lines, int max_mb, int esize) {
  return 2 * tma_buf_bytes(dir, lines, max_mb, esize) + (size_t)14 * lines * (max_mb + 2) * esize;
}

bool flux_tma_applies(const MeshView& v, int recon, const FluxShape& fs, int max_mb) {
  const Geom& g = v.g;
  if (!fs.plm_tma || recon != REC_PLM || !v.a.tmw || g.ng != 2) return false;
  if (fs.plm_lines != 4 && fs.plm_lines != 8 && fs.plm_lines != 16) return false;
  if (max_mb + 4 > 256) return false;
  const int es = v.a.mixed ? 4 : 8;
  for (int d = 0; d < 3; ++d)
    if (tma_smem(d, fs.plm_lines, max_mb, es) > PLM_SMEM_MAX) return false;
  return true;
}

long long tiles_flux_tma(const Geom& g, int dir, int lines) {
  const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
  const long long na = g.mb[ta] + 2 * g.flux_halo, nbl = g.mb[tb] + 2 * g.flux_halo;
  return (long long)g.nblk * nbl * ((na + lines - 1) / lines);
}

bool encode_w_maps(const Geom& g, const void* w, int esize, void* maps, const char** why) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) {
    *why = "the driver offers no cuTensorMapEncodeTiled";
    return false;
  }
  if (g.ng != 2 || (esize != 4 && esize != 8) || ((uintptr_t)w & 255u) || (g.sx * esize) % 16) {
    *why = "w does not meet the TMA layout rules (two ghost layers, 16-byte rows)";
    return false;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)g.sx, (cuuint64_t)g.sy, (cuuint64_t)g.sz, (cuuint64_t)g.nblk * 8};
  const cuuint64_t strides[3] = {(cuuint64_t)g.sx * esize, (cuuint64_t)g.sx * g.sy * esize, (cuuint64_t)g.box * esize};
  const cuuint32_t unit[4] = {1, 1, 1, 1};
  if (dims[3] > 0xffffffffull) {
    *why = "too many MeshBlocks for a TMA tensor";
    return false;
  }
  CUtensorMap* out = static_cast<CUtensorMap*>(maps);
  const int heights[3] = {4, 8, 16};
  for (int dir = 0; dir < 3; ++dir)
    for (int lines : heights) {
      int box[4], xoff;
      tma_w_box(g, dir, lines, esize, box, &xoff);
      cuuint32_t bd[4];
      for (int q = 0; q < 4; ++q) {
        if (box[q] < 1 || box[q] > 256) {
          *why = "a MeshBlock edge is too long for a TMA box";
          return false;
        }
        bd[q] = (cuuint32_t)box[q];
      }
      const CUresult r = encode(&out[tma_map_index(dir, lines)],
                                esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                                const_cast<void*>(w), dims, strides, bd, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled rejected the primitive tensor";
        return false;
      }
    }
  return true;
}

// Resident CTAs per SM of k_flux_tma with this shared memory, cached per instantiation.  The occupancy query
// is not made while `st` is being captured into a graph (a capture records stream work only); an uncached
// shape there takes one CTA per SM, which changes no result.
template <int DIR, int RS, class T>
static int tma_ctas_per_sm(size_t shmem, cudaStream_t st) {
  static std::atomic<long long> cache{-1};  // (shmem << 8) | CTAs per SM
  const long long c = cache.load();
  if (c >= 0 && (size_t)(c >> 8) == shmem) return (int)(c & 255);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flux_tma<DIR, RS, T>, 256, shmem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    return 1;
  }
  per_sm = std::min(per_sm, 255);
  cache.store(((long long)shmem << 8) | per_sm);
  return per_sm;
}

template <int DIR, int RS, class T>
static cudaError_t launch_tma(const MeshView& v, const Dispatch* d, int reg, const FluxShape& fs, int max_mb,
                              cudaStream_t st) {
  const int P = fs.plm_lines;
  const size_t wcap = tma_buf_bytes(DIR, P, max_mb, (int)sizeof(T));
  const size_t shmem = tma_smem(DIR, P, max_mb, (int)sizeof(T));
  const long long items = d ? d->nwork : tiles_flux_tma(v.g, DIR, P);
  if (items <= 0) return cudaSuccess;
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  const long long grid = std::min<long long>(items, (long long)tma_ctas_per_sm<DIR, RS, T>(shmem, st) * sm_count());
  k_flux_tma<DIR, RS, T><<<(unsigned)grid, 256, shmem, st>>>(v, d ? d->views : nullptr, d ? d->work : nullptr,
                                                             (int)items, reg, P, (int)wcap);
  return cudaGetLastError();
}

template <class K>
static cudaError_t set_smem_attr(K kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PLM_SMEM_MAX);
}

template <int DIR, int RS, class T>
static cudaError_t launch_typed(const MeshView& v, const Dispatch* d, int reg, int recon, const FluxShape& fs,
                                int max_mb, cudaStream_t st) {
  const Geom& g = v.g;
  if (flux_tma_applies(v, recon, fs, max_mb)) return launch_tma<DIR, RS, T>(v, d, reg, fs, max_mb, st);
  if (recon == REC_PLM || recon == REC_PPM || recon == REC_PLM_CHAR || recon == REC_PPM_CHAR) {
    FluxShape f2 = fs;
    f2.plm_lines = plm_lines_for(g, DIR, fs, max_mb, recon);
    const size_t shmem = (size_t)f2.plm_lines * line_bytes(max_mb, recon, sizeof(T));
    const long long grid = d ? d->nwork : tiles_flux_plm(g, DIR, f2);
    if (grid <= 0) return cudaSuccess;
    if (recon == REC_PPM)
      k_flux_plm<DIR, RS, T, REC_PPM><<<(unsigned)grid, 256, shmem, st>>>(v, d ? d->views : nullptr,
                                                                         d ? d->work : nullptr, reg, f2.plm_lines);
    else if (recon == REC_PLM_CHAR)
      k_flux_plm<DIR, RS, T, REC_PLM_CHAR><<<(unsigned)grid, 256, shmem, st>>>(
          v, d ? d->views : nullptr, d ? d->work : nullptr, reg, f2.plm_lines);
    else if (recon == REC_PPM_CHAR)
      k_flux_plm<DIR, RS, T, REC_PPM_CHAR><<<(unsigned)grid, 256, shmem, st>>>(
          v, d ? d->views : nullptr, d ? d->work : nullptr, reg, f2.plm_lines);
    else
      k_flux_plm<DIR, RS, T, REC_PLM><<<(unsigned)grid, 256, shmem, st>>>(v, d ? d->views : nullptr,
                                                                         d ? d->work : nullptr, reg, f2.plm_lines);
    return cudaGetLastError();
  }
  const long long grid = d ? d->nwork : tiles_flux_dc(g, DIR, fs);
  if (grid <= 0) return cudaSuccess;
  k_flux<DIR, REC_DC, RS, T><<<(unsigned)grid, fs.dc_threads, 0, st>>>(v, d ? d->views : nullptr,
                                                                        d ? d->work : nullptr, reg);
  return cudaGetLastError();
}

template <int DIR>
static cudaError_t launch_dir(const MeshView& v, const Dispatch* d, int reg, int recon, int riemann,
                              const FluxShape& fs, int max_mb, cudaStream_t st) {
  if (v.a.mixed)
    return riemann == RS_HLLD ? launch_typed<DIR, RS_HLLD, float>(v, d, reg, recon, fs, max_mb, st)
                              : launch_typed<DIR, RS_HLLE, float>(v, d, reg, recon, fs, max_mb, st);
  return riemann == RS_HLLD ? launch_typed<DIR, RS_HLLD, double>(v, d, reg, recon, fs, max_mb, st)
                            : launch_typed<DIR, RS_HLLE, double>(v, d, reg, recon, fs, max_mb, st);
}

template <class T>
static void prime_typed(int riemann, size_t shmem0, size_t shmem1, size_t shmem2, cudaStream_t st) {
  if (riemann == RS_HLLD) {
    tma_ctas_per_sm<0, RS_HLLD, T>(shmem0, st);
    tma_ctas_per_sm<1, RS_HLLD, T>(shmem1, st);
    tma_ctas_per_sm<2, RS_HLLD, T>(shmem2, st);
  } else {
    tma_ctas_per_sm<0, RS_HLLE, T>(shmem0, st);
    tma_ctas_per_sm<1, RS_HLLE, T>(shmem1, st);
    tma_ctas_per_sm<2, RS_HLLE, T>(shmem2, st);
  }
}

void prime_flux_tma(const MeshView& v, int recon, int riemann, const FluxShape& fs, int max_mb, cudaStream_t st) {
  if (!flux_tma_applies(v, recon, fs, max_mb)) return;
  const int es = v.a.mixed ? 4 : 8;
  const size_t s0 = tma_smem(0, fs.plm_lines, max_mb, es), s1 = tma_smem(1, fs.plm_lines, max_mb, es),
               s2 = tma_smem(2, fs.plm_lines, max_mb, es);
  if (v.a.mixed)
    prime_typed<float>(riemann, s0, s1, s2, st);
  else
    prime_typed<double>(riemann, s0, s1, s2, st);
}

cudaError_t launch_flux(const MeshView& v, const Dispatch* d, int reg, int recon, int riemann, int dir,
                        const FluxShape& fs, int max_mb, cudaStream_t st) {
  if (dir == 0) return launch_dir<0>(v, d, reg, recon, riemann, fs, max_mb, st);
  if (dir == 1) return launch_dir<1>(v, d, reg, recon, riemann, fs, max_mb, st);
  return launch_dir<2>(v, d, reg, recon, riemann, fs, max_mb, st);
}

// The PLM kernels need more than the default 48 KB of dynamic shared memory; the attribute is set on the
// current device before any launch (and so before any stream capture).
cudaError_t prepare_kernel_attributes() {
  cudaError_t e = cudaSuccess;
#define VL2_ATTR(DIR, RS, T)                                                      \
  if (e == cudaSuccess) e = set_smem_attr(k_flux_tma<DIR, RS, T>);              \
  if (e == cudaSuccess) e = set_smem_attr(k_flux_plm<DIR, RS, T, REC_PLM>);     \
  if (e == cudaSuccess) e = set_smem_attr(k_flux_plm<DIR, RS, T, REC_PLM_CHAR>); \
  if (e == cudaSuccess) e = set_smem_attr(k_flux_plm<DIR, RS, T, REC_PPM_CHAR>); \
  if (e == cudaSuccess) e = set_smem_attr(k_flux_plm<DIR, RS, T, REC_PPM>);
  VL2_ATTR(0, RS_HLLD, double) VL2_ATTR(1, RS_HLLD, double) VL2_ATTR(2, RS_HLLD, double)
  VL2_ATTR(0, RS_HLLE, double) VL2_ATTR(1, RS_HLLE, double) VL2_ATTR(2, RS_HLLE, double)
  VL2_ATTR(0, RS_HLLD, float) VL2_ATTR(1, RS_HLLD, float) VL2_ATTR(2, RS_HLLD, float)
  VL2_ATTR(0, RS_HLLE, float) VL2_ATTR(1, RS_HLLE, float) VL2_ATTR(2, RS_HLLE, float)
#undef VL2_ATTR
  return e;
}

}  // namespace vl2
