// Face-flux kernels of the VL2 MHD step: reconstruction (donor cell or PLM with the van Leer limiter,
// Sec. 3.2.1) and the HLLD / HLLE Riemann fluxes (Sec. 3.2.2) on every face a MeshBlock needs.
#include "vl2_internal.h"
#include "vl2_physics.cuh"

namespace vl2 {

// One thread per face.  Faces of direction DIR cover the block's active faces along DIR (ng .. ng+mb)
// and the active cells plus one ghost layer transversally (ng-1 .. ng+mb), which feed the corner EMFs
// on the block surface.  W: [nblk][8][box] primitives incl. ghosts; Bn: face field of direction DIR.
template <int DIR, int REC, int RS, class T>
__global__ void __launch_bounds__(128) k_flux(Geom g, const T* __restrict__ W, const double* __restrict__ Bn,
                                              T* __restrict__ F) {
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
  const T* Wb = W + (long long)b * 8 * g.box;
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
  const T bn = (T)Bn[(long long)b * g.box + c];
  T f[7];
  if (RS == RS_HLLD)
    flux_hlld<T>(wl, wr, bn, (T)g.gamma, (T)g.igm1, f);
  else
    flux_hlle<T>(wl, wr, bn, (T)g.gamma, (T)g.igm1, f);
  T* Fb = F + (long long)b * 7 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = f[n];
}

// Corrector fluxes with each cell's PLM reconstruction formed once (Sec. 3.2.1).  A CTA takes P lines
// of faces along DIR: phase A reconstructs the mb+2 cells of each line (ng-1 .. ng+mb) into shared
// memory (face values q -+ delta/2 of 7 variables), phase B solves the mb+1 Riemann problems of each line
// from shared memory.  The 7 limiter denominators of a cell share one division (simultaneous inversion:
// reciprocals of a product and of its prefix products); a product outside the normal range falls back
// to one division per variable.
template <int DIR>
struct LineMap {
  // transverse directions ordered so that the fastest-varying memory index comes first
  static constexpr int TA = (DIR == 0) ? 1 : 0;
  static constexpr int TB = (DIR == 2) ? 1 : 2;
};

__device__ __forceinline__ bool normal_pos(double x) {
  const long long e = (__double_as_longlong(x) >> 52) & 0x7ff;
  return e != 0 && e != 0x7ff;
}

template <int DIR, int RS, class T>
__global__ void __launch_bounds__(256, 2) k_flux_plm(Geom g, const T* __restrict__ W,
                                                     const double* __restrict__ Bn, T* __restrict__ F, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
  constexpr int TA = LineMap<DIR>::TA, TB = LineMap<DIR>::TB;
  const int L = g.mb[DIR] + 2;   // reconstructed cells per line
  const int NF = g.mb[DIR] + 1;  // faces per line
  const int na = g.mb[TA] + 2, nb = g.mb[TB] + 2;
  const int nlines = na * nb;
  const int tiles = (nlines + P - 1) / P;
  const int b = blockIdx.x / tiles;
  const int tile = blockIdx.x - b * tiles;
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const long long sd = stride[DIR];
  const T* Wb = W + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  // shared layout: the fastest thread index is contiguous
  auto sidx = [&](int v, int side, int p, int c) -> int {
    return (DIR == 0) ? (((v * 2 + side) * P + p) * L + c) : (((v * 2 + side) * L + c) * P + p);
  };
  // phase A: reconstruct cells
  for (int t = threadIdx.x; t < P * L; t += blockDim.x) {
    const int p = (DIR == 0) ? t / L : t % P;
    const int c = (DIR == 0) ? t % L : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = NG - 1 + c;
    li[TA] = NG - 1 + line % na;
    li[TB] = NG - 1 + line / na;
    const long long o = cell_off(g, li[2], li[1], li[0]);
    T q0[7], dl[7], dr[7], den[7];
    bool pos[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const T* q = Wb + (long long)var[n] * g.box + o;
      const T qm = q[-sd], qc = q[0], qp = q[sd];
      q0[n] = qc;
      dl[n] = qc - qm;
      dr[n] = qp - qc;
      pos[n] = gt0(dl[n] * dr[n]);
      den[n] = pos[n] ? dl[n] + dr[n] : T(1);
    }
    T rec[7];
    if (sizeof(T) == 8) {
      T pre[7];
      pre[0] = den[0];
#pragma unroll
      for (int n = 1; n < 7; ++n) pre[n] = pre[n - 1] * den[n];
      if (normal_pos((double)fabs(pre[6]))) {
        T inv = T(1) / pre[6];
#pragma unroll
        for (int n = 6; n > 0; --n) {
          rec[n] = inv * pre[n - 1];
          inv = inv * den[n];
        }
        rec[0] = inv;
      } else {
#pragma unroll
        for (int n = 0; n < 7; ++n) rec[n] = T(1) / den[n];
      }
    } else {  // FP32: divisions are cheap, and a 7-fold product could leave the float range
#pragma unroll
      for (int n = 0; n < 7; ++n) rec[n] = T(1) / den[n];
    }
#pragma unroll
    for (int n = 0; n < 7; ++n) {
      const T delta = pos[n] ? (T(2) * (dl[n] * dr[n])) * rec[n] : T(0);
      smem[sidx(n, 0, p, c)] = q0[n] - T(0.5) * delta;  // value at the cell's lower face
      smem[sidx(n, 1, p, c)] = q0[n] + T(0.5) * delta;  // value at the cell's upper face
    }
  }
  __syncthreads();
  // phase B: Riemann problems of the faces ng .. ng+mb of every line
  for (int t = threadIdx.x; t < P * NF; t += blockDim.x) {
    const int p = (DIR == 0) ? t / NF : t % P;
    const int f = (DIR == 0) ? t % NF : t / P;
    const int line = tile * P + p;
    if (line >= nlines) continue;
    int li[3];
    li[DIR] = NG + f;
    li[TA] = NG - 1 + line % na;
    li[TB] = NG - 1 + line / na;
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
      flux_hlld<T>(wl, wr, bn, (T)g.gamma, (T)g.igm1, fl);
    else
      flux_hlle<T>(wl, wr, bn, (T)g.gamma, (T)g.igm1, fl);
    T* Fb = F + (long long)b * 7 * g.box + o;
#pragma unroll
    for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = fl[n];
  }
}

constexpr size_t PLM_SMEM_MAX = 64 * 1024;  // shared bytes per CTA (two CTAs per SM)

template <int DIR, int RS, class T>
static cudaError_t launch_plm(const Geom& g, const T* w, const double* bn, T* f, cudaStream_t st) {
  constexpr int TA = LineMap<DIR>::TA, TB = LineMap<DIR>::TB;
  const size_t per_line = (size_t)(g.mb[DIR] + 2) * 14 * sizeof(T);
  int P = (int)(PLM_SMEM_MAX / per_line);
  P = P < 1 ? 1 : (P > 16 ? 16 : P);
  const int nlines = (g.mb[TA] + 2) * (g.mb[TB] + 2);
  const int tiles = (nlines + P - 1) / P;
  const size_t shmem = (size_t)P * per_line;
  if (shmem > PLM_SMEM_MAX) return cudaErrorInvalidValue;  // a line longer than the shared budget
  cudaError_t e = cudaFuncSetAttribute(k_flux_plm<DIR, RS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PLM_SMEM_MAX);
  if (e != cudaSuccess) return e;
  k_flux_plm<DIR, RS, T><<<(unsigned)((long long)tiles * g.nblk), 256, shmem, st>>>(g, w, bn, f, P);
  return cudaGetLastError();
}

template <int DIR, int REC, int RS, class T>
static cudaError_t launch_one(const Geom& g, const T* w, const double* bn, T* f, cudaStream_t st) {
  const long long per = (long long)(g.mb[0] + (DIR == 0 ? 1 : 2)) * (g.mb[1] + (DIR == 1 ? 1 : 2)) *
                        (g.mb[2] + (DIR == 2 ? 1 : 2));
  const long long n = per * g.nblk;
  const int threads = 128;
  const long long blocks = (n + threads - 1) / threads;
  k_flux<DIR, REC, RS, T><<<(unsigned)blocks, threads, 0, st>>>(g, w, bn, f);
  return cudaGetLastError();
}

template <int DIR, int RS, class T>
static cudaError_t launch_typed(const Geom& g, const Arrays& a, int reg, int recon, cudaStream_t st) {
  const T* w = static_cast<const T*>(a.w);
  T* f = static_cast<T*>(a.f[DIR]);
  if (recon == REC_PLM) return launch_plm<DIR, RS, T>(g, w, a.b[reg][DIR], f, st);
  return launch_one<DIR, REC_DC, RS, T>(g, w, a.b[reg][DIR], f, st);
}

template <int DIR>
static cudaError_t launch_dir(const Geom& g, const Arrays& a, int reg, int recon, int riemann, cudaStream_t st) {
  if (a.mixed)
    return riemann == RS_HLLD ? launch_typed<DIR, RS_HLLD, float>(g, a, reg, recon, st)
                              : launch_typed<DIR, RS_HLLE, float>(g, a, reg, recon, st);
  return riemann == RS_HLLD ? launch_typed<DIR, RS_HLLD, double>(g, a, reg, recon, st)
                            : launch_typed<DIR, RS_HLLE, double>(g, a, reg, recon, st);
}

cudaError_t launch_flux(const Geom& g, const Arrays& a, int reg, int recon, int riemann, int dir, cudaStream_t st) {
  if (dir == 0) return launch_dir<0>(g, a, reg, recon, riemann, st);
  if (dir == 1) return launch_dir<1>(g, a, reg, recon, riemann, st);
  return launch_dir<2>(g, a, reg, recon, riemann, st);
}

}  // namespace vl2
