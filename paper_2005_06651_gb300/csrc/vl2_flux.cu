// Face-flux kernels of the VL2 MHD step: reconstruction (donor cell or PLM with the van Leer limiter,
// Sec. 3.2.1) and the HLLD / HLLE Riemann fluxes (Sec. 3.2.2) on every face a MeshBlock needs.
#include "vl2_internal.h"
#include "vl2_physics.cuh"

namespace vl2 {

// One thread per face.  Faces of direction DIR cover the block's active faces along DIR (ng .. ng+mb)
// and the active cells plus one ghost layer transversally (ng-1 .. ng+mb), which feed the corner EMFs
// on the block surface.  W: [nblk][8][box] primitives incl. ghosts; Bn: face field of direction DIR.
template <int DIR, int REC, int RS>
__global__ void __launch_bounds__(128) k_flux(Geom g, const double* __restrict__ W, const double* __restrict__ Bn,
                                              double* __restrict__ F) {
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
  const double* Wb = W + (long long)b * 8 * g.box;
  const int var[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4, 5 + T1, 5 + T2};
  double wl[7], wr[7];
#pragma unroll
  for (int n = 0; n < 7; ++n) {
    const double* q = Wb + (long long)var[n] * g.box + c;
    if (REC == REC_DC) {
      wl[n] = q[-sd];
      wr[n] = q[0];
    } else {
      const double qm2 = q[-2 * sd], qm1 = q[-sd], q0 = q[0], qp1 = q[sd];
      wl[n] = qm1 + 0.5 * vl_slope(qm2, qm1, q0);
      wr[n] = q0 - 0.5 * vl_slope(qm1, q0, qp1);
    }
  }
  const double bn = Bn[(long long)b * g.box + c];
  double f[7];
  if (RS == RS_HLLD)
    flux_hlld<double>(wl, wr, bn, g.gamma, g.igm1, f);
  else
    flux_hlle<double>(wl, wr, bn, g.gamma, g.igm1, f);
  double* Fb = F + (long long)b * 7 * g.box + c;
#pragma unroll
  for (int n = 0; n < 7; ++n) Fb[(long long)n * g.box] = f[n];
}

template <int DIR, int REC, int RS>
static cudaError_t launch_one(const Geom& g, const double* w, const double* bn, double* f, cudaStream_t st) {
  const long long per = (long long)(g.mb[0] + (DIR == 0 ? 1 : 2)) * (g.mb[1] + (DIR == 1 ? 1 : 2)) *
                        (g.mb[2] + (DIR == 2 ? 1 : 2));
  const long long n = per * g.nblk;
  const int threads = 128;
  const long long blocks = (n + threads - 1) / threads;
  k_flux<DIR, REC, RS><<<(unsigned)blocks, threads, 0, st>>>(g, w, bn, f);
  return cudaGetLastError();
}

template <int REC, int RS>
static cudaError_t launch_dir(const Geom& g, const Arrays& a, int reg, int dir, cudaStream_t st) {
  if (dir == 0) return launch_one<0, REC, RS>(g, a.w, a.b[reg][0], a.f[0], st);
  if (dir == 1) return launch_one<1, REC, RS>(g, a.w, a.b[reg][1], a.f[1], st);
  return launch_one<2, REC, RS>(g, a.w, a.b[reg][2], a.f[2], st);
}

cudaError_t launch_flux(const Geom& g, const Arrays& a, int reg, int recon, int riemann, int dir, cudaStream_t st) {
  if (recon == REC_DC)
    return riemann == RS_HLLD ? launch_dir<REC_DC, RS_HLLD>(g, a, reg, dir, st) : launch_dir<REC_DC, RS_HLLE>(g, a, reg, dir, st);
  return riemann == RS_HLLD ? launch_dir<REC_PLM, RS_HLLD>(g, a, reg, dir, st) : launch_dir<REC_PLM, RS_HLLE>(g, a, reg, dir, st);
}

}  // namespace vl2
