// Non-flux kernels of the VL2 MHD step: cons->prim with the fused CFL reduction, ghost exchange
// between MeshBlocks, upwind-CT corner EMFs, the register update, global-array I/O and the
// diagnostic reductions.
#include "vl2_internal.h"
#include "vl2_physics.cuh"

namespace vl2 {

static inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

__device__ __forceinline__ void block_loc(const Geom& g, int b, int* loc) {
  loc[0] = b % g.nb[0];
  loc[1] = (b / g.nb[0]) % g.nb[1];
  loc[2] = b / (g.nb[0] * g.nb[1]);
}

// ------------------------------------------------------------------------------------------------
// cons -> prim (Sec. 3.1): b_c = mean of the two face values, v = M / rho,
// p = (gamma-1)(E - |M|^2 / (2 rho) - |b_c|^2 / 2); floors rho >= dfloor, p >= pfloor (an active cell
// whose floor fires gets U rewritten and is counted).  With DT, the active cells also reduce the CFL
// rate max_d (|v_d| + C_f,d) / dx_d (Sec. 2.1.7) into scal[SC_MAXRATE] (bit pattern of a positive
// double, so an integer max is the floating max).
// ------------------------------------------------------------------------------------------------
template <class TW> __device__ __forceinline__ TW to_wtype(double x);
template <> __device__ __forceinline__ double to_wtype<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_wtype<float>(double x) { return to_f32(x); }

template <bool DT, class TW>
__global__ void __launch_bounds__(256) k_prim(MeshView single, const MeshView* views, const WorkItem* work, int reg,
                                              int all) {
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, views, work, tile);
  const Geom& g = V.g;
  const int off = all ? 0 : g.ng;
  const int ex = g.mb[0] + (all ? 2 * g.ng : 0), ey = g.mb[1] + (all ? 2 * g.ng : 0), ez = g.mb[2] + (all ? 2 * g.ng : 0);
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  // kept for the CFL rate: the cell's FP64 primitives and a single-precision estimate of its rate
#ifndef VL2_VALUE_SAFE
  constexpr bool LEAN = sizeof(TW) == 4;
#else
  constexpr bool LEAN = false;
#endif
  bool active = false;
  double id = 0.0, p = 0.0, vx = 0.0, vy = 0.0, vz = 0.0, bcx = 0.0, bcy = 0.0, bcz = 0.0;
  [[maybe_unused]] float s32v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float r32 = 0.0f;
  float s32[3] = {0.0f, 0.0f, 0.0f};  // the single-precision rate of each direction
  if (t < per * g.nblk) {
    const int b = (int)(t / per);
    int rem = (int)(t - (long long)b * per);
    const int i = rem % ex + off;
    rem /= ex;
    const int j = rem % ey + off;
    const int k = rem / ey + off;
    const long long c = cell_off(g, k, j, i);
    const long long fb = (long long)b * g.box + c;
    const double* B0 = V.a.b[reg][0];
    const double* B1 = V.a.b[reg][1];
    const double* B2 = V.a.b[reg][2];
    // LEAN (FP32 primitives): bc* hold the sums of the two face values (2 b_c) and v* the momenta; the
    // halvings and the FP64 products M / rho are taken only where an FP64 result needs them (the CFL
    // candidates), the stored FP32 velocity being the FP32 product of M and 1/rho
    bcx = LEAN ? B0[fb] + B0[fb + 1] : 0.5 * (B0[fb] + B0[fb + 1]);
    bcy = LEAN ? B1[fb] + B1[fb + g.sx] : 0.5 * (B1[fb] + B1[fb + g.sx]);
    bcz = LEAN ? B2[fb] + B2[fb + (long long)g.sx * g.sy] : 0.5 * (B2[fb] + B2[fb + (long long)g.sx * g.sy]);
    double* Ub = V.a.u[reg] + (long long)b * 5 * g.box + c;
    double d = Ub[0];
    const double m1 = Ub[g.box], m2 = Ub[2 * g.box], m3 = Ub[3 * g.box];
    double e = Ub[4 * g.box];
    active = i >= g.ng && i < g.ng + g.mb[0] && j >= g.ng && j < g.ng + g.mb[1] && k >= g.ng && k < g.ng + g.mb[2];
    bool fired = false;
    if (d < g.dfloor) {
      d = g.dfloor;
      fired = true;
    }
    id = rcp_nr(d);  // d >= dfloor, a positive normal number
    vx = LEAN ? m1 : m1 * id;
    vy = LEAN ? m2 : m2 * id;
    vz = LEAN ? m3 : m3 * id;
    const double ke = 0.5 * ((m1 * m1 + m2 * m2) + m3 * m3) * id;
    // (2 b)^2 / 8 is b^2 / 2 exactly (powers of two), so both forms give the same bits
    const double me = (LEAN ? 0.125 : 0.5) * ((bcx * bcx + bcy * bcy) + bcz * bcz);
    p = g.gm1 * (e - ke - me);
    if (p < g.pfloor) {
      p = g.pfloor;
      e = p * g.igm1 + ke + me;
      fired = true;
    }
    if (fired && active) {
      atomicAdd(V.a.scal + SC_FLOORS, 1ULL);
      Ub[0] = d;
      Ub[4 * g.box] = e;
    }
    if (g.ns) {
      // concentrations C = (rho C) / rho: the reciprocal's quotient with one correction step (exactly 1
      // for C = 1, so that a unit scalar is carried exactly like the density)
      const double* Sb = V.a.s[reg] + (long long)b * g.ns * g.box + c;
      double* Cb = V.a.cs + (long long)b * g.ns * g.box + c;
      for (int q = 0; q < g.ns; ++q) {
        const double sq = Sb[(long long)q * g.box];
#ifndef VL2_VALUE_SAFE
        const double c0 = sq * id;
        Cb[(long long)q * g.box] = fma(fma(-d, c0, sq), id, c0);
#else
        Cb[(long long)q * g.box] = sq / d;
#endif
      }
    }
    TW* Wb = static_cast<TW*>(V.a.w) + (long long)b * 8 * g.box + c;
    TW wx, wy, wz, ux, uy, uz;
    if constexpr (LEAN) {
      const float fid = to_f32(id);
      wx = to_f32(vx) * fid;
      wy = to_f32(vy) * fid;
      wz = to_f32(vz) * fid;
      ux = 0.5f * to_f32(bcx);
      uy = 0.5f * to_f32(bcy);
      uz = 0.5f * to_f32(bcz);
    } else {
      wx = to_wtype<TW>(vx), wy = to_wtype<TW>(vy), wz = to_wtype<TW>(vz);
      ux = to_wtype<TW>(bcx), uy = to_wtype<TW>(bcy), uz = to_wtype<TW>(bcz);
    }
    if constexpr (LEAN) {  // the FP32 screen below reads the FP32 primitives
      s32v[0] = (float)wx;
      s32v[1] = (float)wy;
      s32v[2] = (float)wz;
      s32v[3] = (float)ux;
      s32v[4] = (float)uy;
      s32v[5] = (float)uz;
    }
    Wb[0] = to_wtype<TW>(d);
    Wb[g.box] = wx;
    Wb[2 * g.box] = wy;
    Wb[3 * g.box] = wz;
    Wb[4 * g.box] = to_wtype<TW>(p);
    Wb[5 * g.box] = ux;
    Wb[6 * g.box] = uy;
    Wb[7 * g.box] = uz;
    // cell EMFs -(v x b_c) of the stored primitives, for the CT corners (each is used by four corners of
    // its family): computed in the stage's precision, as the corners' face EMFs are
    TW* Eb = static_cast<TW*>(V.a.ec) + (long long)b * 3 * g.box + c;
    Eb[0] = wz * uy - wy * uz;
    Eb[g.box] = wx * uz - wz * ux;
    Eb[2 * g.box] = wy * ux - wx * uy;
    if (DT && active) {
      // single-precision estimate of the rate (relative error well below 1e-5)
      const float fid = to_f32(id), fp = to_f32(p), fg = g.gamma_f;
      const float fx = LEAN ? s32v[3] : to_f32(bcx), fy = LEAN ? s32v[4] : to_f32(bcy), fz = LEAN ? s32v[5] : to_f32(bcz);
      const float ax = LEAN ? s32v[0] : to_f32(vx), ay = LEAN ? s32v[1] : to_f32(vy), az = LEAN ? s32v[2] : to_f32(vz);
      const float x2 = fx * fx, y2 = fy * fy, z2 = fz * fz;
      const float sx = (fabsf(ax) + fast_speed_r(fid, fp, x2, y2 + z2, fg)) * g.idx_f[0];
      const float sy = (fabsf(ay) + fast_speed_r(fid, fp, y2, z2 + x2, fg)) * g.idx_f[1];
      const float sz = (fabsf(az) + fast_speed_r(fid, fp, z2, x2 + y2, fg)) * g.idx_f[2];
      s32[0] = sx;
      s32[1] = sy;
      s32[2] = sz;
      r32 = fmaxf(fmaxf(sx, sy), sz);
      if (sx != sx || sy != sy || sz != sz) r32 = __int_as_float(0x7fc00000);  // keep a NaN visible
    }
  }
  if (DT) {
    // The CFL rate max_d (|v_d| + C_f,d) / dx_d of the CTA's cells, in FP64.  Only (cell, direction) pairs
    // whose single-precision rate is within 1e-4 of the CTA's single-precision maximum can hold the FP64
    // maximum, so only they are evaluated in FP64 (every direction of a cell whose estimate is not a number,
    // and everything when the estimate overflowed); the result equals the FP64 maximum over all cells.
    // The rate is a function of (1/rho, p, v, b_c) alone: candidates of a warp whose eight inputs are
    // bitwise equal (a region at rest makes whole warps of them) keep one representative, and the
    // representatives of the CTA are gathered into shared memory and evaluated by its first threads, so
    // the FP64 work runs in as few warps as there are distinct candidates.
    __shared__ float redf[8];
    __shared__ unsigned long long red[8];
    __shared__ double cin[8][THREADS];
    __shared__ unsigned char cdir[THREADS];  // the candidate's directions to evaluate (bits 0, 1, 2)
    __shared__ int ncand;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float m32 = r32;
    for (int o = 16; o > 0; o >>= 1) m32 = fmaxf(m32, __shfl_xor_sync(0xffffffffu, m32, o));
    if (lane == 0) redf[wid] = m32;
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    m32 = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m32 = fmaxf(m32, redf[q]);
    const float thr = m32 * 0.9999f;
    int dirs = 0;
    if (active) {
      if (isnan(r32) || isinf(m32))  // an unreliable estimate (an overflowed one: every cell)
        dirs = 7;
      else
        dirs = (!(s32[0] < thr) ? 1 : 0) | (!(s32[1] < thr) ? 2 : 0) | (!(s32[2] < thr) ? 4 : 0);
    }
    const bool cand = dirs != 0;  // the cell's rate max_d s_d reaches the threshold
    const unsigned cmask = __ballot_sync(0xffffffffu, cand);
    bool lead = false;
    if (cand) {
      unsigned grp = __match_any_sync(cmask, __double_as_longlong(id));
      grp &= __match_any_sync(cmask, __double_as_longlong(p));
      grp &= __match_any_sync(cmask, __double_as_longlong(vx));
      grp &= __match_any_sync(cmask, __double_as_longlong(vy));
      grp &= __match_any_sync(cmask, __double_as_longlong(vz));
      grp &= __match_any_sync(cmask, __double_as_longlong(bcx));
      grp &= __match_any_sync(cmask, __double_as_longlong(bcy));
      grp &= __match_any_sync(cmask, __double_as_longlong(bcz));
      lead = (grp & ((1u << lane) - 1u)) == 0u;  // the lowest lane of its group
    }
    const unsigned lmask = __ballot_sync(0xffffffffu, lead);
    int base = 0;
    if (lane == 0 && lmask) base = atomicAdd(&ncand, __popc(lmask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lead) {
      const int slot = base + __popc(lmask & ((1u << lane) - 1u));  // < blockDim.x: one slot per thread at most
      cin[0][slot] = id;
      cin[1][slot] = p;
      cin[2][slot] = LEAN ? vx * id : vx;  // the FP64 velocity and cell field, as in the FP64 form
      cin[3][slot] = LEAN ? vy * id : vy;
      cin[4][slot] = LEAN ? vz * id : vz;
      cin[5][slot] = LEAN ? 0.5 * bcx : bcx;
      cin[6][slot] = LEAN ? 0.5 * bcy : bcy;
      cin[7][slot] = LEAN ? 0.5 * bcz : bcz;
      cdir[slot] = (unsigned char)dirs;  // equal inputs give equal estimates, so the group shares it
    }
    __syncthreads();
    const int nc = ncand;  // CTA-uniform
    if (nc <= 32 && wid > 0) return;  // the first warp evaluates every candidate and reduces alone
    unsigned long long rate_bits = 0ULL;
    if ((int)threadIdx.x < nc) {
      const int q = threadIdx.x;
      const double cid = cin[0][q], cp = cin[1][q];
      const double bx2 = cin[5][q] * cin[5][q], by2 = cin[6][q] * cin[6][q], bz2 = cin[7][q] * cin[7][q];
      const int dq = cdir[q];
      unsigned long long ax = 0ULL, ay = 0ULL, az = 0ULL;  // a direction left out cannot hold the maximum
      if (dq & 1)
        ax = __double_as_longlong((fabs(cin[2][q]) + fast_speed_r(cid, cp, bx2, by2 + bz2, g.gamma)) * g.idx[0]);
      if (dq & 2)
        ay = __double_as_longlong((fabs(cin[3][q]) + fast_speed_r(cid, cp, by2, bz2 + bx2, g.gamma)) * g.idx[1]);
      if (dq & 4)
        az = __double_as_longlong((fabs(cin[4][q]) + fast_speed_r(cid, cp, bz2, bx2 + by2, g.gamma)) * g.idx[2]);
      rate_bits = ax > ay ? ax : ay;
      rate_bits = rate_bits > az ? rate_bits : az;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, rate_bits, o);
      rate_bits = v > rate_bits ? v : rate_bits;
    }
    if (nc <= 32) {
      if (lane == 0 && rate_bits) atomicMax(V.a.scal + SC_MAXRATE, rate_bits);
      return;
    }
    if (lane == 0) red[wid] = rate_bits;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0ULL;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = red[q] > m ? red[q] : m;
      if (m) atomicMax(V.a.scal + SC_MAXRATE, m);
    }
  }
}

long long tiles_prim(const Geom& g) {
  return ((long long)(g.mb[0] + 2 * g.ng) * (g.mb[1] + 2 * g.ng) * (g.mb[2] + 2 * g.ng) * g.nblk + THREADS - 1) / THREADS;
}

cudaError_t launch_prim(const MeshView& v, const Dispatch* d, int reg, bool all_cells, bool want_dt, cudaStream_t st) {
  const Geom& g = v.g;
  long long grid;
  if (d)
    grid = d->nwork;  // batched launches always cover every cell
  else if (all_cells)
    grid = tiles_prim(g);
  else
    grid = ((long long)g.mb[0] * g.mb[1] * g.mb[2] * g.nblk + THREADS - 1) / THREADS;
  if (grid <= 0) return cudaSuccess;
  const MeshView* vs = d ? d->views : nullptr;
  const WorkItem* wk = d ? d->work : nullptr;
  const int all = (d || all_cells) ? 1 : 0;
  if (v.a.mixed) {
    if (want_dt)
      k_prim<true, float><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, reg, all);
    else
      k_prim<false, float><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, reg, all);
  } else {
    if (want_dt)
      k_prim<true, double><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, reg, all);
    else
      k_prim<false, double><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, reg, all);
  }
  return cudaGetLastError();
}

// per-box time step from the CFL rate each box's last prim pass reduced; the rate is reset for the next pass
__global__ void k_batch_dt(const MeshView* views, int nbox, const double* cfl, double* dt) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nbox) return;
  unsigned long long* rp = views[q].a.scal + SC_MAXRATE;
  if (cfl) {
    const double rate = __longlong_as_double((long long)*rp);
    dt[q] = cfl[q] / rate;
  }
  *rp = 0ULL;
}

// dt = cfl / (the mesh's reduced CFL rate), on the device (one mesh; the rate slot is left for the caller)
__global__ void k_mesh_dt(const unsigned long long* scal, double cfl, double* dt) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *dt = cfl / __longlong_as_double((long long)scal[SC_MAXRATE]);
}

cudaError_t launch_mesh_dt(const unsigned long long* scal, double cfl, double* dt, cudaStream_t st) {
  k_mesh_dt<<<1, 32, 0, st>>>(scal, cfl, dt);
  return cudaGetLastError();
}

cudaError_t launch_batch_dt(const MeshView* views, int nbox, const double* cfl, double* dt, cudaStream_t st) {
  k_batch_dt<<<(nbox + 127) / 128, 128, 0, st>>>(views, nbox, cfl, dt);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Ghost exchange (Sec. 2.1.1): every ghost cell and ghost face of every block is copied from the block
// that owns the (periodically wrapped, or outflow-clamped) global index.  Faces on a block's surface
// are active and not overwritten.  A face on the boundary between two blocks is read from the block
// where it is the lower face; global face N from the last block's upper face.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void source_of(const Geom& g, int q, int gi, bool face, int& blk, int& loc) {
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
    loc = g.mb[q] + g.ng;
  } else {
    blk = m / g.mb[q];
    loc = m - blk * g.mb[q] + g.ng;
  }
}

// Ghost elements lie in the shell of the padded box: index triples 0 .. mb+2ng (one more than the cells,
// for the faces) with at least one coordinate outside the interior ng .. ng+mb-1.  A thread per shell
// element; the shell is decoded as z-slabs (k outside the interior), then y-slabs (k inside, j outside),
// then x-slabs (k, j inside, i outside).
__device__ __forceinline__ long long shell_size(const Geom& g) {
  const long long ex = g.mb[0] + 2 * g.ng + 1, ey = g.mb[1] + 2 * g.ng + 1, ez = g.mb[2] + 2 * g.ng + 1;
  return ex * ey * ez - (long long)g.mb[0] * g.mb[1] * g.mb[2];
}
__device__ __forceinline__ void shell_index(const Geom& g, int s, int* li) {
  const int ex = g.mb[0] + 2 * g.ng + 1, ey = g.mb[1] + 2 * g.ng + 1, ez = g.mb[2] + 2 * g.ng + 1;
  const int gx = ex - g.mb[0], gy = ey - g.mb[1], gz = ez - g.mb[2];  // ghost layers per direction
  auto unfold = [&](int gidx, int q) { return gidx < g.ng ? gidx : gidx + g.mb[q]; };
  const int nz = gz * ey * ex;
  if (s < nz) {
    li[2] = unfold(s / (ey * ex), 2);
    const int r = s % (ey * ex);
    li[1] = r / ex;
    li[0] = r % ex;
    return;
  }
  s -= nz;
  const int ny = g.mb[2] * gy * ex;
  if (s < ny) {
    li[2] = s / (gy * ex) + g.ng;
    const int r = s % (gy * ex);
    li[1] = unfold(r / ex, 1);
    li[0] = r % ex;
    return;
  }
  s -= ny;
  li[2] = s / (g.mb[1] * gx) + g.ng;
  const int r = s % (g.mb[1] * gx);
  li[1] = r / gx + g.ng;
  li[0] = unfold(r % gx, 0);
}

__global__ void __launch_bounds__(256) k_ghosts(MeshView single, const MeshView* views, const WorkItem* work, int reg) {
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, views, work, tile);
  const Geom& g = V.g;
  double* U = V.a.u[reg];
  double* B0 = V.a.b[reg][0];
  double* B1 = V.a.b[reg][1];
  double* B2 = V.a.b[reg][2];
  const long long per = shell_size(g);
  int b, e;
  if (work || gridDim.y == 1) {  // a flat index over (block, shell element)
    const long long t = (long long)tile * blockDim.x + threadIdx.x;
    if (t >= per * g.nblk) return;
    b = (int)(t / per);
    e = (int)(t - (long long)b * per);
  } else {  // one grid row per block: no 64-bit division
    b = (int)blockIdx.y;
    e = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= per) return;
  }
  int li[3];
  shell_index(g, e, li);
  int loc[3];
  block_loc(g, b, loc);
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const int cmax[3] = {g.mb[0] + 2 * g.ng, g.mb[1] + 2 * g.ng, g.mb[2] + 2 * g.ng};
  // source block and index of each coordinate as a cell index (faces re-map their own direction)
  int sb[3], sl[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) source_of(g, q, loc[q] * g.mb[q] + li[q] - g.ng, false, sb[q], sl[q]);
  // Every source is an active cell or face of its block, which no thread of this launch writes, so all of a
  // thread's loads are issued before its stores (one memory round trip instead of one per copied value).
  bool cell = false;
  int ublk = 0;
  long long ucell = 0, usrc = 0;
  if (li[0] < cmax[0] && li[1] < cmax[1] && li[2] < cmax[2]) {
    for (int q = 0; q < 3; ++q) cell |= (li[q] < g.ng || li[q] >= g.ng + g.mb[q]);
    if (cell) {
      ublk = (sb[2] * g.nb[1] + sb[1]) * g.nb[0] + sb[0];
      ucell = cell_off(g, sl[2], sl[1], sl[0]);
      usrc = (long long)ublk * 5 * g.box + ucell;
    }
  }
  double* Bf[3] = {B0, B1, B2};
  bool face[3];
  long long fsrc[3];
#pragma unroll
  for (int fd = 0; fd < 3; ++fd) {
    bool valid = true, ghost = false;
    for (int q = 0; q < 3; ++q) {
      const int hi_valid = (q == fd) ? cmax[q] : cmax[q] - 1;
      const int hi_active = (q == fd) ? g.ng + g.mb[q] : g.ng + g.mb[q] - 1;
      valid &= li[q] <= hi_valid;
      ghost |= (li[q] < g.ng || li[q] > hi_active);
    }
    face[fd] = valid && ghost;
    fsrc[fd] = 0;
    if (face[fd]) {
      int fb[3] = {sb[0], sb[1], sb[2]}, fl[3] = {sl[0], sl[1], sl[2]};
      source_of(g, fd, loc[fd] * g.mb[fd] + li[fd] - g.ng, true, fb[fd], fl[fd]);
      fsrc[fd] = (long long)((fb[2] * g.nb[1] + fb[1]) * g.nb[0] + fb[0]) * g.box + cell_off(g, fl[2], fl[1], fl[0]);
    }
  }
  double uv[5], fv[3];
  if (cell) {
#pragma unroll
    for (int v = 0; v < 5; ++v) uv[v] = U[usrc + (long long)v * g.box];
  }
#pragma unroll
  for (int fd = 0; fd < 3; ++fd)
    if (face[fd]) fv[fd] = Bf[fd][fsrc[fd]];
  // cell-centred conserved variables
  if (cell) {
    double* Ud = U + (long long)b * 5 * g.box + c;
#pragma unroll
    for (int v = 0; v < 5; ++v) Ud[(long long)v * g.box] = uv[v];
    if (g.ns) {  // passive scalars ride with the conserved variables
      const double* Ss = V.a.s[reg] + (long long)ublk * g.ns * g.box + ucell;
      double* Sd = V.a.s[reg] + (long long)b * g.ns * g.box + c;
      for (int q = 0; q < g.ns; ++q) Sd[(long long)q * g.box] = Ss[(long long)q * g.box];
    }
  }
  // face-centred field
#pragma unroll
  for (int fd = 0; fd < 3; ++fd)
    if (face[fd]) Bf[fd][(long long)b * g.box + c] = fv[fd];
}

long long tiles_ghosts(const Geom& g) {
  const long long per = (long long)(g.mb[0] + 2 * g.ng + 1) * (g.mb[1] + 2 * g.ng + 1) * (g.mb[2] + 2 * g.ng + 1) -
                        (long long)g.mb[0] * g.mb[1] * g.mb[2];
  return (per * g.nblk + THREADS - 1) / THREADS;
}

cudaError_t launch_ghosts(const MeshView& v, const Dispatch* d, int reg, cudaStream_t st) {
  const Geom& g = v.g;
  if (!d && g.nblk > 1 && g.nblk <= 65535) {  // one grid row per MeshBlock
    const long long per = (long long)(g.mb[0] + 2 * g.ng + 1) * (g.mb[1] + 2 * g.ng + 1) * (g.mb[2] + 2 * g.ng + 1) -
                          (long long)g.mb[0] * g.mb[1] * g.mb[2];
    const dim3 grid((unsigned)((per + THREADS - 1) / THREADS), (unsigned)g.nblk);
    k_ghosts<<<grid, THREADS, 0, st>>>(v, nullptr, nullptr, reg);
    return cudaGetLastError();
  }
  const long long grid = d ? d->nwork : tiles_ghosts(g);
  if (grid <= 0) return cudaSuccess;
  k_ghosts<<<(unsigned)grid, THREADS, 0, st>>>(v, d ? d->views : nullptr, d ? d->work : nullptr, reg);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Passive scalars (eq. passive_scalars): d(rho C)/dt + div(rho v C) = 0.  C is reconstructed along the sweep
// with the stage's reconstruction (donor cell, PLM or PPM, as for the primitives) and carried by the
// Riemann mass flux from the upwind side: F = F_rho C_L if F_rho >= 0, else F_rho C_R.  One thread per face of
// the block's active cells (the scalars feed no corner EMF).
// ------------------------------------------------------------------------------------------------
template <int DIR, int REC, class TF>
__global__ void __launch_bounds__(256) k_scalar_flux(MeshView V) {
  const Geom& g = V.g;
  const int rx = g.mb[0] + (DIR == 0), ry = g.mb[1] + (DIR == 1), rz = g.mb[2] + (DIR == 2);
  const long long per = (long long)rx * ry * rz;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % rx + g.ng;
  rem /= rx;
  const int j = rem % ry + g.ng;
  const int k = rem / ry + g.ng;
  const long long c = cell_off(g, k, j, i);
  const long long sd = (DIR == 0) ? 1LL : ((DIR == 1) ? (long long)g.sx : (long long)g.sx * g.sy);
  const double m = to_f64(static_cast<const TF*>(V.a.f[DIR])[(long long)b * 7 * g.box + c]);
  const bool up = ge0(m);
  for (int q = 0; q < g.ns; ++q) {
    const long long o = ((long long)b * g.ns + q) * g.box + c;
    const double* C = V.a.cs + o;
    double cl, cr;
    if (REC == REC_DC) {
      cl = C[-sd];
      cr = C[0];
    } else if (REC == REC_PPM) {
      double e0, e1;
      ppm_edges(C[-3 * sd], C[-2 * sd], C[-sd], C[0], C[sd], e0, e1);
      cl = e1;
      ppm_edges(C[-2 * sd], C[-sd], C[0], C[sd], C[2 * sd], e0, e1);
      cr = e0;
    } else {
      cl = C[-sd] + 0.5 * vl_slope(C[-2 * sd], C[-sd], C[0]);
      cr = C[0] - 0.5 * vl_slope(C[-sd], C[0], C[sd]);
    }
    V.a.fsc[DIR][o] = up ? m * cl : m * cr;
  }
}

template <int DIR, class TF>
static cudaError_t launch_scalar_dir(const MeshView& v, int recon, cudaStream_t st) {
  const Geom& g = v.g;
  const long long n = (long long)g.nblk * (g.mb[0] + (DIR == 0)) * (g.mb[1] + (DIR == 1)) * (g.mb[2] + (DIR == 2));
  const unsigned grid = (unsigned)((n + THREADS - 1) / THREADS);
  if (n <= 0) return cudaSuccess;
  if (recon == REC_DC)
    k_scalar_flux<DIR, REC_DC, TF><<<grid, THREADS, 0, st>>>(v);
  else if (recon == REC_PPM || recon == REC_PPM_CHAR)
    k_scalar_flux<DIR, REC_PPM, TF><<<grid, THREADS, 0, st>>>(v);
  else
    k_scalar_flux<DIR, REC_PLM, TF><<<grid, THREADS, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_scalar_fluxes(const MeshView& v, int recon, int dir, cudaStream_t st) {
  if (v.a.mixed) {
    if (dir == 0) return launch_scalar_dir<0, float>(v, recon, st);
    if (dir == 1) return launch_scalar_dir<1, float>(v, recon, st);
    return launch_scalar_dir<2, float>(v, recon, st);
  }
  if (dir == 0) return launch_scalar_dir<0, double>(v, recon, st);
  if (dir == 1) return launch_scalar_dir<1, double>(v, recon, st);
  return launch_scalar_dir<2, double>(v, recon, st);
}

// The L form of the register update with its roundings written out (fused multiply-adds in the fast build,
// separate products and sums in the value-safe build, which contracts nothing), so that every kernel that
// applies it (the one-node and two-node updates, the scalar update) gives the same bits:
//   div = ((dF_x/dx + dF_y/dy) + dF_z/dz),  out = base + h L,  base = g_base U_base + g_other U_other.
__device__ __forceinline__ double div3(const double* df, const double* idx) {
#ifndef VL2_VALUE_SAFE
  return fma(df[2], idx[2], fma(df[1], idx[1], df[0] * idx[0]));
#else
  return (df[0] * idx[0] + df[1] * idx[1]) + df[2] * idx[2];
#endif
}
__device__ __forceinline__ double stage_base(bool plain, double ub, double uo, double g_base, double g_other) {
#ifndef VL2_VALUE_SAFE
  return plain ? ub : fma(g_other, uo, g_base * ub);
#else
  return plain ? ub : g_base * ub + g_other * uo;
#endif
}
__device__ __forceinline__ double plus_hl(double base, double h, double L) {
#ifndef VL2_VALUE_SAFE
  return fma(h, L, base);
#else
  return base + h * L;
#endif
}
// (dE_b / dx_a - dE_a / dx_b) of a face field's CT curl
__device__ __forceinline__ double curl2(double deb, double ia, double dea, double ib) {
#ifndef VL2_VALUE_SAFE
  return fma(deb, ia, -(dea * ib));
#else
  return deb * ia - dea * ib;
#endif
}

// Register update of the scalar masses, written as the FP64 conserved variables' update in k_update (same
// association, same weights), so that a unit scalar stays bitwise equal to the density.
template <bool PLAIN>
__global__ void __launch_bounds__(256) k_scalar_update(MeshView V, int base_reg, int out_reg, double h, double g_base,
                                                       double g_other) {
  const Geom& g = V.g;
  const long long per = (long long)g.mb[0] * g.mb[1] * g.mb[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % g.mb[0] + g.ng;
  rem /= g.mb[0];
  const int j = rem % g.mb[1] + g.ng;
  const int k = rem / g.mb[1] + g.ng;
  const long long c = cell_off(g, k, j, i);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const double* Sbase = V.a.s[base_reg];
  const double* Soth = V.a.s[1 - base_reg];
  double* Sout = V.a.s[out_reg];
  for (int q = 0; q < g.ns; ++q) {
    const long long o = ((long long)b * g.ns + q) * g.box + c;
    double df[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) df[d] = V.a.fsc[d][o + stride[d]] - V.a.fsc[d][o];
    const double L = -div3(df, g.idx);
    Sout[o] = plus_hl(stage_base(PLAIN, Sbase[o], PLAIN ? 0.0 : Soth[o], g_base, g_other), h, L);
  }
}

cudaError_t launch_scalar_update(const MeshView& v, int base_reg, int out_reg, double h, double g_base,
                                 double g_other, cudaStream_t st) {
  const Geom& g = v.g;
  const long long n = (long long)g.nblk * g.mb[0] * g.mb[1] * g.mb[2];
  const unsigned grid = (unsigned)((n + THREADS - 1) / THREADS);
  if (n <= 0 || g.ns == 0) return cudaSuccess;
  if (g_base == 1.0 && g_other == 0.0)
    k_scalar_update<true><<<grid, THREADS, 0, st>>>(v, base_reg, out_reg, h, g_base, g_other);
  else
    k_scalar_update<false><<<grid, THREADS, 0, st>>>(v, base_reg, out_reg, h, g_base, g_other);
  return cudaGetLastError();
}

// Global-array I/O of the scalars: rho C = rho c on the active cells of register 0 (from concentrations
// c[q][NZ][NY][NX]), and the masses out[q][NZ][NY][NX].
__global__ void k_scalars_io(Geom g, Arrays a, const double* c, double* out) {
  const long long per = (long long)g.mb[0] * g.mb[1] * g.mb[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % g.mb[0];
  rem /= g.mb[0];
  const int j = rem % g.mb[1];
  const int k = rem / g.mb[1];
  int loc[3];
  block_loc(g, b, loc);
  const long long gi = ((long long)(loc[2] * g.mb[2] + k) * g.N[1] + (loc[1] * g.mb[1] + j)) * g.N[0] +
                       (loc[0] * g.mb[0] + i);
  const long long nc = (long long)g.N[0] * g.N[1] * g.N[2];
  const long long cc = cell_off(g, k + g.ng, j + g.ng, i + g.ng);
  const double rho = a.u[0][(long long)b * 5 * g.box + cc];
  for (int q = 0; q < g.ns; ++q) {
    const long long o = ((long long)b * g.ns + q) * g.box + cc;
    if (c)
      a.s[0][o] = rho * c[q * nc + gi];
    else
      out[q * nc + gi] = a.s[0][o];
  }
}

// forcing acceleration a[3][NZ][NY][NX] (global cell layout) into acc[nblk][3][box] at the active cells
__global__ void __launch_bounds__(256) k_scatter_forcing(Geom g, double* acc, const double* __restrict__ a) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)g.mb[0] * g.mb[1] * g.mb[2];
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % g.mb[0];
  rem /= g.mb[0];
  const int j = rem % g.mb[1];
  const int k = rem / g.mb[1];
  int loc[3];
  block_loc(g, b, loc);
  const long long gi = ((long long)(loc[2] * g.mb[2] + k) * g.N[1] + (loc[1] * g.mb[1] + j)) * g.N[0] +
                       (loc[0] * g.mb[0] + i);
  const long long nc = (long long)g.N[0] * g.N[1] * g.N[2];
  const long long cc = cell_off(g, k + g.ng, j + g.ng, i + g.ng);
  for (int d = 0; d < 3; ++d) acc[((long long)b * 3 + d) * g.box + cc] = a[d * nc + gi];
}

cudaError_t launch_scatter_forcing(const Geom& g, double* acc, const double* a, cudaStream_t st) {
  const long long n = (long long)g.nblk * g.mb[0] * g.mb[1] * g.mb[2];
  k_scatter_forcing<<<(unsigned)((n + THREADS - 1) / THREADS), THREADS, 0, st>>>(g, acc, a);
  return cudaGetLastError();
}

cudaError_t launch_scatter_scalars(const Geom& g, const Arrays& a, const double* c, cudaStream_t st) {
  const long long n = (long long)g.nblk * g.mb[0] * g.mb[1] * g.mb[2];
  k_scalars_io<<<(unsigned)((n + THREADS - 1) / THREADS), THREADS, 0, st>>>(g, a, c, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gather_scalars(const Geom& g, const Arrays& a, double* out, cudaStream_t st) {
  const long long n = (long long)g.nblk * g.mb[0] * g.mb[1] * g.mb[2];
  k_scalars_io<<<(unsigned)((n + THREADS - 1) / THREADS), THREADS, 0, st>>>(g, a, nullptr, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Upwind CT corner EMFs (Sec. 3.1 / Sec. 2.1.1).  Edge family e (E1 along x, E2 along y, E3 along z),
// transverse directions a = e+1, b = e+2.  Face EMFs of that component: -F_a[B_t1] on a-faces and
// +F_b[B_t2] on b-faces (E = -v x B); cell EMFs as cons->prim wrote them.  One thread per corner node.
// ------------------------------------------------------------------------------------------------
template <class T, bool SMOOTH>
__global__ void __launch_bounds__(256) k_emf(MeshView single, const MeshView* views, const WorkItem* work) {
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, views, work, tile);
  const Geom& g = V.g;
  const T* F0 = static_cast<const T*>(V.a.f[0]);
  const T* F1 = static_cast<const T*>(V.a.f[1]);
  const T* F2 = static_cast<const T*>(V.a.f[2]);
  T* E0 = static_cast<T*>(V.a.e[0]);
  T* E1 = static_cast<T*>(V.a.e[1]);
  T* E2 = static_cast<T*>(V.a.e[2]);
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex + g.ng, (rem / ex) % ey + g.ng, rem / (ex * ey) + g.ng};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const T* F[3] = {F0, F1, F2};
  T* E[3] = {E0, E1, E2};
  const T* Ecb = static_cast<const T*>(V.a.ec) + (long long)b * 3 * g.box;
  // smoothed weights: the node's own three faces serve two edge families each, so 9 weights per node, not 12
  [[maybe_unused]] const T delta = (T)g.ct_delta, band = T(20) * delta;
  [[maybe_unused]] T wown[3];
  if constexpr (SMOOTH) {
#pragma unroll
    for (int d = 0; d < 3; ++d) wown[d] = ct_weight(F[d][(long long)b * 7 * g.box + c], delta, band);
  }
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (li[e] > g.ng + g.mb[e] - 1) continue;
    const int a = (e + 1) % 3, bq = (e + 2) % 3;
    const long long sa = stride[a], sb = stride[bq];
    const T* Fa = F[a] + (long long)b * 7 * g.box;
    const T* Fb = F[bq] + (long long)b * 7 * g.box;
    T ea[2], eb[2], ec[4], ma[2], mb[2];
    ea[0] = -Fa[5 * g.box + c - sb];
    ea[1] = -Fa[5 * g.box + c];
    eb[0] = Fb[6 * g.box + c - sa];
    eb[1] = Fb[6 * g.box + c];
    if constexpr (SMOOTH) {
      ma[0] = ct_weight(Fa[c - sb], delta, band);
      ma[1] = wown[a];
      mb[0] = ct_weight(Fb[c - sa], delta, band);
      mb[1] = wown[bq];
    } else {
      ma[0] = Fa[c - sb];
      ma[1] = Fa[c];
      mb[0] = Fb[c - sa];
      mb[1] = Fb[c];
    }
    const T* Ec = Ecb + (long long)e * g.box;
    ec[0] = Ec[c - sa - sb];
    ec[1] = Ec[c - sb];
    ec[2] = Ec[c - sa];
    ec[3] = Ec[c];
    E[e][(long long)b * g.box + c] = ct_corner<T, SMOOTH>(ea, eb, ec, ma, mb);
  }
}

long long tiles_nodes(const Geom& g) {
  return ((long long)(g.mb[0] + 1) * (g.mb[1] + 1) * (g.mb[2] + 1) * g.nblk + THREADS - 1) / THREADS;
}

cudaError_t launch_emfs(const MeshView& v, const Dispatch* d, cudaStream_t st) {
  const long long grid = d ? d->nwork : tiles_nodes(v.g);
  if (grid <= 0) return cudaSuccess;
  const MeshView* vs = d ? d->views : nullptr;
  const WorkItem* wk = d ? d->work : nullptr;
  const bool smooth = v.g.ct_delta > 0.0;
  if (v.a.mixed) {
    if (smooth)
      k_emf<float, true><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk);
    else
      k_emf<float, false><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk);
  } else {
    if (smooth)
      k_emf<double, true><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk);
    else
      k_emf<double, false><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Register update of one stage (Sec. 3.2.3, eq. rk-2s):
//   U_out = (g_base U_base + g_other U_other) + h L,  L = -[(F_x(i+1/2) - F_x(i-1/2))/dx + (F_y..)/dy + ..]
//   B_out = (g_base B_base + g_other B_other) - h curl_h E   (B1 uses E3 along y and E2 along z, cyclically)
// with U_other the register that is not U_base.  g_base = 1, g_other = 0 is the plain U_base + h L (VL2's
// stages, gamma_s = {0, 1}, written with the base register named directly).
// With a forcing acceleration a set, L of the cell-centred variables also holds the body-force source terms of
// the stage state (register stage_reg, the one the fluxes were formed from): rho a for the momentum and
// M . a for the energy, L = -div F + S, in FP64 in every precision.
// U_base / U_out may alias (stages update a register in place), so no __restrict__ here.
// In the mixed precision the plain form is accumulated as U_base - sum_d (h/dx_d) dF_d (+ h S) with fused
// multiply-adds, and B_base - (h/dx_a) dE_b + (h/dx_b) dE_a: a third fewer FP64 operations than forming L
// first (measured 8% faster there; in FP64, where the loads dominate, the chain of dependent FMAs measured 4%
// slower, so FP64 and the value-safe build keep the L form, which the oracle uses).
// ------------------------------------------------------------------------------------------------
template <class T, bool PLAIN>
__global__ void __launch_bounds__(256, 4) k_update(MeshView single, const MeshView* views, const WorkItem* work,
                                                int base_reg, int out_reg, double h, const double* dtbox, double beta,
                                                double g_base, double g_other, int stage_reg) {
  __shared__ MeshView sv;
  int tile, box;
  const MeshView& V = stage_view(sv, single, views, work, tile, &box);
  const Geom& g = V.g;
  if (dtbox) h = beta * dtbox[box];
  // h / dx_d, formed once per thread (the accumulated form's coefficients in the mixed precision)
  [[maybe_unused]] const double hidx[3] = {h * g.idx[0], h * g.idx[1], h * g.idx[2]};
  const double* Ubase = V.a.u[base_reg];
  const double* Uoth = V.a.u[1 - base_reg];
  double* Uout = V.a.u[out_reg];
  const double* Bb0 = V.a.b[base_reg][0];
  const double* Bb1 = V.a.b[base_reg][1];
  const double* Bb2 = V.a.b[base_reg][2];
  double* Bo0 = V.a.b[out_reg][0];
  double* Bo1 = V.a.b[out_reg][1];
  double* Bo2 = V.a.b[out_reg][2];
  const T* F0 = static_cast<const T*>(V.a.f[0]);
  const T* F1 = static_cast<const T*>(V.a.f[1]);
  const T* F2 = static_cast<const T*>(V.a.f[2]);
  const T* E0 = static_cast<const T*>(V.a.e[0]);
  const T* E1 = static_cast<const T*>(V.a.e[1]);
  const T* E2 = static_cast<const T*>(V.a.e[2]);
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int li[3] = {rem % ex + g.ng, (rem / ex) % ey + g.ng, rem / (ex * ey) + g.ng};
  const long long c = cell_off(g, li[2], li[1], li[0]);
  const long long stride[3] = {1LL, (long long)g.sx, (long long)g.sx * g.sy};
  const bool inside[3] = {li[0] < g.ng + g.mb[0], li[1] < g.ng + g.mb[1], li[2] < g.ng + g.mb[2]};
  if (inside[0] && inside[1] && inside[2]) {
    const T* F[3] = {F0 + (long long)b * 7 * g.box + c, F1 + (long long)b * 7 * g.box + c,
                     F2 + (long long)b * 7 * g.box + c};
    const long long ub = (long long)b * 5 * g.box + c;
    double src[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const bool forced = V.a.acc != nullptr;
    if (forced) {  // from the stage state, before an in-place update overwrites it
      const double* Us = V.a.u[stage_reg] + ub;
      const double* Ab = V.a.acc + (long long)b * 3 * g.box + c;
      const double rho = Us[0], ax = Ab[0], ay = Ab[g.box], az = Ab[2 * g.box];
      src[1] = rho * ax;
      src[2] = rho * ay;
      src[3] = rho * az;
      src[4] = fma(Us[3 * g.box], az, fma(Us[2 * g.box], ay, Us[g.box] * ax));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double df[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int comp;
        if (v == 0)
          comp = 0;
        else if (v == 4)
          comp = 4;
        else {
          const int m = v - 1;
          comp = (m == d) ? 1 : ((m == (d + 1) % 3) ? 2 : 3);
        }
        const T* fp = F[d] + (long long)comp * g.box;
        df[d] = to_f64(fp[stride[d]]) - to_f64(fp[0]);  // FP64 accumulation
      }
      const long long o = ub + (long long)v * g.box;
#ifndef VL2_VALUE_SAFE
      if (PLAIN && sizeof(T) == 4) {
        double acc = Ubase[o];
#pragma unroll
        for (int d = 0; d < 3; ++d) acc = fma(-hidx[d], df[d], acc);
        Uout[o] = forced ? fma(h, src[v], acc) : acc;
        continue;
      }
#endif
      const double dv = div3(df, g.idx);
      const double L = forced ? src[v] - dv : -dv;
      Uout[o] = plus_hl(stage_base(PLAIN, Ubase[o], PLAIN ? 0.0 : Uoth[o], g_base, g_other), h, L);
    }
  }
  const double* Bb[3] = {Bb0, Bb1, Bb2};
  const double* Bx[3] = {V.a.b[1 - base_reg][0], V.a.b[1 - base_reg][1], V.a.b[1 - base_reg][2]};
  double* Bo[3] = {Bo0, Bo1, Bo2};
  const T* E[3] = {E0 + (long long)b * g.box + c, E1 + (long long)b * g.box + c, E2 + (long long)b * g.box + c};
#pragma unroll
  for (int fd = 0; fd < 3; ++fd) {
    const int a = (fd + 1) % 3, bq = (fd + 2) % 3;
    if (!inside[a] || !inside[bq]) continue;
    const double deb = to_f64(E[bq][stride[a]]) - to_f64(E[bq][0]);
    const double dea = to_f64(E[a][stride[bq]]) - to_f64(E[a][0]);
    const long long o = (long long)b * g.box + c;
#ifndef VL2_VALUE_SAFE
    if (PLAIN && sizeof(T) == 4) {
      Bo[fd][o] = fma(hidx[bq], dea, fma(-hidx[a], deb, Bb[fd][o]));
      continue;
    }
#endif
    const double curl = curl2(deb, g.idx[a], dea, g.idx[bq]);
    Bo[fd][o] = plus_hl(stage_base(PLAIN, Bb[fd][o], PLAIN ? 0.0 : Bx[fd][o], g_base, g_other), h, -curl);
  }
}

// The plain (VL2-stage) update for two adjacent nodes along x per thread, with paired loads and stores
// (float2 / double2 for the fluxes and EMFs, double2 for the FP64 registers; the first node's x index
// ng + 2p is even, and rows and arrays start on 16-byte boundaries).  Per node it performs the operations of
// k_update<T, true> in the same order (the accumulated form with FP32 fluxes, the L form in FP64), so it
// gives the same bits; a face shared by the two cells is read once.  Meshes with an even ghost width only;
// the second node of the last pair of a row lies past the block when mb_x is even and is skipped.
template <class T>
__device__ __forceinline__ void ld_pair(const T* p, T& a, T& b);
template <>
__device__ __forceinline__ void ld_pair<float>(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x;
  b = v.y;
}
template <>
__device__ __forceinline__ void ld_pair<double>(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void st_pair(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }

template <class T>
__global__ void __launch_bounds__(256, 4) k_update_pair(MeshView single, int base_reg, int out_reg, double h,
                                                        const double* dtbox, double beta, int stage_reg) {
  constexpr bool ACC = sizeof(T) == 4;  // the accumulated form (FP32 fluxes); else the L form
  __shared__ MeshView sv;
  int tile;
  const MeshView& V = stage_view(sv, single, nullptr, nullptr, tile);
  const Geom& g = V.g;
  if (dtbox) h = beta * dtbox[0];  // the step formed on the device
  // h / dx_d, formed once per thread (the accumulated form's coefficients)
  const double hidx[3] = {h * g.idx[0], h * g.idx[1], h * g.idx[2]};
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const int px = (ex + 1) / 2;
  const long long per = (long long)px * ey * ez;
  const long long t = (long long)tile * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return;
  const int b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i0 = 2 * (rem % px) + g.ng;
  const int j = (rem / px) % ey + g.ng, k = rem / (px * ey) + g.ng;
  const bool node1 = i0 + 1 <= g.ng + g.mb[0];  // the second node exists
  const bool in0 = i0 < g.ng + g.mb[0], in1 = i0 + 1 < g.ng + g.mb[0];  // cells along x
  const bool iny = j < g.ng + g.mb[1], inz = k < g.ng + g.mb[2];
  const long long c = cell_off(g, k, j, i0);
  const long long sy = g.sx, sz = (long long)g.sx * g.sy;
  const double* Ubase = V.a.u[base_reg];
  double* Uout = V.a.u[out_reg];
  const T* F[3] = {static_cast<const T*>(V.a.f[0]) + (long long)b * 7 * g.box + c,
                   static_cast<const T*>(V.a.f[1]) + (long long)b * 7 * g.box + c,
                   static_cast<const T*>(V.a.f[2]) + (long long)b * 7 * g.box + c};
  if (in0 && iny && inz) {
    const long long ub = (long long)b * 5 * g.box + c;
    double src0[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, src1[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const bool forced = V.a.acc != nullptr;
    if (forced) {  // from the stage state, before an in-place update overwrites it
      const double* Us = V.a.u[stage_reg] + ub;
      const double* Ab = V.a.acc + (long long)b * 3 * g.box + c;
      double r0, r1, ax0, ax1, ay0, ay1, az0, az1, m10, m11, m20, m21, m30, m31;
      ld_pair(Us, r0, r1);
      ld_pair(Ab, ax0, ax1);
      ld_pair(Ab + g.box, ay0, ay1);
      ld_pair(Ab + 2 * g.box, az0, az1);
      ld_pair(Us + g.box, m10, m11);
      ld_pair(Us + 2 * g.box, m20, m21);
      ld_pair(Us + 3 * g.box, m30, m31);
      src0[1] = r0 * ax0;
      src0[2] = r0 * ay0;
      src0[3] = r0 * az0;
      src0[4] = fma(m30, az0, fma(m20, ay0, m10 * ax0));
      src1[1] = r1 * ax1;
      src1[2] = r1 * ay1;
      src1[3] = r1 * az1;
      src1[4] = fma(m31, az1, fma(m21, ay1, m11 * ax1));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double d0[3], d1[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int comp;
        if (v == 0)
          comp = 0;
        else if (v == 4)
          comp = 4;
        else {
          const int m = v - 1;
          comp = (m == d) ? 1 : ((m == (d + 1) % 3) ? 2 : 3);
        }
        const T* fp = F[d] + (long long)comp * g.box;
        T a0, a1, b0, b1;
        ld_pair(fp, a0, a1);
        if (d == 0) {
          b0 = a1;
          b1 = in1 ? fp[2] : T(0);
        } else {
          ld_pair(fp + (d == 1 ? sy : sz), b0, b1);
        }
        d0[d] = to_f64(b0) - to_f64(a0);
        d1[d] = to_f64(b1) - to_f64(a1);
      }
      const long long o = ub + (long long)v * g.box;
      double acc0, acc1;
      ld_pair(Ubase + o, acc0, acc1);
      if constexpr (ACC) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          acc0 = fma(-hidx[d], d0[d], acc0);
          acc1 = fma(-hidx[d], d1[d], acc1);
        }
        if (forced) {
          acc0 = fma(h, src0[v], acc0);
          acc1 = fma(h, src1[v], acc1);
        }
      } else {
        const double dv0 = div3(d0, g.idx), dv1 = div3(d1, g.idx);
        acc0 = plus_hl(acc0, h, forced ? src0[v] - dv0 : -dv0);
        acc1 = plus_hl(acc1, h, forced ? src1[v] - dv1 : -dv1);
      }
      if (in1)
        st_pair(Uout + o, acc0, acc1);
      else
        Uout[o] = acc0;
    }
  }
  const T* E[3] = {static_cast<const T*>(V.a.e[0]) + (long long)b * g.box + c,
                   static_cast<const T*>(V.a.e[1]) + (long long)b * g.box + c,
                   static_cast<const T*>(V.a.e[2]) + (long long)b * g.box + c};
  // B_out of one node from dE_b (along a) and dE_a (along b): the accumulated form or the L form
  auto bnew = [&](double base, double deb, int a, double dea, int bq) -> double {
    if constexpr (ACC)
      return fma(hidx[bq], dea, fma(-hidx[a], deb, base));
    else
      return plus_hl(base, h, -curl2(deb, g.idx[a], dea, g.idx[bq]));
  };
  const long long o = (long long)b * g.box + c;
  // face field fd = 0: B1 -= (h/dy) dE3/dy, += (h/dz) dE2/dz at both nodes (transversally inside)
  if (iny && inz) {
    T p0, p1, q0, q1, r0, r1, s0, s1;
    ld_pair(E[2], p0, p1);
    ld_pair(E[2] + sy, q0, q1);
    ld_pair(E[1], r0, r1);
    ld_pair(E[1] + sz, s0, s1);
    double b0, b1;
    ld_pair(V.a.b[base_reg][0] + o, b0, b1);
    const double n0 = bnew(b0, to_f64(q0) - to_f64(p0), 1, to_f64(s0) - to_f64(r0), 2);
    const double n1 = bnew(b1, to_f64(q1) - to_f64(p1), 1, to_f64(s1) - to_f64(r1), 2);
    if (node1)
      st_pair(V.a.b[out_reg][0] + o, n0, n1);
    else
      V.a.b[out_reg][0][o] = n0;
  }
  // fd = 1: B2 -= (h/dz) dE1/dz, += (h/dx) dE3/dx (inside along z and x)
  if (inz && in0) {
    T p0, p1, q0, q1, r0, r1;
    ld_pair(E[0], p0, p1);
    ld_pair(E[0] + sz, q0, q1);
    ld_pair(E[2], r0, r1);
    const T r2 = in1 ? E[2][2] : T(0);
    double b0, b1;
    ld_pair(V.a.b[base_reg][1] + o, b0, b1);
    const double n0 = bnew(b0, to_f64(q0) - to_f64(p0), 2, to_f64(r1) - to_f64(r0), 0);
    const double n1 = bnew(b1, to_f64(q1) - to_f64(p1), 2, to_f64(r2) - to_f64(r1), 0);
    if (in1)
      st_pair(V.a.b[out_reg][1] + o, n0, n1);
    else
      V.a.b[out_reg][1][o] = n0;
  }
  // fd = 2: B3 -= (h/dx) dE2/dx, += (h/dy) dE1/dy (inside along x and y)
  if (in0 && iny) {
    T p0, p1, q0, q1, r0, r1;
    ld_pair(E[1], p0, p1);
    const T p2 = in1 ? E[1][2] : T(0);
    ld_pair(E[0], q0, q1);
    ld_pair(E[0] + sy, r0, r1);
    double b0, b1;
    ld_pair(V.a.b[base_reg][2] + o, b0, b1);
    const double n0 = bnew(b0, to_f64(p1) - to_f64(p0), 0, to_f64(r0) - to_f64(q0), 1);
    const double n1 = bnew(b1, to_f64(p2) - to_f64(p1), 0, to_f64(r1) - to_f64(q1), 1);
    if (in1)
      st_pair(V.a.b[out_reg][2] + o, n0, n1);
    else
      V.a.b[out_reg][2][o] = n0;
  }
}

cudaError_t launch_update(const MeshView& v, const Dispatch* d, int base_reg, int out_reg, double h,
                          const double* dtbox, double beta, cudaStream_t st, double g_base, double g_other,
                          int stage_reg) {
  if (stage_reg < 0) stage_reg = base_reg;
  const long long grid = d ? d->nwork : tiles_nodes(v.g);
  if (grid <= 0) return cudaSuccess;
  const MeshView* vs = d ? d->views : nullptr;
  const WorkItem* wk = d ? d->work : nullptr;
  const bool plain = g_other == 0.0 && g_base == 1.0;  // U_base + h L: the VL2 stages
#ifndef VL2_VALUE_SAFE
  // two nodes per thread (one mesh, even ghost width) in the mixed precision; in FP64 the paired kernel
  // measured no faster (3.39 against 3.35 ms per 256^3 cycle), so FP64 keeps one node per thread
  if (v.a.mixed && plain && !d && v.g.ng % 2 == 0) {
    const Geom& g = v.g;
    const long long pairs = (long long)((g.mb[0] + 2) / 2) * (g.mb[1] + 1) * (g.mb[2] + 1) * g.nblk;
    k_update_pair<float><<<(unsigned)((pairs + THREADS - 1) / THREADS), THREADS, 0, st>>>(v, base_reg, out_reg, h,
                                                                                          dtbox, beta, stage_reg);
    return cudaGetLastError();
  }
#endif
  if (v.a.mixed) {
    if (plain)
      k_update<float, true><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, base_reg, out_reg, h, dtbox, beta, g_base,
                                                                g_other, stage_reg);
    else
      k_update<float, false><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, base_reg, out_reg, h, dtbox, beta,
                                                                 g_base, g_other, stage_reg);
  } else {
    if (plain)
      k_update<double, true><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, base_reg, out_reg, h, dtbox, beta,
                                                                 g_base, g_other, stage_reg);
    else
      k_update<double, false><<<(unsigned)grid, THREADS, 0, st>>>(v, vs, wk, base_reg, out_reg, h, dtbox, beta,
                                                                  g_base, g_other, stage_reg);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Global-array I/O.  Threads cover (block, k, j, i) with i, j, k in [0, mb] (faces need the +1).
// ------------------------------------------------------------------------------------------------
struct IoIdx {
  int b, li[3], gi[3];
};

__device__ __forceinline__ bool io_index(const Geom& g, IoIdx& x) {
  const int ex = g.mb[0] + 1, ey = g.mb[1] + 1, ez = g.mb[2] + 1;
  const long long per = (long long)ex * ey * ez;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * g.nblk) return false;
  x.b = (int)(t / per);
  int rem = (int)(t - (long long)x.b * per);
  x.li[0] = rem % ex;
  x.li[1] = (rem / ex) % ey;
  x.li[2] = rem / (ex * ey);
  int loc[3];
  block_loc(g, x.b, loc);
  for (int q = 0; q < 3; ++q) x.gi[q] = loc[q] * g.mb[q] + x.li[q];
  return true;
}

static inline unsigned io_grid(const Geom& g) {
  return grid_for((long long)(g.mb[0] + 1) * (g.mb[1] + 1) * (g.mb[2] + 1) * g.nblk, 256);
}

__global__ void __launch_bounds__(256) k_scatter_prims(Geom g, double* U, double* B0, double* B1, double* B2,
                                                       const double* __restrict__ w, const double* __restrict__ b1,
                                                       const double* __restrict__ b2, const double* __restrict__ b3) {
  IoIdx x;
  if (!io_index(g, x)) return;
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long c = cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng);
  const long long o = (long long)x.b * g.box + c;
  const bool in[3] = {x.li[0] < g.mb[0], x.li[1] < g.mb[1], x.li[2] < g.mb[2]};
  const long long f1 = ((long long)x.gi[2] * NY + x.gi[1]) * (NX + 1) + x.gi[0];
  const long long f2 = ((long long)x.gi[2] * (NY + 1) + x.gi[1]) * NX + x.gi[0];
  const long long f3 = ((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0];
  if (in[1] && in[2]) B0[o] = b1[f1];
  if (in[0] && in[2]) B1[o] = b2[f2];
  if (in[0] && in[1]) B2[o] = b3[f3];
  if (in[0] && in[1] && in[2]) {
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0];
    const double d = w[gc], vx = w[n + gc], vy = w[2 * n + gc], vz = w[3 * n + gc], p = w[4 * n + gc];
    const double bcx = 0.5 * (b1[f1] + b1[f1 + 1]);
    const double bcy = 0.5 * (b2[f2] + b2[f2 + NX]);
    const double bcz = 0.5 * (b3[f3] + b3[f3 + (long long)NX * NY]);
    double* Ub = U + (long long)x.b * 5 * g.box + c;
    Ub[0] = d;
    Ub[g.box] = d * vx;
    Ub[2 * g.box] = d * vy;
    Ub[3 * g.box] = d * vz;
    Ub[4 * g.box] = p * g.igm1 + 0.5 * d * ((vx * vx + vy * vy) + vz * vz) + 0.5 * ((bcx * bcx + bcy * bcy) + bcz * bcz);
  }
}

cudaError_t launch_scatter_prims(const Geom& g, const Arrays& a, const double* w, const double* b1, const double* b2,
                                 const double* b3, cudaStream_t st) {
  k_scatter_prims<<<io_grid(g), 256, 0, st>>>(g, a.u[0], a.b[0][0], a.b[0][1], a.b[0][2], w, b1, b2, b3);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_scatter_cons(Geom g, double* U, double* B0, double* B1, double* B2,
                                                      const double* __restrict__ u, const double* __restrict__ b1,
                                                      const double* __restrict__ b2, const double* __restrict__ b3) {
  IoIdx x;
  if (!io_index(g, x)) return;
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long c = cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng);
  const long long o = (long long)x.b * g.box + c;
  const bool in[3] = {x.li[0] < g.mb[0], x.li[1] < g.mb[1], x.li[2] < g.mb[2]};
  if (in[1] && in[2]) B0[o] = b1[((long long)x.gi[2] * NY + x.gi[1]) * (NX + 1) + x.gi[0]];
  if (in[0] && in[2]) B1[o] = b2[((long long)x.gi[2] * (NY + 1) + x.gi[1]) * NX + x.gi[0]];
  if (in[0] && in[1]) B2[o] = b3[((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0]];
  if (in[0] && in[1] && in[2]) {
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0];
    double* Ub = U + (long long)x.b * 5 * g.box + c;
    for (int v = 0; v < 5; ++v) Ub[(long long)v * g.box] = u[v * n + gc];
  }
}

cudaError_t launch_scatter_cons(const Geom& g, const Arrays& a, const double* u, const double* b1, const double* b2,
                                const double* b3, cudaStream_t st) {
  k_scatter_cons<<<io_grid(g), 256, 0, st>>>(g, a.u[0], a.b[0][0], a.b[0][1], a.b[0][2], u, b1, b2, b3);
  return cudaGetLastError();
}

// periodic duplicate faces (face N and face 0) must be bitwise equal
__global__ void k_check_periodic(Geom g, const double* b1, const double* b2, const double* b3, unsigned long long* cnt) {
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nxy = (long long)NX * NY, nyz = (long long)NY * NZ, nxz = (long long)NX * NZ;
  if (t < nyz && g.bc[0] == BC_PERIODIC) {
    const long long r = t * (NX + 1);
    if (b1[r] != b1[r + NX]) atomicAdd(cnt, 1ULL);
  }
  if (t < nxz && g.bc[2] == BC_PERIODIC) {
    const long long kk = t / NX, ii = t % NX;
    const long long r0 = (kk * (NY + 1)) * NX + ii;
    if (b2[r0] != b2[r0 + (long long)NY * NX]) atomicAdd(cnt, 1ULL);
  }
  if (t < nxy && g.bc[4] == BC_PERIODIC) {
    if (b3[t] != b3[t + (long long)NZ * nxy]) atomicAdd(cnt, 1ULL);
  }
}

cudaError_t launch_check_periodic(const Geom& g, const double* b1, const double* b2, const double* b3,
                                  unsigned long long* count, cudaStream_t st) {
  long long n = (long long)g.N[1] * g.N[2];
  n = n > (long long)g.N[0] * g.N[2] ? n : (long long)g.N[0] * g.N[2];
  n = n > (long long)g.N[0] * g.N[1] ? n : (long long)g.N[0] * g.N[1];
  k_check_periodic<<<grid_for(n, 256), 256, 0, st>>>(g, b1, b2, b3, count);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_gather_cons(Geom g, const double* __restrict__ U, const double* __restrict__ B0,
                                                     const double* __restrict__ B1, const double* __restrict__ B2,
                                                     double* u, double* b1, double* b2, double* b3) {
  IoIdx x;
  if (!io_index(g, x)) return;
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long c = cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng);
  const long long o = (long long)x.b * g.box + c;
  const bool in[3] = {x.li[0] < g.mb[0], x.li[1] < g.mb[1], x.li[2] < g.mb[2]};
  const bool own[3] = {in[0] || x.gi[0] == NX, in[1] || x.gi[1] == NY, in[2] || x.gi[2] == NZ};
  if (b1 && own[0] && in[1] && in[2]) b1[((long long)x.gi[2] * NY + x.gi[1]) * (NX + 1) + x.gi[0]] = B0[o];
  if (b2 && own[1] && in[0] && in[2]) b2[((long long)x.gi[2] * (NY + 1) + x.gi[1]) * NX + x.gi[0]] = B1[o];
  if (b3 && own[2] && in[0] && in[1]) b3[((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0]] = B2[o];
  if (u && in[0] && in[1] && in[2]) {
    const long long n = (long long)NX * NY * NZ;
    const long long gc = ((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0];
    const double* Ub = U + (long long)x.b * 5 * g.box + c;
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v * n + gc] = Ub[(long long)v * g.box];
  }
}

cudaError_t launch_gather_cons(const Geom& g, const Arrays& a, double* u, double* b1, double* b2, double* b3,
                               cudaStream_t st) {
  k_gather_cons<<<io_grid(g), 256, 0, st>>>(g, a.u[0], a.b[0][0], a.b[0][1], a.b[0][2], u, b1, b2, b3);
  return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(256) k_gather_prims(Geom g, const T* __restrict__ W, double* w) {
  IoIdx x;
  if (!io_index(g, x)) return;
  if (x.li[0] >= g.mb[0] || x.li[1] >= g.mb[1] || x.li[2] >= g.mb[2]) return;
  const int NX = g.N[0], NY = g.N[1], NZ = g.N[2];
  const long long n = (long long)NX * NY * NZ;
  const long long gc = ((long long)x.gi[2] * NY + x.gi[1]) * NX + x.gi[0];
  const T* Wb = W + (long long)x.b * 8 * g.box + cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng);
#pragma unroll
  for (int v = 0; v < 8; ++v) w[v * n + gc] = (double)Wb[(long long)v * g.box];
}

cudaError_t launch_gather_prims(const Geom& g, const Arrays& a, double* w, cudaStream_t st) {
  if (a.mixed)
    k_gather_prims<float><<<io_grid(g), 256, 0, st>>>(g, static_cast<const float*>(a.w), w);
  else
    k_gather_prims<double><<<io_grid(g), 256, 0, st>>>(g, static_cast<const double*>(a.w), w);
  return cudaGetLastError();
}

// fluxes of sweep `dir` on the global face grid [7][..]; a face on a block boundary is taken from the
// block where it is the lower face (global face N from the last block)
template <class T>
__global__ void __launch_bounds__(256) k_gather_fluxes(Geom g, int dir, const T* __restrict__ F, double* out) {
  IoIdx x;
  if (!io_index(g, x)) return;
  int gd[3] = {g.N[0], g.N[1], g.N[2]};
  gd[dir] += 1;
  for (int q = 0; q < 3; ++q) {
    if (q == dir) {
      if (x.li[q] == g.mb[q] && x.gi[q] != g.N[q]) return;
    } else if (x.li[q] >= g.mb[q]) {
      return;
    }
  }
  const long long nf = (long long)gd[0] * gd[1] * gd[2];
  const long long gf = ((long long)x.gi[2] * gd[1] + x.gi[1]) * gd[0] + x.gi[0];
  const T* Fb = F + (long long)x.b * 7 * g.box + cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng);
#pragma unroll
  for (int n = 0; n < 7; ++n) out[n * nf + gf] = (double)Fb[(long long)n * g.box];
}

cudaError_t launch_gather_fluxes(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st) {
  if (a.mixed)
    k_gather_fluxes<float><<<io_grid(g), 256, 0, st>>>(g, dir, static_cast<const float*>(a.f[dir]), out);
  else
    k_gather_fluxes<double><<<io_grid(g), 256, 0, st>>>(g, dir, static_cast<const double*>(a.f[dir]), out);
  return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(256) k_gather_emfs(Geom g, int e, const T* __restrict__ E, double* out) {
  IoIdx x;
  if (!io_index(g, x)) return;
  int gd[3] = {g.N[0] + 1, g.N[1] + 1, g.N[2] + 1};
  gd[e] -= 1;
  for (int q = 0; q < 3; ++q) {
    if (q == e) {
      if (x.li[q] >= g.mb[q]) return;
    } else if (x.li[q] == g.mb[q] && x.gi[q] != g.N[q]) {
      return;
    }
  }
  const long long gf = ((long long)x.gi[2] * gd[1] + x.gi[1]) * gd[0] + x.gi[0];
  out[gf] = (double)E[(long long)x.b * g.box + cell_off(g, x.li[2] + g.ng, x.li[1] + g.ng, x.li[0] + g.ng)];
}

cudaError_t launch_gather_emfs(const Geom& g, const Arrays& a, int dir, double* out, cudaStream_t st) {
  if (a.mixed)
    k_gather_emfs<float><<<io_grid(g), 256, 0, st>>>(g, dir, static_cast<const float*>(a.e[dir]), out);
  else
    k_gather_emfs<double><<<io_grid(g), 256, 0, st>>>(g, dir, static_cast<const double*>(a.e[dir]), out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Diagnostics: fixed grid, grid-stride loops, per-CTA partials, then one CTA combines the partials in a
// fixed order (deterministic results).
// ------------------------------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__device__ __forceinline__ void active_cell(const Geom& g, long long t, int& b, long long& c) {
  const long long per = (long long)g.mb[0] * g.mb[1] * g.mb[2];
  b = (int)(t / per);
  int rem = (int)(t - (long long)b * per);
  const int i = rem % g.mb[0] + g.ng;
  rem /= g.mb[0];
  const int j = rem % g.mb[1] + g.ng;
  const int k = rem / g.mb[1] + g.ng;
  c = cell_off(g, k, j, i);
}

__global__ void __launch_bounds__(RED_THREADS) k_divb_partial(Geom g, const double* __restrict__ B0,
                                                              const double* __restrict__ B1,
                                                              const double* __restrict__ B2, double* part) {
  const long long n = (long long)g.mb[0] * g.mb[1] * g.mb[2] * g.nblk;
  double mx = 0.0, s2 = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int b;
    long long c;
    active_cell(g, t, b, c);
    const long long o = (long long)b * g.box + c;
    const long long sy = g.sx, sz = (long long)g.sx * g.sy;
    const double dv = (B0[o + 1] - B0[o]) * g.idx[0] + (B1[o + sy] - B1[o]) * g.idx[1] + (B2[o + sz] - B2[o]) * g.idx[2];
    mx = fmax(mx, fabs(dv));
    const double bx = 0.5 * (B0[o] + B0[o + 1]), by = 0.5 * (B1[o] + B1[o + sy]), bz = 0.5 * (B2[o] + B2[o + sz]);
    s2 += bx * bx + by * by + bz * bz;
  }
  __shared__ double smx[RED_THREADS], ss[RED_THREADS];
  smx[threadIdx.x] = mx;
  ss[threadIdx.x] = s2;
  __syncthreads();
  for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
      ss[threadIdx.x] += ss[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = smx[0];
    part[2 * blockIdx.x + 1] = ss[0];
  }
}

__global__ void k_combine(const double* part, int nparts, int width, unsigned max_mask, double* out) {
  // thread v combines component v over the partials, sequentially (max, or a Neumaier sum)
  const int v = threadIdx.x;
  if (v >= width) return;
  if ((max_mask >> v) & 1u) {
    double m = 0.0;
    for (int q = 0; q < nparts; ++q) m = fmax(m, part[q * width + v]);
    out[v] = m;
  } else {
    double s = 0.0, comp = 0.0;
    for (int q = 0; q < nparts; ++q) {
      const double y = part[q * width + v];
      const double t = s + y;
      if (fabs(s) >= fabs(y))
        comp += (s - t) + y;
      else
        comp += (y - t) + s;
      s = t;
    }
    out[v] = s + comp;
  }
}

cudaError_t launch_divb(const Geom& g, const Arrays& a, double* result2, cudaStream_t st) {
  k_divb_partial<<<a.red_ctas, RED_THREADS, 0, st>>>(g, a.b[0][0], a.b[0][1], a.b[0][2], a.red);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_combine<<<1, 32, 0, st>>>(a.red, a.red_ctas, 2, 1u, result2);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(RED_THREADS) k_totals_partial(Geom g, const double* __restrict__ U,
                                                                const double* __restrict__ B0,
                                                                const double* __restrict__ B1,
                                                                const double* __restrict__ B2, double* part) {
  const long long n = (long long)g.mb[0] * g.mb[1] * g.mb[2] * g.nblk;
  const double dv = g.dx[0] * g.dx[1] * g.dx[2];
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int b;
    long long c;
    active_cell(g, t, b, c);
    const double* Ub = U + (long long)b * 5 * g.box + c;
    for (int v = 0; v < 5; ++v) s[v] += Ub[(long long)v * g.box] * dv;
    const long long o = (long long)b * g.box + c;
    s[5] += 0.5 * (B0[o] + B0[o + 1]) * dv;
    s[6] += 0.5 * (B1[o] + B1[o + g.sx]) * dv;
    s[7] += 0.5 * (B2[o] + B2[o + (long long)g.sx * g.sy]) * dv;
  }
  __shared__ double sh[8][RED_THREADS];
  for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] = s[v];
  __syncthreads();
  for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[8 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

cudaError_t launch_totals(const Geom& g, const Arrays& a, double* result8, cudaStream_t st) {
  k_totals_partial<<<a.red_ctas, RED_THREADS, 0, st>>>(g, a.u[0], a.b[0][0], a.b[0][1], a.b[0][2], a.red);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_combine<<<1, 32, 0, st>>>(a.red, a.red_ctas, 8, 0u, result8);
  return cudaGetLastError();
}

}  // namespace vl2
