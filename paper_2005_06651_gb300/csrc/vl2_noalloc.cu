// vl2_totals_noalloc: the conserved-totals reduction for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host that has handed all device memory to its own pool and
// forbids further allocations, or a pipeline that must not take the device-wide synchronisation that
// cudaMalloc / cudaFree can cause.  This entry point therefore allocates nothing.  The caller passes
// the state (device arrays in the global layout) and the output; the per-plane partial sums live in
// the file-scope array below, which every GPU that loads this library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "vl2_internal.h"
#include "vl2mhd.h"

namespace {

constexpr int kMaxPlanes = VL2_NOALLOC_MAX_NZ;  // one partial row of 8 sums per z-plane
constexpr int kThreads = 256;

// Shared by every call on a device: calls that overlap on the GPU race on it.  Every slot a call
// reads is written earlier in the same call, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_plane_sums[kMaxPlanes * 8];

// Device address of g_plane_sums per device, looked up once with that device current and kept for the life of
// the process (a reset of the device's context makes it stale; the header says so).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

vl2_status noalloc_fail(vl2_status s, const char* msg) {
  vl2::record_error(msg);  // read back through vl2_last_error(NULL)
  return s;
}

// One CTA per z-plane k: sums of rho, M1..3, E and the cell-centred field over the plane (times dV),
// in a fixed order (thread-strided, then a shared-memory tree), written to scratch row k.
__global__ void __launch_bounds__(kThreads) k_plane_sums(const double* __restrict__ u, const double* __restrict__ b1,
                                                         const double* __restrict__ b2, const double* __restrict__ b3,
                                                         int nx, int ny, int nz, double dv, double* rows) {
  const int k = blockIdx.x;
  const long long plane = (long long)nx * ny;
  const long long ncell = plane * nz;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long t = threadIdx.x; t < plane; t += blockDim.x) {
    const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
    const long long c = (long long)k * plane + t;
    for (int v = 0; v < 5; ++v) s[v] += u[v * ncell + c] * dv;
    const long long f1 = ((long long)k * ny + j) * (nx + 1) + i;
    const long long f2 = ((long long)k * (ny + 1) + j) * nx + i;
    const long long f3 = c;
    s[5] += 0.5 * (b1[f1] + b1[f1 + 1]) * dv;
    s[6] += 0.5 * (b2[f2] + b2[f2 + nx]) * dv;
    s[7] += 0.5 * (b3[f3] + b3[f3 + plane]) * dv;
  }
  __shared__ double sh[8][kThreads];
  for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] = s[v];
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int v = 0; v < 8; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 8) rows[8 * k + threadIdx.x] = sh[threadIdx.x][0];
}

// Thread v adds component v over the planes in order (Neumaier-compensated) into out[v].
__global__ void k_plane_combine(const double* rows, int nz, double* out) {
  const int v = threadIdx.x;
  if (v >= 8) return;
  double s = 0.0, comp = 0.0;
  for (int k = 0; k < nz; ++k) {
    const double y = rows[8 * k + v];
    const double t = s + y;
    comp += (fabs(s) >= fabs(y)) ? (s - t) + y : (y - t) + s;
    s = t;
  }
  out[v] = s + comp;
}

}  // namespace

extern "C" vl2_status vl2_totals_noalloc(const double* u, const double* b1, const double* b2, const double* b3,
                                         const int* nx, const double* dx, double* out, void* stream) {
  if (!u || !b1 || !b2 || !b3 || !nx || !dx || !out) return noalloc_fail(VL2_E_ARG, "NULL argument");
  if (nx[0] <= 0 || nx[1] <= 0 || nx[2] <= 0) return noalloc_fail(VL2_E_ARG, "grid sizes must be positive");
  if (nx[2] > kMaxPlanes)
    return noalloc_fail(VL2_E_ARG, "nz exceeds VL2_NOALLOC_MAX_NZ (the fixed scratch holds one row per z-plane)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(VL2_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(VL2_E_ARG, "device ordinal out of range");
  double* rows = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
      // first call on this device (it is current here): look up the device address of the scratch
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_plane_sums);
      if (e != cudaSuccess) return noalloc_fail(VL2_E_CUDA, cudaGetErrorString(e));
      g_scratch[dev] = static_cast<double*>(p);
    }
    rows = g_scratch[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double dv = dx[0] * dx[1] * dx[2];
  k_plane_sums<<<nx[2], kThreads, 0, st>>>(u, b1, b2, b3, nx[0], nx[1], nx[2], dv, rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(VL2_E_CUDA, cudaGetErrorString(e));
  k_plane_combine<<<1, 32, 0, st>>>(rows, nx[2], out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(VL2_E_CUDA, cudaGetErrorString(e));
  return VL2_OK;
}
