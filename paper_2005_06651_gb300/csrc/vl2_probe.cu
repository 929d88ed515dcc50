// Measurement aids with no counterpart in the paper:
//  - vl2_debug_fp64_peak: the FP64 fused multiply-add throughput of the device, the peak that the roofline of
//    the FP64-bound flux kernels is stated against;
//  - vl2_debug_arith: pointwise evaluation of this library's FP64 reciprocal / square-root forms and its
//    integer-pipe float <-> double conversions, next to CUDA's own operations, so that tests can bound them.
#include <cuda_runtime.h>

#include "vl2_internal.h"
#include "vl2_physics.cuh"
#include "vl2_tma.cuh"
#include "vl2mhd.h"

namespace vl2 {
namespace {

constexpr int kChains = 16;  // independent FMA chains per thread (enough to hide the FMA latency)

// Every thread runs kChains independent chains a <- a * m + c for `iters` rounds: 2 FP64 operations per FMA.
// The fixed point c / (1 - m) keeps every value finite and normal.  The single store is conditional on a
// value no chain reaches, so the chains cannot be removed as dead code.
__global__ void __launch_bounds__(256) k_dfma_peak(long long iters, double m, double c, double* out) {
  double a[kChains];
#pragma unroll
  for (int u = 0; u < kChains; ++u) a[u] = 1.0 + 1e-3 * (threadIdx.x + u);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < kChains; ++u) s += a[u];
  if (s == -1.0) out[0] = s;
}

__global__ void k_arith(int fn, long long n, const double* __restrict__ x, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double v = x[t];
  double r = 0.0;
  switch (fn) {
    case VL2_AR_RCP_NR: r = rcp_nr(v); break;
    case VL2_AR_RSQRT_NR: r = rsqrt_nr(v); break;
    case VL2_AR_SQRT_NR: r = sqrt_nr(v); break;
    case VL2_AR_INV_ANY: r = inv_any<double>(v); break;
    case VL2_AR_ROOT_ANY: r = root_any<double>(v); break;
    case VL2_AR_RROOT_ANY: r = rroot_any<double>(v); break;
    case VL2_AR_TO_F32: r = (double)to_f32(v); break;
    case VL2_AR_TO_F64: r = to_f64((float)v); break;
    case VL2_AR_IEEE_RCP: r = 1.0 / v; break;
    case VL2_AR_IEEE_SQRT: r = sqrt(v); break;
    case VL2_AR_CUDA_RSQRT: r = rsqrt(v); break;
    case VL2_AR_CUDA_D2F: r = (double)__double2float_rn(v); break;
    default: break;
  }
  out[t] = r;
}

// One thread waits, with the same bounded wait as the TMA-staged kernels, on an mbarrier phase that
// nothing completes (no arrival, no copy); out[0] = 1 when the wait gave up, 0 if it (wrongly) completed.
__global__ void k_mbar_timeout(int polls, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  out[0] = mbar_wait_bounded(&bar, 0u, polls) ? 0 : 1;
}

}  // namespace
}  // namespace vl2

extern "C" {

vl2_status vl2_debug_wait_timeout(int polls, int* out, void* stream) {
  if (!out || polls <= 0 || polls > (1 << 20)) {
    vl2::record_error("vl2_debug_wait_timeout: out must be non-NULL and polls in 1 .. 2^20");
    return VL2_E_ARG;
  }
  vl2::k_mbar_timeout<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(polls, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vl2::record_error(cudaGetErrorString(e));
    return VL2_E_CUDA;
  }
  return VL2_OK;
}

vl2_status vl2_debug_fp64_peak(long long iters, int ctas, int threads, double* out, void* stream) {
  if (!out || iters <= 0 || ctas <= 0 || threads <= 0 || threads > 256 || threads % 32 != 0) {
    vl2::record_error("vl2_debug_fp64_peak: out must be non-NULL, iters and ctas positive, threads 32..256 "
                      "in steps of 32");
    return VL2_E_ARG;
  }
  vl2::k_dfma_peak<<<ctas, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.9999999, 1e-7, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vl2::record_error(cudaGetErrorString(e));
    return VL2_E_CUDA;
  }
  return VL2_OK;
}

vl2_status vl2_debug_arith(int fn, long long n, const double* x, double* out, void* stream) {
  if (fn < 0 || fn >= VL2_AR_COUNT || n < 0 || (n > 0 && (!x || !out))) {
    vl2::record_error("vl2_debug_arith: fn out of range, n < 0, or NULL array");
    return VL2_E_ARG;
  }
  if (n == 0) return VL2_OK;
  const long long blocks = (n + 255) / 256;
  vl2::k_arith<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, n, x, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vl2::record_error(cudaGetErrorString(e));
    return VL2_E_CUDA;
  }
  return VL2_OK;
}

}  // extern "C"
