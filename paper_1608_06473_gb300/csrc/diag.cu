// Diagnostics that are not part of the method:
//
//  * hhg_peak_rate: throughput of the arithmetic pipes the stencil kernels
//    use (FP64 FMA, FP32 FMA, INT32 multiply-add), measured by a kernel of
//    independent multiply-add chains that fills every SM.  These are the
//    denominators of the roofline fractions of the FP64 and FP32 kernels.
//  * hhg_check_arith: the hand-written arithmetic helpers of arith.cuh
//    applied elementwise to device arrays, so that a test can compare them
//    with the IEEE operations they stand for.
#include <algorithm>
#include <string>

#include <cuda_runtime.h>

#include "arith.cuh"
#include "common.h"

namespace hhg {

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 8;
constexpr int CHAINS = 8;  // independent multiply-add chains per thread

// x <- x m + c on CHAINS independent chains; with 0 < m < 1 every chain
// settles at c / (1 - m), so nothing overflows or goes subnormal.
template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) peak_fma_kernel(int64_t iters, T m, T c, T* out) {
  T x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = (T)(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], m, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) peak_imad_kernel(int64_t iters, unsigned m, unsigned c, unsigned* out) {
  unsigned x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = threadIdx.x + k;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = x[k] * m + c;
  }
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s ^= x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void check_rcp_kernel(const long long* a, const int* e, double* out, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = rcp_i64_scaled(a[t], e[t]);
}
__global__ void check_cvt_scaled_kernel(const long long* a, const int* e, double* out, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = i64_to_f64_scaled(a[t], e[t]);
}
__global__ void check_div32_kernel(const float* a, const float* b, float* out, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = div_nr32(a[t], b[t]);
}

template <class F>
hhg_status guarded_diag(F&& fn) {
  try {
    fn();
    set_error("");
    return HHG_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.st;
  }
}

}  // namespace

}  // namespace hhg

using namespace hhg;

extern "C" hhg_status hhg_peak_rate(int kind, double* ops_per_s, double* ms_out, void* stream) {
  return guarded_diag([&] {
    HHG_CHECK(kind >= 0 && kind <= 2, HHG_EINVAL, "kind must be 0 (FP64 FMA), 1 (FP32 FMA) or 2 (INT32 IMAD)");
    HHG_CHECK(ops_per_s != nullptr, HHG_EINVAL, "NULL ops_per_s");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    HHG_CUDA(cudaGetDevice(&dev));
    HHG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const int64_t threads = (int64_t)blocks * PEAK_THREADS;
    void* out = nullptr;
    HHG_CUDA(cudaMallocAsync(&out, (size_t)threads * 8, st));
    cudaEvent_t e0, e1;
    HHG_CUDA(cudaEventCreate(&e0));
    HHG_CUDA(cudaEventCreate(&e1));
    auto run = [&](int64_t iters) -> float {
      HHG_CUDA(cudaEventRecord(e0, st));
      if (kind == 0)
        peak_fma_kernel<double><<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999999, 1e-6, (double*)out);
      else if (kind == 1)
        peak_fma_kernel<float><<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.9999f, 1e-4f, (float*)out);
      else
        peak_imad_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, 1664525u, 1013904223u, (unsigned*)out);
      HHG_CUDA(cudaGetLastError());
      count_launch();
      HHG_CUDA(cudaEventRecord(e1, st));
      HHG_CUDA(cudaEventSynchronize(e1));
      float t = 0.0f;
      HHG_CUDA(cudaEventElapsedTime(&t, e0, e1));
      return t;
    };
    // calibrate to about 150 ms, then keep the best of three
    int64_t iters = 1024;
    float t = run(iters);
    while (t < 20.0f && iters < ((int64_t)1 << 40)) {
      iters *= 4;
      t = run(iters);
    }
    iters = std::max<int64_t>(1, (int64_t)((double)iters * 150.0 / t));
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) best = std::min(best, run(iters));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HHG_CUDA(cudaFreeAsync(out, st));
    *ops_per_s = (double)threads * (double)iters * CHAINS / (best * 1e-3);
    if (ms_out) *ms_out = best;
  });
}

extern "C" hhg_status hhg_check_arith(int which, const void* a, const void* b, void* out, int64_t n, void* stream) {
  return guarded_diag([&] {
    HHG_CHECK(which >= 0 && which <= 2, HHG_EINVAL, "which must be 0, 1 or 2");
    HHG_CHECK(n >= 0 && a && b && out, HHG_EINVAL, "NULL argument or negative n");
    if (n == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (which == 0)
      check_div32_kernel<<<g, 256, 0, st>>>((const float*)a, (const float*)b, (float*)out, n);
    else if (which == 1)
      check_rcp_kernel<<<g, 256, 0, st>>>((const long long*)a, (const int*)b, (double*)out, n);
    else
      check_cvt_scaled_kernel<<<g, 256, 0, st>>>((const long long*)a, (const int*)b, (double*)out, n);
    HHG_CUDA(cudaGetLastError());
    count_launch();
  });
}
