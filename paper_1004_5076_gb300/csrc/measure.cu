// Instrumentation: the FMA-pipe peak of the current GPU, measured by a
// kernel of independent fused multiply-add chains held in registers (no
// memory traffic), timed with CUDA events on the caller's stream.  It is the
// denominator of the arithmetic rooflines (complex128 path: FP64 FMA;
// complex64 path: packed FP32x2 FMA); not part of the paper's method.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_THREADS = 256;

// Every thread advances FMA_CHAINS independent chains a <- a * m + c for
// iters rounds; the sum goes to out only if it is negative (it never is:
// every chain stays near 1), so the chains are live but nothing is written.
__global__ void __launch_bounds__(FMA_THREADS) k_fma_f64(int iters, double m, double c, double* out) {
  double a[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = fma(a[k], m, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) s += a[k];
  if (s < 0.0) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(FMA_THREADS) k_fma_f32x2(int iters, float m, float c, float* out) {
  float2 a[FMA_CHAINS];
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) a[k] = make_float2(1.f + 1e-3f * threadIdx.x, 1.f + 1e-3f * k);
  const float2 mm = make_float2(m, m), cc = make_float2(c, c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = __ffma2_rn(a[k], mm, cc);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) s += a[k].x + a[k].y;
  if (s < 0.f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int scabem_peak_fma(int32_t prec, double* tflops, void* stream) {
  if (!tflops || (prec != SCABEM_C64 && prec != SCABEM_C128)) {
    set_error("scabem_peak_fma: bad argument");
    return SCABEM_E_ARG;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = 8 * nsm;  // 8 CTAs of 8 warps per SM: 64 warps, every scheduler busy
  const int iters = prec == SCABEM_C128 ? 4096 : 65536;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SCABEM_OK;
  float ms = 0.f;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "cudaEventCreate");
      break;
    }
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms the clocks up
      if (cudaEventRecord(e0, s) != cudaSuccess) break;
      if (prec == SCABEM_C128)
        k_fma_f64<<<blocks, FMA_THREADS, 0, s>>>(iters, 0.9999999, 1e-7, out);
      else
        k_fma_f32x2<<<blocks, FMA_THREADS, 0, s>>>(iters, 0.9999f, 1e-4f, reinterpret_cast<float*>(out));
      cudaEventRecord(e1, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_fail(e, "scabem_peak_fma");
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return rc;
  // FP64: one FMA (2 flops) per chain step; FP32x2: two FMAs (4 flops)
  const double flops_per_step = prec == SCABEM_C128 ? 2.0 : 4.0;
  const double flops = flops_per_step * FMA_CHAINS * (double)iters * blocks * FMA_THREADS;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SCABEM_OK;
}
