// Measured throughput of the arithmetic pipes the hot path is bound by, for its rooflines: FP32 FMA
// (the pixel kernels), the special-function unit's base-2 exponential (45 per pixel evaluation) and
// FP64 FMA (the trust-region step).  Not part of the method; the benchmark reports the kernels'
// achieved rates against these.
//
// Each kernel runs independent dependency chains (8 per thread, 1024 threads per SM) so that the
// pipe, not the latency of one chain, sets the rate; the grid is a multiple of the SM count.  The
// chains' values stay bounded (a contraction for the FMAs, x <- 2^-x for the exponential) and are
// stored, so nothing is optimised away.
#include <algorithm>

#include "celeste_internal.cuh"
#include "problem.h"

namespace celeste {

constexpr int PK_CHAINS = 8;
constexpr int PK_THREADS = 256;
constexpr int PK_CTAS_PER_SM = 4;

__global__ void __launch_bounds__(PK_THREADS) peak_ffma_kernel(float* out, int iters, float a, float b) {
  float x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same chains two lanes wide (Blackwell's packed FP32 multiply-add): PK_CHAINS / 2 packed
// chains do PK_CHAINS multiply-adds per step, the count the FP32 kernel above does.
__global__ void __launch_bounds__(PK_THREADS) peak_ffma2_kernel(float* out, int iters, float a, float b) {
  float2 x[PK_CHAINS / 2];
#pragma unroll
  for (int c = 0; c < PK_CHAINS / 2; ++c) x[c] = make_float2(1e-3f * (threadIdx.x + 2 * c), 1e-3f * (threadIdx.x + 2 * c + 1));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PK_CHAINS / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CHAINS / 2; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(PK_THREADS) peak_ex2_kernel(float* out, int iters) {
  float x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PK_CHAINS; ++c) x[c] = ex2_approx(-x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) peak_dfma_kernel(double* out, int iters, double a, double b) {
  double x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_measure_peak(int kind, double* ops_per_s, double* seconds, celeste_stream_t stream) {
  if (!ops_per_s || kind < 0 || kind > 3) return fail(CELESTE_ERR_INVALID_ARG, "kind must be 0, 1, 2 or 3");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  const int grid = n_sm * PK_CTAS_PER_SM;
  const size_t n_out = (size_t)grid * PK_THREADS;
  // the chains' results (a few MB); a measurement utility outside the evaluation path, so it
  // allocates and frees its own buffer
  void* buf = nullptr;
  if ((e = cudaMalloc(&buf, n_out * sizeof(double))) != cudaSuccess) return cuda_fail(e, "peak buffer");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  int rc = CELESTE_OK;
  float ms = 0.f;
  // pipe operations per inner iteration of one thread
  const double per_iter = 16.0 * PK_CHAINS;
  int iters = kind == 2 ? 64 : 1024;
  if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
    rc = cuda_fail(e, "events");
  } else {
    auto launch = [&](int it) {
      if (kind == 0)
        peak_ffma_kernel<<<grid, PK_THREADS, 0, st>>>(static_cast<float*>(buf), it, 0.9999f, 1e-4f);
      else if (kind == 1)
        peak_ex2_kernel<<<grid, PK_THREADS, 0, st>>>(static_cast<float*>(buf), it);
      else if (kind == 3)
        peak_ffma2_kernel<<<grid, PK_THREADS, 0, st>>>(static_cast<float*>(buf), it, 0.9999f, 1e-4f);
      else
        peak_dfma_kernel<<<grid, PK_THREADS, 0, st>>>(static_cast<double*>(buf), it, 0.9999, 1e-4);
    };
    launch(iters);   // warm-up
    // grow the launch until it lasts ~50 ms, then time the best of three
    for (int grow = 0; grow < 12 && rc == CELESTE_OK; ++grow) {
      cudaEventRecord(t0, st);
      launch(iters);
      cudaEventRecord(t1, st);
      if ((e = cudaEventSynchronize(t1)) != cudaSuccess) {
        rc = cuda_fail(e, "peak kernel");
        break;
      }
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms >= 25.f) break;
      iters *= 2;
    }
    float best = 1e30f;
    for (int r = 0; r < 3 && rc == CELESTE_OK; ++r) {
      cudaEventRecord(t0, st);
      launch(iters);
      cudaEventRecord(t1, st);
      if ((e = cudaEventSynchronize(t1)) != cudaSuccess) {
        rc = cuda_fail(e, "peak kernel");
        break;
      }
      cudaEventElapsedTime(&ms, t0, t1);
      best = std::min(best, ms);
    }
    if (rc == CELESTE_OK) {
      const double ops = (double)n_out * iters * per_iter * (kind == 1 ? 1.0 : 2.0);   // FMA = 2 flops
      *ops_per_s = ops / (best * 1e-3);
      if (seconds) *seconds = best * 1e-3;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(buf);
  return rc;
}
