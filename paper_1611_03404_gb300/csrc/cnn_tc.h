// Tensor-core (tcgen05) forward products of the warm-start network: shared between the network's
// entry points (cnn.cu) and the kernel (cnn_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace celeste {
namespace cnn_tc {

// D[M x N] = A[M x K] B[K x N]: A the layer input (im2col of a 3x3, padding-1 convolution over an
// NHWC tensor when conv is set), B the weights [N][K] (K-major), bias [N]; D stored as BF16 after
// ReLU into out [M][N], or as FP32 into out_f [M][N] (times scale plus shift when scale is set).
struct Args {
  int M, N, K;
  int conv;
  int B, H, W, Cin, OH, OW, stride;
  const __nv_bfloat16* in;
  const __nv_bfloat16* w;
  const float* bias;
  __nv_bfloat16* out;
  float* out_f;
  const float* scale;
  const float* shift;
  int* err;                      // error word, set when a bounded wait runs out
};

}  // namespace cnn_tc

cudaError_t tc_gemm_forward(const cnn_tc::Args& a, cudaStream_t st);

}  // namespace celeste
