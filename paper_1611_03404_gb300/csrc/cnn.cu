// Learned warm start: a small CNN from a source's 5-band 32 x 32 patch to initial variational
// parameters, trained and run by the kernels below (BF16 operands, FP32 accumulation, FP32
// master weights).  Newton remains the solver: the network only supplies its starting point.
//
// Network (NHWC activations, BF16):
//   x [B,32,32,5] -conv3x3 s1-> a1 [B,32,32,32] -conv3x3 s2-> a2 [B,16,16,64]
//     -conv3x3 s2-> a3 [B,8,8,64] -conv3x3 s2-> a4 [B,4,4,64] = [B,1024]
//     -fc-> a5 [B,256] -fc-> y [B,27] (FP32); ReLU after every layer but the last; padding 1.
// Parameters, one FP32 vector (and its BF16 copy), in this order:
//   W1 [32][3][3][5], b1 [32], W2 [64][3][3][32], b2, W3 [64][3][3][64], b3, W4 [64][3][3][64],
//   b4, W5 [256][1024], b5 [256], W6 [27][256], b6 [27].
//
// Every convolution and product runs through one implicit-GEMM kernel: 64 x 64 output tiles,
// k-steps of 32, four warps of 32 x 32 issuing mma.sync m16n8k16 (BF16 in, FP32 accumulate).
// The operand loaders gather straight from the NHWC tensors (im2col on the fly), so forward,
// input-gradient and weight-gradient passes differ only in their gather and epilogue.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "celeste_internal.cuh"
#include "cnn_tc.h"
#include "problem.h"

namespace celeste {
namespace cnn {

using bf16 = __nv_bfloat16;

constexpr int IMG = 32, CIN = 5, NOUT = 27;
constexpr int C1 = 32, C2 = 64, C3 = 64, C4 = 64, F5 = 256, FLAT = 4 * 4 * C4;

struct Offsets {
  int64_t w1, b1, w2, b2, w3, b3, w4, b4, w5, b5, w6, b6, total;
};
__host__ __device__ constexpr Offsets offsets() {
  Offsets o{};
  int64_t p = 0;
  o.w1 = p; p += (int64_t)C1 * 9 * CIN;
  o.b1 = p; p += C1;
  o.w2 = p; p += (int64_t)C2 * 9 * C1;
  o.b2 = p; p += C2;
  o.w3 = p; p += (int64_t)C3 * 9 * C2;
  o.b3 = p; p += C3;
  o.w4 = p; p += (int64_t)C4 * 9 * C3;
  o.b4 = p; p += C4;
  o.w5 = p; p += (int64_t)F5 * FLAT;
  o.b5 = p; p += F5;
  o.w6 = p; p += (int64_t)NOUT * F5;
  o.b6 = p; p += NOUT;
  o.total = p;
  return o;
}

// Activation and gradient buffers for a batch of B (BF16 elements, each buffer 256-byte aligned).
struct Ws {
  bf16 *a1, *a2, *a3, *a4, *a5;   // activations after ReLU
  bf16 *d1, *d2, *d3, *d4, *d5;   // gradients w.r.t. those activations' pre-ReLU values
  size_t bytes;
};
inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
inline void ws_sizes(int B, size_t (&sz)[5]) {
  sz[0] = (size_t)B * IMG * IMG * C1;
  sz[1] = (size_t)B * 16 * 16 * C2;
  sz[2] = (size_t)B * 8 * 8 * C3;
  sz[3] = (size_t)B * FLAT;
  sz[4] = (size_t)B * F5;
}
inline size_t ws_bytes(int B) {
  size_t sz[5], off = 0;
  ws_sizes(B, sz);
  for (int i = 0; i < 5; ++i) off += 2 * al256(sz[i] * sizeof(bf16));
  return off;
}
inline Ws ws_layout(char* base, int B) {
  size_t sz[5];
  ws_sizes(B, sz);
  Ws w{};
  bf16** act[5] = {&w.a1, &w.a2, &w.a3, &w.a4, &w.a5};
  bf16** grd[5] = {&w.d1, &w.d2, &w.d3, &w.d4, &w.d5};
  size_t off = 0;
  for (int i = 0; i < 5; ++i) {
    *act[i] = reinterpret_cast<bf16*>(base + off);
    off += al256(sz[i] * sizeof(bf16));
    *grd[i] = reinterpret_cast<bf16*>(base + off);
    off += al256(sz[i] * sizeof(bf16));
  }
  w.bytes = off;
  return w;
}

__device__ __forceinline__ bf16 bzero() { return __float2bfloat16(0.f); }

// ------------------------------------------------------------------------------ GEMM core
constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M x N] = sum_k A(m, k) B(k, n) over k in this block's K chunk (blockIdx.z), handed to
// op.store(m, n, value).  op.a / op.b return BF16 operands (zero outside the tensors).
template <class Op>
__global__ void __launch_bounds__(128) gemm_kernel(Op op, int M, int N, int K, int k_chunk) {
  __shared__ __align__(16) bf16 As[BM][LDS];
  __shared__ __align__(16) bf16 Bs[BN][LDS];   // B transposed: Bs[n][k]
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32, g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      const int r = e / BK, c = e % BK, k = k0 + c;
      As[r][c] = (m0 + r < M && k < ke) ? op.a(m0 + r, k) : bzero();
      Bs[r][c] = (n0 + r < N && k < ke) ? op.b(k, n0 + r) : bzero();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
        a[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
        a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + g;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t + 8]);
#pragma unroll
        for (int i = 0; i < 2; ++i) mma16816(acc[i][j], a[i], b0, b1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int m = m0 + wm + 16 * i + g + (e >> 1) * 8, n = n0 + wn + 8 * j + 2 * t + (e & 1);
        if (m < M && n < N) op.store(m, n, acc[i][j][e]);
      }
}

template <class Op>
cudaError_t gemm(const Op& op, int M, int N, int K, int splits, cudaStream_t st) {
  splits = std::max(1, std::min(splits, (K + BK - 1) / BK));
  int chunk = (K + splits - 1) / splits;
  chunk = (chunk + BK - 1) / BK * BK;
  splits = (K + chunk - 1) / chunk;
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
  gemm_kernel<Op><<<grid, 128, 0, st>>>(op, M, N, K, chunk);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ convolution ops
struct ConvGeom {
  int B, H, W, Cin, OH, OW, Cout, stride;
};

// out[b, oh, ow, co] = relu(bias[co] + sum_{kh, kw, ci} in[b, oh s + kh - 1, ow s + kw - 1, ci] W[co, kh, kw, ci])
struct ConvFwd {
  ConvGeom g;
  const bf16* in;
  const bf16* w;
  const float* bias;
  bf16* out;
  __device__ bf16 a(int m, int k) const {
    const int ow = m % g.OW, r = m / g.OW, oh = r % g.OH, b = r / g.OH;
    const int ci = k % g.Cin, kk = k / g.Cin, kh = kk / 3, kw = kk % 3;
    const int ih = oh * g.stride + kh - 1, iw = ow * g.stride + kw - 1;
    if (ih < 0 || ih >= g.H || iw < 0 || iw >= g.W) return bzero();
    return in[(((size_t)b * g.H + ih) * g.W + iw) * g.Cin + ci];
  }
  __device__ bf16 b(int k, int n) const { return w[(size_t)n * 9 * g.Cin + k]; }
  __device__ void store(int m, int n, float v) const {
    out[(size_t)m * g.Cout + n] = __float2bfloat16(fmaxf(v + bias[n], 0.f));
  }
};

// din[b, ih, iw, ci] = [in > 0] sum_{co, kh, kw} dout[b, oh, ow, co] W[co, kh, kw, ci],
// ih = oh s + kh - 1 (the mask turns the gradient w.r.t. the input activation into the gradient
// w.r.t. the previous layer's pre-ReLU value)
struct ConvDgrad {
  ConvGeom g;
  const bf16* dout;
  const bf16* w;
  const bf16* in;
  bf16* din;
  __device__ bf16 a(int m, int k) const {
    const int iw = m % g.W, r = m / g.W, ih = r % g.H, b = r / g.H;
    const int co = k % g.Cout, kk = k / g.Cout, kh = kk / 3, kw = kk % 3;
    const int th = ih + 1 - kh, tw = iw + 1 - kw;
    if (th < 0 || tw < 0 || th % g.stride || tw % g.stride) return bzero();
    const int oh = th / g.stride, ow = tw / g.stride;
    if (oh >= g.OH || ow >= g.OW) return bzero();
    return dout[(((size_t)b * g.OH + oh) * g.OW + ow) * g.Cout + co];
  }
  __device__ bf16 b(int k, int n) const {
    const int co = k % g.Cout, kk = k / g.Cout;
    return w[((size_t)co * 9 + kk) * g.Cin + n];
  }
  __device__ void store(int m, int n, float v) const {
    const size_t i = (size_t)m * g.Cin + n;
    din[i] = __float2bfloat16(__bfloat162float(in[i]) > 0.f ? v : 0.f);
  }
};

// dW[co, kh, kw, ci] += sum_{b, oh, ow} dout[b, oh, ow, co] in[b, oh s + kh - 1, ow s + kw - 1, ci]
struct ConvWgrad {
  ConvGeom g;
  const bf16* dout;
  const bf16* in;
  float* dw;
  __device__ bf16 a(int m, int k) const { return dout[(size_t)k * g.Cout + m]; }
  __device__ bf16 b(int k, int n) const {
    const int ow = k % g.OW, r = k / g.OW, oh = r % g.OH, b = r / g.OH;
    const int ci = n % g.Cin, kk = n / g.Cin, kh = kk / 3, kw = kk % 3;
    const int ih = oh * g.stride + kh - 1, iw = ow * g.stride + kw - 1;
    if (ih < 0 || ih >= g.H || iw < 0 || iw >= g.W) return bzero();
    return in[(((size_t)b * g.H + ih) * g.W + iw) * g.Cin + ci];
  }
  __device__ void store(int m, int n, float v) const { atomicAdd(dw + (size_t)m * 9 * g.Cin + n, v); }
};

// ------------------------------------------------------------------------------ dense ops
// y[b, o] = act(bias[o] + sum_i x[b, i] W[o, i]); the last layer writes FP32, optionally mapped
// to parameter space as y * scale[o] + shift[o].
struct FcFwd {
  int Nin, Nout;
  const bf16* x;
  const bf16* w;
  const float* bias;
  bf16* out_bf;
  float* out_f;
  const float* scale;
  const float* shift;
  __device__ bf16 a(int m, int k) const { return x[(size_t)m * Nin + k]; }
  __device__ bf16 b(int k, int n) const { return w[(size_t)n * Nin + k]; }
  __device__ void store(int m, int n, float v) const {
    v += bias[n];
    if (out_bf) {
      out_bf[(size_t)m * Nout + n] = __float2bfloat16(fmaxf(v, 0.f));
    } else {
      if (scale) v = v * scale[n] + shift[n];
      out_f[(size_t)m * Nout + n] = v;
    }
  }
};

// dx[b, i] = [x > 0] sum_o dy[b, o] W[o, i]   (dy BF16, or FP32 for the last layer)
template <class T>
struct FcDgrad {
  int Nin, Nout;
  const T* dy;
  const bf16* w;
  const bf16* x;
  bf16* dx;
  __device__ bf16 a(int m, int k) const { return __float2bfloat16((float)dy[(size_t)m * Nout + k]); }
  __device__ bf16 b(int k, int n) const { return w[(size_t)k * Nin + n]; }
  __device__ void store(int m, int n, float v) const {
    const size_t i = (size_t)m * Nin + n;
    dx[i] = __float2bfloat16(__bfloat162float(x[i]) > 0.f ? v : 0.f);
  }
};

// dW[o, i] += sum_b dy[b, o] x[b, i]
template <class T>
struct FcWgrad {
  int Nin, Nout;
  const T* dy;
  const bf16* x;
  float* dw;
  __device__ bf16 a(int m, int k) const { return __float2bfloat16((float)dy[(size_t)k * Nout + m]); }
  __device__ bf16 b(int k, int n) const { return x[(size_t)k * Nin + n]; }
  __device__ void store(int m, int n, float v) const { atomicAdd(dw + (size_t)m * Nin + n, v); }
};

// db[c] += sum over rows of g[r, c]
template <class T>
__global__ void bias_grad_kernel(const T* g, int64_t rows, int C, float* db) {
  const int c = threadIdx.x % C, lanes = blockDim.x / C;
  if ((int)threadIdx.x >= lanes * C) return;
  float s = 0.f;
  for (int64_t r = (int64_t)blockIdx.x * lanes + threadIdx.x / C; r < rows; r += (int64_t)gridDim.x * lanes)
    s += (float)g[r * C + c];
  atomicAdd(db + c, s);
}

template <class T>
cudaError_t bias_grad(const T* g, int64_t rows, int C, float* db, cudaStream_t st) {
  const int lanes = std::max(1, 256 / C);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + lanes - 1) / lanes, 1024));
  bias_grad_kernel<T><<<blocks, lanes * C, 0, st>>>(g, rows, C, db);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------ small kernels
// Counter-based standard normal (SplitMix64 of seed and index, Box-Muller).
__device__ inline uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ inline float normal_at(uint64_t seed, int64_t i) {
  const uint64_t h1 = splitmix64(seed * 0x100000001B3ULL + 2 * (uint64_t)i);
  const uint64_t h2 = splitmix64(seed * 0x100000001B3ULL + 2 * (uint64_t)i + 1);
  const float u1 = ((h1 >> 40) + 0.5f) * (1.0f / 16777216.0f), u2 = (h2 >> 40) * (1.0f / 16777216.0f);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// He-normal weights (std sqrt(2 / fan_in)), zero biases; the last layer scaled by 0.1.
__global__ void init_kernel(float* p, bf16* pb, uint64_t seed) {
  constexpr Offsets o = offsets();
  const int64_t n = o.total;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float fan = 0.f, scale = 1.f;
    if (i < o.b1) fan = 9 * CIN;
    else if (i >= o.w2 && i < o.b2) fan = 9 * C1;
    else if (i >= o.w3 && i < o.b3) fan = 9 * C2;
    else if (i >= o.w4 && i < o.b4) fan = 9 * C3;
    else if (i >= o.w5 && i < o.b5) fan = FLAT;
    else if (i >= o.w6 && i < o.b6) { fan = F5; scale = 0.1f; }
    const float v = fan > 0.f ? scale * sqrtf(2.f / fan) * normal_at(seed, i) : 0.f;
    p[i] = v;
    pb[i] = __float2bfloat16(v);
  }
}

// loss += sum_{b, j} w_j (y - t)^2 / (B * 27);  dy = 2 w_j (y - t) / (B * 27)
__global__ void mse_kernel(const float* y, const float* t, const float* w, int n, float* dy, double* loss) {
  __shared__ float red[8];
  const float inv = 1.f / (float)n;
  float s = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float wj = w ? w[i % NOUT] : 1.f, d = y[i] - t[i];
    s += wj * d * d * inv;
    dy[i] = 2.f * wj * d * inv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    atomicAdd(loss, (double)v);
  }
}

// AdamW with bias correction; the BF16 copy follows the FP32 master weights.
__global__ void adamw_kernel(float* p, bf16* pb, float* m, float* v, const float* g, int64_t n, float lr, float b1,
                             float b2, float eps, float wd, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] * (1.f - lr * wd) - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
  }
}

// x[s, i, j, b] = asinh((pixel - sky) / sqrt(sky)) on the 32 x 32 window whose pixel (16, 16) is
// the source's patch centre, taken from the first exposure of band b that holds the source (zero
// where the band is missing or the window leaves the image).
__global__ void extract_patches_kernel(ProblemDev P, bf16* x) {
  const int s = blockIdx.x;
  int img[5] = {-1, -1, -1, -1, -1}, cx[5], cy[5];
  for (int q = P.src_patch[s]; q < P.src_patch[s + 1]; ++q) {
    const PatchDev pt = P.patches[q];
    const ImageDev& im = P.images[pt.image];
    if (img[im.band] >= 0) continue;
    img[im.band] = pt.image;
    const double u = P.u0[2 * s], v = P.u0[2 * s + 1];
    cx[im.band] = (int)floor(im.A[0] * u + im.A[1] * v + im.o[0] + 0.5);
    cy[im.band] = (int)floor(im.A[2] * u + im.A[3] * v + im.o[1] + 0.5);
  }
  for (int e = threadIdx.x; e < IMG * IMG * CIN; e += blockDim.x) {
    const int b = e % CIN, j = (e / CIN) % IMG, i = e / (CIN * IMG);
    float val = 0.f;
    if (img[b] >= 0) {
      const ImageDev& im = P.images[img[b]];
      const int r = cy[b] - 16 + i, c = cx[b] - 16 + j;
      if (r >= 0 && r < im.H && c >= 0 && c < im.W)
        val = asinhf((im.pixels[(size_t)r * im.W + c] - im.sky) * rsqrtf(im.sky));
    }
    x[(size_t)s * IMG * IMG * CIN + e] = __float2bfloat16(val);
  }
}

}  // namespace cnn
}  // namespace celeste

using namespace celeste;
using namespace celeste::cnn;

extern "C" int64_t celeste_cnn_param_count(void) { return offsets().total; }

extern "C" size_t celeste_cnn_workspace_bytes(int batch) {
  if (batch <= 0) return 0;
  return ws_bytes(batch);
}

extern "C" int celeste_cnn_init(float* params, uint16_t* params_bf16, uint64_t seed, celeste_stream_t stream) {
  if (!params || !params_bf16) return fail(CELESTE_ERR_INVALID_ARG, "null parameter buffer");
  init_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(params, reinterpret_cast<bf16*>(params_bf16), seed);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CELESTE_OK : cuda_fail(e, "cnn init");
}

static int check_ws(int batch, const void* ws, size_t bytes) {
  if (batch <= 0) return fail(CELESTE_ERR_INVALID_ARG, "batch must be > 0");
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return fail(CELESTE_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < ws_bytes(batch)) return fail(CELESTE_ERR_WORKSPACE, "workspace needs %zu bytes", ws_bytes(batch));
  return CELESTE_OK;
}

// Error word of the tensor-core forward path (a bounded wait that ran out).
static __device__ int g_cnn_tc_err;

extern "C" int celeste_cnn_status(void) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_cnn_tc_err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cnn status");
  if (!v) return CELESTE_OK;
  const int zero = 0;
  cudaMemcpyToSymbol(g_cnn_tc_err, &zero, sizeof(int));
  return fail(CELESTE_ERR_TIMEOUT, "a tensor-core product of the network did not complete in time");
}

extern "C" int celeste_cnn_forward(const float* params, const uint16_t* params_bf16, const uint16_t* x, int batch,
                                   const float* out_scale, const float* out_shift, float* y, void* ws,
                                   size_t ws_bytes, celeste_stream_t stream) {
  return celeste_cnn_forward_ex(params, params_bf16, x, batch, out_scale, out_shift, y, ws, ws_bytes,
                                CELESTE_CNN_TCGEN05, stream);
}

extern "C" int celeste_cnn_forward_ex(const float* params, const uint16_t* params_bf16, const uint16_t* x, int batch,
                                      const float* out_scale, const float* out_shift, float* y, void* ws,
                                      size_t ws_bytes, int engine, celeste_stream_t stream) {
  if (!params || !params_bf16 || !x || !y) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  if ((out_scale == nullptr) != (out_shift == nullptr)) return fail(CELESTE_ERR_INVALID_ARG, "scale and shift go together");
  if (engine != CELESTE_CNN_MMA_SYNC && engine != CELESTE_CNN_TCGEN05)
    return fail(CELESTE_ERR_INVALID_ARG, "engine must be CELESTE_CNN_MMA_SYNC or CELESTE_CNN_TCGEN05");
  int rc = check_ws(batch, ws, ws_bytes);
  if (rc != CELESTE_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  constexpr Offsets o = offsets();
  const bf16* pb = reinterpret_cast<const bf16*>(params_bf16);
  const Ws w = ws_layout(static_cast<char*>(ws), batch);
  const int B = batch;
  const bf16* xin = reinterpret_cast<const bf16*>(x);
  cudaError_t e;
  ConvGeom g1{B, 32, 32, CIN, 32, 32, C1, 1}, g2{B, 32, 32, C1, 16, 16, C2, 2};
  ConvGeom g3{B, 16, 16, C2, 8, 8, C3, 2}, g4{B, 8, 8, C3, 4, 4, C4, 2};
  if (engine == CELESTE_CNN_TCGEN05) {
    int* err = nullptr;
    if ((e = cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_cnn_tc_err)) != cudaSuccess)
      return cuda_fail(e, "cnn error word");
    auto conv = [&](const ConvGeom& g, const bf16* in, int64_t wo, int64_t bo, bf16* out) {
      cnn_tc::Args a{};
      a.M = g.B * g.OH * g.OW;
      a.N = g.Cout;
      a.K = 9 * g.Cin;
      a.conv = 1;
      a.B = g.B, a.H = g.H, a.W = g.W, a.Cin = g.Cin, a.OH = g.OH, a.OW = g.OW, a.stride = g.stride;
      a.in = in, a.w = pb + wo, a.bias = params + bo, a.out = out, a.err = err;
      return tc_gemm_forward(a, st);
    };
    auto fc = [&](int nin, int nout, const bf16* in, int64_t wo, int64_t bo, bf16* out, float* outf) {
      cnn_tc::Args a{};
      a.M = B, a.N = nout, a.K = nin, a.conv = 0;
      a.in = in, a.w = pb + wo, a.bias = params + bo, a.out = out, a.out_f = outf, a.scale = out_scale,
      a.shift = out_shift, a.err = err;
      return tc_gemm_forward(a, st);
    };
    if ((e = conv(g1, xin, o.w1, o.b1, w.a1)) != cudaSuccess || (e = conv(g2, w.a1, o.w2, o.b2, w.a2)) != cudaSuccess ||
        (e = conv(g3, w.a2, o.w3, o.b3, w.a3)) != cudaSuccess || (e = conv(g4, w.a3, o.w4, o.b4, w.a4)) != cudaSuccess ||
        (e = fc(FLAT, F5, w.a4, o.w5, o.b5, w.a5, nullptr)) != cudaSuccess ||
        (e = fc(F5, NOUT, w.a5, o.w6, o.b6, nullptr, y)) != cudaSuccess)
      return cuda_fail(e, "cnn forward (tensor cores)");
    return CELESTE_OK;
  }
  if ((e = gemm(ConvFwd{g1, xin, pb + o.w1, params + o.b1, w.a1}, B * 1024, C1, 9 * CIN, 1, st)) != cudaSuccess ||
      (e = gemm(ConvFwd{g2, w.a1, pb + o.w2, params + o.b2, w.a2}, B * 256, C2, 9 * C1, 1, st)) != cudaSuccess ||
      (e = gemm(ConvFwd{g3, w.a2, pb + o.w3, params + o.b3, w.a3}, B * 64, C3, 9 * C2, 1, st)) != cudaSuccess ||
      (e = gemm(ConvFwd{g4, w.a3, pb + o.w4, params + o.b4, w.a4}, B * 16, C4, 9 * C3, 1, st)) != cudaSuccess ||
      (e = gemm(FcFwd{FLAT, F5, w.a4, pb + o.w5, params + o.b5, w.a5, nullptr, nullptr, nullptr}, B, F5, FLAT, 1, st)) !=
          cudaSuccess ||
      (e = gemm(FcFwd{F5, NOUT, w.a5, pb + o.w6, params + o.b6, nullptr, y, out_scale, out_shift}, B, NOUT, F5, 1, st)) !=
          cudaSuccess)
    return cuda_fail(e, "cnn forward");
  return CELESTE_OK;
}

extern "C" int celeste_cnn_backward(const float* params, const uint16_t* params_bf16, const uint16_t* x, const float* dy,
                                    int batch, float* grad, void* ws, size_t ws_bytes, celeste_stream_t stream) {
  if (!params || !params_bf16 || !x || !dy || !grad) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  int rc = check_ws(batch, ws, ws_bytes);
  if (rc != CELESTE_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  constexpr Offsets o = offsets();
  const bf16* pb = reinterpret_cast<const bf16*>(params_bf16);
  const Ws w = ws_layout(static_cast<char*>(ws), batch);
  const int B = batch;
  const bf16* xin = reinterpret_cast<const bf16*>(x);
  ConvGeom g1{B, 32, 32, CIN, 32, 32, C1, 1}, g2{B, 32, 32, C1, 16, 16, C2, 2};
  ConvGeom g3{B, 16, 16, C2, 8, 8, C3, 2}, g4{B, 8, 8, C3, 4, 4, C4, 2};
  cudaError_t e;
  auto splits_for = [](int64_t K) { return (int)std::max<int64_t>(1, std::min<int64_t>(256, K / 1024)); };
  // fc2
  if ((e = gemm(FcWgrad<float>{F5, NOUT, dy, w.a5, grad + o.w6}, NOUT, F5, B, splits_for(B), st)) != cudaSuccess ||
      (e = bias_grad(dy, B, NOUT, grad + o.b6, st)) != cudaSuccess ||
      (e = gemm(FcDgrad<float>{F5, NOUT, dy, pb + o.w6, w.a5, w.d5}, B, F5, NOUT, 1, st)) != cudaSuccess)
    return cuda_fail(e, "cnn backward fc2");
  // fc1
  if ((e = gemm(FcWgrad<bf16>{FLAT, F5, w.d5, w.a4, grad + o.w5}, F5, FLAT, B, splits_for(B), st)) != cudaSuccess ||
      (e = bias_grad(w.d5, B, F5, grad + o.b5, st)) != cudaSuccess ||
      (e = gemm(FcDgrad<bf16>{FLAT, F5, w.d5, pb + o.w5, w.a4, w.d4}, B, FLAT, F5, 1, st)) != cudaSuccess)
    return cuda_fail(e, "cnn backward fc1");
  // conv4 .. conv1
  struct L {
    ConvGeom g;
    const bf16* in;
    const bf16* d;
    bf16* din;
    int64_t w, b;
  } layers[4] = {{g4, w.a3, w.d4, w.d3, o.w4, o.b4},
                 {g3, w.a2, w.d3, w.d2, o.w3, o.b3},
                 {g2, w.a1, w.d2, w.d1, o.w2, o.b2},
                 {g1, xin, w.d1, nullptr, o.w1, o.b1}};
  for (const L& l : layers) {
    const int64_t Kw = (int64_t)l.g.B * l.g.OH * l.g.OW;
    if ((e = gemm(ConvWgrad{l.g, l.d, l.in, grad + l.w}, l.g.Cout, 9 * l.g.Cin, (int)Kw, splits_for(Kw), st)) !=
            cudaSuccess ||
        (e = bias_grad(l.d, Kw, l.g.Cout, grad + l.b, st)) != cudaSuccess)
      return cuda_fail(e, "cnn backward weights");
    if (l.din &&
        (e = gemm(ConvDgrad{l.g, l.d, pb + l.w, l.in, l.din}, l.g.B * l.g.H * l.g.W, l.g.Cin, 9 * l.g.Cout, 1, st)) !=
            cudaSuccess)
      return cuda_fail(e, "cnn backward data");
  }
  return CELESTE_OK;
}

extern "C" int celeste_cnn_mse(const float* y, const float* target, const float* weight, int batch, float* dy,
                               double* loss, celeste_stream_t stream) {
  if (!y || !target || !dy || !loss || batch <= 0) return fail(CELESTE_ERR_INVALID_ARG, "null argument or empty batch");
  const int n = batch * NOUT;
  mse_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y, target, weight, n, dy, loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CELESTE_OK : cuda_fail(e, "cnn mse");
}

extern "C" int celeste_cnn_adamw(float* params, uint16_t* params_bf16, float* m, float* v, const float* grad, float lr,
                                 float beta1, float beta2, float eps, float weight_decay, int step,
                                 celeste_stream_t stream) {
  if (!params || !params_bf16 || !m || !v || !grad || step < 1) return fail(CELESTE_ERR_INVALID_ARG, "bad argument");
  const int64_t n = offsets().total;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adamw_kernel<<<256, 256, 0, (cudaStream_t)stream>>>(params, reinterpret_cast<bf16*>(params_bf16), m, v, grad, n, lr,
                                                      beta1, beta2, eps, weight_decay, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CELESTE_OK : cuda_fail(e, "cnn adamw");
}

extern "C" int celeste_extract_patches(celeste_problem* p, uint16_t* x, celeste_stream_t stream) {
  if (!p || !x) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "bind the problem first");
  extract_patches_kernel<<<p->S, 256, 0, (cudaStream_t)stream>>>(p->dev, reinterpret_cast<bf16*>(x));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CELESTE_OK : cuda_fail(e, "extract patches");
}
