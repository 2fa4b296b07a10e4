// Forward layers of the warm-start network on the fifth-generation tensor cores (tcgen05): the
// convolution and dense products as GEMMs D[M x N] = A[M x K] B[K x N] with BF16 operands and an
// FP32 accumulator in tensor memory.
//
// One CTA (4 warps) per 128-row tile of D and N_TILE columns.  A is the layer input gathered on the
// fly (im2col for the convolutions: row m = output pixel, k = (kh * 3 + kw) * Cin + ci), B the
// weights [N][K]; both K-major.  Per K-step of 64 the threads write A (128 x 64) and B (N_TILE x 64)
// into shared memory in the 128-byte-swizzled layout (8-row atoms of 1024 bytes, 16-byte chunk c of
// row r at chunk c ^ (r % 8)), two stages deep; thread 0 issues four tcgen05.mma (K = 16 each) and
// a tcgen05.commit that arrives on the stage's mbarrier once the products have read the stage.
// After the last step each warp reads its 32 accumulator lanes (tcgen05.ld 32x32b), adds the bias,
// applies ReLU (or the last layer's scale and shift) and stores.
//
// Tensor memory: N_TILE columns per CTA (32, 64 or 128), allocated by warp 0 and freed before the
// CTA exits; the dynamic shared memory per CTA (>= 40 KB) keeps at most 5 CTAs on an SM, so the
// columns in use never exceed the SM's 512 and an allocation never waits on another CTA.  Every
// wait on an mbarrier is bounded; on a timeout the CTA records it in the error word, waits once
// more for the products in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "celeste_internal.cuh"
#include "cnn_tc.h"
#include "problem.h"

namespace celeste {
namespace cnn_tc {

using bf16 = __nv_bfloat16;

constexpr int TM = 128;        // rows of D per CTA (the MMA's M)
constexpr int TK = 64;         // K per stage: one 128-byte row per operand row
constexpr int STAGES = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand in the 128-byte-swizzled layout, 8-row atoms
// 1024 bytes apart (stride byte offset), start address in 16-byte units, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset: next 8-row atom
  d |= (uint64_t)1u << 46;                          // descriptor version
  d |= (uint64_t)2u << 61;                          // swizzle: 128 bytes
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128, N.
__device__ __forceinline__ uint32_t instr_desc_bf16(int n) {
  uint32_t d = 0;
  d |= 1u << 4;                      // D format: F32
  d |= 1u << 7;                      // A format: BF16
  d |= 1u << 10;                     // B format: BF16
  d |= (uint32_t)(n >> 3) << 17;     // N / 8
  d |= (uint32_t)(TM >> 4) << 24;    // M / 16
  return d;
}

__device__ __forceinline__ void mma_bf16_tmem(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Eight consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk c of row r in a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// Eight consecutive K entries (k, ..., k + 7) of row m of A, zero outside the operand.
__device__ __forceinline__ uint4 load_a(const Args& a, int m, int k) {
  uint4 z = make_uint4(0u, 0u, 0u, 0u);
  if (m >= a.M || k >= a.K) return z;
  if (!a.conv) return *reinterpret_cast<const uint4*>(a.in + (size_t)m * a.K + k);
  const int ow = m % a.OW, r = m / a.OW, oh = r % a.OH, b = r / a.OH;
  if ((a.Cin & 7) == 0) {
    // one tap, 8 consecutive channels: one 16-byte load
    const int ci = k % a.Cin, tap = k / a.Cin, kh = tap / 3, kw = tap % 3;
    const int ih = oh * a.stride + kh - 1, iw = ow * a.stride + kw - 1;
    if (ih < 0 || ih >= a.H || iw < 0 || iw >= a.W) return z;
    return *reinterpret_cast<const uint4*>(a.in + (((size_t)b * a.H + ih) * a.W + iw) * a.Cin + ci);
  }
  // channels not a multiple of 8 (the first layer): element by element
  __align__(16) bf16 e[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int kk = k + j;
    bf16 v = __float2bfloat16(0.f);
    if (kk < a.K) {
      const int ci = kk % a.Cin, tap = kk / a.Cin, kh = tap / 3, kw = tap % 3;
      const int ih = oh * a.stride + kh - 1, iw = ow * a.stride + kw - 1;
      if (ih >= 0 && ih < a.H && iw >= 0 && iw < a.W) v = a.in[(((size_t)b * a.H + ih) * a.W + iw) * a.Cin + ci];
    }
    e[j] = v;
  }
  return *reinterpret_cast<const uint4*>(e);
}

// Eight consecutive K entries of row n of B (the weights [N][K]), zero outside.
__device__ __forceinline__ uint4 load_b(const Args& a, int n, int k) {
  if (n >= a.N || k >= a.K) return make_uint4(0u, 0u, 0u, 0u);
  if ((a.K & 7) == 0) return *reinterpret_cast<const uint4*>(a.w + (size_t)n * a.K + k);
  __align__(16) bf16 e[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) e[j] = k + j < a.K ? a.w[(size_t)n * a.K + k + j] : __float2bfloat16(0.f);
  return *reinterpret_cast<const uint4*>(e);
}

template <int NT>
__global__ void __launch_bounds__(128) tc_gemm_kernel(Args a) {
  extern __shared__ unsigned char dyn[];
  __shared__ __align__(8) uint64_t bar[STAGES];
  __shared__ uint32_t tmem_base;
  constexpr int A_BYTES = TM * TK * 2, B_BYTES = NT * TK * 2, STAGE = A_BYTES + B_BYTES;
  // 1024-byte aligned stage buffers (the swizzle atom)
  unsigned char* base = dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * NT;
  const int nk = (a.K + TK - 1) / TK;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"((uint32_t)NT)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc_bf16(NT);

  bool ok = true;
  for (int ks = 0; ks < nk && ok; ++ks) {
    const int s = ks & 1;
    unsigned char* As = base + s * STAGE;
    unsigned char* Bs = As + A_BYTES;
    if (ks >= STAGES) {
      // the products of step ks - 2 have read this stage
      const bool w = mbar_wait(&bar[s], ((ks - STAGES) >> 1) & 1u, WAIT_BUDGET_DEFAULT);
      if (!__syncthreads_and(w)) {
        ok = false;
        break;
      }
    }
    const int k0 = ks * TK;
    for (int e = tid; e < TM * (TK / 8); e += 128) {
      const int r = e >> 3, c = e & 7;
      *reinterpret_cast<uint4*>(As + sw128(r, c)) = load_a(a, m0 + r, k0 + 8 * c);
    }
    for (int e = tid; e < NT * (TK / 8); e += 128) {
      const int r = e >> 3, c = e & 7;
      *reinterpret_cast<uint4*>(Bs + sw128(r, c)) = load_b(a, n0 + r, k0 + 8 * c);
    }
    fence_proxy_async_smem();   // the generic-proxy writes above, before the tensor cores read them
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t ab = smem_u32(As), bb = smem_u32(Bs);
#pragma unroll
      for (int j = 0; j < TK / 16; ++j)   // K = 16 per product: 32 bytes along the swizzled row
        mma_bf16_tmem(tmem, smem_desc_sw128(ab + 32 * j), smem_desc_sw128(bb + 32 * j), idesc,
                      (ks > 0 || j > 0) ? 1u : 0u);
      mma_commit(&bar[s]);
    }
  }
  if (ok) {
    const int last = nk - 1;
    ok = mbar_wait(&bar[last & 1], (last >> 1) & 1u, WAIT_BUDGET_DEFAULT);
    ok = __syncthreads_and(ok);
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // the products already issued: wait once more (bounded) before the memory they use is released
    const int last = nk - 1;
    mbar_wait(&bar[last & 1], (last >> 1) & 1u, WAIT_BUDGET_DEFAULT);
  } else {
    fence_after_sync();
    // warp w owns accumulator lanes 32 w .. 32 w + 31: row m0 + 32 w + lane
    const int m = m0 + 32 * warp + lane;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 8) {
      float v[8];
      tmem_ld8(trow + (uint32_t)c0, v);
      const int n = n0 + c0;
      if (m < a.M && n < a.N) {
        if (a.out) {
          __align__(16) bf16 o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16(fmaxf(v[i] + (n + i < a.N ? a.bias[n + i] : 0.f), 0.f));
          if (n + 8 <= a.N && (a.N & 7) == 0) {
            *reinterpret_cast<uint4*>(a.out + (size_t)m * a.N + n) = *reinterpret_cast<const uint4*>(o);
          } else {
            for (int i = 0; i < 8 && n + i < a.N; ++i) a.out[(size_t)m * a.N + n + i] = o[i];
          }
        } else {
          for (int i = 0; i < 8 && n + i < a.N; ++i) {
            float y = v[i] + a.bias[n + i];
            if (a.scale) y = y * a.scale[n + i] + a.shift[n + i];
            a.out_f[(size_t)m * a.N + n + i] = y;
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NT) : "memory");
  }
}

template <int NT>
static cudaError_t launch(const Args& a, cudaStream_t st) {
  // stage buffers plus 1 KB for the alignment; at least 40 KB so that no more than 5 CTAs share an
  // SM (5 x 128 columns of tensor memory at most = the SM's 512)
  const int smem = std::max(STAGES * (TM * TK * 2 + NT * TK * 2) + 1024, 40 * 1024);
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((a.M + TM - 1) / TM, (a.N + NT - 1) / NT);
  tc_gemm_kernel<NT><<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace cnn_tc

// D = A B on the tensor cores, the tile width chosen from N (32, 64 or 128 columns per CTA).
cudaError_t tc_gemm_forward(const cnn_tc::Args& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.N <= 32) return cnn_tc::launch<32>(a, st);
  if (a.N <= 64) return cnn_tc::launch<64>(a, st);
  return cnn_tc::launch<128>(a, st);
}

}  // namespace celeste
