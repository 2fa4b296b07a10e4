// Pixel kernels: ELBO + gradient + Hessian tile sums, and value-only tile sums.
//
// Paper, Sec. "The Celeste Model": x_nm ~ Poisson(F_nm) with F_nm deterministic in the catalog
// and Lambda_n.  Sec. "Variational Inference": L = E_q[log p(x, z) - log q(z)] (Eq. 1-2), each
// source optimised with neighbours fixed, with the exact gradient and dense Hessian.
//
// Per pixel m of a source's patch in image n (band b):
//   E[G] = A0 f0 + A1 f1,  E[G^2] = B0 f0^2 + B1 f1^2      (A_i = a_i E[l_b|i], B_i = a_i E[l_b^2|i])
//   E = bE + iota E[G],    V = bV + iota^2 Var[G]          (bE, bV: sky + fixed neighbours)
//   l = x (log E - V / (2 E^2)) - E - log x!               (delta method for E_q[log F])
// The gradient and Hessian are assembled from 108 per-tile sums (layout in celeste_internal.cuh):
//   grad = sum_m w1 dE[G] + w2 dE[G^2]
//   Hess = sum_m Y_m^T C_m Y_m + w1 d2E[G] + w2 d2E[G^2]
// with Y_m = [dE[G]; dE[G^2]] written in an 11-column reduced basis (the brightness columns of
// dE[G] are f_i times a per-(source, image) constant vector), C_m the 2x2 curvature of the
// pixel term, w1 = iota l_E - 2 iota^2 E[G] l_V and w2 = iota^2 l_V.
//
// A CTA of 128 threads takes tiles (up to 128 * PPT consecutive pixels of one patch) from the
// work queue.  Thread 0 brings each tile's patch table and pixel records into shared memory with
// two TMA bulk copies on one mbarrier, the next tile's while the current one is evaluated.  Each
// thread evaluates its pixels; each warp reduce-scatters the 108 per-pixel contributions so that
// lane l keeps sums l, l+32, l+64, l+96 (4 registers, not 108).
#include <cuda_bf16.h>

#include <algorithm>
#include <utility>

#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

__host__ __device__ constexpr int tri5(int i, int j) { return i * 5 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int tri6(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int tri_row(int q, int n) {
  int i = 0;
  while (q >= n - i) {
    q -= n - i;
    ++i;
  }
  return i;
}
__host__ __device__ constexpr int tri_col(int q, int n) {
  int i = 0;
  while (q >= n - i) {
    q -= n - i;
    ++i;
  }
  return i + q;
}

// Warp reduce-scatter: on return lane l holds the warp sum of v[l] (v is clobbered).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = up ? v[i] : v[i + off];
      const float keep = up ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// The same through shared memory (T: the warp's 32 x XP_LD scratch): lane l writes its 32 values as
// row l (eight 16-byte stores; rows XP_LD = 36 floats apart, so each quarter-warp phase of 16-byte
// stores covers all 32 banks), then sums column l (conflict-free: consecutive lanes, consecutive
// words), pairwise in packed adds.  About half the instructions of the shuffle form, which needs two
// selects, a shuffle and an add per value and level.
constexpr int XP_LD = 36;
__device__ __forceinline__ float warp_reduce_scatter32_smem(const float (&v)[32], float* T, int lane) {
  float4* row = reinterpret_cast<float4*>(T + lane * XP_LD);
#pragma unroll
  for (int i = 0; i < 8; ++i) row[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  __syncwarp();
  float2 p[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) p[r] = make_float2(T[(2 * r) * XP_LD + lane], T[(2 * r + 1) * XP_LD + lane]);
  __syncwarp();   // the scratch is rewritten by the next call
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int r = 0; r < w; ++r) p[r] = __fadd2_rn(p[r], p[r + w]);
  return p[0].x + p[0].y;
}

// Thread 0's feed of tiles from the work queue.  Staging a tile takes four dependent global round
// trips (queue position, list entry, tile record, then the copies); done in one go they would hold
// the CTA at its next barrier.  The feed runs them as a pipeline over three tiles: each call issues
// the copies of the tile whose records arrived during the previous call, starts the record copies
// of the next tile (cp.async into shared memory, so nothing stays in registers across the pixel
// work), the list load of the one after, and the queue take after that (its result, one register,
// is first needed by the next call).  The patch record comes with the tile's bulk copies.
static_assert(sizeof(PatchDev) % 16 == 0, "the patch record is bulk-copied");
struct TileFeed {
  TileDev t;        // records of the tile to issue next (when s >= 0)
  long long pix;
  int s;            // its slot, or -1
  int s_next;       // slot of the tile after it, or -1
  int n;            // tiles in the worklist
};

__device__ __forceinline__ void feed_start(const ProblemDev& P, TileFeed& F, int& i_next) {
  const int n = P.wl_count[WL_TILES];
  const int* list = wl_list(P, WL_TILES);
  F.n = n;
  int i = atomicAdd(P.wl_count + 3 + WL_TILES, 1);
  F.s = i < n ? list[i] : -1;
  if (F.s >= 0) {
    F.t = P.tiles[F.s];
    F.pix = P.tile_pix[F.s];
  }
  i = atomicAdd(P.wl_count + 3 + WL_TILES, 1);
  F.s_next = i < n ? list[i] : -1;
  i_next = atomicAdd(P.wl_count + 3 + WL_TILES, 1);
}

// Issues the copies of the feed's ready tile into (tab, spix, pm) on bar and advances the feed;
// returns the tile's slot (-1: the queue is exhausted).  The caller has synchronised the CTA since
// the buffer was last read.
// value = true: only the table's value-only prefix (TB_VFLOATS floats); otherwise everything but the
// paired value copies (the prefix up to TB_VAL and the galaxy entries, at their table offsets).
__device__ __forceinline__ int feed_issue(const ProblemDev& P, TileFeed& F, int& i_next, float* tab, float4* spix,
                                          uint64_t* bar, TileDev* tm, PatchDev* pm, bool value = false) {
  cp_async_wait_all();   // the records copied by the previous call
  const int s = F.s;
  if (s >= 0) {
    const TileDev t = F.t;
    fence_proxy_async_smem();
    const float* src = P.ptab + (size_t)t.patch * TB_FLOATS;
    const uint32_t pb = (uint32_t)t.count * 16u, mb = (uint32_t)sizeof(PatchDev);
    if (value) {
      mbar_expect_tx(bar, TB_VFLOATS * 4u + pb + mb);
      bulk_copy(tab, src, TB_VFLOATS * 4u, bar);
    } else {
      constexpr uint32_t gb = (TB_FLOATS - TB_GAL) * 4u;
      mbar_expect_tx(bar, TB_VAL * 4u + gb + pb + mb);
      bulk_copy(tab, src, TB_VAL * 4u, bar);
      bulk_copy(tab + TB_GAL, src + TB_GAL, gb, bar);
    }
    bulk_copy(spix, P.pix + F.pix, pb, bar);
    bulk_copy(pm, P.patches + t.patch, mb, bar);
    *tm = t;
  }
  const int sn = F.s_next;
  F.s = sn;
  if (sn >= 0) {
    cp_async<16>(&F.t, P.tiles + sn);
    cp_async<8>(&F.pix, P.tile_pix + sn);
  }
  const int n = F.n;
  if (i_next < n) cp_async<4>(&F.s_next, wl_list(P, WL_TILES) + i_next);
  else F.s_next = -1;
  i_next = i_next < n ? atomicAdd(P.wl_count + 3 + WL_TILES, 1) : n;
  cp_async_commit();
  return s;
}

// All threads: wait (bounded by P.wait_budget) for a staged buffer.  On a timeout: error word, a
// last wait with the full budget for these copies and for the other buffer's when they are in
// flight (so that no copy lands after the CTA has left), and false on every thread.
__device__ __forceinline__ bool wait_tile(const ProblemDev& P, uint64_t* bar, uint32_t phase, uint64_t* other,
                                          uint32_t other_phase, bool other_busy) {
  bool ok = P.wait_budget >= 0 && mbar_wait(bar, phase, P.wait_budget);
  if (!ok) {
    atomicExch(P.err + ERR_TIMEOUT, 1);
    mbar_wait(bar, phase, WAIT_BUDGET_DEFAULT);
  }
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0) {
    if (other_busy) mbar_wait(other, other_phase, WAIT_BUDGET_DEFAULT);
    cp_async_wait_all();   // the tile feed's record copies
  }
  return ok;
}

// Per-pixel quantities that the 108 sums are built from.
struct PixelCtx {
  float ell, w1, w2, u1, u2, A0w1, B0w2x2;
  float f0, f0m[2], f0mm[3];
  float f1, f1g[6], f1gg[21];
  float yE[NRED], yV[NRED], ta[NRED], ua[NRED];
};

// Contribution of one pixel to sum Q (resolved at compile time).
template <int Q>
__device__ __forceinline__ float slot(const PixelCtx& c) {
  if constexpr (Q == ACC_L) {
    return c.ell;
  } else if constexpr (Q < ACC_S2) {
    constexpr int k = Q - ACC_S1;
    if constexpr (k == 0) return c.w1 * c.f0;
    else if constexpr (k < 3) return c.w1 * c.f0m[k - 1];
    else if constexpr (k == 3) return c.w1 * c.f1;
    else return c.w1 * c.f1g[k - 4];
  } else if constexpr (Q < ACC_HP) {
    constexpr int k = Q - ACC_S2;
    if constexpr (k == 0) return c.w2 * c.f0 * c.f0;
    else if constexpr (k < 3) return 2.f * c.w2 * c.f0 * c.f0m[k - 1];
    else if constexpr (k == 3) return c.w2 * c.f1 * c.f1;
    else return 2.f * c.w2 * c.f1 * c.f1g[k - 4];
  } else if constexpr (Q < ACC_M) {
    constexpr int k = Q - ACC_HP, a = tri_row(k, 6), b = tri_col(k, 6);
    float h = c.u1 * c.f1gg[k] + c.u2 * (c.f1g[a] * c.f1g[b] + c.f1 * c.f1gg[k]);
    if constexpr (a < 2 && b < 2) {
      constexpr int qs = a + b;   // (0,0) -> 0, (0,1) -> 1, (1,1) -> 2
      h += c.A0w1 * c.f0mm[qs] + c.B0w2x2 * (c.f0m[a] * c.f0m[b] + c.f0 * c.f0mm[qs]);
    }
    return h;
  } else if constexpr (Q < NACC) {
    constexpr int k = Q - ACC_M, a = tri_row(k, NRED), b = tri_col(k, NRED);
    if constexpr (b < 7) return c.ta[a] * c.yE[b] + c.ua[a] * c.yV[b];
    else if constexpr (b < 9) return c.ta[a] * c.yE[b];    // yV[7], yV[8] are zero
    else return c.ua[a] * c.yV[b];                          // yE[9], yE[10] are zero
  } else {
    return 0.f;
  }
}

// NoM: leave out the Jacobian cross-product sums (formed on the tensor cores instead).
template <int CH, bool NoM = false, int... I>
__device__ __forceinline__ void fill_chunk(float (&v)[32], const PixelCtx& c, std::integer_sequence<int, I...>) {
  ((v[I] = (NoM && 32 * CH + I >= ACC_M) ? 0.f : slot<32 * CH + I>(c)), ...);
}

// ---------------------------------------------------------------- tensor-core Jacobian SYRK
// The cross-product block M_ab = sum_m ta_a yE_b + ua_a yV_b (a, b < 11) as one small GEMM per
// warp and 32 pixels: M = A' B' with A' = [ta | ua] (11 x 64, padded to 16 rows) and
// B' = [yE ; yV] (64 x 11, padded to 16 columns), K = 2 x 32 pixel terms.  Each lane stages its
// pixel's 44 numbers in shared memory (A' rows and B'^T rows of 68 floats: conflict-free stores
// and fragment loads), then the warp issues mma.sync with float32 accumulators kept in registers
// across the tile's pixels.  Operand forms (HM):
//   1  TF32 (m16n8k8, 8 k-steps x 2 n-tiles): 11 significant bits per operand;
//   2  BF16 hi + lo (m16n8k16, 4 k-steps x 2 n-tiles x 3 products hi.hi + hi.lo + lo.hi): the
//      dropped lo.lo and the split's remainder leave ~2^-17 of each product;
//   3  BF16 hi + mid + lo (x 6 products: every pair whose bit weights reach 2^-16 of the product,
//      hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid): ~2^-24 of each product, float32's own level;
//   4  TF32 big + small (m16n8k8 x 3 products big.big + big.small + small.big): ~2^-21.
// A split takes x -> hi = round(x), then the remainder's rounding, and so on; each remainder is
// exact in float32, so the parts sum to x up to the last part's rounding.
constexpr int SYRK_LD = 68;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Two consecutive floats (k, k+1) split into bf16 hi and lo pairs, the lower k in the low half.
__device__ __forceinline__ void split_bf16x2(const float* p, uint32_t& hi, uint32_t& lo) {
  const float2 x = *reinterpret_cast<const float2*>(p);
  const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Two consecutive floats split into bf16 hi, mid and lo pairs (each pair the lower k in the low half).
__device__ __forceinline__ void split3_bf16x2(const float* p, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  const float2 x = *reinterpret_cast<const float2*>(p);
  const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
  const float2 hf = __bfloat1622float2(h);
  const float r0 = x.x - hf.x, r1 = x.y - hf.y;
  const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(m);
  const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  mid = *reinterpret_cast<const uint32_t*>(&m);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// x split into TF32 big + small (the remainder x - big is exact in float32).
__device__ __forceinline__ void split_tf32(float x, uint32_t& big, uint32_t& small) {
  big = to_tf32(x);
  small = to_tf32(x - __uint_as_float(big));
}

// D[nt] (16 x 8 tiles nt = 0, 1) += A' B' for this warp's staged 32 pixels.
// Rows 11..15 of the 16-row fragments are the zero padding of the 11 x 11 block: they read `zrow`
// (a zero row in shared memory) instead of staged rows.
template <int HM>
__device__ __forceinline__ void syrk_mma(const float (*As)[SYRK_LD], const float (*Bt)[SYRK_LD], const float* zrow,
                                         float (&d)[2][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  const float* A0 = As[g];
  const float* A1 = g + 8 < NRED ? As[g + 8] : zrow;
  const float* Bn[2] = {Bt[g], g + 8 < NRED ? Bt[g + 8] : zrow};
  if constexpr (HM == 4) {
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 8) {
      uint32_t ab[4], as[4];
      split_tf32(A0[k0 + t], ab[0], as[0]);
      split_tf32(A1[k0 + t], ab[1], as[1]);
      split_tf32(A0[k0 + t + 4], ab[2], as[2]);
      split_tf32(A1[k0 + t + 4], ab[3], as[3]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        uint32_t bb0, bs0, bb1, bs1;
        split_tf32(Bn[nt][k0 + t], bb0, bs0);
        split_tf32(Bn[nt][k0 + t + 4], bb1, bs1);
        mma_tf32(d[nt], as[0], as[1], as[2], as[3], bb0, bb1);   // small terms first
        mma_tf32(d[nt], ab[0], ab[1], ab[2], ab[3], bs0, bs1);
        mma_tf32(d[nt], ab[0], ab[1], ab[2], ab[3], bb0, bb1);
      }
    }
  } else if constexpr (HM == 3) {
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 16) {
      uint32_t ah[4], am[4], al[4];
      split3_bf16x2(&A0[k0 + 2 * t], ah[0], am[0], al[0]);
      split3_bf16x2(&A1[k0 + 2 * t], ah[1], am[1], al[1]);
      split3_bf16x2(&A0[k0 + 2 * t + 8], ah[2], am[2], al[2]);
      split3_bf16x2(&A1[k0 + 2 * t + 8], ah[3], am[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        uint32_t bh0, bm0, bl0, bh1, bm1, bl1;
        split3_bf16x2(&Bn[nt][k0 + 2 * t], bh0, bm0, bl0);
        split3_bf16x2(&Bn[nt][k0 + 2 * t + 8], bh1, bm1, bl1);
        mma_bf16(d[nt], al[0], al[1], al[2], al[3], bh0, bh1);   // small terms first
        mma_bf16(d[nt], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
        mma_bf16(d[nt], am[0], am[1], am[2], am[3], bm0, bm1);
        mma_bf16(d[nt], am[0], am[1], am[2], am[3], bh0, bh1);
        mma_bf16(d[nt], ah[0], ah[1], ah[2], ah[3], bm0, bm1);
        mma_bf16(d[nt], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
      }
    }
  } else if constexpr (HM == 1) {
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 8) {
      const uint32_t a0 = to_tf32(A0[k0 + t]), a1 = to_tf32(A1[k0 + t]);
      const uint32_t a2 = to_tf32(A0[k0 + t + 4]), a3 = to_tf32(A1[k0 + t + 4]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const uint32_t b0 = to_tf32(Bn[nt][k0 + t]), b1 = to_tf32(Bn[nt][k0 + t + 4]);
        mma_tf32(d[nt], a0, a1, a2, a3, b0, b1);
      }
    }
  } else {
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 16) {
      uint32_t ah[4], al[4];
      split_bf16x2(&A0[k0 + 2 * t], ah[0], al[0]);
      split_bf16x2(&A1[k0 + 2 * t], ah[1], al[1]);
      split_bf16x2(&A0[k0 + 2 * t + 8], ah[2], al[2]);
      split_bf16x2(&A1[k0 + 2 * t + 8], ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        uint32_t bh0, bl0, bh1, bl1;
        split_bf16x2(&Bn[nt][k0 + 2 * t], bh0, bl0);
        split_bf16x2(&Bn[nt][k0 + 2 * t + 8], bh1, bl1);
        mma_bf16(d[nt], ah[0], ah[1], ah[2], ah[3], bh0, bh1);
        mma_bf16(d[nt], ah[0], ah[1], ah[2], ah[3], bl0, bl1);
        mma_bf16(d[nt], al[0], al[1], al[2], al[3], bh0, bh1);
      }
    }
  }
}

// Two-wide float32 arithmetic (one packed instruction for two independent multiply-adds: half
// the issue slots of the scalar form, which bounds this kernel).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// One galaxy family's sums over its components at a pixel: value F, first derivatives over
// v5 = (mu0, mu1, axis, angle, scale) and second derivatives, the latter kept in the pairs that the
// packed updates below form.
struct GalAcc {
  float F;
  float2 v01, v23;              // d/dv (0, 1), (2, 3)
  float v4;
  float2 vv00_01;               // d2/dv dv: (0,0), (0,1)
  float vv11;                   // (1,1)
  float2 vv02_03, vv12_13;      // (0,2), (0,3); (1,2), (1,3)
  float2 vv04_14;               // (0,4), (1,4)
  float2 vv22_23, vv24_33, vv34_44;
  __device__ __forceinline__ void zero() {
    F = v4 = vv11 = 0.f;
    v01 = v23 = vv00_01 = vv02_03 = vv12_13 = vv04_14 = vv22_23 = vv24_33 = vv34_44 = f2(0.f, 0.f);
  }
  __device__ __forceinline__ float v(int a) const {
    return a == 0 ? v01.x : a == 1 ? v01.y : a == 2 ? v23.x : a == 3 ? v23.y : v4;
  }
  // (a, b) with a <= b
  __device__ __forceinline__ float vv(int a, int b) const {
    switch (a * 5 + b) {
      case 0: return vv00_01.x;
      case 1: return vv00_01.y;
      case 2: return vv02_03.x;
      case 3: return vv02_03.y;
      case 4: return vv04_14.x;
      case 6: return vv11;
      case 7: return vv12_13.x;
      case 8: return vv12_13.y;
      case 9: return vv04_14.y;
      case 12: return vv22_23.x;
      case 13: return vv22_23.y;
      case 14: return vv24_33.x;
      case 18: return vv24_33.y;
      case 19: return vv34_44.x;
      default: return vv34_44.y;   // 24: (4, 4)
    }
  }
};

// One galaxy mixture component's contribution at pixel offset d (squares s; D0, D1, S0-S2 the
// same numbers in both halves of a pair): value, 5 first and 15 second derivatives over v5,
// accumulated into its family's sums.  z = P d, q = d.P.d = z.d; b_a = l_a + Q_a.s and
// t_a = (Q_a d) for a = axis, angle, scale; the second derivatives N (z z^T - P),
// N (z_i b_a - 2 t_a,i), N (b_a b_b + c_ab) with c_ab = l_ab + Q_ab.s.
// Far from a narrow component its Gaussian underflows to exactly 0 (q > ~207): where that holds on
// every lane of the warp (lanes without a pixel count as 0) the component adds exactly nothing, and
// the warp skips its derivative terms (on the mosaic ~19 % of warp-component pairs).  All lanes of
// the warp must be active.
__device__ __forceinline__ void gal_component(const float* ep, float2 D0, float2 D1, float2 S0, float2 S1, float2 S2,
                                              bool valid, GalAcc& A) {
  float e[GT_STRIDE];
  const float4* e4 = reinterpret_cast<const float4*>(ep);
#pragma unroll
  for (int w = 0; w < GT_STRIDE / 4; ++w) {
    const float4 t4 = e4[w];
    e[4 * w + 0] = t4.x;
    e[4 * w + 1] = t4.y;
    e[4 * w + 2] = t4.z;
    e[4 * w + 3] = t4.w;
  }
  const float q = fmaf(e[GT_P + 2], S2.x, fmaf(e[GT_P + 1], S1.x, e[GT_P] * S0.x));
  const float N = e[GT_W] * exp2f(q * (-0.5f * LOG2E));
  if (__all_sync(0xffffffffu, N == 0.f || !valid)) return;
  const float2 z = fma2(f2(e[GT_PZ], e[GT_PZ + 1]), D1, mul2(f2(e[GT_P], e[GT_P + 1]), D0));   // (z0, z1)
  // axis and angle together, scale alone
  const float2 Q0 = f2(e[GT_Q01], e[GT_Q01 + 1]), Q1 = f2(e[GT_Q01 + 2], e[GT_Q01 + 3]),
               Q2 = f2(e[GT_Q01 + 4], e[GT_Q01 + 5]);                       // (Q_0[i], Q_1[i])
  const float2 b01 = fma2(Q2, S2, fma2(Q1, S1, fma2(Q0, S0, f2(e[GT_LA01], e[GT_LA01 + 1]))));
  const float2 t0 = fma2(Q1, D1, mul2(Q0, D0));     // (t_0[0], t_1[0])
  const float2 t1 = fma2(Q2, D1, mul2(Q1, D0));     // (t_0[1], t_1[1])
  const float b2 = fmaf(e[GT_Q2 + 3], S2.x, fmaf(e[GT_Q2 + 1], S1.x, fmaf(e[GT_Q2], S0.x, e[GT_LA2])));
  const float2 t2 = fma2(f2(e[GT_Q2 + 2], e[GT_Q2 + 3]), D1, mul2(f2(e[GT_Q2], e[GT_Q2 + 1]), D0));   // t_2
  const float2 NN = f2(N, N);
  const float2 Nz = mul2(NN, z);
  const float2 Nm2 = f2(-2.f * N, -2.f * N);
  const float2 Nb01 = mul2(NN, b01);
  const float Nb2 = N * b2;
  A.F += N;
  A.v01 = add2(A.v01, Nz);
  A.v23 = add2(A.v23, Nb01);
  A.v4 += Nb2;
  A.vv00_01 = fma2(f2(-N, -N), f2(e[GT_P], e[GT_P + 1]), fma2(f2(Nz.x, Nz.x), z, A.vv00_01));
  A.vv11 = fmaf(-N, e[GT_P + 2], fmaf(Nz.y, z.y, A.vv11));
  A.vv02_03 = fma2(Nm2, t0, fma2(f2(Nz.x, Nz.x), b01, A.vv02_03));
  A.vv12_13 = fma2(Nm2, t1, fma2(f2(Nz.y, Nz.y), b01, A.vv12_13));
  A.vv04_14 = fma2(Nm2, t2, fma2(Nz, f2(b2, b2), A.vv04_14));
  // c_ab for the pairs (00, 01), (02, 11), (12, 22)
  float2 c[3];
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const float* G = e + GT_CAB + 8 * g;
    c[g] = fma2(f2(G[6], G[7]), S2, fma2(f2(G[4], G[5]), S1, fma2(f2(G[2], G[3]), S0, f2(G[0], G[1]))));
  }
  A.vv22_23 = fma2(NN, c[0], fma2(f2(Nb01.x, Nb01.x), b01, A.vv22_23));
  A.vv24_33 = fma2(NN, c[1], fma2(Nb01, f2(b2, b01.y), A.vv24_33));
  A.vv34_44 = fma2(NN, c[2], fma2(f2(Nb01.y, Nb2), f2(b2, b2), A.vv34_44));
}

// ------------------------------------------------------------------------------ full kernel
// HM: 0 all sums on the FP32 pipes; 1 / 2 the Jacobian cross-product on the tensor cores with
// TF32 / BF16 hi+lo operands.
// Tiles are double-buffered: the next tile's copies are issued before the current one is
// evaluated.  (The tensor-core variants' staging area holds the 11 rows of A' and B'^T per warp;
// the fragments' padding rows read one shared zero row, which keeps both buffers within the 48 KB
// of static shared memory.)
template <int PPT, int HM>
__global__ void __launch_bounds__(BLOCK) elbo_full_kernel(ProblemDev P) {
  constexpr int NB = PPT >= 8 ? 1 : 2;   // (1024-pixel tiles: two pixel buffers would pass 48 KB)
  __shared__ __align__(16) float tab_buf[NB][TB_FLOATS];
  __shared__ __align__(16) float4 spix_buf[NB][BLOCK * PPT];
  __shared__ __align__(8) uint64_t bar[NB];
  __shared__ TileDev tmeta[NB];
  __shared__ __align__(16) PatchDev pmeta[NB];
  __shared__ __align__(16) TileFeed feed;
  __shared__ float red[BLOCK / 32][128];
  // per-warp scratch: the tensor-core forms' staging of A' and B'^T, or the FP32 form's transposes
  // for the reduce-scatter with 128-pixel tiles (with larger tiles the 18 KB cost a CTA per SM,
  // more than the transposes save)
  constexpr bool XP = HM == 0 && PPT == 1;
  constexpr int WB = HM ? 2 * NRED * SYRK_LD : (XP ? 32 * XP_LD : 4);
  __shared__ __align__(16) float wbuf[BLOCK / 32][WB];
  __shared__ __align__(16) float zrow[HM ? SYRK_LD : 4];

  __shared__ int slot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0)
    for (int b = 0; b < NB; ++b) mbar_init(&bar[b], 1);
  if constexpr (HM != 0) {   // the zero row standing for rows 11..15 of A' and B'^T
    for (int i = tid; i < SYRK_LD; i += BLOCK) zrow[i] = 0.f;
  }
  // Iteration it uses buffer it % NB for its (it / NB + 1)-th time: the barrier's phase parity is
  // (it / NB) & 1.  Thread 0 takes the next tile from the queue and issues its copies; the wait's
  // barrier publishes its index in `slot`, which thread 0 rewrites only after the iteration's
  // closing barrier.
  int i_next = 0;   // thread 0: the feed's pending queue position
  if (tid == 0) {
    feed_start(P, feed, i_next);
    slot = feed_issue(P, feed, i_next, tab_buf[0], spix_buf[0], &bar[0], &tmeta[0], &pmeta[0]);
  }
  __syncthreads();
  int tile = slot;
  for (uint32_t it = 0; tile >= 0; ++it) {
  const int b = NB == 2 ? (int)(it & 1u) : 0;
  if (NB == 2 && tid == 0)
    slot = feed_issue(P, feed, i_next, tab_buf[b ^ 1], spix_buf[b ^ 1], &bar[b ^ 1], &tmeta[b ^ 1], &pmeta[b ^ 1]);
  if (!wait_tile(P, &bar[b], (it / NB) & 1u, &bar[b ^ (NB - 1)], ((it + 1) / NB) & 1u, NB == 2 && slot >= 0)) {
    if (tid < NACC) P.partials[(size_t)tile * NACC + tid] = __int_as_float(0x7fc00000);
    return;
  }
  const float* tab = tab_buf[b];
  const float4* spix = spix_buf[b];
  const TileDev t = tmeta[b];
  const PatchDev pt = pmeta[b];
  if (tid == 0) atomicAdd(P.counters + 0, (unsigned long long)t.count);
  const SNConst c = *reinterpret_cast<const SNConst*>(&tab[TB_SNC]);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float dm[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};   // tensor-core M block (HM != 0)

#pragma unroll 1
  for (int r = 0; r < PPT; ++r) {
    if (r * BLOCK + warp * 32 >= t.count) break;   // warp-uniform
    const int i = r * BLOCK + tid;
    const bool valid = i < t.count;
    const int idx = t.start + (valid ? i : 0);
    const int row = idx / pt.w, col = idx - row * pt.w;
    const float fx = (float)col, fy = (float)row;
    const float4 pv = valid ? spix[i] : make_float4(0.f, 1.f, 0.f, 0.f);

    // ---- profiles: star (value, d/dmu, d2/dmu2); galaxy families exp/deV over
    //      v5 = (mu0, mu1, axis, angle, scale): value, 5 first, 15 second derivatives
    float f0 = 0.f, f0m[2] = {0.f, 0.f}, f0mm[3] = {0.f, 0.f, 0.f};
    GalAcc G[2];
    G[0].zero();
    G[1].zero();
#pragma unroll 1
    for (int k = 0; k < CELESTE_NPSF; ++k) {
      const float d0 = fx - tab[TB_MU + 2 * k], d1 = fy - tab[TB_MU + 2 * k + 1];
      const float s0 = d0 * d0, s1 = 2.f * d0 * d1, s2 = d1 * d1;
      const float2 D0 = f2(d0, d0), D1 = f2(d1, d1), S0 = f2(s0, s0), S1 = f2(s1, s1), S2 = f2(s2, s2);
      {
        const float4 st = *reinterpret_cast<const float4*>(&tab[TB_STAR + 4 * k]);
        const float q = fmaf(st.w, s2, fmaf(st.z, s1, st.y * s0));
        const float N = st.x * exp2f(q * (-0.5f * LOG2E));
        const float z0 = st.y * d0 + st.z * d1, z1 = st.z * d0 + st.w * d1;
        f0 += N;
        f0m[0] += N * z0;
        f0m[1] += N * z1;
        f0mm[0] += N * (z0 * z0 - st.y);
        f0mm[1] += N * (z0 * z1 - st.z);
        f0mm[2] += N * (z1 * z1 - st.w);
      }
      // one family at a time, rolled loops: the component body stays small enough for the
      // instruction cache, and each family's accumulators stay statically indexed
#pragma unroll 1
      for (int j = 0; j < CELESTE_NEXP; ++j)
        gal_component(&tab[TB_GAL + (k * NMIX + j) * GT_STRIDE], D0, D1, S0, S1, S2, valid, G[0]);
#pragma unroll 1
      for (int j = CELESTE_NEXP; j < NMIX; ++j)
        gal_component(&tab[TB_GAL + (k * NMIX + j) * GT_STRIDE], D0, D1, S0, S1, S2, valid, G[1]);
    }

    // ---- galaxy profile over G6 = (mu0, mu1, dev, axis, angle, scale);  v5 index -> G6 index:
    //      0 -> 0, 1 -> 1, 2 -> 3, 3 -> 4, 4 -> 5
    PixelCtx cx;
    cx.f0 = f0;
    cx.f0m[0] = f0m[0];
    cx.f0m[1] = f0m[1];
    cx.f0mm[0] = f0mm[0];
    cx.f0mm[1] = f0mm[1];
    cx.f0mm[2] = f0mm[2];
    const float F0 = G[0].F, F1 = G[1].F;
    const float dF = F1 - F0;
    cx.f1 = F0 + c.e * dF;
    cx.f1g[2] = c.e1 * dF;
    cx.f1gg[tri6(2, 2)] = c.e2 * dF;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const int ga = a < 2 ? a : a + 1;
      cx.f1g[ga] = G[0].v(a) + c.e * (G[1].v(a) - G[0].v(a));
      cx.f1gg[ga < 2 ? tri6(ga, 2) : tri6(2, ga)] = c.e1 * (G[1].v(a) - G[0].v(a));
#pragma unroll
      for (int bb = a; bb < 5; ++bb) {
        const int gb = bb < 2 ? bb : bb + 1;
        cx.f1gg[tri6(ga, gb)] = G[0].vv(a, bb) + c.e * (G[1].vv(a, bb) - G[0].vv(a, bb));
      }
    }
    const float f1 = cx.f1;

    // ---- pixel rate moments and the pixel term
    const float iota = c.iota, iota2 = iota * iota;
    const float EG = c.A0 * f0 + c.A1 * f1;
    const float dxv = c.L10 * f0 - c.L11 * f1;
    const float VG = c.C0 * f0 * f0 + c.C1 * f1 * f1 + c.Cx * dxv * dxv;
    const float E = pv.y + iota * EG;
    const float V = pv.z + iota2 * VG;
    const float x = pv.x;
    if (valid) P.srcmom[pt.pix_off + idx] = make_float2(EG, VG);
    const float rE = 1.f / E;
    const float rE2 = rE * rE;
    float ell;
    if (x > 0.f) {
      const float dEx = E - x;
      ell = pv.w + x * log1pf(dEx / x) - dEx - 0.5f * x * V * rE2;
    } else {
      ell = -E;
    }
    const float lE = (x - E) * rE + x * V * rE2 * rE;
    const float lV = -0.5f * x * rE2;
    const float lEE = -x * rE2 - 3.f * x * V * rE2 * rE2;
    const float lEV = x * rE2 * rE;
    const float vm = valid ? 1.f : 0.f;
    cx.ell = ell * vm;
    cx.w1 = vm * (iota * lE - 2.f * iota2 * EG * lV);
    cx.w2 = vm * (iota2 * lV);
    const float c00 = vm * (iota2 * lEE - 4.f * iota2 * iota * EG * lEV - 2.f * iota2 * lV);
    const float c01 = vm * (iota2 * iota * lEV);

    // ---- reduced Jacobian rows
    cx.yE[0] = c.A0 * f0m[0] + c.A1 * cx.f1g[0];
    cx.yE[1] = c.A0 * f0m[1] + c.A1 * cx.f1g[1];
    cx.yV[0] = 2.f * (c.B0 * f0 * f0m[0] + c.B1 * f1 * cx.f1g[0]);
    cx.yV[1] = 2.f * (c.B0 * f0 * f0m[1] + c.B1 * f1 * cx.f1g[1]);
#pragma unroll
    for (int a = 2; a < 6; ++a) {
      cx.yE[a] = c.A1 * cx.f1g[a];
      cx.yV[a] = 2.f * c.B1 * f1 * cx.f1g[a];
    }
    cx.yE[6] = c.aE1 * f1 - c.aE0 * f0;
    cx.yV[6] = c.aV1 * f1 * f1 - c.aV0 * f0 * f0;
    cx.yE[7] = f0;
    cx.yE[8] = f1;
    cx.yE[9] = 0.f;
    cx.yE[10] = 0.f;
    cx.yV[7] = 0.f;
    cx.yV[8] = 0.f;
    cx.yV[9] = f0 * f0;
    cx.yV[10] = f1 * f1;
#pragma unroll
    for (int a = 0; a < NRED; ++a) {
      cx.ta[a] = c00 * cx.yE[a] + c01 * cx.yV[a];
      cx.ua[a] = c01 * cx.yE[a];
    }
    cx.u1 = cx.w1 * c.A1;
    cx.u2 = 2.f * cx.w2 * c.B1;
    cx.A0w1 = cx.w1 * c.A0;
    cx.B0w2x2 = 2.f * cx.w2 * c.B0;

    if constexpr (HM == 0 && XP) {
      float v[32];
      float* T = wbuf[warp];
      fill_chunk<0>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[0] += warp_reduce_scatter32_smem(v, T, lane);
      fill_chunk<1>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[1] += warp_reduce_scatter32_smem(v, T, lane);
      fill_chunk<2>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[2] += warp_reduce_scatter32_smem(v, T, lane);
      fill_chunk<3>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[3] += warp_reduce_scatter32_smem(v, T, lane);
    } else if constexpr (HM == 0) {
      float v[32];
      fill_chunk<0>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[0] += warp_reduce_scatter32(v, lane);
      fill_chunk<1>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[1] += warp_reduce_scatter32(v, lane);
      fill_chunk<2>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[2] += warp_reduce_scatter32(v, lane);
      fill_chunk<3>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[3] += warp_reduce_scatter32(v, lane);
    } else {
      // chunks 0 and 1 hold every sum but the cross-product block (slots >= ACC_M = 42)
      float v[32];
      fill_chunk<0, true>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[0] += warp_reduce_scatter32(v, lane);
      fill_chunk<1, true>(v, cx, std::make_integer_sequence<int, 32>{});
      acc[1] += warp_reduce_scatter32(v, lane);
      float (*As)[SYRK_LD] = reinterpret_cast<float (*)[SYRK_LD]>(wbuf[warp]);
      float (*Bt)[SYRK_LD] = reinterpret_cast<float (*)[SYRK_LD]>(wbuf[warp] + NRED * SYRK_LD);
#pragma unroll
      for (int a = 0; a < NRED; ++a) {
        As[a][lane] = cx.ta[a];
        As[a][32 + lane] = cx.ua[a];
        Bt[a][lane] = cx.yE[a];
        Bt[a][32 + lane] = cx.yV[a];
      }
      __syncwarp();
      syrk_mma<HM>(As, Bt, zrow, dm, lane);
      __syncwarp();   // the staging area is rewritten for the next 32 pixels
    }
  }

  // ---- combine the warps: sum q lives in lane q % 32 of chunk q / 32
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) red[warp][32 * ch + lane] = acc[ch];
  if constexpr (HM != 0) {
    // D fragment (tile nt): rows g, g + 8; columns 8 nt + 2 t, 8 nt + 2 t + 1.  Entry (a, b) with
    // a <= b < 11 is sum ACC_M + tri(a, b) (the block is symmetric; its upper half is kept).
    __syncwarp();
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int a = g + (e >> 1) * 8, b = 8 * nt + 2 * tq + (e & 1);
        if (a <= b && b < NRED) red[warp][ACC_M + a * NRED - a * (a - 1) / 2 + (b - a)] = dm[nt][e];
      }
  }
  __syncthreads();
  if (tid < NACC) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) v += red[w][tid];
    P.partials[(size_t)tile * NACC + tid] = v;
  }
  const int next = slot;
  __syncthreads();   // this buffer, red and slot are rewritten after this point
  if constexpr (NB == 1) {
    if (tid == 0) slot = feed_issue(P, feed, i_next, tab_buf[0], spix_buf[0], &bar[0], &tmeta[0], &pmeta[0]);
    __syncthreads();
    tile = slot;
  } else {
    tile = next;
  }
  }
  if (tid == 0) cp_async_wait_all();   // no record copy lands after the CTA has left
}

// ------------------------------------------------------------------------------ value kernel
// diff = 0: sum of the pixel terms at the table's parameters.
// diff = 1: sum of l(theta) - l(theta_ref) per pixel, where theta_ref is the point of the source's
//           last full evaluation (its E[G], Var[G] kept in srcmom): the change of the ELBO's pixel
//           part without the rounding of two large sums.
template <int PPT>
__global__ void __launch_bounds__(BLOCK) elbo_value_kernel(ProblemDev P, int diff) {
  __shared__ __align__(16) float tab_buf[2][TB_VFLOATS];   // the table's value-only prefix
  __shared__ __align__(16) float4 spix_buf[2][BLOCK * PPT];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ TileDev tmeta[2];
  __shared__ __align__(16) PatchDev pmeta[2];
  __shared__ __align__(16) TileFeed feed;
  __shared__ float red[BLOCK / 32];

  __shared__ int slot;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  int i_next = 0;   // thread 0: the feed's pending queue position
  if (tid == 0) {
    feed_start(P, feed, i_next);
    slot = feed_issue(P, feed, i_next, tab_buf[0], spix_buf[0], &bar[0], &tmeta[0], &pmeta[0], true);
  }
  __syncthreads();
  int tile = slot;
  for (uint32_t it = 0; tile >= 0; ++it) {
  const int b = (int)(it & 1u);
  if (tid == 0)
    slot = feed_issue(P, feed, i_next, tab_buf[b ^ 1], spix_buf[b ^ 1], &bar[b ^ 1], &tmeta[b ^ 1], &pmeta[b ^ 1],
                      true);
  if (!wait_tile(P, &bar[b], (it >> 1) & 1u, &bar[b ^ 1], ((it + 1) >> 1) & 1u, slot >= 0)) {
    if (tid == 0) P.vpartials[tile] = __int_as_float(0x7fc00000);
    return;
  }
  const float* tab = tab_buf[b];
  const float4* spix = spix_buf[b];
  const TileDev t = tmeta[b];
  const PatchDev pt = pmeta[b];
  if (tid == 0) atomicAdd(P.counters + 1, (unsigned long long)t.count);
  const SNConst c = *reinterpret_cast<const SNConst*>(&tab[TB_SNC]);
  float sum = 0.f;
#pragma unroll 1
  for (int r = 0; r < PPT; ++r) {
    const int i = r * BLOCK + tid;
    if (i >= t.count) break;
    const int idx = t.start + i;
    const int row = idx / pt.w, col = idx - row * pt.w;
    const float fx = (float)col, fy = (float)row;
    const float4 pv = spix[i];
    // the pixel's reference values, loaded ahead of the profiles so that their latency overlaps them
    float2 ref = make_float2(0.f, 0.f);
    float wpx = 1.f;
    if (diff == 2) {
      ref = P.refEV[pt.pix_off + idx];
      wpx = P.pweight[pt.pix_off + idx];
    } else if (diff) {
      ref = P.srcmom[pt.pix_off + idx];
    } else if (P.pweight) {
      wpx = P.pweight[pt.pix_off + idx];
    }
    // components two at a time (the paired copies of the table's value prefix), with the full
    // kernel's formulas; the sums' association differs from it (pairs), a rounding difference of
    // ~1e-7 of a pixel's rate, far below what the ELBO tolerance resolves
    float f0 = 0.f;
    float2 fE = make_float2(0.f, 0.f), fD = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < CELESTE_NPSF; ++k) {
      const float d0 = fx - tab[TB_MU + 2 * k], d1 = fy - tab[TB_MU + 2 * k + 1];
      const float s0 = d0 * d0, s1 = 2.f * d0 * d1, s2 = d1 * d1;
      const float4 st = *reinterpret_cast<const float4*>(&tab[TB_STAR + 4 * k]);
      f0 += st.x * exp2f(fmaf(st.w, s2, fmaf(st.z, s1, st.y * s0)) * (-0.5f * LOG2E));
      const float2 S0 = f2(s0, s0), S1 = f2(s1, s1), S2 = f2(s2, s2);
      const float4* vp = reinterpret_cast<const float4*>(&tab[TB_VAL + 8 * (k * NMIX / 2)]);
#pragma unroll
      for (int pr = 0; pr < NMIX / 2; ++pr) {
        const float4 a = vp[2 * pr], w = vp[2 * pr + 1];   // (P00, P00', P01, P01'), (P11, P11', W, W')
        const float2 q = fma2(f2(w.x, w.y), S2, fma2(f2(a.z, a.w), S1, mul2(f2(a.x, a.y), S0)));
        const float2 qs = mul2(q, f2(-0.5f * LOG2E, -0.5f * LOG2E));
        const float2 g = mul2(f2(w.z, w.w), f2(exp2f(qs.x), exp2f(qs.y)));
        if (pr < CELESTE_NEXP / 2)
          fE = add2(fE, g);
        else
          fD = add2(fD, g);
      }
    }
    const float fEs = fE.x + fE.y, fDs = fD.x + fD.y;
    const float f1 = fEs + c.e * (fDs - fEs);
    const float EG = c.A0 * f0 + c.A1 * f1;
    const float dxv = c.L10 * f0 - c.L11 * f1;
    const float VG = c.C0 * f0 * f0 + c.C1 * f1 * f1 + c.Cx * dxv * dxv;
    const float E = pv.y + c.iota * EG;
    const float V = pv.z + c.iota * c.iota * VG;
    const float x = pv.x;
    if (diff == 2) {
      // joint objective: every source may have moved; the change from the stored pixel rates at
      // the reference point, weighted by 1 / (windows holding the pixel)
      const float dE = E - ref.x;
      sum += wpx * (x > 0.f ? x * log1pf(dE / ref.x) - dE - 0.5f * x * (V / (E * E) - ref.y / (ref.x * ref.x)) : -dE);
    } else if (diff) {
      const float dE = c.iota * (EG - ref.x);                  // E(theta) - E(theta_ref)
      const float Er = pv.y + c.iota * ref.x;
      const float Vr = pv.z + c.iota * c.iota * ref.y;
      sum += x > 0.f ? x * log1pf(dE / Er) - dE - 0.5f * x * (V / (E * E) - Vr / (Er * Er)) : -dE;
    } else {
      // pixel weight: 1 / (windows holding the pixel) for the joint objective, else 1
      const float dEx = E - x;
      sum += wpx * (x > 0.f ? pv.w + x * log1pf(dEx / x) - dEx - 0.5f * x * V / (E * E) : -E);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((tid & 31) == 0) red[tid >> 5] = sum;
  __syncthreads();
  if (tid == 0) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) v += red[w];
    P.vpartials[tile] = v;
  }
  const int next = slot;
  __syncthreads();   // this buffer, red and slot are rewritten after this point
  tile = next;
  }
  if (tid == 0) cp_async_wait_all();   // no record copy lands after the CTA has left
}

// ------------------------------------------------------------------------------ launchers
// Persistent grids: a fixed number of CTAs per SM takes tiles from the device work queue over the
// tile worklist, whose length is known only on the device.
constexpr int FULL_CTAS_PER_SM = 4;    // 128 registers x 128 threads: 4 CTAs fill the register file
constexpr int VALUE_CTAS_PER_SM = 8;

cudaError_t launch_full(const ProblemDev& P, const double* theta, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  cudaError_t e = launch_tables(P, theta, true, st);
  if (e != cudaSuccess) return e;
  return launch_full_kernel(P, st);
}

cudaError_t launch_full_kernel(const ProblemDev& P, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  const int g = std::max(1, std::min(P.n_tiles, P.n_sm * FULL_CTAS_PER_SM));
  if (P.hmode == 1) {
    elbo_full_kernel<1, 1><<<g, BLOCK, 0, st>>>(P);   // the create call admits these only with 128-pixel tiles
    return cudaGetLastError();
  }
  if (P.hmode == 2) {
    elbo_full_kernel<1, 2><<<g, BLOCK, 0, st>>>(P);
    return cudaGetLastError();
  }
  if (P.hmode == 3) {
    elbo_full_kernel<1, 3><<<g, BLOCK, 0, st>>>(P);
    return cudaGetLastError();
  }
  if (P.hmode == 4) {
    elbo_full_kernel<1, 4><<<g, BLOCK, 0, st>>>(P);
    return cudaGetLastError();
  }
  switch (P.tile_pixels) {
    case 128: elbo_full_kernel<1, 0><<<g, BLOCK, 0, st>>>(P); break;
    case 256: elbo_full_kernel<2, 0><<<g, BLOCK, 0, st>>>(P); break;
    case 512: elbo_full_kernel<4, 0><<<g, BLOCK, 0, st>>>(P); break;
    default: elbo_full_kernel<8, 0><<<g, BLOCK, 0, st>>>(P); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_value(const ProblemDev& P, const double* theta, bool diff, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  cudaError_t e = launch_tables(P, theta, false, st);
  if (e != cudaSuccess) return e;
  return launch_value_kernel(P, diff, st);
}

cudaError_t launch_value_kernel(const ProblemDev& P, bool diff, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  const int d = diff ? (P.refEV ? 2 : 1) : 0;   // difference from the joint reference rates when set
  const int g = std::max(1, std::min(P.n_tiles, P.n_sm * VALUE_CTAS_PER_SM));
  switch (P.tile_pixels) {
    case 128: elbo_value_kernel<1><<<g, BLOCK, 0, st>>>(P, d); break;
    case 256: elbo_value_kernel<2><<<g, BLOCK, 0, st>>>(P, d); break;
    case 512: elbo_value_kernel<4><<<g, BLOCK, 0, st>>>(P, d); break;
    default: elbo_value_kernel<8><<<g, BLOCK, 0, st>>>(P, d); break;
  }
  return cudaGetLastError();
}

}  // namespace celeste
