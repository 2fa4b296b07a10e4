// Internal device-side layout and helpers of the Celeste GB300 library.
//
// Model (paper, Sec. "The Celeste Model" and "Variational Inference"): the pixel rate of
// image n is F = sky + iota * sum_s G_s with G_s = l_b(s) * f_type(s)(pixel); the ELBO uses
// E[F], Var[F] under q and the delta method for E[log F].  Everything in this header is
// layout or small arithmetic used by several kernels of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "celeste.h"

namespace celeste {

constexpr int NP = CELESTE_NPARAM;       // 27 free parameters per source
constexpr int NSTAR = CELESTE_NPSF;      // star components (one per PSF component)
constexpr int NMIX = CELESTE_NEXP + CELESTE_NDEV;   // 14 profile components per PSF component
constexpr int NGAL = CELESTE_NPSF * NMIX;           // 42 galaxy components
constexpr int NCOMP = NSTAR + NGAL;                 // 45
constexpr int BLOCK = 128;               // threads per CTA of the pixel kernels

// Per-tile partial sums written by the ELBO+gradient+Hessian pixel kernel (float32 within a tile,
// summed across tiles in float64).  Reduced basis (11): mu0, mu1, dev, axis, angle, scale, alpha,
// f0 (E-row, star brightness), f1 (E-row, galaxy brightness), f0^2 (V-row), f1^2 (V-row).
constexpr int ACC_L = 0;                 // sum of pixel ELBO terms
constexpr int ACC_S1 = 1;                // 10: sum w1 * [f0, d_mu f0 (2), f1, d f1 (6: mu0 mu1 dev axis angle scale)]
constexpr int ACC_S2 = 11;               // 10: sum w2 * [f0^2, d_mu f0^2 (2), f1^2, d f1^2 (6)]
constexpr int ACC_HP = 21;               // 21: packed upper triangle over (mu0 mu1 dev axis angle scale)
constexpr int ACC_M = 42;                // 66: packed upper triangle of the 11x11 Jacobian cross-product
constexpr int NACC = 108;
constexpr int NRED = 11;

// Per-patch table (floats) written by the table kernel at the source's current parameters and
// bulk-copied into shared memory by every tile of the patch.  Positions are relative to the patch
// origin; quadratic forms use s = (d0^2, 2 d0 d1, d1^2) with d = pixel - mean of PSF component k
// (the same for the star component k and the 14 galaxy components (k, j)).  The first TB_VFLOATS
// floats are all that the value-only kernel reads (it stages only them): the galaxy components'
// precisions and normalisers again, two components interleaved for two-wide float32 arithmetic.
constexpr int TB_MU = 0;      // 3 x (x, y) mean of PSF component k, + 2 pad
constexpr int TB_STAR = 8;    // 3 x (W, P00, P01, P11)
constexpr int TB_SNC = 20;    // SNConst (20 floats)
constexpr int TB_VAL = 40;    // per k, per pair of components (j, j + 1), j even: (P00, P00'),
                              // (P01, P01'), (P11, P11'), (W, W'); pair index k * NMIX / 2 + j / 2
constexpr int TB_VFLOATS = TB_VAL + NGAL * 4;   // 208 floats = 832 bytes
constexpr int TB_GAL = TB_VFLOATS;              // NGAL x GT_STRIDE, component g = k * NMIX + j
// A galaxy component's entry is laid out for the pixel kernel's two-wide float32 arithmetic: the
// numbers combined in one packed operation sit side by side at an even offset (a few are stored
// twice).  Q_a = -1/2 dP/da (entries 00, 01, 11; a = axis, angle, scale), l_a = -1/2 d logdet/da,
// Q_ab and l_ab their second derivatives for the pairs ab = 00 01 02 11 12 22 (index pq 0-5).
constexpr int GT_P = 0;       // 3: precision matrix (00, 01, 11)
constexpr int GT_W = 3;       // weight * Gaussian normaliser, w_k nu_j / (2 pi sqrt(det)) (fracDev mixing applied later)
constexpr int GT_PZ = 4;      // (P01, P11): with (P00, P01) the rows of P
constexpr int GT_LA01 = 6;    // (l_0, l_1)
constexpr int GT_Q01 = 8;     // (Q_0[i], Q_1[i]) for i = 00, 01, 11
constexpr int GT_Q2 = 14;     // (Q_2[00], Q_2[01]), (Q_2[01], Q_2[11])
constexpr int GT_LA2 = 18;    // l_2 (19: pad)
constexpr int GT_CAB = 20;    // 3 groups of two pairs pq = (0, 1), (2, 3), (4, 5), 8 floats each:
                              // (l_p, l_q), then (Q_p[i], Q_q[i]) for i = 00, 01, 11
constexpr int GT_STRIDE = 44;
// Offsets of the single numbers (the first of a number stored twice).
__host__ __device__ constexpr int gt_qa(int a, int i) {
  return a < 2 ? GT_Q01 + 2 * i + a : GT_Q2 + (i == 0 ? 0 : (i == 1 ? 1 : 3));
}
__host__ __device__ constexpr int gt_la(int a) { return a < 2 ? GT_LA01 + a : GT_LA2; }
__host__ __device__ constexpr int gt_qab(int pq, int i) { return GT_CAB + 8 * (pq / 2) + 2 * (i + 1) + (pq % 2); }
__host__ __device__ constexpr int gt_lab(int pq) { return GT_CAB + 8 * (pq / 2) + (pq % 2); }
constexpr int TB_FLOATS = TB_GAL + NGAL * GT_STRIDE;   // 2056 floats = 8224 bytes (multiple of 16)
static_assert(NMIX % 2 == 0 && CELESTE_NEXP % 2 == 0, "component pairs never straddle the two families");
static_assert(TB_VFLOATS % 4 == 0 && TB_FLOATS % 4 == 0, "bulk-copied in multiples of 16 bytes");

// Per-(source, image) scalar constants used by the pixel kernels.
struct SNConst {
  float A0, A1, B0, B1;          // a_i E[l_b|i], a_i E[l_b^2|i]
  float aE0, aE1, aV0, aV1;      // a0 a1 E[l_b|i], a0 a1 E[l_b^2|i]
  float iota, e, e1, e2;         // calibration, sigma(dev), its first and second derivative
  // Var[G] = C0 f0^2 + C1 f1^2 + Cx (L10 f0 - L11 f1)^2 without cancellation:
  // C_i = a_i (E[l^2|i] - E[l|i]^2) = a_i E[l|i]^2 expm1(v_i), Cx = a0 a1.
  float C0, C1, Cx, L10, L11;
};
static_assert(sizeof(SNConst) <= 20 * sizeof(float), "SNConst fits its 20 table floats");

struct ImageDev {
  const float* pixels;
  int H, W, band, pad;
  float sky, iota;
  double A[4], o[2];
};

struct PatchDev {
  int source, image, x0, y0, w, h;
  long long pix_off;             // first float4 of this patch in the pixel buffer
  int tile_begin, tile_end, nbr_begin, nbr_end;
};

struct TileDev {
  int patch, start, count, pad;
};

// Worklists (offsets into ProblemDev::wl and indices of ProblemDev::wl_count).
constexpr int WL_TILES = 0, WL_PATCHES = 1, WL_SOURCES = 2;
constexpr int WL_INTS = 8;
// Doubles per source kept by the trust-region step for a repeated subproblem (Householder
// vectors, tridiagonal form, reflected gradient, reflection coefficients, squared off-diagonal).
constexpr int TR_CACHE = NP * NP + 5 * NP;

// Device view of a bound problem (passed by value to kernels).
struct ProblemDev {
  const ImageDev* images;
  const PatchDev* patches;
  const TileDev* tiles;
  const int* src_patch;          // [S+1] CSR of each source's patches
  const int* nbr;                // neighbour patch ids (same image)
  const double* u0;              // [S][2]
  const double* psf_coef;        // [n_images][3][6][6]
  float* psf;                    // [n_patches][18]: per PSF comp (w, mx, my, s00, s01, s11)
  float4* pix;                   // [n_pix]: (x, fixed rate, fixed variance, log-factorial term)
  float2* srcmom;                // [n_pix]: the target source's (E[G], Var[G]) at its last full evaluation
  float* ptab;                   // [n_patches][TB_FLOATS] per-patch tables
  const long long* tile_pix;     // [n_tiles] the tile's first float4 in pix (patch offset + start)
  float* partials;               // [n_tiles][NACC]
  float* vpartials;              // [n_tiles]
  int* flags;                    // [S] per-source work flags
  SNConst* snc;                  // [S][5] per-source, per-band brightness constants (iota unset)
  int* wl;                       // worklists built from the flags: tiles [n_tiles], patches [n_patches], sources [S]
  int* wl_count;                 // [WL_INTS]: number of tiles, patches, sources in the worklists,
                                 // then the three queue heads
  int* err;                      // [4] device error words
  unsigned long long* counters;  // [4]: full-kernel pixels, value-kernel pixels
  float* pweight;                 // [n_pix] or null: 1 / (number of windows holding the pixel), written by the
                                 // window-mode background and applied by the value kernel (joint objective)
  float2* refEV;                 // [n_pix] or null: each pixel's (E, V) at the joint solver's current point
  int S, n_patches, n_tiles, tile_pixels, n_sm, hmode;
  long long wait_budget;         // SM cycles the pixel kernels' first wait on a tile's bulk copies may take
                                 // (< 0: give up at once, the timeout path's test hook)
  double priors[5];
  double log_var_r, log_var_c, log_phi, log1m_phi, logit_phi;   // logs of the priors (host-computed)
  double inv_var_r, inv_var_c;   // reciprocals of the prior variances (host-computed)
  float nu[NMIX], tau[NMIX];     // exp (0..5) then deV (6..13)
};

__device__ inline int* wl_list(const ProblemDev& P, int which) {
  return P.wl + (which == WL_TILES ? 0 : which == WL_PATCHES ? P.n_tiles : P.n_tiles + P.n_patches);
}

// Work queue over a worklist: the CTA's next item (one atomic by thread 0, broadcast through
// shared memory), or -1 once the list is exhausted.  Every thread of the CTA must call it.
__device__ inline int wl_next_cta(const ProblemDev& P, int which, int& slot) {
  if (threadIdx.x == 0) {
    const int i = atomicAdd(P.wl_count + 3 + which, 1);
    slot = i < P.wl_count[which] ? wl_list(P, which)[i] : -1;
  }
  __syncthreads();
  const int item = slot;
  __syncthreads();   // the slot is rewritten only after every thread has read it
  return item;
}

// One thread's fetch from the work queue (the caller publishes the result to the CTA).
__device__ inline int wl_take(const ProblemDev& P, int which) {
  const int i = atomicAdd(P.wl_count + 3 + which, 1);
  return i < P.wl_count[which] ? wl_list(P, which)[i] : -1;
}

// The same for one warp (lane 0 takes the item, a shuffle broadcasts it).
__device__ inline int wl_next_warp(const ProblemDev& P, int which) {
  int item = -1;
  if ((threadIdx.x & 31) == 0) {
    const int i = atomicAdd(P.wl_count + 3 + which, 1);
    item = i < P.wl_count[which] ? wl_list(P, which)[i] : -1;
  }
  return __shfl_sync(0xffffffffu, item, 0);
}

// Work flags per source.
constexpr int FLAG_FULL = 1;     // evaluate value + gradient + Hessian
constexpr int FLAG_VALUE = 2;    // evaluate value only (trial point)

// Error words.
constexpr int ERR_BAD_PIXEL = 0;
constexpr int ERR_TIMEOUT = 1;

// Budget of a bounded wait on a bulk copy: ~2 s of SM clock.  A copy of a few KB completes in
// microseconds; a wait that runs out means the copy engine is stuck or the phase is wrong.
constexpr long long WAIT_BUDGET_DEFAULT = 4000000000LL;

// -------------------------------------------------------------------------------- small math
__host__ __device__ inline double sigmoid_d(double x) {
  return x >= 0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}

// Symmetric 2x2 stored as (00, 01, 11), and a general 2x2, in float (the kernels' arithmetic) or
// double (the table kernel's path for ill-conditioned galaxy components).
template <class T>
struct Sym2T {
  T a, b, c;
};
template <class T>
struct Mat2T {
  T m00, m01, m10, m11;
};
using Sym2 = Sym2T<float>;
using Mat2 = Mat2T<float>;

template <class T>
__device__ inline Mat2T<T> mul(const Sym2T<T>& x, const Sym2T<T>& y) {
  return {x.a * y.a + x.b * y.b, x.a * y.b + x.b * y.c, x.b * y.a + x.c * y.b, x.b * y.b + x.c * y.c};
}
template <class T>
__device__ inline Mat2T<T> mul(const Mat2T<T>& x, const Sym2T<T>& y) {
  return {x.m00 * y.a + x.m01 * y.b, x.m00 * y.b + x.m01 * y.c, x.m10 * y.a + x.m11 * y.b, x.m10 * y.b + x.m11 * y.c};
}
template <class T>
__device__ inline Mat2T<T> mul(const Mat2T<T>& x, const Mat2T<T>& y) {
  return {x.m00 * y.m00 + x.m01 * y.m10, x.m00 * y.m01 + x.m01 * y.m11, x.m10 * y.m00 + x.m11 * y.m10,
          x.m10 * y.m01 + x.m11 * y.m11};
}
template <class T>
__device__ inline T trace(const Mat2T<T>& x) { return x.m00 + x.m11; }
// symmetric part of x + x^T stored as Sym2
template <class T>
__device__ inline Sym2T<T> sym_plus_t(const Mat2T<T>& x) { return {T(2) * x.m00, x.m01 + x.m10, T(2) * x.m11}; }
template <class T>
__device__ inline Sym2T<T> to_sym(const Mat2T<T>& x) { return {x.m00, T(0.5) * (x.m01 + x.m10), x.m11}; }
// A S A^T for a general 2x2 A (row-major a00 a01 a10 a11)
template <class T>
__device__ inline Sym2T<T> congruence(const T A[4], const Sym2T<T>& S) {
  T t00 = A[0] * S.a + A[1] * S.b, t01 = A[0] * S.b + A[1] * S.c;
  T t10 = A[2] * S.a + A[3] * S.b, t11 = A[2] * S.b + A[3] * S.c;
  return {t00 * A[0] + t01 * A[1], t10 * A[0] + t11 * A[1], t10 * A[2] + t11 * A[3]};
}

// PSF component c of a patch: weight, mean (pixels), covariance.
struct PsfComp {
  float w, mx, my;
  Sym2 S;
};
__device__ inline PsfComp load_psf(const float* psf_patch, int k) {
  const float* q = psf_patch + 6 * k;
  return {q[0], q[1], q[2], {q[3], q[4], q[5]}};
}

// Brightness parameter indices of type t (r1, rho, c1 x4, gamma x4).  In band b the log flux of
// type t is normal, log l_b ~ N(m, v) with m = r1 + a_b.c1 and v = exp(rho) + (a_b^2).exp(gam), so
// E[l] = exp(m + v/2) and E[l^2] = exp(2m + 2v).
__device__ inline int bvar(int type, int v) {
  if (v == 0) return type ? 9 : 7;
  if (v == 1) return type ? 10 : 8;
  if (v < 6) return (type ? 19 : 11) + (v - 2);
  return (type ? 23 : 15) + (v - 6);
}

// Inverse of bvar for a brightness parameter index j >= 7: type and variable number.
__device__ inline void bvar_inv(int j, int& t, int& v) {
  t = (j == 9 || j == 10 || j >= 19) ? 1 : 0;
  if (j == 7 || j == 9) v = 0;
  else if (j == 8 || j == 10) v = 1;
  else if (j < 15) v = 2 + (j - 11);
  else if (j < 19) v = 6 + (j - 15);
  else if (j < 23) v = 2 + (j - 19);
  else v = 6 + (j - 23);
}

// a_bj in {-1, 0, 1}: u = r - c1 - c2, g = r - c2, r, i = r + c3, z = r + c3 + c4 (log fluxes; no
// table, so a run-time band indexes no local memory).
__host__ __device__ inline double color_coef(int band, int j) {
  return (band < 2 && j >= band && j < 2) ? -1.0 : ((band > 2 && j >= 2 && j < band) ? 1.0 : 0.0);
}
__host__ __device__ inline void color_row(int band, double a[4]) {
  for (int j = 0; j < 4; ++j) a[j] = color_coef(band, j);
}

// float64 -> float32 saturating at the float32 maximum (NaN stays NaN).  A brightness moment can
// exceed float32's range where a type's probability has all but vanished: its brightness
// parameters then barely move the objective, and Newton may carry their variance far out.  An
// infinite constant would turn the profile's zeros far from the source into inf * 0 = NaN.
__host__ __device__ inline float sat_f(double x) { return (float)(x > 3.4028234663852886e38 ? 3.4028234663852886e38 : x); }

// Galaxy world covariance Sigma_g = scale^2 R diag(1, axis^2) R^T and its first/second
// derivatives w.r.t. (logit axis, angle, log scale); pairs ordered 00 01 02 11 12 22.
template <class T>
struct GalShapeT {
  Sym2T<T> S, d[3], d2[6];
};
using GalShape = GalShapeT<float>;
__device__ inline Sym2 inv2(const Sym2& S, float& logdet) {
  // det = a c - b^2 with the rounding of b^2 compensated (one FMA recovers its exact error)
  const float bb = S.b * S.b;
  const float det = fmaf(S.a, S.c, -bb) - fmaf(S.b, S.b, -bb);
  logdet = logf(det);
  float r = 1.f / det;
  return {S.c * r, -S.b * r, S.a * r};
}

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LOG_2PI = 1.8378770664093453f;

// Position of the source in image pixels relative to (ox, oy), in float64.
__device__ inline void source_pixel_pos(const ImageDev& im, const double* th, double ox, double oy, double& px, double& py) {
  px = im.A[0] * th[0] + im.A[1] * th[1] + im.o[0] - ox;
  py = im.A[2] * th[0] + im.A[3] * th[1] + im.o[1] - oy;
}

// Weight times Gaussian normaliser, w / (2 pi sqrt(det)): a few correctly rounded float32 steps
// (det with its b^2 rounding compensated), ~2 ulp in all.
__device__ inline float gauss_weight(float w, const Sym2& S) {
  const float bb = S.b * S.b;
  const float det = fmaf(S.a, S.c, -bb) - fmaf(S.b, S.b, -bb);
  return w / (6.2831853071795865f * sqrtf(det));
}

// Bounded wait on an mbarrier phase (returns false if the budget ran out).
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t phase, long long budget_cycles) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(phase)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > budget_cycles) return false;
  }
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before later async-proxy
// (bulk copy) accesses; issued before a bulk copy overwrites a buffer that was just read.
__device__ inline void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on `bar` expecting `bytes` of asynchronous copies to complete on it.
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}

// One-dimensional bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst/src 16-byte aligned, bytes a multiple of 16.
__device__ inline void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(src), "r"(bytes), "r"(b)
               : "memory");
}

// Asynchronous global -> shared copies of 4, 8 or 16 bytes (naturally aligned), no registers
// involved; cp_async_wait_all waits for every group this thread committed.
template <int BYTES>
__device__ inline void cp_async(void* dst, const void* src) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace celeste
