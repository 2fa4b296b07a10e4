// Per-(source, image) tables for the pixel kernels, computed once per evaluation and patch.
//
// For the source's current parameters, each of the 45 profile components of the patch (3 star =
// PSF components; 42 galaxy = 3 PSF x (6 exponential + 8 de Vaucouleurs) mixture components) gets
// its precision matrix and weighted normaliser and, for the galaxy components, the first and second
// derivatives of both w.r.t. (logit axis ratio, angle, log scale):
//   Sigma_kj = tau_j A Sigma_g A^T + S_k,   P = Sigma^-1,
//   dP = -P dSigma P,  d2P = P dSa P dSb P + P dSb P dSa P - P d2S P,
//   d logdet = tr(P dSigma),  d2 logdet = tr(P d2S) - tr(P dSa P dSb),
// with Sigma_g = scale^2 R(angle) diag(1, axis^2) R(angle)^T (the galaxy shape of the paper's
// Sec. "The Celeste Model") mapped to pixels by the WCS matrix A.  Also the per-patch brightness
// constants (lognormal moments of the band flux times the type probabilities).
#include <algorithm>

#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

// Galaxy shape derivatives in float32 from float64 parameters (angle reduced first).
__device__ inline void galaxy_shape_f(double eta, double phi, double kappa, GalShape& g) {
  const double two_pi = 6.283185307179586;
  const float ph = (float)(phi - two_pi * rint(phi / two_pi));
  // e = sigmoid(eta) and 1 - e = sigmoid(-eta), each evaluated directly (no cancellation in 1 - e)
  const float e = 1.f / (1.f + expf(-(float)eta)), em = 1.f / (1.f + expf((float)eta)), e2 = e * e;
  const float s2 = expf(2.f * (float)kappa);
  float sn, c;
  sincosf(ph, &sn, &c);
  Sym2 A = {c * c, c * sn, sn * sn};
  Sym2 B = {sn * sn, -c * sn, c * c};
  Sym2 dA = {-2.f * c * sn, c * c - sn * sn, 2.f * c * sn};
  Sym2 d2A = {-2.f * (c * c - sn * sn), -4.f * c * sn, 2.f * (c * c - sn * sn)};
  float de2 = 2.f * e2 * em;
  float d2e2 = 2.f * e2 * em * (2.f - 3.f * e);
  g.S = {s2 * (A.a + e2 * B.a), s2 * (A.b + e2 * B.b), s2 * (A.c + e2 * B.c)};
  g.d[0] = {s2 * de2 * B.a, s2 * de2 * B.b, s2 * de2 * B.c};
  float k1 = s2 * em * (1.f + e);   // s2 (1 - e^2)
  g.d[1] = {k1 * dA.a, k1 * dA.b, k1 * dA.c};
  g.d[2] = {2.f * g.S.a, 2.f * g.S.b, 2.f * g.S.c};
  g.d2[0] = {s2 * d2e2 * B.a, s2 * d2e2 * B.b, s2 * d2e2 * B.c};
  g.d2[1] = {-s2 * de2 * dA.a, -s2 * de2 * dA.b, -s2 * de2 * dA.c};
  g.d2[2] = {2.f * g.d[0].a, 2.f * g.d[0].b, 2.f * g.d[0].c};
  g.d2[3] = {k1 * d2A.a, k1 * d2A.b, k1 * d2A.c};
  g.d2[4] = {2.f * g.d[1].a, 2.f * g.d[1].b, 2.f * g.d[1].c};
  g.d2[5] = {4.f * g.S.a, 4.f * g.S.b, 4.f * g.S.c};
}

// The same derivatives in float64, for components whose covariance is ill-conditioned (below).
__device__ inline void galaxy_shape_d(double eta, double phi, double kappa, GalShapeT<double>& g) {
  const double e = sigmoid_d(eta), em = sigmoid_d(-eta), e2 = e * e;
  const double s2 = exp(2.0 * kappa);
  double sn, c;
  sincos(phi, &sn, &c);
  const Sym2T<double> A = {c * c, c * sn, sn * sn};
  const Sym2T<double> B = {sn * sn, -c * sn, c * c};
  const Sym2T<double> dA = {-2.0 * c * sn, c * c - sn * sn, 2.0 * c * sn};
  const Sym2T<double> d2A = {-2.0 * (c * c - sn * sn), -4.0 * c * sn, 2.0 * (c * c - sn * sn)};
  const double de2 = 2.0 * e2 * em, d2e2 = 2.0 * e2 * em * (2.0 - 3.0 * e);
  g.S = {s2 * (A.a + e2 * B.a), s2 * (A.b + e2 * B.b), s2 * (A.c + e2 * B.c)};
  g.d[0] = {s2 * de2 * B.a, s2 * de2 * B.b, s2 * de2 * B.c};
  const double k1 = s2 * em * (1.0 + e);   // s2 (1 - e^2)
  g.d[1] = {k1 * dA.a, k1 * dA.b, k1 * dA.c};
  g.d[2] = {2.0 * g.S.a, 2.0 * g.S.b, 2.0 * g.S.c};
  g.d2[0] = {s2 * d2e2 * B.a, s2 * d2e2 * B.b, s2 * d2e2 * B.c};
  g.d2[1] = {-s2 * de2 * dA.a, -s2 * de2 * dA.b, -s2 * de2 * dA.c};
  g.d2[2] = {2.0 * g.d[0].a, 2.0 * g.d[0].b, 2.0 * g.d[0].c};
  g.d2[3] = {k1 * d2A.a, k1 * d2A.b, k1 * d2A.c};
  g.d2[4] = {2.0 * g.d[1].a, 2.0 * g.d[1].b, 2.0 * g.d[1].c};
  g.d2[5] = {4.0 * g.S.a, 4.0 * g.S.b, 4.0 * g.S.c};
}

__device__ inline Sym2T<double> inv2(const Sym2T<double>& S, double& logdet) {
  const double det = S.a * S.c - S.b * S.b;
  logdet = log(det);
  const double r = 1.0 / det;
  return {S.c * r, -S.b * r, S.a * r};
}
__device__ inline double gauss_weight(double w, const Sym2T<double>& S) {
  return w / (6.283185307179586 * sqrt(S.a * S.c - S.b * S.b));
}

// One galaxy component's table entry, computed in T and stored as float: precision P of
// Sigma = tau A Sigma_g A^T + S_k, weighted normaliser, and with `full` -1/2 dP, -1/2 d logdet and
// their second derivatives over (axis, angle, scale).
template <class T>
__device__ inline void gal_entry(const GalShapeT<T>& gs, const T A[4], const Sym2T<T>& Sk, T w, T tau, bool full,
                                 float* e) {
  const Sym2T<T> Sp = congruence(A, gs.S);
  const Sym2T<T> S = {tau * Sp.a + Sk.a, tau * Sp.b + Sk.b, tau * Sp.c + Sk.c};
  T ld;
  const Sym2T<T> Pm = inv2(S, ld);
  e[GT_P + 0] = (float)Pm.a;
  e[GT_P + 1] = (float)Pm.b;
  e[GT_P + 2] = (float)Pm.c;
  e[GT_W] = (float)gauss_weight(w, S);
  if (!full) return;
  e[GT_PZ + 0] = (float)Pm.b;
  e[GT_PZ + 1] = (float)Pm.c;
  e[GT_LA2 + 1] = 0.f;
  Mat2T<T> PdS[3];
  for (int a = 0; a < 3; ++a) {
    const Sym2T<T> t = congruence(A, gs.d[a]);
    PdS[a] = mul(Pm, Sym2T<T>{tau * t.a, tau * t.b, tau * t.c});
    const Sym2T<T> dP = to_sym(mul(PdS[a], Pm));   // P dS P = -dP/da
    e[gt_qa(a, 0)] = (float)(T(0.5) * dP.a);
    e[gt_qa(a, 1)] = (float)(T(0.5) * dP.b);
    e[gt_qa(a, 2)] = (float)(T(0.5) * dP.c);
    if (a == 2) e[GT_Q2 + 2] = (float)(T(0.5) * dP.b);   // Q_2[01], second copy
    e[gt_la(a)] = (float)(T(-0.5) * trace(PdS[a]));
  }
  int q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++q) {
      const Sym2T<T> t = congruence(A, gs.d2[q]);
      const Sym2T<T> d2S = {tau * t.a, tau * t.b, tau * t.c};
      const Mat2T<T> X = mul(PdS[a], PdS[b]);
      const Sym2T<T> two = sym_plus_t(mul(X, Pm));
      const Mat2T<T> Pd2 = mul(Pm, d2S);
      const Sym2T<T> third = to_sym(mul(Pd2, Pm));
      e[gt_qab(q, 0)] = (float)(T(-0.5) * (two.a - third.a));
      e[gt_qab(q, 1)] = (float)(T(-0.5) * (two.b - third.b));
      e[gt_qab(q, 2)] = (float)(T(-0.5) * (two.c - third.c));
      e[gt_lab(q)] = (float)(T(-0.5) * (trace(Pd2) - trace(X)));
    }
}

// Brightness constants of every listed source for all five bands, in float64.  One warp per
// source: lane 5t + b (t = type, b = band, lanes 0-9) evaluates the lognormal moments of l_b for
// type t, lanes 0-4 then combine both types for band b.  Spreading the transcendental functions
// over the lanes keeps the count of float64 warp instructions (each ~64 cycles here) per source
// low; the tables below only copy the result.
__global__ void source_const_kernel(ProblemDev P, const double* __restrict__ theta) {
  const int lane = threadIdx.x & 31;
  const int n = P.wl_count[WL_SOURCES];
  const int* items = wl_list(P, WL_SOURCES);
  const int nw = gridDim.x * (blockDim.x >> 5);
  const int t = lane < 5 ? 0 : 1, b = lane % 5;   // meaningful for lanes < 10
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n; w += nw) {   // warp-uniform
    const int s = items[w];
    const double* th = theta + (size_t)s * NP;
    // exp of the log-variances, lane 5t + k: k = 0 log flux, k = 1..4 colours j = k - 1
    double ev = 0.0;
    if (lane < 10) {
      const int k = lane % 5;
      ev = exp(th[k == 0 ? (t ? 10 : 8) : (t ? 23 : 15) + k - 1]);
    }
    double evk[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) evk[k] = __shfl_sync(0xffffffffu, ev, 5 * t + k);
    double a[4];
    color_row(b, a);
    double m = th[t ? 9 : 7], v = evk[0];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m = fma(a[j], th[(t ? 19 : 11) + j], m);
      v = fma(a[j] * a[j], evk[1 + j], v);
    }
    double L1 = 0.0, L2 = 0.0, em = 0.0;
    if (lane < 10) {
      L1 = exp(m + 0.5 * v);
      L2 = exp(2.0 * m + 2.0 * v);
      em = expm1(v);
    }
    const double L10 = __shfl_sync(0xffffffffu, L1, b), L20 = __shfl_sync(0xffffffffu, L2, b);
    const double em0 = __shfl_sync(0xffffffffu, em, b);
    const double L11 = __shfl_sync(0xffffffffu, L1, 5 + b), L21 = __shfl_sync(0xffffffffu, L2, 5 + b);
    const double em1 = __shfl_sync(0xffffffffu, em, 5 + b);
    if (lane < 5) {
      const double a1 = sigmoid_d(th[6]), a0 = sigmoid_d(-th[6]), aa = a0 * a1;
      const double e = sigmoid_d(th[2]), ee = e * sigmoid_d(-th[2]);
      SNConst c;
      c.C0 = sat_f(a0 * L10 * L10 * em0);
      c.C1 = sat_f(a1 * L11 * L11 * em1);
      c.Cx = (float)aa;
      c.L10 = sat_f(L10);
      c.L11 = sat_f(L11);
      c.A0 = sat_f(a0 * L10);
      c.A1 = sat_f(a1 * L11);
      c.B0 = sat_f(a0 * L20);
      c.B1 = sat_f(a1 * L21);
      c.aE0 = sat_f(aa * L10);
      c.aE1 = sat_f(aa * L11);
      c.aV0 = sat_f(aa * L20);
      c.aV1 = sat_f(aa * L21);
      c.iota = 0.f;
      c.e = (float)e;
      c.e1 = (float)ee;
      c.e2 = (float)(ee * (1.0 - 2.0 * e));
      P.snc[(size_t)s * 5 + b] = c;
    }
  }
}

// full = 1: galaxy derivative entries too; full = 0: precision and normaliser only.
// 64-thread CTAs taking patches from the device work queue over the patch worklist.
__global__ void __launch_bounds__(64) table_kernel(ProblemDev P, const double* __restrict__ theta, int full) {
  __shared__ int slot;
  const int tid = threadIdx.x;
  for (int patch = wl_next_cta(P, WL_PATCHES, slot); patch >= 0; patch = wl_next_cta(P, WL_PATCHES, slot)) {
  const PatchDev pt = P.patches[patch];
  const ImageDev im = P.images[pt.image];
  const double* th = theta + (size_t)pt.source * NP;
  float* out = P.ptab + (size_t)patch * TB_FLOATS;
  const float* psf = P.psf + (size_t)patch * 18;
  if (tid < NGAL) {
    const int k = tid / NMIX, j = tid % NMIX;
    const PsfComp pc = load_psf(psf, k);
    GalShape gs;
    galaxy_shape_f(th[3], th[4], th[5], gs);
    const float A[4] = {(float)im.A[0], (float)im.A[1], (float)im.A[2], (float)im.A[3]};
    const float tau = P.tau[j], nu = P.nu[j];
    float* e = out + TB_GAL + tid * GT_STRIDE;
    // A long, thin galaxy (axis ratio ~1e-4, radius ~1e3 px) gives Sigma entries ~1e6 whose
    // determinant cancels to ~1e-6 of a c: float32 would leave P and its shape derivatives with a
    // few correct bits.  Where a c exceeds 16 det such a component is built in float64.
    const Sym2 Sp = congruence(A, gs.S);
    const Sym2 S = {tau * Sp.a + pc.S.a, tau * Sp.b + pc.S.b, tau * Sp.c + pc.S.c};
    const float bb = S.b * S.b;
    const float det = fmaf(S.a, S.c, -bb) - fmaf(S.b, S.b, -bb);
    if (S.a * S.c <= 16.f * det) {
      gal_entry<float>(gs, A, pc.S, pc.w * nu, tau, full != 0, e);
    } else {
      GalShapeT<double> gd;
      galaxy_shape_d(th[3], th[4], th[5], gd);
      const double Ad[4] = {im.A[0], im.A[1], im.A[2], im.A[3]};
      gal_entry<double>(gd, Ad, Sym2T<double>{pc.S.a, pc.S.b, pc.S.c}, (double)pc.w * nu, (double)tau, full != 0, e);
    }
    // the value-only copy, interleaved with the other component of its pair
    float* v = out + TB_VAL + 8 * (tid / 2) + (j & 1);
    v[0] = e[GT_P];
    v[2] = e[GT_P + 1];
    v[4] = e[GT_P + 2];
    v[6] = e[GT_W];
  } else if (tid < NGAL + NSTAR) {
    const int k = tid - NGAL;
    const PsfComp pc = load_psf(psf, k);
    double px, py;
    source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
    float ld;
    const Sym2 Pm = inv2(pc.S, ld);
    out[TB_MU + 2 * k + 0] = (float)(px + pc.mx);
    out[TB_MU + 2 * k + 1] = (float)(py + pc.my);
    out[TB_STAR + 4 * k + 0] = gauss_weight(pc.w, pc.S);
    out[TB_STAR + 4 * k + 1] = Pm.a;
    out[TB_STAR + 4 * k + 2] = Pm.b;
    out[TB_STAR + 4 * k + 3] = Pm.c;
  } else if (tid == NGAL + NSTAR) {
    SNConst c = P.snc[(size_t)pt.source * 5 + im.band];
    c.iota = im.iota;
    const float* cf = reinterpret_cast<const float*>(&c);
    for (int q = 0; q < (int)(sizeof(SNConst) / sizeof(float)); ++q) out[TB_SNC + q] = cf[q];
  }
  }
}

cudaError_t launch_tables(const ProblemDev& P, const double* theta, bool full, cudaStream_t st) {
  if (P.n_patches == 0) return cudaSuccess;
  source_const_kernel<<<std::max(1, std::min((P.S + 3) / 4, P.n_sm * 8)), 128, 0, st>>>(P, theta);
  const int blocks = std::max(1, std::min(P.n_patches, P.n_sm * 16));
  table_kernel<<<blocks, 64, 0, st>>>(P, theta, full ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace celeste
