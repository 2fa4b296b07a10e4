// Assembly of each source's ELBO, gradient and Hessian from the per-tile pixel sums,
// plus the KL term of q (paper, Sec. "Variational Inference": Eq. (1)-(3); q(a) Bernoulli,
// q(r|a) lognormal, q(c|a) normal, each conjugate to its prior).
//
// Work in the "E-space" of a patch: the 27 parameters with the world position u replaced by
// the pixel-space mean mu = A u + o (so the pixel sums need no WCS); the u rows/columns are
// mapped back with A before summing over the source's images.
//
// A float64 warp instruction occupies its SM sub-partition's FP64 pipe for ~64 cycles on this
// part, whatever the number of active lanes, so every transcendental is evaluated once per source
// and in parallel across threads, and only the objective and gradient are lifted in float64.
#include <algorithm>

#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

__device__ constexpr int tri11d(int i, int j) { return i * 11 - i * (i - 1) / 2 + (j - i); }

// One normal-KL term of type t: k = 0 the log flux, k = 1..4 the colours j = k - 1, with v the
// exp of its log-variance parameter.
// KL_N(m, v || mu, s2) = (log s2 - log v + (v + (m - mu)^2) / s2 - 1) / 2.
__device__ inline double kl_normal_term(const double* th, double v, const ProblemDev& P, int t, int k) {
  const double m = k == 0 ? th[bvar(t, 0)] : th[bvar(t, 1 + k)];
  const double lv = k == 0 ? th[bvar(t, 1)] : th[bvar(t, 5 + k)];
  const double mu = k == 0 ? P.priors[1] : P.priors[3], is2 = k == 0 ? P.inv_var_r : P.inv_var_c;
  const double ls2 = k == 0 ? P.log_var_r : P.log_var_c;
  return 0.5 * (ls2 - lv + (v + (m - mu) * (m - mu)) * is2 - 1.0);
}

// Per-source quantities shared by the source's patches, for all five bands: the type
// probabilities, the band moments of the lognormal flux and their derivatives over the type's
// brightness parameters, and the KL term with its derivatives.  Built once per source by the
// whole CTA, so a patch's lift needs no transcendental and almost no float64 arithmetic.
struct SrcTab {
  double ev[2][10];                       // exp of the log-variance parameters (v = 1, 6..9), 0 elsewhere
  double a0, a1, aa, la0, la1;            // P(star), P(galaxy), their product, their logs
  double L1[2][5], L2[2][5];              // E[l_b | t], E[l_b^2 | t]
  double gc[5][8];                        // per band: a0 L1_0, a1 L1_1, a0 L2_0, a1 L2_1, aa x (L1_0, L1_1, L2_0, L2_1)
  double kd1[2][5][10], kd2[2][5][10];    // a_t dL1_t / d(brightness v), a_t dL2_t / d(v): the lift's coefficients
  double klg[NP], klhd[NP], klh6[NP];     // KL gradient; KL Hessian diagonal and row (= column) 6
  double kterm[10], kl;                   // the ten normal-KL terms; the KL
  float fL1[2][5], fL2[2][5];
  float kf1[2][5][10], kf2[2][5][10];     // kd1, kd2
  float fdL1[2][5][10], fdL2[2][5][10];   // dL1, dL2
  float fdl1[2][5][10], fdl2[2][5][10];   // d log L1, d log L2
  float fd2l1[2][5][10], fd2l2[2][5][10]; // diagonal second derivatives of log L1, log L2
  float fa0, fa1, faa;
};

// Builds the source table (every thread of the CTA calls it; ends with a barrier).
__device__ inline void build_src_tab(const ProblemDev& P, const double* __restrict__ th, SrcTab& T, int tid) {
  // ---- exps of the log-variances (warp 0), type probabilities (warp 1), zeros (warp 2)
  if (tid < 10) {
    const int t = tid / 5, k = tid % 5, v = k == 0 ? 1 : 5 + k;
    T.ev[t][v] = exp(th[bvar(t, v)]);
  } else if (tid == 32) {
    const double al = th[6];
    const double e = exp(-fabs(al)), l1p = log1p(e);
    T.la1 = al >= 0 ? -l1p : al - l1p;   // log sigmoid(alpha)
    T.la0 = T.la1 - al;                  // log sigmoid(-alpha)
    const double sg = 1.0 / (1.0 + e);
    T.a1 = al >= 0 ? sg : e * sg;
    T.a0 = al >= 0 ? e * sg : sg;
    T.aa = T.a0 * T.a1;
    T.fa0 = (float)T.a0;
    T.fa1 = (float)T.a1;
    T.faa = (float)T.aa;
  } else if (tid >= 64 && tid < 74) {
    const int k = tid - 64, t = k / 5, kk = k % 5, v = kk == 0 ? 0 : kk + 1;   // v = 0, 2..5
    T.ev[t][v] = 0.0;
  }
  __syncthreads();
  // ---- band moments (warp 0), KL derivative tables (warp 1), normal-KL terms (warp 2)
  if (tid < 20) {
    const int t = tid / 10, b = (tid >> 1) % 5, which = tid & 1;
    double m = th[bvar(t, 0)], v = T.ev[t][1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double c = color_coef(b, j);
      m = fma(c, th[bvar(t, 2 + j)], m);
      v = fma(c * c, T.ev[t][6 + j], v);
    }
    const double L = which ? exp(2.0 * m + 2.0 * v) : exp(m + 0.5 * v);
    if (which) {
      T.L2[t][b] = L;
      T.fL2[t][b] = (float)L;
    } else {
      T.L1[t][b] = L;
      T.fL1[t][b] = (float)L;
    }
  } else if (tid >= 32 && tid < 32 + NP) {
    // dK_t/dth_j and d2K_t/dth_j^2 of the normal-KL sum K_t of j's type (closed forms); row 6
    // (alpha) is set once K_0 and K_1 are known
    const int j = tid - 32;
    double g = 0.0, hd = 0.0, h6 = 0.0;
    if (j >= 7) {
      int t, v;
      bvar_inv(j, t, v);
      const double is2 = v <= 1 ? P.inv_var_r : P.inv_var_c;
      double dK, d2K;
      if (v == 0 || (v >= 2 && v < 6)) {
        dK = (th[j] - (v == 0 ? P.priors[1] : P.priors[3])) * is2;
        d2K = is2;
      } else {
        d2K = 0.5 * T.ev[t][v] * is2;
        dK = d2K - 0.5;
      }
      const double at = t ? T.a1 : T.a0;
      g = at * dK;
      hd = at * d2K;
      h6 = (t ? T.aa : -T.aa) * dK;
    }
    if (j != 6) {
      T.klg[j] = g;
      T.klhd[j] = hd;
      T.klh6[j] = h6;
    }
  } else if (tid >= 64 && tid < 74) {
    const int k = tid - 64, t = k / 5, kk = k % 5;
    T.kterm[k] = kl_normal_term(th, T.ev[t][kk == 0 ? 1 : 5 + kk], P, t, kk);
  }
  __syncthreads();
  // ---- derivatives of the band moments (items 0..199), the gradient coefficients per band
  //      (200..239); the last thread adds up the KL and its alpha row
  for (int i = tid; i < 240; i += blockDim.x) {
    if (i < 200) {
      const int t = i / 100, b = (i / 20) % 5, which = (i / 10) & 1, v = i % 10;
      const bool var = v == 1 || v >= 6;
      double c = v < 2 ? 1.0 : color_coef(b, (v - 2) & 3);
      if (v >= 6) c *= c;
      const double dl = (which ? 2.0 : (var ? 0.5 : 1.0)) * c * (var ? T.ev[t][v] : 1.0);   // d log L
      const double L = which ? T.L2[t][b] : T.L1[t][b];
      const double dL = L * dl, kd = (t ? T.a1 : T.a0) * dL;
      if (which) {
        T.kd2[t][b][v] = kd;
        T.kf2[t][b][v] = (float)kd;
        T.fdL2[t][b][v] = (float)dL;
        T.fdl2[t][b][v] = (float)dl;
        T.fd2l2[t][b][v] = var ? (float)dl : 0.f;
      } else {
        T.kd1[t][b][v] = kd;
        T.kf1[t][b][v] = (float)kd;
        T.fdL1[t][b][v] = (float)dL;
        T.fdl1[t][b][v] = (float)dl;
        T.fd2l1[t][b][v] = var ? (float)dl : 0.f;
      }
    } else {
      const int b = (i - 200) >> 3, k = (i - 200) & 7, t = k & 1;
      const double L = (k & 2) ? T.L2[t][b] : T.L1[t][b];
      T.gc[b][k] = (k < 4 ? (t ? T.a1 : T.a0) : T.aa) * L;
    }
  }
  if (tid == blockDim.x - 1) {
    // KL = a1 (log a1 - log Phi) + a0 (log a0 - log(1 - Phi)) + a0 K_0 + a1 K_1
    double K0 = 0.0, K1 = 0.0;
    for (int i = 0; i < 5; ++i) {
      K0 += T.kterm[i];
      K1 += T.kterm[5 + i];
    }
    const double dlg = th[6] - P.logit_phi, dK = K1 - K0, s = 1.0 - 2.0 * T.a1;
    T.kl = T.a1 * (T.la1 - P.log_phi) + T.a0 * (T.la0 - P.log1m_phi) + T.a0 * K0 + T.a1 * K1;
    T.klg[6] = T.aa * dlg + T.aa * dK;
    T.klhd[6] = T.aa * (s * dlg + 1.0) + T.aa * s * dK;
    T.klh6[6] = 0.0;
  }
  __syncthreads();
}

// Per-warp working set of one patch's lift.
struct WarpLift {
  double sd[ACC_HP];                                  // float64 sums: L, S1, S2
  double gs[NP], gE[NP], nzK[NP], nzL[NP], ghat[NRED];
  double A[4];                                        // the image's WCS linear part
  double Lsum;
  float sdf[ACC_HP], sf[NACC - ACC_HP];               // float32 copies / compensated sums: HP, M
  float Hs[NP * NP], H2[NP * NP];                     // accumulated Hessian; per-patch second-order part
  float Msym[NRED * NRED], nzKf[NP], nzLf[NP], Af[4];
  int nzA[NP], nzB[NP];
};

// ELBO and gradient are summed and lifted in float64 (the cross-pixel sums of the objective and
// its gradient); the Hessian, whose per-pixel terms are float32 to begin with, in float32 with
// compensated cross-tile sums.  On this part a float64 warp instruction costs ~64 cycles of its
// SM sub-partition and a float32 one a single issue slot, so every transcendental and every
// derivative of the band moments is formed once per source (SrcTab) and a patch's lift keeps
// only the sums' float64 work.  A CTA takes one source; each of its four warps lifts every
// fourth patch of the source into warp-private accumulators (the four sub-partitions' float64
// pipes run in parallel), then the warps' sums are added.
__global__ void __launch_bounds__(128) assemble_kernel(ProblemDev P, const double* __restrict__ theta, int full,
                                                       double* elbo, double* grad, double* hess) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = 4;                 // warps per CTA
  constexpr int ND = ACC_HP;            // float64 sums: L, S1, S2
  constexpr int NF = NACC - ACC_HP;     // float32 sums: HP, M
  constexpr int NTRI = NP * (NP + 1) / 2;
  __shared__ WarpLift wl[NW];
  __shared__ SrcTab T;
  __shared__ float Hs[NP * NP];
  __shared__ double gs[NP];
  __shared__ double Lsum;
  __shared__ unsigned short tri[NTRI];   // packed upper triangle index -> (row << 8) | column
  __shared__ int slot;
  WarpLift& W = wl[warp];
  for (int q = tid; q < NTRI; q += nt) {
    int r = 0, rem = q;
    while (rem >= NP - r) {
      rem -= NP - r;
      ++r;
    }
    tri[q] = (unsigned short)((r << 8) | (r + rem));
  }
  for (int s = wl_next_cta(P, WL_SOURCES, slot); s >= 0; s = wl_next_cta(P, WL_SOURCES, slot)) {
  const double* th = theta + (size_t)s * NP;
  for (int i = lane; i < NP * NP; i += 32) W.Hs[i] = 0.f;
  if (lane < NP) W.gs[lane] = 0.0;
  if (lane == 0) W.Lsum = 0.0;
  build_src_tab(P, th, T, tid);
  for (int p = P.src_patch[s] + warp; p < P.src_patch[s + 1]; p += NW) {
    const PatchDev pt = P.patches[p];
    const ImageDev& im = P.images[pt.image];
    const int b = im.band;
    // ---- tile sums (fixed order; float64 for the objective and gradient, compensated float32 for
    //      the Hessian-only sums)
    if (lane < ND) {
      double v = 0.0;
      const float* src = P.partials + lane;
#pragma unroll 4
      for (int t = pt.tile_begin; t < pt.tile_end; ++t) v += (double)src[(size_t)t * NACC];
      W.sd[lane] = v;
      W.sdf[lane] = (float)v;
    } else if (lane < ND + 4) {
      const double a = im.A[lane - ND];
      W.A[lane - ND] = a;
      W.Af[lane - ND] = (float)a;
    }
    for (int q = lane; q < NF; q += 32) {
      float v = 0.f, comp = 0.f;
      const float* src = P.partials + ND + q;
#pragma unroll 4
      for (int t = pt.tile_begin; t < pt.tile_end; ++t) {
        const float y = src[(size_t)t * NACC] - comp;
        const float u = v + y;
        comp = (u - v) - y;
        v = u;
      }
      W.sf[q] = v;
    }
    __syncwarp();
    if (lane == 0) W.Lsum += W.sd[ACC_L];
    const double* S1 = W.sd + ACC_S1;
    const double* S2 = W.sd + ACC_S2;
    const float* S1h = W.sdf + ACC_S1;
    const float* S2h = W.sdf + ACC_S2;
    // ---- reduced gradient (float64): ghat_a = c0 S1[i0] + c1 S1[i1] + c2 S2[i0] + c3 S2[i1]
    if (lane < NRED) {
      const int a = lane;
      const double* g = T.gc[b];
      int i0 = 0, i1 = 3;
      double c0, c1, c2, c3;
      if (a < 2) {
        i0 = 1 + a;
        i1 = 4 + a;
        c0 = g[0];
        c1 = g[1];
        c2 = g[2];
        c3 = g[3];
      } else if (a < 6) {
        i1 = 4 + a;
        c0 = 0.0;
        c1 = g[1];
        c2 = 0.0;
        c3 = g[3];
      } else if (a == 6) {
        c0 = -g[4];
        c1 = g[5];
        c2 = -g[6];
        c3 = g[7];
      } else {
        c0 = a == 7 ? 1.0 : 0.0;
        c1 = a == 8 ? 1.0 : 0.0;
        c2 = a == 9 ? 1.0 : 0.0;
        c3 = a == 10 ? 1.0 : 0.0;
      }
      W.ghat[a] = fma(c0, S1[i0], fma(c1, S1[i1], fma(c2, S2[i0], c3 * S2[i1])));
    }
    // Lift from the 11-column reduced basis to the 27 parameters: column j of K has at most two
    // nonzeros (a, k): j < 7 -> (j, 1); brightness parameter v of type t -> (7 + t, a_t dL1_t[v])
    // from the E-row and (9 + t, a_t dL2_t[v]) from the V-row.  H_E = K^T M K + H2, g_E = K^T ghat.
    if (lane < NP) {
      const int j = lane;
      if (j < 7) {
        W.nzA[j] = j;
        W.nzB[j] = -1;
        W.nzK[j] = 1.0;
        W.nzL[j] = 0.0;
        W.nzKf[j] = 1.f;
        W.nzLf[j] = 0.f;
      } else {
        int t, v;
        bvar_inv(j, t, v);
        W.nzA[j] = 7 + t;
        W.nzB[j] = 9 + t;
        W.nzK[j] = T.kd1[t][b][v];
        W.nzL[j] = T.kd2[t][b][v];
        W.nzKf[j] = T.kf1[t][b][v];
        W.nzLf[j] = T.kf2[t][b][v];
      }
    }
    for (int i = lane; i < NRED * NRED; i += 32) {
      const int a = i / NRED, c = i % NRED;
      W.Msym[i] = W.sf[ACC_M - ND + (a <= c ? tri11d(a, c) : tri11d(c, a))];
    }
    // second-order part  sum_m w1 d2E[G] + w2 d2E[G^2] (float32), filled block by block:
    // G6 x G6 from the kernel's sums; G6 x alpha; alpha x alpha; G6 x brightness;
    // alpha x brightness; brightness x brightness (same type only)
    float* H2 = W.H2;
    for (int i = lane; i < NP * NP; i += 32) H2[i] = 0.f;
    __syncwarp();
    for (int q = lane; q < 21; q += 32) {
      int a = 0, rem = q;
      while (rem >= 6 - a) {
        rem -= 6 - a;
        ++a;
      }
      const int c = a + rem;
      H2[a * NP + c] = H2[c * NP + a] = W.sf[ACC_HP - ND + q];
    }
    const float S1f0 = S1h[0], S1f1 = S1h[3], S2f0 = S2h[0], S2f1 = S2h[3];
    const float fa0 = T.fa0, fa1 = T.fa1, faa = T.faa;
    const float L10 = T.fL1[0][b], L11 = T.fL1[1][b], L20 = T.fL2[0][b], L21 = T.fL2[1][b];
    for (int i = lane; i < 6 + 1 + 120 + 20 + 200; i += 32) {
      if (i < 6) {
        const int a = i;
        const float s1f0 = a < 2 ? S1h[1 + a] : 0.f, s2f0 = a < 2 ? S2h[1 + a] : 0.f;
        H2[a * NP + 6] = H2[6 * NP + a] = faa * (L11 * S1h[4 + a] - L10 * s1f0 + L21 * S2h[4 + a] - L20 * s2f0);
      } else if (i == 6) {
        H2[6 * NP + 6] = faa * (1.f - 2.f * fa1) * (L11 * S1f1 - L10 * S1f0 + L21 * S2f1 - L20 * S2f0);
      } else if (i < 127) {
        const int k = i - 7, t = k / 60, a = (k % 60) / 10, v = k % 10, j = bvar(t, v);
        const float s1 = t ? S1h[4 + a] : (a < 2 ? S1h[1 + a] : 0.f);
        const float s2 = t ? S2h[4 + a] : (a < 2 ? S2h[1 + a] : 0.f);
        H2[a * NP + j] = H2[j * NP + a] = (t ? fa1 : fa0) * (s1 * T.fdL1[t][b][v] + s2 * T.fdL2[t][b][v]);
      } else if (i < 147) {
        const int k = i - 127, t = k / 10, v = k % 10, j = bvar(t, v);
        H2[6 * NP + j] = H2[j * NP + 6] =
            (t ? faa : -faa) * ((t ? S1f1 : S1f0) * T.fdL1[t][b][v] + (t ? S2f1 : S2f0) * T.fdL2[t][b][v]);
      } else {
        // d2 L = L (dlogL dlogL^T + diag(d2 log L)) within a type
        const int k = i - 147, t = k / 100, v = (k % 100) / 10, w = k % 10;
        const float d2L1 = T.fL1[t][b] * (T.fdl1[t][b][v] * T.fdl1[t][b][w] + (v == w ? T.fd2l1[t][b][v] : 0.f));
        const float d2L2 = T.fL2[t][b] * (T.fdl2[t][b][v] * T.fdl2[t][b][w] + (v == w ? T.fd2l2[t][b][v] : 0.f));
        H2[bvar(t, v) * NP + bvar(t, w)] = (t ? fa1 : fa0) * ((t ? S1f1 : S1f0) * d2L1 + (t ? S2f1 : S2f0) * d2L2);
      }
    }
    __syncwarp();
    // H_E = K^T M K + H2, in place over H2 (each pair (r <= col) reads only its own upper entry)
    for (int q = lane; q < NTRI; q += 32) {
      const int rc = tri[q], r = rc >> 8, col = rc & 0xff;
      float v = W.nzKf[r] * W.nzKf[col] * W.Msym[W.nzA[r] * NRED + W.nzA[col]];
      if (W.nzB[col] >= 0) v += W.nzKf[r] * W.nzLf[col] * W.Msym[W.nzA[r] * NRED + W.nzB[col]];
      if (W.nzB[r] >= 0) {
        v += W.nzLf[r] * W.nzKf[col] * W.Msym[W.nzB[r] * NRED + W.nzA[col]];
        if (W.nzB[col] >= 0) v += W.nzLf[r] * W.nzLf[col] * W.Msym[W.nzB[r] * NRED + W.nzB[col]];
      }
      v += H2[r * NP + col];
      H2[r * NP + col] = v;
      H2[col * NP + r] = v;
    }
    if (lane < NP) {
      const int j = lane;
      W.gE[j] = W.nzK[j] * W.ghat[W.nzA[j]] + (W.nzB[j] >= 0 ? W.nzL[j] * W.ghat[W.nzB[j]] : 0.0);
    }
    __syncwarp();
    // map mu -> u: d/du_b = sum_a A[a][b] d/dmu_a
    const float* HE = H2;
    const float* Af = W.Af;
    for (int i = lane; i < NP * NP; i += 32) {
      const int r = i / NP, q = i % NP;
      float v;
      if (r < 2 && q < 2) {
        v = 0.f;
        for (int a = 0; a < 2; ++a)
          for (int c = 0; c < 2; ++c) v += Af[a * 2 + r] * Af[c * 2 + q] * HE[a * NP + c];
      } else if (r < 2) {
        v = Af[0 * 2 + r] * HE[0 * NP + q] + Af[1 * 2 + r] * HE[1 * NP + q];
      } else if (q < 2) {
        v = Af[0 * 2 + q] * HE[r * NP + 0] + Af[1 * 2 + q] * HE[r * NP + 1];
      } else {
        v = HE[i];
      }
      W.Hs[i] += v;
    }
    if (lane < NP) {
      const int j = lane;
      W.gs[j] += j < 2 ? W.A[0 * 2 + j] * W.gE[0] + W.A[1 * 2 + j] * W.gE[1] : W.gE[j];
    }
    __syncwarp();
  }
  __syncthreads();
  // ---- the warps' sums (fixed order)
  for (int i = tid; i < NP * NP; i += nt) Hs[i] = (wl[0].Hs[i] + wl[1].Hs[i]) + (wl[2].Hs[i] + wl[3].Hs[i]);
  if (tid < NP) gs[tid] = (wl[0].gs[tid] + wl[1].gs[tid]) + (wl[2].gs[tid] + wl[3].gs[tid]);
  if (tid == 0) Lsum = (wl[0].Lsum + wl[1].Lsum) + (wl[2].Lsum + wl[3].Lsum);
  __syncthreads();
  // ---- ELBO = pixel sum - KL, and the KL's derivatives (closed forms from the source table)
  if (elbo && tid == 0) elbo[s] = Lsum - T.kl;
  if (full) {
    if (hess) {
      for (int i = tid; i < NP * NP; i += nt) {
        const int r = i / NP, q = i % NP;
        const double h = (r == q ? T.klhd[r] : 0.0) + (r == 6 ? T.klh6[q] : (q == 6 ? T.klh6[r] : 0.0));
        hess[(size_t)s * NP * NP + i] = (double)Hs[i] - h;
      }
    }
    if (grad && tid < NP) grad[(size_t)s * NP + tid] = gs[tid] - T.klg[tid];
  }
  __syncthreads();   // shared state is reused by the next source
  }
}

// Value-only assembly, one warp per source: sum of the value tile sums minus the KL at theta
// (plus the KL at theta_ref when the pixel sums are differences from theta_ref).
__global__ void assemble_value_kernel(ProblemDev P, const double* __restrict__ theta, const double* __restrict__ theta_ref,
                                      double* out) {
  const int lane = threadIdx.x & 31;
  for (int s = wl_next_warp(P, WL_SOURCES); s >= 0; s = wl_next_warp(P, WL_SOURCES)) {   // warp-uniform
  double v = 0.0;
  for (int p = P.src_patch[s]; p < P.src_patch[s + 1]; ++p) {
    const PatchDev& pt = P.patches[p];
    for (int t = pt.tile_begin + lane; t < pt.tile_end; t += 32) v += (double)P.vpartials[t];
  }
  // KL terms: lanes 0..10 at theta, lanes 16..26 at theta_ref (subtracted / added)
  const int which = lane >> 4, k = lane & 15;
  const double* th = which ? theta_ref : theta;
  if (th && k <= 10) {
    th += (size_t)s * NP;   // (per-lane pointer; th is reset each source)
    const double al = th[6], e = exp(-fabs(al)), sg = 1.0 / (1.0 + e);
    const double a1 = al >= 0 ? sg : e * sg, a0 = al >= 0 ? e * sg : sg;
    double klp;
    if (k < 10) {
      const int t = k / 5, kk = k % 5;
      const double ev = exp(th[bvar(t, kk == 0 ? 1 : 5 + kk)]);
      klp = (t ? a1 : a0) * kl_normal_term(th, ev, P, t, kk);
    } else {
      const double l1p = log1p(e);
      const double la1 = al >= 0 ? -l1p : al - l1p, la0 = la1 - al;
      klp = a1 * (la1 - P.log_phi) + a0 * (la0 - P.log1m_phi);
    }
    v += which ? klp : -klp;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[s] = v;
  }
}

cudaError_t launch_assemble_value(const ProblemDev& P, const double* theta, const double* theta_ref, double* out,
                                  cudaStream_t st) {
  const int warps_per_block = 4;
  const int blocks = std::max(1, std::min((P.S + warps_per_block - 1) / warps_per_block, P.n_sm * 8));
  assemble_value_kernel<<<blocks, 32 * warps_per_block, 0, st>>>(P, theta, theta_ref, out);
  return cudaGetLastError();
}

__global__ void set_flags_kernel(int* flags, int S, int value) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) flags[s] = value;
}

// Worklists of the tiles, patches and sources whose source's flags match `mask` (warp-aggregated
// appends; the order inside a list is not significant: results are indexed by item).
__global__ void worklist_kernel(ProblemDev P, int mask) {
  int* lists[3] = {wl_list(P, WL_TILES), wl_list(P, WL_PATCHES), wl_list(P, WL_SOURCES)};
  const int lane = threadIdx.x & 31;
  const int total = P.n_tiles + P.n_patches + P.S;
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    int which = -1, item = 0;
    bool act = false;
    if (i < P.n_tiles) {
      which = WL_TILES;
      item = i;
      act = (P.flags[P.patches[P.tiles[i].patch].source] & mask) != 0;
    } else if (i < P.n_tiles + P.n_patches) {
      which = WL_PATCHES;
      item = i - P.n_tiles;
      act = (P.flags[P.patches[item].source] & mask) != 0;
    } else if (i < total) {
      which = WL_SOURCES;
      item = i - P.n_tiles - P.n_patches;
      act = (P.flags[item] & mask) != 0;
    }
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const bool mine = act && which == w;
      const unsigned m = __ballot_sync(0xffffffffu, mine);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(P.wl_count + w, __popc(m));
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (mine) lists[w][pos + __popc(m & ((1u << lane) - 1u))] = item;
    }
  }
}

cudaError_t launch_worklists(const ProblemDev& P, int mask, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(P.wl_count, 0, sizeof(int) * WL_INTS, st);
  if (e != cudaSuccess) return e;
  const int total = P.n_tiles + P.n_patches + P.S;
  const int blocks = std::max(1, std::min((total + 255) / 256, P.n_sm * 4));
  worklist_kernel<<<blocks, 256, 0, st>>>(P, mask);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const ProblemDev& P, const double* theta, bool full, double* elbo, double* grad,
                            double* hess, cudaStream_t st) {
  const int blocks = std::max(1, std::min(P.S, P.n_sm * 4));
  assemble_kernel<<<blocks, 128, 0, st>>>(P, theta, full ? 1 : 0, elbo, grad, hess);
  return cudaGetLastError();
}

cudaError_t launch_set_flags(const ProblemDev& P, int value, cudaStream_t st) {
  set_flags_kernel<<<(P.S + 255) / 256, 256, 0, st>>>(P.flags, P.S, value);
  return cudaGetLastError();
}

}  // namespace celeste
