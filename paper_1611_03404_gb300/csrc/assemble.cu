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

// Brightness parameter indices of type t (r1, rho, c1 x4, gamma x4).
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

// Source-level quantities shared by all patches (exps of the log-variances, type probabilities).
struct SourceConst {
  double a0, a1, aa, la0, la1;   // P(star), P(galaxy), product, their logs
  double ev[2][10];              // exp of the log-variance parameters (v = 1, 6..9), 0 elsewhere
};

__device__ inline void source_const_parallel(const double* th, SourceConst& sc, int tid) {
  if (tid < 10) {
    const int t = tid / 5, k = tid % 5, v = k == 0 ? 1 : 5 + k;
    sc.ev[t][v] = exp(th[bvar(t, v)]);
  } else if (tid < 20) {
    const int t = (tid - 10) / 5, k = (tid - 10) % 5, v = k == 0 ? 0 : k + 1;   // v = 0, 2..5
    sc.ev[t][v] = 0.0;
  } else if (tid == 20) {
    const double al = th[6];
    const double e = exp(-fabs(al)), l1p = log1p(e);
    sc.la1 = al >= 0 ? -l1p : al - l1p;   // log sigmoid(alpha)
    sc.la0 = sc.la1 - al;                  // log sigmoid(-alpha)
    const double sg = 1.0 / (1.0 + e);
    sc.a1 = al >= 0 ? sg : e * sg;
    sc.a0 = al >= 0 ? e * sg : sg;
    sc.aa = sc.a0 * sc.a1;
  }
}

// One normal-KL term of type t: k = 0 the log flux, k = 1..4 the colours j = k - 1.
// KL_N(m, v || mu, s2) = (log s2 - log v + (v + (m - mu)^2) / s2 - 1) / 2 with v = exp(log v).
__device__ inline double kl_normal_term(const double* th, const double* ev, const ProblemDev& P, int t, int k) {
  const double m = k == 0 ? th[bvar(t, 0)] : th[bvar(t, 1 + k)];
  const double lv = k == 0 ? th[bvar(t, 1)] : th[bvar(t, 5 + k)];
  const double v = k == 0 ? ev[1] : ev[5 + k];
  const double mu = k == 0 ? P.priors[1] : P.priors[3], s2 = k == 0 ? P.priors[2] : P.priors[4];
  const double ls2 = k == 0 ? P.log_var_r : P.log_var_c;
  return 0.5 * (ls2 - lv + (v + (m - mu) * (m - mu)) / s2 - 1.0);
}

// First and second derivative of K_t w.r.t. brightness parameter j of type t.
__device__ inline void kl_normal_derivs(const double* th, const SourceConst& sc, const ProblemDev& P, int j, int& t,
                                        double& dK, double& d2K) {
  int v;
  bvar_inv(j, t, v);
  if (v == 0 || (v >= 2 && v < 6)) {
    const double mu = v == 0 ? P.priors[1] : P.priors[3], s2 = v == 0 ? P.priors[2] : P.priors[4];
    dK = (th[j] - mu) / s2;
    d2K = 1.0 / s2;
  } else {
    const double s2 = v == 1 ? P.priors[2] : P.priors[4];
    dK = 0.5 * (sc.ev[t][v] / s2 - 1.0);
    d2K = 0.5 * sc.ev[t][v] / s2;
  }
}

struct PatchLift {
  double L1[2], L2[2];                     // E[l_b|i], E[l_b^2|i]
  double dL1[2][10], dL2[2][10];           // gradients over the type's brightness parameters
  double d2l1[2][10], d2l2[2][10];         // diagonal second derivatives of log L1, log L2
  double A[4];                             // WCS linear part
  int band;
};

// Float32 copies of the lift quantities that only the Hessian uses.
struct PatchLiftF {
  float L1[2], L2[2], dL1[2][10], dL2[2][10], d2l1[2][10], d2l2[2][10], A[4];
  float a0, a1, aa;
};

// Per-warp working set of one patch's lift.
struct WarpLift {
  double sd[ACC_HP];                                  // float64 sums: L, S1, S2
  double gs[NP], gE[NP], nzK[NP], nzL[NP], ghat[NRED];
  double Lsum;
  PatchLift c;
  float sdf[ACC_HP], sf[NACC - ACC_HP];               // float32 copies / compensated sums: HP, M
  float Hs[NP * NP], H2[NP * NP];                     // accumulated Hessian; per-patch second-order part
  float Msym[NRED * NRED], nzKf[NP], nzLf[NP];
  PatchLiftF cf;
  int nzA[NP], nzB[NP];
};

// ELBO and gradient are summed and lifted in float64 (the cross-pixel sums of the objective and
// its gradient); the Hessian, whose per-pixel terms are float32 to begin with, in float32 with
// compensated cross-tile sums.  On this part a float64 warp instruction costs ~64 cycles of its
// SM sub-partition, a float32 one a single issue slot, so the split cuts the kernel's float64
// instructions about fourfold.  A CTA takes one source; each of its four warps lifts every fourth
// patch of the source into warp-private accumulators (the four sub-partitions' float64 pipes run
// in parallel), then the warps' sums are added.
__global__ void __launch_bounds__(128) assemble_kernel(ProblemDev P, const double* __restrict__ theta, int full,
                                                       double* elbo, double* grad, double* hess) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = 4;                 // warps per CTA
  constexpr int ND = ACC_HP;            // float64 sums: L, S1, S2
  constexpr int NF = NACC - ACC_HP;     // float32 sums: HP, M
  __shared__ WarpLift wl[NW];
  __shared__ float Hs[NP * NP];
  __shared__ double gs[NP];
  __shared__ SourceConst sc;
  __shared__ double Lsum, red[16];
  __shared__ int slot;
  WarpLift& W = wl[warp];
  PatchLift& c = W.c;
  PatchLiftF& cf = W.cf;
  for (int s = wl_next_cta(P, WL_SOURCES, slot); s >= 0; s = wl_next_cta(P, WL_SOURCES, slot)) {
  const double* th = theta + (size_t)s * NP;
  for (int i = lane; i < NP * NP; i += 32) W.Hs[i] = 0.f;
  if (lane < NP) W.gs[lane] = 0.0;
  if (lane == 0) W.Lsum = 0.0;
  source_const_parallel(th, sc, tid);
  __syncthreads();
  if (lane == 0) {
    cf.a0 = (float)sc.a0;
    cf.a1 = (float)sc.a1;
    cf.aa = (float)sc.aa;
  }
  for (int p = P.src_patch[s] + warp; p < P.src_patch[s + 1]; p += NW) {
    const PatchDev pt = P.patches[p];
    // ---- tile sums (fixed order; float64 for the objective and gradient, compensated float32 for
    //      the Hessian-only sums) and the band moments
    if (lane < ND) {
      double v = 0.0;
      for (int t = pt.tile_begin; t < pt.tile_end; ++t) v += (double)P.partials[(size_t)t * NACC + lane];
      W.sd[lane] = v;
      W.sdf[lane] = (float)v;
    } else if (lane < ND + 4) {
      const int k = lane - ND, t = k & 1, second = k >> 1;
      const int band = P.images[pt.image].band;
      double arow[4];
      color_row(band, arow);
      double m = th[bvar(t, 0)], v = sc.ev[t][1];
      for (int j = 0; j < 4; ++j) {
        m += arow[j] * th[bvar(t, 2 + j)];
        v += arow[j] * arow[j] * sc.ev[t][6 + j];
      }
      if (second) {
        c.L2[t] = exp(2.0 * m + 2.0 * v);
        cf.L2[t] = (float)c.L2[t];
      } else {
        c.L1[t] = exp(m + 0.5 * v);
        cf.L1[t] = (float)c.L1[t];
      }
      if (k == 0) c.band = band;
    } else if (lane < ND + 8) {
      c.A[lane - ND - 4] = P.images[pt.image].A[lane - ND - 4];
      cf.A[lane - ND - 4] = (float)c.A[lane - ND - 4];
    }
    for (int q = lane; q < NF; q += 32) {
      float v = 0.f, comp = 0.f;
      for (int t = pt.tile_begin; t < pt.tile_end; ++t) {
        const float y = P.partials[(size_t)t * NACC + ND + q] - comp;
        const float u = v + y;
        comp = (u - v) - y;
        v = u;
      }
      W.sf[q] = v;
    }
    __syncwarp();
    // ---- derivatives of the band moments over the type's brightness parameters
    for (int q = lane; q < 40; q += 32) {
      const int t = q / 20, which = (q % 20) / 10, v = q % 10;
      double arow[4];
      color_row(c.band, arow);
      double dl, d2;
      if (v == 0) {
        dl = which ? 2.0 : 1.0;
        d2 = 0.0;
      } else if (v == 1) {
        dl = (which ? 2.0 : 0.5) * sc.ev[t][1];
        d2 = dl;
      } else if (v < 6) {
        dl = (which ? 2.0 : 1.0) * arow[v - 2];
        d2 = 0.0;
      } else {
        dl = (which ? 2.0 : 0.5) * arow[v - 6] * arow[v - 6] * sc.ev[t][v];
        d2 = dl;
      }
      if (which) {
        c.dL2[t][v] = c.L2[t] * dl;
        cf.dL2[t][v] = (float)c.dL2[t][v];
        cf.d2l2[t][v] = (float)d2;
      } else {
        c.dL1[t][v] = c.L1[t] * dl;
        cf.dL1[t][v] = (float)c.dL1[t][v];
        cf.d2l1[t][v] = (float)d2;
      }
    }
    if (lane == 0) W.Lsum += W.sd[ACC_L];
    __syncwarp();
    const double* S1 = W.sd + ACC_S1;
    const double* S2 = W.sd + ACC_S2;
    const float* S1h = W.sdf + ACC_S1;
    const float* S2h = W.sdf + ACC_S2;
    // ---- reduced gradient (float64)
    if (lane < NRED) {
      const double A0 = sc.a0 * c.L1[0], A1 = sc.a1 * c.L1[1], B0 = sc.a0 * c.L2[0], B1 = sc.a1 * c.L2[1];
      const int a = lane;
      double v;
      if (a < 2)
        v = A0 * S1[1 + a] + A1 * S1[4 + a] + B0 * S2[1 + a] + B1 * S2[4 + a];
      else if (a < 6)
        v = A1 * S1[4 + a] + B1 * S2[4 + a];
      else if (a == 6)
        v = sc.aa * (c.L1[1] * S1[3] - c.L1[0] * S1[0] + c.L2[1] * S2[3] - c.L2[0] * S2[0]);
      else
        v = a == 7 ? S1[0] : a == 8 ? S1[3] : a == 9 ? S2[0] : S2[3];
      W.ghat[a] = v;
    }
    // Lift from the 11-column reduced basis to the 27 parameters: column j of K has at most two
    // nonzeros (a, k): j < 7 -> (j, 1); brightness parameter v of type t -> (7 + t, a_t dL1_t[v])
    // from the E-row and (9 + t, a_t dL2_t[v]) from the V-row.  H_E = K^T M K + H2, g_E = K^T ghat.
    if (lane < NP) {
      const int j = lane;
      if (j < 7) {
        W.nzA[j] = j;
        W.nzK[j] = 1.0;
        W.nzB[j] = -1;
        W.nzL[j] = 0.0;
      } else {
        int t, v;
        bvar_inv(j, t, v);
        const double at = t ? sc.a1 : sc.a0;
        W.nzA[j] = 7 + t;
        W.nzK[j] = at * c.dL1[t][v];
        W.nzB[j] = 9 + t;
        W.nzL[j] = at * c.dL2[t][v];
      }
      W.nzKf[j] = (float)W.nzK[j];
      W.nzLf[j] = (float)W.nzL[j];
    }
    for (int i = lane; i < NRED * NRED; i += 32) {
      const int a = i / NRED, b = i % NRED;
      W.Msym[i] = W.sf[ACC_M - ND + (a <= b ? tri11d(a, b) : tri11d(b, a))];
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
      const int b = a + rem;
      H2[a * NP + b] = H2[b * NP + a] = W.sf[ACC_HP - ND + q];
    }
    const float S1f[2] = {S1h[0], S1h[3]}, S2f[2] = {S2h[0], S2h[3]};
    for (int i = lane; i < 6 + 1 + 120 + 20 + 200; i += 32) {
      if (i < 6) {
        const int a = i;
        const float s1f0 = a < 2 ? S1h[1 + a] : 0.f, s2f0 = a < 2 ? S2h[1 + a] : 0.f;
        H2[a * NP + 6] = H2[6 * NP + a] =
            cf.aa * (cf.L1[1] * S1h[4 + a] - cf.L1[0] * s1f0 + cf.L2[1] * S2h[4 + a] - cf.L2[0] * s2f0);
      } else if (i == 6) {
        H2[6 * NP + 6] = cf.aa * (1.f - 2.f * cf.a1) *
                         (cf.L1[1] * S1f[1] - cf.L1[0] * S1f[0] + cf.L2[1] * S2f[1] - cf.L2[0] * S2f[0]);
      } else if (i < 127) {
        const int k = i - 7, t = k / 60, a = (k % 60) / 10, v = k % 10, j = bvar(t, v);
        const float s1 = t ? S1h[4 + a] : (a < 2 ? S1h[1 + a] : 0.f);
        const float s2 = t ? S2h[4 + a] : (a < 2 ? S2h[1 + a] : 0.f);
        H2[a * NP + j] = H2[j * NP + a] = (t ? cf.a1 : cf.a0) * (s1 * cf.dL1[t][v] + s2 * cf.dL2[t][v]);
      } else if (i < 147) {
        const int k = i - 127, t = k / 10, v = k % 10, j = bvar(t, v);
        H2[6 * NP + j] = H2[j * NP + 6] = (t ? cf.aa : -cf.aa) * (S1f[t] * cf.dL1[t][v] + S2f[t] * cf.dL2[t][v]);
      } else {
        // d2 L = L (dlogL dlogL^T + diag(d2 log L)) within a type
        const int k = i - 147, t = k / 100, v = (k % 100) / 10, w = k % 10;
        const float dl1v = cf.dL1[t][v] / cf.L1[t], dl1w = cf.dL1[t][w] / cf.L1[t];
        const float dl2v = cf.dL2[t][v] / cf.L2[t], dl2w = cf.dL2[t][w] / cf.L2[t];
        const float d2L1 = cf.L1[t] * (dl1v * dl1w + (v == w ? cf.d2l1[t][v] : 0.f));
        const float d2L2 = cf.L2[t] * (dl2v * dl2w + (v == w ? cf.d2l2[t][v] : 0.f));
        H2[bvar(t, v) * NP + bvar(t, w)] = (t ? cf.a1 : cf.a0) * (S1f[t] * d2L1 + S2f[t] * d2L2);
      }
    }
    __syncwarp();
    // H_E = K^T M K + H2, in place over H2 (each pair (r <= col) reads only its own upper entry)
    for (int q = lane; q < NP * (NP + 1) / 2; q += 32) {
      int r = 0, rem = q;   // q -> (r, col) with r <= col
      while (rem >= NP - r) {
        rem -= NP - r;
        ++r;
      }
      const int col = r + rem;
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
    for (int i = lane; i < NP * NP; i += 32) {
      const int r = i / NP, q = i % NP;
      float v;
      if (r < 2 && q < 2) {
        v = 0.f;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) v += cf.A[a * 2 + r] * cf.A[b * 2 + q] * HE[a * NP + b];
      } else if (r < 2) {
        v = cf.A[0 * 2 + r] * HE[0 * NP + q] + cf.A[1 * 2 + r] * HE[1 * NP + q];
      } else if (q < 2) {
        v = cf.A[0 * 2 + q] * HE[r * NP + 0] + cf.A[1 * 2 + q] * HE[r * NP + 1];
      } else {
        v = HE[i];
      }
      W.Hs[i] += v;
    }
    if (lane < NP) {
      const int j = lane;
      W.gs[j] += j < 2 ? c.A[0 * 2 + j] * W.gE[0] + c.A[1 * 2 + j] * W.gE[1] : W.gE[j];
    }
    __syncwarp();
  }
  __syncthreads();
  // ---- the warps' sums (fixed order)
  for (int i = tid; i < NP * NP; i += nt) Hs[i] = (wl[0].Hs[i] + wl[1].Hs[i]) + (wl[2].Hs[i] + wl[3].Hs[i]);
  if (tid < NP) gs[tid] = (wl[0].gs[tid] + wl[1].gs[tid]) + (wl[2].gs[tid] + wl[3].gs[tid]);
  if (tid == 0) Lsum = (wl[0].Lsum + wl[1].Lsum) + (wl[2].Lsum + wl[3].Lsum);
  __syncthreads();

  // ---- KL = a1 (log a1 - log Phi) + a0 (log a0 - log(1 - Phi)) + a0 K_0 + a1 K_1 and its
  //      derivatives (closed forms from the source constants; no further transcendentals)
  if (tid < 10) red[tid] = kl_normal_term(th, sc.ev[tid / 5], P, tid / 5, tid % 5);
  __syncthreads();
  if (tid == 0) {
    double K0 = 0.0, K1 = 0.0;
    for (int i = 0; i < 5; ++i) {
      K0 += red[i];
      K1 += red[5 + i];
    }
    red[10] = K0;
    red[11] = K1;
    const double kl = sc.a1 * (sc.la1 - P.log_phi) + sc.a0 * (sc.la0 - P.log1m_phi) + sc.a0 * K0 + sc.a1 * K1;
    if (elbo) elbo[s] = Lsum - kl;
  }
  __syncthreads();
  if (full) {
    const double K0 = red[10], K1 = red[11];
    const double ga = sc.aa * (th[6] - P.logit_phi) + sc.aa * (K1 - K0);
    if (hess) {
      for (int i = tid; i < NP * NP; i += nt) {
        const int r = i / NP, q = i % NP;
        double h = 0.0;
        if (r == 6 && q == 6) {
          h = sc.aa * ((1.0 - 2.0 * sc.a1) * (th[6] - P.logit_phi) + 1.0) + sc.aa * (1.0 - 2.0 * sc.a1) * (K1 - K0);
        } else if ((r == 6 && q >= 7) || (q == 6 && r >= 7)) {
          int t;
          double dK, d2K;
          kl_normal_derivs(th, sc, P, r == 6 ? q : r, t, dK, d2K);
          h = (t ? sc.aa : -sc.aa) * dK;
        } else if (r == q && r >= 7) {
          int t;
          double dK, d2K;
          kl_normal_derivs(th, sc, P, r, t, dK, d2K);
          h = (t ? sc.a1 : sc.a0) * d2K;
        }
        hess[(size_t)s * NP * NP + i] = (double)Hs[i] - h;
      }
    }
    if (grad && tid < NP) {
      const int j = tid;
      double gk = 0.0;
      if (j == 6) {
        gk = ga;
      } else if (j >= 7) {
        int t;
        double dK, d2K;
        kl_normal_derivs(th, sc, P, j, t, dK, d2K);
        gk = (t ? sc.a1 : sc.a0) * dK;
      }
      grad[(size_t)s * NP + j] = gs[j] - gk;
    }
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
      double ev[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      const int vi = kk == 0 ? 1 : 5 + kk;
      ev[vi] = exp(th[bvar(t, vi)]);
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
