// Float64 assembly of each source's ELBO, gradient and Hessian from the per-tile pixel sums,
// plus the KL term of q (paper, Sec. "Variational Inference": Eq. (1)-(3); q(a) Bernoulli,
// q(r|a) lognormal, q(c|a) normal, each conjugate to its prior).
//
// Work in the "E-space" of a patch: the 27 parameters with the world position u replaced by
// the pixel-space mean mu = A u + o (so the pixel sums need no WCS); the u rows/columns are
// mapped back with A before summing over the source's images.
#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

__device__ constexpr int tri6d(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }
__device__ constexpr int tri11d(int i, int j) { return i * 11 - i * (i - 1) / 2 + (j - i); }

// Brightness parameter indices of type i (r1, rho, c1 x4, gamma x4).
__device__ inline int bvar(int type, int v) {
  if (v == 0) return type ? 9 : 7;
  if (v == 1) return type ? 10 : 8;
  if (v < 6) return (type ? 19 : 11) + (v - 2);
  return (type ? 23 : 15) + (v - 6);
}

// Category of a parameter index: 0..5 -> G6 (mu0 mu1 dev axis angle scale), 6 alpha,
// 7.. brightness (type, v) encoded as 100 + 10 * type + v.
__device__ inline int category(int i) {
  if (i < 6) return i;
  if (i == 6) return 6;
  if (i == 7) return 100;
  if (i == 8) return 101;
  if (i == 9) return 110;
  if (i == 10) return 111;
  if (i < 15) return 100 + 2 + (i - 11);
  if (i < 19) return 100 + 6 + (i - 15);
  if (i < 23) return 110 + 2 + (i - 19);
  return 110 + 6 + (i - 23);
}

struct PatchLift {
  double a0, a1, aa;                       // P(star), P(galaxy), a0 a1
  double L1[2], L2[2];                     // E[l_b|i], E[l_b^2|i]
  double dL1[2][10], dL2[2][10];           // gradients over the type's brightness parameters
  double d2l1[2][10], d2l2[2][10];         // diagonal second derivatives of log L1, log L2
  double S1[10], S2[10], Hp[21];           // tile sums (float64)
  double A[4];                             // WCS linear part
};

__device__ double h2_entry(const PatchLift& c, int ci, int cj) {
  // symmetric: order so that ci <= cj in the category encoding
  if (ci > cj) {
    int t = ci;
    ci = cj;
    cj = t;
  }
  auto s1f0g = [&](int a) { return a < 2 ? c.S1[1 + a] : 0.0; };
  auto s2f0g = [&](int a) { return a < 2 ? c.S2[1 + a] : 0.0; };
  auto s1fg = [&](int type, int a) { return type ? c.S1[4 + a] : s1f0g(a); };
  auto s2fg = [&](int type, int a) { return type ? c.S2[4 + a] : s2f0g(a); };
  const double S1f[2] = {c.S1[0], c.S1[3]}, S2f[2] = {c.S2[0], c.S2[3]};
  if (cj < 6) return c.Hp[tri6d(ci, cj)];
  if (cj == 6) {
    if (ci < 6)
      return c.aa * (c.L1[1] * s1fg(1, ci) - c.L1[0] * s1fg(0, ci) + c.L2[1] * s2fg(1, ci) - c.L2[0] * s2fg(0, ci));
    return c.aa * (1.0 - 2.0 * c.a1) * (c.L1[1] * S1f[1] - c.L1[0] * S1f[0] + c.L2[1] * S2f[1] - c.L2[0] * S2f[0]);
  }
  const int tj = (cj - 100) / 10, vj = (cj - 100) % 10;
  const double ai = tj ? c.a1 : c.a0;
  if (ci < 6) return ai * (s1fg(tj, ci) * c.dL1[tj][vj] + s2fg(tj, ci) * c.dL2[tj][vj]);
  if (ci == 6) return (tj ? c.aa : -c.aa) * (S1f[tj] * c.dL1[tj][vj] + S2f[tj] * c.dL2[tj][vj]);
  const int ti = (ci - 100) / 10, vi = (ci - 100) % 10;
  if (ti != tj) return 0.0;
  // d2 L = L (dlogL dlogL^T + diag(d2 log L))
  const double dl1i = c.dL1[ti][vi] / c.L1[ti], dl1j = c.dL1[tj][vj] / c.L1[tj];
  const double dl2i = c.dL2[ti][vi] / c.L2[ti], dl2j = c.dL2[tj][vj] / c.L2[tj];
  double d2L1 = c.L1[ti] * (dl1i * dl1j + (vi == vj ? c.d2l1[ti][vi] : 0.0));
  double d2L2 = c.L2[ti] * (dl2i * dl2j + (vi == vj ? c.d2l2[ti][vi] : 0.0));
  return ai * (S1f[ti] * d2L1 + S2f[ti] * d2L2);
}

// KL of one source and its derivatives (closed forms).
__device__ void kl_terms(const double* th, const double* pri, double& kl, double* g, double* h /*27x27*/, int tid,
                         int nthreads) {
  const double phi = pri[0], mu_r = pri[1], var_r = pri[2], mu_c = pri[3], var_c = pri[4];
  const double al = th[6];
  const double a1 = sigmoid_d(al), a0 = sigmoid_d(-al), aa = a0 * a1;
  const double la1 = al >= 0 ? -log1p(exp(-al)) : al - log1p(exp(al));
  const double la0 = la1 - al;
  const double lgt = log(phi) - log1p(-phi);
  double K[2], dK[2][10], d2K[2][10];
  for (int t = 0; t < 2; ++t) {
    K[t] = 0.0;
    for (int v = 0; v < 10; ++v) {
      const int idx = bvar(t, v);
      if (v == 0 || (v >= 2 && v < 6)) {
        const double mu = v == 0 ? mu_r : mu_c, s2 = v == 0 ? var_r : var_c;
        const int rho_idx = v == 0 ? bvar(t, 1) : bvar(t, v + 4);
        const double m = th[idx], rho = th[rho_idx];
        K[t] += 0.5 * (log(s2) - rho + (exp(rho) + (m - mu) * (m - mu)) / s2 - 1.0);
        dK[t][v] = (m - mu) / s2;
        d2K[t][v] = 1.0 / s2;
      } else {
        const double s2 = v == 1 ? var_r : var_c;
        const double rho = th[idx];
        dK[t][v] = 0.5 * (exp(rho) / s2 - 1.0);
        d2K[t][v] = 0.5 * exp(rho) / s2;
      }
    }
  }
  kl = a1 * (la1 - log(phi)) + a0 * (la0 - log1p(-phi)) + a0 * K[0] + a1 * K[1];
  for (int i = tid; i < NP; i += nthreads) g[i] = 0.0;
  for (int i = tid; i < NP * NP; i += nthreads) h[i] = 0.0;
  __syncthreads();
  if (tid == 0) {
    g[6] = aa * (al - lgt) + aa * (K[1] - K[0]);
    h[6 * NP + 6] = aa * ((1.0 - 2.0 * a1) * (al - lgt) + 1.0) + aa * (1.0 - 2.0 * a1) * (K[1] - K[0]);
    for (int t = 0; t < 2; ++t) {
      const double at = t ? a1 : a0, sa = t ? aa : -aa;
      for (int v = 0; v < 10; ++v) {
        const int idx = bvar(t, v);
        g[idx] = at * dK[t][v];
        h[idx * NP + idx] = at * d2K[t][v];
        h[6 * NP + idx] = h[idx * NP + 6] = sa * dK[t][v];
      }
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(128) assemble_kernel(ProblemDev P, const double* __restrict__ theta, int full,
                                                       int flag_mask, double* elbo, double* grad, double* hess) {
  const int s = blockIdx.x;
  if (!(P.flags[s] & flag_mask)) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ double sums[NACC];
  __shared__ double Hs[NP * NP], gs[NP], HE[NP * NP], gE[NP];
  __shared__ double Kd[NRED * NP], T[NRED * NP], ghat[NRED];
  __shared__ PatchLift c;
  __shared__ double Lsum;
  const double* th = theta + (size_t)s * NP;
  for (int i = tid; i < NP * NP; i += nt) Hs[i] = 0.0;
  for (int i = tid; i < NP; i += nt) gs[i] = 0.0;
  if (tid == 0) Lsum = 0.0;
  __syncthreads();
  for (int p = P.src_patch[s]; p < P.src_patch[s + 1]; ++p) {
    const PatchDev pt = P.patches[p];
    if (!full) {
      if (tid == 0) {
        double v = 0.0;
        for (int t = pt.tile_begin; t < pt.tile_end; ++t) v += (double)P.vpartials[t];
        Lsum += v;
      }
      continue;
    }
    for (int q = tid; q < NACC; q += nt) {
      double v = 0.0;
      for (int t = pt.tile_begin; t < pt.tile_end; ++t) v += (double)P.partials[(size_t)t * NACC + q];
      sums[q] = v;
    }
    __syncthreads();
    if (tid == 0) {
      const ImageDev& im = P.images[pt.image];
      c.a1 = sigmoid_d(th[6]);
      c.a0 = sigmoid_d(-th[6]);
      c.aa = c.a0 * c.a1;
      double arow[4];
      color_row(im.band, arow);
      for (int t = 0; t < 2; ++t) {
        lognormal_moments(th, t, im.band, c.L1[t], c.L2[t]);
        double dl1[10], dl2[10];
        dl1[0] = 1.0;
        dl2[0] = 2.0;
        const double er = exp(th[bvar(t, 1)]);
        dl1[1] = 0.5 * er;
        dl2[1] = 2.0 * er;
        c.d2l1[t][0] = 0.0;
        c.d2l2[t][0] = 0.0;
        c.d2l1[t][1] = 0.5 * er;
        c.d2l2[t][1] = 2.0 * er;
        for (int j = 0; j < 4; ++j) {
          const double eg = exp(th[bvar(t, 6 + j)]);
          dl1[2 + j] = arow[j];
          dl2[2 + j] = 2.0 * arow[j];
          dl1[6 + j] = 0.5 * arow[j] * arow[j] * eg;
          dl2[6 + j] = 2.0 * arow[j] * arow[j] * eg;
          c.d2l1[t][2 + j] = 0.0;
          c.d2l2[t][2 + j] = 0.0;
          c.d2l1[t][6 + j] = 0.5 * arow[j] * arow[j] * eg;
          c.d2l2[t][6 + j] = 2.0 * arow[j] * arow[j] * eg;
        }
        for (int v = 0; v < 10; ++v) {
          c.dL1[t][v] = c.L1[t] * dl1[v];
          c.dL2[t][v] = c.L2[t] * dl2[v];
        }
      }
      for (int q = 0; q < 10; ++q) {
        c.S1[q] = sums[ACC_S1 + q];
        c.S2[q] = sums[ACC_S2 + q];
      }
      for (int q = 0; q < 21; ++q) c.Hp[q] = sums[ACC_HP + q];
      for (int q = 0; q < 4; ++q) c.A[q] = im.A[q];
      Lsum += sums[ACC_L];
      // reduced gradient
      const double A0 = c.a0 * c.L1[0], A1 = c.a1 * c.L1[1], B0 = c.a0 * c.L2[0], B1 = c.a1 * c.L2[1];
      for (int a = 0; a < 2; ++a) ghat[a] = A0 * c.S1[1 + a] + A1 * c.S1[4 + a] + B0 * c.S2[1 + a] + B1 * c.S2[4 + a];
      for (int a = 2; a < 6; ++a) ghat[a] = A1 * c.S1[4 + a] + B1 * c.S2[4 + a];
      ghat[6] = c.aa * (c.L1[1] * c.S1[3] - c.L1[0] * c.S1[0] + c.L2[1] * c.S2[3] - c.L2[0] * c.S2[0]);
      ghat[7] = c.S1[0];
      ghat[8] = c.S1[3];
      ghat[9] = c.S2[0];
      ghat[10] = c.S2[3];
    }
    // lift matrix K (11 x 27) in E-space
    for (int i = tid; i < NRED * NP; i += nt) Kd[i] = 0.0;
    __syncthreads();
    if (tid < 7) Kd[tid * NP + tid] = 1.0;
    if (tid >= 32 && tid < 72) {
      const int r = (tid - 32) / 10, v = (tid - 32) % 10;   // r: 0 -> row 7 (f0,E), 1 -> 8, 2 -> 9, 3 -> 10
      const int type = r & 1;
      const double at = type ? c.a1 : c.a0;
      const double val = r < 2 ? at * c.dL1[type][v] : at * c.dL2[type][v];
      Kd[(7 + r) * NP + bvar(type, v)] = val;
    }
    __syncthreads();
    // T = M K  (M symmetric 11x11 from packed sums)
    for (int i = tid; i < NRED * NP; i += nt) {
      const int a = i / NP, j = i % NP;
      double v = 0.0;
      for (int b = 0; b < NRED; ++b) {
        const double m = sums[ACC_M + (a <= b ? tri11d(a, b) : tri11d(b, a))];
        v += m * Kd[b * NP + j];
      }
      T[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < NP * NP; i += nt) {
      const int r = i / NP, q = i % NP;
      double v = 0.0;
      for (int a = 0; a < NRED; ++a) v += Kd[a * NP + r] * T[a * NP + q];
      HE[i] = v + h2_entry(c, category(r), category(q));
    }
    for (int j = tid; j < NP; j += nt) {
      double v = 0.0;
      for (int a = 0; a < NRED; ++a) v += ghat[a] * Kd[a * NP + j];
      gE[j] = v;
    }
    __syncthreads();
    // map mu -> u: d/du_b = sum_a A[a][b] d/dmu_a
    for (int i = tid; i < NP * NP; i += nt) {
      const int r = i / NP, q = i % NP;
      double v;
      if (r < 2 && q < 2) {
        v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) v += c.A[a * 2 + r] * c.A[b * 2 + q] * HE[a * NP + b];
      } else if (r < 2) {
        v = c.A[0 * 2 + r] * HE[0 * NP + q] + c.A[1 * 2 + r] * HE[1 * NP + q];
      } else if (q < 2) {
        v = c.A[0 * 2 + q] * HE[r * NP + 0] + c.A[1 * 2 + q] * HE[r * NP + 1];
      } else {
        v = HE[i];
      }
      Hs[i] += v;
    }
    for (int j = tid; j < NP; j += nt) {
      double v = j < 2 ? c.A[0 * 2 + j] * gE[0] + c.A[1 * 2 + j] * gE[1] : gE[j];
      gs[j] += v;
    }
    __syncthreads();
  }
  __syncthreads();
  double kl;
  kl_terms(th, P.priors, kl, gE, HE, tid, nt);
  if (tid == 0 && elbo) elbo[s] = Lsum - kl;
  if (full) {
    if (grad)
      for (int j = tid; j < NP; j += nt) grad[(size_t)s * NP + j] = gs[j] - gE[j];
    if (hess)
      for (int i = tid; i < NP * NP; i += nt) hess[(size_t)s * NP * NP + i] = Hs[i] - HE[i];
  }
}

__global__ void set_flags_kernel(int* flags, int S, int value) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) flags[s] = value;
}

cudaError_t launch_assemble(const ProblemDev& P, const double* theta, bool full, int flag_mask, double* elbo,
                            double* grad, double* hess, cudaStream_t st) {
  assemble_kernel<<<P.S, 128, 0, st>>>(P, theta, full ? 1 : 0, flag_mask, elbo, grad, hess);
  return cudaGetLastError();
}

cudaError_t launch_set_flags(const ProblemDev& P, int value, cudaStream_t st) {
  set_flags_kernel<<<(P.S + 255) / 256, 256, 0, st>>>(P.flags, P.S, value);
  return cudaGetLastError();
}

}  // namespace celeste
