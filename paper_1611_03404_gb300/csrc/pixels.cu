// Pixel kernels: neighbour background, ELBO + gradient + Hessian tile sums, value-only tile sums.
//
// Paper, Sec. "The Celeste Model": x_nm ~ Poisson(F_nm) with F_nm deterministic in the catalog
// and Lambda_n.  Sec. "Variational Inference": L = E_q[log p(x, z) - log q(z)] (Eq. 1-2), each
// source optimised with neighbours fixed, with the exact gradient and dense Hessian.
//
// Per pixel m of a source's patch in image n (band b):
//   E[G] = A0 f0 + A1 f1,  E[G^2] = B0 f0^2 + B1 f1^2      (A_i = a_i E[l_b|i], B_i = a_i E[l_b^2|i])
//   E = bE + iota E[G],    V = bV + iota^2 Var[G]          (bE, bV: sky + fixed neighbours)
//   l = x (log E - V / (2 E^2)) - E - log x!               (delta method for E_q[log F])
// The gradient and Hessian are assembled from 108 per-tile sums (see celeste_internal.cuh):
//   grad = sum_m w1 dE[G] + w2 dE[G^2]
//   Hess = sum_m Y_m^T C_m Y_m + w1 d2E[G] + w2 d2E[G^2]
// with Y_m = [dE[G]; dE[G^2]] written in an 11-column reduced basis (the brightness columns of
// dE[G] are f_i times a per-(source, image) constant vector), C_m the 2x2 curvature of the
// pixel term, w1 = iota l_E - 2 iota^2 E[G] l_V and w2 = iota^2 l_V.
#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

__host__ __device__ constexpr int tri5(int i, int j) { return i * 5 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int tri6(int i, int j) { return i * 6 - i * (i - 1) / 2 + (j - i); }
__host__ __device__ constexpr int tri11(int i, int j) { return i * 11 - i * (i - 1) / 2 + (j - i); }

constexpr long long WAIT_BUDGET = 4000000000LL;   // ~2 s of SM clock for a bulk copy

// ------------------------------------------------------------------------------ table setup
// Full derivative table of galaxy component g = k * NMIX + j for a source with parameters th.
__device__ void gal_full_entry(const ProblemDev& P, const ImageDev& im, const PatchDev& pt, int patch, const double* th,
                               int g, float* out) {
  const int k = g / NMIX, j = g % NMIX;
  PsfComp pc = load_psf(P.psf + (size_t)patch * 18, k);
  double px, py;
  source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
  GalShape gs;
  galaxy_shape(th[3], th[4], th[5], gs);
  const float A[4] = {(float)im.A[0], (float)im.A[1], (float)im.A[2], (float)im.A[3]};
  const float tau = P.tau[j], nu = P.nu[j];
  Sym2 Sp = congruence(A, gs.S);
  Sym2 S = {tau * Sp.a + pc.S.a, tau * Sp.b + pc.S.b, tau * Sp.c + pc.S.c};
  float ld;
  Sym2 Pm = inv2(S, ld);
  Sym2 dS[3];
  Mat2 PdS[3];
  for (int a = 0; a < 3; ++a) {
    Sym2 t = congruence(A, gs.d[a]);
    dS[a] = {tau * t.a, tau * t.b, tau * t.c};
    PdS[a] = mul(Pm, dS[a]);
  }
  out[GT_MU + 0] = (float)(px + pc.mx);
  out[GT_MU + 1] = (float)(py + pc.my);
  out[GT_LW2] = (logf(pc.w * nu) - 0.5f * ld - LOG_2PI) * LOG2E;
  out[GT_P + 0] = Pm.a;
  out[GT_P + 1] = Pm.b;
  out[GT_P + 2] = Pm.c;
  for (int a = 0; a < 3; ++a) {
    Sym2 dP = to_sym(mul(PdS[a], Pm));   // P dS P; dP/da = -P dS P
    out[GT_QA + 3 * a + 0] = 0.5f * dP.a;
    out[GT_QA + 3 * a + 1] = 0.5f * dP.b;
    out[GT_QA + 3 * a + 2] = 0.5f * dP.c;
    out[GT_LA + a] = -0.5f * trace(PdS[a]);
  }
  int q = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++q) {
      Sym2 t = congruence(A, gs.d2[q]);
      Sym2 d2S = {tau * t.a, tau * t.b, tau * t.c};
      Mat2 X = mul(PdS[a], PdS[b]);            // P dSa P dSb
      Sym2 two = sym_plus_t(mul(X, Pm));       // P dSa P dSb P + P dSb P dSa P
      Mat2 Pd2 = mul(Pm, d2S);
      Sym2 third = to_sym(mul(Pd2, Pm));       // P d2S P
      // d2P = two - third ; store -1/2 d2P
      out[GT_QAB + 3 * q + 0] = -0.5f * (two.a - third.a);
      out[GT_QAB + 3 * q + 1] = -0.5f * (two.b - third.b);
      out[GT_QAB + 3 * q + 2] = -0.5f * (two.c - third.c);
      out[GT_LAB + q] = -0.5f * (trace(Pd2) - trace(X));
    }
  out[42] = 0.f;
  out[43] = 0.f;
}

__device__ void star_entry(const ProblemDev& P, const ImageDev& im, const PatchDev& pt, int patch, const double* th,
                           double ox, double oy, int k, float* out) {
  PsfComp pc = load_psf(P.psf + (size_t)patch * 18, k);
  double px, py;
  source_pixel_pos(im, th, ox, oy, px, py);
  star_value_entry(pc, px, py, out);
  out[6] = out[7] = 0.f;
}

// ------------------------------------------------------------------------------ background
constexpr int NB_CHUNK = 8;   // neighbours staged per pass

__global__ void __launch_bounds__(BLOCK) background_kernel(ProblemDev P, const double* __restrict__ nbr_theta) {
  __shared__ __align__(16) float tab[NB_CHUNK][NCOMP * 6];
  __shared__ float cst[NB_CHUNK][10];   // A0 A1 C0 C1 Cx L10 L11 e
  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const ImageDev im = P.images[pt.image];
  const int tid = threadIdx.x;
  const int nn = pt.nbr_end - pt.nbr_begin;
  float bE[8], bV[8];
  constexpr int MAXPPT = 8;
  const int ppt = (t.count + BLOCK - 1) / BLOCK;
#pragma unroll
  for (int r = 0; r < MAXPPT; ++r) bE[r] = bV[r] = 0.f;
  for (int c0 = 0; c0 < nn; c0 += NB_CHUNK) {
    const int nc = min(NB_CHUNK, nn - c0);
    __syncthreads();
    for (int w = tid; w < nc * (NCOMP + 1); w += BLOCK) {
      const int q = w / (NCOMP + 1), c = w % (NCOMP + 1);
      const int np = P.nbr[pt.nbr_begin + c0 + q];
      const PatchDev nb = P.patches[np];
      const double* th = nbr_theta + (size_t)nb.source * NP;
      if (c < NSTAR) {
        PsfComp pc = load_psf(P.psf + (size_t)np * 18, c);
        double px, py;
        source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
        star_value_entry(pc, px, py, &tab[q][6 * c]);
      } else if (c < NCOMP) {
        const int g = c - NSTAR, k = g / NMIX, j = g % NMIX;
        PsfComp pc = load_psf(P.psf + (size_t)np * 18, k);
        double px, py;
        source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
        GalShape gs;
        galaxy_shape(th[3], th[4], th[5], gs);
        const float A[4] = {(float)im.A[0], (float)im.A[1], (float)im.A[2], (float)im.A[3]};
        gal_value_entry(pc, congruence(A, gs.S), P.nu[j], P.tau[j], px, py, &tab[q][6 * c]);
      } else {
        SNConst sc;
        sn_constants(th, im.band, im.iota, sc);
        cst[q][0] = sc.A0;
        cst[q][1] = sc.A1;
        cst[q][2] = sc.C0;
        cst[q][3] = sc.C1;
        cst[q][4] = sc.Cx;
        cst[q][5] = sc.L10;
        cst[q][6] = sc.L11;
        cst[q][7] = sc.e;
      }
    }
    __syncthreads();
    for (int r = 0; r < ppt && r < MAXPPT; ++r) {
      const int i = r * BLOCK + tid;
      if (i >= t.count) break;
      const int idx = t.start + i;
      const int row = idx / pt.w, col = idx - row * pt.w;
      const float fx = (float)col, fy = (float)row;
      for (int q = 0; q < nc; ++q) {
        float f0 = 0.f, fE = 0.f, fD = 0.f;
#pragma unroll
        for (int c = 0; c < NSTAR; ++c) f0 += gauss_value(&tab[q][6 * c], fx, fy);
        for (int k = 0; k < CELESTE_NPSF; ++k) {
#pragma unroll
          for (int j = 0; j < CELESTE_NEXP; ++j) fE += gauss_value(&tab[q][6 * (NSTAR + k * NMIX + j)], fx, fy);
#pragma unroll
          for (int j = CELESTE_NEXP; j < NMIX; ++j) fD += gauss_value(&tab[q][6 * (NSTAR + k * NMIX + j)], fx, fy);
        }
        const float f1 = fE + cst[q][7] * (fD - fE);
        bE[r] += cst[q][0] * f0 + cst[q][1] * f1;
        const float dx = cst[q][5] * f0 - cst[q][6] * f1;
        bV[r] += cst[q][2] * f0 * f0 + cst[q][3] * f1 * f1 + cst[q][4] * dx * dx;
      }
    }
  }
  for (int r = 0; r < ppt && r < MAXPPT; ++r) {
    const int i = r * BLOCK + tid;
    if (i >= t.count) break;
    float4* v = P.pix + pt.pix_off + t.start + i;
    float4 o = *v;
    o.y = im.sky + im.iota * bE[r];
    o.z = im.iota * im.iota * bV[r];
    *v = o;
  }
}

// ------------------------------------------------------------------------------ full kernel
struct Acc {
  float v[NACC];
};

template <int PPT>
__global__ void __launch_bounds__(BLOCK) elbo_full_kernel(ProblemDev P, const double* __restrict__ theta) {
  __shared__ __align__(16) float gtab[NGAL * GT_STRIDE];
  __shared__ __align__(16) float stab[NSTAR * ST_STRIDE];
  __shared__ __align__(16) float4 spix[BLOCK * PPT];
  __shared__ SNConst cst;
  __shared__ __align__(8) uint64_t bar;
  __shared__ float red[BLOCK / 32][NACC];

  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const int s = pt.source;
  if (!(P.flags[s] & FLAG_FULL)) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    atomicAdd(P.counters + 0, (unsigned long long)t.count);
  }
  __syncthreads();
  if (tid == 0) bulk_load(spix, P.pix + pt.pix_off + t.start, (uint32_t)t.count * 16u, &bar);
  const ImageDev im = P.images[pt.image];
  const double* th = theta + (size_t)s * NP;
  if (tid < NSTAR) {
    star_entry(P, im, pt, t.patch, th, pt.x0, pt.y0, tid, &stab[tid * ST_STRIDE]);
  } else if (tid < NSTAR + NGAL) {
    gal_full_entry(P, im, pt, t.patch, th, tid - NSTAR, &gtab[(tid - NSTAR) * GT_STRIDE]);
  } else if (tid == 64) {
    sn_constants(th, im.band, im.iota, cst);
  }
  bool ok = mbar_wait(&bar, 0, WAIT_BUDGET);
  if (!ok) {
    atomicExch(P.err + ERR_TIMEOUT, 1);
    mbar_wait(&bar, 0, WAIT_BUDGET);
  }
  __syncthreads();
  if (!ok) {
    if (tid < NACC) P.partials[(size_t)blockIdx.x * NACC + tid] = __int_as_float(0x7fc00000);
    return;
  }

  float acc[NACC];
#pragma unroll
  for (int q = 0; q < NACC; ++q) acc[q] = 0.f;

  const SNConst c = cst;
#pragma unroll 1
  for (int r = 0; r < PPT; ++r) {
    const int i = r * BLOCK + tid;
    if (i >= t.count) break;
    const int idx = t.start + i;
    const int row = idx / pt.w, col = idx - row * pt.w;
    const float fx = (float)col, fy = (float)row;
    const float4 pv = spix[i];

    // ---- star profile: value, d/dmu, d2/dmu2
    float f0 = 0.f, f0m[2] = {0.f, 0.f}, f0mm[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NSTAR; ++k) {
      const float* tb = &stab[k * ST_STRIDE];
      const float d0 = fx - tb[0], d1 = fy - tb[1];
      const float q = tb[3] * d0 * d0 + 2.f * tb[4] * d0 * d1 + tb[5] * d1 * d1;
      const float N = exp2f(fmaf(q, -0.5f * LOG2E, tb[2]));
      const float z0 = tb[3] * d0 + tb[4] * d1, z1 = tb[4] * d0 + tb[5] * d1;
      f0 += N;
      f0m[0] += N * z0;
      f0m[1] += N * z1;
      f0mm[0] += N * (z0 * z0 - tb[3]);
      f0mm[1] += N * (z0 * z1 - tb[4]);
      f0mm[2] += N * (z1 * z1 - tb[5]);
    }

    // ---- galaxy families (exp, deV): value and derivatives over (mu0, mu1, axis, angle, scale)
    float F[2], Fv[2][5], Fvv[2][15];
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
      F[fam] = 0.f;
#pragma unroll
      for (int a = 0; a < 5; ++a) Fv[fam][a] = 0.f;
#pragma unroll
      for (int a = 0; a < 15; ++a) Fvv[fam][a] = 0.f;
    }
#pragma unroll 1
    for (int k = 0; k < CELESTE_NPSF; ++k) {
#pragma unroll
      for (int j = 0; j < NMIX; ++j) {
        const int fam = j < CELESTE_NEXP ? 0 : 1;
        const float* tb = &gtab[(k * NMIX + j) * GT_STRIDE];
        const float d0 = fx - tb[GT_MU], d1 = fy - tb[GT_MU + 1];
        const float s0 = d0 * d0, s1 = 2.f * d0 * d1, s2 = d1 * d1;
        const float q = tb[GT_P] * s0 + tb[GT_P + 1] * s1 + tb[GT_P + 2] * s2;
        const float N = exp2f(fmaf(q, -0.5f * LOG2E, tb[GT_LW2]));
        const float z0 = tb[GT_P] * d0 + tb[GT_P + 1] * d1, z1 = tb[GT_P + 1] * d0 + tb[GT_P + 2] * d1;
        float b[3], y0[3], y1[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float* Q = tb + GT_QA + 3 * a;
          b[a] = tb[GT_LA + a] + Q[0] * s0 + Q[1] * s1 + Q[2] * s2;
          // (dP/da) d = -2 (Q_a d)
          y0[a] = -2.f * (Q[0] * d0 + Q[1] * d1);
          y1[a] = -2.f * (Q[1] * d0 + Q[2] * d1);
        }
        const float Nz0 = N * z0, Nz1 = N * z1;
        F[fam] += N;
        Fv[fam][0] += Nz0;
        Fv[fam][1] += Nz1;
        float Nb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Nb[a] = N * b[a];
          Fv[fam][2 + a] += Nb[a];
        }
        Fvv[fam][tri5(0, 0)] += Nz0 * z0 - N * tb[GT_P];
        Fvv[fam][tri5(0, 1)] += Nz0 * z1 - N * tb[GT_P + 1];
        Fvv[fam][tri5(1, 1)] += Nz1 * z1 - N * tb[GT_P + 2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          Fvv[fam][tri5(0, 2 + a)] += Nz0 * b[a] + N * y0[a];
          Fvv[fam][tri5(1, 2 + a)] += Nz1 * b[a] + N * y1[a];
        }
        int pq = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int bb = a; bb < 3; ++bb, ++pq) {
            const float* Q = tb + GT_QAB + 3 * pq;
            const float cab = tb[GT_LAB + pq] + Q[0] * s0 + Q[1] * s1 + Q[2] * s2;
            Fvv[fam][tri5(2 + a, 2 + bb)] += Nb[a] * b[bb] + N * cab;
          }
      }
    }

    // ---- galaxy profile over G6 = (mu0, mu1, dev, axis, angle, scale)
    const int v2g[5] = {0, 1, 3, 4, 5};
    float f1 = F[0] + c.e * (F[1] - F[0]);
    float f1g[6], f1gg[21];
    f1g[2] = c.e1 * (F[1] - F[0]);
#pragma unroll
    for (int a = 0; a < 5; ++a) f1g[v2g[a]] = Fv[0][a] + c.e * (Fv[1][a] - Fv[0][a]);
    f1gg[tri6(2, 2)] = c.e2 * (F[1] - F[0]);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const int ga = v2g[a];
      f1gg[ga < 2 ? tri6(ga, 2) : tri6(2, ga)] = c.e1 * (Fv[1][a] - Fv[0][a]);
#pragma unroll
      for (int bb = a; bb < 5; ++bb)
        f1gg[tri6(ga, v2g[bb])] = Fvv[0][tri5(a, bb)] + c.e * (Fvv[1][tri5(a, bb)] - Fvv[0][tri5(a, bb)]);
    }

    // ---- pixel rate moments and the pixel term
    const float iota = c.iota, iota2 = iota * iota;
    const float EG = c.A0 * f0 + c.A1 * f1;
    const float dxv = c.L10 * f0 - c.L11 * f1;
    const float VG = c.C0 * f0 * f0 + c.C1 * f1 * f1 + c.Cx * dxv * dxv;
    const float E = pv.y + iota * EG;
    const float V = pv.z + iota2 * VG;
    const float x = pv.x;
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
    const float w1 = iota * lE - 2.f * iota2 * EG * lV;
    const float w2 = iota2 * lV;
    const float c00 = iota2 * lEE - 4.f * iota2 * iota * EG * lEV - 2.f * iota2 * lV;
    const float c01 = iota2 * iota * lEV;

    // ---- reduced Jacobian rows
    float yE[NRED], yV[NRED];
    yE[0] = c.A0 * f0m[0] + c.A1 * f1g[0];
    yE[1] = c.A0 * f0m[1] + c.A1 * f1g[1];
    yV[0] = 2.f * (c.B0 * f0 * f0m[0] + c.B1 * f1 * f1g[0]);
    yV[1] = 2.f * (c.B0 * f0 * f0m[1] + c.B1 * f1 * f1g[1]);
#pragma unroll
    for (int a = 2; a < 6; ++a) {
      yE[a] = c.A1 * f1g[a];
      yV[a] = 2.f * c.B1 * f1 * f1g[a];
    }
    yE[6] = c.aE1 * f1 - c.aE0 * f0;
    yV[6] = c.aV1 * f1 * f1 - c.aV0 * f0 * f0;
    yE[7] = f0;
    yE[8] = f1;
    yE[9] = 0.f;
    yE[10] = 0.f;
    yV[7] = 0.f;
    yV[8] = 0.f;
    yV[9] = f0 * f0;
    yV[10] = f1 * f1;

    acc[ACC_L] += ell;
    // S1 = w1 [f0, f0_mu(2), f1, f1_g(6)] ; S2 = w2 [f0^2, d f0^2 (2), f1^2, d f1^2 (6)]
    acc[ACC_S1 + 0] += w1 * f0;
    acc[ACC_S1 + 1] += w1 * f0m[0];
    acc[ACC_S1 + 2] += w1 * f0m[1];
    acc[ACC_S1 + 3] += w1 * f1;
    acc[ACC_S2 + 0] += w2 * f0 * f0;
    acc[ACC_S2 + 1] += w2 * 2.f * f0 * f0m[0];
    acc[ACC_S2 + 2] += w2 * 2.f * f0 * f0m[1];
    acc[ACC_S2 + 3] += w2 * f1 * f1;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      acc[ACC_S1 + 4 + a] += w1 * f1g[a];
      acc[ACC_S2 + 4 + a] += w2 * 2.f * f1 * f1g[a];
    }
    // second-order profile block: w1 (A0 d2f0 + A1 d2f1) + w2 (B0 d2 f0^2 + B1 d2 f1^2)
    const float u1 = w1 * c.A1, u2 = 2.f * w2 * c.B1;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int bb = a; bb < 6; ++bb) {
        const int q = tri6(a, bb);
        float h = u1 * f1gg[q] + u2 * (f1g[a] * f1g[bb] + f1 * f1gg[q]);
        if (a < 2 && bb < 2) {
          const int qs = a + bb;   // (0,0)->0, (0,1)->1, (1,1)->2
          h += w1 * c.A0 * f0mm[qs] + 2.f * w2 * c.B0 * (f0m[a] * f0m[bb] + f0 * f0mm[qs]);
        }
        acc[ACC_HP + q] += h;
      }
    // Jacobian cross-product: c00 yE yE^T + c01 (yE yV^T + yV yE^T)
#pragma unroll
    for (int a = 0; a < NRED; ++a) {
      const float ta = c00 * yE[a] + c01 * yV[a];
      const float ua = c01 * yE[a];
#pragma unroll
      for (int bb = a; bb < NRED; ++bb) acc[ACC_M + tri11(a, bb)] += ta * yE[bb] + ua * yV[bb];
    }
  }

  // ---- block reduction of the 108 sums
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NACC; ++q) {
    float v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (tid < NACC) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < BLOCK / 32; ++w) v += red[w][tid];
    P.partials[(size_t)blockIdx.x * NACC + tid] = v;
  }
}

// ------------------------------------------------------------------------------ value kernel
template <int PPT>
__global__ void __launch_bounds__(BLOCK) elbo_value_kernel(ProblemDev P, const double* __restrict__ theta, int flag_mask) {
  __shared__ __align__(16) float tab[NCOMP * 6];
  __shared__ __align__(16) float4 spix[BLOCK * PPT];
  __shared__ SNConst cst;
  __shared__ __align__(8) uint64_t bar;
  __shared__ float red[BLOCK / 32];

  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const int s = pt.source;
  if (!(P.flags[s] & flag_mask)) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    atomicAdd(P.counters + 1, (unsigned long long)t.count);
  }
  __syncthreads();
  if (tid == 0) bulk_load(spix, P.pix + pt.pix_off + t.start, (uint32_t)t.count * 16u, &bar);
  const ImageDev im = P.images[pt.image];
  const double* th = theta + (size_t)s * NP;
  if (tid < NSTAR) {
    PsfComp pc = load_psf(P.psf + (size_t)t.patch * 18, tid);
    double px, py;
    source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
    star_value_entry(pc, px, py, &tab[6 * tid]);
  } else if (tid < NCOMP) {
    const int g = tid - NSTAR, k = g / NMIX, j = g % NMIX;
    PsfComp pc = load_psf(P.psf + (size_t)t.patch * 18, k);
    double px, py;
    source_pixel_pos(im, th, pt.x0, pt.y0, px, py);
    GalShape gs;
    galaxy_shape(th[3], th[4], th[5], gs);
    const float A[4] = {(float)im.A[0], (float)im.A[1], (float)im.A[2], (float)im.A[3]};
    gal_value_entry(pc, congruence(A, gs.S), P.nu[j], P.tau[j], px, py, &tab[6 * tid]);
  } else if (tid == 64) {
    sn_constants(th, im.band, im.iota, cst);
  }
  bool ok = mbar_wait(&bar, 0, WAIT_BUDGET);
  if (!ok) {
    atomicExch(P.err + ERR_TIMEOUT, 1);
    mbar_wait(&bar, 0, WAIT_BUDGET);
  }
  __syncthreads();
  if (!ok) {
    if (tid == 0) P.vpartials[blockIdx.x] = __int_as_float(0x7fc00000);
    return;
  }
  const SNConst c = cst;
  float sum = 0.f;
#pragma unroll 1
  for (int r = 0; r < PPT; ++r) {
    const int i = r * BLOCK + tid;
    if (i >= t.count) break;
    const int idx = t.start + i;
    const int row = idx / pt.w, col = idx - row * pt.w;
    const float fx = (float)col, fy = (float)row;
    const float4 pv = spix[i];
    float f0 = 0.f, fE = 0.f, fD = 0.f;
#pragma unroll
    for (int k = 0; k < NSTAR; ++k) f0 += gauss_value(&tab[6 * k], fx, fy);
#pragma unroll 1
    for (int k = 0; k < CELESTE_NPSF; ++k) {
#pragma unroll
      for (int j = 0; j < CELESTE_NEXP; ++j) fE += gauss_value(&tab[6 * (NSTAR + k * NMIX + j)], fx, fy);
#pragma unroll
      for (int j = CELESTE_NEXP; j < NMIX; ++j) fD += gauss_value(&tab[6 * (NSTAR + k * NMIX + j)], fx, fy);
    }
    const float f1 = fE + c.e * (fD - fE);
    const float EG = c.A0 * f0 + c.A1 * f1;
    const float dxv = c.L10 * f0 - c.L11 * f1;
    const float VG = c.C0 * f0 * f0 + c.C1 * f1 * f1 + c.Cx * dxv * dxv;
    const float E = pv.y + c.iota * EG;
    const float V = pv.z + c.iota * c.iota * VG;
    const float x = pv.x;
    if (x > 0.f) {
      const float dEx = E - x;
      sum += pv.w + x * log1pf(dEx / x) - dEx - 0.5f * x * V / (E * E);
    } else {
      sum += -E;
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
    P.vpartials[blockIdx.x] = v;
  }
}

// ------------------------------------------------------------------------------ launchers
cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  background_kernel<<<P.n_tiles, BLOCK, 0, st>>>(P, nbr_theta);
  return cudaGetLastError();
}

cudaError_t launch_full(const ProblemDev& P, const double* theta, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  switch (P.tile_pixels) {
    case 128: elbo_full_kernel<1><<<P.n_tiles, BLOCK, 0, st>>>(P, theta); break;
    case 256: elbo_full_kernel<2><<<P.n_tiles, BLOCK, 0, st>>>(P, theta); break;
    case 512: elbo_full_kernel<4><<<P.n_tiles, BLOCK, 0, st>>>(P, theta); break;
    default: elbo_full_kernel<8><<<P.n_tiles, BLOCK, 0, st>>>(P, theta); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_value(const ProblemDev& P, const double* theta, int flag_mask, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  switch (P.tile_pixels) {
    case 128: elbo_value_kernel<1><<<P.n_tiles, BLOCK, 0, st>>>(P, theta, flag_mask); break;
    case 256: elbo_value_kernel<2><<<P.n_tiles, BLOCK, 0, st>>>(P, theta, flag_mask); break;
    case 512: elbo_value_kernel<4><<<P.n_tiles, BLOCK, 0, st>>>(P, theta, flag_mask); break;
    default: elbo_value_kernel<8><<<P.n_tiles, BLOCK, 0, st>>>(P, theta, flag_mask); break;
  }
  return cudaGetLastError();
}

}  // namespace celeste
