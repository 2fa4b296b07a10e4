// Neighbour background of every patch pixel (paper, Sec. "Variational Inference": each source is
// optimised with its neighbours held fixed).  For pixel m of source s's patch in image n:
//   bE(m) = sky_n + iota_n sum_{s' in nbr(s, n)} E[G_s'](m),  bV(m) = iota_n^2 sum Var[G_s'](m),
// with the neighbours' full variational moments (value-only profiles, no derivatives).
// clip = 1 (the joint objective's per-source blocks): a neighbour counts only on the pixels of its
// own window, as every source does in the objective over all sources jointly.
#include "celeste_internal.cuh"
#include "kernels.h"

namespace celeste {

// ------------------------------------------------------------------------------ background
// The neighbours' value tables come from the table kernel, run once per rendering on every patch
// at nbr_theta (component means relative to the neighbour's own patch origin, precisions, weighted
// normalisers, brightness constants): per tile only a shift of the means and float4 copies remain.
constexpr int NB_CHUNK = 8;   // neighbours staged per pass

struct NbrStage {
  float4 gal[NGAL];            // per pair of components (the table's value prefix): (P00, P00', P01,
                               // P01') * (-1/2 log2 e), then (P11, P11') * (-1/2 log2 e), (W, W')
  float4 star[NSTAR];
  float mu[2 * CELESTE_NPSF];  // component means relative to the target patch's origin
  float c[8];                  // A0 A1 C0 C1 Cx L10 L11 e
  int win[4];                  // the neighbour's window relative to the target patch: x0, y0, x1, y1 (exclusive)
};

__global__ void __launch_bounds__(BLOCK) background_kernel(ProblemDev P, int clip) {
  __shared__ NbrStage nbs[NB_CHUNK];
  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const ImageDev im = P.images[pt.image];
  const int tid = threadIdx.x;
  const int nn = pt.nbr_end - pt.nbr_begin;
  constexpr int MAXPPT = 8;
  constexpr float NL2 = -0.5f * LOG2E;
  float bE[MAXPPT], bV[MAXPPT];
  int cover[MAXPPT];   // windows holding the pixel (its own and the neighbours'), window mode
  const int ppt = (t.count + BLOCK - 1) / BLOCK;
#pragma unroll
  for (int r = 0; r < MAXPPT; ++r) {
    bE[r] = bV[r] = 0.f;
    cover[r] = 1;
  }
  constexpr int ITEMS = NGAL + NSTAR + 2;
  for (int c0 = 0; c0 < nn; c0 += NB_CHUNK) {
    const int nc = min(NB_CHUNK, nn - c0);
    __syncthreads();
    for (int w = tid; w < nc * ITEMS; w += BLOCK) {
      const int q = w / ITEMS, e = w % ITEMS;
      const int np = P.nbr[pt.nbr_begin + c0 + q];
      const float* tb = P.ptab + (size_t)np * TB_FLOATS;
      NbrStage& S = nbs[q];
      if (e < NGAL) {
        const float4 g = *reinterpret_cast<const float4*>(tb + TB_VAL + 4 * e);
        S.gal[e] = (e & 1) ? make_float4(g.x * NL2, g.y * NL2, g.z, g.w)
                           : make_float4(g.x * NL2, g.y * NL2, g.z * NL2, g.w * NL2);
      } else if (e < NGAL + NSTAR) {
        const float4 g = *reinterpret_cast<const float4*>(tb + TB_STAR + 4 * (e - NGAL));
        S.star[e - NGAL] = make_float4(g.x, g.y * NL2, g.z * NL2, g.w * NL2);
      } else if (e == NGAL + NSTAR) {
        const PatchDev nb = P.patches[np];
        const float dx = (float)(nb.x0 - pt.x0), dy = (float)(nb.y0 - pt.y0);
#pragma unroll
        for (int k = 0; k < CELESTE_NPSF; ++k) {
          S.mu[2 * k] = tb[TB_MU + 2 * k] + dx;
          S.mu[2 * k + 1] = tb[TB_MU + 2 * k + 1] + dy;
        }
        S.win[0] = nb.x0 - pt.x0;
        S.win[1] = nb.y0 - pt.y0;
        S.win[2] = nb.x0 - pt.x0 + nb.w;
        S.win[3] = nb.y0 - pt.y0 + nb.h;
      } else {
        const SNConst& sc = *reinterpret_cast<const SNConst*>(tb + TB_SNC);
        S.c[0] = sc.A0;
        S.c[1] = sc.A1;
        S.c[2] = sc.C0;
        S.c[3] = sc.C1;
        S.c[4] = sc.Cx;
        S.c[5] = sc.L10;
        S.c[6] = sc.L11;
        S.c[7] = sc.e;
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
        const NbrStage& S = nbs[q];
        if (clip && (col < S.win[0] || col >= S.win[2] || row < S.win[1] || row >= S.win[3])) continue;
        cover[r] += 1;
        // galaxy components two at a time, on packed two-wide float32 arithmetic
        float f0 = 0.f;
        float2 fE = make_float2(0.f, 0.f), fD = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < CELESTE_NPSF; ++k) {
          const float d0 = fx - S.mu[2 * k], d1 = fy - S.mu[2 * k + 1];
          const float s0 = d0 * d0, s1 = 2.f * d0 * d1, s2 = d1 * d1;
          const float4 st = S.star[k];
          f0 += st.x * exp2f(st.y * s0 + st.z * s1 + st.w * s2);
          const float2 S0 = make_float2(s0, s0), S1 = make_float2(s1, s1), S2 = make_float2(s2, s2);
#pragma unroll
          for (int pr = 0; pr < NMIX / 2; ++pr) {
            const float4 a = S.gal[2 * (k * NMIX / 2 + pr)], b = S.gal[2 * (k * NMIX / 2 + pr) + 1];
            const float2 q = __ffma2_rn(make_float2(b.x, b.y), S2,
                                        __ffma2_rn(make_float2(a.z, a.w), S1, __fmul2_rn(make_float2(a.x, a.y), S0)));
            const float2 v = __fmul2_rn(make_float2(b.z, b.w), make_float2(exp2f(q.x), exp2f(q.y)));
            if (pr < CELESTE_NEXP / 2)
              fE = __fadd2_rn(fE, v);
            else
              fD = __fadd2_rn(fD, v);
          }
        }
        const float fEs = fE.x + fE.y, fDs = fD.x + fD.y;
        const float f1 = fEs + S.c[7] * (fDs - fEs);
        bE[r] += S.c[0] * f0 + S.c[1] * f1;
        const float dx = S.c[5] * f0 - S.c[6] * f1;
        bV[r] += S.c[2] * f0 * f0 + S.c[3] * f1 * f1 + S.c[4] * dx * dx;
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
    if (clip && P.pweight) P.pweight[pt.pix_off + t.start + i] = 1.f / (float)cover[r];
  }
}

// Value tables of every patch at nbr_theta (all sources flagged; the flags, worklists and tables are
// working state that every later evaluation rebuilds), then the background of every tile.
cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, int clip, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  cudaError_t e = launch_set_flags(P, FLAG_VALUE, st);
  if (e == cudaSuccess) e = launch_worklists(P, FLAG_VALUE, st);
  if (e == cudaSuccess) e = launch_tables(P, nbr_theta, false, st);
  if (e != cudaSuccess) return e;
  background_kernel<<<P.n_tiles, BLOCK, 0, st>>>(P, clip);
  return cudaGetLastError();
}

}  // namespace celeste
