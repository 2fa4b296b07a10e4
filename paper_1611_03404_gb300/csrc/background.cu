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
constexpr int NB_CHUNK = 8;   // neighbours staged per pass

__global__ void __launch_bounds__(BLOCK) background_kernel(ProblemDev P, const double* __restrict__ nbr_theta,
                                                           int clip) {
  __shared__ __align__(16) float tab[NB_CHUNK][NCOMP * 6];
  __shared__ float cst[NB_CHUNK][10];   // A0 A1 C0 C1 Cx L10 L11 e
  __shared__ int win[NB_CHUNK][4];      // neighbour's window relative to this patch: x0, y0, x1, y1 (exclusive)
  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const ImageDev im = P.images[pt.image];
  const int tid = threadIdx.x;
  const int nn = pt.nbr_end - pt.nbr_begin;
  float bE[8], bV[8];
  int cover[8];   // windows holding the pixel (its own and the neighbours'), window mode
  constexpr int MAXPPT = 8;
  const int ppt = (t.count + BLOCK - 1) / BLOCK;
#pragma unroll
  for (int r = 0; r < MAXPPT; ++r) {
    bE[r] = bV[r] = 0.f;
    cover[r] = 1;
  }
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
        win[q][0] = nb.x0 - pt.x0;
        win[q][1] = nb.y0 - pt.y0;
        win[q][2] = nb.x0 - pt.x0 + nb.w;
        win[q][3] = nb.y0 - pt.y0 + nb.h;
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
        if (clip && (col < win[q][0] || col >= win[q][2] || row < win[q][1] || row >= win[q][3])) continue;
        cover[r] += 1;
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
    if (clip && P.pweight) P.pweight[pt.pix_off + t.start + i] = 1.f / (float)cover[r];
  }
}

cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, int clip, cudaStream_t st) {
  if (P.n_tiles == 0) return cudaSuccess;
  background_kernel<<<P.n_tiles, BLOCK, 0, st>>>(P, nbr_theta, clip);
  return cudaGetLastError();
}

}  // namespace celeste
