// Problem layout, validation, workspace binding and the per-patch PSF / pixel-gather kernels.
//
// Paper, Sec. "Parallel Work Decomposition": to optimise one light source Celeste needs
// every image containing it, the source's initial estimate and the initial estimates of
// nearby sources that may overlap it.  Here that is laid out once on the host: every
// (source, image) patch, its neighbours in the same image, and fixed-size pixel tiles that
// the kernels process; the images themselves stay resident in device memory.
#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "celeste_internal.cuh"
#include "problem.h"

namespace celeste {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(CELESTE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaError_t clear_timeout(const ProblemDev& D, cudaStream_t st) {
  return cudaMemsetAsync(D.err + ERR_TIMEOUT, 0, sizeof(int), st);
}

int device_errors(const ProblemDev& D, cudaStream_t st) {
  int err[4];
  cudaError_t e = cudaMemcpyAsync(err, D.err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error words");
  if (err[ERR_TIMEOUT]) return fail(CELESTE_ERR_TIMEOUT, "a pixel kernel's bulk copy did not complete in time");
  if (err[ERR_BAD_PIXEL]) return fail(CELESTE_ERR_INVALID_ARG, "an image holds negative or non-finite counts");
  return CELESTE_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------------------ kernels
// PSF of every patch, evaluated at the source's catalog position in that image.
__global__ void psf_setup_kernel(ProblemDev P) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n_patches) return;
  const PatchDev pt = P.patches[p];
  const ImageDev im = P.images[pt.image];
  const double* u = P.u0 + 2 * pt.source;
  double x = im.A[0] * u[0] + im.A[1] * u[1] + im.o[0];
  double y = im.A[2] * u[0] + im.A[3] * u[1] + im.o[1];
  double xh = 2.0 * x / (im.W - 1) - 1.0, yh = 2.0 * y / (im.H - 1) - 1.0;
  double basis[6] = {1.0, xh, yh, xh * xh, xh * yh, yh * yh};
  double par[CELESTE_NPSF][6];
  const double* psf = P.psf_coef + (size_t)pt.image * CELESTE_NPSF * 36;
  for (int k = 0; k < CELESTE_NPSF; ++k)
    for (int q = 0; q < 6; ++q) {
      double v = 0.0;
      for (int b = 0; b < 6; ++b) v += psf[(k * 6 + q) * 6 + b] * basis[b];
      par[k][q] = v;
    }
  double mx = fmax(par[0][0], fmax(par[1][0], par[2][0]));
  double wsum = 0.0, w[CELESTE_NPSF];
  for (int k = 0; k < CELESTE_NPSF; ++k) {
    w[k] = exp(par[k][0] - mx);
    wsum += w[k];
  }
  float* out = P.psf + (size_t)p * 18;
  for (int k = 0; k < CELESTE_NPSF; ++k) {
    double sx = exp(par[k][3]), sy = exp(par[k][4]), rho = tanh(par[k][5]);
    out[6 * k + 0] = (float)(w[k] / wsum);
    out[6 * k + 1] = (float)par[k][1];
    out[6 * k + 2] = (float)par[k][2];
    out[6 * k + 3] = (float)(sx * sx);
    out[6 * k + 4] = (float)(rho * sx * sy);
    out[6 * k + 5] = (float)(sy * sy);
  }
}

// Gather each patch pixel's count and its log-factorial term x log x - x - lgamma(x+1)
// (float64, so that the float32 pixel term keeps its precision), once per bind.
__global__ void gather_pixels_kernel(ProblemDev P) {
  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const ImageDev im = P.images[pt.image];
  for (int i = threadIdx.x; i < t.count; i += blockDim.x) {
    int idx = t.start + i;
    int row = idx / pt.w, col = idx - row * pt.w;
    float x = im.pixels[(size_t)(pt.y0 + row) * im.W + (pt.x0 + col)];
    if (!(x >= 0.f) || !isfinite(x)) {
      atomicExch(P.err + ERR_BAD_PIXEL, 1);
      x = 0.f;
    }
    double xd = x;
    double kappa = xd > 0 ? xd * log(xd) - xd - lgamma(xd + 1.0) : 0.0;
    float4 v = P.pix[pt.pix_off + idx];
    v.x = x;
    v.w = (float)kappa;
    P.pix[pt.pix_off + idx] = v;
  }
}

}  // namespace celeste

using namespace celeste;

// ------------------------------------------------------------------------------ host API
static bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

extern "C" int celeste_problem_create(const celeste_problem_desc* d, celeste_problem** out) {
  if (!d || !out) return fail(CELESTE_ERR_INVALID_ARG, "null descriptor or output pointer");
  *out = nullptr;
  if (d->n_images <= 0 || !d->images) return fail(CELESTE_ERR_INVALID_ARG, "n_images must be > 0");
  if (d->n_sources <= 0 || !d->u0 || !d->radius) return fail(CELESTE_ERR_INVALID_ARG, "n_sources must be > 0");
  int tp = d->tile_pixels ? d->tile_pixels : 128;
  if (tp != 128 && tp != 256 && tp != 512 && tp != 1024)
    return fail(CELESTE_ERR_INVALID_ARG, "tile_pixels must be 128, 256, 512 or 1024");
  if (d->hessian_mode < CELESTE_HESS_FP32 || d->hessian_mode > CELESTE_HESS_TF32X3)
    return fail(CELESTE_ERR_INVALID_ARG, "hessian_mode must be 0 to 4");
  if (d->hessian_mode != CELESTE_HESS_FP32 && tp != 128)
    return fail(CELESTE_ERR_INVALID_ARG, "tensor-core hessian modes need tile_pixels 128");
  for (int n = 0; n < d->n_images; ++n) {
    const celeste_image_desc& im = d->images[n];
    if (im.height < 2 || im.width < 2 || im.height > (1 << 20) || im.width > (1 << 20))
      return fail(CELESTE_ERR_INVALID_ARG, "image %d: size %dx%d out of range", n, im.height, im.width);
    if (im.band < 0 || im.band > 4) return fail(CELESTE_ERR_INVALID_ARG, "image %d: band %d not in 0..4", n, im.band);
    if (!im.pixels) return fail(CELESTE_ERR_INVALID_ARG, "image %d: null pixels", n);
    if (!(im.sky > 0) || !std::isfinite(im.sky)) return fail(CELESTE_ERR_INVALID_ARG, "image %d: sky must be > 0", n);
    if (!(im.iota > 0) || !std::isfinite(im.iota)) return fail(CELESTE_ERR_INVALID_ARG, "image %d: iota must be > 0", n);
    if (!finite_all(im.wcs, 6)) return fail(CELESTE_ERR_INVALID_ARG, "image %d: non-finite wcs", n);
    double det = im.wcs[0] * im.wcs[3] - im.wcs[1] * im.wcs[2];
    if (!(std::fabs(det) > 1e-12)) return fail(CELESTE_ERR_INVALID_ARG, "image %d: singular wcs", n);
    if (!finite_all(&im.psf[0][0][0], CELESTE_NPSF * 36)) return fail(CELESTE_ERR_INVALID_ARG, "image %d: non-finite psf", n);
    // PSF parameters at the image corners stay in a sane range (sigma in [1e-3, 1e3] px, |rho| < 1).
    for (int c = 0; c < 4; ++c) {
      double xh = (c & 1) ? 1.0 : -1.0, yh = (c & 2) ? 1.0 : -1.0;
      double b[6] = {1, xh, yh, xh * xh, xh * yh, yh * yh};
      for (int k = 0; k < CELESTE_NPSF; ++k)
        for (int q = 3; q < 6; ++q) {
          double v = 0;
          for (int j = 0; j < 6; ++j) v += im.psf[k][q][j] * b[j];
          if (q < 5 && std::fabs(v) > 6.9) return fail(CELESTE_ERR_INVALID_ARG, "image %d: psf sigma out of range", n);
          if (q == 5 && std::fabs(v) > 5.0) return fail(CELESTE_ERR_INVALID_ARG, "image %d: psf correlation out of range", n);
        }
    }
  }
  for (int s = 0; s < d->n_sources; ++s) {
    if (!finite_all(d->u0 + 2 * s, 2)) return fail(CELESTE_ERR_INVALID_ARG, "source %d: non-finite position", s);
    if (d->radius[s] < 1 || d->radius[s] > CELESTE_MAX_RADIUS)
      return fail(CELESTE_ERR_INVALID_ARG, "source %d: radius %d not in 1..%d", s, d->radius[s], CELESTE_MAX_RADIUS);
  }
  if (!(d->priors[0] > 0 && d->priors[0] < 1) || !(d->priors[2] > 0) || !(d->priors[4] > 0) || !finite_all(d->priors, 5))
    return fail(CELESTE_ERR_INVALID_ARG, "priors must have 0<Phi<1 and positive variances");
  double se = 0, sd = 0;
  for (int j = 0; j < CELESTE_NEXP; ++j) {
    if (!(d->exp_nu[j] > 0) || !(d->exp_tau[j] > 0)) return fail(CELESTE_ERR_INVALID_ARG, "exp mixture entries must be > 0");
    se += d->exp_nu[j];
  }
  for (int j = 0; j < CELESTE_NDEV; ++j) {
    if (!(d->dev_nu[j] > 0) || !(d->dev_tau[j] > 0)) return fail(CELESTE_ERR_INVALID_ARG, "deV mixture entries must be > 0");
    sd += d->dev_nu[j];
  }
  if (std::fabs(se - 1) > 1e-6 || std::fabs(sd - 1) > 1e-6) return fail(CELESTE_ERR_INVALID_ARG, "mixture weights must sum to 1");

  celeste_problem* p = new celeste_problem();
  p->S = d->n_sources;
  p->tile_pixels = tp;
  p->hessian_mode = d->hessian_mode;
  p->images.assign(d->images, d->images + d->n_images);
  p->u0.assign(d->u0, d->u0 + 2 * (size_t)d->n_sources);
  p->radius.assign(d->radius, d->radius + d->n_sources);
  std::memcpy(p->priors, d->priors, sizeof(p->priors));
  for (int j = 0; j < CELESTE_NEXP; ++j) {
    p->nu[j] = (float)d->exp_nu[j];
    p->tau[j] = (float)d->exp_tau[j];
  }
  for (int j = 0; j < CELESTE_NDEV; ++j) {
    p->nu[CELESTE_NEXP + j] = (float)d->dev_nu[j];
    p->tau[CELESTE_NEXP + j] = (float)d->dev_tau[j];
  }
  build_layout(p);
  *out = p;
  return CELESTE_OK;
}

namespace celeste {

void build_layout(celeste_problem* p) {
  const int S = p->S, N = (int)p->images.size();
  p->src_patch.assign(S + 1, 0);
  p->patches.clear();
  for (int s = 0; s < S; ++s) {
    p->src_patch[s] = (int)p->patches.size();
    for (int n = 0; n < N; ++n) {
      const celeste_image_desc& im = p->images[n];
      double x = im.wcs[0] * p->u0[2 * s] + im.wcs[1] * p->u0[2 * s + 1] + im.wcs[4];
      double y = im.wcs[2] * p->u0[2 * s] + im.wcs[3] * p->u0[2 * s + 1] + im.wcs[5];
      double cxd = std::floor(x + 0.5), cyd = std::floor(y + 0.5);
      if (!(cxd >= 0 && cxd <= im.width - 1 && cyd >= 0 && cyd <= im.height - 1)) continue;
      int cx = (int)cxd, cy = (int)cyd, R = p->radius[s];
      PatchDev pt{};
      pt.source = s;
      pt.image = n;
      pt.x0 = std::max(cx - R, 0);
      pt.y0 = std::max(cy - R, 0);
      pt.w = std::min(cx + R, im.width - 1) - pt.x0 + 1;
      pt.h = std::min(cy + R, im.height - 1) - pt.y0 + 1;
      p->patches.push_back(pt);
    }
  }
  p->src_patch[S] = (int)p->patches.size();
  const int NPch = (int)p->patches.size();

  // neighbours: other sources whose patch in the same image overlaps (grid binning per image)
  const int CELL = 128;
  std::vector<std::vector<int>> nbr(NPch);
  for (int n = 0; n < N; ++n) {
    const celeste_image_desc& im = p->images[n];
    int gx = (im.width + CELL - 1) / CELL, gy = (im.height + CELL - 1) / CELL;
    std::vector<std::vector<int>> cells((size_t)gx * gy);
    for (int q = 0; q < NPch; ++q) {
      const PatchDev& a = p->patches[q];
      if (a.image != n) continue;
      for (int cy = a.y0 / CELL; cy <= (a.y0 + a.h - 1) / CELL; ++cy)
        for (int cx = a.x0 / CELL; cx <= (a.x0 + a.w - 1) / CELL; ++cx) cells[(size_t)cy * gx + cx].push_back(q);
    }
    for (int q = 0; q < NPch; ++q) {
      const PatchDev& a = p->patches[q];
      if (a.image != n) continue;
      std::vector<int>& lst = nbr[q];
      for (int cy = a.y0 / CELL; cy <= (a.y0 + a.h - 1) / CELL; ++cy)
        for (int cx = a.x0 / CELL; cx <= (a.x0 + a.w - 1) / CELL; ++cx)
          for (int r : cells[(size_t)cy * gx + cx]) {
            const PatchDev& b = p->patches[r];
            if (b.source == a.source) continue;
            if (b.x0 <= a.x0 + a.w - 1 && a.x0 <= b.x0 + b.w - 1 && b.y0 <= a.y0 + a.h - 1 && a.y0 <= b.y0 + b.h - 1)
              lst.push_back(r);
          }
      std::sort(lst.begin(), lst.end());
      lst.erase(std::unique(lst.begin(), lst.end()), lst.end());
    }
  }
  p->nbr.clear();
  p->tiles.clear();
  p->tile_pix.clear();
  long long off = 0;
  for (int q = 0; q < NPch; ++q) {
    PatchDev& a = p->patches[q];
    a.nbr_begin = (int)p->nbr.size();
    p->nbr.insert(p->nbr.end(), nbr[q].begin(), nbr[q].end());
    a.nbr_end = (int)p->nbr.size();
    a.pix_off = off;
    int npix = a.w * a.h;
    off += npix;
    a.tile_begin = (int)p->tiles.size();
    for (int st = 0; st < npix; st += p->tile_pixels) {
      p->tiles.push_back({q, st, std::min(p->tile_pixels, npix - st), 0});
      p->tile_pix.push_back(a.pix_off + st);
    }
    a.tile_end = (int)p->tiles.size();
  }
  p->n_pix = off;

  p->imgdev.resize(N);
  p->psf_coef.resize((size_t)N * CELESTE_NPSF * 36);
  for (int n = 0; n < N; ++n) {
    const celeste_image_desc& im = p->images[n];
    ImageDev& g = p->imgdev[n];
    g.pixels = im.pixels;
    g.H = im.height;
    g.W = im.width;
    g.band = im.band;
    g.sky = (float)im.sky;
    g.iota = (float)im.iota;
    for (int j = 0; j < 4; ++j) g.A[j] = im.wcs[j];
    g.o[0] = im.wcs[4];
    g.o[1] = im.wcs[5];
    std::memcpy(&p->psf_coef[(size_t)n * CELESTE_NPSF * 36], &im.psf[0][0][0], sizeof(double) * CELESTE_NPSF * 36);
  }

  // workspace layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  WsLayout& L = p->ws;
  L.images = take(sizeof(ImageDev) * N);
  L.patches = take(sizeof(PatchDev) * std::max(NPch, 1));
  L.tiles = take(sizeof(TileDev) * std::max<size_t>(p->tiles.size(), 1));
  L.tile_pix = take(sizeof(long long) * std::max<size_t>(p->tiles.size(), 1));
  L.src_patch = take(sizeof(int) * (S + 1));
  L.nbr = take(sizeof(int) * std::max<size_t>(p->nbr.size(), 1));
  L.u0 = take(sizeof(double) * 2 * S);
  L.psf_coef = take(sizeof(double) * p->psf_coef.size());
  L.psf = take(sizeof(float) * 18 * std::max(NPch, 1));
  L.pix = take(sizeof(float4) * std::max<long long>(p->n_pix, 1));
  L.srcmom = take(sizeof(float2) * std::max<long long>(p->n_pix, 1));
  L.ptab = take(sizeof(float) * TB_FLOATS * std::max(NPch, 1));
  L.partials = take(sizeof(float) * NACC * std::max<size_t>(p->tiles.size(), 1));
  L.vpartials = take(sizeof(float) * std::max<size_t>(p->tiles.size(), 1));
  L.flags = take(sizeof(int) * S);
  L.err = take(sizeof(int) * 4);
  L.counters = take(sizeof(unsigned long long) * 4);
  L.wl = take(sizeof(int) * (p->tiles.size() + NPch + S + 1));
  L.wl_count = take(sizeof(int) * WL_INTS);
  L.snc = take(sizeof(SNConst) * 5 * S);
  // trust-region state
  L.nt_f = take(sizeof(double) * S);
  L.nt_g = take(sizeof(double) * NP * S);
  L.nt_H = take(sizeof(double) * NP * NP * S);
  L.nt_trial = take(sizeof(double) * NP * S);
  L.nt_pred = take(sizeof(double) * S);
  L.nt_ftrial = take(sizeof(double) * S);
  L.nt_state = take(sizeof(int) * 8 * S);
  L.nt_tcache = take(sizeof(double) * TR_CACHE * S);
  L.nt_count = take(sizeof(int) * 4);
  L.nt_lam = take(sizeof(double) * S);
  L.nt_list = take(sizeof(int) * S);
  L.total = o;
}

}  // namespace celeste

extern "C" size_t celeste_problem_workspace_bytes(const celeste_problem* p) { return p ? p->ws.total : 0; }

extern "C" int celeste_problem_counts(const celeste_problem* p, int64_t counts[5]) {
  if (!p || !counts) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  counts[0] = p->S;
  counts[1] = (int64_t)p->patches.size();
  counts[2] = (int64_t)p->tiles.size();
  counts[3] = p->n_pix;
  counts[4] = (int64_t)p->nbr.size();
  return CELESTE_OK;
}

template <class T>
static cudaError_t upload(char* base, size_t off, const std::vector<T>& v, cudaStream_t st) {
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(base + off, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}

extern "C" int celeste_problem_bind(celeste_problem* p, void* workspace, size_t bytes, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!workspace || bytes < p->ws.total) return fail(CELESTE_ERR_WORKSPACE, "workspace needs %zu bytes", p->ws.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(CELESTE_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* base = static_cast<char*>(workspace);
  const WsLayout& L = p->ws;
  cudaError_t e;
  if ((e = upload(base, L.images, p->imgdev, st)) != cudaSuccess) return cuda_fail(e, "upload images");
  if ((e = upload(base, L.patches, p->patches, st)) != cudaSuccess) return cuda_fail(e, "upload patches");
  if ((e = upload(base, L.tiles, p->tiles, st)) != cudaSuccess) return cuda_fail(e, "upload tiles");
  if ((e = upload(base, L.tile_pix, p->tile_pix, st)) != cudaSuccess) return cuda_fail(e, "upload tile offsets");
  if ((e = upload(base, L.src_patch, p->src_patch, st)) != cudaSuccess) return cuda_fail(e, "upload src_patch");
  if ((e = upload(base, L.nbr, p->nbr, st)) != cudaSuccess) return cuda_fail(e, "upload nbr");
  if ((e = upload(base, L.u0, p->u0, st)) != cudaSuccess) return cuda_fail(e, "upload u0");
  if ((e = upload(base, L.psf_coef, p->psf_coef, st)) != cudaSuccess) return cuda_fail(e, "upload psf");
  if ((e = cudaMemsetAsync(base + L.pix, 0, sizeof(float4) * std::max<long long>(p->n_pix, 1), st)) != cudaSuccess)
    return cuda_fail(e, "clear pixels");
  if ((e = cudaMemsetAsync(base + L.flags, 0, sizeof(int) * p->S, st)) != cudaSuccess) return cuda_fail(e, "clear flags");
  if ((e = cudaMemsetAsync(base + L.err, 0, sizeof(int) * 4, st)) != cudaSuccess) return cuda_fail(e, "clear err");
  if ((e = cudaMemsetAsync(base + L.counters, 0, sizeof(unsigned long long) * 4, st)) != cudaSuccess)
    return cuda_fail(e, "clear counters");
  if ((e = cudaMemsetAsync(base + L.wl_count, 0, sizeof(int) * WL_INTS, st)) != cudaSuccess)
    return cuda_fail(e, "clear worklists");
  int dev_id = 0, n_sm = 0;
  if ((e = cudaGetDevice(&dev_id)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev_id)) != cudaSuccess)
    return cuda_fail(e, "SM count");

  ProblemDev& D = p->dev;
  D.images = reinterpret_cast<const ImageDev*>(base + L.images);
  D.patches = reinterpret_cast<const PatchDev*>(base + L.patches);
  D.tiles = reinterpret_cast<const TileDev*>(base + L.tiles);
  D.tile_pix = reinterpret_cast<const long long*>(base + L.tile_pix);
  D.src_patch = reinterpret_cast<const int*>(base + L.src_patch);
  D.nbr = reinterpret_cast<const int*>(base + L.nbr);
  D.u0 = reinterpret_cast<const double*>(base + L.u0);
  D.psf_coef = reinterpret_cast<const double*>(base + L.psf_coef);
  D.psf = reinterpret_cast<float*>(base + L.psf);
  D.pix = reinterpret_cast<float4*>(base + L.pix);
  D.srcmom = reinterpret_cast<float2*>(base + L.srcmom);
  D.ptab = reinterpret_cast<float*>(base + L.ptab);
  D.partials = reinterpret_cast<float*>(base + L.partials);
  D.vpartials = reinterpret_cast<float*>(base + L.vpartials);
  D.flags = reinterpret_cast<int*>(base + L.flags);
  D.err = reinterpret_cast<int*>(base + L.err);
  D.counters = reinterpret_cast<unsigned long long*>(base + L.counters);
  D.wl = reinterpret_cast<int*>(base + L.wl);
  D.wl_count = reinterpret_cast<int*>(base + L.wl_count);
  D.snc = reinterpret_cast<SNConst*>(base + L.snc);
  D.pweight = nullptr;   // set only on the joint solver's copies
  D.refEV = nullptr;
  D.n_sm = std::max(n_sm, 1);
  D.wait_budget = p->wait_budget ? p->wait_budget : WAIT_BUDGET_DEFAULT;
  D.S = p->S;
  D.n_patches = (int)p->patches.size();
  D.n_tiles = (int)p->tiles.size();
  D.tile_pixels = p->tile_pixels;
  D.hmode = p->hessian_mode;
  std::memcpy(D.priors, p->priors, sizeof(D.priors));
  D.log_var_r = std::log(p->priors[2]);
  D.log_var_c = std::log(p->priors[4]);
  D.log_phi = std::log(p->priors[0]);
  D.log1m_phi = std::log1p(-p->priors[0]);
  D.logit_phi = D.log_phi - D.log1m_phi;
  D.inv_var_r = 1.0 / p->priors[2];
  D.inv_var_c = 1.0 / p->priors[4];
  std::memcpy(D.nu, p->nu, sizeof(D.nu));
  std::memcpy(D.tau, p->tau, sizeof(D.tau));
  p->base = base;
  if (D.n_patches > 0) {
    psf_setup_kernel<<<(D.n_patches + 127) / 128, 128, 0, st>>>(D);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "psf_setup_kernel");
  }
  if (D.n_tiles > 0) {
    gather_pixels_kernel<<<D.n_tiles, 256, 0, st>>>(D);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gather_pixels_kernel");
  }
  p->bound = true;
  p->background_ready = false;
  return CELESTE_OK;
}

extern "C" int celeste_problem_refresh_pixels(celeste_problem* p, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  cudaStream_t st = (cudaStream_t)stream;
  const ProblemDev& D = p->dev;
  cudaError_t e = cudaMemsetAsync(D.err, 0, sizeof(int) * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear err");
  if (D.n_tiles > 0) {
    gather_pixels_kernel<<<D.n_tiles, 256, 0, st>>>(D);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gather_pixels_kernel");
  }
  p->background_ready = false;
  return CELESTE_OK;
}

celeste_problem::~celeste_problem() {
  for (cudaEvent_t ev : prof_events) cudaEventDestroy(ev);
  for (cudaEvent_t ev : iter_events) cudaEventDestroy(ev);
  if (newton_exec) cudaGraphExecDestroy(newton_exec);
  if (capture_stream) cudaStreamDestroy(capture_stream);
}

extern "C" void celeste_problem_destroy(celeste_problem* p) { delete p; }

namespace celeste {
int prof_mark(celeste_problem* p, cudaStream_t st) {
  if (!p->prof_on) return -1;
  if (p->prof_used == p->prof_events.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return -1;
    p->prof_events.push_back(ev);
  }
  cudaEvent_t ev = p->prof_events[p->prof_used];
  if (cudaEventRecord(ev, st) != cudaSuccess) return -1;
  return (int)p->prof_used++;
}
}  // namespace celeste

extern "C" int celeste_profile_start(celeste_problem* p) {
  if (!p || !p->bound) return fail(CELESTE_ERR_STATE, "profiling needs a bound problem");
  cudaError_t e = cudaMemset(p->dev.counters, 0, sizeof(unsigned long long) * 4);
  if (e != cudaSuccess) return cuda_fail(e, "reset counters");
  p->prof_on = true;
  p->prof_used = 0;
  p->prof_full.clear();
  p->prof_value.clear();
  p->prof_launches = 0;
  p->prof_iters = 0;
  p->prof_full_acc = p->prof_value_acc = p->prof_tr_acc = 0.0;
  p->prof_full_n = p->prof_value_n = p->prof_tr_n = 0;
  return CELESTE_OK;
}

extern "C" int celeste_profile_stop(celeste_problem* p, celeste_profile_stats* out) {
  if (!p || !out) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  p->prof_on = false;
  std::memset(out, 0, sizeof(*out));
  cudaError_t e;
  auto span = [&](const std::vector<std::pair<int, int>>& v, double& ms) -> cudaError_t {
    for (auto& pr : v) {
      if (pr.first < 0 || pr.second < 0) continue;
      cudaError_t e2 = cudaEventSynchronize(p->prof_events[pr.second]);
      if (e2 != cudaSuccess) return e2;
      float t = 0.f;
      e2 = cudaEventElapsedTime(&t, p->prof_events[pr.first], p->prof_events[pr.second]);
      if (e2 != cudaSuccess) return e2;
      ms += t;
    }
    return cudaSuccess;
  };
  if ((e = span(p->prof_full, out->full_ms)) != cudaSuccess) return cuda_fail(e, "full-kernel events");
  if ((e = span(p->prof_value, out->value_ms)) != cudaSuccess) return cuda_fail(e, "value-kernel events");
  out->full_ms += p->prof_full_acc;
  out->value_ms += p->prof_value_acc;
  out->full_launches = (int64_t)p->prof_full.size() + p->prof_full_n;
  out->value_launches = (int64_t)p->prof_value.size() + p->prof_value_n;
  unsigned long long c[4];
  if ((e = cudaMemcpy(c, p->dev.counters, sizeof(c), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read counters");
  out->full_pixels = (int64_t)c[0];
  out->value_pixels = (int64_t)c[1];
  out->kernel_launches = p->prof_launches;
  out->newton_iterations = p->prof_iters;
  out->tr_ms = p->prof_tr_acc;
  out->tr_launches = p->prof_tr_n;
  return CELESTE_OK;
}

extern "C" const char* celeste_strerror(int code) {
  switch (code) {
    case CELESTE_OK: return "ok";
    case CELESTE_ERR_INVALID_ARG: return "invalid argument";
    case CELESTE_ERR_CUDA: return "CUDA error";
    case CELESTE_ERR_TIMEOUT: return "device wait timed out";
    case CELESTE_ERR_WORKSPACE: return "bad workspace";
    case CELESTE_ERR_STATE: return "call order violated";
    default: return "unknown error";
  }
}

extern "C" const char* celeste_last_error_detail(void) { return g_last_error.c_str(); }
