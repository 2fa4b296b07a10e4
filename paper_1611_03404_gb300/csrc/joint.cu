// Cross-source Hessian blocks of the joint objective (paper, concluding section: a stationary
// point of the objective over all light sources at once, beyond the per-source optimisation with
// the neighbours held fixed).
//
//   J(theta) = sum over the pixels of the union of the windows (each counted once) of
//              l(x, E, V) - sum_s KL_s,   each source's light counted on its own window.
//
// E and V are sums over sources, so two sources s, t couple only through the pixels their windows
// share, and only through first derivatives:
//   d2J / ds dt = sum_{m in W_s cap W_t} l_EE e_s e_t^T + l_EV (e_s v_t^T + v_s e_t^T),
//   e = dE/dtheta = iota dE[G],  v = dV/dtheta = iota^2 (dE[G^2] - 2 E[G] dE[G]).
// Per pixel both sources' rows are formed in the 11-column reduced basis of the pixel kernel
// (position mu, dev, axis, angle, scale, alpha; the E-rows f_0, f_1 and V-rows f_0^2, f_1^2 that
// the band-dependent brightness derivatives multiply), from each source's own patch table; the
// 11 x 11 cross product is summed per tile of the overlap in float32 (warp reduce-scatter), and
// each pair's tiles are summed and lifted to the 27 parameters in float64.
#include <algorithm>
#include <cstring>
#include <vector>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"

namespace celeste {

struct JointItem {   // an overlap rectangle (image pixels) of patch p (source s) and patch q (source t)
  int p, q, x0, y0, w, h, tile_begin, tile_end;
};
struct JointTile {
  int item, start, count, pad;
};
constexpr int JT_PIX = 128;             // overlap pixels per tile (one per thread)
constexpr int NCROSS = NRED * NRED;     // 121 reduced cross sums

struct JointDev {
  const JointItem* items;
  const JointTile* tiles;
  const int* pair_items;                // CSR [n_pairs + 1] over the items (sorted by pair)
  const int* pairs;                     // [n_pairs][2]
  float* partials;                      // [n_tiles][NCROSS]
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Offsets of the joint buffers inside p->joint_dev.
struct JointLayout {
  size_t items, tiles, pair_items, pairs, partials, total;
};
static JointLayout joint_layout(int n_items, int n_tiles, int n_pairs) {
  JointLayout L{};
  size_t o = 0;
  L.items = o;
  o = align256(o + sizeof(JointItem) * std::max(n_items, 1));
  L.tiles = o;
  o = align256(o + sizeof(JointTile) * std::max(n_tiles, 1));
  L.pair_items = o;
  o = align256(o + sizeof(int) * (n_pairs + 1));
  L.pairs = o;
  o = align256(o + sizeof(int) * 2 * std::max(n_pairs, 1));
  L.partials = o;
  o = align256(o + sizeof(float) * NCROSS * std::max(n_tiles, 1));
  L.total = o;
  return L;
}

static JointDev joint_view(const celeste_problem* p) {
  const int n_pairs = (int)p->joint_pairs.size() / 2;
  const JointLayout L = joint_layout(p->joint_n_items, p->joint_n_tiles, n_pairs);
  char* b = static_cast<char*>(p->joint_dev);
  return {reinterpret_cast<const JointItem*>(b + L.items), reinterpret_cast<const JointTile*>(b + L.tiles),
          reinterpret_cast<const int*>(b + L.pair_items), reinterpret_cast<const int*>(b + L.pairs),
          reinterpret_cast<float*>(b + L.partials)};
}

// Overlap items of every pair of patches that share an image and whose windows intersect, grouped
// by source pair; tiles of at most JT_PIX pixels over each rectangle (row-major).
static int joint_build(celeste_problem* p) {
  if (p->joint_built) return CELESTE_OK;
  struct Raw {
    int s, t;
    JointItem it;
  };
  std::vector<Raw> raw;
  for (int pi = 0; pi < (int)p->patches.size(); ++pi) {
    const PatchDev& A = p->patches[pi];
    for (int k = A.nbr_begin; k < A.nbr_end; ++k) {
      const int qi = p->nbr[k];
      const PatchDev& B = p->patches[qi];
      if (B.source <= A.source) continue;   // each unordered pair once per image
      const int x0 = std::max(A.x0, B.x0), x1 = std::min(A.x0 + A.w, B.x0 + B.w);
      const int y0 = std::max(A.y0, B.y0), y1 = std::min(A.y0 + A.h, B.y0 + B.h);
      if (x1 <= x0 || y1 <= y0) continue;
      raw.push_back({A.source, B.source, {pi, qi, x0, y0, x1 - x0, y1 - y0, 0, 0}});
    }
  }
  std::stable_sort(raw.begin(), raw.end(),
                   [](const Raw& a, const Raw& b) { return a.s != b.s ? a.s < b.s : a.t < b.t; });
  std::vector<JointItem> items;
  std::vector<JointTile> tiles;
  std::vector<int> pair_items, pairs;
  for (size_t i = 0; i < raw.size(); ++i) {
    if (i == 0 || raw[i].s != raw[i - 1].s || raw[i].t != raw[i - 1].t) {
      pair_items.push_back((int)items.size());
      pairs.push_back(raw[i].s);
      pairs.push_back(raw[i].t);
    }
    JointItem it = raw[i].it;
    it.tile_begin = (int)tiles.size();
    const int n = it.w * it.h;
    for (int st = 0; st < n; st += JT_PIX) tiles.push_back({(int)items.size(), st, std::min(JT_PIX, n - st), 0});
    it.tile_end = (int)tiles.size();
    items.push_back(it);
  }
  pair_items.push_back((int)items.size());
  const int n_pairs = (int)pairs.size() / 2;
  const JointLayout L = joint_layout((int)items.size(), (int)tiles.size(), n_pairs);
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, L.total);
  if (e != cudaSuccess) return cuda_fail(e, "joint buffers");
  char* b = static_cast<char*>(dev);
  if (!items.empty()) e = cudaMemcpy(b + L.items, items.data(), sizeof(JointItem) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(b + L.tiles, tiles.data(), sizeof(JointTile) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b + L.pair_items, pair_items.data(), sizeof(int) * pair_items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pairs.empty())
    e = cudaMemcpy(b + L.pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "joint upload");
  }
  p->joint_dev = dev;
  p->joint_pairs = pairs;
  p->joint_n_items = (int)items.size();
  p->joint_n_tiles = (int)tiles.size();
  p->joint_built = true;
  return CELESTE_OK;
}

// Value and first derivatives of one source's E[G] and E[G^2] at pixel (fx, fy) of its patch, as
// rows in the reduced basis (the same columns as the pixel kernel's Jacobian rows).
struct JacRows {
  float EG, VG, yE[NRED], yV[NRED];
};

__device__ inline void jac_rows(const float* tab, float fx, float fy, JacRows& r) {
  const SNConst& c = *reinterpret_cast<const SNConst*>(&tab[TB_SNC]);
  float f0 = 0.f, f0m[2] = {0.f, 0.f};
  float F[2] = {0.f, 0.f}, Fv[2][5];
#pragma unroll
  for (int fam = 0; fam < 2; ++fam)
#pragma unroll
    for (int a = 0; a < 5; ++a) Fv[fam][a] = 0.f;
#pragma unroll 1
  for (int k = 0; k < CELESTE_NPSF; ++k) {
    const float d0 = fx - tab[TB_MU + 2 * k], d1 = fy - tab[TB_MU + 2 * k + 1];
    const float s0 = d0 * d0, s1 = 2.f * d0 * d1, s2 = d1 * d1;
    {
      const float* st = &tab[TB_STAR + 4 * k];
      const float N = st[0] * exp2f((st[1] * s0 + st[2] * s1 + st[3] * s2) * (-0.5f * LOG2E));
      f0 += N;
      f0m[0] += N * (st[1] * d0 + st[2] * d1);
      f0m[1] += N * (st[2] * d0 + st[3] * d1);
    }
#pragma unroll 1
    for (int j = 0; j < NMIX; ++j) {
      const float* e = &tab[TB_GAL + (k * NMIX + j) * GT_STRIDE];
      const float N = e[GT_W] * exp2f((e[GT_P] * s0 + e[GT_P + 1] * s1 + e[GT_P + 2] * s2) * (-0.5f * LOG2E));
      const int fam = j < CELESTE_NEXP ? 0 : 1;
      float b[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float* Q = e + GT_QA + 3 * a;
        b[a] = e[GT_LA + a] + Q[0] * s0 + Q[1] * s1 + Q[2] * s2;
      }
      const float z0 = e[GT_P] * d0 + e[GT_P + 1] * d1, z1 = e[GT_P + 1] * d0 + e[GT_P + 2] * d1;
      const float v[6] = {N, N * z0, N * z1, N * b[0], N * b[1], N * b[2]};
      // (statically indexed accumulators: one branch per family)
      if (fam == 0) {
        F[0] += v[0];
#pragma unroll
        for (int a = 0; a < 5; ++a) Fv[0][a] += v[1 + a];
      } else {
        F[1] += v[0];
#pragma unroll
        for (int a = 0; a < 5; ++a) Fv[1][a] += v[1 + a];
      }
    }
  }
  // galaxy over G6 = (mu0, mu1, dev, axis, angle, scale)
  const float dF = F[1] - F[0];
  const float f1 = F[0] + c.e * dF;
  float f1g[6];
  f1g[0] = Fv[0][0] + c.e * (Fv[1][0] - Fv[0][0]);
  f1g[1] = Fv[0][1] + c.e * (Fv[1][1] - Fv[0][1]);
  f1g[2] = c.e1 * dF;
#pragma unroll
  for (int a = 2; a < 5; ++a) f1g[a + 1] = Fv[0][a] + c.e * (Fv[1][a] - Fv[0][a]);
  r.EG = c.A0 * f0 + c.A1 * f1;
  const float dx = c.L10 * f0 - c.L11 * f1;
  r.VG = c.C0 * f0 * f0 + c.C1 * f1 * f1 + c.Cx * dx * dx;
  r.yE[0] = c.A0 * f0m[0] + c.A1 * f1g[0];
  r.yE[1] = c.A0 * f0m[1] + c.A1 * f1g[1];
  r.yV[0] = 2.f * (c.B0 * f0 * f0m[0] + c.B1 * f1 * f1g[0]);
  r.yV[1] = 2.f * (c.B0 * f0 * f0m[1] + c.B1 * f1 * f1g[1]);
#pragma unroll
  for (int a = 2; a < 6; ++a) {
    r.yE[a] = c.A1 * f1g[a];
    r.yV[a] = 2.f * c.B1 * f1 * f1g[a];
  }
  r.yE[6] = c.aE1 * f1 - c.aE0 * f0;
  r.yV[6] = c.aV1 * f1 * f1 - c.aV0 * f0 * f0;
  r.yE[7] = f0;
  r.yE[8] = f1;
  r.yE[9] = 0.f;
  r.yE[10] = 0.f;
  r.yV[7] = 0.f;
  r.yV[8] = 0.f;
  r.yV[9] = f0 * f0;
  r.yV[10] = f1 * f1;
}

// Warp reduce-scatter: on return lane l holds the warp sum of v[l] (v is clobbered).
__device__ __forceinline__ float joint_reduce_scatter32(float (&v)[32], int lane) {
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

// One overlap tile: per pixel the rows of both sources and the pixel's l_EE, l_EV; the 121
// reduced cross sums M[a][b] = sum_m ts[a] e_t[b] + us[a] v_t[b] with ts = l_EE e_s + l_EV v_s and
// us = l_EV e_s.
__global__ void __launch_bounds__(JT_PIX, 1) cross_kernel(ProblemDev P, JointDev JD) {
  __shared__ __align__(16) float tabs[2][TB_FLOATS];
  __shared__ float red[JT_PIX / 32][128];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const JointTile jt = JD.tiles[blockIdx.x];
  const JointItem it = JD.items[jt.item];
  const PatchDev ps = P.patches[it.p], pq = P.patches[it.q];
  for (int i = tid; i < TB_FLOATS; i += JT_PIX) {
    tabs[0][i] = P.ptab[(size_t)it.p * TB_FLOATS + i];
    tabs[1][i] = P.ptab[(size_t)it.q * TB_FLOATS + i];
  }
  __syncthreads();
  const bool valid = tid < jt.count;
  const int i = jt.start + (valid ? tid : 0);
  const int X = it.x0 + i % it.w, Y = it.y0 + i / it.w;
  const int cs = X - ps.x0, rs = Y - ps.y0;
  const float4 pv = P.pix[ps.pix_off + (long long)rs * ps.w + cs];
  JacRows a, b;
  jac_rows(tabs[0], (float)cs, (float)rs, a);
  jac_rows(tabs[1], (float)(X - pq.x0), (float)(Y - pq.y0), b);
  const float iota = reinterpret_cast<const SNConst*>(&tabs[0][TB_SNC])->iota, iota2 = iota * iota;
  const float E = pv.y + iota * a.EG, V = pv.z + iota2 * a.VG, x = pv.x;
  const float rE = 1.f / E, rE2 = rE * rE;
  const float lEE = valid ? -x * rE2 - 3.f * x * V * rE2 * rE2 : 0.f;
  const float lEV = valid ? x * rE2 * rE : 0.f;
  float ts[NRED], us[NRED], et[NRED], vt[NRED];
#pragma unroll
  for (int k = 0; k < NRED; ++k) {
    const float es = iota * a.yE[k], vs = iota2 * (a.yV[k] - 2.f * a.EG * a.yE[k]);
    ts[k] = lEE * es + lEV * vs;
    us[k] = lEV * es;
    et[k] = iota * b.yE[k];
    vt[k] = iota2 * (b.yV[k] - 2.f * b.EG * b.yE[k]);
  }
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int q = ch * 32 + j;
      v[j] = q < NCROSS ? ts[q / NRED] * et[q % NRED] + us[q / NRED] * vt[q % NRED] : 0.f;
    }
    red[warp][ch * 32 + lane] = joint_reduce_scatter32(v, lane);
  }
  __syncthreads();
  if (tid < NCROSS)
    JD.partials[(size_t)blockIdx.x * NCROSS + tid] = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
}

// Lift coefficients of one source for band `band`, lane j < 27: column j of K (11 -> 27) has the
// nonzeros (nzA, nzK) and (nzB, nzL): j < 7 -> (j, 1); brightness parameter v of type t ->
// (7 + t, a_t dE[l_b|t]/dv) from the E-row and (9 + t, a_t dE[l_b^2|t]/dv) from the V-row.
__device__ inline void lift_column(const double* __restrict__ th, int band, int j, int& nzA, double& nzK, int& nzB,
                                   double& nzL) {
  if (j < 7) {
    nzA = j;
    nzK = 1.0;
    nzB = -1;
    nzL = 0.0;
    return;
  }
  int t, v;
  bvar_inv(j, t, v);
  double m = th[bvar(t, 0)], var = exp(th[bvar(t, 1)]);
  for (int q = 0; q < 4; ++q) {
    const double cq = color_coef(band, q);
    m += cq * th[bvar(t, 2 + q)];
    var += cq * cq * exp(th[bvar(t, 6 + q)]);
  }
  const bool isvar = v == 1 || v >= 6;
  double cf = v < 2 ? 1.0 : color_coef(band, (v - 2) & 3);
  if (v >= 6) cf *= cf;
  const double e = isvar ? exp(th[bvar(t, v)]) : 1.0;
  const double dl1 = (isvar ? 0.5 : 1.0) * cf * e, dl2 = 2.0 * cf * e;   // d log E[l], d log E[l^2]
  const double at = t ? sigmoid_d(th[6]) : sigmoid_d(-th[6]);
  nzA = 7 + t;
  nzK = at * exp(m + 0.5 * var) * dl1;
  nzB = 9 + t;
  nzL = at * exp(2.0 * m + 2.0 * var) * dl2;
}

// One CTA per pair: for each of its images, sum the overlap tiles' cross sums (float64), lift
// both sides to the 27 parameters with the image's band and map pixel position to world position
// through the image's WCS; the images' blocks are added in a fixed order.
__global__ void __launch_bounds__(128, 1) cross_assemble_kernel(ProblemDev P, JointDev JD, const double* __restrict__ theta,
                                                             double* __restrict__ blocks) {
  __shared__ double M[NCROSS];
  __shared__ double HE[NP * NP], H[NP * NP];
  __shared__ double kK[2][NP], kL[2][NP], A[4];
  __shared__ int kA[2][NP], kB[2][NP];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int pr = blockIdx.x;
  const int s0 = JD.pairs[2 * pr], s1 = JD.pairs[2 * pr + 1];
  for (int i = tid; i < NP * NP; i += nt) H[i] = 0.0;
  for (int k = JD.pair_items[pr]; k < JD.pair_items[pr + 1]; ++k) {
    const JointItem it = JD.items[k];
    const ImageDev& im = P.images[P.patches[it.p].image];
    if (tid < NCROSS) {
      double v = 0.0;
      for (int t = it.tile_begin; t < it.tile_end; ++t) v += (double)JD.partials[(size_t)t * NCROSS + tid];
      M[tid] = v;
    } else if (tid < NCROSS + 4) {
      A[tid - NCROSS] = im.A[tid - NCROSS];
    }
    if (tid < 64) {
      const int side = tid >> 5, j = tid & 31;
      if (j < NP) {
        int a, b;
        double kk, kl;
        lift_column(theta + (size_t)(side ? s1 : s0) * NP, im.band, j, a, kk, b, kl);
        kA[side][j] = a;
        kK[side][j] = kk;
        kB[side][j] = b;
        kL[side][j] = kl;
      }
    }
    __syncthreads();
    // H_E = K_s^T M K_t (at most four terms per entry)
    for (int i = tid; i < NP * NP; i += nt) {
      const int r = i / NP, c = i % NP;
      const int ar = kA[0][r], br = kB[0][r], ac = kA[1][c], bc = kB[1][c];
      double v = kK[1][c] * M[ar * NRED + ac] + (bc >= 0 ? kL[1][c] * M[ar * NRED + bc] : 0.0);
      v *= kK[0][r];
      if (br >= 0) v += kL[0][r] * (kK[1][c] * M[br * NRED + ac] + (bc >= 0 ? kL[1][c] * M[br * NRED + bc] : 0.0));
      HE[i] = v;
    }
    __syncthreads();
    // d/du_b = sum_a A[a][b] d/dmu_a on both sides (same image)
    for (int i = tid; i < NP * NP; i += nt) {
      const int r = i / NP, c = i % NP;
      double v;
      if (r < 2 && c < 2) {
        v = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) v += A[a * 2 + r] * A[b * 2 + c] * HE[a * NP + b];
      } else if (r < 2) {
        v = A[0 * 2 + r] * HE[0 * NP + c] + A[1 * 2 + r] * HE[1 * NP + c];
      } else if (c < 2) {
        v = A[0 * 2 + c] * HE[r * NP + 0] + A[1 * 2 + c] * HE[r * NP + 1];
      } else {
        v = HE[i];
      }
      H[i] += v;
    }
    __syncthreads();
  }
  for (int i = tid; i < NP * NP; i += nt) blocks[(size_t)pr * NP * NP + i] = H[i];
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_joint_pairs(celeste_problem* p, int32_t* pairs, int64_t capacity, int64_t* n_pairs) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  if (!n_pairs) return fail(CELESTE_ERR_INVALID_ARG, "null n_pairs");
  const int rc = joint_build(p);
  if (rc != CELESTE_OK) return rc;
  const int64_t n = (int64_t)p->joint_pairs.size() / 2;
  *n_pairs = n;
  if (!pairs) return CELESTE_OK;
  if (capacity < n) return fail(CELESTE_ERR_INVALID_ARG, "pairs holds %lld pairs, %lld needed", (long long)capacity,
                                (long long)n);
  if (n) std::memcpy(pairs, p->joint_pairs.data(), sizeof(int32_t) * 2 * n);
  return CELESTE_OK;
}

extern "C" int celeste_joint_cross_hessian(celeste_problem* p, const double* theta, double* blocks,
                                           celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound || !p->background_ready)
    return fail(CELESTE_ERR_STATE, "bind the problem and render the background first");
  if (p->background_mode != CELESTE_NBR_WINDOW)
    return fail(CELESTE_ERR_STATE, "the background must be rendered with CELESTE_NBR_WINDOW");
  if (!theta || !blocks) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  int rc = joint_build(p);
  if (rc != CELESTE_OK) return rc;
  const int n_pairs = (int)p->joint_pairs.size() / 2;
  if (n_pairs == 0) return CELESTE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const ProblemDev& D = p->dev;
  cudaError_t e;
  if ((e = launch_set_flags(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "set flags");
  if ((e = launch_worklists(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  if ((e = launch_tables(D, theta, true, st)) != cudaSuccess) return cuda_fail(e, "tables");
  const JointDev JD = joint_view(p);
  if (p->joint_n_tiles > 0) {
    cross_kernel<<<p->joint_n_tiles, JT_PIX, 0, st>>>(D, JD);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "cross_kernel");
  }
  cross_assemble_kernel<<<n_pairs, 128, 0, st>>>(D, JD, theta, blocks);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "cross_assemble_kernel");
  prof_count(p, 6);
  return CELESTE_OK;
}
