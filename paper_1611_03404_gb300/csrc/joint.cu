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
#include <cmath>
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
// by source pair; tiles of at most JT_PIX pixels over each rectangle (row-major).  Host only: the
// lists are kept on the problem (flat int records) until the first device use uploads them.
static void joint_host(celeste_problem* p) {
  if (p->joint_host_built) return;
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
  static_assert(sizeof(JointItem) == 8 * sizeof(int) && sizeof(JointTile) == 4 * sizeof(int), "flat records");
  p->joint_items_h.resize(8 * items.size());
  p->joint_tiles_h.resize(4 * tiles.size());
  if (!items.empty()) std::memcpy(p->joint_items_h.data(), items.data(), sizeof(JointItem) * items.size());
  if (!tiles.empty()) std::memcpy(p->joint_tiles_h.data(), tiles.data(), sizeof(JointTile) * tiles.size());
  p->joint_pair_items_h = pair_items;
  p->joint_pairs = pairs;
  p->joint_n_items = (int)items.size();
  p->joint_n_tiles = (int)tiles.size();
  p->joint_host_built = true;
}

// The joint structures live in a caller-bound workspace (celeste_joint_bind): the overlap lists,
// then the joint Newton state.
static int joint_build(celeste_problem* p) {
  joint_host(p);
  if (!p->joint_built) return fail(CELESTE_ERR_STATE, "bind the joint workspace first (celeste_joint_bind)");
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
      for (int a = 0; a < 3; ++a)
        b[a] = e[gt_la(a)] + e[gt_qa(a, 0)] * s0 + e[gt_qa(a, 1)] * s1 + e[gt_qa(a, 2)] * s2;
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

// ------------------------------------------------------------------------------ joint Newton
// Trust-region Newton on f = -J over all sources at once (Nocedal & Wright Alg. 4.1 for the outer
// iteration; the same acceptance, radius and stopping rules as the per-source solve).  The
// subproblem min g.p + p.B.p/2, |p|_M <= delta, B = -d2J, is solved by preconditioned conjugate
// gradients with Steihaug's stopping rules (Nocedal & Wright Alg. 7.2): stop on negative
// curvature or on reaching the boundary (then step to it), or once |r| <= 1e-2 |g| (an interior
// step is then an accurate Newton step, and only such a step's predicted decrease is taken as the
// Newton decrement of the stopping rule).
// The preconditioner is block-diagonal, M = blockdiag(-H_ss + mu_s I) with mu_s the first shift of
// a short ladder that makes the block positive definite, and the radius is measured in its norm.
// B is block-sparse: a block per source and one per overlapping pair.  J's change at a trial point
// is summed per pixel against the stored rates at the current point, each pixel weighted by
// 1 / (windows holding it), so every pixel counts once.

struct JNScalars {
  double rz, alpha, beta, tau, delta, xMx, xMd, dMd, eps, gnorm, gmax, pred, dJ;
  int cur, stop, mode, boundary, cg_iters, rstop, pad1, pad2;
};

struct JNDev {
  int S;
  const double* gJ;     // [S][27] dJ/dtheta (f = -J: gradient -gJ)
  const double* Hd;     // [S][27][27] d2J/dtheta_s^2 (B_ss = -Hd)
  const double* Hc;     // [n_pairs][27][27] d2J/dtheta_s dtheta_t (B_st = -Hc)
  const int* row_ptr;   // [S + 1] each source's coupling entries
  const int* row_ent;   // pair index * 2 + side (side 1: the source is the pair's second)
  const int* pairs;     // [n_pairs][2]
  double* Mf;           // [S][27][27] L D L^T of M_s: L below the diagonal, 1/D on it
  double *x, *r, *z, *d0, *d1, *Bd;   // [S][27]
  double* part;         // [3][S] per-source partial sums
  JNScalars* sc;
};

constexpr int JN_WARPS = 4;
constexpr int JN_CHUNK = 4;   // CG iterations enqueued between two reads of the stop flag

__device__ inline double jn_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double jn_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// z = M_s^-1 r (lane i holds r_i and receives z_i; lanes >= 27 hold 0).
__device__ inline double jn_minv(const double* __restrict__ Mf, double ri, int lane) {
  const bool row = lane < NP;
  double y = row ? ri : 0.0;
  for (int k = 0; k < NP - 1; ++k) {
    const double yk = __shfl_sync(0xffffffffu, y, k);
    if (row && lane > k) y = fma(-Mf[lane * NP + k], yk, y);
  }
  if (row) y *= Mf[lane * NP + lane];
  for (int k = NP - 1; k > 0; --k) {
    const double yk = __shfl_sync(0xffffffffu, y, k);
    if (lane < k) y = fma(-Mf[k * NP + lane], yk, y);
  }
  return row ? y : 0.0;
}

// Row `lane` of B_ss v_s + sum over the coupled sources B_st v_t, with v read through `vec`
// (lanes < 27; the caller passes each source's vector entry held by the lane).
template <class Vec>
__device__ inline double jn_rowmul(const JNDev& J, int s, int lane, Vec vec) {
  const bool row = lane < NP;
  const double* H = J.Hd + (size_t)s * NP * NP;
  const double vs = vec(s);
  double y = 0.0;
  for (int j = 0; j < NP; ++j) {
    const double vj = __shfl_sync(0xffffffffu, vs, j);
    if (row) y = fma(-H[lane * NP + j], vj, y);
  }
  for (int e = J.row_ptr[s]; e < J.row_ptr[s + 1]; ++e) {
    const int ent = J.row_ent[e], k = ent >> 1, side = ent & 1;
    const int t = J.pairs[2 * k + (side ? 0 : 1)];
    const double* blk = J.Hc + (size_t)k * NP * NP;
    const double vt = vec(t);
    for (int j = 0; j < NP; ++j) {
      const double vj = __shfl_sync(0xffffffffu, vt, j);
      if (row) y = fma(-(side ? blk[j * NP + lane] : blk[lane * NP + j]), vj, y);
    }
  }
  return row ? y : 0.0;
}

// Preconditioner blocks: L D L^T of -H_ss + mu I for the first mu in {1e-4, 1e-3, .., 10} x max_i |H_ii|
// that gives positive pivots, else the positive diagonal |H_ii| + max_i |H_ii|.  The floor 1e-4
// keeps the norm of M from stretching along the block's flat directions (a step there is measured
// at least at 1e-4 of the block's largest curvature), where the quadratic model is poor.
__global__ void __launch_bounds__(32 * JN_WARPS) jn_precond_kernel(JNDev J) {
  __shared__ double As[JN_WARPS][NP * NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * JN_WARPS + warp;
  if (s >= J.S) return;
  double* A = As[warp];
  const double* H = J.Hd + (size_t)s * NP * NP;
  double* out = J.Mf + (size_t)s * NP * NP;
  const double scale = fmax(jn_warp_max(lane < NP ? fabs(H[lane * NP + lane]) : 0.0), 1e-300);
  const double ladder[6] = {1e-4, 1e-3, 1e-2, 1e-1, 1.0, 10.0};
  bool pd = false;
  for (int a = 0; a < 6 && !pd; ++a) {
    const double mu = ladder[a] * scale;
    for (int i = lane; i < NP * NP; i += 32) A[i] = -H[i] + ((i / NP) == (i % NP) ? mu : 0.0);
    __syncwarp();
    pd = true;
    for (int k = 0; k < NP && pd; ++k) {
      const double dk = A[k * NP + k];
      pd = dk > 0.0 && isfinite(dk);   // same value in every lane
      if (!pd) break;
      const double rk = 1.0 / dk;
      const bool act = lane > k && lane < NP;
      const double li = act ? A[lane * NP + k] * rk : 0.0;
      __syncwarp();
      if (act) {
        for (int j = k + 1; j < NP; ++j) A[lane * NP + j] = fma(-li, A[k * NP + j], A[lane * NP + j]);
        A[lane * NP + k] = li;
      }
      __syncwarp();
      if (lane == 0) A[k * NP + k] = rk;
      __syncwarp();
    }
    __syncwarp();
  }
  if (!pd) {
    for (int i = lane; i < NP * NP; i += 32) {
      const int r = i / NP, c = i % NP;
      A[i] = r == c ? 1.0 / (fabs(H[i]) + scale) : 0.0;
    }
    __syncwarp();
  }
  for (int i = lane; i < NP * NP; i += 32) out[i] = (i / NP) > (i % NP) || (i / NP) == (i % NP) ? A[i] : 0.0;
}

// x = 0, r = g = -gJ, z = M^-1 r; partial sums r.z, g.g and max |g|.
__global__ void __launch_bounds__(32 * JN_WARPS) jn_cg_init_kernel(JNDev J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * JN_WARPS + warp;
  if (s >= J.S) return;
  const size_t o = (size_t)s * NP + lane;
  const bool row = lane < NP;
  const double g = row ? -J.gJ[o] : 0.0;
  const double z = jn_minv(J.Mf + (size_t)s * NP * NP, g, lane);
  if (row) {
    J.x[o] = 0.0;
    J.r[o] = g;
    J.z[o] = z;
    J.d0[o] = 0.0;
    J.d1[o] = 0.0;
  }
  const double rz = jn_warp_sum(g * z), gg = jn_warp_sum(g * g), gm = jn_warp_max(fabs(g));
  if (lane == 0) {
    J.part[s] = rz;
    J.part[J.S + s] = gg;
    J.part[2 * J.S + s] = gm;
  }
}

// Fixed-order sums over the sources of part[q] (one block).
__device__ inline double jn_block_sum(const double* __restrict__ v, int n, bool take_max) {
  __shared__ double red[256];
  double a = 0.0;   // (the maxima taken here are of non-negative values)
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = take_max ? fmax(a, v[i]) : a + v[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = take_max ? fmax(red[threadIdx.x], red[threadIdx.x + w]) : red[threadIdx.x] + red[threadIdx.x + w];
    __syncthreads();
  }
  const double out = red[0];
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(256) jn_scalar_init_kernel(JNDev J, double delta) {
  const double rz = jn_block_sum(J.part, J.S, false);
  const double gg = jn_block_sum(J.part + J.S, J.S, false);
  const double gm = jn_block_sum(J.part + 2 * J.S, J.S, true);
  if (threadIdx.x == 0) {
    JNScalars& c = *J.sc;
    c.rz = rz;
    c.gnorm = sqrt(gg);
    c.gmax = gm;
    c.eps = 1e-2 * c.gnorm;   // relative residual: each subproblem an accurate Newton step
    c.rstop = 0;
    c.delta = delta;
    c.xMx = 0.0;
    c.xMd = 0.0;
    c.dMd = rz;
    c.beta = 0.0;
    c.alpha = 0.0;
    c.tau = 0.0;
    c.cur = 0;
    c.stop = !(c.gnorm > 0.0) || !(rz > 0.0);
    c.mode = 0;
    c.boundary = 0;
    c.cg_iters = 0;
  }
}

// d_new = -z + beta d (on the fly for the coupled sources; the owner stores it in the other
// buffer), Bd = B d_new, partial d_new.Bd.
__global__ void __launch_bounds__(32 * JN_WARPS) jn_matvec_kernel(JNDev J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * JN_WARPS + warp;
  if (s >= J.S || J.sc->stop) return;
  const double beta = J.sc->beta;
  const double* dc = J.sc->cur ? J.d1 : J.d0;
  double* dn = J.sc->cur ? J.d0 : J.d1;
  const bool row = lane < NP;
  auto dnew = [&](int t) { return row ? -J.z[(size_t)t * NP + lane] + beta * dc[(size_t)t * NP + lane] : 0.0; };
  const double ds = dnew(s);
  const double y = jn_rowmul(J, s, lane, dnew);
  if (row) {
    dn[(size_t)s * NP + lane] = ds;
    J.Bd[(size_t)s * NP + lane] = y;
  }
  const double k = jn_warp_sum(ds * y);
  if (lane == 0) J.part[s] = k;
}

__device__ inline double jn_boundary_tau(const JNScalars& c) {
  const double d2 = c.delta * c.delta;
  const double disc = fmax(c.xMd * c.xMd + c.dMd * (d2 - c.xMx), 0.0);
  return (-c.xMd + sqrt(disc)) / c.dMd;
}

// Curvature test and step length (the direction buffers swap here).
__global__ void __launch_bounds__(256) jn_scalar_a_kernel(JNDev J) {
  if (J.sc->stop) return;
  const double kappa = jn_block_sum(J.part, J.S, false);
  if (threadIdx.x == 0) {
    JNScalars& c = *J.sc;
    c.cur ^= 1;
    if (!(kappa > 0.0)) {
      c.tau = jn_boundary_tau(c);
      c.mode = 2;
    } else {
      c.alpha = c.rz / kappa;
      if (c.xMx + 2.0 * c.alpha * c.xMd + c.alpha * c.alpha * c.dMd >= c.delta * c.delta) {
        c.tau = jn_boundary_tau(c);
        c.mode = 2;
      } else {
        c.mode = 1;
      }
    }
  }
}

// x += alpha d, r += alpha Bd, z = M^-1 r (or x += tau d onto the boundary); partial r.z, r.r.
__global__ void __launch_bounds__(32 * JN_WARPS) jn_update_kernel(JNDev J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * JN_WARPS + warp;
  if (s >= J.S || J.sc->stop) return;
  const JNScalars c = *J.sc;
  const double* d = c.cur ? J.d1 : J.d0;
  const size_t o = (size_t)s * NP + lane;
  const bool row = lane < NP;
  if (c.mode == 2) {
    if (row) J.x[o] += c.tau * d[o];
    return;
  }
  double r = 0.0;
  if (row) {
    J.x[o] += c.alpha * d[o];
    r = J.r[o] + c.alpha * J.Bd[o];
    J.r[o] = r;
  }
  const double z = jn_minv(J.Mf + (size_t)s * NP * NP, r, lane);
  if (row) J.z[o] = z;
  const double rz = jn_warp_sum(r * z), rr = jn_warp_sum(r * r);
  if (lane == 0) {
    J.part[s] = rz;
    J.part[J.S + s] = rr;
  }
}

// Residual test and the next direction's coefficient; the M-norm recurrences of Steihaug's method.
__global__ void __launch_bounds__(256) jn_scalar_b_kernel(JNDev J) {
  if (J.sc->stop) return;
  if (J.sc->mode == 2) {
    if (threadIdx.x == 0) {
      JNScalars& c = *J.sc;
      c.stop = 1;
      c.boundary = 1;
      c.xMx = c.delta * c.delta;
      c.cg_iters += 1;
    }
    return;
  }
  const double rz = jn_block_sum(J.part, J.S, false);
  const double rr = jn_block_sum(J.part + J.S, J.S, false);
  if (threadIdx.x == 0) {
    JNScalars& c = *J.sc;
    c.xMx += 2.0 * c.alpha * c.xMd + c.alpha * c.alpha * c.dMd;
    c.cg_iters += 1;
    if (sqrt(rr) <= c.eps) {
      c.stop = 1;
      c.rstop = 1;
    } else {
      c.beta = rz / c.rz;
      c.rz = rz;
      c.xMd = c.beta * (c.xMd + c.alpha * c.dMd);
      c.dMd = rz + c.beta * c.beta * c.dMd;
    }
  }
}

// Model decrease of the step: pred = -(g.x + x.Bx/2), g = -gJ.
__global__ void __launch_bounds__(32 * JN_WARPS) jn_model_kernel(JNDev J) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * JN_WARPS + warp;
  if (s >= J.S) return;
  const bool row = lane < NP;
  auto xv = [&](int t) { return row ? J.x[(size_t)t * NP + lane] : 0.0; };
  const double Bx = jn_rowmul(J, s, lane, xv);
  const double xs = xv(s);
  const double g = row ? -J.gJ[(size_t)s * NP + lane] : 0.0;
  const double q = jn_warp_sum(g * xs + 0.5 * xs * Bx);
  if (lane == 0) J.part[s] = q;
}

__global__ void __launch_bounds__(256) jn_scalar_model_kernel(JNDev J) {
  const double q = jn_block_sum(J.part, J.S, false);
  if (threadIdx.x == 0) J.sc->pred = -q;
}

// trial = theta + x
__global__ void jn_trial_kernel(const double* __restrict__ theta, const double* __restrict__ x, double* trial, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) trial[i] = theta[i] + x[i];
}

// Sum over sources of the per-source value sums (the change of J from the reference point).
__global__ void __launch_bounds__(256) jn_sum_kernel(const double* __restrict__ v, int n, JNScalars* sc) {
  const double a = jn_block_sum(v, n, false);
  if (threadIdx.x == 0) sc->dJ = a;
}

// Reference rates of every patch pixel at the current point: E = bE + iota E[G_s], V = bV +
// iota^2 Var[G_s] (the background and the source's moments of the last full evaluation).
__global__ void jn_refev_kernel(ProblemDev P) {
  const TileDev t = P.tiles[blockIdx.x];
  const PatchDev pt = P.patches[t.patch];
  const float iota = P.images[pt.image].iota;
  for (int i = threadIdx.x; i < t.count; i += blockDim.x) {
    const long long o = pt.pix_off + t.start + i;
    const float4 pv = P.pix[o];
    const float2 m = P.srcmom[o];
    P.refEV[o] = make_float2(pv.y + iota * m.x, pv.z + iota * iota * m.y);
  }
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_joint_pairs(celeste_problem* p, int32_t* pairs, int64_t capacity, int64_t* n_pairs) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!n_pairs) return fail(CELESTE_ERR_INVALID_ARG, "null n_pairs");
  joint_host(p);
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

namespace {

struct JNLayout {
  size_t gJ, Hd, Hc, Mf, x, r, z, d0, d1, Bd, trial, part, vals, elbo, pweight, refEV, row_ptr, row_ent, sc, total;
};

JNLayout jn_layout(int S, int n_pairs, long long n_pix) {
  JNLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + std::max(bytes, (size_t)1) + 255) & ~size_t(255);
    return at;
  };
  const size_t vec = sizeof(double) * NP * S, blk = sizeof(double) * NP * NP;
  L.gJ = take(vec);
  L.Hd = take(blk * S);
  L.Hc = take(blk * std::max(n_pairs, 1));
  L.Mf = take(blk * S);
  L.x = take(vec);
  L.r = take(vec);
  L.z = take(vec);
  L.d0 = take(vec);
  L.d1 = take(vec);
  L.Bd = take(vec);
  L.trial = take(vec);
  L.part = take(sizeof(double) * 3 * S);
  L.vals = take(sizeof(double) * S);
  L.elbo = take(sizeof(double) * S);
  L.pweight = take(sizeof(float) * n_pix);
  L.refEV = take(sizeof(float2) * n_pix);
  L.row_ptr = take(sizeof(int) * (S + 1));
  L.row_ent = take(sizeof(int) * 2 * std::max(n_pairs, 1));
  L.sc = take(sizeof(JNScalars));
  L.total = o;
  return L;
}


// Each source's coupling entries (pair index * 2 + side), CSR over the sources: host lists kept on
// the problem for the upload at bind.
void jn_rows(celeste_problem* p) {
  const int S = p->S, n_pairs = (int)p->joint_pairs.size() / 2;
  std::vector<int>& row_ptr = p->jn_row_ptr_h;
  std::vector<int>& row_ent = p->jn_row_ent_h;
  row_ptr.assign(S + 1, 0);
  row_ent.assign(2 * std::max(n_pairs, 1), 0);
  for (int k = 0; k < n_pairs; ++k) {
    row_ptr[p->joint_pairs[2 * k] + 1] += 1;
    row_ptr[p->joint_pairs[2 * k + 1] + 1] += 1;
  }
  for (int s = 0; s < S; ++s) row_ptr[s + 1] += row_ptr[s];
  std::vector<int> fill(row_ptr.begin(), row_ptr.end() - 1);
  for (int k = 0; k < n_pairs; ++k) {
    row_ent[fill[p->joint_pairs[2 * k]]++] = 2 * k;
    row_ent[fill[p->joint_pairs[2 * k + 1]]++] = 2 * k + 1;
  }
}

int jn_state(celeste_problem* p, const JNLayout&) {
  if (!p->jn_dev) return fail(CELESTE_ERR_STATE, "bind the joint workspace first (celeste_joint_bind)");
  return CELESTE_OK;
}

}  // namespace

extern "C" int celeste_joint_newton(celeste_problem* p, double* theta, const celeste_newton_opts* opts, int32_t max_cg,
                                    int32_t* iters_out, int32_t* status_out, double* J_out, int32_t* cg_iters_out,
                                    celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  if (!theta || !iters_out || !status_out || !J_out) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  int rc = joint_build(p);
  if (rc != CELESTE_OK) return rc;
  celeste_newton_opts o{};
  if (opts) o = *opts;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 50;
  const double ftol = o.ftol > 0 ? o.ftol : 1e-8, gtol = o.gtol > 0 ? o.gtol : 1e-10;
  const double eta = o.eta > 0 ? o.eta : 0.1, delta_min = o.delta_min > 0 ? o.delta_min : 1e-12;
  const double delta_max_factor = o.delta_max > 0 ? o.delta_max : 1e4;
  const int ncg = max_cg > 0 ? max_cg : 100;
  const int S = p->S, n_pairs = (int)p->joint_pairs.size() / 2;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  const JNLayout L = jn_layout(S, n_pairs, p->n_pix);
  if ((rc = jn_state(p, L)) != CELESTE_OK) return rc;
  char* b = static_cast<char*>(p->jn_dev);
  double* gJ = reinterpret_cast<double*>(b + L.gJ);
  double* Hd = reinterpret_cast<double*>(b + L.Hd);
  double* Hc = reinterpret_cast<double*>(b + L.Hc);
  double* trial = reinterpret_cast<double*>(b + L.trial);
  double* vals = reinterpret_cast<double*>(b + L.vals);
  double* elbo = reinterpret_cast<double*>(b + L.elbo);
  JNScalars* scd = reinterpret_cast<JNScalars*>(b + L.sc);
  JNDev J{S, gJ, Hd, Hc, reinterpret_cast<const int*>(b + L.row_ptr), reinterpret_cast<const int*>(b + L.row_ent),
          nullptr, reinterpret_cast<double*>(b + L.Mf), reinterpret_cast<double*>(b + L.x),
          reinterpret_cast<double*>(b + L.r), reinterpret_cast<double*>(b + L.z), reinterpret_cast<double*>(b + L.d0),
          reinterpret_cast<double*>(b + L.d1), reinterpret_cast<double*>(b + L.Bd),
          reinterpret_cast<double*>(b + L.part), scd};
  const JointDev JD = joint_view(p);
  J.pairs = JD.pairs;
  ProblemDev Dj = p->dev;
  Dj.pweight = reinterpret_cast<float*>(b + L.pweight);
  ProblemDev Dd = Dj;
  Dd.refEV = reinterpret_cast<float2*>(b + L.refEV);
  const int wb = (S + JN_WARPS - 1) / JN_WARPS;
  long long launches = 0;

#define JN_TRY(call, what)                                  \
  do {                                                      \
    if ((e = (call)) != cudaSuccess) return cuda_fail(e, what); \
  } while (0)
#define JN_LAUNCHED(what)                                   \
  do {                                                      \
    ++launches;                                             \
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, what); \
  } while (0)

  // ELBO gradient, diagonal and cross blocks, reference rates and preconditioner at th
  auto full_eval = [&](const double* th) -> int {
    JN_TRY(launch_background(Dj, th, 1, st), "background");
    JN_TRY(launch_set_flags(Dj, FLAG_FULL, st), "set flags");
    JN_TRY(launch_worklists(Dj, FLAG_FULL, st), "worklists");
    JN_TRY(launch_full(Dj, th, st), "pixel kernel");
    JN_TRY(launch_assemble(Dj, th, true, elbo, gJ, Hd, st), "assemble");
    launches += 7;
    if (p->joint_n_tiles > 0) {
      cross_kernel<<<p->joint_n_tiles, JT_PIX, 0, st>>>(Dj, JD);
      JN_LAUNCHED("cross_kernel");
    }
    if (n_pairs > 0) {
      cross_assemble_kernel<<<n_pairs, 128, 0, st>>>(Dj, JD, th, Hc);
      JN_LAUNCHED("cross_assemble_kernel");
    }
    if (Dd.n_tiles > 0) {
      jn_refev_kernel<<<Dd.n_tiles, 128, 0, st>>>(Dd);
      JN_LAUNCHED("refev");
    }
    jn_precond_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
    JN_LAUNCHED("precond");
    return CELESTE_OK;
  };
  // per-source value sums at th (difference from ref when ref is given) and their total
  auto value_eval = [&](const double* th, const double* ref, double& out) -> int {
    const ProblemDev& D = ref ? Dd : Dj;
    JN_TRY(launch_background(D, th, 1, st), "background");
    JN_TRY(launch_set_flags(D, FLAG_VALUE, st), "set flags");
    JN_TRY(launch_worklists(D, FLAG_VALUE, st), "worklists");
    JN_TRY(launch_value(D, th, ref != nullptr, st), "value kernel");
    JN_TRY(launch_assemble_value(D, th, ref, vals, st), "assemble value");
    jn_sum_kernel<<<1, 256, 0, st>>>(vals, S, scd);
    JN_LAUNCHED("sum");
    launches += 7;
    JNScalars h;
    JN_TRY(cudaMemcpyAsync(&h, scd, sizeof(h), cudaMemcpyDeviceToHost, st), "scalars");
    JN_TRY(cudaStreamSynchronize(st), "sync");
    out = h.dJ;
    return CELESTE_OK;
  };
  auto read_scalars = [&](JNScalars& h) -> int {
    JN_TRY(cudaMemcpyAsync(&h, scd, sizeof(h), cudaMemcpyDeviceToHost, st), "scalars");
    JN_TRY(cudaStreamSynchronize(st), "sync");
    return CELESTE_OK;
  };

  double Jcur = 0.0;
  JN_TRY(clear_timeout(Dj, st), "clear timeout word");
  if ((rc = value_eval(theta, nullptr, Jcur)) != CELESTE_OK) return rc;
  if ((rc = full_eval(theta)) != CELESTE_OK) return rc;
  // initial radius: the M-norm of the block-diagonal Newton step, sqrt(g^T M^-1 g)
  jn_cg_init_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
  JN_LAUNCHED("cg init");
  jn_scalar_init_kernel<<<1, 256, 0, st>>>(J, 1.0);
  JN_LAUNCHED("cg scalars");
  JNScalars h;
  if ((rc = read_scalars(h)) != CELESTE_OK) return rc;
  double delta = h.rz > 0.0 ? sqrt(h.rz) : 1.0;
  const double delta_cap = delta_max_factor * delta;
  double f = -Jcur;
  int status = CELESTE_STATUS_MAX_ITER, iters = 0, cg_total = 0;
  while (iters < max_iter) {
    jn_cg_init_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
    JN_LAUNCHED("cg init");
    jn_scalar_init_kernel<<<1, 256, 0, st>>>(J, delta);
    JN_LAUNCHED("cg scalars");
    // CG iterations in chunks of JN_CHUNK, the stop flag read back after each chunk (a converged
    // or truncated subproblem usually stops within the first chunk; the kernels of a chunk that
    // runs past the stop return at once)
    for (int j = 0; j < ncg; j += JN_CHUNK) {
      for (int q = 0; q < JN_CHUNK && j + q < ncg; ++q) {
        jn_matvec_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
        JN_LAUNCHED("matvec");
        jn_scalar_a_kernel<<<1, 256, 0, st>>>(J);
        JN_LAUNCHED("cg step");
        jn_update_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
        JN_LAUNCHED("cg update");
        jn_scalar_b_kernel<<<1, 256, 0, st>>>(J);
        JN_LAUNCHED("cg direction");
      }
      int stop = 0;
      JN_TRY(cudaMemcpyAsync(&stop, &scd->stop, sizeof(int), cudaMemcpyDeviceToHost, st), "stop flag");
      JN_TRY(cudaStreamSynchronize(st), "sync");
      if (stop) break;
    }
    jn_model_kernel<<<wb, 32 * JN_WARPS, 0, st>>>(J);
    JN_LAUNCHED("model");
    jn_scalar_model_kernel<<<1, 256, 0, st>>>(J);
    JN_LAUNCHED("model scalars");
    if ((rc = read_scalars(h)) != CELESTE_OK) return rc;
    cg_total += h.cg_iters;
    if (!(std::isfinite(f) && std::isfinite(h.gmax))) {
      status = CELESTE_STATUS_NONFINITE;
      break;
    }
    if (h.gmax <= gtol) {
      status = CELESTE_STATUS_CONVERGED;
      break;
    }
    ++iters;
    const double pred = h.pred;
    if (!h.boundary && h.rstop && pred <= ftol * std::fabs(f)) {   // Newton decrement
      status = CELESTE_STATUS_CONVERGED;
      break;
    }
    const int n = S * NP;
    jn_trial_kernel<<<(n + 255) / 256, 256, 0, st>>>(theta, J.x, trial, n);
    JN_LAUNCHED("trial");
    double dJ = 0.0;
    if ((rc = value_eval(trial, theta, dJ)) != CELESTE_OK) return rc;   // J(trial) - J(theta)
    double rho = pred > 0.0 ? dJ / pred : -1.0;
    if (!std::isfinite(dJ)) rho = -1.0;
    if (rho <= eta && pred <= ftol * std::fabs(f)) {   // a rejected step that promised <= ftol |f|
      status = CELESTE_STATUS_CONVERGED;
      break;
    }
    if (rho < 0.25)
      delta *= 0.25;
    else if (rho > 0.75 && h.boundary)
      delta = std::min(2.0 * delta, delta_cap);
    if (rho > eta) {
      const double f_new = f - dJ;
      const bool done = std::fabs(dJ) <= ftol * std::fabs(f_new);
      JN_TRY(cudaMemcpyAsync(theta, trial, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "accept");
      f = f_new;
      if ((rc = full_eval(theta)) != CELESTE_OK) return rc;
      if (done) {
        status = CELESTE_STATUS_CONVERGED;
        break;
      }
    }
    if (delta < delta_min) {
      status = CELESTE_STATUS_RADIUS_COLLAPSE;
      break;
    }
  }
  // leave the background at the returned point
  JN_TRY(launch_background(Dj, theta, 1, st), "background");
  ++launches;
  JN_TRY(cudaStreamSynchronize(st), "sync");
  p->background_ready = true;
  p->background_mode = CELESTE_NBR_WINDOW;
  *iters_out = iters;
  *status_out = status;
  *J_out = -f;
  if (cg_iters_out) *cg_iters_out = cg_total;
  prof_count(p, (int)std::min(launches, (long long)1 << 30));
#undef JN_TRY
#undef JN_LAUNCHED
  return device_errors(Dj, st);
}

extern "C" int celeste_joint_value(celeste_problem* p, const double* theta, double* J_out, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  if (!theta || !J_out) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  int rc = joint_build(p);
  if (rc != CELESTE_OK) return rc;
  const int S = p->S;
  const JNLayout L = jn_layout(S, (int)p->joint_pairs.size() / 2, p->n_pix);
  if ((rc = jn_state(p, L)) != CELESTE_OK) return rc;
  char* b = static_cast<char*>(p->jn_dev);
  cudaStream_t st = (cudaStream_t)stream;
  ProblemDev Dj = p->dev;
  Dj.pweight = reinterpret_cast<float*>(b + L.pweight);
  double* vals = reinterpret_cast<double*>(b + L.vals);
  JNScalars* scd = reinterpret_cast<JNScalars*>(b + L.sc);
  cudaError_t e;
  if ((e = clear_timeout(Dj, st)) != cudaSuccess) return cuda_fail(e, "clear timeout word");
  if ((e = launch_background(Dj, theta, 1, st)) != cudaSuccess) return cuda_fail(e, "background");
  if ((e = launch_set_flags(Dj, FLAG_VALUE, st)) != cudaSuccess) return cuda_fail(e, "set flags");
  if ((e = launch_worklists(Dj, FLAG_VALUE, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  if ((e = launch_value(Dj, theta, false, st)) != cudaSuccess) return cuda_fail(e, "value kernel");
  if ((e = launch_assemble_value(Dj, theta, nullptr, vals, st)) != cudaSuccess) return cuda_fail(e, "assemble value");
  jn_sum_kernel<<<1, 256, 0, st>>>(vals, S, scd);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sum");
  JNScalars h;
  if ((e = cudaMemcpyAsync(&h, scd, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e, "scalars");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sync");
  p->background_ready = true;
  p->background_mode = CELESTE_NBR_WINDOW;
  *J_out = h.dJ;
  prof_count(p, 8);
  return device_errors(Dj, st);
}

extern "C" size_t celeste_joint_workspace_bytes(celeste_problem* p) {
  if (!p) return 0;
  joint_host(p);
  const int n_pairs = (int)p->joint_pairs.size() / 2;
  return joint_layout(p->joint_n_items, p->joint_n_tiles, n_pairs).total + jn_layout(p->S, n_pairs, p->n_pix).total;
}

extern "C" int celeste_joint_bind(celeste_problem* p, void* workspace, size_t bytes, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "bind the problem first");
  joint_host(p);
  const int n_pairs = (int)p->joint_pairs.size() / 2;
  const JointLayout L = joint_layout(p->joint_n_items, p->joint_n_tiles, n_pairs);
  const JNLayout J = jn_layout(p->S, n_pairs, p->n_pix);
  if (!workspace || bytes < L.total + J.total)
    return fail(CELESTE_ERR_WORKSPACE, "joint workspace needs %zu bytes", L.total + J.total);
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(CELESTE_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  char* b = static_cast<char*>(workspace);
  jn_rows(p);
  cudaError_t e = cudaSuccess;
  auto up = [&](size_t off, const std::vector<int>& v) {
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(b + off, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, st);
  };
  up(L.items, p->joint_items_h);
  up(L.tiles, p->joint_tiles_h);
  up(L.pair_items, p->joint_pair_items_h);
  up(L.pairs, p->joint_pairs);
  up(L.total + J.row_ptr, p->jn_row_ptr_h);
  up(L.total + J.row_ent, p->jn_row_ent_h);
  if (e != cudaSuccess) return cuda_fail(e, "joint upload");
  p->joint_dev = b;
  p->jn_dev = b + L.total;
  p->joint_built = true;
  return CELESTE_OK;
}
