// Trust-region subproblem in float64 on four warps (one CTA of 128 threads per problem): the same
// method as the one-warp solver of trsolve.cuh (Nocedal & Wright Sec. 4.3, More-Sorensen), spread
// over the SM's four sub-partitions for the iterations where only a few sources are left.
//
// A warp's float64 instruction stream is what bounds one subproblem on this part (an SM
// sub-partition retires a float64 warp instruction only every few tens of cycles), so when fewer
// subproblems than SMs are in flight, three of every four float64 pipes idle under the one-warp
// solver.  Here:
//   * the L D L^T factorisation and the Householder reduction split the matrix by columns, column j
//     belonging to warp j mod 4 (each warp updates and multiplies its own columns for every row,
//     lane i owning row i); the scalars of a step (norms, reflection coefficients, the reductions
//     of v.p and v.g) are formed by every warp from the same data in the same order, so all warps
//     hold the same values, and two CTA barriers per step order the partial products and the next
//     column;
//   * the multiplier search evaluates 128 multipliers per pass (32 per warp, lane-private
//     recurrences on the tridiagonal form), the warps' minima and maxima combined through shared
//     memory in a fixed order;
//   * the hard case and the back-transformation run on warp 0 as in the one-warp solver.
// Every branch that contains a barrier depends only on values all threads hold identically.
#pragma once

#include "trsolve.cuh"

namespace celeste {

struct TrSmemQ {
  double A[TR_N * TR_LD];         // B; its L D L^T factors, or the Householder vectors below the diagonal
  double beta[TR_N];
  double v[4][32], w[4][32];      // per-warp copies of the reflection vector and of w
  double up[4][32];               // per-warp partial products (A v) over the warp's columns
  double d[TR_N], off[TR_N], o2[TR_N], gh[TR_N], y[TR_N], z[TR_N], D[TR_N], L[TR_N];
  double rd[4][8];                // per-warp results of a multiplier pass
  int ri[4][4];
  int flag[4];
  double PL[4][TR_N][32], PR[4][TR_N][32], PY[4][TR_N][32];
};

// Newton step p = -B^-1 g by L D L^T of S.A in place, columns split over the warps.  Returns false
// if a pivot is not positive (in every thread); otherwise lane i < 27 of every warp holds p_i.
__device__ inline bool tr_newton_step_q(TrSmemQ& S, double gi, double& p_i) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool row = lane < TR_N;
  double* ar = S.A + lane * TR_LD;
  for (int k = 0; k < TR_N; ++k) {
    const double dk = S.A[k * TR_LD + k];
    if (!(dk > 0.0)) return false;   // same value in every thread
    const double r = tr_rcp(dk);
    const bool act = row && lane > k;
    const double li = act ? ar[k] * r : 0.0;
    if (act) {
      // this warp's columns j > k (j = w mod 4)
      for (int j = k + 1 + ((w - (k + 1)) & 3); j < TR_N; j += 4) ar[j] = fma(-li, S.A[k * TR_LD + j], ar[j]);
    }
    __syncthreads();   // row k + 1 and column k + 1 complete; every warp has read column k
    if (act && w == (k & 3)) ar[k] = li;   // L below the diagonal (column k is not read again)
    if (tid == k) S.D[k] = r;
  }
  __syncthreads();
  // L y = -g (column by column), y *= D^-1, L^T x = y (from the bottom); every warp alike
  double y = row ? -gi : 0.0;
  for (int k = 0; k < TR_N - 1; ++k) {
    const double yk = __shfl_sync(0xffffffffu, y, k);
    if (row && lane > k) y = fma(-ar[k], yk, y);
  }
  if (row) y *= S.D[lane];
  for (int k = TR_N - 1; k > 0; --k) {
    const double xk = __shfl_sync(0xffffffffu, y, k);
    if (lane < k) y = fma(-S.A[k * TR_LD + lane], xk, y);
  }
  p_i = row ? y : 0.0;
  return true;
}

// Copies candidate (warp src_w, lane src_l)'s y into S.y; a barrier after, so that the candidate's
// warp may overwrite its scratch in the next pass.
__device__ inline void tr_take_y_q(TrSmemQ& S, int src_w, int src_l) {
  const int tid = threadIdx.x;
  if (tid < TR_N) S.y[tid] = S.PY[src_w][tid][src_l];
  __syncthreads();
}

// The multiplier search of tr_lambda_parallel with 128 candidates per pass (candidate c = 32 warp +
// lane).  Candidate layout: without a Newton point, c = 0 at 0 (first pass, when the interior step
// is to be tested) or the bracket's middle, c = 1-63 geometric from L (2^-47.25 .. 2^-0.75 of the
// bracket), c = 64-127 uniform (1/65 .. 64/65); in the first pass with a hint, c >= 1 on a
// geometric grid around it (2^-7.94 .. 2^7.94, ratio 2^(1/8)); with a Newton point and no secant
// point, c = 0 at it, c = 1-63 above and 64-127 below at 2^-0.75 .. 2^-47.25 of the distance to the
// bracket's ends; with both (the Newton point below the root, the secant point above it, phi being
// concave), c = 0 and 1 at the two, c = 2-111 evenly between them, c = 112-119 above the secant
// point and 120-127 below the Newton point at 2^-2 .. 2^-16 of the distance to the bracket's ends.
// Same return values as tr_lambda_parallel, in every thread.
__device__ inline int tr_lambda_q(TrSmemQ& S, double lo, double hi, double delta, bool try_zero, double spec,
                                  double hint, double& lam_out) {
  constexpr double TOL = 1e-10;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, c = tid;
  double L = lo, H = hi, lamH = hi;
  bool have_h = false;
  double lamN = -1.0, lamS = -1.0;
  double lamL = -INFINITY, phiL = 0.0, dphiL = 1.0, phiH = 0.0;
  const double gfac = c < 64 ? exp2(-0.75 * (double)(64 - c)) : (double)(c - 63) / 65.0;
  const double nfac = exp2(-0.75 * (double)((c & 63) + (c < 64 ? 0 : 1)));
  const double ufac = (double)(c - 1) / 111.0;
  const double afac = exp2(-2.0 * (double)((c & 7) + 1));
  const double hfac = exp2((double)(c - 64) / 8.0 + 0.0625);
  for (int pass = 0; pass < 16; ++pass) {
    double lam;
    const double span = H - L;
    if (pass > 0 && lamN > L && lamN < H && lamS > lamN && lamS <= H)
      lam = c == 0   ? lamN
            : c == 1 ? lamS
            : c < 112 ? lamN + (lamS - lamN) * ufac
            : c < 120 ? lamS + (H - lamS) * afac
                      : lamN - (lamN - L) * afac;
    else if (pass > 0 && lamN > L && lamN < H)
      lam = c == 0 ? lamN : (c < 64 ? lamN + (H - lamN) * nfac : lamN - (lamN - L) * nfac);
    else
      lam = c == 0 ? ((pass == 0 && try_zero) ? 0.0 : L + 0.5 * span) : L + span * gfac;
    if (pass == 0 && hint > L && hint < H && c > 0) {
      const double lh = hint * hfac;
      if (lh > L && lh < H) lam = lh;
    }
    __syncwarp();
    double pn = 0.0, qn2 = 0.0;
    const bool pd = tr_eval_lane(S, S.PL[w], S.PR[w], S.PY[w], lane, lam, pn, qn2);
    // ---- this warp's part: best error, bracket ends, largest left point
    const double err = pd ? fabs(pn - delta) : INFINITY;
    const double bw = tr_warp_min(err);
    const int iw = __ffs(__ballot_sync(0xffffffffu, err == bw)) - 1;
    const bool right = pd && pn <= delta;
    const double nLw = tr_warp_max(right ? -INFINITY : lam);
    const double nHw = tr_warp_min(right ? lam : INFINITY);
    const unsigned mh = __ballot_sync(0xffffffffu, right && lam == nHw);
    const int iHw = mh ? __ffs(mh) - 1 : 0;
    const double pnHw = __shfl_sync(0xffffffffu, pn, iHw);
    const bool lft = pd && pn > delta;
    const double lbw = tr_warp_max(lft ? lam : -INFINITY);
    const unsigned ml = __ballot_sync(0xffffffffu, lft && lam == lbw);
    const int ilw = ml ? __ffs(ml) - 1 : 0;
    const double pnbw = __shfl_sync(0xffffffffu, pn, ilw), qbw = __shfl_sync(0xffffffffu, qn2, ilw);
    const double lamBw = __shfl_sync(0xffffffffu, lam, iw);
    const int int0 = __shfl_sync(0xffffffffu, (int)(pd && pn <= delta), 0);
    if (lane == 0) {
      S.rd[w][0] = bw;
      S.rd[w][1] = nLw;
      S.rd[w][2] = nHw;
      S.rd[w][3] = pnHw;
      S.rd[w][4] = lbw;
      S.rd[w][5] = pnbw;
      S.rd[w][6] = qbw;
      S.rd[w][7] = lamBw;
      S.ri[w][0] = iw;
      S.ri[w][1] = iHw;
      S.ri[w][2] = int0;
    }
    __syncthreads();
    // ---- combined in a fixed order (the first warp wins ties), identically in every thread
    if (pass == 0 && try_zero && S.ri[0][2]) {
      tr_take_y_q(S, 0, 0);
      lam_out = 0.0;
      return 0;
    }
    int wb = 0;
    for (int q = 1; q < 4; ++q)
      if (S.rd[q][0] < S.rd[wb][0]) wb = q;
    if (S.rd[wb][0] <= TOL * delta) {
      lam_out = S.rd[wb][7];
      tr_take_y_q(S, wb, S.ri[wb][0]);
      return 0;
    }
    double newL = S.rd[0][1];
    int wh = 0, wl = 0;
    for (int q = 1; q < 4; ++q) {
      newL = fmax(newL, S.rd[q][1]);
      if (S.rd[q][2] < S.rd[wh][2]) wh = q;
      if (S.rd[q][4] > S.rd[wl][4]) wl = q;
    }
    const double newH = S.rd[wh][2], pnH = S.rd[wh][3];
    const double lbest = S.rd[wl][4], pnb = S.rd[wl][5], qb = S.rd[wl][6];
    const int iH = S.ri[wh][1];
    // every thread has read rd / ri; the copy's barrier orders them before the next pass's writes
    if (newH < H) {
      tr_take_y_q(S, wh, iH);
      H = newH;
      lamH = newH;
      phiH = tr_rcp(pnH) - tr_rcp(delta);
      have_h = true;
    } else {
      __syncthreads();
    }
    L = fmax(L, newL);
    if (lbest > lamL) {
      lamL = lbest;
      phiL = tr_rcp(pnb) - tr_rcp(delta);
      dphiL = qb * tr_rcp(pnb * pnb * pnb);
    }
    lamN = lamL > -INFINITY ? lamL - phiL * tr_rcp(dphiL) : -1.0;
    lamS = have_h && lamL > -INFINITY && phiH > phiL ? lamL + (H - lamL) * (-phiL * tr_rcp(phiH - phiL)) : -1.0;
    if (H - L <= 4.0 * DBL_EPSILON * fmax(fabs(H), spec)) {
      if (!have_h) return 1;
      lam_out = lamH;   // (the hard case only without a positive definite point past delta: see tr_lambda_parallel)
      return lamL == -INFINITY && tr_norm(S.y) < delta * (1.0 - 1e-6) ? 1 : 0;
    }
  }
  lam_out = lamH;
  return have_h ? 0 : 1;
}

// Solves the subproblem on the CTA's four warps; the arguments are those of tr_solve_warp (gi: the
// gradient entry of lane i, the same in every warp).  On return warp 0's lane i < 27 holds p_i
// and warp 0 holds pred, hard and lam_out (every warp, when the Newton step was taken).
__device__ inline bool tr_solve_q(TrSmemQ& S, const double* __restrict__ Bsrc, double bsign, double gi, double delta,
                                  bool try_newton, const double* __restrict__ cache_in, double* __restrict__ cache_out,
                                  double lam_hint, double& lam_out, double& p_i, double& pred, int& hard) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = TR_N;
  const bool row = lane < n;
  const double gnorm = sqrt(tr_warp_sum(gi * gi));
  bool stored = false;
  if (cache_in) {
    for (int i = tid; i < TR_N * TR_N; i += 128) S.A[(i / TR_N) * TR_LD + (i % TR_N)] = cache_in[i];
    if (tid < n) {
      S.d[tid] = cache_in[TR_N * TR_N + tid];
      S.off[tid] = cache_in[TR_N * TR_N + TR_N + tid];
      S.o2[tid] = cache_in[TR_N * TR_N + 2 * TR_N + tid];
      S.gh[tid] = cache_in[TR_N * TR_N + 3 * TR_N + tid];
      S.beta[tid] = cache_in[TR_N * TR_N + 4 * TR_N + tid];
    }
    __syncthreads();
  } else {
    if (try_newton) {
      for (int i = tid; i < TR_N * TR_N; i += 128) S.A[i] = bsign * Bsrc[i];
      __syncthreads();
      double pn;
      const bool pdef = tr_newton_step_q(S, gi, pn);
      if (pdef) {
        const double pp = tr_warp_sum(pn * pn);
        if (sqrt(pp) <= delta) {
          p_i = pn;
          pred = -0.5 * tr_warp_sum(gi * pn);
          hard = 0;
          lam_out = 0.0;
          return false;
        }
      }
      __syncthreads();   // every warp is done with the factors before B is loaded again
    }
    for (int i = tid; i < TR_N * TR_N; i += 128) S.A[i] = bsign * Bsrc[i];
    __syncthreads();
    // ---- Householder tridiagonalisation: lane i owns row i, warp w the columns j = w mod 4
    double gh = row ? gi : 0.0;
    double* ar = S.A + lane * TR_LD;
    for (int k = 0; k < n - 2; ++k) {
      const double xi = lane > k && row ? ar[k] : 0.0;
      const double s2 = tr_warp_sum(xi * xi);
      const double x0 = S.A[(k + 1) * TR_LD + k];
      if (s2 == 0.0) {   // same in every warp
        if (tid == 0) {
          S.beta[k] = 0.0;
          S.off[k + 1] = 0.0;
        }
        continue;
      }
      const double alpha = -copysign(sqrt(s2), x0);
      const double vi = lane == k + 1 ? x0 - alpha : xi;
      const double beta = tr_rcp(s2 - alpha * x0);
      S.v[w][lane] = vi;
      __syncwarp();
      const int j0 = k + 1 + ((w - (k + 1)) & 3);   // this warp's first column > k
      double u0 = 0.0, u1 = 0.0;
      if (lane > k && row) {
        int j = j0;
        for (; j + 4 < n; j += 8) {
          u0 = fma(ar[j], S.v[w][j], u0);
          u1 = fma(ar[j + 4], S.v[w][j + 4], u1);
        }
        if (j < n) u0 = fma(ar[j], S.v[w][j], u0);
      }
      S.up[w][lane] = u0 + u1;
      __syncthreads();   // (a) the four partial products
      const double u = (S.up[0][lane] + S.up[1][lane]) + (S.up[2][lane] + S.up[3][lane]);
      const double pi = beta * u;
      double vp = vi * pi, vg = vi * gh;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vp += __shfl_xor_sync(0xffffffffu, vp, o);
        vg += __shfl_xor_sync(0xffffffffu, vg, o);
      }
      const double K = 0.5 * beta * vp;
      const double wi = pi - K * vi;
      gh = fma(-beta * vg, vi, gh);
      S.w[w][lane] = wi;
      __syncwarp();
      if (lane > k && row) {
        for (int j = j0; j < n; j += 4) ar[j] = fma(-vi, S.w[w][j], fma(-wi, S.v[w][j], ar[j]));
        if (w == (k & 3)) ar[k] = vi;   // the reflection vector (column k is not read again)
      }
      if (tid == 0) {
        S.beta[k] = beta;
        S.off[k + 1] = alpha;
      }
      __syncthreads();   // (b) column k + 1 complete before the next step reads it
    }
    if (tid < n) S.d[tid] = S.A[tid * TR_LD + tid];
    if (w == 0 && row) S.gh[lane] = gh;
    if (tid == 0) {
      S.off[n - 1] = S.A[(n - 1) * TR_LD + n - 2];
      S.off[0] = 0.0;
    }
    __syncthreads();
    if (tid < n) S.o2[tid] = S.off[tid] * S.off[tid];
    __syncthreads();
    if (cache_out) {
      for (int i = tid; i < TR_N * TR_N; i += 128) cache_out[i] = S.A[(i / TR_N) * TR_LD + (i % TR_N)];
      if (tid < n) {
        cache_out[TR_N * TR_N + tid] = S.d[tid];
        cache_out[TR_N * TR_N + TR_N + tid] = S.off[tid];
        cache_out[TR_N * TR_N + 2 * TR_N + tid] = S.o2[tid];
        cache_out[TR_N * TR_N + 3 * TR_N + tid] = S.gh[tid];
        cache_out[TR_N * TR_N + 4 * TR_N + tid] = S.beta[tid];
      }
      stored = true;
    }
  }

  // ---- multiplier (bounds as in tr_solve_warp, formed by every warp alike)
  const int li = row ? lane : 0, ln = lane + 1 < n ? lane + 1 : 0;
  const double di = S.d[li], oi = fabs(S.off[li]), on = lane + 1 < n ? fabs(S.off[ln]) : 0.0;
  const double a = tr_warp_min(row ? di - (oi + on) : INFINITY);
  const double dmin = tr_warp_min(row ? di : INFINITY);
  const double dmax = tr_warp_max(row ? fabs(di) : 0.0);
  const double omax = tr_warp_max(row ? oi : 0.0);
  const double spec = dmax + 2.0 * omax;
  const double scale = fmax(1.0, spec);
  const double lo = fmax(0.0, -dmin);
  const double hi = fmax(lo, gnorm / delta - a) * (1.0 + 1e-12) + 1e-300;
  if (tid == 0) S.flag[2] = 0;
  __syncthreads();
  lam_out = -1.0;
  const int hc = tr_lambda_q(S, lo, hi, delta, lo == 0.0, spec, lam_hint, lam_out);
  if (hc) {
    lam_out = -1.0;
    // hard case on warp 0, as in tr_solve_warp
    if (w == 0) {
      float fa = (float)a, fb = (float)(dmin);
      for (int it = 0; it < 6; ++it) {
        const float x = fa + (fb - fa) * (float)(lane + 1) / 33.f;
        const unsigned m = __ballot_sync(0xffffffffu, tr_sturm_f(S, x) >= 1);
        const int f = m ? __ffs(m) - 1 : 32;
        const float na = f > 0 ? fa + (fb - fa) * (float)f / 33.f : fa;
        const float nb = f < 32 ? fa + (fb - fa) * (float)(f + 1) / 33.f : fb;
        fa = na;
        fb = nb;
      }
      const double ab = fmax(a, (double)fa - 1e-5 * scale), bb = fmin((double)dmin, (double)fb + 1e-5 * scale);
      if (lane == 0) {
        tr_ldl(S, -(ab - 1e-8 * scale));
        for (int i = 0; i < n; ++i) S.z[i] = 1.0;
        for (int r = 0; r < 4; ++r) {
          tr_ldl_solve(S, S.z, S.z);
          const double rz = tr_rcp(tr_norm(S.z));
          for (int i = 0; i < n; ++i) S.z[i] *= rz;
        }
        double lmin = 0.0, zg = 0.0;
        for (int i = 0; i < n; ++i) {
          double Tz = S.d[i] * S.z[i];
          if (i > 0) Tz += S.off[i] * S.z[i - 1];
          if (i + 1 < n) Tz += S.off[i + 1] * S.z[i + 1];
          lmin += S.z[i] * Tz;
          zg += S.z[i] * S.gh[i];
        }
        lmin = fmin(lmin, bb);
        tr_ldl(S, fmax(0.0, -lmin) + 1e-9 * scale);
        for (int i = 0; i < n; ++i) S.y[i] = -S.gh[i];
        tr_ldl_solve(S, S.y, S.y);
        double zy = 0.0;
        for (int i = 0; i < n; ++i) zy += S.z[i] * S.y[i];
        for (int i = 0; i < n; ++i) S.y[i] -= zy * S.z[i];
        const double yn = tr_norm(S.y);
        if (yn > delta) {
          for (int i = 0; i < n; ++i) S.y[i] *= delta / yn;
        } else {
          const double tau = copysign(sqrt(fmax(delta * delta - yn * yn, 0.0)), -zg);
          for (int i = 0; i < n; ++i) S.y[i] += tau * S.z[i];
        }
        S.flag[2] = 1;
      }
    }
  } else if (tid == 0) {
    const double yn = tr_norm(S.y);
    if (yn > delta)
      for (int i = 0; i < n; ++i) S.y[i] *= delta / yn;
  }
  __syncthreads();
  hard = S.flag[2];
  // ---- p = Q y and the model value, on warp 0
  if (w == 0) {
    double yi = row ? S.y[lane] : 0.0;
    double Ty = 0.0;
    if (row) {
      Ty = S.d[lane] * yi + (lane > 0 ? S.off[lane] * S.y[lane - 1] : 0.0) +
           (lane + 1 < n ? S.off[lane + 1] * S.y[lane + 1] : 0.0);
    }
    const double gy = tr_warp_sum(row ? S.gh[lane] * yi : 0.0);
    const double yTy = tr_warp_sum(yi * Ty);
    pred = -(gy + 0.5 * yTy);
    for (int k = n - 3; k >= 0; --k) {
      const double vk = lane > k && row ? S.A[lane * TR_LD + k] : 0.0;
      const double t = tr_warp_sum(vk * yi);
      yi -= S.beta[k] * vk * t;
    }
    p_i = yi;
  }
  __syncthreads();
  return stored;
}

}  // namespace celeste
