// Trust-region subproblem in float64, one warp per problem:
//     minimise  g.p + p.B.p / 2   subject to  |p| <= delta      (B symmetric 27 x 27)
// More-Sorensen characterisation (Nocedal & Wright, Sec. 4.3): p = -(B + lambda I)^-1 g with
// lambda >= max(0, -lambda_min(B)), lambda (|p| - delta) = 0, plus the "hard case" where g has no
// component along the eigenvector of lambda_min.
//
// On GB300 one warp's float64 work is bounded by the number of FP64 instructions it issues (the
// FP64 pipe of an SM sub-partition retires a warp-wide FMA only every several tens of cycles), so
// the solver keeps that count low:
//   * Newton step first: where the caller expects it (the previous step was interior), B is
//     factored B = L D L^T in place (lane i owns row i); if every pivot is positive and
//     |B^-1 g| <= delta the Newton step is the solution and nothing else runs;
//   * otherwise B is reduced once to tridiagonal form T = Q^T B Q by Householder reflections
//     (lane-parallel; g is reflected in the same reductions), after which every solve with
//     T + lambda I is an O(n) LDL^T recurrence:
//   * the multiplier lambda >= max(0, -lambda_min) with |p(lambda)| = delta (Nocedal & Wright
//     Sec. 4.3, Moré-Sorensen) by passes of 32 multipliers at once, one per lane (each lane
//     factors T + lambda I and solves with it): a geometric-plus-uniform grid over the bracket,
//     then points around the Newton iterate of phi(lambda) = 1/|p| - 1/delta from the largest
//     left point (phi concave and increasing: Newton from the left stays left).  A float64
//     warp instruction costs the same for 1 or 32 lanes here, so a pass costs one evaluation;
//     positive definiteness of T + lambda I (Sylvester: all LDL^T pivots positive) tells the
//     points left of the pole -lambda_min; lambda = 0 tests the interior step;
//   * hard case (the bracket closes on the pole with |p| < delta): eigenvector of lambda_min by
//     inverse iteration on T after a float32 Sturm bracket, p = y + tau z;
//   * lane-dependent choices are selects and every lane finishes its evaluation, so the warp
//     stays converged through the float64 passes (a split warp issues them once per part).
// The step is mapped back with the reflections, p = Q y.
#pragma once

#include <cfloat>

#include "celeste_internal.cuh"

namespace celeste {

constexpr int TR_N = NP;          // 27
constexpr int TR_LD = NP;         // row length of the matrix in shared memory (27 doubles: the
                                  // rows of a warp's lanes start on distinct bank pairs)

struct TrSmem {
  double A[TR_N * TR_LD];         // B; its L D L^T factors, or the Householder vectors below
                                  // the diagonal after the reduction
  double beta[TR_N];              // reflection coefficients
  double v[32], w[32];            // per-step temporaries
  double d[TR_N], off[TR_N];      // T: diagonal, off[i] = T[i][i-1]
  double o2[TR_N];                // off[i]^2
  double gh[TR_N], y[TR_N], z[TR_N];
  double D[TR_N], L[TR_N];        // LDL^T of T + lambda I (D holds the reciprocal pivots)
  double sc[4];                   // broadcast scalars
  int flag[4];
  // lane-private factors of T + lambda_lane I for the parallel secular-equation passes
  double PL[TR_N][32], PR[TR_N][32], PY[TR_N][32];
};

// 1/a in float64 with few float64-pipe instructions (a float64 division issues a dozen, and the
// solver's recurrences divide once per row): the approximate reciprocal of the PTX ISA
// (rcp.approx.ftz.f64, special-function unit) refined by two Newton-Raphson steps for f(r) = 1/r - a,
// r <- r + r (1 - a r) (Ypma, "Historical development of the Newton-Raphson method", SIAM Review
// 1995), each squaring the relative error: a seed good to 2^-14 ends within an ulp or two of 1/a.
// Normal a only: |a| < 2^-1022 or a = 0 gives NaN (the solver masks those rows as not positive
// definite), |a| > 2^1022 gives 0.
__device__ __forceinline__ double tr_rcp(double a) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
  double e = fma(-a, r, 1.0);
  r = fma(r, e, r);
  e = fma(-a, r, 1.0);
  return fma(r, e, r);
}

__device__ inline double tr_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// LDL^T of T + lambda I into S.D (reciprocal pivots), S.L; returns false if a pivot is not positive.
// (The helpers below take any shared-memory layout with the members they use: the one-warp
// solver's TrSmem and the four-warp solver's.)
template <class SM>
__device__ inline bool tr_ldl(SM& S, double lambda) {
  double Dp = S.d[0] + lambda;
  bool pd = Dp > 0.0;
  double r = tr_rcp(Dp);
  S.D[0] = r;
  for (int i = 1; i < TR_N; ++i) {
    S.L[i] = S.off[i] * r;                 // off the pivot chain
    Dp = fma(-S.o2[i], r, S.d[i] + lambda);
    pd = pd && Dp > 0.0;
    r = tr_rcp(Dp);
    S.D[i] = r;
  }
  return pd;
}

// Solve (L D L^T) x = b (b may alias x).
template <class SM>
__device__ inline void tr_ldl_solve(const SM& S, const double* b, double* x) {
  x[0] = b[0];
  for (int i = 1; i < TR_N; ++i) x[i] = b[i] - S.L[i] * x[i - 1];
  for (int i = 0; i < TR_N; ++i) x[i] *= S.D[i];
  for (int i = TR_N - 2; i >= 0; --i) x[i] -= S.L[i + 1] * x[i + 1];
}

__device__ inline double tr_norm(const double* x) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;   // four chains instead of one
#pragma unroll
  for (int i = 0; i + 3 < TR_N; i += 4) {
    s0 = fma(x[i], x[i], s0);
    s1 = fma(x[i + 1], x[i + 1], s1);
    s2 = fma(x[i + 2], x[i + 2], s2);
    s3 = fma(x[i + 3], x[i + 3], s3);
  }
#pragma unroll
  for (int i = TR_N & ~3; i < TR_N; ++i) s0 = fma(x[i], x[i], s0);
  return sqrt((s0 + s1) + (s2 + s3));
}

// Float32 Sturm count (only used to bracket lambda_min; the bracket is widened afterwards).
template <class SM>
__device__ inline int tr_sturm_f(const SM& S, float x) {
  float q = (float)S.d[0] - x;
  int c = q < 0.f;
  for (int i = 1; i < TR_N; ++i) {
    if (q == 0.f) q = -1e-30f;
    const float o = (float)S.off[i];
    q = (float)S.d[i] - x - o * o / q;
    c += q < 0.f;
  }
  return c;
}

// Lane-private evaluation at the lane's own multiplier lam: L D L^T = T + lam I (reciprocal
// pivots in PR), y = -(T + lam I)^-1 gh in PY (PL, PR, PY: the warp's [TR_N][32] scratch); returns
// false if a pivot is not positive.
// Otherwise pn = |y| and qn2 = y^T (T + lam I)^-1 y (phi'(lam) = qn2 / pn^3 for
// phi = 1/|y| - 1/delta).  All lanes run the same instruction stream on their own lam, so a pass
// costs one evaluation's float64 instructions for 32 multipliers.
template <class SM>
__device__ inline bool tr_eval_lane(const SM& S, double (*PL)[32], double (*PR)[32], double (*PY)[32], int lane,
                                    double lam, double& pn, double& qn2) {
  double Dp = S.d[0] + lam;
  bool pd = Dp > 0.0;
  double r = tr_rcp(Dp);
  double w = -S.gh[0];
  PR[0][lane] = r;
  PY[0][lane] = w;
  for (int i = 1; i < TR_N; ++i) {
    const double l = S.off[i] * r;
    Dp = fma(-S.o2[i], r, S.d[i] + lam);
    pd = pd && Dp > 0.0;
    r = tr_rcp(Dp);
    w = fma(-l, w, -S.gh[i]);
    PL[i][lane] = l;
    PR[i][lane] = r;
    PY[i][lane] = w;
  }
  // (finished whatever the pivots' signs, so the warp stays converged; the caller masks by pd)
  double y = PY[TR_N - 1][lane] * PR[TR_N - 1][lane];
  PY[TR_N - 1][lane] = y;
  double p2 = y * y;
  for (int i = TR_N - 2; i >= 0; --i) {
    y = fma(-PL[i + 1][lane], y, PY[i][lane] * PR[i][lane]);
    PY[i][lane] = y;
    p2 = fma(y, y, p2);
  }
  double z = PY[0][lane], q2 = z * z * PR[0][lane];
  for (int i = 1; i < TR_N; ++i) {
    z = fma(-PL[i][lane], z, PY[i][lane]);
    q2 = fma(z * z, PR[i][lane], q2);
  }
  pn = sqrt(p2);
  qn2 = q2;
  return pd;
}

__device__ inline double tr_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double tr_warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Copies lane src's y into S.y (lanes < 27 in parallel).
__device__ inline void tr_take_y(TrSmem& S, int lane, int src) {
  __syncwarp();
  if (lane < TR_N) S.y[lane] = S.PY[lane][src];
  __syncwarp();
}

// Root of phi(lambda) = 1/|y(lambda)| - 1/delta over [lo, hi] (lo <= lambda*, phi(hi) >= 0), or
// lambda* = 0 when T is positive definite and |T^-1 gh| <= delta.  Each pass evaluates 32
// multipliers: a geometric grid over the bracket, refined around the Newton point of the
// largest evaluated multiplier on the left (phi < 0; phi is concave and increasing, so Newton
// from the left stays left).  Non-positive-definite points lie left of -lambda_min <= lambda*.
// spec bounds |eigenvalues of T| (Gershgorin): the bracket counts as closed once it is narrower
// than 4 ulps of max(|lambda|, spec).  hint (> 0, or negative for none): the multiplier of this
// source's previous subproblem; the root moves little from one Newton iteration to the next, so
// the first pass puts its points on a geometric grid around the hint (factors 2^-7.75 .. 2^7.75)
// instead of across the whole bracket.  On return S.y holds the step in the T basis and lam_out
// its multiplier; returns 1 for the hard case (the bracket closes on the pole with phi > 0 to its
// right), in which S.y is not set.
__device__ inline int tr_lambda_parallel(TrSmem& S, int lane, double lo, double hi, double delta, bool try_zero,
                                         double spec, double hint, double& lam_out) {
  constexpr double TOL = 1e-10;
  double L = lo, H = hi;            // L <= lambda* <= H
  bool have_h = false;              // S.y holds the point H (phi(H) >= 0)
  double lamN = -1.0;               // Newton point from the best left evaluation (< 0: none)
  double lamS = -1.0;               // secant point through the best left point and H (< 0: none)
  double lamL = -INFINITY, phiL = 0.0, dphiL = 1.0;   // largest left multiplier with phi < 0: phi, phi'
  double phiH = 0.0;                // phi at H, once evaluated
  // Lane offsets.  Without a Newton point: lanes 1-15 geometric from L (2^-45 .. 2^-3 of the
  // bracket, for a root or pole just above L), lanes 16-31 uniform (1/17 .. 16/17, so the bracket
  // shrinks at least 17-fold).  With one but no secant point: lane 0 at it, lanes 1-15 above and
  // 16-31 below at 2^-3 .. 2^-48 of the distance to the bracket's ends.  With both: phi concave,
  // so the Newton point from the left lies below the root and the secant point through a left
  // point and a right one above it; lanes 0 and 1 at the two, lanes 2-23 evenly between them
  // (the bracket shrinks at least 23-fold), lanes 24-27 above the secant point and 28-31 below
  // the Newton point at 2^-4 .. 2^-16 of the distance to the bracket's ends (in case rounding
  // has moved either across the root).
  const double gfac = lane < 16 ? ldexp(1.0, -3 * (16 - lane)) : (double)(lane - 15) / 17.0;
  const double nfac = ldexp(1.0, -3 * ((lane & 15) + 1));
  const double ufac = (double)(lane - 1) / 23.0;
  const double afac = ldexp(1.0, -4 * ((lane & 3) + 1));
  const double hfac = exp2(0.5 * (double)(lane - 16) + 0.25);   // 2^-7.75 .. 2^7.75 around the hint
  double lamH = H;                  // multiplier of the point H
  for (int pass = 0; pass < 16; ++pass) {
    // ---- this lane's multiplier
    double lam;
    const double span = H - L;
    if (pass > 0 && lamN > L && lamN < H && lamS > lamN && lamS <= H)
      lam = lane == 0   ? lamN
            : lane == 1 ? lamS
            : lane < 24 ? lamN + (lamS - lamN) * ufac
            : lane < 28 ? lamS + (H - lamS) * afac
                        : lamN - (lamN - L) * afac;
    else if (pass > 0 && lamN > L && lamN < H)
      lam = lane == 0 ? lamN : (lane < 16 ? lamN + (H - lamN) * nfac : lamN - (lamN - L) * nfac);
    else
      lam = lane == 0 ? ((pass == 0 && try_zero) ? 0.0 : L + 0.5 * span) : L + span * gfac;
    if (pass == 0 && hint > L && hint < H && lane > 0) {
      const double lh = hint * hfac;
      if (lh > L && lh < H) lam = lh;   // else the lane keeps its bracket point
    }
    __syncwarp();   // (lane choices are selects; the evaluation below must issue once, converged)
    double pn = 0.0, qn2 = 0.0;
    const bool pd = tr_eval_lane(S, S.PL, S.PR, S.PY, lane, lam, pn, qn2);
    // ---- interior solution
    if (pass == 0 && try_zero) {
      const bool interior = __shfl_sync(0xffffffffu, (int)(pd && pn <= delta), 0) != 0;
      if (interior) {
        tr_take_y(S, lane, 0);
        lam_out = 0.0;
        return 0;
      }
    }
    // ---- converged lane?
    const double err = pd ? fabs(pn - delta) : INFINITY;
    const double best = tr_warp_min(err);
    if (best <= TOL * delta) {
      const unsigned m = __ballot_sync(0xffffffffu, err == best);
      tr_take_y(S, lane, __ffs(m) - 1);
      lam_out = __shfl_sync(0xffffffffu, lam, __ffs(m) - 1);
      return 0;
    }
    // ---- new bracket
    const bool right = pd && pn <= delta;
    const double newL = tr_warp_max(right ? -INFINITY : lam);
    const double newH = tr_warp_min(right ? lam : INFINITY);
    if (newH < H) {
      const unsigned m = __ballot_sync(0xffffffffu, right && lam == newH);
      tr_take_y(S, lane, __ffs(m) - 1);
      H = newH;
      lamH = newH;
      phiH = tr_rcp(__shfl_sync(0xffffffffu, pn, __ffs(m) - 1)) - tr_rcp(delta);
      have_h = true;
    }
    L = fmax(L, newL);
    // ---- Newton point from the largest left evaluation with phi < 0 (phi' = q^2 / |p|^3)
    const bool lft = pd && pn > delta;
    const double lbest = tr_warp_max(lft ? lam : -INFINITY);
    if (lbest > lamL) {
      const unsigned m = __ballot_sync(0xffffffffu, lft && lam == lbest);
      const int src = __ffs(m) - 1;
      const double pnb = __shfl_sync(0xffffffffu, pn, src), qb = __shfl_sync(0xffffffffu, qn2, src);
      lamL = lbest;
      phiL = tr_rcp(pnb) - tr_rcp(delta);
      dphiL = qb * tr_rcp(pnb * pnb * pnb);
    }
    lamN = lamL > -INFINITY ? lamL - phiL * tr_rcp(dphiL) : -1.0;
    // ---- secant point through (lamL, phiL < 0) and (H, phiH >= 0)
    lamS = have_h && lamL > -INFINITY && phiH > phiL ? lamL + (H - lamL) * (-phiL * tr_rcp(phiH - phiL)) : -1.0;
    // ---- bracket closed: no multiplier left between L and H that T + lambda I could tell apart
    //      (its entries carry rounding of a few ulps of the spectrum's scale `spec`, so a bracket
    //      that narrow around a root next to the pole is resolved as far as float64 allows)
    if (H - L <= 4.0 * DBL_EPSILON * fmax(fabs(H), spec)) {
      if (!have_h) return 1;
      // phi(H) >= 0 with H next to L: the root, unless |y| jumps across delta within the last
      // ulps of lambda -- the pole, where g's component along the eigenvector of lambda_min is
      // too small to resolve (the hard case, numerically).  A positive definite point with
      // |y| > delta (lamL) rules the hard case out: there g's component along that eigenvector
      // lifts |y| above delta right of the pole, so the root lies in [lamL, H] and y(H) stands.
      lam_out = lamH;
      return lamL == -INFINITY && tr_norm(S.y) < delta * (1.0 - 1e-6) ? 1 : 0;
    }
  }
  lam_out = lamH;
  return have_h ? 0 : 1;
}

// Loads B (scaled by bsign) into S.A, lane-parallel and coalesced.
__device__ inline void tr_load(TrSmem& S, const double* __restrict__ B, double bsign) {
  for (int i = threadIdx.x & 31; i < TR_N * TR_N; i += 32) S.A[i] = bsign * B[i];
  __syncwarp();
}

// Newton step p = -B^-1 g by L D L^T of S.A in place (lane i owns row i; the rows are kept full,
// so row k holds the current a_kj when step k needs it).  Returns false if a pivot is not
// positive; otherwise lane i < 27 holds p_i.
__device__ inline bool tr_newton_step(TrSmem& S, double gi, double& p_i) {
  const int lane = threadIdx.x & 31;
  const bool row = lane < TR_N;
  double* ar = S.A + lane * TR_LD;
  for (int k = 0; k < TR_N; ++k) {
    const double dk = S.A[k * TR_LD + k];
    if (!(dk > 0.0)) return false;   // same value in every lane
    const double r = tr_rcp(dk);
    const bool act = row && lane > k;
    const double li = act ? ar[k] * r : 0.0;
    __syncwarp();
    if (act) {
      for (int j = k + 1; j < TR_N; ++j) ar[j] = fma(-li, S.A[k * TR_LD + j], ar[j]);
      ar[k] = li;   // L below the diagonal
    }
    if (lane == k) S.D[k] = r;
    __syncwarp();
  }
  // L y = -g (column by column), y *= D^-1, L^T x = y (from the bottom)
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

// Solves the subproblem for B (device, row-major 27 x 27, times bsign) and the gradient g_i held by
// lane i (0 for lanes >= 27).  On return lane i < 27 holds p_i; pred = -(g.p + p.B.p/2); hard =
// hard case taken.  try_newton: attempt the Newton step first.  cache_in (or null): the
// tridiagonal form of this same B and g, stored by an earlier call, replaces the reduction;
// cache_out (or null): where to store the reduction when one is made.  lam_hint: the multiplier
// of this source's previous subproblem (negative: none); lam_out: this one's (0 for an interior
// step, negative after the hard case).  Returns true when the reduction was made and stored.
__device__ inline bool tr_solve_warp(TrSmem& S, const double* __restrict__ Bsrc, double bsign, double gi,
                                     double delta, bool try_newton, const double* __restrict__ cache_in,
                                     double* __restrict__ cache_out, double lam_hint, double& lam_out,
                                     double& p_i, double& pred, int& hard) {
  const int lane = threadIdx.x & 31;
  const int n = TR_N;
  const bool row = lane < n;
  const double gnorm = sqrt(tr_warp_sum(gi * gi));
  bool stored = false;
  if (cache_in) {
    // layout: A [27][27], d, off, o2, gh, beta [27] each
    for (int i = lane; i < TR_N * TR_N; i += 32) S.A[(i / TR_N) * TR_LD + (i % TR_N)] = cache_in[i];
    if (row) {
      S.d[lane] = cache_in[TR_N * TR_N + lane];
      S.off[lane] = cache_in[TR_N * TR_N + TR_N + lane];
      S.o2[lane] = cache_in[TR_N * TR_N + 2 * TR_N + lane];
      S.gh[lane] = cache_in[TR_N * TR_N + 3 * TR_N + lane];
      S.beta[lane] = cache_in[TR_N * TR_N + 4 * TR_N + lane];
    }
    __syncwarp();
  } else {
  if (try_newton) {
    tr_load(S, Bsrc, bsign);
    double pn;
    if (tr_newton_step(S, gi, pn)) {
      const double pp = tr_warp_sum(pn * pn);
      if (sqrt(pp) <= delta) {
        p_i = pn;
        pred = -0.5 * tr_warp_sum(gi * pn);   // -(g.p + p.B.p/2) with B p = -g
        hard = 0;
        lam_out = 0.0;
        return false;
      }
    }
  }
  tr_load(S, Bsrc, bsign);
  // ---- Householder tridiagonalisation, lane i owns row i (in shared memory); gh = Q^T g is
  //      reflected along, its reductions paired with the reduction's own
  double gh = row ? gi : 0.0;
  for (int k = 0; k < n - 2; ++k) {
    const double xi = lane > k && row ? S.A[lane * TR_LD + k] : 0.0;
    const double s2 = tr_warp_sum(xi * xi);
    const double x0 = S.A[(k + 1) * TR_LD + k];
    if (s2 == 0.0) {
      if (lane == 0) {
        S.beta[k] = 0.0;
        S.off[k + 1] = 0.0;
      }
      __syncwarp();
      continue;
    }
    const double alpha = -copysign(sqrt(s2), x0);
    const double vi = lane == k + 1 ? x0 - alpha : xi;
    const double beta = tr_rcp(s2 - alpha * x0);   // 2 / v.v with v.v = 2 (s2 - alpha x0)
    S.v[lane] = vi;
    __syncwarp();
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    if (lane > k && row) {
      const double* ar = S.A + lane * TR_LD;
      int j = k + 1;
      for (; j + 3 < n; j += 4) {
        u[0] = fma(ar[j], S.v[j], u[0]);
        u[1] = fma(ar[j + 1], S.v[j + 1], u[1]);
        u[2] = fma(ar[j + 2], S.v[j + 2], u[2]);
        u[3] = fma(ar[j + 3], S.v[j + 3], u[3]);
      }
      for (; j < n; ++j) u[0] = fma(ar[j], S.v[j], u[0]);
    }
    const double pi = beta * ((u[0] + u[1]) + (u[2] + u[3]));
    double vp = vi * pi, vg = vi * gh;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vp += __shfl_xor_sync(0xffffffffu, vp, o);
      vg += __shfl_xor_sync(0xffffffffu, vg, o);
    }
    const double K = 0.5 * beta * vp;
    const double wi = pi - K * vi;
    gh = fma(-beta * vg, vi, gh);
    S.w[lane] = wi;
    __syncwarp();
    if (lane > k && row) {
      double* ar = S.A + lane * TR_LD;
      for (int j = k + 1; j < n; ++j) ar[j] = fma(-vi, S.w[j], fma(-wi, S.v[j], ar[j]));
      ar[k] = vi;   // keep the reflection vector
    }
    if (lane == 0) {
      S.beta[k] = beta;
      S.off[k + 1] = alpha;
    }
    __syncwarp();
  }
  if (row) {
    S.d[lane] = S.A[lane * TR_LD + lane];
    S.gh[lane] = gh;
  }
  if (lane == 0) {
    S.off[n - 1] = S.A[(n - 1) * TR_LD + n - 2];
    S.off[0] = 0.0;
  }
  __syncwarp();
  if (row) S.o2[lane] = S.off[lane] * S.off[lane];
  __syncwarp();
  if (cache_out) {
    for (int i = lane; i < TR_N * TR_N; i += 32) cache_out[i] = S.A[(i / TR_N) * TR_LD + (i % TR_N)];
    if (row) {
      cache_out[TR_N * TR_N + lane] = S.d[lane];
      cache_out[TR_N * TR_N + TR_N + lane] = S.off[lane];
      cache_out[TR_N * TR_N + 2 * TR_N + lane] = S.o2[lane];
      cache_out[TR_N * TR_N + 3 * TR_N + lane] = S.gh[lane];
      cache_out[TR_N * TR_N + 4 * TR_N + lane] = S.beta[lane];
    }
    stored = true;
  }
  }   // reduction

  // ---- multiplier: lambda* >= max(0, -lambda_min) >= max(0, -min_i d_i); at
  //      hi = |g| / delta - a (a <= lambda_min, Gershgorin) |p(hi)| <= |g| / (hi + lambda_min) <= delta
  // (lane-parallel, with selects: a lane-divergent branch here can leave the warp split through
  // the multiplier search)
  const int li = row ? lane : 0, ln = lane + 1 < n ? lane + 1 : 0;
  const double di = S.d[li], oi = fabs(S.off[li]), on = lane + 1 < n ? fabs(S.off[ln]) : 0.0;
  double a = tr_warp_min(row ? di - (oi + on) : INFINITY);
  const double dmin = tr_warp_min(row ? di : INFINITY);
  const double dmax = tr_warp_max(row ? fabs(di) : 0.0);
  const double omax = tr_warp_max(row ? oi : 0.0);
  const double spec = dmax + 2.0 * omax;   // >= |eigenvalues of T| (Gershgorin)
  const double scale = fmax(1.0, spec);
  const double lo = fmax(0.0, -dmin);
  const double hi = fmax(lo, gnorm / delta - a) * (1.0 + 1e-12) + 1e-300;
  if (lane == 0) S.flag[2] = 0;
  __syncwarp();
  lam_out = -1.0;
  if (tr_lambda_parallel(S, lane, lo, hi, delta, lo == 0.0, spec, lam_hint, lam_out)) {
    lam_out = -1.0;
    // hard case: g has (almost) no component along the eigenvector z of lambda_min.  lambda_min
    // from a float32 Sturm bracket refined by inverse iteration (lane 0), then
    // p = y(-lambda_min) + tau z with |p| = delta.
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
        // the sign that lowers the model: tau z.g < 0 (either sign when z.g = 0 exactly)
        const double tau = copysign(sqrt(fmax(delta * delta - yn * yn, 0.0)), -zg);
        for (int i = 0; i < n; ++i) S.y[i] += tau * S.z[i];
      }
      S.flag[2] = 1;
    }
    __syncwarp();
  } else if (lane == 0) {
    // next to the pole the last ulp of lambda can move |y| by ~1e-8 relative; keep the step feasible
    const double yn = tr_norm(S.y);
    if (yn > delta)
      for (int i = 0; i < n; ++i) S.y[i] *= delta / yn;
  }
  __syncwarp();
  hard = S.flag[2];
  // ---- p = Q y, and the model value through T: g.p = gh.y, p.B.p = y.T.y
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
  __syncwarp();
  return stored;
}

}  // namespace celeste
