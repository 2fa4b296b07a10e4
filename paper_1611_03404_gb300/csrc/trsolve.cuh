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
//   * positive definiteness of B  <=>  all LDL^T pivots of T positive (Sylvester);
//   * lambda_min(T): a float32 Sturm-sequence multisection bracket (each lane tests its own shift),
//     refined in float64 by inverse iteration and the Rayleigh quotient;
//   * |p(lambda)| = delta by the safeguarded Newton iteration on 1/|p| - 1/delta
//     (Nocedal & Wright Algorithm 4.3), phi'(lambda) = |w|^2/|p|^3, L D w = p;
//   * hard case: eigenvector of lambda_min by inverse iteration on T.
// The step is mapped back with the reflections, p = Q y.
#pragma once

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
};

__device__ inline double tr_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// LDL^T of T + lambda I into S.D (reciprocal pivots), S.L; returns false if a pivot is not positive.
__device__ inline bool tr_ldl(TrSmem& S, double lambda) {
  double Dp = S.d[0] + lambda;
  bool pd = Dp > 0.0;
  double r = 1.0 / Dp;
  S.D[0] = r;
  for (int i = 1; i < TR_N; ++i) {
    S.L[i] = S.off[i] * r;                 // off the pivot chain
    Dp = fma(-S.o2[i], r, S.d[i] + lambda);
    pd = pd && Dp > 0.0;
    r = 1.0 / Dp;
    S.D[i] = r;
  }
  return pd;
}

// Solve (L D L^T) x = b (b may alias x).
__device__ inline void tr_ldl_solve(const TrSmem& S, const double* b, double* x) {
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

// Number of eigenvalues of T below x (negative pivots of T - x I).
__device__ inline int tr_sturm(const TrSmem& S, double x) {
  double q = S.d[0] - x;
  int c = q < 0.0;
  for (int i = 1; i < TR_N; ++i) {
    if (q == 0.0) q = -1e-300;
    q = S.d[i] - x - S.off[i] * S.off[i] / q;
    c += q < 0.0;
  }
  return c;
}

// Float32 Sturm count (only used to bracket lambda_min; the bracket is widened afterwards).
__device__ inline int tr_sturm_f(const TrSmem& S, float x) {
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

// Lane 0 only: float32 Newton iterations on phi(lambda) = 1/|y| - 1/delta to a starting point for
// the float64 iteration (|y| within ~1e-5 of delta).  The float32 phi can have the wrong sign close
// to the pole, so this phase keeps its own bracket and leaves the float64 safeguards untouched.
__device__ inline double tr_newton_lambda_f32(const TrSmem& S, double lambda, double lo, double hi, double delta) {
  float D[TR_N], L[TR_N], y[TR_N];
  for (int it = 0; it < 30; ++it) {
    const float lam = (float)lambda;
    float Dp = (float)S.d[0] + lam;
    bool pd = Dp > 0.f;
    D[0] = 1.f / Dp;
    for (int i = 1; i < TR_N; ++i) {
      const float o = (float)S.off[i];
      L[i] = o * D[i - 1];
      Dp = (float)S.d[i] + lam - L[i] * o;
      pd = pd && Dp > 0.f;
      D[i] = 1.f / Dp;
    }
    if (!pd) {
      lo = lambda;
      lambda = 0.5 * (lo + hi);
      continue;
    }
    y[0] = -(float)S.gh[0];
    for (int i = 1; i < TR_N; ++i) y[i] = -(float)S.gh[i] - L[i] * y[i - 1];
    for (int i = 0; i < TR_N; ++i) y[i] *= D[i];
    for (int i = TR_N - 2; i >= 0; --i) y[i] -= L[i + 1] * y[i + 1];
    float pn2 = 0.f;
    for (int i = 0; i < TR_N; ++i) pn2 += y[i] * y[i];
    const float pn = sqrtf(pn2);
    float wv = y[0], qn2 = wv * wv * D[0];
    for (int i = 1; i < TR_N; ++i) {
      wv = y[i] - L[i] * wv;
      qn2 += wv * wv * D[i];
    }
    if (!(pn > 0.f) || !isfinite(pn)) break;
    if (fabsf(pn - (float)delta) <= 1e-5f * (float)delta) break;
    const double phi = 1.0 / pn - 1.0 / delta;
    if (phi > 0)
      hi = lambda;
    else
      lo = lambda;
    double ln = lambda - phi / ((double)qn2 / ((double)pn * pn * pn));
    if (!(lo < ln && ln < hi)) ln = 0.5 * (lo + hi);
    if (ln == lambda) break;
    lambda = ln;
  }
  return lambda;
}

// Lane 0 only: safeguarded Newton on phi(lambda) = 1/|y| - 1/delta over (lo, hi); result in S.y.
__device__ inline void tr_newton_lambda(TrSmem& S, double lambda, double lo, double hi, double delta) {
  double mg[TR_N];
  for (int i = 0; i < TR_N; ++i) mg[i] = -S.gh[i];
  bool have = false;
  // float32 estimate, checked in float64: on the near (phi < 0) side it is the starting point of the
  // monotone float64 Newton iteration; beyond the root or below the pole it only tightens the
  // bracket and the iteration starts from the given point, where phi < 0.
  const double lam_f = tr_newton_lambda_f32(S, lambda, lo, hi, delta);
  if (lam_f != lambda && lam_f > lo && lam_f < hi) {
    if (tr_ldl(S, lam_f)) {
      tr_ldl_solve(S, mg, S.y);
      if (tr_norm(S.y) > delta)
        lambda = lam_f;
      else
        hi = lam_f;
    } else {
      lo = lam_f;
      if (lambda <= lo) lambda = 0.5 * (lo + hi);
    }
  }
  for (int it = 0; it < 60; ++it) {
    if (!tr_ldl(S, lambda)) {   // below lambda_min: move up by bisection
      lo = lambda;
      lambda = 0.5 * (lo + hi);
      continue;
    }
    tr_ldl_solve(S, mg, S.y);
    have = true;
    const double pn = tr_norm(S.y);
    double wv = S.y[0], qn2 = wv * wv * S.D[0];
    for (int i = 1; i < TR_N; ++i) {
      wv = S.y[i] - S.L[i] * wv;
      qn2 += wv * wv * S.D[i];
    }
    if (fabs(pn - delta) <= 1e-10 * delta) break;
    const double phi = 1.0 / pn - 1.0 / delta;
    if (phi > 0)
      hi = lambda;
    else
      lo = lambda;
    double ln = lambda - phi / (qn2 / (pn * pn * pn));
    if (!(lo < ln && ln < hi)) ln = 0.5 * (lo + hi);
    if (ln == lambda) break;
    lambda = ln;
  }
  if (!have || !tr_ldl(S, lambda)) {   // fall back to the upper bracket end, always admissible
    tr_ldl(S, hi);
    tr_ldl_solve(S, mg, S.y);
  }
  // Near the pole lambda = -lambda_min the last ulp of lambda can move |y| by ~1e-8 relative;
  // keep the step feasible.
  const double yn = tr_norm(S.y);
  if (yn > delta) {
    const double r = delta / yn;
    for (int i = 0; i < TR_N; ++i) S.y[i] *= r;
  }
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
    const double r = 1.0 / dk;
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
// hard case taken.  try_newton: attempt the Newton step first.
__device__ inline void tr_solve_warp(TrSmem& S, const double* __restrict__ Bsrc, double bsign, double gi, double delta,
                                     bool try_newton, double& p_i, double& pred, int& hard) {
  const int lane = threadIdx.x & 31;
  const int n = TR_N;
  const bool row = lane < n;
  const double gnorm = sqrt(tr_warp_sum(gi * gi));
  if (try_newton) {
    tr_load(S, Bsrc, bsign);
    double pn;
    if (tr_newton_step(S, gi, pn)) {
      const double pp = tr_warp_sum(pn * pn);
      if (sqrt(pp) <= delta) {
        p_i = pn;
        pred = -0.5 * tr_warp_sum(gi * pn);   // -(g.p + p.B.p/2) with B p = -g
        hard = 0;
        return;
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
    const double beta = 1.0 / (s2 - alpha * x0);   // 2 / v.v with v.v = 2 (s2 - alpha x0)
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

  // ---- positive definite and interior?
  if (lane == 0) {
    S.flag[0] = tr_ldl(S, 0.0);
    S.flag[1] = 0;   // done
    S.flag[2] = 0;   // hard case
    if (S.flag[0]) {
      for (int i = 0; i < n; ++i) S.y[i] = -S.gh[i];
      tr_ldl_solve(S, S.y, S.y);
      if (tr_norm(S.y) <= delta) S.flag[1] = 1;
    }
  }
  __syncwarp();
  if (!S.flag[1]) {
    double lo = 0.0, lam0 = 0.0, scale = 1.0;
    if (!S.flag[0]) {
      // lambda_min of T by multisection of its Gershgorin interval (one shift per lane)
      double a = INFINITY, b = -INFINITY, dmax = 0.0, omax = 0.0;
      for (int i = 0; i < n; ++i) {
        const double r = fabs(S.off[i]) + (i + 1 < n ? fabs(S.off[i + 1]) : 0.0);
        a = fmin(a, S.d[i] - r);
        b = fmax(b, S.d[i] + r);
        dmax = fmax(dmax, fabs(S.d[i]));
        omax = fmax(omax, fabs(S.off[i]));
      }
      scale = fmax(1.0, dmax + 2.0 * omax);
      // Bracket [a, b] of lambda_min by Sturm multisection in float32 (one shift per lane), widened by
      // 1e-5 of the spectrum scale to cover the rounding; it supplies the shift of the float64
      // inverse iteration below.
      {
        float fa = (float)a, fb = (float)b;
        for (int it = 0; it < 6; ++it) {
          const float x = fa + (fb - fa) * (float)(lane + 1) / 33.f;
          const unsigned m = __ballot_sync(0xffffffffu, tr_sturm_f(S, x) >= 1);
          const int f = m ? __ffs(m) - 1 : 32;
          const float na = f > 0 ? fa + (fb - fa) * (float)f / 33.f : fa;
          const float nb = f < 32 ? fa + (fb - fa) * (float)(f + 1) / 33.f : fb;
          fa = na;
          fb = nb;
          if (fb - fa <= 1e-6f * (float)scale) break;
        }
        a = fmax(a, (double)fa - 1e-5 * scale);
        b = fmin(b, (double)fb + 1e-5 * scale);
      }
      if (lane == 0) {
        // float64 refinement: eigenvector z of lambda_min by inverse iteration with a shift below the
        // bracket, lambda_min from its Rayleigh quotient (>= lambda_min, so -lambda_R is a lower bound
        // of the admissible lambdas).  The hard case needs g to have (almost) no component on z.
        tr_ldl(S, -(a - 1e-8 * scale));
        for (int i = 0; i < n; ++i) S.z[i] = 1.0;
        for (int r = 0; r < 4; ++r) {
          tr_ldl_solve(S, S.z, S.z);
          const double rz = 1.0 / tr_norm(S.z);
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
        lmin = fmin(lmin, b);
        S.sc[0] = fmax(0.0, -lmin);
        S.sc[1] = fmax(0.0, -lmin) + 1e-12 * scale;
        if (fabs(zg) <= 1e-12 * fmax(gnorm, 1e-300)) {
          tr_ldl(S, fmax(0.0, -lmin) + 1e-9 * scale);
          for (int i = 0; i < n; ++i) S.y[i] = -S.gh[i];
          tr_ldl_solve(S, S.y, S.y);
          double zy = 0.0;
          for (int i = 0; i < n; ++i) zy += S.z[i] * S.y[i];
          for (int i = 0; i < n; ++i) S.y[i] -= zy * S.z[i];
          const double yn = tr_norm(S.y);
          if (yn <= delta) {
            const double tau = sqrt(fmax(delta * delta - yn * yn, 0.0));
            for (int i = 0; i < n; ++i) S.y[i] += tau * S.z[i];
            S.flag[1] = 1;
            S.flag[2] = 1;
          }
        }
      }
      __syncwarp();
      lo = S.sc[0];
      lam0 = S.sc[1];
    }
    // upper end: |p(lambda)| <= |g| / (lambda + lambda_min) <= delta there (lam0 >= -lambda_min up
    // to the Rayleigh-quotient error, covered by the + 1)
    if (!S.flag[1] && lane == 0) tr_newton_lambda(S, lam0, lo, lam0 + gnorm / delta + 1.0, delta);
    __syncwarp();
  }
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
}

}  // namespace celeste
