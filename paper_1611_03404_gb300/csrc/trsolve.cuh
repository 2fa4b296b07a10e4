// Trust-region subproblem in float64, one warp per problem:
//     minimise  g.p + p.B.p / 2   subject to  |p| <= delta      (B symmetric 27 x 27)
// More-Sorensen characterisation (Nocedal & Wright, Sec. 4.3): p = -(B + lambda I)^-1 g with
// lambda >= max(0, -lambda_min(B)), lambda (|p| - delta) = 0, plus the "hard case" where g has no
// component along the eigenvector of lambda_min.
//
// GB300 float64 throughput is low, so instead of a full eigendecomposition the matrix is reduced
// once to tridiagonal form T = Q^T B Q by Householder reflections (lane-parallel), after which
// every solve with T + lambda I is an O(n) LDL^T recurrence:
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
constexpr int TR_LD = NP + 1;     // padded row length of the matrix in shared memory

struct TrSmem {
  double A[TR_N * TR_LD];         // B on entry; Householder vectors below the diagonal afterwards
  double v[32], w[32];            // per-step temporaries
  double d[TR_N], off[TR_N];      // T: diagonal, off[i] = T[i][i-1]
  double beta[TR_N];              // reflection coefficients
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
    const double l = S.off[i] * r;
    Dp = S.d[i] + lambda - l * S.off[i];
    pd = pd && Dp > 0.0;
    r = 1.0 / Dp;
    S.L[i] = l;
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
  double s = 0.0;
  for (int i = 0; i < TR_N; ++i) s += x[i] * x[i];
  return sqrt(s);
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

// Solves the subproblem for the matrix in S.A and the gradient g_i held by lane i (0 for lanes
// >= 27).  On return lane i < 27 holds p_i; pred = -(g.p + p.B.p/2); hard = hard case taken.
__device__ inline void tr_solve_warp(TrSmem& S, double gi, double delta, double& p_i, double& pred, int& hard) {
  const int lane = threadIdx.x & 31;
  const int n = TR_N;
  // ---- Householder tridiagonalisation, lane i owns row i
  for (int k = 0; k < n - 2; ++k) {
    const double xi = lane > k && lane < n ? S.A[lane * TR_LD + k] : 0.0;
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
    if (lane > k && lane < n) S.v[lane] = vi;
    __syncwarp();
    double pi = 0.0;
    if (lane > k && lane < n) {
      for (int j = k + 1; j < n; ++j) pi += S.A[lane * TR_LD + j] * S.v[j];
      pi *= beta;
    }
    const double K = 0.5 * beta * tr_warp_sum(lane > k && lane < n ? vi * pi : 0.0);
    const double wi = pi - K * vi;
    if (lane > k && lane < n) S.w[lane] = wi;
    __syncwarp();
    if (lane > k && lane < n) {
      for (int j = k + 1; j < n; ++j) S.A[lane * TR_LD + j] -= vi * S.w[j] + wi * S.v[j];
      S.A[lane * TR_LD + k] = vi;   // keep the reflection vector
    }
    if (lane == 0) {
      S.beta[k] = beta;
      S.off[k + 1] = alpha;
    }
    __syncwarp();
  }
  if (lane < n) S.d[lane] = S.A[lane * TR_LD + lane];
  if (lane == 0) {
    S.off[n - 1] = S.A[(n - 1) * TR_LD + n - 2];
    S.off[0] = 0.0;
  }
  // ---- gh = Q^T g
  double gh = lane < n ? gi : 0.0;
  for (int k = 0; k < n - 2; ++k) {
    const double vk = lane > k && lane < n ? S.A[lane * TR_LD + k] : 0.0;
    const double t = tr_warp_sum(vk * gh);
    gh -= S.beta[k] * vk * t;
  }
  if (lane < n) S.gh[lane] = gh;
  const double gnorm = sqrt(tr_warp_sum(gi * gi));
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
          const double nz = tr_norm(S.z);
          for (int i = 0; i < n; ++i) S.z[i] /= nz;
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
  double yi = lane < n ? S.y[lane] : 0.0;
  double Ty = 0.0;
  if (lane < n) {
    Ty = S.d[lane] * yi + (lane > 0 ? S.off[lane] * S.y[lane - 1] : 0.0) +
         (lane + 1 < n ? S.off[lane + 1] * S.y[lane + 1] : 0.0);
  }
  const double gy = tr_warp_sum(lane < n ? S.gh[lane] * yi : 0.0);
  const double yTy = tr_warp_sum(yi * Ty);
  pred = -(gy + 0.5 * yTy);
  for (int k = n - 3; k >= 0; --k) {
    const double vk = lane > k && lane < n ? S.A[lane * TR_LD + k] : 0.0;
    const double t = tr_warp_sum(vk * yi);
    yi -= S.beta[k] * vk * t;
  }
  p_i = yi;
  __syncwarp();
}

}  // namespace celeste
