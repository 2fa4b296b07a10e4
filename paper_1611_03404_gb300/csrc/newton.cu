// Batched trust-region Newton over per-source subproblems (paper, Sec. "Variational Inference":
// each source optimised with its neighbours fixed, Newton's method with a trust region, using
// the exact gradient and dense Hessian; machine tolerance within 50 iterations).
//
// The subproblem min g.p + p.B.p/2 s.t. |p| <= delta (f = -ELBO, g = -grad, B = -Hessian) is
// solved in float64 the More-Sorensen way (Nocedal & Wright, Sec. 4.3): eigendecomposition of B
// (cyclic Jacobi, one warp per source), then a safeguarded Newton iteration on
// 1/|p(lambda)| - 1/delta, with the hard case handled explicitly.  The outer iteration follows
// Nocedal & Wright Algorithm 4.1.
#include <cmath>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"

namespace celeste {

constexpr int TR_WARPS = 4;     // sources per CTA of the step kernel
constexpr int LD = NP + 1;      // padded leading dimension of the 27x27 matrices in shared memory

// Per-source integer state.
constexpr int ST_ACTIVE = 0, ST_ITERS = 1, ST_STATUS = 2, ST_BOUNDARY = 3;

struct NewtonDev {
  double* theta;        // [S][27] current iterate (caller memory)
  double* delta;        // [S] trust radius (caller memory)
  double* L;            // [S] ELBO at theta
  double* gL;           // [S][27] gradient of the ELBO at theta
  double* HL;           // [S][27][27] Hessian of the ELBO at theta
  double* trial;        // [S][27]
  double* pred;         // [S] predicted reduction of f = -ELBO
  double* Ltrial;       // [S]
  int* state;           // [S][4]
  int* count;           // [0]: active sources after the update
  int S;
  double ftol, gtol, delta0, delta_max, eta, delta_min;
};

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void newton_init_kernel(NewtonDev N, int* flags) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N.S) return;
  N.state[4 * s + ST_ACTIVE] = 1;
  N.state[4 * s + ST_ITERS] = 0;
  N.state[4 * s + ST_STATUS] = CELESTE_STATUS_MAX_ITER;
  N.state[4 * s + ST_BOUNDARY] = 0;
  if (!(N.delta[s] > 0.0)) N.delta[s] = N.delta0;
  flags[s] = FLAG_FULL;
}

// One warp per source: convergence tests, eigendecomposition, subproblem, trial point.
__global__ void __launch_bounds__(32 * TR_WARPS) tr_step_kernel(NewtonDev N, int* flags) {
  __shared__ double Ash[TR_WARPS][NP * LD];
  __shared__ double Vsh[TR_WARPS][NP * LD];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * TR_WARPS + warp;
  if (s >= N.S) return;
  int* st = N.state + 4 * s;
  if (!st[ST_ACTIVE]) {
    if (lane == 0) flags[s] = 0;
    return;
  }
  double* A = Ash[warp];
  double* V = Vsh[warp];
  const double* HL = N.HL + (size_t)s * NP * NP;
  const double* gL = N.gL + (size_t)s * NP;
  // f = -L, g = -gL, B = -HL
  double gk = lane < NP ? -gL[lane] : 0.0;
  bool finite = isfinite(N.L[s]) && isfinite(gk);
  for (int i = lane; i < NP * NP; i += 32) {
    const double b = -HL[i];
    finite = finite && isfinite(b);
    A[(i / NP) * LD + (i % NP)] = b;
    V[(i / NP) * LD + (i % NP)] = (i / NP == i % NP) ? 1.0 : 0.0;
  }
  finite = __all_sync(0xffffffffu, finite);
  if (!finite) {
    if (lane == 0) {
      st[ST_ACTIVE] = 0;
      st[ST_STATUS] = CELESTE_STATUS_NONFINITE;
      flags[s] = 0;
    }
    return;
  }
  const double gmax = warp_max(fabs(gk));
  if (gmax <= N.gtol) {
    if (lane == 0) {
      st[ST_ACTIVE] = 0;
      st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
      flags[s] = 0;
    }
    return;
  }
  __syncwarp();

  // ---- cyclic Jacobi: A <- J^T A J, V <- V J until the off-diagonal part is negligible
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dia = 0.0;
    if (lane < NP) {
      for (int j = 0; j < NP; ++j) {
        const double a = A[lane * LD + j];
        if (j == lane)
          dia += a * a;
        else
          off += a * a;
      }
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (off <= 1e-26 * dia || off == 0.0) break;
    for (int p = 0; p < NP - 1; ++p)
      for (int q = p + 1; q < NP; ++q) {
        const double apq = A[p * LD + q];
        if (apq == 0.0) continue;
        const double app = A[p * LD + p], aqq = A[q * LD + q];
        const double th = (aqq - app) / (2.0 * apq);
        double t;
        if (fabs(th) > 1e150)
          t = 0.5 / th;
        else
          t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
        __syncwarp();
        if (lane < NP) {
          const double akp = A[lane * LD + p], akq = A[lane * LD + q];
          A[lane * LD + p] = c * akp - sn * akq;
          A[lane * LD + q] = sn * akp + c * akq;
        }
        __syncwarp();
        if (lane < NP) {
          const double apk = A[p * LD + lane], aqk = A[q * LD + lane];
          A[p * LD + lane] = c * apk - sn * aqk;
          A[q * LD + lane] = sn * apk + c * aqk;
          const double vkp = V[lane * LD + p], vkq = V[lane * LD + q];
          V[lane * LD + p] = c * vkp - sn * vkq;
          V[lane * LD + q] = sn * vkp + c * vkq;
        }
        __syncwarp();
      }
  }
  __syncwarp();

  // ---- subproblem in the eigenbasis: lambda_i = A_ii, gamma_i = v_i . g
  const double lam = lane < NP ? A[lane * LD + lane] : INFINITY;
  double gam = 0.0;
  if (lane < NP)
    for (int k = 0; k < NP; ++k) gam += V[k * LD + lane] * (-gL[k]);
  const double delta = N.delta[s];
  const double gnorm = sqrt(warp_sum(gk * gk));
  double lmin = lam;
  int imin = lane;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ol = __shfl_xor_sync(0xffffffffu, lmin, o);
    const int oi = __shfl_xor_sync(0xffffffffu, imin, o);
    if (ol < lmin || (ol == lmin && oi < imin)) {
      lmin = ol;
      imin = oi;
    }
  }
  double coef = 0.0;   // p = sum_i coef_i v_i
  bool have = false;
  if (lmin > 0.0) {
    coef = lane < NP ? -gam / lam : 0.0;
    const double pn = sqrt(warp_sum(coef * coef));
    if (pn <= delta) have = true;
  }
  if (!have) {
    double lo = fmax(0.0, -lmin);
    const double lmaxabs = warp_max(lane < NP ? fabs(lam) : 0.0);
    const double scale = fmax(1.0, lmaxabs);
    const bool small = lane < NP && fabs(lam - lmin) <= 1e-12 * scale;
    const bool gsmall = !small || fabs(gam) <= 1e-12 * fmax(gnorm, 1e-300);
    if (__all_sync(0xffffffffu, gsmall)) {
      const double ch = (lane < NP && !small) ? -gam / (lam - lmin) : 0.0;
      const double phn2 = warp_sum(ch * ch);
      if (sqrt(phn2) <= delta) {
        const double tau = sqrt(fmax(delta * delta - phn2, 0.0));
        coef = ch + (lane == imin ? tau : 0.0);
        have = true;
      }
    }
    if (!have) {
      double hi = lo + gnorm / delta + 1.0;
      for (int it = 0; it < 2000; ++it) {
        const double d = lane < NP ? gam / (lam + hi) : 0.0;
        if (sqrt(warp_sum(d * d)) <= delta) break;
        hi = 2.0 * hi + 1.0;
      }
      double l = hi;
      for (int it = 0; it < 200; ++it) {
        const double dd = lam + l;
        const double r = lane < NP ? gam / dd : 0.0;
        const double pn = sqrt(warp_sum(r * r));
        const double qn2 = warp_sum(lane < NP ? gam * gam / (dd * dd * dd) : 0.0);
        const double phi = 1.0 / pn - 1.0 / delta;
        if (fabs(pn - delta) <= 1e-12 * delta) break;
        if (phi > 0)
          hi = l;
        else
          lo = l;
        double ln = l - phi / (qn2 / (pn * pn * pn));
        if (!(lo < ln && ln < hi)) ln = 0.5 * (lo + hi);
        if (ln == l) break;
        l = ln;
      }
      coef = lane < NP ? -gam / (lam + l) : 0.0;
    }
  }
  // p = V coef; row 0 of A (no longer needed: the eigenvalues are in registers) holds p
  double pk = 0.0;
  for (int i = 0; i < NP; ++i) {
    const double ci = __shfl_sync(0xffffffffu, coef, i);
    if (lane < NP) pk += V[lane * LD + i] * ci;
  }
  __syncwarp();
  if (lane < NP) A[lane] = pk;
  __syncwarp();
  double Bp = 0.0;
  if (lane < NP)
    for (int k = 0; k < NP; ++k) Bp += -HL[lane * NP + k] * A[k];
  const double gp = warp_sum(gk * pk), pBp = warp_sum(pk * Bp);
  const double pnorm = sqrt(warp_sum(pk * pk));
  if (lane < NP) N.trial[(size_t)s * NP + lane] = N.theta[(size_t)s * NP + lane] + pk;
  if (lane == 0) {
    N.pred[s] = -(gp + 0.5 * pBp);
    st[ST_ITERS] += 1;
    st[ST_BOUNDARY] = pnorm >= (1.0 - 1e-9) * delta;
    flags[s] = FLAG_VALUE;
  }
}

// Accept or reject the trial point and update the radius (Nocedal & Wright Alg. 4.1).
__global__ void tr_update_kernel(NewtonDev N, int* flags) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int active = 0;
  if (s < N.S) {
    int* st = N.state + 4 * s;
    if (flags[s] & FLAG_VALUE) {
      const double f = -N.L[s], fn = -N.Ltrial[s], pred = N.pred[s];
      double rho = pred > 0 ? (f - fn) / pred : -1.0;
      if (!isfinite(fn)) rho = -1.0;
      double delta = N.delta[s];
      if (rho < 0.25)
        delta = 0.25 * delta;
      else if (rho > 0.75 && st[ST_BOUNDARY])
        delta = fmin(2.0 * delta, N.delta_max);
      N.delta[s] = delta;
      int fl = 0;
      if (rho > N.eta) {
        const bool done = fabs(f - fn) <= N.ftol * fabs(fn);
        for (int k = 0; k < NP; ++k) N.theta[(size_t)s * NP + k] = N.trial[(size_t)s * NP + k];
        N.L[s] = N.Ltrial[s];
        if (done) {
          st[ST_ACTIVE] = 0;
          st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
        } else {
          fl = FLAG_FULL;
        }
      }
      if (st[ST_ACTIVE] && delta < N.delta_min) {
        st[ST_ACTIVE] = 0;
        st[ST_STATUS] = CELESTE_STATUS_RADIUS_COLLAPSE;
        fl = 0;
      }
      flags[s] = fl;
    } else {
      flags[s] = 0;
    }
    active = st[ST_ACTIVE];
  }
  // count active sources (one atomic per warp)
  const unsigned m = __ballot_sync(0xffffffffu, active);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(N.count, __popc(m));
}

__global__ void newton_finish_kernel(NewtonDev N, int32_t* iters, int32_t* status, double* elbo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N.S) return;
  if (iters) iters[s] = N.state[4 * s + ST_ITERS];
  if (status) status[s] = N.state[4 * s + ST_STATUS];
  if (elbo) elbo[s] = N.L[s];
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_newton_batch(celeste_problem* p, double* theta, const celeste_newton_opts* opts, double* delta,
                                    int32_t* iters_out, int32_t* status_out, double* elbo_out,
                                    celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound || !p->background_ready)
    return fail(CELESTE_ERR_STATE, "bind the problem and render the background first");
  if (!theta || !delta || !iters_out || !status_out) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  celeste_newton_opts o{};
  if (opts) o = *opts;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 50;
  NewtonDev N;
  const WsLayout& L = p->ws;
  N.theta = theta;
  N.delta = delta;
  N.L = reinterpret_cast<double*>(p->base + L.nt_f);
  N.gL = reinterpret_cast<double*>(p->base + L.nt_g);
  N.HL = reinterpret_cast<double*>(p->base + L.nt_H);
  N.trial = reinterpret_cast<double*>(p->base + L.nt_trial);
  N.pred = reinterpret_cast<double*>(p->base + L.nt_pred);
  N.Ltrial = reinterpret_cast<double*>(p->base + L.nt_ftrial);
  N.state = reinterpret_cast<int*>(p->base + L.nt_state);
  N.count = reinterpret_cast<int*>(p->base + L.nt_count);
  N.S = p->S;
  N.ftol = o.ftol > 0 ? o.ftol : 1e-8;
  N.gtol = o.gtol > 0 ? o.gtol : 1e-10;
  N.delta0 = o.delta0 > 0 ? o.delta0 : 1.0;
  N.delta_max = o.delta_max > 0 ? o.delta_max : 1e4;
  N.eta = o.eta > 0 ? o.eta : 0.1;
  N.delta_min = o.delta_min > 0 ? o.delta_min : 1e-12;
  const ProblemDev& D = p->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int S = p->S;
  cudaError_t e;
  auto full_eval = [&](const double* th) -> cudaError_t {
    const int m0 = prof_mark(p, st);
    cudaError_t e2 = launch_full(D, th, st);
    const int m1 = prof_mark(p, st);
    if (p->prof_on) p->prof_full.push_back({m0, m1});
    return e2;
  };
  auto value_eval = [&](const double* th) -> cudaError_t {
    const int m0 = prof_mark(p, st);
    cudaError_t e2 = launch_value(D, th, FLAG_VALUE, st);
    const int m1 = prof_mark(p, st);
    if (p->prof_on) p->prof_value.push_back({m0, m1});
    return e2;
  };
  newton_init_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, D.flags);
  if ((e = full_eval(theta)) != cudaSuccess) return cuda_fail(e, "full eval");
  if ((e = launch_assemble(D, theta, true, FLAG_FULL, N.L, N.gL, N.HL, st)) != cudaSuccess) return cuda_fail(e, "assemble");
  for (int it = 0; it < max_iter; ++it) {
    tr_step_kernel<<<(S + TR_WARPS - 1) / TR_WARPS, 32 * TR_WARPS, 0, st>>>(N, D.flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "tr_step");
    if ((e = value_eval(N.trial)) != cudaSuccess) return cuda_fail(e, "trial eval");
    if ((e = launch_assemble(D, N.trial, false, FLAG_VALUE, N.Ltrial, nullptr, nullptr, st)) != cudaSuccess)
      return cuda_fail(e, "trial assemble");
    if ((e = cudaMemsetAsync(N.count, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "count reset");
    tr_update_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, D.flags);
    if ((e = full_eval(theta)) != cudaSuccess) return cuda_fail(e, "full eval");
    if ((e = launch_assemble(D, theta, true, FLAG_FULL, N.L, N.gL, N.HL, st)) != cudaSuccess)
      return cuda_fail(e, "assemble");
    int active = 0;
    if ((e = cudaMemcpyAsync(&active, N.count, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(e, "count read");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "newton iteration");
    prof_count(p, 6);
    if (p->prof_on) p->prof_iters += 1;
    if (active == 0) break;
  }
  newton_finish_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, iters_out, status_out, elbo_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "finish");
  prof_count(p, 4);
  int err[4];
  if ((e = cudaMemcpyAsync(err, D.err, sizeof(err), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e, "err read");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "newton finish");
  if (err[ERR_TIMEOUT]) return fail(CELESTE_ERR_TIMEOUT, "a pixel kernel's bulk copy did not complete in time");
  if (err[ERR_BAD_PIXEL]) return fail(CELESTE_ERR_INVALID_ARG, "an image holds negative or non-finite counts");
  return CELESTE_OK;
}
