// Batched trust-region Newton over per-source subproblems (paper, Sec. "Variational Inference":
// each source optimised with its neighbours fixed, Newton's method with a trust region, using
// the exact gradient and dense Hessian; machine tolerance within 50 iterations).
//
// The subproblem min g.p + p.B.p/2 s.t. |p| <= delta (f = -ELBO, g = -grad, B = -Hessian) is
// solved in float64 the More-Sorensen way (trsolve.cuh: tridiagonal reduction, Sturm
// multisection, safeguarded Newton on 1/|p(lambda)| - 1/delta, hard case).  The outer iteration
// follows Nocedal & Wright Algorithm 4.1.
#include <cmath>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"
#include "trsolve.cuh"

namespace celeste {

constexpr int TR_WARPS = 4;     // sources per CTA of the step kernel

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
  double* Ltrial;       // [S] ELBO change from theta to the trial point
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

// One warp per source: convergence tests, subproblem, trial point.
__global__ void __launch_bounds__(32 * TR_WARPS) tr_step_kernel(NewtonDev N, int* flags) {
  __shared__ TrSmem sm[TR_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * TR_WARPS + warp;
  if (s >= N.S) return;
  int* st = N.state + 4 * s;
  if (!st[ST_ACTIVE]) {
    if (lane == 0) flags[s] = 0;
    return;
  }
  TrSmem& S = sm[warp];
  const double* HL = N.HL + (size_t)s * NP * NP;
  const double* gL = N.gL + (size_t)s * NP;
  // f = -L, g = -gL, B = -HL
  const double gk = lane < NP ? -gL[lane] : 0.0;
  bool finite = isfinite(N.L[s]) && isfinite(gk);
  for (int i = lane; i < NP * NP; i += 32) {
    const double b = -HL[i];
    finite = finite && isfinite(b);
    S.A[(i / NP) * TR_LD + (i % NP)] = b;
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
  const double delta = N.delta[s];
  double pk, pred;
  int hard;
  tr_solve_warp(S, gk, delta, pk, pred, hard);
  const double pnorm = sqrt(warp_sum(lane < NP ? pk * pk : 0.0));
  if (lane < NP) N.trial[(size_t)s * NP + lane] = N.theta[(size_t)s * NP + lane] + pk;
  if (lane == 0) {
    N.pred[s] = pred;
    st[ST_ITERS] += 1;
    st[ST_BOUNDARY] = pnorm >= (1.0 - 1e-9) * delta;
    // Newton decrement: an interior step that promises less than ftol |f| ends the solve
    if (!st[ST_BOUNDARY] && pred <= N.ftol * fabs(N.L[s])) {
      st[ST_ACTIVE] = 0;
      st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
      flags[s] = 0;
    } else {
      flags[s] = FLAG_VALUE;
    }
  }
}

// Batched subproblem solve for testing and standalone use: one warp per problem.
__global__ void __launch_bounds__(32 * TR_WARPS) tr_solve_batch_kernel(const double* __restrict__ B,
                                                                       const double* __restrict__ g,
                                                                       const double* __restrict__ delta, int n,
                                                                       double* p, double* pred, int* hard) {
  __shared__ TrSmem sm[TR_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * TR_WARPS + warp;
  if (q >= n) return;
  TrSmem& S = sm[warp];
  for (int i = lane; i < NP * NP; i += 32) S.A[(i / NP) * TR_LD + (i % NP)] = B[(size_t)q * NP * NP + i];
  const double gk = lane < NP ? g[(size_t)q * NP + lane] : 0.0;
  __syncwarp();
  double pk, pr;
  int hc;
  tr_solve_warp(S, gk, delta[q], pk, pr, hc);
  if (lane < NP) p[(size_t)q * NP + lane] = pk;
  if (lane == 0) {
    if (pred) pred[q] = pr;
    if (hard) hard[q] = hc;
  }
}

// Accept or reject the trial point and update the radius (Nocedal & Wright Alg. 4.1).
__global__ void tr_update_kernel(NewtonDev N, int* flags) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int active = 0;
  if (s < N.S) {
    int* st = N.state + 4 * s;
    if (flags[s] & FLAG_VALUE) {
      const double dL = N.Ltrial[s], pred = N.pred[s];   // f - f_new = L_new - L = dL
      double rho = pred > 0 ? dL / pred : -1.0;
      if (!isfinite(dL)) rho = -1.0;
      double delta = N.delta[s];
      if (rho < 0.25)
        delta = 0.25 * delta;
      else if (rho > 0.75 && st[ST_BOUNDARY])
        delta = fmin(2.0 * delta, N.delta_max);
      N.delta[s] = delta;
      int fl = 0;
      if (rho > N.eta) {
        const double Lnew = N.L[s] + dL;
        const bool done = fabs(dL) <= N.ftol * fabs(Lnew);
        for (int k = 0; k < NP; ++k) N.theta[(size_t)s * NP + k] = N.trial[(size_t)s * NP + k];
        N.L[s] = Lnew;
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
    cudaError_t e2 = launch_value(D, th, FLAG_VALUE, true, st);
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
    if ((e = launch_assemble_value(D, N.trial, theta, FLAG_VALUE, N.Ltrial, st)) != cudaSuccess)
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

extern "C" int celeste_tr_solve_batch(const double* B, const double* g, const double* delta, int n, double* p,
                                      double* pred, int32_t* hard, celeste_stream_t stream) {
  if (n < 0 || (n > 0 && (!B || !g || !delta || !p))) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  if (n == 0) return CELESTE_OK;
  tr_solve_batch_kernel<<<(n + TR_WARPS - 1) / TR_WARPS, 32 * TR_WARPS, 0, (cudaStream_t)stream>>>(B, g, delta, n, p,
                                                                                                 pred, hard);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tr_solve_batch_kernel");
  return CELESTE_OK;
}
