// Batched trust-region Newton over per-source subproblems (paper, Sec. "Variational Inference":
// each source optimised with its neighbours fixed, Newton's method with a trust region, using
// the exact gradient and dense Hessian; machine tolerance within 50 iterations).
//
// The subproblem min g.p + p.B.p/2 s.t. |p| <= delta (f = -ELBO, g = -grad, B = -Hessian) is
// solved in float64 the More-Sorensen way (trsolve.cuh: tridiagonal reduction, Sturm
// multisection, safeguarded Newton on 1/|p(lambda)| - 1/delta, hard case).  The outer iteration
// follows Nocedal & Wright Algorithm 4.1.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"
#include "trsolve.cuh"
#include "trsolve_cta.cuh"

namespace celeste {

constexpr int TR_WARPS = 1;     // sources per CTA of the step kernel (one warp: 29 KB of shared memory)

// Per-source integer state (ST_STRIDE ints).  ST_SAME: the last step was rejected, so the next
// subproblem has the same B and g; ST_CACHED: the tridiagonal form of that B is in the cache.
constexpr int ST_ACTIVE = 0, ST_ITERS = 1, ST_STATUS = 2, ST_BOUNDARY = 3, ST_SAME = 4, ST_CACHED = 5;
constexpr int ST_STRIDE = 8;

struct NewtonDev {
  double* theta;        // [S][27] current iterate (caller memory)
  double* delta;        // [S] trust radius (caller memory)
  double* L;            // [S] ELBO at theta
  double* gL;           // [S][27] gradient of the ELBO at theta
  double* HL;           // [S][27][27] Hessian of the ELBO at theta
  double* trial;        // [S][27]
  double* pred;         // [S] predicted reduction of f = -ELBO
  double* Ltrial;       // [S] ELBO change from theta to the trial point
  double* tcache;       // [S][TR_CACHE] tridiagonal form of the last Householder-reduced B
  double* lam;          // [S] multiplier of the last subproblem (negative: none)
  int* state;           // [S][ST_STRIDE]
  int* count;           // [0]: active sources after the update
  int* list;            // [S]: the active sources after the update (count[0] of them, any order)
  int cta_max;          // at most this many active sources: four warps per subproblem
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
  N.state[ST_STRIDE * s + ST_ACTIVE] = 1;
  N.state[ST_STRIDE * s + ST_ITERS] = 0;
  N.state[ST_STRIDE * s + ST_STATUS] = CELESTE_STATUS_MAX_ITER;
  N.state[ST_STRIDE * s + ST_BOUNDARY] = 0;
  N.state[ST_STRIDE * s + ST_SAME] = 0;
  N.state[ST_STRIDE * s + ST_CACHED] = 0;
  if (!(N.delta[s] > 0.0)) N.delta[s] = N.delta0;
  N.lam[s] = -1.0;
  N.list[s] = s;                  // every source active, listed in order
  if (s == 0) N.count[0] = N.S;
  flags[s] = FLAG_FULL;
}

// One warp per source: convergence tests, subproblem, trial point.
__global__ void __launch_bounds__(32 * TR_WARPS) tr_step_kernel(NewtonDev N, int* flags) {
  __shared__ TrSmem sm[TR_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * TR_WARPS + warp;
  if (s >= N.S) return;
  int* st = N.state + ST_STRIDE * s;
  if (!st[ST_ACTIVE]) {
    if (lane == 0) flags[s] = 0;
    return;
  }
  if (*N.count <= N.cta_max) return;   // few sources left: tr_step_cta_kernel takes them
  TrSmem& S = sm[warp];
  const double* HL = N.HL + (size_t)s * NP * NP;
  const double* gL = N.gL + (size_t)s * NP;
  // f = -L, g = -gL, B = -HL
  const double gk = lane < NP ? -gL[lane] : 0.0;
  // (no short-circuit: the loads are independent and issue together)
  bool finite = isfinite(N.L[s]) & isfinite(gk);
#pragma unroll
  for (int i = lane; i < NP * NP; i += 32) finite &= isfinite(HL[i]);
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
  const double delta = N.delta[s];
  double pk, pred;
  int hard;
  // A rejected step leaves B and g as they were: reuse their tridiagonal form if it was cached
  // (the Newton step, tried first where the previous step was interior, cannot fit the smaller
  // radius then).
  const bool same = st[ST_SAME] != 0;
  const bool use_cache = same && st[ST_CACHED];
  const bool try_newton = !same && st[ST_ITERS] > 0 && !st[ST_BOUNDARY];
  double* cache = N.tcache + (size_t)s * TR_CACHE;
  double lam;
  const bool reduced = tr_solve_warp(S, HL, -1.0, gk, delta, try_newton, use_cache ? cache : nullptr, cache,
                                     N.lam[s], lam, pk, pred, hard);
  if (lane == 0) {
    st[ST_CACHED] = use_cache || reduced;
    N.lam[s] = lam;
  }
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

// The same step on four warps per source (trsolve_cta.cuh), for iterations that start with at most
// N.cta_max active sources: one CTA per listed source.  The float64 pipes of all four SM
// sub-partitions then work on one subproblem, where the one-warp kernel would leave three idle.
__global__ void __launch_bounds__(128, 2) tr_step_cta_kernel(NewtonDev N, int* flags) {
  extern __shared__ __align__(16) unsigned char tr_cta_smem[];
  TrSmemQ& S = *reinterpret_cast<TrSmemQ*>(tr_cta_smem);
  const int count = *N.count;
  if (count > N.cta_max) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int q = blockIdx.x; q < count; q += gridDim.x) {
    const int s = N.list[q];
    int* st = N.state + ST_STRIDE * s;
    const double* HL = N.HL + (size_t)s * NP * NP;
    const double* gL = N.gL + (size_t)s * NP;
    const double gk = lane < NP ? -gL[lane] : 0.0;
    bool finite = isfinite(N.L[s]) & isfinite(gk);
#pragma unroll
    for (int i = lane; i < NP * NP; i += 32) finite &= isfinite(HL[i]);
    finite = __all_sync(0xffffffffu, finite);   // (every warp reads the same data: same decision)
    if (!finite) {
      if (tid == 0) {
        st[ST_ACTIVE] = 0;
        st[ST_STATUS] = CELESTE_STATUS_NONFINITE;
        flags[s] = 0;
      }
      continue;
    }
    if (warp_max(fabs(gk)) <= N.gtol) {
      if (tid == 0) {
        st[ST_ACTIVE] = 0;
        st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
        flags[s] = 0;
      }
      continue;
    }
    const double delta = N.delta[s];
    const bool same = st[ST_SAME] != 0;
    const bool use_cache = same && st[ST_CACHED];
    const bool try_newton = !same && st[ST_ITERS] > 0 && !st[ST_BOUNDARY];
    double* cache = N.tcache + (size_t)s * TR_CACHE;
    double pk = 0.0, pred = 0.0, lam = -1.0;
    int hard = 0;
    // (every thread has read the source's state before the solver's first barrier; warp 0
    // writes it back below)
    const bool reduced = tr_solve_q(S, HL, -1.0, gk, delta, try_newton, use_cache ? cache : nullptr, cache,
                                    N.lam[s], lam, pk, pred, hard);
    if (w == 0) {
      const double pnorm = sqrt(warp_sum(lane < NP ? pk * pk : 0.0));
      if (lane < NP) N.trial[(size_t)s * NP + lane] = N.theta[(size_t)s * NP + lane] + pk;
      if (lane == 0) {
        st[ST_CACHED] = use_cache || reduced;
        N.lam[s] = lam;
        N.pred[s] = pred;
        st[ST_ITERS] += 1;
        st[ST_BOUNDARY] = pnorm >= (1.0 - 1e-9) * delta;
        if (!st[ST_BOUNDARY] && pred <= N.ftol * fabs(N.L[s])) {
          st[ST_ACTIVE] = 0;
          st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
          flags[s] = 0;
        } else {
          flags[s] = FLAG_VALUE;
        }
      }
    }
    __syncthreads();
  }
}

// Batched subproblem solve for testing and standalone use: one warp per problem.
__global__ void __launch_bounds__(32 * TR_WARPS) tr_solve_batch_kernel(const double* __restrict__ B,
                                                                       const double* __restrict__ g,
                                                                       const double* __restrict__ delta, int n,
                                                                       const double* __restrict__ hint, double* p,
                                                                       double* pred, int* hard, double* lam_out) {
  __shared__ TrSmem sm[TR_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * TR_WARPS + warp;
  if (q >= n) return;
  TrSmem& S = sm[warp];
  const double gk = lane < NP ? g[(size_t)q * NP + lane] : 0.0;
  double pk, pr, lam;
  int hc;
  tr_solve_warp(S, B + (size_t)q * NP * NP, 1.0, gk, delta[q], true, nullptr, nullptr, hint ? hint[q] : -1.0, lam,
                pk, pr, hc);
  if (lane < NP) p[(size_t)q * NP + lane] = pk;
  if (lane == 0) {
    if (pred) pred[q] = pr;
    if (hard) hard[q] = hc;
    if (lam_out) lam_out[q] = lam;
  }
}

// The same on four warps per problem (one CTA each).
__global__ void __launch_bounds__(128, 2) tr_solve_batch_cta_kernel(const double* __restrict__ B,
                                                                   const double* __restrict__ g,
                                                                   const double* __restrict__ delta, int n,
                                                                   const double* __restrict__ hint, double* p,
                                                                   double* pred, int* hard, double* lam_out) {
  extern __shared__ __align__(16) unsigned char tr_cta_smem[];
  TrSmemQ& S = *reinterpret_cast<TrSmemQ*>(tr_cta_smem);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = blockIdx.x; q < n; q += gridDim.x) {
    const double gk = lane < NP ? g[(size_t)q * NP + lane] : 0.0;
    double pk = 0.0, pr = 0.0, lam = -1.0;
    int hc = 0;
    tr_solve_q(S, B + (size_t)q * NP * NP, 1.0, gk, delta[q], true, nullptr, nullptr, hint ? hint[q] : -1.0, lam, pk,
               pr, hc);
    if (w == 0) {
      if (lane < NP) p[(size_t)q * NP + lane] = pk;
      if (lane == 0) {
        if (pred) pred[q] = pr;
        if (hard) hard[q] = hc;
        if (lam_out) lam_out[q] = lam;
      }
    }
    __syncthreads();
  }
}

// The solver's float64 reciprocal applied elementwise (for its error-bound test).
__global__ void tr_reciprocal_kernel(const double* __restrict__ x, double* __restrict__ r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = tr_rcp(x[i]);
}

// Accept or reject the trial point and update the radius (Nocedal & Wright Alg. 4.1).
__global__ void tr_update_kernel(NewtonDev N, int* flags) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  int active = 0;
  if (s < N.S) {
    int* st = N.state + ST_STRIDE * s;
    if (flags[s] & FLAG_VALUE) {
      const double dL = N.Ltrial[s], pred = N.pred[s];   // f - f_new = L_new - L = dL
      double rho = pred > 0 ? dL / pred : -1.0;
      if (!isfinite(dL)) rho = -1.0;
      int fl = 0;
      if (rho <= N.eta && pred <= N.ftol * fabs(N.L[s])) {
        // a rejected step that had promised no more than ftol |f|: the radius only shrinks from
        // here, so the model has nothing left above the tolerance (the evaluation's rounding floor)
        st[ST_ACTIVE] = 0;
        st[ST_STATUS] = CELESTE_STATUS_CONVERGED;
      } else {
        double delta = N.delta[s];
        if (rho < 0.25)
          delta = 0.25 * delta;
        else if (rho > 0.75 && st[ST_BOUNDARY])
          delta = fmin(2.0 * delta, N.delta_max);
        N.delta[s] = delta;
        st[ST_SAME] = 1;   // until accepted below
        if (rho > N.eta) {
          st[ST_SAME] = 0;
          st[ST_CACHED] = 0;
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
      }
      flags[s] = fl;
    } else {
      flags[s] = 0;
    }
    active = st[ST_ACTIVE];
  }
  // count and list the active sources (one atomic per warp)
  const unsigned m = __ballot_sync(0xffffffffu, active);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && m) base = atomicAdd(N.count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (active) N.list[base + __popc(m & ((1u << lane) - 1u))] = s;
}

__global__ void newton_finish_kernel(NewtonDev N, int32_t* iters, int32_t* status, double* elbo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N.S) return;
  if (iters) iters[s] = N.state[ST_STRIDE * s + ST_ITERS];
  if (status) status[s] = N.state[ST_STRIDE * s + ST_STATUS];
  if (elbo) elbo[s] = N.L[s];
}

// Kernels launched by one Newton iteration (newton_iteration below), and profiling events recorded
// by it: value kernel (0, 1), full kernel (2, 3), subproblem step (4, 5).
constexpr int NEWTON_KERNELS_PER_ITER = 13;
constexpr int EV_PER_ITER = 6;

// The launches of one Newton iteration: subproblem step, value at the trial point, accept/reject,
// full evaluation at the accepted points.  ev (EV_PER_ITER events, or null) brackets the value and
// the full pixel kernels and the subproblem step; inside a stream capture they become event-record
// nodes.
static cudaError_t newton_iteration(const ProblemDev& D, const NewtonDev& N, cudaStream_t st, cudaEvent_t* ev,
                                    bool capturing) {
  auto mark = [&](int k) -> cudaError_t {
    if (!ev) return cudaSuccess;
    return capturing ? cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal) : cudaEventRecord(ev[k], st);
  };
  const int S = N.S;
  cudaError_t e;
  if ((e = mark(4)) != cudaSuccess) return e;
  tr_step_kernel<<<(S + TR_WARPS - 1) / TR_WARPS, 32 * TR_WARPS, 0, st>>>(N, D.flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tr_step_cta_kernel<<<std::max(1, std::min(N.cta_max, 2 * D.n_sm)), 128, sizeof(TrSmemQ), st>>>(N, D.flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(5)) != cudaSuccess) return e;
  if ((e = launch_worklists(D, FLAG_VALUE, st)) != cudaSuccess) return e;
  if ((e = launch_tables(D, N.trial, false, st)) != cudaSuccess) return e;
  if ((e = mark(0)) != cudaSuccess) return e;
  if ((e = launch_value_kernel(D, true, st)) != cudaSuccess) return e;
  if ((e = mark(1)) != cudaSuccess) return e;
  if ((e = launch_assemble_value(D, N.trial, N.theta, N.Ltrial, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(N.count, 0, sizeof(int), st)) != cudaSuccess) return e;
  tr_update_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, D.flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_worklists(D, FLAG_FULL, st)) != cudaSuccess) return e;
  if ((e = launch_tables(D, N.theta, true, st)) != cudaSuccess) return e;
  if ((e = mark(2)) != cudaSuccess) return e;
  if ((e = launch_full_kernel(D, st)) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  return launch_assemble(D, N.theta, true, N.L, N.gL, N.HL, st);
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
  N.tcache = reinterpret_cast<double*>(p->base + L.nt_tcache);
  N.count = reinterpret_cast<int*>(p->base + L.nt_count);
  N.lam = reinterpret_cast<double*>(p->base + L.nt_lam);
  N.list = reinterpret_cast<int*>(p->base + L.nt_list);
  N.cta_max = o.cta_sources > 0 ? o.cta_sources : (o.cta_sources == 0 ? 2 * p->dev.n_sm : -1);
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
  const int K = std::max(1, std::min(o.graph_iters > 0 ? o.graph_iters : 4, max_iter));
  const bool prof = p->prof_on;
  cudaError_t e;
  {
    static bool attr_set[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "device");
    if (dev < 64 && !attr_set[dev]) {
      if ((e = cudaFuncSetAttribute(tr_step_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(TrSmemQ))) != cudaSuccess)
        return cuda_fail(e, "tr_step_cta_kernel shared memory");
      attr_set[dev] = true;
    }
  }
  // events bracketing each iteration's value and full evaluation (profiling only)
  while (prof && p->iter_events.size() < (size_t)(EV_PER_ITER * K)) {
    cudaEvent_t ev;
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "event create");
    p->iter_events.push_back(ev);
  }
  auto read_events = [&](int n_iter) -> cudaError_t {
    if (!prof) return cudaSuccess;
    for (int k = 0; k < n_iter; ++k) {
      float tv = 0.f, tf = 0.f, tt = 0.f;
      const cudaEvent_t* ev = &p->iter_events[EV_PER_ITER * k];
      cudaError_t e2 = cudaEventElapsedTime(&tv, ev[0], ev[1]);
      if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(&tf, ev[2], ev[3]);
      if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(&tt, ev[4], ev[5]);
      if (e2 != cudaSuccess) return e2;
      p->prof_value_acc += tv;
      p->prof_full_acc += tf;
      p->prof_tr_acc += tt;
    }
    p->prof_tr_n += n_iter;
    p->prof_value_n += n_iter;
    p->prof_full_n += n_iter;
    p->prof_iters += n_iter;
    p->prof_launches += (long long)n_iter * NEWTON_KERNELS_PER_ITER;
    return cudaSuccess;
  };
  auto read_active = [&](int& active) -> cudaError_t {
    cudaError_t e2 = cudaMemcpyAsync(&active, N.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    return e2;
  };

  if ((e = clear_timeout(D, st)) != cudaSuccess) return cuda_fail(e, "clear timeout word");
  newton_init_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, D.flags);
  if ((e = launch_worklists(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  {
    if ((e = launch_tables(D, theta, true, st)) != cudaSuccess) return cuda_fail(e, "tables");
    const int m0 = prof_mark(p, st);
    if ((e = launch_full_kernel(D, st)) != cudaSuccess) return cuda_fail(e, "full eval");
    const int m1 = prof_mark(p, st);
    if (prof) p->prof_full.push_back({m0, m1});
  }
  if ((e = launch_assemble(D, theta, true, N.L, N.gL, N.HL, st)) != cudaSuccess) return cuda_fail(e, "assemble");
  prof_count(p, 6);

  int it = 0, active = S;
  if (K > 1) {
    // (re)capture K iterations unless the graph kept from an earlier call has the same arguments
    struct {
      NewtonDev N;
      const char* base;
      long long wait_budget;
      int K, prof;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.N = N;
    key.base = p->base;
    key.wait_budget = D.wait_budget;
    key.K = K;
    key.prof = prof ? 1 : 0;
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&key);
    if (!p->newton_exec || p->newton_key.size() != sizeof(key) ||
        std::memcmp(p->newton_key.data(), kb, sizeof(key)) != 0) {
      if (p->newton_exec) {
        cudaGraphExecDestroy(p->newton_exec);
        p->newton_exec = nullptr;
      }
      p->newton_key.clear();
      if (!p->capture_stream &&
          (e = cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "capture stream");
      cudaStream_t cs = p->capture_stream;
      if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
      cudaError_t ec = cudaSuccess;
      for (int k = 0; k < K && ec == cudaSuccess; ++k)
        ec = newton_iteration(D, N, cs, prof ? &p->iter_events[EV_PER_ITER * k] : nullptr, true);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      if (ec != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ec != cudaSuccess ? ec : e, "capture of the Newton iterations");
      }
      e = cudaGraphInstantiate(&p->newton_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        p->newton_exec = nullptr;
        return cuda_fail(e, "graph instantiate");
      }
      p->newton_key.assign(kb, kb + sizeof(key));
    }
    while (active > 0 && it + K <= max_iter) {
      if ((e = cudaGraphLaunch(p->newton_exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
      if ((e = read_active(active)) != cudaSuccess) return cuda_fail(e, "newton iterations");
      if ((e = read_events(K)) != cudaSuccess) return cuda_fail(e, "iteration events");
      it += K;
    }
  }
  // plain launches: every iteration when K == 1, else the iterations left over after the graphs
  while (active > 0 && it < max_iter) {
    if ((e = newton_iteration(D, N, st, prof ? &p->iter_events[0] : nullptr, false)) != cudaSuccess)
      return cuda_fail(e, "newton iteration");
    if ((e = read_active(active)) != cudaSuccess) return cuda_fail(e, "newton iteration");
    if ((e = read_events(1)) != cudaSuccess) return cuda_fail(e, "iteration events");
    ++it;
  }
  newton_finish_kernel<<<(S + 127) / 128, 128, 0, st>>>(N, iters_out, status_out, elbo_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "finish");
  prof_count(p, 4);
  return device_errors(D, st);
}

extern "C" int celeste_tr_solve_batch(const double* B, const double* g, const double* delta, int n, double* p,
                                      double* pred, int32_t* hard, celeste_stream_t stream) {
  return celeste_tr_solve_batch_ex(B, g, delta, n, 1, nullptr, p, pred, hard, nullptr, stream);
}

extern "C" int celeste_tr_solve_batch_ex(const double* B, const double* g, const double* delta, int n, int warps,
                                         const double* lam_hint, double* p, double* pred, int32_t* hard, double* lam,
                                         celeste_stream_t stream) {
  if (n < 0 || (n > 0 && (!B || !g || !delta || !p))) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  if (warps != 1 && warps != 4) return fail(CELESTE_ERR_INVALID_ARG, "warps must be 1 or 4");
  if (n == 0) return CELESTE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (warps == 1) {
    tr_solve_batch_kernel<<<(n + TR_WARPS - 1) / TR_WARPS, 32 * TR_WARPS, 0, st>>>(B, g, delta, n, lam_hint, p, pred,
                                                                                   hard, lam);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tr_solve_batch_kernel");
    return CELESTE_OK;
  }
  static bool attr_set[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "device");
  if (dev < 64 && !attr_set[dev]) {
    if ((e = cudaFuncSetAttribute(tr_solve_batch_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(TrSmemQ))) != cudaSuccess)
      return cuda_fail(e, "tr_solve_batch_cta_kernel shared memory");
    attr_set[dev] = true;
  }
  tr_solve_batch_cta_kernel<<<std::min(n, 1024), 128, sizeof(TrSmemQ), st>>>(B, g, delta, n, lam_hint, p, pred, hard,
                                                                              lam);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tr_solve_batch_cta_kernel");
  return CELESTE_OK;
}

extern "C" int celeste_tr_reciprocal(const double* x, double* r, int n, celeste_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !r))) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  if (n == 0) return CELESTE_OK;
  tr_reciprocal_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, r, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tr_reciprocal_kernel");
  return CELESTE_OK;
}
