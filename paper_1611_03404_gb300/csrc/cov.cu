// Linear-response covariance of each source's variational parameters (paper, Sec. "Variational
// Inference": the per-source objective's curvature at its optimum, reused from the Newton
// solver's exact Hessian): Sigma = (-H)^-1, where H is the ELBO Hessian w.r.t. the 27 free
// parameters.  Defined only where -H is positive definite (a strict local maximum).
//
// One warp per source, float64: -H = L D L^T in place (lane i owns row i), then the 27 columns of
// the inverse solved at once, lane j carrying the right-hand side e_j (a float64 warp instruction
// costs the same for 1 or 32 lanes on this part, so the 27 solves cost one).
#include <algorithm>

#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"

namespace celeste {

struct CovSmem {
  double A[NP * NP];     // -H, then L below the diagonal
  double r[NP];          // reciprocal pivots
  double Y[NP][32];      // lane j: the solve for e_j
};

__global__ void __launch_bounds__(32) cov_kernel(const double* __restrict__ H, int S, double* cov, int32_t* ok) {
  __shared__ CovSmem sm;
  const int s = blockIdx.x, lane = threadIdx.x;
  if (s >= S) return;
  const double* h = H + (size_t)s * NP * NP;
  for (int i = lane; i < NP * NP; i += 32) sm.A[i] = -h[i];
  __syncwarp();
  // L D L^T with full rows kept current (row k holds the Schur complement's row when step k reads it)
  bool pd = true;
  for (int k = 0; k < NP && pd; ++k) {
    const double dk = sm.A[k * NP + k];
    pd = dk > 0.0 && isfinite(dk);   // same value in every lane
    if (!pd) break;
    const double rk = 1.0 / dk;
    const bool act = lane > k && lane < NP;
    const double li = act ? sm.A[lane * NP + k] * rk : 0.0;
    __syncwarp();
    if (act) {
      for (int j = k + 1; j < NP; ++j) sm.A[lane * NP + j] = fma(-li, sm.A[k * NP + j], sm.A[lane * NP + j]);
      sm.A[lane * NP + k] = li;
    }
    if (lane == 0) sm.r[k] = rk;
    __syncwarp();
  }
  if (lane == 0) ok[s] = pd ? 1 : 0;
  double* out = cov + (size_t)s * NP * NP;
  if (!pd) {
    for (int i = lane; i < NP * NP; i += 32) out[i] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  // lane j < 27: L y = e_j, y *= D^-1, L^T x = y
  if (lane < NP) {
    for (int i = 0; i < NP; ++i) {
      double acc = i == lane ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) acc = fma(-sm.A[i * NP + k], sm.Y[k][lane], acc);
      sm.Y[i][lane] = acc;
    }
    for (int i = 0; i < NP; ++i) sm.Y[i][lane] *= sm.r[i];
    for (int i = NP - 2; i >= 0; --i) {
      double acc = sm.Y[i][lane];
      for (int k = i + 1; k < NP; ++k) acc = fma(-sm.A[k * NP + i], sm.Y[k][lane], acc);
      sm.Y[i][lane] = acc;
    }
    for (int i = 0; i < NP; ++i) out[(size_t)i * NP + lane] = sm.Y[i][lane];
  }
}

}  // namespace celeste

using namespace celeste;

extern "C" int celeste_covariance_batch(celeste_problem* p, const double* theta, double* cov, int32_t* ok,
                                        celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound || !p->background_ready)
    return fail(CELESTE_ERR_STATE, "bind the problem and render the background first");
  if (!theta || !cov || !ok) return fail(CELESTE_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const ProblemDev& D = p->dev;
  const WsLayout& L = p->ws;
  double* f = reinterpret_cast<double*>(p->base + L.nt_f);
  double* g = reinterpret_cast<double*>(p->base + L.nt_g);
  double* H = reinterpret_cast<double*>(p->base + L.nt_H);
  cudaError_t e;
  if ((e = clear_timeout(D, st)) != cudaSuccess) return cuda_fail(e, "clear timeout word");
  if ((e = launch_set_flags(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "set flags");
  if ((e = launch_worklists(D, FLAG_FULL, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  if ((e = launch_full(D, theta, st)) != cudaSuccess) return cuda_fail(e, "pixel kernel");
  if ((e = launch_assemble(D, theta, true, f, g, H, st)) != cudaSuccess) return cuda_fail(e, "assemble");
  cov_kernel<<<p->S, 32, 0, st>>>(H, p->S, cov, ok);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "cov_kernel");
  prof_count(p, 7);
  return CELESTE_OK;
}
