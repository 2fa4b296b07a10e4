// C ABI entry points: background rendering and batched ELBO / gradient / Hessian.
#include "celeste_internal.cuh"
#include "kernels.h"
#include "problem.h"

using namespace celeste;

extern "C" int celeste_render_background_mode(celeste_problem* p, const double* nbr_theta, int mode,
                                              celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  if (!nbr_theta) return fail(CELESTE_ERR_INVALID_ARG, "null nbr_theta");
  if (mode != CELESTE_NBR_FULL && mode != CELESTE_NBR_WINDOW)
    return fail(CELESTE_ERR_INVALID_ARG, "mode must be CELESTE_NBR_FULL or CELESTE_NBR_WINDOW");
  cudaError_t e = launch_background(p->dev, nbr_theta, mode == CELESTE_NBR_WINDOW ? 1 : 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "background kernel");
  prof_count(p, 1);
  p->background_ready = true;
  p->background_mode = mode;
  return CELESTE_OK;
}

extern "C" int celeste_render_background(celeste_problem* p, const double* nbr_theta, celeste_stream_t stream) {
  return celeste_render_background_mode(p, nbr_theta, CELESTE_NBR_FULL, stream);
}

extern "C" int celeste_elbo_batch(celeste_problem* p, const double* theta, unsigned want, double* elbo, double* grad,
                                  double* hess, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound || !p->background_ready)
    return fail(CELESTE_ERR_STATE, "bind the problem and render the background first");
  if (!theta) return fail(CELESTE_ERR_INVALID_ARG, "null theta");
  if (!want || (want & ~7u)) return fail(CELESTE_ERR_INVALID_ARG, "want must be a non-empty OR of CELESTE_WANT_*");
  if ((want & CELESTE_WANT_ELBO) && !elbo) return fail(CELESTE_ERR_INVALID_ARG, "elbo output is NULL");
  if ((want & CELESTE_WANT_GRAD) && !grad) return fail(CELESTE_ERR_INVALID_ARG, "grad output is NULL");
  if ((want & CELESTE_WANT_HESS) && !hess) return fail(CELESTE_ERR_INVALID_ARG, "hess output is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const bool full = (want & (CELESTE_WANT_GRAD | CELESTE_WANT_HESS)) != 0;
  const int flag = full ? FLAG_FULL : FLAG_VALUE;
  cudaError_t e = clear_timeout(p->dev, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear timeout word");
  if ((e = launch_set_flags(p->dev, flag, st)) != cudaSuccess) return cuda_fail(e, "set flags");
  if ((e = launch_worklists(p->dev, flag, st)) != cudaSuccess) return cuda_fail(e, "worklists");
  if ((e = launch_tables(p->dev, theta, full, st)) != cudaSuccess) return cuda_fail(e, "tables");
  const int m0 = prof_mark(p, st);
  e = full ? launch_full_kernel(p->dev, st) : launch_value_kernel(p->dev, false, st);
  if (e != cudaSuccess) return cuda_fail(e, "pixel kernel");
  const int m1 = prof_mark(p, st);
  if (p->prof_on) (full ? p->prof_full : p->prof_value).push_back({m0, m1});
  prof_count(p, 6);
  e = full ? launch_assemble(p->dev, theta, true, (want & CELESTE_WANT_ELBO) ? elbo : nullptr,
                             (want & CELESTE_WANT_GRAD) ? grad : nullptr, (want & CELESTE_WANT_HESS) ? hess : nullptr, st)
           : launch_assemble_value(p->dev, theta, nullptr, elbo, st);
  if (e != cudaSuccess) return cuda_fail(e, "assemble kernel");
  return CELESTE_OK;
}

extern "C" int celeste_problem_check(celeste_problem* p, celeste_stream_t stream) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  if (!p->bound) return fail(CELESTE_ERR_STATE, "problem is not bound to a workspace");
  return device_errors(p->dev, (cudaStream_t)stream);
}

extern "C" int celeste_problem_set_wait_budget(celeste_problem* p, long long cycles) {
  if (!p) return fail(CELESTE_ERR_INVALID_ARG, "null problem");
  p->wait_budget = cycles;
  p->dev.wait_budget = cycles ? cycles : WAIT_BUDGET_DEFAULT;
  return CELESTE_OK;
}
