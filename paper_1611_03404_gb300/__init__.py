"""GB300-native (sm_103a) Celeste hot path: per-source ELBO, exact gradient and dense Hessian over
every pixel of a light source's patches, and batched trust-region Newton, behind a C ABI
(include/celeste.h) with a thin ctypes binding."""
from .celeste import (WANT_ELBO, WANT_GRAD, WANT_HESS, STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_NONFINITE,
                      STATUS_RADIUS_COLLAPSE, HESS_FP32, HESS_TF32, HESS_BF16X3, HESS_BF16X6, HESS_TF32X3, NBR_FULL, NBR_WINDOW, NPARAM, CelesteError, HostProblem, Problem, lib, load_library,
                      tr_solve_batch, tr_reciprocal, measure_peak)

__all__ = ["Problem", "HostProblem", "CelesteError", "lib", "load_library", "NPARAM", "WANT_ELBO", "WANT_GRAD",
           "WANT_HESS", "STATUS_CONVERGED", "STATUS_MAX_ITER", "STATUS_NONFINITE", "STATUS_RADIUS_COLLAPSE", "HESS_FP32", "HESS_TF32", "HESS_BF16X3", "HESS_BF16X6", "HESS_TF32X3", "NBR_FULL", "NBR_WINDOW",
           "tr_solve_batch", "tr_reciprocal", "measure_peak"]
