// Launchers shared between the library's translation units.
#pragma once

#include "celeste_internal.cuh"

namespace celeste {

cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, cudaStream_t st);
// Per-patch tables at theta for sources whose flags match (full: with the shape derivatives).
cudaError_t launch_tables(const ProblemDev& P, const double* theta, int flag_mask, bool full, cudaStream_t st);
// Tables (full) + ELBO/gradient/Hessian tile sums for sources flagged FLAG_FULL.
cudaError_t launch_full(const ProblemDev& P, const double* theta, cudaStream_t st);
cudaError_t launch_value(const ProblemDev& P, const double* theta, int flag_mask, bool diff, cudaStream_t st);
// Per-source float64 sum of the value-only tile sums minus the KL at theta; with theta_ref the
// result is the ELBO change from theta_ref (value kernel run in difference mode).
cudaError_t launch_assemble_value(const ProblemDev& P, const double* theta, const double* theta_ref, int flag_mask,
                                  double* out, cudaStream_t st);
// Per-source float64 assembly of the tile sums into (ELBO, gradient, Hessian), KL included.
//   full: use the 108 full sums (else the value-only sums); flag_mask selects sources.
cudaError_t launch_assemble(const ProblemDev& P, const double* theta, bool full, int flag_mask, double* elbo,
                            double* grad, double* hess, cudaStream_t st);
cudaError_t launch_set_flags(const ProblemDev& P, int value, cudaStream_t st);

}  // namespace celeste
