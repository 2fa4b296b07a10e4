// Launchers shared between the library's translation units.
#pragma once

#include "celeste_internal.cuh"

namespace celeste {

cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, cudaStream_t st);
cudaError_t launch_full(const ProblemDev& P, const double* theta, cudaStream_t st);
cudaError_t launch_value(const ProblemDev& P, const double* theta, int flag_mask, cudaStream_t st);
// Per-source float64 assembly of the tile sums into (ELBO, gradient, Hessian), KL included.
//   full: use the 108 full sums (else the value-only sums); flag_mask selects sources.
cudaError_t launch_assemble(const ProblemDev& P, const double* theta, bool full, int flag_mask, double* elbo,
                            double* grad, double* hess, cudaStream_t st);
cudaError_t launch_set_flags(const ProblemDev& P, int value, cudaStream_t st);

}  // namespace celeste
