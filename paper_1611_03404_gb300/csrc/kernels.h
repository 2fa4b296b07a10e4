// Launchers shared between the library's translation units.
#pragma once

#include "celeste_internal.cuh"

namespace celeste {

// clip: neighbours counted on their own windows only (the joint objective's per-source blocks).
cudaError_t launch_background(const ProblemDev& P, const double* nbr_theta, int clip, cudaStream_t st);
// Rebuilds the tile/patch/source worklists from the sources whose flags match `mask`. Every
// launcher below works on the current worklists, whose counts live on the device, so a sequence
// of launches needs no host round trip and can be captured in a CUDA graph.
cudaError_t launch_worklists(const ProblemDev& P, int mask, cudaStream_t st);
// Per-patch tables at theta for the listed patches (full: with the shape derivatives).
cudaError_t launch_tables(const ProblemDev& P, const double* theta, bool full, cudaStream_t st);
// Tables (full) + ELBO/gradient/Hessian tile sums for the listed tiles.
cudaError_t launch_full(const ProblemDev& P, const double* theta, cudaStream_t st);
// Tables (value) + value-only tile sums for the listed tiles (diff: differences from the stored
// per-pixel source moments).
cudaError_t launch_value(const ProblemDev& P, const double* theta, bool diff, cudaStream_t st);
// The pixel kernels alone, on tables already built for the listed patches.
cudaError_t launch_full_kernel(const ProblemDev& P, cudaStream_t st);
cudaError_t launch_value_kernel(const ProblemDev& P, bool diff, cudaStream_t st);
// Per-source float64 sum of the value-only tile sums minus the KL at theta; with theta_ref the
// result is the ELBO change from theta_ref (value kernel run in difference mode).
cudaError_t launch_assemble_value(const ProblemDev& P, const double* theta, const double* theta_ref, double* out,
                                  cudaStream_t st);
// Per-source float64 assembly of the tile sums into (ELBO, gradient, Hessian), KL included.
//   full: use the 108 full sums (else the value-only sums); the listed sources only.
cudaError_t launch_assemble(const ProblemDev& P, const double* theta, bool full, double* elbo, double* grad,
                            double* hess, cudaStream_t st);
cudaError_t launch_set_flags(const ProblemDev& P, int value, cudaStream_t st);

}  // namespace celeste
