// pflb_chem.cuh -- host entry of the chemistry pre-pass (implicit Newton
// integrator or learned surrogate with Newton fallback).  The kernels read
// only T, Y, phi and the scalar block of a state, so they are compiled once
// per (species count, compute type) in pflb_chem.cu and shared by every
// lattice and storage precision.
#pragma once

#include <cuda_runtime.h>

#include "pflb_kernels.cuh"
#include "pflb_surrogate.cuh"

namespace pflb {

// Queue the chemistry increments of state S (T, Y, phi, scal) into src
// ([K+1][N], the step's source terms).  P.chem == 2: backward-Euler Newton
// per fluid cell; P.chem == 3: network pre-pass with `surr` (K = 6), cells it
// rejects listed in fb_idx / fb_count and integrated by Newton, counters in
// stats.  When `out` is non-null the increments (dY, dT) are also written
// there as doubles ([K+1][N]).
template <int K, class Real>
cudaError_t chem_pass_launch(const Params<Real, K>& P, const State<Real, Real>& S, Real* src,
                             const SurrArgs* surr, int* fb_idx, unsigned* fb_count,
                             double* stats, double* out, cudaStream_t st);

extern template cudaError_t chem_pass_launch<5, double>(const Params<double, 5>&,
                                                        const State<double, double>&, double*,
                                                        const SurrArgs*, int*, unsigned*, double*,
                                                        double*, cudaStream_t);
extern template cudaError_t chem_pass_launch<6, double>(const Params<double, 6>&,
                                                        const State<double, double>&, double*,
                                                        const SurrArgs*, int*, unsigned*, double*,
                                                        double*, cudaStream_t);
extern template cudaError_t chem_pass_launch<5, float>(const Params<float, 5>&,
                                                       const State<float, float>&, float*,
                                                       const SurrArgs*, int*, unsigned*, double*,
                                                       double*, cudaStream_t);
extern template cudaError_t chem_pass_launch<6, float>(const Params<float, 6>&,
                                                       const State<float, float>&, float*,
                                                       const SurrArgs*, int*, unsigned*, double*,
                                                       double*, cudaStream_t);

}  // namespace pflb
