// Chemistry pre-pass kernels with double arithmetic (one translation unit per
// compute type so that the build compiles them in parallel).
#include "pflb_chem_impl.cuh"

namespace pflb {

template cudaError_t chem_pass_launch<5, double>(const Params<double, 5>&, const State<double, double>&, double*,
                                             const SurrArgs*, int*, unsigned*, double*, double*,
                                             cudaStream_t);
template cudaError_t chem_pass_launch<6, double>(const Params<double, 6>&, const State<double, double>&, double*,
                                             const SurrArgs*, int*, unsigned*, double*, double*,
                                             cudaStream_t);

}  // namespace pflb
