// Chemistry pre-pass kernels with float arithmetic (one translation unit per
// compute type so that the build compiles them in parallel).
#include "pflb_chem_impl.cuh"

namespace pflb {

template cudaError_t chem_pass_launch<5, float>(const Params<float, 5>&, const State<float, float>&, float*,
                                             const SurrArgs*, int*, unsigned*, double*, double*,
                                             cudaStream_t);
template cudaError_t chem_pass_launch<6, float>(const Params<float, 6>&, const State<float, float>&, float*,
                                             const SurrArgs*, int*, unsigned*, double*, double*,
                                             cudaStream_t);

}  // namespace pflb
