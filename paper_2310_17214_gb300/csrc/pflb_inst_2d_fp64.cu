// Instantiations of the 2-D fp64 kernels (one translation unit per lattice
// and precision so that the build compiles them in parallel).
#include "pflb_launch.cuh"

namespace pflb {

Launcher* make_launcher_2d_fp64(int K, const pflb_domain_desc& d, const pflb_mechanism& m) {
  switch (K) {
    case 0: return new LauncherImpl<2, 0, MODE_FP64>(d, m);
    case 5: return new LauncherImpl<2, 5, MODE_FP64>(d, m);
    case 6: return new LauncherImpl<2, 6, MODE_FP64>(d, m);
    default: return nullptr;
  }
}

}  // namespace pflb
