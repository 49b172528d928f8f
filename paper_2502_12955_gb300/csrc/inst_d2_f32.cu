// inst_d2_f32.cu -- kernels for lattice D2 with float population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d2_f32() {
  static const KernelSet k = Launchers<D2, float>::make();
  return k;
}
}  // namespace lbm
