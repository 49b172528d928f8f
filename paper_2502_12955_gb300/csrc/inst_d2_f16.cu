// inst_d2_f16.cu -- kernels for lattice D2 with __half population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d2_f16() {
  static const KernelSet k = Launchers<D2, __half>::make();
  return k;
}
}  // namespace lbm
