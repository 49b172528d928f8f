// inst_d3_f32.cu -- kernels for lattice D3 with float population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d3_f32() {
  static const KernelSet k = Launchers<D3, float>::make();
  return k;
}
}  // namespace lbm
