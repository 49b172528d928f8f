// inst_d3_f16.cu -- kernels for lattice D3 with __half population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d3_f16() {
  static const KernelSet k = Launchers<D3, __half>::make();
  return k;
}
}  // namespace lbm
