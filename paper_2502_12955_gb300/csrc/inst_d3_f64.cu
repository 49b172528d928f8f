// inst_d3_f64.cu -- kernels for lattice D3 with double population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d3_f64() {
  static const KernelSet k = Launchers<D3, double>::make();
  return k;
}
}  // namespace lbm
