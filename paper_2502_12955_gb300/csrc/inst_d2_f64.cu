// inst_d2_f64.cu -- kernels for lattice D2 with double population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d2_f64() {
  static const KernelSet k = Launchers<D2, double>::make();
  return k;
}
}  // namespace lbm
