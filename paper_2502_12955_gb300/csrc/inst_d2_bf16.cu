// inst_d2_bf16.cu -- kernels for lattice D2 with __nv_bfloat16 population storage.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d2_bf16() {
  static const KernelSet k = Launchers<D2, __nv_bfloat16>::make();
  return k;
}
}  // namespace lbm
