// inst_d2_bf16s32.cu -- kernels for lattice D2 with BF16 flow populations and FP32 scalar populations.
#include <type_traits>

#include "launch.cuh"

namespace lbm {
const KernelSet& kernels_d2_bf16s32() {
  static const KernelSet k = Launchers<D2, bf16_s32>::make();
  return k;
}
}  // namespace lbm
