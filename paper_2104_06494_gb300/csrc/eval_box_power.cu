// Evaluate kernels of the box-power family (sum of squares to a power), dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_box_power() {
  static const FamilyKernels k = make_family_kernels<Fixed<BoxPower>::template type, 64>();
  return k;
}

}  // namespace pg
