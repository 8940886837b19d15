// Evaluate kernels of the oscillatory family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_oscillatory() {
  static const FamilyKernels k = make_family_kernels<Fixed<Oscillatory>::template type, 64>();
  return k;
}

}  // namespace pg
