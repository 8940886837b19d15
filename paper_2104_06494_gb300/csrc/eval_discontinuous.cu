// Evaluate kernels of the discontinuous family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_discontinuous() {
  static const FamilyKernels k = make_family_kernels<Fixed<Discontinuous>::template type, 128>();
  return k;
}

}  // namespace pg
