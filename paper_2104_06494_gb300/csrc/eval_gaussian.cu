// Evaluate kernels of the gaussian family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_gaussian() {
  static const FamilyKernels k = make_family_kernels<Fixed<Gaussian>::template type, 128>();
  return k;
}

}  // namespace pg
