// Evaluate kernels of the corner peak family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_corner_peak() {
  static const FamilyKernels k = make_family_kernels<CornerPeak, 128>();
  return k;
}

}  // namespace pg
