// Evaluate kernels of the c0 family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_c0() {
  static const FamilyKernels k = make_family_kernels<Fixed<C0Fam>::template type, 128>();
  return k;
}

}  // namespace pg
