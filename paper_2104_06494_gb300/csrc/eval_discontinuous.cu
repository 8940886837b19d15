// Evaluate kernels of the discontinuous family, dimensions 2..8.
#include "pagani_kernels.cuh"

namespace pg {

#ifdef PAGANI_GM7
// compiled a second time with -DPAGANI_GM7: the Genz-Malik degree-7 variant
const FamilyKernels& kernels_discontinuous_gm7() {
  static const FamilyKernels k = make_family_kernels_gm7<Fixed<Discontinuous>::template type, 128>();
  return k;
}
#else
const FamilyKernels& kernels_discontinuous() {
  static const FamilyKernels k = make_family_kernels<Fixed<Discontinuous>::template type, 128>();
  return k;
}
#endif

}  // namespace pg
