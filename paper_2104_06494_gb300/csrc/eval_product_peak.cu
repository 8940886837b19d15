// Evaluate kernels of the product peak family, dimensions 2..8.
#include "pagani_kernels.cuh"

namespace pg {

#ifdef PAGANI_GM7
// compiled a second time with -DPAGANI_GM7: the Genz-Malik degree-7 variant
const FamilyKernels& kernels_product_peak_gm7() {
  static const FamilyKernels k = make_family_kernels_gm7<Fixed<ProductPeak>::template type, 128>();
  return k;
}
#else
const FamilyKernels& kernels_product_peak() {
  static const FamilyKernels k = make_family_kernels<Fixed<ProductPeak>::template type, 128>();
  return k;
}
#endif

}  // namespace pg
