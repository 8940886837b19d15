// Evaluate kernels of the product peak family, dimensions 2..8.
#include "pagani_eval.cuh"

namespace pg {

const FamilyKernels& kernels_product_peak() {
  static const FamilyKernels k = make_family_kernels<Fixed<ProductPeak>::template type, 128>();
  return k;
}

}  // namespace pg
