// Kernels and launchers instantiated for storage precision WD_B16N.
#include "wd_kernels.cuh"

namespace wd {
const PrecOps* ops_b16() {
  static const PrecOps ops = Impl<WD_B16N>::make();
  return &ops;
}
}  // namespace wd
