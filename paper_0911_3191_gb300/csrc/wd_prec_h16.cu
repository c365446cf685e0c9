// Kernels and launchers instantiated for storage precision WD_H16N.
#include "wd_kernels.cuh"

namespace wd {
const PrecOps* ops_h16() {
  static const PrecOps ops = Impl<WD_H16N>::make();
  return &ops;
}
}  // namespace wd
