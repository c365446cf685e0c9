// Kernels and launchers instantiated for storage precision WD_F64.
#include "wd_kernels.cuh"

namespace wd {
const PrecOps* ops_f64() {
  static const PrecOps ops = Impl<WD_F64>::make();
  return &ops;
}
}  // namespace wd
