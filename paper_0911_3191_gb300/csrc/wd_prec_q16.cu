// Kernels and launchers instantiated for storage precision WD_Q16.
#include "wd_kernels.cuh"

namespace wd {
const PrecOps* ops_q16() {
  static const PrecOps ops = Impl<WD_Q16>::make();
  return &ops;
}
}  // namespace wd
