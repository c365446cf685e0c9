// Kernels and launchers instantiated for storage precision WD_F32.
#include "wd_kernels.cuh"

namespace wd {
const PrecOps* ops_f32() {
  static const PrecOps ops = Impl<WD_F32>::make();
  return &ops;
}
}  // namespace wd
