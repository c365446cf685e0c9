// Kernels and launchers instantiated for storage precision WD_F32.
#include "wd_batch.cuh"

namespace wd {
const PrecOps* ops_f32() {
  static const PrecOps ops = [] {
    PrecOps o = Impl<WD_F32>::make();
    o.dslash_batch = &ImplBatch<WD_F32>::dslash;
    o.batch_setup = &ImplBatch<WD_F32>::setup;
    o.batch_iteration = &ImplBatch<WD_F32>::iteration;
    o.batch_update = &ImplBatch<WD_F32>::update;
    return o;
  }();
  return &ops;
}
}  // namespace wd
