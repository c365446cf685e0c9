// Kernels and launchers instantiated for storage precision WD_F64.
#include "wd_batch.cuh"

namespace wd {
const PrecOps* ops_f64() {
  static const PrecOps ops = [] {
    PrecOps o = Impl<WD_F64>::make();
    o.dslash_batch = &ImplBatch<WD_F64>::dslash;
    o.batch_setup = &ImplBatch<WD_F64>::setup;
    o.batch_iteration = &ImplBatch<WD_F64>::iteration;
    o.batch_update = &ImplBatch<WD_F64>::update;
    return o;
  }();
  return &ops;
}
}  // namespace wd
