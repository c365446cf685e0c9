// Kernels and launchers instantiated for storage precision WD_Q16.
#include "wd_batch.cuh"

namespace wd {
const PrecOps* ops_q16() {
  static const PrecOps ops = [] {
    PrecOps o = Impl<WD_Q16>::make();
    o.dslash_batch = &ImplBatch<WD_Q16>::dslash;
    o.batch_setup = &ImplBatch<WD_Q16>::setup;
    o.batch_iteration = &ImplBatch<WD_Q16>::iteration;
    o.batch_update = &ImplBatch<WD_Q16>::update;
    return o;
  }();
  return &ops;
}
}  // namespace wd
