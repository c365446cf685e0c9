// Kernels and launchers instantiated for storage precision WD_B16N.
#include "wd_batch.cuh"

namespace wd {
const PrecOps* ops_b16() {
  static const PrecOps ops = [] {
    PrecOps o = Impl<WD_B16N>::make();
    o.dslash_batch = &ImplBatch<WD_B16N>::dslash;
    o.batch_setup = &ImplBatch<WD_B16N>::setup;
    o.batch_iteration = &ImplBatch<WD_B16N>::iteration;
    o.batch_update = &ImplBatch<WD_B16N>::update;
    return o;
  }();
  return &ops;
}
}  // namespace wd
