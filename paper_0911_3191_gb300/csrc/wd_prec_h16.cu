// Kernels and launchers instantiated for storage precision WD_H16N.
#include "wd_batch.cuh"

namespace wd {
const PrecOps* ops_h16() {
  static const PrecOps ops = [] {
    PrecOps o = Impl<WD_H16N>::make();
    o.dslash_batch = &ImplBatch<WD_H16N>::dslash;
    o.batch_setup = &ImplBatch<WD_H16N>::setup;
    o.batch_iteration = &ImplBatch<WD_H16N>::iteration;
    o.batch_update = &ImplBatch<WD_H16N>::update;
    return o;
  }();
  return &ops;
}
}  // namespace wd
