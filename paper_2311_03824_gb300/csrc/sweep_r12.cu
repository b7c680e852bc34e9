// Instantiation of the per-column Gaussian sweep for rank width 12.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r12(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<12, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<12, false>);
}
}  // namespace lrs
