// Instantiation of the per-column Gaussian sweep for rank width 2.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r2(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<2, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<2, false>);
}
}  // namespace lrs
