// Instantiation of the per-column Gaussian sweep for rank width 5.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r5(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<5, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<5, false>);
}
}  // namespace lrs
