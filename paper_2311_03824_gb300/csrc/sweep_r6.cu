// Instantiation of the per-column Gaussian sweep for rank width 6.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r6(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<6, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<6, false>);
}
}  // namespace lrs
