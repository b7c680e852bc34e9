// Instantiation of the per-column Gaussian sweep for rank width 4.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r4(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<4, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<4, false>);
}
}  // namespace lrs
