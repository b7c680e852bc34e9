// Instantiation of the per-column Gaussian sweep for rank width 3.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r3(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<3, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<3, false>);
}
}  // namespace lrs
