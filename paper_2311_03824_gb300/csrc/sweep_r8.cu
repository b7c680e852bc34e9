// Instantiation of the per-column Gaussian sweep for rank width 8.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r8(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<8, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<8, false>);
}
}  // namespace lrs
