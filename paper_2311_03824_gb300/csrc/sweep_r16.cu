// Instantiation of the per-column Gaussian sweep for rank width 16.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r16(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<16, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<16, false>);
}
}  // namespace lrs
