// Instantiation of the per-column Gaussian sweep for rank width 10.
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r10(int resident) {
  return resident ? reinterpret_cast<void*>(&sweep::sweep_kernel<10, true>)
                  : reinterpret_cast<void*>(&sweep::sweep_kernel<10, false>);
}
}  // namespace lrs
