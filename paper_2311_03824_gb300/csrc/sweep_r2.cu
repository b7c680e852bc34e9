// Instantiation of the per-column Gaussian sweep for rank width 2 (all
// stored forms of A_k, resident and streamed slabs).
#include "sweep_gauss_impl.cuh"

namespace lrs {
void* sweep_kernel_r2(int resident, int et) {
  using namespace sweep;
  switch (et) {
    case 1: return resident ? reinterpret_cast<void*>(&sweep_kernel<2, true, 1>)
                            : reinterpret_cast<void*>(&sweep_kernel<2, false, 1>);
    case 2: return resident ? reinterpret_cast<void*>(&sweep_kernel<2, true, 2>)
                            : reinterpret_cast<void*>(&sweep_kernel<2, false, 2>);
    case 3: return resident ? reinterpret_cast<void*>(&sweep_kernel<2, true, 3>)
                            : reinterpret_cast<void*>(&sweep_kernel<2, false, 3>);
    default: return resident ? reinterpret_cast<void*>(&sweep_kernel<2, true, 0>)
                             : reinterpret_cast<void*>(&sweep_kernel<2, false, 0>);
  }
}
}  // namespace lrs
