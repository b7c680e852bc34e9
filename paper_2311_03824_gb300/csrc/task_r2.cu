// Instantiation of the persistent task engine for rank width 2 (all
// stored forms of A_k).
#include "task_sweep_impl.cuh"

namespace lrs {
void* task_kernel_r2(int et) {
  using namespace task;
  switch (et) {
    case 1: return reinterpret_cast<void*>(&task_kernel<2, 1>);
    case 2: return reinterpret_cast<void*>(&task_kernel<2, 2>);
    case 3: return reinterpret_cast<void*>(&task_kernel<2, 3>);
    default: return reinterpret_cast<void*>(&task_kernel<2, 0>);
  }
}
}  // namespace lrs
