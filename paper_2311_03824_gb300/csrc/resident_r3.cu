// Register-resident cluster engine instantiated for rank width 3, rows per
// lane 1..6 (m <= 192).
#include "resident_impl.cuh"

namespace lrs {
void* res_kernel_r3(int MR) {
  switch (MR) {
    case 1: return reinterpret_cast<void*>(&res::resident_kernel<3, 1>);
    case 2: return reinterpret_cast<void*>(&res::resident_kernel<3, 2>);
    case 3: return reinterpret_cast<void*>(&res::resident_kernel<3, 3>);
    case 4: return reinterpret_cast<void*>(&res::resident_kernel<3, 4>);
    case 5: return reinterpret_cast<void*>(&res::resident_kernel<3, 5>);
    case 6: return reinterpret_cast<void*>(&res::resident_kernel<3, 6>);
    default: return nullptr;
  }
}
}  // namespace lrs
