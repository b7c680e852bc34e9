// Register-resident cluster engine instantiated for rank width 8, rows per
// lane 1..6 (m <= 192).
#include "resident_impl.cuh"

namespace lrs {
void* res_kernel_r8(int MR) {
  switch (MR) {
    case 1: return reinterpret_cast<void*>(&res::resident_kernel<8, 1>);
    case 2: return reinterpret_cast<void*>(&res::resident_kernel<8, 2>);
    case 3: return reinterpret_cast<void*>(&res::resident_kernel<8, 3>);
    case 4: return reinterpret_cast<void*>(&res::resident_kernel<8, 4>);
    case 5: return reinterpret_cast<void*>(&res::resident_kernel<8, 5>);
    case 6: return reinterpret_cast<void*>(&res::resident_kernel<8, 6>);
    default: return nullptr;
  }
}
}  // namespace lrs
