// Instantiations of the walk kernel with int64 deltas (one translation unit
// per delta width so the two compile in parallel).
#include "qap_kernels.cuh"

namespace qapk {

WalkKernelFn walk_kernel_i64(int nt, int maxpt) {
  using DT = int64_t;
  switch (nt * 100 + maxpt) {
    case 12804: return walk_kernel<DT, 128, 4>;
    case 12808: return walk_kernel<DT, 128, 8>;
    case 25604: return walk_kernel<DT, 256, 4>;
    case 25608: return walk_kernel<DT, 256, 8>;
    case 51204: return walk_kernel<DT, 512, 4>;
    case 51208: return walk_kernel<DT, 512, 8>;
    case 102408: return walk_kernel<DT, 1024, 8>;
    case 102412: return walk_kernel<DT, 1024, 12>;
    case 102416: return walk_kernel<DT, 1024, 16>;
    default: return nullptr;
  }
}

}  // namespace qapk
