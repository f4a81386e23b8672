// Instantiations of the walk kernel with int64 deltas and int16 flow storage
// (one translation unit per combination so they compile in parallel), for
// one instance (walk_kernel) and for a batch of instances (batch_kernel).
#include "qap_kernels.cuh"

namespace qapk {

WalkKernelFn walk_kernel_i64_f16(int nt, int maxpt) {
  using DT = int64_t;
  using FE = int16_t;
  switch (nt * 100 + maxpt) {
    case 12804: return walk_kernel<DT, FE, 128, 4>;
    case 12812: return walk_kernel<DT, FE, 128, 12>;
    case 25606: return walk_kernel<DT, FE, 256, 6>;
    case 25608: return walk_kernel<DT, FE, 256, 8>;
    case 51204: return walk_kernel<DT, FE, 512, 4>;
    case 51208: return walk_kernel<DT, FE, 512, 8>;
    case 51212: return walk_kernel<DT, FE, 512, 12>;
    case 102408: return walk_kernel<DT, FE, 1024, 8>;
    case 102412: return walk_kernel<DT, FE, 1024, 12>;
    case 102416: return walk_kernel<DT, FE, 1024, 16>;
    case 102420: return walk_kernel<DT, FE, 1024, 20>;
    default: return nullptr;
  }
}

BatchKernelFn batch_kernel_i64_f16(int nt, int maxpt) {
  using DT = int64_t;
  using FE = int16_t;
  switch (nt * 100 + maxpt) {
    case 12804: return batch_kernel<DT, FE, 128, 4>;
    case 12812: return batch_kernel<DT, FE, 128, 12>;
    case 25606: return batch_kernel<DT, FE, 256, 6>;
    case 25608: return batch_kernel<DT, FE, 256, 8>;
    case 51204: return batch_kernel<DT, FE, 512, 4>;
    case 51208: return batch_kernel<DT, FE, 512, 8>;
    case 51212: return batch_kernel<DT, FE, 512, 12>;
    case 102408: return batch_kernel<DT, FE, 1024, 8>;
    case 102412: return batch_kernel<DT, FE, 1024, 12>;
    case 102416: return batch_kernel<DT, FE, 1024, 16>;
    case 102420: return batch_kernel<DT, FE, 1024, 20>;
    default: return nullptr;
  }
}

}  // namespace qapk
