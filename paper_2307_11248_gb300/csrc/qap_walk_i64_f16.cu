// Instantiations of the walk kernels with int64 deltas and int16 flow storage
// (one translation unit per combination so they compile in parallel), for
// one instance (walk_kernel); qap_batch_* holds the batch kernels.
#include "qap_kernels.cuh"

namespace qapk {

WalkKernelFn walk_kernel_i64_f16m(int nt, int maxpt, int store);  // qap_walk_i64_f16m.cu

#define QAP_PLANS(K)                                             \
  switch (nt * 1000 + maxpt * 10 + store) {                      \
    case 128040: return K<DT, FE, 128, 4, 0>;                    \
    case 128120: return K<DT, FE, 128, 12, 0>;                   \
    case 256060: return K<DT, FE, 256, 6, 0>;                    \
    case 256080: return K<DT, FE, 256, 8, 0>;                    \
    case 256120: return K<DT, FE, 256, 12, 0>;                   \
    case 256160: return K<DT, FE, 256, 16, 0>;                   \
    case 256240: return K<DT, FE, 256, 24, 0>;                   \
    case 512040: return K<DT, FE, 512, 4, 0>;                    \
    case 512080: return K<DT, FE, 512, 8, 0>;                    \
    case 512120: return K<DT, FE, 512, 12, 0>;                   \
    case 512160: return K<DT, FE, 512, 16, 0>;                   \
    case 512200: return K<DT, FE, 512, 20, 0>;                   \
    case 512240: return K<DT, FE, 512, 24, 0>;                   \
    case 512260: return K<DT, FE, 512, 26, 0>;                   \
    case 1024080: return K<DT, FE, 1024, 8, 0>;                  \
    case 1024120: return K<DT, FE, 1024, 12, 0>;                 \
    case 1024160: return K<DT, FE, 1024, 16, 0>;                 \
    case 1024200: return K<DT, FE, 1024, 20, 0>;                 \
    case 1024401: return K<DT, FE, 1024, 40, kGlobalDelta>;      \
    case 1024403: return K<DT, FE, 1024, 40, kGlobalDelta | kGlobalFlow>; \
    default: return nullptr;                                     \
  }

WalkKernelFn walk_kernel_i64_f16(int nt, int maxpt, int store) {
  using DT = int64_t;
  using FE = int16_t;
  if (store & kProductM) return walk_kernel_i64_f16m(nt, maxpt, store);
  QAP_PLANS(walk_kernel)
}

#undef QAP_PLANS

}  // namespace qapk
