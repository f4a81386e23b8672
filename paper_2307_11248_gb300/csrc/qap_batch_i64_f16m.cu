// Instantiations of the batch kernels with int64 deltas, int16 flow storage and
// the maintained products M in shared memory (plans with kProductM), in a
// translation unit of their own so they compile beside the other plans.
#include "qap_kernels.cuh"

namespace qapk {

#define QAP_PLANS(K)                                             \
  switch (nt * 10000 + maxpt * 100 + store) {                  \
    case 1280404: return K<DT, FE, 128, 4, kProductM>;       \
    case 1281204: return K<DT, FE, 128, 12, kProductM>;      \
    case 2560604: return K<DT, FE, 256, 6, kProductM>;       \
    case 2560804: return K<DT, FE, 256, 8, kProductM>;       \
    case 2561204: return K<DT, FE, 256, 12, kProductM>;      \
    case 2561604: return K<DT, FE, 256, 16, kProductM>;      \
    case 2562404: return K<DT, FE, 256, 24, kProductM>;      \
    case 5120404: return K<DT, FE, 512, 4, kProductM>;       \
    case 5120804: return K<DT, FE, 512, 8, kProductM>;       \
    case 5121204: return K<DT, FE, 512, 12, kProductM>;      \
    case 5121604: return K<DT, FE, 512, 16, kProductM>;      \
    case 5122004: return K<DT, FE, 512, 20, kProductM>;      \
    case 5122404: return K<DT, FE, 512, 24, kProductM>;      \
    case 10240804: return K<DT, FE, 1024, 8, kProductM>;     \
    case 10241204: return K<DT, FE, 1024, 12, kProductM>;    \
    case 2561220: return K<DT, FE, 256, 12, kProductM | kNoTransposed>; \
    case 2561620: return K<DT, FE, 256, 16, kProductM | kNoTransposed>; \
    case 2562420: return K<DT, FE, 256, 24, kProductM | kNoTransposed>; \
    case 5121220: return K<DT, FE, 512, 12, kProductM | kNoTransposed>; \
    case 5121620: return K<DT, FE, 512, 16, kProductM | kNoTransposed>; \
    case 5122020: return K<DT, FE, 512, 20, kProductM | kNoTransposed>; \
    case 5122420: return K<DT, FE, 512, 24, kProductM | kNoTransposed>; \
    case 5122604: return K<DT, FE, 512, 26, kProductM>;       \
    case 5122620: return K<DT, FE, 512, 26, kProductM | kNoTransposed>; \
    default: return nullptr;                                     \
  }

BatchKernelFn batch_kernel_i64_f16m(int nt, int maxpt, int store) {
  using DT = int64_t;
  using FE = int16_t;
  QAP_PLANS(batch_kernel)
}

#undef QAP_PLANS

}  // namespace qapk
