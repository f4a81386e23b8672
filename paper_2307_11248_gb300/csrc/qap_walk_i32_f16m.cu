// Instantiations of the walk kernels with int32 deltas, int16 flow storage and
// the maintained products M in shared memory (plans with kProductM), in a
// translation unit of their own so they compile beside the other plans.
#include "qap_kernels.cuh"

namespace qapk {

#define QAP_PLANS(K)                                             \
  switch (nt * 1000 + maxpt * 10 + store) {                      \
    case 128044: return K<DT, FE, 128, 4, kProductM>;            \
    case 128124: return K<DT, FE, 128, 12, kProductM>;           \
    case 256064: return K<DT, FE, 256, 6, kProductM>;            \
    case 256084: return K<DT, FE, 256, 8, kProductM>;            \
    case 256124: return K<DT, FE, 256, 12, kProductM>;           \
    case 256164: return K<DT, FE, 256, 16, kProductM>;           \
    case 256244: return K<DT, FE, 256, 24, kProductM>;           \
    case 512044: return K<DT, FE, 512, 4, kProductM>;            \
    case 512084: return K<DT, FE, 512, 8, kProductM>;            \
    case 512124: return K<DT, FE, 512, 12, kProductM>;           \
    case 512164: return K<DT, FE, 512, 16, kProductM>;           \
    case 512204: return K<DT, FE, 512, 20, kProductM>;           \
    case 512244: return K<DT, FE, 512, 24, kProductM>;           \
    case 1024084: return K<DT, FE, 1024, 8, kProductM>;          \
    case 1024124: return K<DT, FE, 1024, 12, kProductM>;         \
    default: return nullptr;                                     \
  }

WalkKernelFn walk_kernel_i32_f16m(int nt, int maxpt, int store) {
  using DT = int32_t;
  using FE = int16_t;
  QAP_PLANS(walk_kernel)
}

#undef QAP_PLANS

}  // namespace qapk
