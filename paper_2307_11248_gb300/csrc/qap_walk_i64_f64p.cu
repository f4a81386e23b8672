// Instantiations of the walk_kernels with int64 deltas and int64 flows and
// distances whose P and P^T live in the per-CTA workspace (kGlobalP), the
// plans of larger n on the int64 element path; qap_walk_i64_f64.cu holds
// the plans with P in shared memory.
#include "qap_kernels.cuh"

namespace qapk {

#define QAP_PLANS(K)                                  \
  switch (nt * 10000 + maxpt * 100 + store) {         \
    case 1280410: return K<DT, FE, 128, 4, kGlobalFlow | kGlobalP>; \
    case 1281210: return K<DT, FE, 128, 12, kGlobalFlow | kGlobalP>; \
    case 2560610: return K<DT, FE, 256, 6, kGlobalFlow | kGlobalP>; \
    case 2560810: return K<DT, FE, 256, 8, kGlobalFlow | kGlobalP>; \
    case 2561210: return K<DT, FE, 256, 12, kGlobalFlow | kGlobalP>; \
    case 2561610: return K<DT, FE, 256, 16, kGlobalFlow | kGlobalP>; \
    case 2562410: return K<DT, FE, 256, 24, kGlobalFlow | kGlobalP>; \
    case 5120410: return K<DT, FE, 512, 4, kGlobalFlow | kGlobalP>; \
    case 5120810: return K<DT, FE, 512, 8, kGlobalFlow | kGlobalP>; \
    case 5121210: return K<DT, FE, 512, 12, kGlobalFlow | kGlobalP>; \
    case 5121610: return K<DT, FE, 512, 16, kGlobalFlow | kGlobalP>; \
    case 5122010: return K<DT, FE, 512, 20, kGlobalFlow | kGlobalP>; \
    case 5122410: return K<DT, FE, 512, 24, kGlobalFlow | kGlobalP>; \
    case 5122610: return K<DT, FE, 512, 26, kGlobalFlow | kGlobalP>; \
    case 10240810: return K<DT, FE, 1024, 8, kGlobalFlow | kGlobalP>; \
    case 10241210: return K<DT, FE, 1024, 12, kGlobalFlow | kGlobalP>; \
    case 10241610: return K<DT, FE, 1024, 16, kGlobalFlow | kGlobalP>; \
    case 10242010: return K<DT, FE, 1024, 20, kGlobalFlow | kGlobalP>; \
    case 10244011: return K<DT, FE, 1024, 40, kGlobalDelta | kGlobalFlow | kGlobalP>; \
    default: return nullptr;                          \
  }

WalkKernelFn walk_kernel_i64_f64p(int nt, int maxpt, int store) {
  using DT = int64_t;
  using FE = int64_t;
  QAP_PLANS(walk_kernel)
}

#undef QAP_PLANS

}  // namespace qapk
