// Instantiations of the batch_kernels with int64 deltas and int64 flows and
// distances (the wide element path: F and F^T read from global memory, P in
// shared memory); the plans with P in the workspace are in
// qap_batch_i64_f64p.cu.  One translation unit per combination so they
// compile in parallel.
#include "qap_kernels.cuh"

namespace qapk {

BatchKernelFn batch_kernel_i64_f64p(int nt, int maxpt, int store);  // qap_batch_i64_f64p.cu

#define QAP_PLANS(K)                                  \
  switch (nt * 10000 + maxpt * 100 + store) {         \
    case 1280402: return K<DT, FE, 128, 4, kGlobalFlow>; \
    case 1281202: return K<DT, FE, 128, 12, kGlobalFlow>; \
    case 2560602: return K<DT, FE, 256, 6, kGlobalFlow>; \
    case 2560802: return K<DT, FE, 256, 8, kGlobalFlow>; \
    case 2561202: return K<DT, FE, 256, 12, kGlobalFlow>; \
    case 2561602: return K<DT, FE, 256, 16, kGlobalFlow>; \
    case 2562402: return K<DT, FE, 256, 24, kGlobalFlow>; \
    case 5120402: return K<DT, FE, 512, 4, kGlobalFlow>; \
    case 5120802: return K<DT, FE, 512, 8, kGlobalFlow>; \
    case 5121202: return K<DT, FE, 512, 12, kGlobalFlow>; \
    case 5121602: return K<DT, FE, 512, 16, kGlobalFlow>; \
    case 5122002: return K<DT, FE, 512, 20, kGlobalFlow>; \
    case 5122402: return K<DT, FE, 512, 24, kGlobalFlow>; \
    case 5122602: return K<DT, FE, 512, 26, kGlobalFlow>; \
    case 10240802: return K<DT, FE, 1024, 8, kGlobalFlow>; \
    case 10241202: return K<DT, FE, 1024, 12, kGlobalFlow>; \
    case 10241602: return K<DT, FE, 1024, 16, kGlobalFlow>; \
    case 10242002: return K<DT, FE, 1024, 20, kGlobalFlow>; \
    case 10244003: return K<DT, FE, 1024, 40, kGlobalDelta | kGlobalFlow>; \
    default: return nullptr;                          \
  }

BatchKernelFn batch_kernel_i64_f64(int nt, int maxpt, int store) {
  using DT = int64_t;
  using FE = int64_t;
  if (store & kGlobalP) return batch_kernel_i64_f64p(nt, maxpt, store);
  QAP_PLANS(batch_kernel)
}

#undef QAP_PLANS

}  // namespace qapk
