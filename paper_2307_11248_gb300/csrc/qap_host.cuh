// Host-side helpers shared by the C-ABI entry points (qap_api.cu) and the
// serving loop (qap_server.cu): instance inspection and upload images, launch
// planning, argument marshalling and output buffers.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/qap.h"
#include "qap_kernels.cuh"

namespace qapk {
WalkKernelFn walk_kernel_i32_f8(int nt, int maxpt, int store);
WalkKernelFn walk_kernel_i32_f8m(int nt, int maxpt, int store);
WalkKernelFn walk_kernel_i32_f16(int nt, int maxpt, int store);
WalkKernelFn walk_kernel_i64_f16(int nt, int maxpt, int store);
WalkKernelFn walk_kernel_i64_f64(int nt, int maxpt, int store);
BatchKernelFn batch_kernel_i32_f8(int nt, int maxpt, int store);
BatchKernelFn batch_kernel_i32_f8m(int nt, int maxpt, int store);
BatchKernelFn batch_kernel_i32_f16(int nt, int maxpt, int store);
BatchKernelFn batch_kernel_i64_f16(int nt, int maxpt, int store);
BatchKernelFn batch_kernel_i64_f64(int nt, int maxpt, int store);
}  // namespace qapk

namespace qaph {

// Detail of the last QAP_ECUDA (per host thread).
extern thread_local char g_last_error[256];

inline qap_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
  return QAP_ECUDA;
}

#define QAP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

#define QAP_TRY(call)                  \
  do {                                 \
    qap_status s_ = (call);            \
    if (s_ != QAP_OK) return s_;       \
  } while (0)

// Largest n: keys pack (r << 8 | s) into 16 bits.
inline constexpr int kMaxN = 256;

struct Plan {
  int nt;
  int maxpt;
  int store;  // qapk::kGlobalDelta, kGlobalFlow, kProductM, kGlobalP bits (0: all on chip)
};

// The large-n plan: 1024 threads, up to 40 slots each in a global workspace
// (row_segments(256, 40) = 945).
inline constexpr Plan kLargePlan = {1024, 40, qapk::kGlobalDelta};

// Register plans (threads per walk, pair slots per thread) compiled into the
// library.  A plan fits n when its row segments (qapk::row_segments) number
// at most its threads.  The automatic choice takes the fewest threads that fit
// with at most eight slots, or 512 threads with any slot count (measured
// 18-55 % faster than 1024 threads where both fit, n = 90..100), else the
// fewest threads that fit at all; for a given thread count the fewest slots
// that fit.  With walks enough for two CTAs on every SM it also takes 256
// threads with any slot count, when two of them fit an SM's shared memory:
// two walks per SM then beat one at 512 threads (1216 walks: n = 80
// asymmetric 9.1 vs 11.5 ms, n = 100 12.4 vs 14.6 ms, grid100 38.3 vs
// 45.7 ms, int64 n = 100 16.2 vs 18.8 ms).
inline constexpr Plan kPlans[] = {{128, 4, 0},   {128, 12, 0},  {256, 6, 0},   {256, 8, 0},
                       {256, 12, 0},  {256, 16, 0},  {256, 24, 0},
                       {512, 4, 0},   {512, 8, 0},   {512, 12, 0},  {512, 16, 0},
                       {512, 20, 0},  {512, 24, 0},  {512, 26, 0},  {1024, 8, 0},  {1024, 12, 0},
                       {1024, 16, 0}, {1024, 20, 0}};

inline bool plan_for(int n, int nt, Plan* out) {
  for (const Plan& p : kPlans)
    if (p.nt == nt && qapk::row_segments(n, p.maxpt) <= nt) {
      *out = p;
      return true;
    }
  return false;
}

inline bool choose_plan(int n, int threads, bool many, Plan* out) {
  if (threads != 0) return plan_for(n, threads, out);
  for (int pass = 0; pass < 2; ++pass)
    for (int nt : {128, 256, 512, 1024}) {
      Plan p;
      if (plan_for(n, nt, &p) &&
          (pass == 1 || p.maxpt <= 8 || nt == 512 || (many && nt == 256))) {
        *out = p;
        return true;
      }
    }
  return false;
}

// Widest power-of-two group (<= 8 lanes, <= the row chunks) that still gives
// every index of phase X its own group.
inline int group_for(int n, int nt, int fbytes) {
  const int w = 16 / fbytes;
  const int nc = (n + w - 1) / w;
  int g = 8;
  while (g > 1 && (nt / g < n || g > nc)) g >>= 1;
  return g;
}

// One instance's shape on the device: F, F^T in `fbytes` elements with rows
// of an odd number of 16-byte chunks (rows read side by side by the lanes of
// a warp then fall in different banks), D and P in `pbytes_of(fbytes)`.
struct DevInstance {
  int n = 0, ldF = 0, ldP = 0, symF = 0, symD = 0;
  int64_t bound = 0;
  int64_t maxF = 0;
  int bytevec = 0;  // every difference of two F entries, and of two D entries, fits int8
  int diff16 = 0;   // every difference of two F entries fits int16, of two D entries int8
  int wide = 0;     // outside the narrow paths: int64 elements and arithmetic
};

// Largest bound of the int64 path.  With B = (n^2 + 8n + 32) max|F| max|D|
// below 2^62, every cost (at most n^2 max|F| max|D|), delta, dot-product sum
// and element product is below 2^62 in magnitude, and so is the difference
// of two costs below 2^63 (the aspiration test compares a delta with it).
inline constexpr int64_t kMaxBound = (int64_t)1 << 62;

// Element width of F on the device: int8 (dp4a rows, byte vectors for the
// O(1) update) when the instance allows it and the deltas are int32; int16
// on the narrow path otherwise; 8 (int64 F, D and P) on the wide path.
inline int flow_bytes(const DevInstance& di, int dbytes) {
  if (di.wide) return 8;
  return (di.bytevec && dbytes == 4) ? 1 : 2;
}

// P and D are int8 beside int8 or int16 flows and int64 beside int64 flows.
inline int pbytes_of(int fbytes) { return fbytes == 8 ? 8 : 1; }

inline int pad_ldF(int n, int fbytes) { return (16 / fbytes) * (((n * fbytes + 15) / 16) | 1); }
inline int pad_ldP(int n, int pbytes) { return (16 / pbytes) * (((n * pbytes + 15) / 16) | 1); }

// Checks ranges and symmetry of one instance and picks its arithmetic:
//  - narrow (int8 or int16 flows, int8 distances, 32-bit element sums) when
//    F fits int16, D fits int8 and every dot product of two length-n rows
//    pairs, 2 n max|F| max|D|, stays below 2^31;
//  - wide (int64 elements and arithmetic) otherwise;
//  - QAP_EOVERFLOW when B = (n^2 + 8n + 32) max|F| max|D| reaches 2^62.
inline qap_status inspect_instance(const int64_t* F, const int64_t* D, int n, DevInstance* di) {
  if (!F || !D || n < 2) return QAP_EINVAL;
  if (n > kMaxN) return QAP_EUNSUPPORTED;
  uint64_t mF = 0, mD = 0;  // magnitudes (|INT64_MIN| included)
  int64_t loF = F[0], hiF = F[0], loD = D[0], hiD = D[0];
  int symF = 1, symD = 1;
  auto mag = [](int64_t v) { return v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v; };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int64_t f = F[(size_t)i * n + j], d = D[(size_t)i * n + j];
      mF = std::max(mF, mag(f));
      mD = std::max(mD, mag(d));
      loF = std::min(loF, f);
      hiF = std::max(hiF, f);
      loD = std::min(loD, d);
      hiD = std::max(hiD, d);
      if (f != F[(size_t)j * n + i]) symF = 0;
      if (d != D[(size_t)j * n + i]) symD = 0;
    }
  const unsigned __int128 nn = (unsigned)n;
  const unsigned __int128 B = (nn * nn + 8 * nn + 32) * (unsigned __int128)mF * mD;
  if (B >= (unsigned __int128)kMaxBound) return QAP_EOVERFLOW;
  const bool in16 = loF >= INT16_MIN && hiF <= INT16_MAX && loD >= INT8_MIN && hiD <= INT8_MAX;
  const unsigned __int128 dots = 2 * nn * (unsigned __int128)mF * mD;
  di->n = n;
  di->symF = symF;
  di->symD = symD;
  di->bound = (int64_t)B;
  di->maxF = (int64_t)mF;
  di->wide = !(in16 && dots <= (unsigned __int128)INT32_MAX);
  // differences of two F entries and of two D entries fit a byte (no
  // overflow here: on this branch the ranges fit int16 and int8)
  di->bytevec = !di->wide && mF <= 127 && hiF - loF <= 127 && hiD - loD <= 127;
  di->diff16 = !di->wide && hiF - loF <= 32767 && hiD - loD <= 127;
  return QAP_OK;
}

// Host images of F, F^T and D for the chosen element width.
inline void build_images(const int64_t* F, const int64_t* D, const DevInstance& di, int fbytes,
                  std::vector<unsigned char>& img_F, std::vector<unsigned char>& img_Ft,
                  std::vector<unsigned char>& img_D) {
  const int n = di.n, ld = di.ldF;
  const int pbytes = pbytes_of(fbytes);
  img_F.assign((size_t)n * ld * fbytes, 0);
  img_Ft.assign((size_t)n * ld * fbytes, 0);
  img_D.resize((size_t)n * n * pbytes);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int64_t f = F[(size_t)i * n + j];
      if (fbytes == 1) {
        reinterpret_cast<int8_t*>(img_F.data())[(size_t)i * ld + j] = (int8_t)f;
        reinterpret_cast<int8_t*>(img_Ft.data())[(size_t)j * ld + i] = (int8_t)f;
      } else if (fbytes == 2) {
        reinterpret_cast<int16_t*>(img_F.data())[(size_t)i * ld + j] = (int16_t)f;
        reinterpret_cast<int16_t*>(img_Ft.data())[(size_t)j * ld + i] = (int16_t)f;
      } else {
        reinterpret_cast<int64_t*>(img_F.data())[(size_t)i * ld + j] = f;
        reinterpret_cast<int64_t*>(img_Ft.data())[(size_t)j * ld + i] = f;
      }
      const int64_t d = D[(size_t)i * n + j];
      if (pbytes == 1)
        img_D[(size_t)i * n + j] = (unsigned char)(int8_t)d;
      else
        reinterpret_cast<int64_t*>(img_D.data())[(size_t)i * n + j] = d;
    }
}

inline qap_status device_attrs(int* device, int* sms, int* smem_optin) {
  QAP_CUDA(cudaGetDevice(device));
  QAP_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *device));
  QAP_CUDA(cudaDeviceGetAttribute(smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, *device));
  return QAP_OK;
}

inline qapk::WalkKernelFn pick_walk_kernel(int dbytes, int fbytes, const Plan& p) {
  if (fbytes == 8) return qapk::walk_kernel_i64_f64(p.nt, p.maxpt, p.store);
  if (dbytes == 8) return qapk::walk_kernel_i64_f16(p.nt, p.maxpt, p.store);
  if (fbytes == 1) return qapk::walk_kernel_i32_f8(p.nt, p.maxpt, p.store);
  return qapk::walk_kernel_i32_f16(p.nt, p.maxpt, p.store);
}

inline qapk::BatchKernelFn pick_batch_kernel(int dbytes, int fbytes, const Plan& p) {
  if (fbytes == 8) return qapk::batch_kernel_i64_f64(p.nt, p.maxpt, p.store);
  if (dbytes == 8) return qapk::batch_kernel_i64_f16(p.nt, p.maxpt, p.store);
  if (fbytes == 1) return qapk::batch_kernel_i32_f8(p.nt, p.maxpt, p.store);
  return qapk::batch_kernel_i32_f16(p.nt, p.maxpt, p.store);
}

// Shared memory of a plan for the instance shapes `d` (the largest over them).
inline int plan_smem(const Plan& p, const DevInstance* d, int count, int fbytes, int dbytes) {
  int smem = 0;
  for (int i = 0; i < count; ++i)
    smem = std::max(smem, qapk::smem_layout(d[i].n, d[i].ldF, fbytes, d[i].ldP, d[i].symF,
                                            d[i].symD, dbytes, p.nt * p.maxpt, p.store)
                              .bytes);
  return smem;
}

// Register plans compiled with the maintained products M (int8 and int16
// flows): up to 24 slots (12 at 1024 threads), and 512 x 26 for int16 flows.
// Measured against the dot products at 24 slots: the n = 100 grid 153.5 ->
// 150.9 ms per step, asymmetric n = 96 (2 walks per SM) 14.2 -> 12.8 ms,
// n = 135 at 512 x 24 15.0 -> 13.2 ms; at 26 slots symmetric int8 n = 148
// was slower (14.0 -> 14.3 ms), the int16 batch512 classes faster (step
// 2799.6 -> 2782.4 ms).
inline bool has_product_form(const Plan& p, int fbytes) {
  if (p.store != 0) return false;
  if (p.nt == 512 && p.maxpt == 26) return fbytes == 2;
  return p.nt == 1024 ? p.maxpt <= 12 : p.maxpt <= 24;
}

// Products plans also compiled without the transposed copies of F and P
// (kNoTransposed): the plans of the larger n, where M may not fit beside
// them on asymmetric instances.
inline bool has_notrans_form(const Plan& p, int fbytes) {
  return has_product_form(p, fbytes) && p.maxpt >= 12 && (p.nt == 256 || p.nt == 512);
}

// The form a plan reports: 0 dot products, 1 maintained products, 2 the
// same without the transposed copies of F and P.
inline int products_form(const Plan& p) {
  return !(p.store & qapk::kProductM) ? 0 : (p.store & qapk::kNoTransposed) ? 2 : 1;
}

// The products form of a register plan when the flows are stored as int8 or
// int16 and M fits shared memory too (phase X then reads M instead of
// computing dot products), unless the caller asks for the dot products.
// Measured with 2 walks per SM, 4000 iterations: asymmetric n = 60 / 70 /
// 80 8.4 / 10.4 / 12.9 ms against 10.3 / 11.0 / 13.4 for symmetric ones by
// dot products; symmetric n = 50 / 60 / 70 / 80 by products 6.7 / 8.4 /
// 10.3 / 12.7 ms; n = 100 at 512 x 12 symmetric 10.2 against 12.1 ms.
// Where M does not fit beside the transposed copies (or would keep two
// walks from sharing an SM where the plan was taken for that), the form
// without the copies.  `fits` says whether a plan fits.
template <typename Fits>
inline Plan with_products(Plan p, int fbytes, int form, Fits fits) {
  if (form == QAP_PHASE_X_DOTS || fbytes == 8 || !has_product_form(p, fbytes)) return p;
  Plan m = p;
  m.store |= qapk::kProductM;
  if (fits(m)) return m;
  if (!has_notrans_form(p, fbytes)) return p;
  m.store |= qapk::kNoTransposed;
  return fits(m) ? m : p;
}

// The int64 element path reads F and F^T from global memory (L1-cached,
// read-only), and keeps P and P^T in the CTA's workspace too when they do
// not fit shared memory.
inline Plan wide_store(Plan p, const DevInstance* d, int count, int fbytes, int dbytes,
                       int smem_optin, int reserve) {
  if (fbytes != 8) return p;
  p.store |= qapk::kGlobalFlow;
  if (plan_smem(p, d, count, fbytes, dbytes) + reserve > smem_optin) p.store |= qapk::kGlobalP;
  return p;
}

// A register plan when one holds n and fits shared memory (in its products
// form when that fits as well); else the large-n plan, with F in global
// memory when it does not fit shared memory either.  `many`: the launch has
// walks enough for two CTAs on every SM (see choose_plan); a 256-thread plan
// taken for that alone must let two CTAs share an SM (without the products
// form if need be), else the choice is made as without `many`.
inline bool choose_plan_fit(int nmax, int threads, bool many, const DevInstance* d, int count,
                            int fbytes, int dbytes, int smem_optin, int reserve, int form,
                            Plan* out) {
  Plan p;
  if (nmax <= 181 && choose_plan(nmax, threads, many, &p)) {
    p = wide_store(p, d, count, fbytes, dbytes, smem_optin, reserve);
    if (plan_smem(p, d, count, fbytes, dbytes) + reserve <= smem_optin) {
      const bool need_two = many && threads == 0 && p.nt == 256 && p.maxpt > 8;
      // two CTAs per SM: each with its own 1 KB reserved by the hardware
      auto two = [&](const Plan& x) {
        return 2 * (plan_smem(x, d, count, fbytes, dbytes) + reserve + 1024) <=
               smem_optin + 1024;
      };
      if (need_two && !two(p))
        return choose_plan_fit(nmax, threads, false, d, count, fbytes, dbytes, smem_optin,
                               reserve, form, out);
      *out = with_products(p, fbytes, form, [&](const Plan& x) {
        return plan_smem(x, d, count, fbytes, dbytes) + reserve <= smem_optin &&
               (!need_two || two(x));
      });
      return true;
    }
  }
  if (threads != 0 && threads != kLargePlan.nt) return false;
  if (qapk::row_segments(nmax, kLargePlan.maxpt) > kLargePlan.nt) return false;
  p = kLargePlan;
  if (fbytes == 8)
    p = wide_store(p, d, count, fbytes, dbytes, smem_optin, reserve);
  else if (plan_smem(p, d, count, fbytes, dbytes) + reserve > smem_optin)
    p.store |= qapk::kGlobalFlow;
  if (plan_smem(p, d, count, fbytes, dbytes) + reserve > smem_optin) return false;
  *out = p;
  return true;
}

// Per-CTA workspace: the deltas and marks of large-n plans, then P and P^T
// of kGlobalP plans (sized for the largest n), then the tables of the other
// tabu criteria and of the frequency penalty when a search uses them
// (loc_until n x n, unit_until n, applied n x n; int32).
inline size_t delta_workspace(const Plan& p, int dbytes) {
  if (!(p.store & qapk::kGlobalDelta)) return 0;
  const size_t b = (size_t)p.nt * p.maxpt * ((size_t)dbytes + 4);
  return (b + 255) / 256 * 256;
}

inline size_t p_workspace(const Plan& p, int fbytes, int nmax) {
  if (!(p.store & qapk::kGlobalP)) return 0;
  const int pb = pbytes_of(fbytes);
  const size_t b = 2 * (size_t)nmax * pad_ldP(nmax, pb) * pb;
  return (b + 255) / 256 * 256;
}

inline bool uses_rule_tables(const qap_search_params* sp) {
  return sp->iters > 0 && (sp->criterion != QAP_TABU_PAIR || sp->freq_penalty != 0);
}

struct WsLayout {
  size_t p_off;    // P, P^T (kGlobalP plans)
  size_t rws_off;  // tables of the other criteria and of the penalty
  size_t stride;   // bytes per CTA (0: no workspace)
};

inline WsLayout ws_layout(const Plan& p, int dbytes, int fbytes, int nmax,
                          const qap_search_params* sp) {
  WsLayout w;
  w.p_off = delta_workspace(p, dbytes);
  w.rws_off = w.p_off + p_workspace(p, fbytes, nmax);
  w.stride = w.rws_off;
  if (uses_rule_tables(sp)) w.stride += ((size_t)(2 * nmax * nmax + nmax) * 4 + 255) / 256 * 256;
  return w;
}

// With the frequency penalty a non-improving move's rank is delta + lambda *
// count, count <= iters; int32 deltas must hold it below their sentinel, int64
// deltas below the int64 path's bound.
inline qap_status check_penalty(const qap_search_params* sp, int dbytes, int64_t bound) {
  if (sp->freq_penalty == 0 || sp->iters == 0) return QAP_OK;
  const int64_t top = bound + (int64_t)sp->freq_penalty * sp->iters;  // < 2^62 + 2^62
  if (dbytes == 8) return top < kMaxBound ? QAP_OK : QAP_EOVERFLOW;
  return top < (int64_t)INT32_MAX - 1 ? QAP_OK : QAP_EOVERFLOW;
}

extern std::mutex g_attr_mu;

// Makes a device current for the length of an entry point and gives the
// caller's current device back on return, so that a call never leaves the
// calling thread on another device.
class DeviceGuard {
 public:
  DeviceGuard() = default;
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  qap_status set(int device) {
    QAP_CUDA(cudaGetDevice(&prev_));
    if (prev_ != device) {
      QAP_CUDA(cudaSetDevice(device));
      changed_ = true;
    }
    return QAP_OK;
  }
  ~DeviceGuard() {
    if (changed_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = 0;
  bool changed_ = false;
};

// Kernels whose dynamic shared-memory limit has been raised, per device: a
// fixed table, so that the check allocates nothing.  When it is full the
// attribute is simply set again on every launch (an idempotent call).
inline constexpr int kPreparedMax = 1024;
struct PreparedKernel {
  const void* fn;
  int device;
};
extern PreparedKernel g_prepared[kPreparedMax];
extern int g_prepared_count;

inline qap_status prepare_kernel(const void* fn, int smem) {
  // The dynamic shared-memory limit is a property of the function, shared
  // by every launch of it from any thread; raise it once to the device
  // maximum so that no launch can find it lowered by a smaller request.
  std::lock_guard<std::mutex> lk(g_attr_mu);
  int dev = 0, optin = 0;
  QAP_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < g_prepared_count; ++i)
    if (g_prepared[i].fn == fn && g_prepared[i].device == dev) return QAP_OK;
  QAP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  QAP_CUDA(cudaFuncGetAttributes(&fa, fn));
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // the static part counts too
  if (smem > dyn_max) return QAP_EUNSUPPORTED;
  QAP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  if (g_prepared_count < kPreparedMax) g_prepared[g_prepared_count++] = PreparedKernel{fn, dev};
  return QAP_OK;
}

inline qap_status validate_params(const qap_search_params* p) {
  if (!p) return QAP_EINVAL;
  if (p->starts < 1 || p->iters < 0) return QAP_EINVAL;
  if (p->descend != 0 && p->descend != 1) return QAP_EINVAL;
  if (p->aspiration != 0 && p->aspiration != 1) return QAP_EINVAL;
  if (p->iters > 0) {
    if (p->tenure.tmin < 1 || p->tenure.tmax < p->tenure.tmin || p->tenure.period < 0)
      return QAP_EINVAL;
    // tabu_until = it + t must stay below INT_MAX
    if ((int64_t)p->iters + (int64_t)p->tenure.tmax >= (int64_t)INT_MAX) return QAP_EINVAL;
  }
  if (p->launch != QAP_LAUNCH_PERSISTENT && p->launch != QAP_LAUNCH_PLAIN) return QAP_EINVAL;
  if (p->criterion < QAP_TABU_PAIR || p->criterion > QAP_TABU_UNIT || p->freq_penalty < 0)
    return QAP_EINVAL;
  if (p->tenure_per_n != 0 && p->tenure_per_n != 1) return QAP_EINVAL;
  // the kernel forms tmax * n + 99 and period * n in 32-bit integers
  if (p->tenure_per_n && p->iters > 0 &&
      ((int64_t)p->tenure.tmax * kMaxN + 99 > (int64_t)INT_MAX ||
       (int64_t)p->tenure.period * kMaxN > (int64_t)INT_MAX ||
       (int64_t)p->tenure.tmax * kMaxN / 100 + 1 + p->iters >= (int64_t)INT_MAX))
    return QAP_EINVAL;
  const int t = p->threads_per_walk;
  if (t != 0 && t != 128 && t != 256 && t != 512 && t != 1024) return QAP_EINVAL;
  if (p->phase_x != QAP_PHASE_X_AUTO && p->phase_x != QAP_PHASE_X_DOTS) return QAP_EINVAL;
  return QAP_OK;
}

inline qapk::SearchArgs make_search_args(const qap_search_params* p, const qap_walk_outputs* o,
                                  int p_stride) {
  qapk::SearchArgs a{};
  a.walk_base = p->walk_base;
  a.seed = p->seed;
  a.descend = p->descend;
  a.max_descent = p->max_descent;
  a.iters = p->iters;
  a.tmin = p->tenure.tmin;
  a.tmax = p->tenure.tmax;
  a.period = p->tenure.period;
  a.aspiration = p->aspiration;
  a.tenure_per_n = p->tenure_per_n;
  a.crit = p->criterion;
  a.lambda = p->freq_penalty;
  a.p_stride = p_stride;
  a.best_p = o->best_p;
  a.best_cost = o->best_cost;
  a.final_cost = o->final_cost;
  a.best_iter = o->best_iter;
  a.iters_done = o->iters_done;
  a.status = o->status;
  a.descent_moves = o->descent_moves;
  a.hash = o->hash;
  a.descent_hash = o->descent_hash;
  a.freq = o->freq;
  return a;
}

inline bool is_permutation(const int32_t* p, int n, std::vector<char>& seen) {
  seen.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    if (p[i] < 0 || p[i] >= n || seen[p[i]]) return false;
    seen[p[i]] = 1;
  }
  return true;
}

inline qap_status grow(void** buf, size_t* have, size_t bytes) {
  if (bytes <= *have) return QAP_OK;
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(buf, bytes);
  if (e == cudaErrorMemoryAllocation) return QAP_ENOMEM;
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  *have = bytes;
  return QAP_OK;
}

// Device outputs of W walks carved from one buffer; rows of best_p hold
// p_stride elements.
struct OutLayout {
  size_t off_p, off_i64, off_i32, total;
};

inline OutLayout out_layout(int W, int p_stride) {
  OutLayout L;
  const size_t perm = (size_t)W * p_stride * sizeof(int32_t);
  L.off_p = 0;
  L.off_i64 = (perm + 255) / 256 * 256;
  L.off_i32 = L.off_i64 + (size_t)4 * W * 8;
  L.total = L.off_i32 + (size_t)4 * W * 4 + 256;
  return L;
}

inline qap_walk_outputs carve_outputs(char* base, const OutLayout& L, int W) {
  qap_walk_outputs d{};
  d.best_p = reinterpret_cast<int32_t*>(base + L.off_p);
  int64_t* i64 = reinterpret_cast<int64_t*>(base + L.off_i64);
  int32_t* i32 = reinterpret_cast<int32_t*>(base + L.off_i32);
  d.best_cost = i64;
  d.final_cost = i64 + W;
  d.hash = reinterpret_cast<uint64_t*>(i64 + 2 * W);
  d.descent_hash = reinterpret_cast<uint64_t*>(i64 + 3 * W);
  d.best_iter = i32;
  d.iters_done = i32 + W;
  d.status = i32 + 2 * W;
  d.descent_moves = i32 + 3 * W;
  return d;
}

inline qap_status copy_outputs_back(const qap_walk_outputs* out, const qap_walk_outputs& d, int W,
                             int p_stride, cudaStream_t s) {
  auto d2h = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
  };
  QAP_CUDA(d2h(out->best_p, d.best_p, (size_t)W * p_stride * 4));
  QAP_CUDA(d2h(out->best_cost, d.best_cost, (size_t)W * 8));
  QAP_CUDA(d2h(out->final_cost, d.final_cost, (size_t)W * 8));
  QAP_CUDA(d2h(out->hash, d.hash, (size_t)W * 8));
  QAP_CUDA(d2h(out->descent_hash, d.descent_hash, (size_t)W * 8));
  QAP_CUDA(d2h(out->best_iter, d.best_iter, (size_t)W * 4));
  QAP_CUDA(d2h(out->iters_done, d.iters_done, (size_t)W * 4));
  QAP_CUDA(d2h(out->status, d.status, (size_t)W * 4));
  QAP_CUDA(d2h(out->descent_moves, d.descent_moves, (size_t)W * 4));
  QAP_CUDA(d2h(out->freq, d.freq, (size_t)W * p_stride * p_stride * 4));
  QAP_CUDA(cudaStreamSynchronize(s));
  return QAP_OK;
}

inline qapk::InstArgs inst_args(const DevInstance& d, const void* F, const void* Ft, const void* D,
                                int nt, int fbytes) {
  qapk::InstArgs I{};
  I.n = d.n;
  I.ldF = d.ldF;
  I.ldP = d.ldP;
  I.symF = d.symF;
  I.symD = d.symD;
  I.group = group_for(d.n, nt, fbytes);
  I.diff16 = d.diff16;
  I.F = F;
  I.Ft = d.symF ? F : Ft;
  I.D = D;
  return I;
}

}  // namespace qaph
