// C-ABI of the QAP search library: instance upload, validation, launch
// planning and the blocking / stream-ordered search entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/qap.h"
#include "qap_kernels.cuh"

namespace qapk {
WalkKernelFn walk_kernel_i32_f8(int nt, int maxpt);
WalkKernelFn walk_kernel_i32_f16(int nt, int maxpt);
WalkKernelFn walk_kernel_i64_f16(int nt, int maxpt);
}  // namespace qapk

namespace {

thread_local char g_last_error[256] = "";

qap_status cuda_fail(cudaError_t e, const char* where) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
  return QAP_ECUDA;
}

#define QAP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Largest n: keys pack (r << 8 | s), and the largest register plan holds
// 16 pairs per thread for 1024 threads.
constexpr int kMaxN = 181;

struct Plan {
  int nt;
  int maxpt;
};

}  // namespace

struct qap_ctx {
  int device = 0;
  int n = 0, ldF = 0, ldP = 0;
  int symF = 0, symD = 0;
  int dbytes = 4;  // delta width
  int fbytes = 2;  // flow element width in device memory (1: int8, 2: int16)
  int64_t bound = 0;
  int sms = 0;
  int smem_optin = 0;
  void* dF = nullptr;
  void* dFt = nullptr;
  int8_t* dD = nullptr;
  cudaStream_t stream = nullptr;
  // growable device buffers for the blocking entry points
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
};

namespace {

using KernelFn = qapk::WalkKernelFn;

// Register plans (threads per walk, pair slots per thread) compiled into the
// library.  A plan fits n when its row segments (qapk::row_segments) number
// at most its threads.  The automatic choice takes the fewest threads that fit
// with at most eight slots, else the fewest threads that fit at all; for a
// given thread count the fewest slots that fit.
const Plan kPlans[] = {{128, 4},  {128, 12}, {256, 6},  {256, 8},   {512, 4},
                       {512, 8},  {512, 12}, {1024, 8}, {1024, 12}, {1024, 16},
                       {1024, 20}};

bool plan_for(int n, int nt, Plan* out) {
  for (const Plan& p : kPlans)
    if (p.nt == nt && qapk::row_segments(n, p.maxpt) <= nt) {
      *out = p;
      return true;
    }
  return false;
}

bool choose_plan(int n, int threads, Plan* out) {
  if (threads != 0) return plan_for(n, threads, out);
  for (int pass = 0; pass < 2; ++pass)
    for (int nt : {128, 256, 512, 1024}) {
      Plan p;
      if (plan_for(n, nt, &p) && (pass == 1 || p.maxpt <= 8)) {
        *out = p;
        return true;
      }
    }
  return false;
}

KernelFn pick_kernel(const qap_ctx* ctx, const Plan& p) {
  if (ctx->dbytes == 8) return qapk::walk_kernel_i64_f16(p.nt, p.maxpt);
  if (ctx->fbytes == 1) return qapk::walk_kernel_i32_f8(p.nt, p.maxpt);
  return qapk::walk_kernel_i32_f16(p.nt, p.maxpt);
}

std::mutex g_attr_mu;

qap_status prepare_kernel(KernelFn fn, int smem) {
  // cudaFuncSetAttribute is idempotent; serialise to keep it cheap and safe.
  std::lock_guard<std::mutex> lk(g_attr_mu);
  QAP_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  return QAP_OK;
}

struct Launch {
  KernelFn fn;
  Plan plan;
  int group;  // lanes per recompute task
  int smem;
  int ctas_per_sm;
  int grid;
};

qap_status validate_params(const qap_ctx* ctx, const qap_search_params* p) {
  if (!ctx || !p) return QAP_EINVAL;
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
  const int t = p->threads_per_walk;
  if (t != 0 && t != 128 && t != 256 && t != 512 && t != 1024) return QAP_EINVAL;
  return QAP_OK;
}

qap_status plan_launch(qap_ctx* ctx, const qap_search_params* p, Launch* L) {
  if (!choose_plan(ctx->n, p->threads_per_walk, &L->plan)) return QAP_EUNSUPPORTED;
  L->fn = pick_kernel(ctx, L->plan);
  if (!L->fn) return QAP_EUNSUPPORTED;
  const qapk::SmemLayout S =
      qapk::smem_layout(ctx->n, ctx->ldF, ctx->fbytes, ctx->ldP, ctx->symF, ctx->symD,
                        ctx->dbytes, L->plan.nt * L->plan.maxpt);
  L->smem = S.bytes;
  if (L->smem > ctx->smem_optin) return QAP_EUNSUPPORTED;
  qap_status st = prepare_kernel(L->fn, L->smem);
  if (st != QAP_OK) return st;
  int occ = 0;
  QAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, reinterpret_cast<const void*>(L->fn), L->plan.nt, L->smem));
  if (occ < 1) return QAP_EUNSUPPORTED;
  L->ctas_per_sm = occ;
  L->grid = std::min(p->starts, occ * ctx->sms);
  // widest power-of-two group (<= 8 lanes, <= the row chunks) that still
  // gives every index of phase X its own group
  const int nc = (ctx->n + 16 / ctx->fbytes - 1) / (16 / ctx->fbytes);
  L->group = 8;
  while (L->group > 1 && (L->plan.nt / L->group < ctx->n || L->group > nc)) L->group >>= 1;
  return QAP_OK;
}

qapk::WalkArgs make_args(const qap_ctx* ctx, const qap_search_params* p, const int32_t* d_starts,
                         const qap_walk_outputs* o) {
  qapk::WalkArgs a{};
  a.n = ctx->n;
  a.ldF = ctx->ldF;
  a.ldP = ctx->ldP;
  a.symF = ctx->symF;
  a.symD = ctx->symD;
  a.F = ctx->dF;
  a.Ft = ctx->symF ? ctx->dF : ctx->dFt;
  a.D = ctx->dD;
  a.walks = p->starts;
  a.walk_offset = 0;
  a.walk_base = p->walk_base;
  a.seed = p->seed;
  a.starts = d_starts;
  a.descend = p->descend;
  a.max_descent = p->max_descent;
  a.iters = p->iters;
  a.tmin = p->tenure.tmin;
  a.tmax = p->tenure.tmax;
  a.period = p->tenure.period;
  a.aspiration = p->aspiration;
  a.best_p = o->best_p;
  a.best_cost = o->best_cost;
  a.final_cost = o->final_cost;
  a.best_iter = o->best_iter;
  a.iters_done = o->iters_done;
  a.status = o->status;
  a.descent_moves = o->descent_moves;
  a.hash = o->hash;
  a.descent_hash = o->descent_hash;
  return a;
}

bool is_permutation(const int32_t* p, int n, std::vector<char>& seen) {
  seen.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    if (p[i] < 0 || p[i] >= n || seen[p[i]]) return false;
    seen[p[i]] = 1;
  }
  return true;
}

qap_status ensure_scratch(qap_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return QAP_OK;
  if (ctx->scratch) {
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->scratch, bytes);
  if (e == cudaErrorMemoryAllocation) return QAP_ENOMEM;
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  ctx->scratch_bytes = bytes;
  return QAP_OK;
}

}  // namespace

extern "C" {

const char* qap_strerror(qap_status s) {
  switch (s) {
    case QAP_OK: return "ok";
    case QAP_EINVAL: return "invalid argument";
    case QAP_EOVERFLOW: return "cost bound exceeds the int64 path";
    case QAP_ENOMEM: return "out of memory";
    case QAP_ECUDA: return "CUDA error";
    case QAP_ETIMEOUT: return "bounded wait timed out";
    case QAP_EUNSUPPORTED: return "instance outside the supported ranges";
  }
  return "unknown status";
}

const char* qap_last_error(void) { return g_last_error; }

qap_status qap_create(const int64_t* F, const int64_t* D, int32_t n, uint32_t flags,
                      qap_ctx** out) {
  if (!out) return QAP_EINVAL;
  *out = nullptr;
  if (!F || !D || n < 2) return QAP_EINVAL;
  if (flags & ~QAP_FORCE_INT64) return QAP_EINVAL;
  if (n > kMaxN) return QAP_EUNSUPPORTED;
  int64_t mF = 0, mD = 0;
  int symF = 1, symD = 1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int64_t f = F[(size_t)i * n + j], d = D[(size_t)i * n + j];
      if (f < INT16_MIN || f > INT16_MAX || d < INT8_MIN || d > INT8_MAX) return QAP_EUNSUPPORTED;
      mF = std::max<int64_t>(mF, f < 0 ? -f : f);
      mD = std::max<int64_t>(mD, d < 0 ? -d : d);
      if (f != F[(size_t)j * n + i]) symF = 0;
      if (d != D[(size_t)j * n + i]) symD = 0;
    }
  const int64_t nn = (int64_t)n;
  const int64_t bound = (nn * nn + 8 * nn + 32) * mF * mD;  // < 2^40 for n <= 181
  qap_ctx* c = new (std::nothrow) qap_ctx();
  if (!c) return QAP_ENOMEM;
  c->n = n;
  c->symF = symF;
  c->symD = symD;
  c->bound = bound;
  c->dbytes = ((flags & QAP_FORCE_INT64) || bound > (int64_t)INT_MAX - 1) ? 8 : 4;
  // int8 flows (dp4a rows) when they fit and deltas are int32; else int16
  c->fbytes = (mF <= 127 && c->dbytes == 4) ? 1 : 2;
  // F rows: an odd number of 16-byte chunks, so rows read side by side by
  // the lanes of a warp fall in different banks
  c->ldF = (16 / c->fbytes) * (((n * c->fbytes + 15) / 16) | 1);
  // P rows: an odd number of 16-byte chunks, so the column exchanges of a
  // move hit 8 different banks per 32 rows instead of 2
  c->ldP = 16 * (((n + 15) / 16) | 1);
  auto fail = [&](qap_status s) {
    qap_destroy(c);
    return s;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
  e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
  const size_t fcount = (size_t)n * c->ldF;
  std::vector<int16_t> hF16, hFt16;
  std::vector<int8_t> hF8, hFt8;
  if (c->fbytes == 1) {
    hF8.assign(fcount, 0);
    hFt8.assign(fcount, 0);
  } else {
    hF16.assign(fcount, 0);
    hFt16.assign(fcount, 0);
  }
  std::vector<int8_t> hD((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int64_t f = F[(size_t)i * n + j];
      if (c->fbytes == 1) {
        hF8[(size_t)i * c->ldF + j] = (int8_t)f;
        hFt8[(size_t)j * c->ldF + i] = (int8_t)f;
      } else {
        hF16[(size_t)i * c->ldF + j] = (int16_t)f;
        hFt16[(size_t)j * c->ldF + i] = (int16_t)f;
      }
      hD[(size_t)i * n + j] = (int8_t)D[(size_t)i * n + j];
    }
  const void* srcF = c->fbytes == 1 ? (const void*)hF8.data() : (const void*)hF16.data();
  const void* srcFt = c->fbytes == 1 ? (const void*)hFt8.data() : (const void*)hFt16.data();
  const size_t fbytes = fcount * c->fbytes;
  if (cudaMalloc(&c->dF, fbytes) != cudaSuccess) return fail(QAP_ENOMEM);
  if (!symF && cudaMalloc(&c->dFt, fbytes) != cudaSuccess) return fail(QAP_ENOMEM);
  if (cudaMalloc(&c->dD, hD.size()) != cudaSuccess) return fail(QAP_ENOMEM);
  e = cudaMemcpy(c->dF, srcF, fbytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !symF) e = cudaMemcpy(c->dFt, srcFt, fbytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->dD, hD.data(), hD.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
  e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreateWithFlags"));
  *out = c;
  return QAP_OK;
}

void qap_destroy(qap_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->dF) cudaFree(ctx->dF);
  if (ctx->dFt) cudaFree(ctx->dFt);
  if (ctx->dD) cudaFree(ctx->dD);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

qap_status qap_info(const qap_ctx* ctx, qap_ctx_info* out) {
  if (!ctx || !out) return QAP_EINVAL;
  out->n = ctx->n;
  out->delta_bytes = ctx->dbytes;
  out->sym_flow = ctx->symF;
  out->sym_dist = ctx->symD;
  out->bound = ctx->bound;
  return QAP_OK;
}

qap_status qap_plan(qap_ctx* ctx, const qap_search_params* params, qap_plan_info* out) {
  qap_status st = validate_params(ctx, params);
  if (st != QAP_OK) return st;
  if (!out) return QAP_EINVAL;
  QAP_CUDA(cudaSetDevice(ctx->device));
  Launch L;
  st = plan_launch(ctx, params, &L);
  if (st != QAP_OK) return st;
  out->threads_per_walk = L.plan.nt;
  out->pairs_per_thread = L.plan.maxpt;
  out->smem_bytes = L.smem;
  out->grid = params->launch == QAP_LAUNCH_PLAIN ? 1 : L.grid;
  out->ctas_per_sm = L.ctas_per_sm;
  out->sms = ctx->sms;
  return QAP_OK;
}

qap_status qap_search_async(qap_ctx* ctx, const qap_search_params* params,
                            const int32_t* d_starts, const qap_walk_outputs* out,
                            void* stream) {
  qap_status st = validate_params(ctx, params);
  if (st != QAP_OK) return st;
  if (!out || !out->best_cost) return QAP_EINVAL;
  QAP_CUDA(cudaSetDevice(ctx->device));
  Launch L;
  st = plan_launch(ctx, params, &L);
  if (st != QAP_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  qapk::WalkArgs a = make_args(ctx, params, d_starts, out);
  a.group = L.group;
  if (params->launch == QAP_LAUNCH_PLAIN) {
    a.walks = 1;
    for (int w = 0; w < params->starts; ++w) {
      a.walk_offset = w;
      L.fn<<<1, L.plan.nt, L.smem, s>>>(a);
    }
  } else {
    L.fn<<<L.grid, L.plan.nt, L.smem, s>>>(a);
  }
  QAP_CUDA(cudaGetLastError());
  return QAP_OK;
}

qap_status qap_search(qap_ctx* ctx, const qap_search_params* params, const int32_t* starts,
                      const qap_walk_outputs* out) {
  qap_status st = validate_params(ctx, params);
  if (st != QAP_OK) return st;
  if (!out || !out->best_cost) return QAP_EINVAL;
  const int n = ctx->n, W = params->starts;
  if (starts) {
    std::vector<char> seen;
    for (int w = 0; w < W; ++w)
      if (!is_permutation(starts + (size_t)w * n, n, seen)) return QAP_EINVAL;
  }
  QAP_CUDA(cudaSetDevice(ctx->device));
  // device layout of the scratch block: starts | best_p | 64-bit outputs | 32-bit outputs
  const size_t perm_bytes = (size_t)W * n * sizeof(int32_t);
  const size_t off_best_p = 0;
  const size_t off_starts = off_best_p + ((perm_bytes + 255) / 256) * 256;
  const size_t off_i64 = off_starts + ((perm_bytes + 255) / 256) * 256;
  const size_t n64 = 4, n32 = 5;
  const size_t off_i32 = off_i64 + n64 * W * 8;
  const size_t total = off_i32 + n32 * W * 4 + 256;
  st = ensure_scratch(ctx, total);
  if (st != QAP_OK) return st;
  char* base = static_cast<char*>(ctx->scratch);
  qap_walk_outputs d{};
  d.best_p = reinterpret_cast<int32_t*>(base + off_best_p);
  int32_t* d_starts = reinterpret_cast<int32_t*>(base + off_starts);
  int64_t* i64 = reinterpret_cast<int64_t*>(base + off_i64);
  int32_t* i32 = reinterpret_cast<int32_t*>(base + off_i32);
  d.best_cost = i64;
  d.final_cost = i64 + W;
  d.hash = reinterpret_cast<uint64_t*>(i64 + 2 * W);
  d.descent_hash = reinterpret_cast<uint64_t*>(i64 + 3 * W);
  d.best_iter = i32;
  d.iters_done = i32 + W;
  d.status = i32 + 2 * W;
  d.descent_moves = i32 + 3 * W;
  cudaStream_t s = ctx->stream;
  if (starts) QAP_CUDA(cudaMemcpyAsync(d_starts, starts, perm_bytes, cudaMemcpyHostToDevice, s));
  st = qap_search_async(ctx, params, starts ? d_starts : nullptr, &d, s);
  if (st != QAP_OK) return st;
  auto d2h = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
  };
  QAP_CUDA(d2h(out->best_p, d.best_p, perm_bytes));
  QAP_CUDA(d2h(out->best_cost, d.best_cost, (size_t)W * 8));
  QAP_CUDA(d2h(out->final_cost, d.final_cost, (size_t)W * 8));
  QAP_CUDA(d2h(out->hash, d.hash, (size_t)W * 8));
  QAP_CUDA(d2h(out->descent_hash, d.descent_hash, (size_t)W * 8));
  QAP_CUDA(d2h(out->best_iter, d.best_iter, (size_t)W * 4));
  QAP_CUDA(d2h(out->iters_done, d.iters_done, (size_t)W * 4));
  QAP_CUDA(d2h(out->status, d.status, (size_t)W * 4));
  QAP_CUDA(d2h(out->descent_moves, d.descent_moves, (size_t)W * 4));
  QAP_CUDA(cudaStreamSynchronize(s));
  return QAP_OK;
}

qap_status qap_cost(qap_ctx* ctx, int32_t count, const int32_t* p, int64_t* cost) {
  if (!ctx || count < 0 || (count > 0 && (!p || !cost))) return QAP_EINVAL;
  if (count == 0) return QAP_OK;
  const int n = ctx->n;
  std::vector<char> seen;
  for (int k = 0; k < count; ++k)
    if (!is_permutation(p + (size_t)k * n, n, seen)) return QAP_EINVAL;
  QAP_CUDA(cudaSetDevice(ctx->device));
  const size_t pbytes = (size_t)count * n * sizeof(int32_t);
  const size_t off_cost = ((pbytes + 255) / 256) * 256;
  qap_status st = ensure_scratch(ctx, off_cost + (size_t)count * 8);
  if (st != QAP_OK) return st;
  char* base = static_cast<char*>(ctx->scratch);
  int32_t* dp = reinterpret_cast<int32_t*>(base);
  int64_t* dc = reinterpret_cast<int64_t*>(base + off_cost);
  cudaStream_t s = ctx->stream;
  QAP_CUDA(cudaMemcpyAsync(dp, p, pbytes, cudaMemcpyHostToDevice, s));
  const int grid = std::min(count, ctx->sms * 8);
  if (ctx->fbytes == 1)
    qapk::cost_kernel<int8_t, 256><<<grid, 256, 0, s>>>(static_cast<const int8_t*>(ctx->dF),
                                                        ctx->ldF, ctx->dD, n, dp, count, dc);
  else
    qapk::cost_kernel<int16_t, 256><<<grid, 256, 0, s>>>(static_cast<const int16_t*>(ctx->dF),
                                                         ctx->ldF, ctx->dD, n, dp, count, dc);
  QAP_CUDA(cudaGetLastError());
  QAP_CUDA(cudaMemcpyAsync(cost, dc, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
  QAP_CUDA(cudaStreamSynchronize(s));
  return QAP_OK;
}

qap_status qap_2opt(qap_ctx* ctx, int32_t starts, uint64_t seed, int32_t max_iters,
                    int32_t* best_p, int64_t* best_cost, int32_t* iters_done) {
  if (!best_p || !best_cost) return QAP_EINVAL;
  qap_search_params p{};
  p.starts = starts;
  p.seed = seed;
  p.descend = 1;
  p.max_descent = max_iters;
  p.iters = 0;
  p.tenure = qap_tenure{1, 1, 0};
  qap_walk_outputs o{};
  o.best_p = best_p;
  o.best_cost = best_cost;
  o.descent_moves = iters_done;
  return qap_search(ctx, &p, nullptr, &o);
}

qap_status qap_tabu(qap_ctx* ctx, int32_t starts, int32_t iters, qap_tenure tenure,
                    int32_t aspiration, uint64_t seed, int32_t* best_p, int64_t* best_cost,
                    int32_t* best_iter, int32_t* status) {
  if (!best_p || !best_cost) return QAP_EINVAL;
  qap_search_params p{};
  p.starts = starts;
  p.seed = seed;
  p.iters = iters;
  p.tenure = tenure;
  p.aspiration = aspiration;
  p.max_descent = -1;
  qap_walk_outputs o{};
  o.best_p = best_p;
  o.best_cost = best_cost;
  o.best_iter = best_iter;
  o.status = status;
  return qap_search(ctx, &p, nullptr, &o);
}

}  // extern "C"
