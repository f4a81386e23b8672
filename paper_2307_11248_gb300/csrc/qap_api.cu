// C-ABI of the QAP search library: instance upload, validation, launch
// planning, and the blocking / stream-ordered search entry points for one
// instance and for a batch of instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/qap.h"
#include "qap_host.cuh"

namespace qaph {
thread_local char g_last_error[256] = "";
std::mutex g_attr_mu;
PreparedKernel g_prepared[kPreparedMax];
int g_prepared_count = 0;
}  // namespace qaph

using namespace qaph;

struct qap_ctx {
  int device = 0, sms = 0, smem_optin = 0;
  DevInstance di;
  int dbytes = 4;  // delta width
  int fbytes = 2;  // flow element width in device memory (1: int8, 2: int16)
  void* dF = nullptr;
  void* dFt = nullptr;
  void* dD = nullptr;
  cudaStream_t stream = nullptr;
  // growable device buffer of the blocking entry points
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // workspace of large-n plans (one slice per CTA of the persistent grid)
  void* ws = nullptr;
  size_t ws_bytes = 0;
};

// Instances of a batch that share one launch plan (a size class).
struct BatchClass {
  Plan plan;
  const void* fn = nullptr;
  int smem = 0, grid = 0, ctas_per_sm = 0;
  std::vector<int> members;  // instance indices, largest n first
  int item_off = 0, items = 0;
  size_t ws_off = 0, ws_stride = 0;
  size_t p_off = 0, rws_off = 0;  // offsets inside a CTA's workspace slice
  cudaStream_t side = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // timing events (qap_batch_set_timing)
  bool timed = false;                      // t0, t1 bracket the class's last launch
};

struct qap_batch {
  int device = 0, sms = 0, smem_optin = 0;
  int count = 0, nmax = 0;
  int dbytes = 4, fbytes = 2;
  std::vector<DevInstance> di;
  std::vector<size_t> offF, offFt, offD;
  void* data = nullptr;  // every instance's F, F^T and D
  qapk::InstArgs* d_insts = nullptr;  // one table per thread count (128..1024)
  int insts_written = 0;              // bit t: the table for 128 << t is written
  int* d_counter = nullptr;           // one work counter per class
  cudaStream_t stream = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* ws = nullptr;  // workspace of large-n plans and rule tables
  size_t ws_bytes = 0;
  // size classes of the last search shape (threads_per_walk, starts)
  std::vector<BatchClass> classes;
  int classes_threads = -1, classes_walks = 0, classes_rules = -1;
  int32_t* d_class_items = nullptr;  // per class item_inst | item_walk, then row_base
  cudaEvent_t fork = nullptr;
  std::vector<Plan> tuned;  // per instance: the autotuner's plan (nt == 0: none)
  int timing = 0;           // record timing events around each class's launch
};

namespace {

constexpr int kCounterStride = 32;  // ints between the classes' work counters

struct Launch {
  const void* fn;
  Plan plan;
  int smem;
  int ctas_per_sm;
  int grid;
};

qap_status occupancy(Launch* L, int sms, int work) {
  int occ = 0;
  QAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, L->fn, L->plan.nt, L->smem));
  if (occ < 1) return QAP_EUNSUPPORTED;
  L->ctas_per_sm = occ;
  L->grid = std::min(work, occ * sms);
  return QAP_OK;
}

qap_status plan_ctx(qap_ctx* ctx, const qap_search_params* p, Launch* L) {
  const bool many = p->starts >= 2 * ctx->sms;
  if (!choose_plan_fit(ctx->di.n, p->threads_per_walk, many, &ctx->di, 1, ctx->fbytes,
                       ctx->dbytes, ctx->smem_optin, 0, p->phase_x, &L->plan))
    return QAP_EUNSUPPORTED;
  L->fn = reinterpret_cast<const void*>(pick_walk_kernel(ctx->dbytes, ctx->fbytes, L->plan));
  if (!L->fn) return QAP_EUNSUPPORTED;
  L->smem = plan_smem(L->plan, &ctx->di, 1, ctx->fbytes, ctx->dbytes);
  QAP_TRY(prepare_kernel(L->fn, L->smem));
  return occupancy(L, ctx->sms, p->starts);
}

qap_status plan_batch(qap_batch* b, const qap_search_params* p, Launch* L) {
  // the batch kernel also holds one static int
  const bool many = (int64_t)b->count * p->starts >= 2 * (int64_t)b->sms;
  if (!choose_plan_fit(b->nmax, p->threads_per_walk, many, b->di.data(), b->count, b->fbytes,
                       b->dbytes, b->smem_optin, 16, p->phase_x, &L->plan))
    return QAP_EUNSUPPORTED;
  L->fn = reinterpret_cast<const void*>(pick_batch_kernel(b->dbytes, b->fbytes, L->plan));
  if (!L->fn) return QAP_EUNSUPPORTED;
  L->smem = plan_smem(L->plan, b->di.data(), b->count, b->fbytes, b->dbytes);
  QAP_TRY(prepare_kernel(L->fn, L->smem));
  return occupancy(L, b->sms, b->count * p->starts);
}

int nt_index(int nt) { return nt == 128 ? 0 : nt == 256 ? 1 : nt == 512 ? 2 : 3; }

void destroy_class_handles(BatchClass& c) {
  if (c.side) {
    cudaStreamSynchronize(c.side);
    cudaStreamDestroy(c.side);
  }
  if (c.done) cudaEventDestroy(c.done);
  if (c.t0) cudaEventDestroy(c.t0);
  if (c.t1) cudaEventDestroy(c.t1);
  c.side = nullptr;
  c.done = c.t0 = c.t1 = nullptr;
}

// Launch shape of a class with W walks per member (smem, kernel, grid,
// workspace) and the instance table for its thread count.
qap_status class_shape(qap_batch* b, BatchClass& c, int W, const qap_search_params* p) {
  std::vector<DevInstance> dm;
  int nmax = 0;
  for (int i : c.members) {
    dm.push_back(b->di[i]);
    nmax = std::max(nmax, b->di[i].n);
  }
  c.smem = plan_smem(c.plan, dm.data(), (int)dm.size(), b->fbytes, b->dbytes);
  c.fn = reinterpret_cast<const void*>(pick_batch_kernel(b->dbytes, b->fbytes, c.plan));
  if (!c.fn) return QAP_EUNSUPPORTED;
  QAP_TRY(prepare_kernel(c.fn, c.smem));
  int occ = 0;
  QAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c.fn, c.plan.nt, c.smem));
  if (occ < 1) return QAP_EUNSUPPORTED;
  c.items = (int)c.members.size() * W;
  c.ctas_per_sm = occ;
  c.grid = std::min(c.items, occ * b->sms);
  const WsLayout wl = ws_layout(c.plan, b->dbytes, b->fbytes, nmax, p);
  c.ws_stride = wl.stride;
  c.p_off = wl.p_off;
  c.rws_off = wl.rws_off;
  const int t = nt_index(c.plan.nt);
  if (!(b->insts_written & (1 << t))) {
    std::vector<qapk::InstArgs> h(b->count);
    char* base = static_cast<char*>(b->data);
    for (int i = 0; i < b->count; ++i)
      h[i] = inst_args(b->di[i], base + b->offF[i], base + b->offFt[i],
                       base + b->offD[i], c.plan.nt, b->fbytes);
    QAP_CUDA(cudaMemcpy(b->d_insts + (size_t)t * b->count, h.data(),
                        sizeof(qapk::InstArgs) * b->count, cudaMemcpyHostToDevice));
    b->insts_written |= 1 << t;
  }
  return QAP_OK;
}

// Size classes of a batch search: every instance takes the plan its own n
// would get alone, and instances with the same plan share one persistent
// launch.  Classes run on side streams, largest n first, so the longest
// walks start first and the other classes fill the SMs as those finish.
// The instance tables (one per thread count) and the item lists are written
// synchronously and cached for the same (threads, starts, rule tables).
qap_status plan_classes(qap_batch* b, const qap_search_params* p) {
  const int rules = uses_rule_tables(p) ? 1 : 0;
  const int W = p->starts;
  if (!b->classes.empty() && b->classes_threads == p->threads_per_walk &&
      b->classes_walks == W && b->classes_rules == rules)
    return QAP_OK;
  if ((size_t)b->count * W > (size_t)INT_MAX / 2) return QAP_EINVAL;
  b->classes_threads = -1;
  std::vector<Plan> plan_of(b->count);
  for (int i = 0; i < b->count; ++i) {
    if (p->threads_per_walk == 0 && !b->tuned.empty() && b->tuned[i].nt != 0) {
      plan_of[i] = b->tuned[i];
      if (p->phase_x == QAP_PHASE_X_DOTS) plan_of[i].store &= ~qapk::kProductM;
      continue;
    }
    // the batch kernel also holds one static int
    // the classes run together: walks of the whole batch fill the SMs
    const bool many = (int64_t)b->count * W >= 2 * (int64_t)b->sms;
    if (!choose_plan_fit(b->di[i].n, p->threads_per_walk, many, &b->di[i], 1, b->fbytes,
                         b->dbytes, b->smem_optin, 16, p->phase_x, &plan_of[i]))
      return QAP_EUNSUPPORTED;
  }
  std::vector<int> order(b->count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->di[x].n > b->di[y].n; });
  // keep the old classes' streams and events for reuse
  std::vector<BatchClass> old;
  old.swap(b->classes);
  auto same = [](const Plan& x, const Plan& y) {
    return x.nt == y.nt && x.maxpt == y.maxpt && x.store == y.store;
  };
  for (int i : order) {  // classes appear in order of their largest n
    BatchClass* c = nullptr;
    for (BatchClass& k : b->classes)
      if (same(k.plan, plan_of[i])) c = &k;
    if (!c) {
      b->classes.emplace_back();
      c = &b->classes.back();
      c->plan = plan_of[i];
    }
    c->members.push_back(i);
  }
  for (size_t k = 0; k < b->classes.size(); ++k) {
    if (k < old.size()) {
      b->classes[k].side = old[k].side;
      b->classes[k].done = old[k].done;
      b->classes[k].t0 = old[k].t0;
      b->classes[k].t1 = old[k].t1;
      old[k].side = nullptr;
      old[k].done = nullptr;
      old[k].t0 = old[k].t1 = nullptr;
    }
  }
  for (BatchClass& c : old) destroy_class_handles(c);
  int item_off = 0;
  size_t ws_off = 0;
  for (BatchClass& c : b->classes) {
    QAP_TRY(class_shape(b, c, W, p));
    c.item_off = item_off;
    item_off += c.items;
    c.ws_off = ws_off;
    ws_off += (c.ws_stride * c.grid + 255) / 256 * 256;
    if (b->classes.size() > 1) {
      if (!c.side) QAP_CUDA(cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking));
      if (!c.done) QAP_CUDA(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    }
    c.timed = false;
  }
  if (b->classes.size() > 1 && !b->fork)
    QAP_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  // item lists: class after class, each longest instances first; row bases
  const size_t total = (size_t)item_off;
  std::vector<int32_t> h(total * 2 + b->count);
  for (const BatchClass& c : b->classes) {
    size_t k = c.item_off;
    for (int inst : c.members)
      for (int w = 0; w < W; ++w, ++k) {
        h[k] = inst;
        h[total + k] = w;
      }
  }
  for (int i = 0; i < b->count; ++i) h[2 * total + i] = i * W;
  if (b->d_class_items) cudaFree(b->d_class_items);
  b->d_class_items = nullptr;
  if (cudaMalloc(&b->d_class_items, h.size() * sizeof(int32_t)) != cudaSuccess)
    return QAP_ENOMEM;
  QAP_CUDA(cudaMemcpy(b->d_class_items, h.data(), h.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice));
  QAP_TRY(grow(&b->ws, &b->ws_bytes, ws_off));
  b->classes_threads = p->threads_per_walk;
  b->classes_walks = W;
  b->classes_rules = rules;
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

// ---------------------------------------------------------------------------
// one instance
// ---------------------------------------------------------------------------

qap_status qap_create(const int64_t* F, const int64_t* D, int32_t n, uint32_t flags,
                      qap_ctx** out) {
  if (!out) return QAP_EINVAL;
  *out = nullptr;
  if (flags & ~QAP_FORCE_INT64) return QAP_EINVAL;
  DevInstance di;
  QAP_TRY(inspect_instance(F, D, n, &di));
  qap_ctx* c = new (std::nothrow) qap_ctx();
  if (!c) return QAP_ENOMEM;
  auto fail = [&](qap_status s) {
    qap_destroy(c);
    return s;
  };
  c->dbytes = ((flags & QAP_FORCE_INT64) || di.wide || di.bound > (int64_t)INT_MAX - 1) ? 8 : 4;
  c->fbytes = flow_bytes(di, c->dbytes);
  di.ldF = pad_ldF(n, c->fbytes);
  di.ldP = pad_ldP(n, pbytes_of(c->fbytes));
  c->di = di;
  qap_status st = device_attrs(&c->device, &c->sms, &c->smem_optin);
  if (st != QAP_OK) return fail(st);
  std::vector<unsigned char> iF, iFt, iD;
  build_images(F, D, di, c->fbytes, iF, iFt, iD);
  if (cudaMalloc(&c->dF, iF.size()) != cudaSuccess) return fail(QAP_ENOMEM);
  if (!di.symF && cudaMalloc(&c->dFt, iFt.size()) != cudaSuccess) return fail(QAP_ENOMEM);
  if (cudaMalloc(&c->dD, iD.size()) != cudaSuccess) return fail(QAP_ENOMEM);
  cudaError_t e = cudaMemcpy(c->dF, iF.data(), iF.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !di.symF)
    e = cudaMemcpy(c->dFt, iFt.data(), iFt.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->dD, iD.data(), iD.size(), cudaMemcpyHostToDevice);
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
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

qap_status qap_info(const qap_ctx* ctx, qap_ctx_info* out) {
  if (!ctx || !out) return QAP_EINVAL;
  out->n = ctx->di.n;
  out->delta_bytes = ctx->dbytes;
  out->sym_flow = ctx->di.symF;
  out->sym_dist = ctx->di.symD;
  out->bound = ctx->di.bound;
  out->flow_bytes = ctx->fbytes;
  out->dist_bytes = pbytes_of(ctx->fbytes);
  return QAP_OK;
}

qap_status qap_plan(qap_ctx* ctx, const qap_search_params* params, qap_plan_info* out) {
  if (!ctx || !out) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  DeviceGuard dg;
  QAP_TRY(dg.set(ctx->device));
  Launch L;
  QAP_TRY(plan_ctx(ctx, params, &L));
  out->threads_per_walk = L.plan.nt;
  out->pairs_per_thread = L.plan.maxpt;
  out->smem_bytes = L.smem;
  out->grid = params->launch == QAP_LAUNCH_PLAIN ? 1 : L.grid;
  out->ctas_per_sm = L.ctas_per_sm;
  out->sms = ctx->sms;
  out->classes = 1;
  out->products = products_form(L.plan);
  out->workspace = (L.plan.store & qapk::kGlobalDelta) != 0;
  return QAP_OK;
}

qap_status qap_search_async(qap_ctx* ctx, const qap_search_params* params,
                            const int32_t* d_starts, const qap_walk_outputs* out,
                            void* stream) {
  if (!ctx) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (!out || !out->best_cost) return QAP_EINVAL;
  QAP_TRY(check_penalty(params, ctx->dbytes, ctx->di.bound));
  DeviceGuard dg;
  QAP_TRY(dg.set(ctx->device));
  Launch L;
  QAP_TRY(plan_ctx(ctx, params, &L));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  qapk::WalkArgs a{};
  a.inst = inst_args(ctx->di, ctx->dF, ctx->dFt, ctx->dD, L.plan.nt, ctx->fbytes);
  a.s = make_search_args(params, out, ctx->di.n);
  a.starts = d_starts;
  a.walks = params->starts;
  a.walk_offset = 0;
  const WsLayout wl = ws_layout(L.plan, ctx->dbytes, ctx->fbytes, ctx->di.n, params);
  a.ws_stride = wl.stride;
  a.s.rws_off = wl.rws_off;
  a.s.p_off = wl.p_off;
  if (a.ws_stride) {
    // the plain form runs one CTA per launch; launches on one stream share it
    const int ctas = params->launch == QAP_LAUNCH_PLAIN ? 1 : L.grid;
    QAP_TRY(grow(&ctx->ws, &ctx->ws_bytes, a.ws_stride * ctas));
    a.ws = static_cast<unsigned char*>(ctx->ws);
  }
  const auto fn = reinterpret_cast<qapk::WalkKernelFn>(const_cast<void*>(L.fn));
  if (params->launch == QAP_LAUNCH_PLAIN) {
    a.walks = 1;
    for (int w = 0; w < params->starts; ++w) {
      a.walk_offset = w;
      fn<<<1, L.plan.nt, L.smem, s>>>(a);
    }
  } else {
    fn<<<L.grid, L.plan.nt, L.smem, s>>>(a);
  }
  QAP_CUDA(cudaGetLastError());
  return QAP_OK;
}

qap_status qap_search(qap_ctx* ctx, const qap_search_params* params, const int32_t* starts,
                      const qap_walk_outputs* out) {
  if (!ctx) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (!out || !out->best_cost) return QAP_EINVAL;
  const int n = ctx->di.n, W = params->starts;
  if (starts) {
    std::vector<char> seen;
    for (int w = 0; w < W; ++w)
      if (!is_permutation(starts + (size_t)w * n, n, seen)) return QAP_EINVAL;
  }
  DeviceGuard dg;
  QAP_TRY(dg.set(ctx->device));
  const OutLayout L = out_layout(W, n);
  const size_t starts_off = (L.total + 255) / 256 * 256;
  const size_t freq_off = starts_off + ((size_t)W * n * 4 + 255) / 256 * 256;
  const size_t freq_bytes = out->freq ? (size_t)W * n * n * 4 : 0;
  QAP_TRY(grow(&ctx->scratch, &ctx->scratch_bytes, freq_off + freq_bytes));
  char* base = static_cast<char*>(ctx->scratch);
  qap_walk_outputs d = carve_outputs(base, L, W);
  if (out->freq) d.freq = reinterpret_cast<int32_t*>(base + freq_off);
  int32_t* d_starts = reinterpret_cast<int32_t*>(base + starts_off);
  cudaStream_t s = ctx->stream;
  if (starts)
    QAP_CUDA(cudaMemcpyAsync(d_starts, starts, (size_t)W * n * 4, cudaMemcpyHostToDevice, s));
  QAP_TRY(qap_search_async(ctx, params, starts ? d_starts : nullptr, &d, s));
  return copy_outputs_back(out, d, W, n, s);
}

qap_status qap_cost(qap_ctx* ctx, int32_t count, const int32_t* p, int64_t* cost) {
  if (!ctx || count < 0 || (count > 0 && (!p || !cost))) return QAP_EINVAL;
  if (count == 0) return QAP_OK;
  const int n = ctx->di.n;
  std::vector<char> seen;
  for (int k = 0; k < count; ++k)
    if (!is_permutation(p + (size_t)k * n, n, seen)) return QAP_EINVAL;
  DeviceGuard dg;
  QAP_TRY(dg.set(ctx->device));
  const size_t pbytes = (size_t)count * n * sizeof(int32_t);
  const size_t off_cost = ((pbytes + 255) / 256) * 256;
  QAP_TRY(grow(&ctx->scratch, &ctx->scratch_bytes, off_cost + (size_t)count * 8));
  char* base = static_cast<char*>(ctx->scratch);
  int32_t* dp = reinterpret_cast<int32_t*>(base);
  int64_t* dc = reinterpret_cast<int64_t*>(base + off_cost);
  cudaStream_t s = ctx->stream;
  QAP_CUDA(cudaMemcpyAsync(dp, p, pbytes, cudaMemcpyHostToDevice, s));
  const int grid = std::min(count, ctx->sms * 8);
  if (ctx->fbytes == 1)
    qapk::cost_kernel<int8_t, int8_t, 256><<<grid, 256, 0, s>>>(
        static_cast<const int8_t*>(ctx->dF), ctx->di.ldF, static_cast<const int8_t*>(ctx->dD), n,
        dp, count, dc);
  else if (ctx->fbytes == 2)
    qapk::cost_kernel<int16_t, int8_t, 256><<<grid, 256, 0, s>>>(
        static_cast<const int16_t*>(ctx->dF), ctx->di.ldF, static_cast<const int8_t*>(ctx->dD),
        n, dp, count, dc);
  else
    qapk::cost_kernel<int64_t, int64_t, 256><<<grid, 256, 0, s>>>(
        static_cast<const int64_t*>(ctx->dF), ctx->di.ldF, static_cast<const int64_t*>(ctx->dD),
        n, dp, count, dc);
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

qap_status qap_best_walks(const int64_t* best_cost, int32_t groups, int32_t walks,
                          int32_t* index) {
  if (groups < 0 || walks < 1 || (groups > 0 && (!best_cost || !index))) return QAP_EINVAL;
  for (int32_t g = 0; g < groups; ++g) {
    const int64_t* c = best_cost + (size_t)g * walks;
    int32_t k = 0;
    for (int32_t w = 1; w < walks; ++w)
      if (c[w] < c[k]) k = w;
    index[g] = k;
  }
  return QAP_OK;
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

// ---------------------------------------------------------------------------
// a batch of instances
// ---------------------------------------------------------------------------

qap_status qap_batch_create(int32_t count, const int64_t* const* F, const int64_t* const* D,
                            const int32_t* n, uint32_t flags, qap_batch** out) {
  if (!out) return QAP_EINVAL;
  *out = nullptr;
  if (count < 1 || !F || !D || !n || (flags & ~QAP_FORCE_INT64)) return QAP_EINVAL;
  qap_batch* b = new (std::nothrow) qap_batch();
  if (!b) return QAP_ENOMEM;
  auto fail = [&](qap_status s) {
    qap_batch_destroy(b);
    return s;
  };
  b->count = count;
  b->di.resize(count);
  int64_t maxB = 0;
  int bytevec = 1, wide = 0;
  for (int i = 0; i < count; ++i) {
    qap_status st = inspect_instance(F[i], D[i], n[i], &b->di[i]);
    if (st != QAP_OK) return fail(st);
    bytevec &= b->di[i].bytevec;
    wide |= b->di[i].wide;
    maxB = std::max(maxB, b->di[i].bound);
    b->nmax = std::max(b->nmax, n[i]);
  }
  // one delta width and one element width for the whole batch
  b->dbytes = ((flags & QAP_FORCE_INT64) || wide || maxB > (int64_t)INT_MAX - 1) ? 8 : 4;
  DevInstance all;
  all.bytevec = bytevec;
  all.wide = wide;
  b->fbytes = flow_bytes(all, b->dbytes);
  qap_status st = device_attrs(&b->device, &b->sms, &b->smem_optin);
  if (st != QAP_OK) return fail(st);
  std::vector<unsigned char> blob;
  b->offF.resize(count);
  b->offFt.resize(count);
  b->offD.resize(count);
  for (int i = 0; i < count; ++i) {
    DevInstance& d = b->di[i];
    d.ldF = pad_ldF(d.n, b->fbytes);
    d.ldP = pad_ldP(d.n, pbytes_of(b->fbytes));
    std::vector<unsigned char> iF, iFt, iD;
    build_images(F[i], D[i], d, b->fbytes, iF, iFt, iD);
    auto append = [&](const std::vector<unsigned char>& v) {
      const size_t off = (blob.size() + 255) / 256 * 256;
      blob.resize(off + v.size());
      std::memcpy(blob.data() + off, v.data(), v.size());
      return off;
    };
    b->offF[i] = append(iF);
    b->offFt[i] = d.symF ? b->offF[i] : append(iFt);
    b->offD[i] = append(iD);
  }
  if (cudaMalloc(&b->data, blob.size()) != cudaSuccess) return fail(QAP_ENOMEM);
  cudaError_t e = cudaMemcpy(b->data, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy"));
  if (cudaMalloc(&b->d_insts, sizeof(qapk::InstArgs) * count * 4) != cudaSuccess)
    return fail(QAP_ENOMEM);
  if (cudaMalloc(&b->d_counter, kCounterStride * 4 * 64) != cudaSuccess) return fail(QAP_ENOMEM);
  e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreateWithFlags"));
  *out = b;
  return QAP_OK;
}

void qap_batch_destroy(qap_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->data) cudaFree(b->data);
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->scratch) cudaFree(b->scratch);
  if (b->ws) cudaFree(b->ws);
  if (b->d_class_items) cudaFree(b->d_class_items);
  for (BatchClass& c : b->classes) destroy_class_handles(c);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

qap_status qap_batch_info(const qap_batch* b, int32_t* count, int32_t* nmax,
                          int32_t* delta_bytes) {
  if (!b) return QAP_EINVAL;
  if (count) *count = b->count;
  if (nmax) *nmax = b->nmax;
  if (delta_bytes) *delta_bytes = b->dbytes;
  return QAP_OK;
}

qap_status qap_batch_plan(qap_batch* b, const qap_search_params* params, qap_plan_info* out) {
  if (!b || !out) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  QAP_TRY(plan_classes(b, params));
  const BatchClass& c = b->classes.front();  // the class of the largest n
  out->threads_per_walk = c.plan.nt;
  out->pairs_per_thread = c.plan.maxpt;
  out->smem_bytes = c.smem;
  out->grid = c.grid;
  out->ctas_per_sm = c.ctas_per_sm;
  out->sms = b->sms;
  out->classes = (int32_t)b->classes.size();
  out->products = products_form(c.plan);
  out->workspace = (c.plan.store & qapk::kGlobalDelta) != 0;
  return QAP_OK;
}

qap_status qap_batch_set_timing(qap_batch* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return QAP_EINVAL;
  b->timing = on;
  return QAP_OK;
}

qap_status qap_batch_classes(qap_batch* b, const qap_search_params* params,
                             qap_class_info* out, int32_t max_out, int32_t* count,
                             int32_t* inst_class) {
  if (!b || max_out < 0 || (max_out > 0 && !out)) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  QAP_TRY(plan_classes(b, params));
  if (count) *count = (int32_t)b->classes.size();
  for (size_t k = 0; k < b->classes.size(); ++k) {
    BatchClass& c = b->classes[k];
    if (inst_class)
      for (int i : c.members) inst_class[i] = (int32_t)k;
    if ((int32_t)k >= max_out) continue;
    qap_class_info& o = out[k];
    o.nmin = INT_MAX;
    o.nmax = 0;
    for (int i : c.members) {
      o.nmin = std::min(o.nmin, b->di[i].n);
      o.nmax = std::max(o.nmax, b->di[i].n);
    }
    o.instances = (int32_t)c.members.size();
    o.walks = c.items;
    o.threads_per_walk = c.plan.nt;
    o.pairs_per_thread = c.plan.maxpt;
    o.products = products_form(c.plan);
    o.workspace = (c.plan.store & qapk::kGlobalDelta) != 0;
    o.grid = c.grid;
    o.ctas_per_sm = c.ctas_per_sm;
    o.smem_bytes = c.smem;
    o.delta_bytes = b->dbytes;
    o.flow_bytes = b->fbytes;
    o.dist_bytes = pbytes_of(b->fbytes);
    o.last_ms = -1.f;
    if (c.timed) {
      QAP_CUDA(cudaEventSynchronize(c.t1));
      QAP_CUDA(cudaEventElapsedTime(&o.last_ms, c.t0, c.t1));
    }
  }
  return QAP_OK;
}

// The autotuner: for every size class of the rule, time each compiled plan
// that holds the class's largest n (each thread count with its fewest slots,
// and the workspace plan) on the class's own instances with the search's
// walk count and `trial_iters` iterations, and keep the fastest.  Every plan
// computes the same walks, so the choice changes only the speed.
qap_status qap_batch_autotune(qap_batch* b, const qap_search_params* params,
                              int32_t trial_iters, qap_tune_result* results,
                              int32_t max_results, int32_t* nresults) {
  if (!b || trial_iters < 1 || max_results < 0 || (max_results > 0 && !results))
    return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (params->launch != QAP_LAUNCH_PERSISTENT || params->threads_per_walk != 0)
    return QAP_EINVAL;
  qap_search_params tp = *params;
  tp.iters = trial_iters;
  QAP_TRY(validate_params(&tp));
  for (const DevInstance& d : b->di) QAP_TRY(check_penalty(&tp, b->dbytes, d.bound));
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  b->tuned.clear();
  b->classes_threads = -1;
  QAP_TRY(plan_classes(b, &tp));
  struct RuleClass { Plan plan; std::vector<int> members; };
  std::vector<RuleClass> rule;
  for (const BatchClass& c : b->classes) rule.push_back({c.plan, c.members});
  const int W = params->starts;
  const size_t rows = (size_t)b->count * W;
  QAP_TRY(grow(&b->scratch, &b->scratch_bytes, rows * 8));
  qap_walk_outputs dout{};
  dout.best_cost = static_cast<int64_t*>(b->scratch);
  int32_t* d_items = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  qap_status st = QAP_OK;
  std::vector<Plan> tuned(b->count);
  int found = 0;
  auto fail = [&](qap_status e) {
    if (d_items) cudaFree(d_items);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return e;
  };
  if (cudaMalloc(&d_items, (rows * 2 + b->count) * sizeof(int32_t)) != cudaSuccess)
    return fail(QAP_ENOMEM);
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
  int* counter = b->d_counter + 63 * kCounterStride;
  auto chk = [](cudaError_t e, const char* where) {
    return e == cudaSuccess ? QAP_OK : cuda_fail(e, where);
  };
  for (const RuleClass& rc : rule) {
    int nmin = INT_MAX, nmax = 0;
    std::vector<DevInstance> dm;
    for (int i : rc.members) {
      nmin = std::min(nmin, b->di[i].n);
      nmax = std::max(nmax, b->di[i].n);
      dm.push_back(b->di[i]);
    }
    auto fits = [&](const Plan& p) {
      return plan_smem(p, dm.data(), (int)dm.size(), b->fbytes, b->dbytes) + 16 <= b->smem_optin;
    };
    std::vector<Plan> cands;
    for (int nt : {128, 256, 512, 1024}) {
      Plan p;
      if (nmax <= 181 && plan_for(nmax, nt, &p) &&
          fits(p = wide_store(p, dm.data(), (int)dm.size(), b->fbytes, b->dbytes,
                              b->smem_optin, 16))) {
        cands.push_back(p);
        const Plan m = with_products(p, b->fbytes, tp.phase_x, fits);
        if (m.store != p.store) cands.push_back(m);
      }
    }
    if (qapk::row_segments(nmax, kLargePlan.maxpt) <= kLargePlan.nt) {
      Plan p = kLargePlan;
      if (b->fbytes == 8)
        p = wide_store(p, dm.data(), (int)dm.size(), b->fbytes, b->dbytes, b->smem_optin, 16);
      else if (!fits(p))
        p.store |= qapk::kGlobalFlow;
      if (fits(p)) cands.push_back(p);
    }
    // items of this class, longest instances first; row bases for all
    const size_t items = rc.members.size() * (size_t)W;
    std::vector<int32_t> h(items * 2 + b->count);
    size_t k = 0;
    for (int inst : rc.members)
      for (int w = 0; w < W; ++w, ++k) {
        h[k] = inst;
        h[items + k] = w;
      }
    for (int i = 0; i < b->count; ++i) h[2 * items + i] = i * W;
    if ((st = chk(cudaMemcpy(d_items, h.data(), h.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice), "cudaMemcpy")) != QAP_OK)
      return fail(st);
    Plan best = rc.plan;
    float best_ms = -1.f, rule_ms = -1.f;
    for (const Plan& cand : cands) {
      BatchClass c;
      c.plan = cand;
      c.members = rc.members;
      if ((st = class_shape(b, c, W, &tp)) != QAP_OK) return fail(st);
      if ((st = grow(&b->ws, &b->ws_bytes, c.ws_stride * c.grid)) != QAP_OK) return fail(st);
      qapk::BatchArgs a{};
      a.insts = b->d_insts + (size_t)nt_index(c.plan.nt) * b->count;
      a.item_inst = d_items;
      a.item_walk = d_items + items;
      a.row_base = d_items + 2 * items;
      a.items = c.items;
      a.counter = counter;
      a.s = make_search_args(&tp, &dout, b->nmax);
      a.s.rws_off = c.rws_off;
      a.s.p_off = c.p_off;
      a.ws_stride = c.ws_stride;
      a.ws = c.ws_stride ? static_cast<unsigned char*>(b->ws) : nullptr;
      const auto fn = reinterpret_cast<qapk::BatchKernelFn>(const_cast<void*>(c.fn));
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // a warm-up run, then the timed one
        cudaMemsetAsync(counter, 0, sizeof(int), b->stream);
        if (rep) cudaEventRecord(t0, b->stream);
        fn<<<c.grid, c.plan.nt, c.smem, b->stream>>>(a);
        if (rep) cudaEventRecord(t1, b->stream);
      }
      // a trial that did not launch would time as the fastest
      if ((st = chk(cudaGetLastError(), "autotune launch")) != QAP_OK) return fail(st);
      if ((st = chk(cudaEventSynchronize(t1), "autotune trial")) != QAP_OK) return fail(st);
      cudaEventElapsedTime(&ms, t0, t1);
      const bool is_rule = cand.nt == rc.plan.nt && cand.maxpt == rc.plan.maxpt &&
                           cand.store == rc.plan.store;
      if (is_rule) rule_ms = ms;
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
    for (int i : rc.members) tuned[i] = best;
    if (found < max_results) {
      qap_tune_result& r = results[found];
      r.nmin = nmin;
      r.nmax = nmax;
      r.instances = (int32_t)rc.members.size();
      r.candidates = (int32_t)cands.size();
      r.threads_per_walk = best.nt;
      r.pairs_per_thread = best.maxpt;
      r.workspace = (best.store & qapk::kGlobalDelta) != 0;
      r.products = products_form(best);
      r.trial_ms = best_ms;
      r.rule_ms = rule_ms;
    }
    ++found;
  }
  if (nresults) *nresults = found;
  b->tuned = tuned;
  b->classes_threads = -1;  // the next search regroups by the tuned plans
  return fail(QAP_OK);
}

qap_status qap_batch_search_async(qap_batch* b, const qap_search_params* params,
                                  const qap_walk_outputs* out, int32_t p_stride, void* stream) {
  if (!b) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (!out || !out->best_cost || p_stride < b->nmax) return QAP_EINVAL;
  if (params->launch != QAP_LAUNCH_PERSISTENT) return QAP_EINVAL;
  for (const DevInstance& d : b->di) QAP_TRY(check_penalty(params, b->dbytes, d.bound));
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  QAP_TRY(plan_classes(b, params));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t total = (size_t)b->count * params->starts;
  const bool fork = b->classes.size() > 1;
  if (fork) QAP_CUDA(cudaEventRecord(b->fork, s));
  for (size_t k = 0; k < b->classes.size(); ++k) {
    BatchClass& c = b->classes[k];
    cudaStream_t cs = fork ? c.side : s;
    if (b->timing && !c.t0) QAP_CUDA(cudaEventCreate(&c.t0));
    if (b->timing && !c.t1) QAP_CUDA(cudaEventCreate(&c.t1));
    if (fork) QAP_CUDA(cudaStreamWaitEvent(cs, b->fork, 0));
    qapk::BatchArgs a{};
    a.insts = b->d_insts + (size_t)nt_index(c.plan.nt) * b->count;
    a.item_inst = b->d_class_items + c.item_off;
    a.item_walk = b->d_class_items + total + c.item_off;
    a.row_base = b->d_class_items + 2 * total;
    a.items = c.items;
    a.counter = b->d_counter + k * kCounterStride;
    a.s = make_search_args(params, out, p_stride);
    a.s.rws_off = c.rws_off;
    a.s.p_off = c.p_off;
    a.ws_stride = c.ws_stride;
    a.ws = c.ws_stride ? static_cast<unsigned char*>(b->ws) + c.ws_off : nullptr;
    QAP_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), cs));
    const auto fn = reinterpret_cast<qapk::BatchKernelFn>(const_cast<void*>(c.fn));
    if (b->timing) QAP_CUDA(cudaEventRecord(c.t0, cs));
    fn<<<c.grid, c.plan.nt, c.smem, cs>>>(a);
    QAP_CUDA(cudaGetLastError());
    if (b->timing) QAP_CUDA(cudaEventRecord(c.t1, cs));
    c.timed = b->timing != 0;
    if (fork) {
      QAP_CUDA(cudaEventRecord(c.done, cs));
      QAP_CUDA(cudaStreamWaitEvent(s, c.done, 0));
    }
  }
  return QAP_OK;
}

qap_status qap_batch_search(qap_batch* b, const qap_search_params* params,
                            const qap_walk_outputs* out, int32_t p_stride) {
  if (!b) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (!out || !out->best_cost || p_stride < b->nmax) return QAP_EINVAL;
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  const int W = b->count * params->starts;
  const OutLayout L = out_layout(W, p_stride);
  const size_t freq_off = (L.total + 255) / 256 * 256;
  const size_t freq_bytes = out->freq ? (size_t)W * p_stride * p_stride * 4 : 0;
  QAP_TRY(grow(&b->scratch, &b->scratch_bytes, freq_off + freq_bytes));
  qap_walk_outputs d = carve_outputs(static_cast<char*>(b->scratch), L, W);
  if (out->freq) d.freq = reinterpret_cast<int32_t*>(static_cast<char*>(b->scratch) + freq_off);
  QAP_TRY(qap_batch_search_async(b, params, &d, p_stride, b->stream));
  return copy_outputs_back(out, d, W, p_stride, b->stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch search without device allocation.
//
// The work-queue counter, the instance table and the item lists of
// qap_batch_search_noalloc live in one file-scope device array instead of
// memory from cudaMalloc.  Every GPU that loads the library holds the array
// (kNoallocBytes) until the process exits.  In host code the array's name
// stands for a host-side shadow, so its device address is looked up once per
// device with cudaGetSymbolAddress and that address is what the kernels get.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoallocMaxInstances = 4096;
constexpr int kNoallocMaxItems = 65536;
constexpr size_t kNoallocInstOff = 256;  // counter in the first 256 bytes
constexpr size_t kNoallocItemsOff =
    kNoallocInstOff + (sizeof(qapk::InstArgs) * kNoallocMaxInstances + 255) / 256 * 256;
constexpr size_t kNoallocBytes =
    kNoallocItemsOff + sizeof(int32_t) * (2 * (size_t)kNoallocMaxItems + kNoallocMaxInstances);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kNoallocMaxDevices] = {};

// Host staging of the tables (static storage: the call allocates no host
// memory either).  Calls serialise on g_noalloc_mu while they use it; a copy
// from pageable host memory has read its source when cudaMemcpyAsync
// returns, so the next call may overwrite the staging.
qapk::InstArgs g_noalloc_h_insts[kNoallocMaxInstances];
int32_t g_noalloc_h_items[2 * kNoallocMaxItems + kNoallocMaxInstances];
int32_t g_noalloc_h_order[kNoallocMaxInstances];
int32_t g_noalloc_h_bucket[kMaxN + 2];

// Device address of the array on the current device (set-up on first use).
qap_status noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= kNoallocMaxDevices) return QAP_EUNSUPPORTED;
  if (!g_noalloc_addr[device]) {
    void* ptr = nullptr;
    QAP_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_addr[device] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_addr[device];
  return QAP_OK;
}

}  // namespace

extern "C" qap_status qap_batch_search_noalloc(qap_batch* b, const qap_search_params* params,
                                               const qap_walk_outputs* out, int32_t p_stride,
                                               void* stream) {
  if (!b) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (!out || !out->best_cost || p_stride < b->nmax) return QAP_EINVAL;
  if (params->launch != QAP_LAUNCH_PERSISTENT) return QAP_EINVAL;
  if (uses_rule_tables(params)) {
    snprintf(g_last_error, sizeof(g_last_error),
             "qap_batch_search_noalloc: the unit criteria and the frequency penalty keep "
             "per-CTA tables in an allocated workspace");
    return QAP_EUNSUPPORTED;
  }
  const int64_t items = (int64_t)b->count * params->starts;
  if (b->count > kNoallocMaxInstances || items > kNoallocMaxItems) {
    snprintf(g_last_error, sizeof(g_last_error),
             "qap_batch_search_noalloc: %d instances x %d walks exceeds the static scratch "
             "limit of %d instances and %d walks in total",
             b->count, params->starts, kNoallocMaxInstances, kNoallocMaxItems);
    return QAP_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  DeviceGuard dg;
  QAP_TRY(dg.set(b->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The tables are copied from static host memory that the next call
  // overwrites; a captured copy would read it again at every replay.
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  QAP_CUDA(cudaStreamIsCapturing(s, &capturing));
  if (capturing != cudaStreamCaptureStatusNone) {
    snprintf(g_last_error, sizeof(g_last_error),
             "qap_batch_search_noalloc: the stream is being captured; the call copies its "
             "tables from host memory that the next call overwrites");
    return QAP_EUNSUPPORTED;
  }
  unsigned char* base = nullptr;
  QAP_TRY(noalloc_scratch(b->device, &base));
  Launch L;
  QAP_TRY(plan_batch(b, params, &L));
  if (ws_layout(L.plan, b->dbytes, b->fbytes, b->nmax, params).stride != 0) {
    snprintf(g_last_error, sizeof(g_last_error),
             "qap_batch_search_noalloc: n = %d needs a plan with a per-CTA workspace, which is "
             "allocated (the large-n plan, or int64 elements beyond shared memory)", b->nmax);
    return QAP_EUNSUPPORTED;
  }
  const int count = b->count, W = params->starts;

  // instance table for this plan's thread count
  char* data = static_cast<char*>(b->data);
  for (int i = 0; i < count; ++i)
    g_noalloc_h_insts[i] = inst_args(b->di[i], data + b->offF[i], data + b->offFt[i],
                                     data + b->offD[i], L.plan.nt,
                                     b->fbytes);
  // items, longest instances first (stable counting sort by n)
  for (int v = 0; v <= kMaxN + 1; ++v) g_noalloc_h_bucket[v] = 0;
  for (int i = 0; i < count; ++i) ++g_noalloc_h_bucket[b->di[i].n];
  int pos = 0;
  for (int v = kMaxN; v >= 0; --v) {
    const int c = g_noalloc_h_bucket[v];
    g_noalloc_h_bucket[v] = pos;
    pos += c;
  }
  for (int i = 0; i < count; ++i) g_noalloc_h_order[g_noalloc_h_bucket[b->di[i].n]++] = i;
  int32_t* h_inst = g_noalloc_h_items;
  int32_t* h_walk = g_noalloc_h_items + items;
  int32_t* h_row = g_noalloc_h_items + 2 * items;
  int64_t k = 0;
  for (int j = 0; j < count; ++j)
    for (int w = 0; w < W; ++w, ++k) {
      h_inst[k] = g_noalloc_h_order[j];
      h_walk[k] = w;
    }
  for (int i = 0; i < count; ++i) h_row[i] = i * W;

  int* d_counter = reinterpret_cast<int*>(base);
  qapk::InstArgs* d_insts = reinterpret_cast<qapk::InstArgs*>(base + kNoallocInstOff);
  int32_t* d_items = reinterpret_cast<int32_t*>(base + kNoallocItemsOff);
  QAP_CUDA(cudaMemcpyAsync(d_insts, g_noalloc_h_insts, sizeof(qapk::InstArgs) * count,
                           cudaMemcpyHostToDevice, s));
  QAP_CUDA(cudaMemcpyAsync(d_items, g_noalloc_h_items, sizeof(int32_t) * (2 * items + count),
                           cudaMemcpyHostToDevice, s));
  QAP_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(int), s));
  qapk::BatchArgs a{};
  a.insts = d_insts;
  a.item_inst = d_items;
  a.item_walk = d_items + items;
  a.row_base = d_items + 2 * items;
  a.items = (int)items;
  a.counter = d_counter;
  a.s = make_search_args(params, out, p_stride);
  const auto fn = reinterpret_cast<qapk::BatchKernelFn>(const_cast<void*>(L.fn));
  fn<<<L.grid, L.plan.nt, L.smem, s>>>(a);
  QAP_CUDA(cudaGetLastError());
  return QAP_OK;
}
