// Serving loop: continuous batching of QAP solve requests.
//
// A worker thread owns the GPU side.  Requests wait in a FIFO queue; the
// head request is admitted as soon as a slot (a CUDA stream) is free and the
// device arena has room for its instance, outputs and workspace.  An
// admitted request is uploaded, searched and copied back on its slot's
// stream, so requests admitted at different times run on the device at the
// same time; completion is detected with events, which frees the slot and
// the arena range for the next request.  The arena is one device allocation
// made at creation and carved first-fit, so no cudaMalloc or cudaFree (and
// none of the device-wide synchronisation cudaFree implies) happens while
// serving.  The submitting thread builds each request's upload images and
// places them in a pinned host slab (also allocated once), so the worker
// only enqueues copies and launches; pinned output buffers are sized at
// creation and, if a request ever needs more, replaced without freeing the
// old ones until the server is destroyed (cudaFreeHost synchronises the
// device).  Every host wait is bounded.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>

#include "qap_host.cuh"

using namespace qaph;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator of offsets in [0, size), 256-byte granules, adjacent
// free ranges merged.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  static size_t round(size_t b) { return (b + 255) / 256 * 256; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  DevInstance di;
  int dbytes = 4, fbytes = 2;
  std::vector<unsigned char> iF, iFt, iD;  // upload images (while not in the pinned slab)
  size_t szF = 0, szFt = 0, szD = 0;       // image sizes
  size_t host_off = 0, host_bytes = 0;     // range of the images in the pinned slab (bytes 0: none)
  qap_search_params params{};
  // placement on the device
  Plan plan{};
  int grid = 0, smem = 0;
  const void* fn = nullptr;
  size_t off = 0, bytes = 0, offF = 0, offFt = 0, offD = 0, offOut = 0, offWs = 0, ws_stride = 0;
  size_t p_off = 0, rws_off = 0;  // offsets inside a CTA's workspace slice
  int slot = -1;
  // results (host copies) and times
  std::vector<unsigned char> out;  // the device output block
  Clock::time_point t_submit, t_admit, t_done;
  double k_start_us = -1, k_end_us = -1;  // device clock of the kernel, from the server's creation
  qap_status result = QAP_OK;
  char err[256] = "";  // CUDA error text recorded by the worker thread
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t k0 = nullptr, k1 = nullptr;  // timing events around the kernel
  unsigned char* pinned = nullptr;  // upload images (when not in the slab), then the outputs
  size_t pinned_bytes = 0;
  Request* req = nullptr;
};

// Pinned bytes each slot starts with: the outputs of 64 walks of n = 256,
// or the images of an int8/int16 instance of n = 256.
constexpr size_t kSlotPinnedBytes = 512 << 10;

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

}  // namespace

struct qap_server {
  int device = 0, sms = 0, smem_optin = 0;
  qap_server_config cfg{};
  unsigned char* arena_base = nullptr;
  Arena arena;
  // pinned host slab of upload images, filled by the submitting threads
  unsigned char* slab = nullptr;
  Arena slab_arena;
  std::mutex slab_mu;
  std::vector<unsigned char*> retired;  // pinned buffers replaced while serving
  cudaEvent_t ref = nullptr;             // device-clock origin of the kernel times
  int64_t peak_in_flight = 0;
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0, in_flight = 0;
  std::thread worker;
  std::atomic<bool> stop{false};
  qap_status fatal = QAP_OK;
};

namespace {

// Plans the launch and sizes the device block of one request.
qap_status place(qap_server* sv, Request* r) {
  const int W = r->params.starts, n = r->di.n;
  // a request's own walks decide (several requests share the GPU)
  const bool many = W >= 2 * sv->sms;
  if (!choose_plan_fit(n, r->params.threads_per_walk, many, &r->di, 1, r->fbytes, r->dbytes,
                       sv->smem_optin, 0, r->params.phase_x, &r->plan))
    return QAP_EUNSUPPORTED;
  r->fn = reinterpret_cast<const void*>(pick_walk_kernel(r->dbytes, r->fbytes, r->plan));
  if (!r->fn) return QAP_EUNSUPPORTED;
  r->smem = plan_smem(r->plan, &r->di, 1, r->fbytes, r->dbytes);
  QAP_TRY(prepare_kernel(r->fn, r->smem));
  int occ = 0;
  QAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->fn, r->plan.nt, r->smem));
  if (occ < 1) return QAP_EUNSUPPORTED;
  r->grid = std::min(W, occ * sv->sms);
  const WsLayout wl = ws_layout(r->plan, r->dbytes, r->fbytes, n, &r->params);
  r->ws_stride = wl.stride;
  r->p_off = wl.p_off;
  r->rws_off = wl.rws_off;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = Arena::round(o + bytes);
    return at;
  };
  r->offF = take(r->iF.size());
  r->offFt = r->di.symF ? r->offF : take(r->iFt.size());
  r->offD = take(r->iD.size());
  r->offOut = take(out_layout(W, n).total);
  r->offWs = take(r->ws_stride * r->grid);
  r->bytes = o;
  return QAP_OK;
}

// A slot's pinned buffer of at least `bytes`; a smaller one is kept aside
// (freed at destruction) because cudaFreeHost would synchronise the device.
qap_status ensure_pinned(qap_server* sv, Slot& sl, size_t bytes) {
  if (sl.pinned_bytes >= bytes) return QAP_OK;
  unsigned char* p = nullptr;
  QAP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&p), bytes, cudaHostAllocDefault));
  if (sl.pinned) sv->retired.push_back(sl.pinned);
  sl.pinned = p;
  sl.pinned_bytes = bytes;
  return QAP_OK;
}

// Upload, search and download of one admitted request on its slot's stream.
qap_status launch(qap_server* sv, Request* r) {
  Slot& sl = sv->slots[r->slot];
  const int W = r->params.starts, n = r->di.n;
  const OutLayout OL = out_layout(W, n);
  const size_t up = r->host_bytes ? 0 : r->iF.size() + r->iFt.size() + r->iD.size();
  QAP_TRY(ensure_pinned(sv, sl, std::max(up, OL.total)));
  unsigned char* dev = sv->arena_base + r->off;
  if (r->host_bytes) {
    // the images are in the pinned slab already: copies only
    const unsigned char* h = sv->slab + r->host_off;
    QAP_CUDA(cudaMemcpyAsync(dev + r->offF, h, r->szF, cudaMemcpyHostToDevice, sl.stream));
    h += Arena::round(r->szF);
    if (!r->di.symF) {
      QAP_CUDA(cudaMemcpyAsync(dev + r->offFt, h, r->szFt, cudaMemcpyHostToDevice, sl.stream));
      h += Arena::round(r->szFt);
    }
    QAP_CUDA(cudaMemcpyAsync(dev + r->offD, h, r->szD, cudaMemcpyHostToDevice, sl.stream));
  } else {
    // stage the images in the slot's pinned memory and upload them
    size_t at = 0;
    auto stage = [&](const std::vector<unsigned char>& v, size_t dev_off) -> cudaError_t {
      if (v.empty()) return cudaSuccess;
      std::memcpy(sl.pinned + at, v.data(), v.size());
      cudaError_t e = cudaMemcpyAsync(dev + dev_off, sl.pinned + at, v.size(),
                                      cudaMemcpyHostToDevice, sl.stream);
      at += v.size();
      return e;
    };
    // the pinned staging is reused for the outputs only after the uploads ran
    QAP_CUDA(stage(r->iF, r->offF));
    if (!r->di.symF) QAP_CUDA(stage(r->iFt, r->offFt));
    QAP_CUDA(stage(r->iD, r->offD));
  }
  qapk::WalkArgs a{};
  a.inst = inst_args(r->di, dev + r->offF, dev + r->offFt,
                     dev + r->offD, r->plan.nt, r->fbytes);
  const qap_walk_outputs d = carve_outputs(reinterpret_cast<char*>(dev + r->offOut), OL, W);
  a.s = make_search_args(&r->params, &d, n);
  a.s.rws_off = r->rws_off;
  a.s.p_off = r->p_off;
  a.walks = W;
  a.walk_offset = 0;
  a.starts = nullptr;
  a.ws_stride = r->ws_stride;
  a.ws = r->ws_stride ? dev + r->offWs : nullptr;
  const auto fn = reinterpret_cast<qapk::WalkKernelFn>(const_cast<void*>(r->fn));
  QAP_CUDA(cudaEventRecord(sl.k0, sl.stream));
  fn<<<r->grid, r->plan.nt, r->smem, sl.stream>>>(a);
  QAP_CUDA(cudaGetLastError());
  QAP_CUDA(cudaEventRecord(sl.k1, sl.stream));
  QAP_CUDA(cudaMemcpyAsync(sl.pinned, dev + r->offOut, OL.total, cudaMemcpyDeviceToHost,
                           sl.stream));
  QAP_CUDA(cudaEventRecord(sl.done, sl.stream));
  return QAP_OK;
}

void finish(qap_server* sv, int slot_idx, qap_status st) {
  Slot& sl = sv->slots[slot_idx];
  Request* r = sl.req;
  if (st == QAP_OK) {
    const OutLayout OL = out_layout(r->params.starts, r->di.n);
    r->out.assign(sl.pinned, sl.pinned + OL.total);
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, sv->ref, sl.k0) == cudaSuccess &&
        cudaEventElapsedTime(&b, sv->ref, sl.k1) == cudaSuccess) {
      r->k_start_us = 1e3 * a;
      r->k_end_us = 1e3 * b;
    }
  }
  if (st == QAP_ECUDA) snprintf(r->err, sizeof(r->err), "%s", g_last_error);
  if (r->host_bytes) {
    std::lock_guard<std::mutex> hk(sv->slab_mu);
    sv->slab_arena.release(r->host_off, r->host_bytes);
    r->host_bytes = 0;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->arena.release(r->off, r->bytes);
  r->iF.clear();
  r->iFt.clear();
  r->iD.clear();
  r->result = st;
  r->t_done = Clock::now();
  r->done = true;
  sl.req = nullptr;
  sv->free_slots.push_back(slot_idx);
  --sv->in_flight;
  ++sv->completed;
  sv->cv_done.notify_all();
}

void worker_loop(qap_server* sv) {
  if (cudaSetDevice(sv->device) != cudaSuccess) {
    sv->fatal = QAP_ECUDA;
    return;
  }
  for (;;) {
    bool progress = false;
    // completions
    for (int i = 0; i < (int)sv->slots.size(); ++i) {
      Slot& sl = sv->slots[i];
      if (!sl.req) continue;
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) continue;
      finish(sv, i, e == cudaSuccess ? QAP_OK : cuda_fail(e, "request"));
      progress = true;
    }
    // admissions, in arrival order
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->pending.empty() && !sv->free_slots.empty()) {
      Request* r = sv->pending.front();
      if (!sv->arena.alloc(r->bytes, &r->off)) break;  // wait for memory
      sv->pending.pop_front();
      r->slot = sv->free_slots.back();
      sv->free_slots.pop_back();
      sv->slots[r->slot].req = r;
      ++sv->in_flight;
      sv->peak_in_flight = std::max(sv->peak_in_flight, sv->in_flight);
      r->t_admit = Clock::now();
      lk.unlock();
      const qap_status st = launch(sv, r);
      if (st != QAP_OK) {
        // nothing of the request is in flight past the failed call; record it
        cudaStreamSynchronize(sv->slots[r->slot].stream);
        finish(sv, r->slot, st);
      }
      progress = true;
      lk.lock();
    }
    if (sv->stop && sv->pending.empty() && sv->in_flight == 0) return;
    if (!progress) {
      // idle: sleep until work arrives (bounded), or poll the device again
      if (sv->in_flight == 0)
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
    }
  }
}

}  // namespace

extern "C" {

qap_status qap_server_create(const qap_server_config* cfg, qap_server** out) {
  if (!cfg || !out) return QAP_EINVAL;
  *out = nullptr;
  if (cfg->slots < 1 || cfg->slots > 128 || cfg->mem_bytes < (1 << 20)) return QAP_EINVAL;
  auto* sv = new (std::nothrow) qap_server();
  if (!sv) return QAP_ENOMEM;
  sv->cfg = *cfg;
  auto fail = [&](qap_status s) {
    qap_server_destroy(sv);
    return s;
  };
  qap_status st = device_attrs(&sv->device, &sv->sms, &sv->smem_optin);
  if (st != QAP_OK) return fail(st);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&sv->arena_base), (size_t)cfg->mem_bytes);
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? QAP_ENOMEM : cuda_fail(e, "cudaMalloc"));
  sv->arena.init((size_t)cfg->mem_bytes);
  // pinned slab of upload images: a quarter of the device arena, 8 to 256 MiB
  const size_t slab = std::min<size_t>(256u << 20, std::max<size_t>(8u << 20, cfg->mem_bytes / 4));
  e = cudaHostAlloc(reinterpret_cast<void**>(&sv->slab), slab, cudaHostAllocDefault);
  if (e != cudaSuccess) return fail(QAP_ENOMEM);
  sv->slab_arena.init(slab);
  sv->slots.resize(cfg->slots);
  for (int i = 0; i < cfg->slots; ++i) {
    Slot& sl = sv->slots[i];
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.k0);
    if (e == cudaSuccess) e = cudaEventCreate(&sl.k1);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate"));
    st = ensure_pinned(sv, sl, kSlotPinnedBytes);
    if (st != QAP_OK) return fail(st);
    sv->free_slots.push_back(cfg->slots - 1 - i);
  }
  e = cudaEventCreate(&sv->ref);
  if (e == cudaSuccess) e = cudaEventRecord(sv->ref, sv->slots[0].stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(sv->ref);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaEventRecord"));
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return QAP_OK;
}

qap_status qap_server_submit(qap_server* sv, const int64_t* F, const int64_t* D, int32_t n,
                             uint32_t flags, const qap_search_params* params, uint64_t* ticket) {
  if (!sv || !ticket) return QAP_EINVAL;
  QAP_TRY(validate_params(params));
  if (params->launch != QAP_LAUNCH_PERSISTENT || (flags & ~QAP_FORCE_INT64)) return QAP_EINVAL;
  if (sv->fatal != QAP_OK) return sv->fatal;
  auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
  if (!r) return QAP_ENOMEM;
  QAP_TRY(inspect_instance(F, D, n, &r->di));
  // int64 deltas when B, or B plus the largest frequency penalty, needs them
  r->dbytes = ((flags & QAP_FORCE_INT64) || r->di.wide || r->di.bound > (int64_t)INT_MAX - 1 ||
               check_penalty(params, 4, r->di.bound) != QAP_OK) ? 8 : 4;
  r->fbytes = flow_bytes(r->di, r->dbytes);
  r->di.ldF = pad_ldF(n, r->fbytes);
  r->di.ldP = pad_ldP(n, pbytes_of(r->fbytes));
  r->params = *params;
  build_images(F, D, r->di, r->fbytes, r->iF, r->iFt, r->iD);
  if (r->di.symF) r->iFt.clear();
  DeviceGuard dg;
  QAP_TRY(dg.set(sv->device));
  QAP_TRY(place(sv, r.get()));
  if (r->bytes > sv->arena.size()) return QAP_ENOMEM;  // could never be admitted
  // the images into the pinned slab when it has room, so the worker only
  // enqueues their copies
  r->szF = r->iF.size();
  r->szFt = r->iFt.size();
  r->szD = r->iD.size();
  const size_t hb = Arena::round(r->szF) + Arena::round(r->szFt) + Arena::round(r->szD);
  {
    std::lock_guard<std::mutex> hk(sv->slab_mu);
    if (sv->slab_arena.alloc(hb, &r->host_off)) r->host_bytes = hb;
  }
  if (r->host_bytes) {
    unsigned char* h = sv->slab + r->host_off;
    std::memcpy(h, r->iF.data(), r->szF);
    h += Arena::round(r->szF);
    if (r->szFt) {
      std::memcpy(h, r->iFt.data(), r->szFt);
      h += Arena::round(r->szFt);
    }
    std::memcpy(h, r->iD.data(), r->szD);
    std::vector<unsigned char>().swap(r->iF);
    std::vector<unsigned char>().swap(r->iFt);
    std::vector<unsigned char>().swap(r->iD);
  }
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->pending.push_back(r.get());
  sv->all.emplace(r->ticket, std::move(r));
  ++sv->submitted;
  sv->cv_work.notify_one();
  return QAP_OK;
}

qap_status qap_server_wait(qap_server* sv, uint64_t ticket, int32_t timeout_ms,
                           const qap_walk_outputs* out, qap_request_times* times) {
  if (!sv || timeout_ms < 0) return QAP_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return QAP_EINVAL;
  Request* r = it->second.get();
  if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
    return QAP_ETIMEOUT;
  const qap_status st = r->result;
  if (st == QAP_ECUDA) snprintf(g_last_error, sizeof(g_last_error), "%s", r->err);
  if (st == QAP_OK && out) {
    const int W = r->params.starts, n = r->di.n;
    const OutLayout OL = out_layout(W, n);
    // the output block's layout on the host equals the device one
    const qap_walk_outputs h = carve_outputs(reinterpret_cast<char*>(r->out.data()), OL, W);
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (dst) std::memcpy(dst, src, bytes);
    };
    cp(out->best_p, h.best_p, (size_t)W * n * 4);
    cp(out->best_cost, h.best_cost, (size_t)W * 8);
    cp(out->final_cost, h.final_cost, (size_t)W * 8);
    cp(out->hash, h.hash, (size_t)W * 8);
    cp(out->descent_hash, h.descent_hash, (size_t)W * 8);
    cp(out->best_iter, h.best_iter, (size_t)W * 4);
    cp(out->iters_done, h.iters_done, (size_t)W * 4);
    cp(out->status, h.status, (size_t)W * 4);
    cp(out->descent_moves, h.descent_moves, (size_t)W * 4);
  }
  if (times) {
    times->queued_us = us_between(r->t_submit, r->t_admit);
    times->device_us = us_between(r->t_admit, r->t_done);
    times->total_us = us_between(r->t_submit, r->t_done);
    times->kernel_start_us = r->k_start_us;
    times->kernel_end_us = r->k_end_us;
  }
  sv->all.erase(it);
  return st;
}

qap_status qap_server_get_stats(qap_server* sv, qap_server_stats* out) {
  if (!sv || !out) return QAP_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->pending = (int64_t)sv->pending.size();
  out->in_flight = sv->in_flight;
  out->arena_bytes = (int64_t)sv->arena.size();
  out->arena_used = (int64_t)sv->arena.used();
  out->peak_in_flight = sv->peak_in_flight;
  return QAP_OK;
}

void qap_server_destroy(qap_server* sv) {
  if (!sv) return;
  if (sv->worker.joinable()) {
    sv->stop = true;
    sv->cv_work.notify_all();
    sv->worker.join();
  }
  for (Slot& sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.k0) cudaEventDestroy(sl.k0);
    if (sl.k1) cudaEventDestroy(sl.k1);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.pinned) cudaFreeHost(sl.pinned);
  }
  for (unsigned char* p : sv->retired) cudaFreeHost(p);
  if (sv->ref) cudaEventDestroy(sv->ref);
  if (sv->slab) cudaFreeHost(sv->slab);
  if (sv->arena_base) cudaFree(sv->arena_base);
  delete sv;
}

}  // extern "C"
