// Continuous-batching prediction service over resident models.
//
// Submitters enqueue requests (host test points, host result buffers).  One
// scheduler thread per server:
//   1. completes in-flight batches whose CUDA event has fired: copies each
//      request's results from the pinned staging arena to the caller's
//      buffers and releases its reservation;
//   2. admits queued requests first-come-first-served while their device
//      bytes fit the budget and their staging fits the pinned arena (their
//      test points are copied into the arena at admission);
//   3. while a stream is free, launches all admitted requests of the model of
//      the oldest admitted request as one batch: host-to-device copies into
//      one stream-ordered allocation, nearest-point lookup + gather-dot over
//      the concatenated points, device-to-host copies of the results, an event;
//   4. sleeps briefly while work is in flight, or waits for a submission.
// Batches on different streams overlap on the device, and requests arriving
// while others run join the next batch of their model.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include "model.cuh"

namespace fmgp {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator of [0, size) (256-byte granules), used for the pinned arena.
class RangeAlloc {
 public:
  explicit RangeAlloc(size_t size) { if (size) free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rem = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rem) free_[start] = rem;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }

 private:
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t id = 0;
  int model = 0;
  const void* Z_host = nullptr;
  int64_t m = 0;
  double* Y_host = nullptr;
  int32_t* N_host = nullptr;
  size_t zbytes = 0, ybytes = 0, nbytes = 0, dev_bytes = 0, stage_bytes = 0, stage_off = 0;
  Clock::time_point t_submit, t_launch, t_done;
  int status = FMGP_OK;
  bool done = false;
};

struct Batch {
  int model = 0;
  int stream = 0;
  std::vector<Request*> reqs;
};

}  // namespace

struct Server {
  std::vector<Model*> models;
  fmgp_server_config cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<Batch*> slot;  // in-flight batch per stream (or null)
  unsigned char* pinned = nullptr;
  RangeAlloc* stage = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> admitted;
  std::unordered_map<uint64_t, Request*> requests;
  int64_t reserved = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  fmgp_server_stats stats{};
  int64_t batched_requests = 0;

  void run();
  void complete(int s);
  void launch(int s, Batch* b);
  bool inflight() const {
    for (auto* b : slot)
      if (b) return true;
    return false;
  }
};

void Server::complete(int s) {
  Batch* b = slot[s];
  cudaError_t e = cudaEventQuery(events[s]);
  if (e == cudaErrorNotReady) return;
  const int status = e == cudaSuccess ? FMGP_OK : FMGP_ECUDA;
  if (e != cudaSuccess) cudaGetLastError();
  const auto now = Clock::now();
  for (Request* r : b->reqs) {
    if (status == FMGP_OK) {
      std::memcpy(r->Y_host, pinned + r->stage_off + r->zbytes, r->ybytes);
      if (r->N_host) std::memcpy(r->N_host, pinned + r->stage_off + r->zbytes + r->ybytes, r->nbytes);
      stats.points += r->m;
    }
    if (r->status == FMGP_OK) r->status = status;
    r->t_done = now;
    r->done = true;
    stage->release(r->stage_off, r->stage_bytes);
    reserved -= (int64_t)r->dev_bytes;
    stats.completed += 1;
  }
  delete b;
  slot[s] = nullptr;
  cv_done.notify_all();
}

void Server::launch(int s, Batch* b) {
  Model& md = *models[b->model];
  cudaStream_t st = streams[s];
  int64_t M = 0;
  for (Request* r : b->reqs) M += r->m;
  const size_t elem = md.dtype == FMGP_F64 ? 8 : 4;
  const size_t zb = RangeAlloc::round((size_t)M * md.d * elem);
  const size_t yb = RangeAlloc::round((size_t)M * md.r * 8);
  const size_t nb = RangeAlloc::round((size_t)M * 4);
  unsigned char* dev = nullptr;
  int rc = FMGP_OK;
  cudaError_t e = cudaMallocAsync((void**)&dev, zb + yb + nb, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = FMGP_ENOMEM;
  }
  const auto now = Clock::now();
  if (rc == FMGP_OK) {
    size_t zo = 0;
    for (Request* r : b->reqs) {
      cudaMemcpyAsync(dev + zo, pinned + r->stage_off, r->zbytes, cudaMemcpyHostToDevice, st);
      zo += r->zbytes;
    }
    double* Yd = (double*)(dev + zb);
    int32_t* Nd = (int32_t*)(dev + zb + yb);
    rc = model_predict(md, dev, M, Yd, Nd, st);
    size_t p = 0;
    for (Request* r : b->reqs) {
      unsigned char* h = pinned + r->stage_off + r->zbytes;
      cudaMemcpyAsync(h, Yd + p * md.r, r->ybytes, cudaMemcpyDeviceToHost, st);
      if (r->N_host) cudaMemcpyAsync(h + r->ybytes, Nd + p, r->nbytes, cudaMemcpyDeviceToHost, st);
      p += r->m;
    }
    cudaFreeAsync(dev, st);
  }
  for (Request* r : b->reqs) {
    r->t_launch = now;
    if (rc != FMGP_OK) r->status = rc;
  }
  cudaEventRecord(events[s], st);
  slot[s] = b;
  stats.batches += 1;
  batched_requests += (int64_t)b->reqs.size();
}

void Server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    for (int s = 0; s < (int)slot.size(); ++s)
      if (slot[s]) complete(s);
    // admission, first come first served, by device bytes and staging space
    while (!queue.empty()) {
      Request* r = queue.front();
      if (reserved + (int64_t)r->dev_bytes > cfg.device_budget_bytes) break;
      size_t off = 0;
      if (!stage->alloc(r->stage_bytes, &off)) break;
      r->stage_off = off;
      std::memcpy(pinned + off, r->Z_host, r->zbytes);
      reserved += (int64_t)r->dev_bytes;
      admitted.push_back(r);
      queue.pop_front();
    }
    // launches: one batch per free stream, model of the oldest admitted request
    for (int s = 0; s < (int)slot.size() && !admitted.empty(); ++s) {
      if (slot[s]) continue;
      Batch* b = new Batch();
      b->model = admitted.front()->model;
      b->stream = s;
      int64_t pts = 0;
      std::vector<Request*> rest;
      for (Request* r : admitted) {
        if (r->model == b->model && (b->reqs.empty() || pts + r->m <= cfg.max_batch_points)) {
          b->reqs.push_back(r);
          pts += r->m;
        } else {
          rest.push_back(r);
        }
      }
      admitted.swap(rest);
      launch(s, b);
    }
    if (stop && queue.empty() && admitted.empty() && !inflight()) break;
    if (inflight()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
}

}  // namespace fmgp

using namespace fmgp;

extern "C" int fmgp_server_create(fmgp_model* const* models, int32_t count,
                                  const fmgp_server_config* cfg, fmgp_server** out) {
  if (!out || !models || count < 1 || !cfg) {
    set_error("models, count >= 1, cfg and out are required");
    return FMGP_EINVAL;
  }
  *out = nullptr;
  if (cfg->streams < 1 || cfg->streams > 16 || cfg->device_budget_bytes <= 0 ||
      cfg->host_staging_bytes <= 0 || cfg->max_batch_points < 1) {
    set_error("server config invalid (streams 1..16, positive budgets and batch cap)");
    return FMGP_EINVAL;
  }
  for (int i = 0; i < count; ++i)
    if (!models[i]) {
      set_error("model %d is NULL", i);
      return FMGP_EINVAL;
    }
  Server* s = new Server();
  s->cfg = *cfg;
  for (int i = 0; i < count; ++i) s->models.push_back(reinterpret_cast<Model*>(models[i]));
  cudaGetDevice(&s->device);
  cudaError_t e = cudaHostAlloc((void**)&s->pinned, (size_t)cfg->host_staging_bytes,
                                cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_error("cudaHostAlloc(%lld) failed", (long long)cfg->host_staging_bytes);
    return FMGP_ENOMEM;
  }
  s->stage = new RangeAlloc((size_t)cfg->host_staging_bytes);
  for (int i = 0; i < cfg->streams; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    s->streams.push_back(st);
    s->events.push_back(ev);
    s->slot.push_back(nullptr);
  }
  s->worker = std::thread([s]() { s->run(); });
  *out = reinterpret_cast<fmgp_server*>(s);
  return FMGP_OK;
}

extern "C" int fmgp_server_submit(fmgp_server* srv, int32_t model, const void* Z_host, int64_t m,
                                  double* Yhat_host, int32_t* nearest_host,
                                  uint64_t* request_id) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !request_id) { set_error("server and request_id are required"); return FMGP_EINVAL; }
  if (model < 0 || model >= (int)s->models.size()) {
    set_error("model %d out of range", model);
    return FMGP_EINVAL;
  }
  if (m < 1 || !Z_host || !Yhat_host) {
    set_error("m >= 1, Z_host and Yhat_host are required");
    return FMGP_EINVAL;
  }
  const Model& md = *s->models[model];
  Request* r = new Request();
  r->model = model;
  r->Z_host = Z_host;
  r->m = m;
  r->Y_host = Yhat_host;
  r->N_host = nearest_host;
  const size_t elem = md.dtype == FMGP_F64 ? 8 : 4;
  r->zbytes = (size_t)m * md.d * elem;
  r->ybytes = (size_t)m * md.r * 8;
  r->nbytes = nearest_host ? (size_t)m * 4 : 0;
  r->stage_bytes = r->zbytes + r->ybytes + r->nbytes;
  // device bytes: inputs, outputs, nearest indices, and the double-float copy of Z
  r->dev_bytes = (size_t)m * (md.d * elem + md.r * 8 + 4 +
                              (md.prec == FMGP_PREC_MIXED ? md.d * 8 : 0)) + 3 * 256;
  if ((int64_t)r->dev_bytes > s->cfg.device_budget_bytes ||
      (int64_t)RangeAlloc::round(r->stage_bytes) > s->cfg.host_staging_bytes) {
    delete r;
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.rejected += 1;
    set_error("request of %lld points exceeds the server's memory budget", (long long)m);
    return FMGP_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      set_error("server is shutting down");
      return FMGP_EINVAL;
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->requests[r->id] = r;
    s->queue.push_back(r);
    s->stats.submitted += 1;
    *request_id = r->id;
  }
  s->cv_work.notify_one();
  return FMGP_OK;
}

extern "C" int fmgp_server_wait(fmgp_server* srv, uint64_t request_id, int32_t timeout_ms) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return FMGP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end()) {
    set_error("unknown request %llu", (unsigned long long)request_id);
    return FMGP_EINVAL;
  }
  Request* r = it->second;
  auto pred = [r]() { return r->done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return FMGP_ETIMEOUT;
  if (r->status != FMGP_OK) set_error("request %llu failed", (unsigned long long)request_id);
  return r->status;
}

extern "C" int fmgp_server_request_times(fmgp_server* srv, uint64_t request_id, double* queue_ms,
                                         double* total_ms) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return FMGP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end() || !it->second->done) return FMGP_EINVAL;
  Request* r = it->second;
  using ms = std::chrono::duration<double, std::milli>;
  if (queue_ms) *queue_ms = ms(r->t_launch - r->t_submit).count();
  if (total_ms) *total_ms = ms(r->t_done - r->t_submit).count();
  return FMGP_OK;
}

extern "C" int fmgp_server_release(fmgp_server* srv, uint64_t request_id) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return FMGP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(request_id);
  if (it == s->requests.end() || !it->second->done) {
    set_error("request %llu is unknown or not finished", (unsigned long long)request_id);
    return FMGP_EINVAL;
  }
  delete it->second;
  s->requests.erase(it);
  return FMGP_OK;
}

extern "C" int fmgp_server_get_stats(fmgp_server* srv, fmgp_server_stats* out) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !out) return FMGP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->mean_batch_requests =
      s->stats.batches ? (double)s->batched_requests / (double)s->stats.batches : 0.0;
  return FMGP_OK;
}

extern "C" int fmgp_server_destroy(fmgp_server* srv) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return FMGP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->requests) delete kv.second;
  for (size_t i = 0; i < s->streams.size(); ++i) {
    cudaStreamSynchronize(s->streams[i]);
    cudaEventDestroy(s->events[i]);
    cudaStreamDestroy(s->streams[i]);
  }
  cudaFreeHost(s->pinned);
  delete s->stage;
  delete s;
  return FMGP_OK;
}
