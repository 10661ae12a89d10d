// Continuous-batching prediction service over resident models.
//
// Submitters enqueue requests (host test points, host result buffers).  One
// scheduler thread per server:
//   1. completes in-flight batches whose CUDA event has fired; a request is
//      finished when the last of its pieces is (its results are then copied
//      from the pinned staging arena to the caller's buffers and its
//      reservation released);
//   2. admits queued requests first-come-first-served while their device
//      bytes fit the budget and their staging fits the pinned arena, and
//      splits each into pieces of at most max_batch_points test points;
//   3. while a stream is free, launches the pending pieces of the model of the
//      oldest pending piece, up to max_batch_points points, as one batch:
//      host-to-device copies into one stream-ordered allocation,
//      nearest-point lookup + gather-dot over the concatenated points,
//      device-to-host copies of the results, an event;
//   4. sleeps briefly while work is in flight, or waits for a submission.
// Batches on different streams overlap on the device; requests arriving
// while others run join the next batch of their model, and a large request
// occupies a stream for one piece at a time, so small requests behind it
// wait for at most one piece.  The server mutex guards only the queues and
// the request table: copies into the staging arena and every CUDA call are
// made by the scheduler thread without it, so submitters never wait on them.
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
  int pending = 0;     // pieces not yet completed
  bool launched = false;
  bool done = false;
};

// Test points [off, off + cnt) of a request.
struct Piece {
  Request* r;
  int64_t off, cnt;
};

struct Batch {
  int model = 0;
  int stream = 0;
  std::vector<Piece> pieces;
  int status = FMGP_OK;
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
  std::deque<Piece> admitted;  // pieces of admitted requests, oldest first
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

// Called with mu held.
void Server::complete(int s) {
  Batch* b = slot[s];
  cudaError_t e = cudaEventQuery(events[s]);
  if (e == cudaErrorNotReady) return;
  const int status = e == cudaSuccess ? b->status : FMGP_ECUDA;
  if (e != cudaSuccess) cudaGetLastError();
  const auto now = Clock::now();
  for (const Piece& pc : b->pieces) {
    Request* r = pc.r;
    if (r->status == FMGP_OK) r->status = status;
    if (--r->pending > 0) continue;
    if (r->status == FMGP_OK) {
      std::memcpy(r->Y_host, pinned + r->stage_off + r->zbytes, r->ybytes);
      if (r->N_host) std::memcpy(r->N_host, pinned + r->stage_off + r->zbytes + r->ybytes, r->nbytes);
      stats.points += r->m;
    }
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

// Called without mu: only the scheduler thread uses the streams, events and
// the staging ranges of admitted requests.
void Server::launch(int s, Batch* b) {
  Model& md = *models[b->model];
  cudaStream_t st = streams[s];
  int64_t M = 0;
  for (const Piece& pc : b->pieces) M += pc.cnt;
  const size_t elem = md.dtype == FMGP_F64 ? 8 : 4;
  const size_t zrow = (size_t)md.d * elem, yrow = (size_t)md.r * 8;
  const size_t zb = RangeAlloc::round((size_t)M * zrow);
  const size_t yb = RangeAlloc::round((size_t)M * yrow);
  const size_t nb = RangeAlloc::round((size_t)M * 4);
  unsigned char* dev = nullptr;
  int rc = FMGP_OK;
  cudaError_t e = cudaMallocAsync((void**)&dev, zb + yb + nb, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = FMGP_ENOMEM;
  }
  if (rc == FMGP_OK) {
    size_t zo = 0;
    for (const Piece& pc : b->pieces) {
      cudaMemcpyAsync(dev + zo, pinned + pc.r->stage_off + pc.off * zrow, pc.cnt * zrow,
                      cudaMemcpyHostToDevice, st);
      zo += pc.cnt * zrow;
    }
    double* Yd = (double*)(dev + zb);
    int32_t* Nd = (int32_t*)(dev + zb + yb);
    rc = model_predict(md, dev, M, Yd, Nd, st);
    int64_t p = 0;
    for (const Piece& pc : b->pieces) {
      Request* r = pc.r;
      unsigned char* h = pinned + r->stage_off + r->zbytes;
      cudaMemcpyAsync(h + pc.off * yrow, Yd + p * md.r, pc.cnt * yrow, cudaMemcpyDeviceToHost, st);
      if (r->N_host)
        cudaMemcpyAsync(h + r->ybytes + pc.off * 4, Nd + p, pc.cnt * 4, cudaMemcpyDeviceToHost, st);
      p += pc.cnt;
    }
    cudaFreeAsync(dev, st);
  }
  b->status = rc;
  cudaEventRecord(events[s], st);
}

void Server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  std::vector<Request*> to_stage;
  std::vector<Batch*> to_launch;
  for (;;) {
    for (int s = 0; s < (int)slot.size(); ++s)
      if (slot[s]) complete(s);
    // admission, first come first served, by device bytes and staging space
    to_stage.clear();
    while (!queue.empty()) {
      Request* r = queue.front();
      if (reserved + (int64_t)r->dev_bytes > cfg.device_budget_bytes) break;
      size_t off = 0;
      if (!stage->alloc(r->stage_bytes, &off)) break;
      r->stage_off = off;
      reserved += (int64_t)r->dev_bytes;
      to_stage.push_back(r);
      queue.pop_front();
    }
    if (!to_stage.empty()) {
      lk.unlock();  // the arena range is this thread's: copy without the lock
      for (Request* r : to_stage) std::memcpy(pinned + r->stage_off, r->Z_host, r->zbytes);
      lk.lock();
      for (Request* r : to_stage) {
        const int64_t piece = cfg.max_batch_points;
        for (int64_t off = 0; off < r->m; off += piece) {
          admitted.push_back(Piece{r, off, std::min<int64_t>(piece, r->m - off)});
          ++r->pending;
        }
      }
    }
    // batches: per free stream, pending pieces of the model of the oldest
    // pending piece, up to max_batch_points points
    to_launch.clear();
    for (int s = 0; s < (int)slot.size() && !admitted.empty(); ++s) {
      if (slot[s]) continue;
      Batch* b = new Batch();
      b->model = admitted.front().r->model;
      b->stream = s;
      int64_t pts = 0;
      std::deque<Piece> rest;
      for (const Piece& pc : admitted) {
        if (pc.r->model == b->model && (b->pieces.empty() || pts + pc.cnt <= cfg.max_batch_points)) {
          b->pieces.push_back(pc);
          pts += pc.cnt;
        } else {
          rest.push_back(pc);
        }
      }
      admitted.swap(rest);
      const auto now = Clock::now();
      for (const Piece& pc : b->pieces)
        if (!pc.r->launched) {
          pc.r->launched = true;
          pc.r->t_launch = now;
        }
      slot[s] = b;
      stats.batches += 1;
      batched_requests += (int64_t)b->pieces.size();
      to_launch.push_back(b);
    }
    if (!to_launch.empty()) {
      lk.unlock();
      for (Batch* b : to_launch) launch(b->stream, b);
      lk.lock();
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
