// Request server: the in-process analogue of serving the tracking chain as a service
// (Sec. 1 Fig. 1 and Sec. 3: clients send events, the server batches the requests,
// runs them on the coprocessor and returns the results; several requests are in
// flight on one GPU, Sec. 3.2 and Sec. 4.2).  No network and no inference server.
//
// Continuous batching: the device budget is split into slots, each a context with its
// own stream and workspace.  Submitted events wait in a FIFO; a dispatcher thread fills
// every free slot with the longest prefix of the queue that fits the slot (events,
// hits, and an estimate of the cells, which grow with the square of the hit count),
// stages it in pinned memory and enqueues the whole chain as the slot's CUDA graph.
// Slots run concurrently on the GPU; as each finishes, its results are copied back
// (counters first, then exactly the ntuplets found) and handed to the waiting tickets,
// and the slot takes the next requests.  A batch that still overflows its slot is split
// into single events, each of which fits by construction.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ptca_internal.cuh"

using namespace ptca;
using Clock = std::chrono::steady_clock;

namespace {

constexpr double kCellsPerHit2 = 1.6e-3;  // cells ~ 1.6e-3 * hits^2 (PU200 calibration)
constexpr int64_t kMaxRequestHits = 65536;

struct Request {
  uint64_t ticket = 0;
  std::vector<float> x, y, z;
  std::vector<uint8_t> layer;
  bool solo = false;  // must run alone (its batch overflowed)
  bool done = false;
  pt_status status = PT_OK;
  std::string err;
  std::vector<int32_t> hits;
  std::vector<uint8_t> nhits;
  std::vector<pt_track> tracks;
  Clock::time_point t_submit, t_done;
  int64_t n() const { return (int64_t)x.size(); }
};
using ReqPtr = std::shared_ptr<Request>;

struct Slot {
  pt_ctx* ctx = nullptr;
  int64_t max_events = 0, max_hits = 0, max_nt = 0;
  double cell_budget = 0;
  float *hx = nullptr, *hy = nullptr, *hz = nullptr;
  uint8_t* hl = nullptr;
  int64_t* hoff = nullptr;
  int32_t* rh = nullptr;
  uint8_t* rn = nullptr;
  pt_track* rt = nullptr;
  int64_t* roff = nullptr;
  cudaEvent_t ev = nullptr;
  int state = 0;  // 0 free, 1 running (counters pending), 2 copying results
  std::vector<ReqPtr> batch;
  int64_t S = 0;
};

double est_cells(int64_t n) { return kCellsPerHit2 * (double)n * (double)n; }

}  // namespace

struct pt_server {
  int device = 0;
  std::vector<Slot> slots;
  std::deque<ReqPtr> queue;
  std::unordered_map<uint64_t, ReqPtr> reqs;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<double> lat_ms;
  int64_t completed = 0;
  int64_t finished = 0;      // requests completed since creation (never reset)
  int64_t batches = 0;       // batches launched
  int64_t split = 0;         // batches that overflowed their slot and were split
  int64_t requeued = 0;      // events those splits sent back to run alone
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

pt_status sfail(pt_status st, const std::string& m) {
  set_last_error(m.c_str());
  return st;
}

void finish(pt_server* s, const ReqPtr& r, pt_status st, const std::string& err) {
  r->status = st;
  r->err = err;
  r->done = true;
  r->t_done = Clock::now();
  s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  s->completed += 1;
  s->finished += 1;
  s->t_last = r->t_done;
}

// Fills a free slot from the front of the queue; returns true if it launched work.
bool dispatch(pt_server* s, Slot& sl) {
  if (s->queue.empty()) return false;
  sl.batch.clear();
  int64_t hits = 0;
  double cells = 0;
  while (!s->queue.empty()) {
    ReqPtr r = s->queue.front();
    const int64_t n = r->n();
    const bool fits = (int64_t)sl.batch.size() < sl.max_events && hits + n <= sl.max_hits &&
                      cells + est_cells(n) <= sl.cell_budget;
    if (!sl.batch.empty() && (!fits || r->solo || sl.batch.front()->solo)) break;
    s->queue.pop_front();
    sl.batch.push_back(r);
    hits += n;
    cells += est_cells(n);
    if (r->solo) break;
  }
  const int E = (int)sl.batch.size();
  sl.hoff[0] = 0;
  for (int e = 0; e < E; ++e) {
    const Request& r = *sl.batch[e];
    const int64_t o = sl.hoff[e], n = r.n();
    std::memcpy(sl.hx + o, r.x.data(), n * 4);
    std::memcpy(sl.hy + o, r.y.data(), n * 4);
    std::memcpy(sl.hz + o, r.z.data(), n * 4);
    std::memcpy(sl.hl + o, r.layer.data(), n);
    sl.hoff[e + 1] = o + n;
  }
  s->batches += 1;
  pt_status st = pt_enqueue_batch(sl.ctx, E, sl.hoff, sl.hx, sl.hy, sl.hz, sl.hl, 0);
  if (st == PT_OK) st = ctx_counters_async(sl.ctx, sl.ev);
  if (st != PT_OK) {
    const std::string m = pt_last_error();
    for (auto& r : sl.batch) finish(s, r, st, m);
    sl.batch.clear();
    s->cv_done.notify_all();
    return true;
  }
  sl.state = 1;
  return true;
}

// Advances a running slot if its current step has completed; returns true on progress.
bool advance(pt_server* s, Slot& sl) {
  if (sl.state == 0) return false;
  const cudaError_t q = cudaEventQuery(sl.ev);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) {
    const std::string m = std::string("CUDA error in a served batch: ") + cudaGetErrorString(q);
    for (auto& r : sl.batch) finish(s, r, PT_ERR_CUDA, m);
    sl.batch.clear();
    sl.state = 0;
    s->cv_done.notify_all();
    return true;
  }
  if (sl.state == 1) {
    int64_t S = 0;
    pt_status st = ctx_read_counters(sl.ctx, &S);
    if (st == PT_ERR_CAPACITY && sl.batch.size() > 1) {
      // split the batch: every event runs alone, ahead of the rest of the queue
      s->split += 1;
      s->requeued += (int64_t)sl.batch.size();
      for (auto it = sl.batch.rbegin(); it != sl.batch.rend(); ++it) {
        (*it)->solo = true;
        s->queue.push_front(*it);
      }
      sl.batch.clear();
      sl.state = 0;
      return true;
    }
    if (st == PT_OK && S > sl.max_nt) st = PT_ERR_CAPACITY;
    if (st == PT_OK) st = ctx_results_async(sl.ctx, S, sl.rh, sl.rn, sl.rt, sl.roff, sl.ev);
    if (st != PT_OK) {
      const std::string m = pt_last_error();
      for (auto& r : sl.batch) finish(s, r, st, m);
      sl.batch.clear();
      sl.state = 0;
      s->cv_done.notify_all();
      return true;
    }
    sl.S = S;
    sl.state = 2;
    return true;
  }
  // state 2: results are in pinned memory; hand them to the requests
  for (size_t e = 0; e < sl.batch.size(); ++e) {
    Request& r = *sl.batch[e];
    const int64_t a = sl.roff[e], b = sl.roff[e + 1];
    r.hits.assign(sl.rh + a * kMaxHits, sl.rh + b * kMaxHits);
    r.nhits.assign(sl.rn + a, sl.rn + b);
    r.tracks.assign(sl.rt + a, sl.rt + b);
    finish(s, sl.batch[e], PT_OK, "");
  }
  sl.batch.clear();
  sl.state = 0;
  s->cv_done.notify_all();
  return true;
}

void run(pt_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progress = false;
    for (auto& sl : s->slots) progress |= advance(s, sl);
    for (auto& sl : s->slots)
      if (sl.state == 0) progress |= dispatch(s, sl);
    bool busy = !s->queue.empty();
    for (auto& sl : s->slots) busy |= sl.state != 0;
    if (s->stop && !busy) break;
    if (!progress) {
      if (busy) {
        // GPU work in flight: poll its events again shortly
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
  }
}

void free_slot(Slot& sl) {
  if (sl.ctx) pt_destroy(sl.ctx);
  for (void* p : {(void*)sl.hx, (void*)sl.hy, (void*)sl.hz, (void*)sl.hl, (void*)sl.hoff,
                  (void*)sl.rh, (void*)sl.rn, (void*)sl.rt, (void*)sl.roff})
    if (p) cudaFreeHost(p);
  if (sl.ev) cudaEventDestroy(sl.ev);
  sl = Slot{};
}

}  // namespace

namespace ptca {
int64_t server_finished(pt_server* s) {
  std::lock_guard<std::mutex> lk(s->mu);
  return s->finished;
}
}  // namespace ptca

extern "C" {

pt_status pt_server_create(const pt_geometry* geom, const pt_cuts* cuts, int device,
                           size_t device_budget_bytes, int max_slots, pt_server** out) {
  set_last_error("");
  if (!out || !geom || !cuts) return sfail(PT_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64) return sfail(PT_ERR_INVALID, "max_slots must be in [1, 64]");
  // largest per-slot capacity (in units of one PU200-sized event) within budget / slots
  const size_t per_slot = device_budget_bytes / (size_t)max_slots;
  auto cap_for = [](int64_t s) {
    pt_capacity c{};
    c.max_events = 4 * s;
    c.max_hits = s * 49152;
    c.max_cells = s * 3500000;
    c.max_links = s * 262144;
    c.max_ntuplets = s * 196608;
    c.phi_bins = 1024;
    return c;
  };
  int64_t units = 0;
  for (int64_t u = 16; u >= 1; --u) {
    pt_capacity c = cap_for(u);
    size_t bytes = 0;
    if (pt_workspace_size(&c, &bytes) == PT_OK && bytes <= per_slot) {
      units = u;
      break;
    }
  }
  if (units == 0)
    return sfail(PT_ERR_NOMEM, "device budget too small for one slot of one PU200-sized event");
  pt_server* s = new pt_server();
  s->device = device;
  s->slots.resize(max_slots);
  for (auto& sl : s->slots) {
    pt_capacity c = cap_for(units);
    pt_status st = pt_create(geom, cuts, &c, device, nullptr, 0, nullptr, &sl.ctx);
    bool ok = st == PT_OK;
    sl.max_events = c.max_events;
    sl.max_hits = c.max_hits;
    sl.max_nt = c.max_ntuplets;
    sl.cell_budget = 0.8 * (double)c.max_cells;
    ok = ok && cudaMallocHost(&sl.hx, c.max_hits * 4) == cudaSuccess &&
         cudaMallocHost(&sl.hy, c.max_hits * 4) == cudaSuccess &&
         cudaMallocHost(&sl.hz, c.max_hits * 4) == cudaSuccess &&
         cudaMallocHost(&sl.hl, c.max_hits) == cudaSuccess &&
         cudaMallocHost(&sl.hoff, (c.max_events + 1) * 8) == cudaSuccess &&
         cudaMallocHost(&sl.rh, c.max_ntuplets * kMaxHits * 4) == cudaSuccess &&
         cudaMallocHost(&sl.rn, c.max_ntuplets) == cudaSuccess &&
         cudaMallocHost(&sl.rt, c.max_ntuplets * sizeof(pt_track)) == cudaSuccess &&
         cudaMallocHost(&sl.roff, (c.max_events + 1) * 8) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      const std::string m = st == PT_OK ? "pinned host allocation failed" : pt_last_error();
      for (auto& t : s->slots) free_slot(t);
      delete s;
      return sfail(st == PT_OK ? PT_ERR_NOMEM : st, m);
    }
  }
  s->worker = std::thread(run, s);
  *out = s;
  return PT_OK;
}

pt_status pt_server_set_gate(pt_server* s, const float* w, float tau) {
  set_last_error("");
  if (!s) return sfail(PT_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  // wait until no slot is running, so no batch mixes forms
  while (true) {
    bool busy = false;
    for (auto& sl : s->slots) busy |= sl.state != 0;
    if (!busy) break;
    lk.unlock();
    std::this_thread::sleep_for(std::chrono::microseconds(100));
    lk.lock();
  }
  for (auto& sl : s->slots) {
    const pt_status st = pt_set_gate(sl.ctx, w, tau);
    if (st != PT_OK) return st;
  }
  return PT_OK;
}

pt_status pt_submit(pt_server* s, int64_t n, const float* x, const float* y, const float* z,
                    const uint8_t* layer, uint64_t* ticket) {
  set_last_error("");
  if (!s || !ticket) return sfail(PT_ERR_INVALID, "NULL argument");
  if (n < 0 || (n > 0 && (!x || !y || !z || !layer))) return sfail(PT_ERR_INVALID, "bad hit arrays");
  if (n > kMaxRequestHits || n > s->slots[0].max_hits ||
      est_cells(n) > s->slots[0].cell_budget)
    return sfail(PT_ERR_CAPACITY, "event too large for a slot of this server's budget");
  for (int64_t i = 0; i < n; ++i)
    if (layer[i] >= kLayers) return sfail(PT_ERR_INVALID, "layer code > 9");
  auto r = std::make_shared<Request>();
  r->x.assign(x, x + n);
  r->y.assign(y, y + n);
  r->z.assign(z, z + n);
  r->layer.assign(layer, layer + n);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return sfail(PT_ERR_INVALID, "server is stopping");
    r->ticket = s->next_ticket++;
    if (!s->any) {
      s->any = true;
      s->t_first = r->t_submit;
    }
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return PT_OK;
}

pt_status pt_poll(pt_server* s, uint64_t ticket, int64_t timeout_us, int32_t* hits,
                  uint8_t* nhits, pt_track* tracks, int64_t cap, int64_t* n) {
  set_last_error("");
  if (!s) return sfail(PT_ERR_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(PT_ERR_INVALID, "unknown ticket");
  ReqPtr r = it->second;
  if (!r->done) {
    if (timeout_us == 0) return sfail(PT_ERR_NOT_READY, "not ready");
    if (timeout_us < 0) {
      s->cv_done.wait(lk, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                    [&] { return r->done; })) {
      return sfail(PT_ERR_TIMEOUT, "timed out");
    }
  }
  const int64_t S = (int64_t)r->nhits.size();
  if (n) *n = S;
  if (r->status != PT_OK) {
    const pt_status st = r->status;
    const std::string m = r->err;
    s->reqs.erase(ticket);
    return sfail(st, m);
  }
  if (cap < S) return sfail(PT_ERR_CAPACITY, "output capacity too small; *n holds the size");
  if (hits && S) std::memcpy(hits, r->hits.data(), (size_t)S * kMaxHits * 4);
  if (nhits && S) std::memcpy(nhits, r->nhits.data(), (size_t)S);
  if (tracks && S) std::memcpy(tracks, r->tracks.data(), (size_t)S * sizeof(pt_track));
  s->reqs.erase(ticket);
  return PT_OK;
}

pt_status pt_server_stats(pt_server* s, double* p50_ms, double* p99_ms, double* events_per_s,
                          int64_t* n_done) {
  set_last_error("");
  if (!s) return sfail(PT_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->lat_ms;
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (events_per_s) {
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    *events_per_s = span > 0 ? (double)s->completed / span : 0.0;
  }
  if (n_done) *n_done = s->completed;
  return PT_OK;
}

pt_status pt_server_counters(pt_server* s, int64_t* batches, int64_t* split_batches,
                             int64_t* requeued_events) {
  set_last_error("");
  if (!s) return sfail(PT_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->batches;
  if (split_batches) *split_batches = s->split;
  if (requeued_events) *requeued_events = s->requeued;
  return PT_OK;
}

pt_status pt_server_reset_stats(pt_server* s) {
  set_last_error("");
  if (!s) return sfail(PT_ERR_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_ms.clear();
  s->completed = 0;
  s->batches = s->split = s->requeued = 0;
  s->any = false;
  return PT_OK;
}

pt_status pt_server_destroy(pt_server* s) {
  if (!s) return PT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& sl : s->slots) free_slot(sl);
  delete s;
  return PT_OK;
}

}  // extern "C"
