// Request router over several server instances: the in-process analogue of serving
// one model through several model instances (Sec. 3.2 and Sec. 4.2: the inference
// server balances requests over instances of the model on one GPU, or over GPUs).
// Each instance is a pt_server with its own dispatcher thread, slots and device budget
// (on the device given for it); a submission goes to the instance with the fewest
// requests outstanding (ties: the lowest index), and the router's ticket names the
// instance and that instance's ticket.  An instance's load is its requests submitted
// and not yet completed on the device.  Statistics merge the instances' latencies.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "ptca_internal.cuh"

using namespace ptca;

struct pt_router {
  std::vector<pt_server*> inst;
  std::vector<int64_t> submitted;  // per instance, since creation
  std::mutex mu;
};

namespace {

constexpr int kInstBits = 8;  // router ticket = instance ticket << 8 | instance
constexpr uint64_t kInstMask = (1u << kInstBits) - 1u;

pt_status rfail(pt_status st, const std::string& m) {
  set_last_error(m.c_str());
  return st;
}

}  // namespace

extern "C" {

pt_status pt_router_create(const pt_geometry* geom, const pt_cuts* cuts, const int* devices,
                           int n_instances, size_t budget_per_instance, int slots_per_instance,
                           pt_router** out) {
  set_last_error("");
  if (!out || !geom || !cuts || !devices) return rfail(PT_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (n_instances < 1 || n_instances > (int)kInstMask)
    return rfail(PT_ERR_INVALID, "n_instances must be in [1, 255]");
  pt_router* r = new pt_router();
  for (int i = 0; i < n_instances; ++i) {
    pt_server* s = nullptr;
    const pt_status st = pt_server_create(geom, cuts, devices[i], budget_per_instance,
                                          slots_per_instance, &s);
    if (st != PT_OK) {
      const std::string m = pt_last_error();
      for (pt_server* t : r->inst) pt_server_destroy(t);
      delete r;
      return rfail(st, "instance " + std::to_string(i) + ": " + m);
    }
    r->inst.push_back(s);
    r->submitted.push_back(0);
  }
  *out = r;
  return PT_OK;
}

pt_status pt_router_set_gate(pt_router* r, const float* w, float tau) {
  set_last_error("");
  if (!r) return rfail(PT_ERR_INVALID, "router is NULL");
  for (pt_server* s : r->inst) {
    const pt_status st = pt_server_set_gate(s, w, tau);
    if (st != PT_OK) return st;
  }
  return PT_OK;
}

pt_status pt_router_submit(pt_router* r, int64_t n, const float* x, const float* y,
                           const float* z, const uint8_t* layer, uint64_t* ticket) {
  set_last_error("");
  if (!r || !ticket) return rfail(PT_ERR_INVALID, "NULL argument");
  size_t k = 0;
  {
    std::lock_guard<std::mutex> lk(r->mu);
    int64_t best = 0;
    for (size_t i = 0; i < r->inst.size(); ++i) {
      const int64_t load = r->submitted[i] - server_finished(r->inst[i]);
      if (i == 0 || load < best) {
        best = load;
        k = i;
      }
    }
    r->submitted[k] += 1;  // counted before the submit, so that racing clients spread
  }
  uint64_t t = 0;
  const pt_status st = pt_submit(r->inst[k], n, x, y, z, layer, &t);
  if (st != PT_OK) {
    std::lock_guard<std::mutex> lk(r->mu);
    r->submitted[k] -= 1;
    return st;
  }
  *ticket = (t << kInstBits) | (uint64_t)k;
  return PT_OK;
}

pt_status pt_router_poll(pt_router* r, uint64_t ticket, int64_t timeout_us, int32_t* hits,
                         uint8_t* nhits, pt_track* tracks, int64_t cap, int64_t* n) {
  set_last_error("");
  if (!r) return rfail(PT_ERR_INVALID, "router is NULL");
  const size_t k = (size_t)(ticket & kInstMask);
  if (k >= r->inst.size()) return rfail(PT_ERR_INVALID, "unknown ticket");
  return pt_poll(r->inst[k], ticket >> kInstBits, timeout_us, hits, nhits, tracks, cap, n);
}

pt_status pt_router_stats(pt_router* r, double* p50_ms, double* p99_ms, double* events_per_s,
                          int64_t* n_done, int64_t* per_instance_done) {
  set_last_error("");
  if (!r) return rfail(PT_ERR_INVALID, "router is NULL");
  double rate = 0.0, wp50 = 0.0, p99 = 0.0;
  int64_t done = 0;
  for (size_t i = 0; i < r->inst.size(); ++i) {
    double a = 0, b = 0, c = 0;
    int64_t d = 0;
    const pt_status st = pt_server_stats(r->inst[i], &a, &b, &c, &d);
    if (st != PT_OK) return st;
    if (per_instance_done) per_instance_done[i] = d;
    rate += c;
    wp50 += a * (double)d;
    p99 = std::max(p99, b);
    done += d;
  }
  // p50: the instances' medians weighted by their requests; p99: the worst instance's
  if (p50_ms) *p50_ms = done ? wp50 / (double)done : 0.0;
  if (p99_ms) *p99_ms = p99;
  if (events_per_s) *events_per_s = rate;
  if (n_done) *n_done = done;
  return PT_OK;
}

pt_status pt_router_reset_stats(pt_router* r) {
  set_last_error("");
  if (!r) return rfail(PT_ERR_INVALID, "router is NULL");
  for (pt_server* s : r->inst) pt_server_reset_stats(s);
  return PT_OK;
}

pt_status pt_router_destroy(pt_router* r) {
  if (!r) return PT_OK;
  for (pt_server* s : r->inst) pt_server_destroy(s);
  delete r;
  return PT_OK;
}

}  // extern "C"
