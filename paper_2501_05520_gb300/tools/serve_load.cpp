// Open-loop load generator for the request server (pt_server_*), native threads only.
//
//   serve_load EVENTS_FILE RATE SECONDS CLIENTS SLOTS BUDGET_BYTES GATE_FILE|- SEED [INSTANCES]
//
// INSTANCES > 1 serves through a pt_router of that many server instances on device 0,
// each with SLOTS slots and BUDGET_BYTES; otherwise one pt_server.
// EVENTS_FILE holds a pool of events, each as int64 n followed by float32 x[n], y[n],
// z[n] and uint8 layer[n] (little-endian).  CLIENTS threads submit events from the pool
// at Poisson arrival times (RATE events/s in all, for SECONDS), never waiting for their
// results: each client has a collector thread that polls its tickets in submission
// order.  GATE_FILE: 5057 float32 weights and a float32 threshold, or "-" for the plain
// form.  Prints one JSON line: the offered rate; sustained events/s = results returned
// within the offered window over its length; throughput = all results over the window
// plus the time the server took to drain the backlog after it; the server's latency
// percentiles (submit to result ready) and the clients' (submit to poll returning).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "pt_ca.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Event {
  std::vector<float> x, y, z;
  std::vector<uint8_t> layer;
};

bool read_events(const char* path, std::vector<Event>* out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  while (true) {
    int64_t n = 0;
    if (std::fread(&n, 8, 1, f) != 1) break;
    if (n < 0 || n > (1 << 20)) {
      std::fclose(f);
      return false;
    }
    Event e;
    e.x.resize(n);
    e.y.resize(n);
    e.z.resize(n);
    e.layer.resize(n);
    bool ok = std::fread(e.x.data(), 4, n, f) == (size_t)n && std::fread(e.y.data(), 4, n, f) == (size_t)n &&
              std::fread(e.z.data(), 4, n, f) == (size_t)n && std::fread(e.layer.data(), 1, n, f) == (size_t)n;
    if (!ok) {
      std::fclose(f);
      return false;
    }
    out->push_back(std::move(e));
  }
  std::fclose(f);
  return !out->empty();
}

struct Pending {
  uint64_t ticket;
  Clock::time_point t_submit;
};

struct Client {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> q;
  bool done = false;
  std::vector<double> lat_ms;
  int64_t in_window = 0;  // results returned before the offered window closed
  int64_t errors = 0;
};

double pct(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  const size_t k = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
  std::nth_element(v.begin(), v.begin() + k, v.end());
  return v[k];
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 9 && argc != 10) {
    std::fprintf(stderr,
                 "usage: %s EVENTS RATE SECONDS CLIENTS SLOTS BUDGET_BYTES GATE|- SEED [INSTANCES]\n",
                 argv[0]);
    return 2;
  }
  const int instances = argc == 10 ? std::atoi(argv[9]) : 1;
  std::vector<Event> pool;
  if (!read_events(argv[1], &pool)) {
    std::fprintf(stderr, "cannot read events from %s\n", argv[1]);
    return 2;
  }
  const double rate = std::atof(argv[2]), seconds = std::atof(argv[3]);
  const int clients = std::atoi(argv[4]), slots = std::atoi(argv[5]);
  const size_t budget = (size_t)std::atoll(argv[6]);
  const unsigned seed = (unsigned)std::atoi(argv[8]);
  if (!(rate > 0) || !(seconds > 0) || clients < 1 || clients > 256 || instances < 1 ||
      instances > 64) {
    std::fprintf(stderr, "bad arguments\n");
    return 2;
  }
  std::vector<float> gate;
  if (std::strcmp(argv[7], "-") != 0) {
    gate.resize(5058);
    FILE* f = std::fopen(argv[7], "rb");
    if (!f || std::fread(gate.data(), 4, 5058, f) != 5058) {
      std::fprintf(stderr, "cannot read the gate file\n");
      return 2;
    }
    std::fclose(f);
  }
  pt_geometry geom{3.8f};
  pt_cuts cuts{};
  {
    // the library's frozen cut constants (pt_min 0.45 GeV), passed in as float32 bits
    const char* env = std::getenv("PT_CUTS");
    if (!env || std::sscanf(env, "%f,%f,%f,%f,%f,%f,%f", &cuts.kmax, &cuts.z0max, &cuts.cotmax,
                            &cuts.rz0, &cuts.rz1, &cuts.dca_b0, &cuts.dca_other) != 7) {
      std::fprintf(stderr, "set PT_CUTS=kmax,z0max,cotmax,rz0,rz1,dca_b0,dca_other\n");
      return 2;
    }
  }
  pt_server* srv = nullptr;
  pt_router* rtr = nullptr;
  if (instances > 1) {
    std::vector<int> devs(instances, 0);
    if (pt_router_create(&geom, &cuts, devs.data(), instances, budget, slots, &rtr) != PT_OK) {
      std::fprintf(stderr, "pt_router_create: %s\n", pt_last_error());
      return 1;
    }
  } else if (pt_server_create(&geom, &cuts, 0, budget, slots, &srv) != PT_OK) {
    std::fprintf(stderr, "pt_server_create: %s\n", pt_last_error());
    return 1;
  }
  auto submit = [&](int64_t n, const float* x, const float* y, const float* z, const uint8_t* l,
                    uint64_t* t) {
    return rtr ? pt_router_submit(rtr, n, x, y, z, l, t) : pt_submit(srv, n, x, y, z, l, t);
  };
  auto poll = [&](uint64_t t, int64_t us, int32_t* h, uint8_t* nh, pt_track* tr, int64_t cap,
                  int64_t* n) {
    return rtr ? pt_router_poll(rtr, t, us, h, nh, tr, cap, n)
               : pt_poll(srv, t, us, h, nh, tr, cap, n);
  };
  if (!gate.empty() &&
      (rtr ? pt_router_set_gate(rtr, gate.data(), gate[5057])
           : pt_server_set_gate(srv, gate.data(), gate[5057])) != PT_OK) {
    std::fprintf(stderr, "set_gate: %s\n", pt_last_error());
    return 1;
  }
  // warm-up: every slot's graph captured, every pool event once
  {
    std::vector<uint64_t> t(pool.size());
    for (size_t i = 0; i < pool.size(); ++i)
      submit((int64_t)pool[i].x.size(), pool[i].x.data(), pool[i].y.data(), pool[i].z.data(),
             pool[i].layer.data(), &t[i]);
    for (uint64_t k : t) {
      int64_t n = 0;
      while (poll(k, -1, nullptr, nullptr, nullptr, 0, &n) == PT_ERR_CAPACITY) {
        std::vector<int32_t> h(6 * n);
        std::vector<uint8_t> nh(n);
        std::vector<pt_track> tr(n);
        if (poll(k, -1, h.data(), nh.data(), tr.data(), n, &n) == PT_OK) break;
      }
    }
    if (rtr) pt_router_reset_stats(rtr);
    else pt_server_reset_stats(srv);
  }
  std::vector<Client> cl(clients);
  std::atomic<int64_t> submitted{0};
  const Clock::time_point t0 = Clock::now() + std::chrono::milliseconds(20);
  const Clock::time_point t_end = t0 + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(seconds));
  auto submitter = [&](int c) {
    std::mt19937_64 rng(seed * 1000003ull + (unsigned)c);
    std::exponential_distribution<double> gap(rate / clients);
    Clock::time_point next = t0;
    size_t k = (size_t)c;
    while (true) {
      next += std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(gap(rng)));
      if (next >= t_end) break;
      std::this_thread::sleep_until(next);
      const Event& e = pool[k % pool.size()];
      k += (size_t)clients;
      uint64_t ticket = 0;
      const Clock::time_point ts = Clock::now();
      if (submit((int64_t)e.x.size(), e.x.data(), e.y.data(), e.z.data(), e.layer.data(),
                 &ticket) != PT_OK) {
        std::lock_guard<std::mutex> lk(cl[c].mu);
        cl[c].errors += 1;
        continue;
      }
      submitted.fetch_add(1);
      {
        std::lock_guard<std::mutex> lk(cl[c].mu);
        cl[c].q.push_back({ticket, ts});
      }
      cl[c].cv.notify_one();
    }
    {
      std::lock_guard<std::mutex> lk(cl[c].mu);
      cl[c].done = true;
    }
    cl[c].cv.notify_one();
  };
  auto collector = [&](int c) {
    std::vector<int32_t> h;
    std::vector<uint8_t> nh;
    std::vector<pt_track> tr;
    while (true) {
      Pending p;
      {
        std::unique_lock<std::mutex> lk(cl[c].mu);
        cl[c].cv.wait(lk, [&] { return !cl[c].q.empty() || cl[c].done; });
        if (cl[c].q.empty()) break;
        p = cl[c].q.front();
        cl[c].q.pop_front();
      }
      int64_t n = 0;
      pt_status st = poll(p.ticket, -1, nullptr, nullptr, nullptr, 0, &n);
      if (st == PT_ERR_CAPACITY) {
        h.resize(6 * n);
        nh.resize(n);
        tr.resize(n);
        st = poll(p.ticket, -1, h.data(), nh.data(), tr.data(), n, &n);
      }
      const Clock::time_point tr_ = Clock::now();
      const double ms = std::chrono::duration<double, std::milli>(tr_ - p.t_submit).count();
      std::lock_guard<std::mutex> lk(cl[c].mu);
      if (st == PT_OK) {
        cl[c].lat_ms.push_back(ms);
        cl[c].in_window += tr_ <= t_end;
      } else {
        cl[c].errors += 1;
      }
    }
  };
  std::vector<std::thread> th;
  for (int c = 0; c < clients; ++c) {
    th.emplace_back(submitter, c);
    th.emplace_back(collector, c);
  }
  for (auto& t : th) t.join();
  const Clock::time_point t_last = Clock::now();
  double p50 = 0, p99 = 0, srv_rate = 0;
  int64_t done = 0, batches = 0, split = 0, requeued = 0;
  if (rtr) {
    pt_router_stats(rtr, &p50, &p99, &srv_rate, &done, nullptr);
  } else {
    pt_server_stats(srv, &p50, &p99, &srv_rate, &done);
    pt_server_counters(srv, &batches, &split, &requeued);
  }
  std::vector<double> all;
  int64_t errors = 0, in_window = 0;
  for (auto& c : cl) {
    all.insert(all.end(), c.lat_ms.begin(), c.lat_ms.end());
    errors += c.errors;
    in_window += c.in_window;
  }
  const double drain_s = std::chrono::duration<double>(t_last - t_end).count();
  const double med = pct(all, 0.5);
  int64_t over3 = 0, over10ms = 0;
  for (double v : all) {
    over3 += v > 3.0 * med;
    over10ms += v > 10.0;
  }
  std::printf(
      "{\"offered_events_per_s\": %.1f, \"seconds\": %.3f, \"clients\": %d, \"slots\": %d, "
      "\"submitted\": %lld, \"completed\": %lld, \"errors\": %lld, "
      "\"sustained_events_per_s\": %.1f, \"throughput_events_per_s\": %.1f, "
      "\"drain_s\": %.4f, \"server_p50_ms\": %.4f, "
      "\"server_p99_ms\": %.4f, \"client_p50_ms\": %.4f, \"client_p99_ms\": %.4f, "
      "\"client_max_ms\": %.4f, \"requests_over_3x_median\": %lld, "
      "\"requests_over_10ms\": %lld, \"batches\": %lld, \"split_batches\": %lld, "
      "\"requeued_events\": %lld, \"instances\": %d}\n",
      rate, seconds, clients, slots, (long long)submitted.load(), (long long)done,
      (long long)errors, (double)in_window / seconds, (double)done / (seconds + drain_s),
      drain_s, p50, p99, pct(all, 0.5),
      pct(all, 0.99), all.empty() ? 0.0 : *std::max_element(all.begin(), all.end()),
      (long long)over3, (long long)over10ms, (long long)batches, (long long)split,
      (long long)requeued, instances);
  if (rtr) pt_router_destroy(rtr);
  else pt_server_destroy(srv);
  return errors ? 1 : 0;
}
