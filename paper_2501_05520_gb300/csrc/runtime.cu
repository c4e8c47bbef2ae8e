// Host runtime of the C ABI declared in pt_ca.h: context lifecycle, workspace layout,
// input staging, stage sequencing on the context's stream, CUDA-graph replay of the
// whole batch, result export and error reporting.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>
#include <initializer_list>
#include <utility>
#include <vector>

#include "brokenline.cuh"
#include "ptca_internal.cuh"

using namespace ptca;

namespace ptca {

// Per-kernel timing of stage calls: a pool of CUDA events, one (start, end) pair per
// traced launch, reduced to per-name totals when read.
struct Tracer {
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  struct Rec {
    const char* name;
    size_t e0, e1;
  };
  std::vector<Rec> recs;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> totals;  // first-seen order
  cudaStream_t last = nullptr;

  size_t take(cudaStream_t s) {
    if (used == ev.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return SIZE_MAX;
      ev.push_back(e);
    }
    cudaEventRecord(ev[used], s);
    last = s;
    return used++;
  }
  void add(const char* name, double ms) {
    for (auto& t : totals)
      if (t.first == name) {
        t.second.first += ms;
        t.second.second += 1;
        return;
      }
    totals.push_back({name, {ms, 1}});
  }
  // events must have completed (the caller synchronised the stream)
  void collect() {
    for (const Rec& r : recs) {
      float ms = 0.0f;
      if (r.e0 != SIZE_MAX && r.e1 != SIZE_MAX &&
          cudaEventElapsedTime(&ms, ev[r.e0], ev[r.e1]) == cudaSuccess)
        add(r.name, ms);
    }
    recs.clear();
    used = 0;
  }
  ~Tracer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

size_t trace_begin(Tracer* t, cudaStream_t s) { return t->take(s); }

bool make_pair_table(int n, const int32_t* in, const int32_t* out, PairTable* t) {
  if (n < 1 || n > kMaxPairs || !in || !out) return false;
  PairTable p;
  std::memset(&p, -1, sizeof(p));
  for (int L = 0; L < kLayers; ++L) p.n_outer[L] = p.n_inner[L] = 0;
  bool adj[kLayers][kLayers] = {};
  for (int i = 0; i < n; ++i) {
    const int a = in[i], c = out[i];
    if (a < 0 || a >= kLayers || c < 0 || c >= kLayers || a == c || adj[a][c]) return false;
    if (p.n_outer[a] >= kMaxOuter || p.n_inner[c] >= kMaxInner) return false;
    adj[a][c] = true;
    p.outer[a][p.n_outer[a]++] = (int8_t)c;
    p.slot[c][a] = p.n_inner[c];
    p.inner[c][p.n_inner[c]++] = (int8_t)a;
  }
  // longest path (in pairs) ending at each layer, by repeated relaxation: a cycle keeps
  // growing it past kLayers, a chain longer than an ntuplet can hold passes kMaxHits - 1
  int depth[kLayers] = {};
  for (int it = 0; it <= kLayers; ++it)
    for (int a = 0; a < kLayers; ++a)
      for (int c = 0; c < kLayers; ++c)
        if (adj[a][c] && depth[c] < depth[a] + 1) depth[c] = depth[a] + 1;
  int8_t mi = 1;
  for (int L = 0; L < kLayers; ++L) {
    if (depth[L] > kMaxHits - 1) return false;
    if (p.n_inner[L] > mi) mi = p.n_inner[L];
  }
  p.max_inner = mi;
  *t = p;
  return true;
}

PairTable default_pair_table() {
  static const int32_t in[13] = {0, 1, 2, 0, 1, 2, 4, 5, 0, 1, 2, 7, 8};
  static const int32_t out[13] = {1, 2, 3, 4, 4, 4, 5, 6, 7, 7, 7, 8, 9};
  PairTable t;
  make_pair_table(13, in, out, &t);
  return t;
}

void trace_end(Tracer* t, const char* name, size_t i0, cudaStream_t s) {
  t->recs.push_back({name, i0, t->take(s)});
  if (t->recs.size() >= 4096) {  // bound the pool: fold completed records into the totals
    cudaStreamSynchronize(s);
    t->collect();
  }
}

}  // namespace ptca

namespace {

thread_local std::string g_err;

pt_status fail(pt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define PT_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(PT_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

#define PT_TRY(call)              \
  do {                            \
    pt_status s_ = (call);        \
    if (s_ != PT_OK) return s_;   \
  } while (0)

constexpr size_t kAlign = 256;

// Carves the workspace; with base == nullptr only computes the size.
size_t layout(const pt_capacity& c, char* base, Buffers* b, GateWeights** gate = nullptr) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + kAlign - 1) / kAlign * kAlign;
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t N = (size_t)c.max_hits, E = (size_t)c.max_events, C = (size_t)c.max_cells;
  const size_t L = (size_t)c.max_links, T = (size_t)c.max_ntuplets;
  const size_t NB = E * kLayers * (size_t)c.phi_bins + 1;
  Buffers t{};
  t.hdr = (BatchHeader*)take(sizeof(BatchHeader));
  t.cnt = (unsigned long long*)take(CNT_N * 8);
  t.in_x = (float*)take(N * 4);
  t.in_y = (float*)take(N * 4);
  t.in_z = (float*)take(N * 4);
  t.in_layer = (uint8_t*)take(N);
  t.hit_off = (int32_t*)take((E + 1) * 4);
  t.in_bin = (uint32_t*)take(N * 4);
  t.in_rank = (uint32_t*)take(N * 4);
  t.hit4 = (float4*)take(N * 16);
  t.perm = (uint32_t*)take(N * 4);
  t.hbin = (uint32_t*)take(N * 4);
  t.bin_cnt = (uint32_t*)take(NB * 4);
  t.bin_start = (uint32_t*)take(NB * 4);
  t.layer_rmax = (uint32_t*)take(E * kLayers * 4);
  t.layer_asin = (float*)take(E * kLayers * 4);
  t.layer_rmin = (uint32_t*)take(E * kLayers * 4);
  t.layer_asin_lo = (float*)take(E * kLayers * 4);
  t.layer_zmin = (uint32_t*)take(E * kLayers * 4);
  t.layer_zmax = (uint32_t*)take(E * kLayers * 4);
  t.seg = (uint2*)take(N * kMaxInner * sizeof(uint2));  // the table's max_inner slots used
  t.cell_in = (uint32_t*)take(C * 4);
  t.cell_out = (uint32_t*)take(C * 4);
  t.has_in = (uint8_t*)take(C);
  t.has_out = (uint8_t*)take(C);
  t.fb_kill = (uint8_t*)take(C);
  t.fb_cnt = (uint32_t*)take((N + 1) * 4);
  t.fb_start = (uint32_t*)take((N + 1) * 4);
  t.fb_rec = (float4*)take(L * 32);
  t.cell_head = (uint32_t*)take(C * 4);
  t.best = (unsigned long long*)take(C * 8);
  t.link_dst = (uint32_t*)take(L * 4);
  t.link_next = (uint32_t*)take(L * 4);
  t.link_walk = (uint2*)take(L * 8);
  t.link_q = (float*)take(L * 4);
  t.nt_hits = (int32_t*)take(T * kMaxHits * 4);
  t.nt_cells = (uint32_t*)take(T * kMaxCellsPerNt * 4);
  t.nt_n = (uint8_t*)take(T);
  t.nt_q = (float*)take(T * 4);
  t.nt_rank = (uint32_t*)take(T * 4);
  t.bucket_cnt = (uint32_t*)take((N + 1) * 4);
  t.bucket_start = (uint32_t*)take((N + 1) * 4);
  t.ord = (uint32_t*)take(T * 4);
  t.alive = (uint32_t*)take(T * 4);
  t.alive_scan = (uint32_t*)take((T + 1) * 4);
  t.used = (uint8_t*)take(N);
  t.sv = (uint32_t*)take(T * 4);
  t.ev_nt_off = (int64_t*)take((E + 1) * 8);
  t.tracks = (pt_track*)take(T * sizeof(pt_track));
  t.vtx_stage = (pt_vertex*)take((T / 2 + 1) * sizeof(pt_vertex));
  t.vtx = (pt_vertex*)take((T / 2 + 1) * sizeof(pt_vertex));
  t.trk_vtx = (int32_t*)take(T * 4);
  t.ev_nv = (uint32_t*)take((E + 1) * 4);
  t.ev_v_scan = (uint32_t*)take((E + 1) * 4);
  t.ev_vtx_off = (int64_t*)take((E + 1) * 8);
  t.gate_x = (uint16_t*)take(L * 16 * 2);
  t.gate_score = (float*)take(L * 4);
  t.gate_keep = (uint8_t*)take(L);
  t.link_src = (uint32_t*)take(L * 4);
  t.exp_hits = (int32_t*)take(T * kMaxHits * 4);
  t.exp_n = (uint8_t*)take(T);
  t.exp_q = (float*)take(T * 4);
  t.exp_ev = (int32_t*)take(T * 4);
  t.scan_part = (uint32_t*)take((kScanBlocks + 1) * 4);
  if (gate) *gate = (GateWeights*)take(sizeof(GateWeights));
  else take(sizeof(GateWeights));
  if (b) *b = t;
  return (off + kAlign - 1) / kAlign * kAlign;
}

pt_status check_capacity(const pt_capacity* c) {
  if (!c) return fail(PT_ERR_INVALID, "capacity is NULL");
  if (c->max_events < 1 || c->max_hits < 1 || c->max_cells < 1 || c->max_links < 1 ||
      c->max_ntuplets < 1)
    return fail(PT_ERR_INVALID, "capacities must be >= 1");
  if (c->max_hits >= (1ll << 29)) return fail(PT_ERR_INVALID, "max_hits must be < 2^29");
  if (c->max_cells >= (1ll << 32) - 1 || c->max_links >= (1ll << 32) - 1)
    return fail(PT_ERR_INVALID, "max_cells and max_links must be < 2^32 - 1");
  if (c->max_ntuplets >= (1ll << kRankBits))
    return fail(PT_ERR_INVALID, "max_ntuplets must be < 2^%d", kRankBits);
  if (c->phi_bins < 16 || c->phi_bins > 4096)
    return fail(PT_ERR_INVALID, "phi_bins must be in [16, 4096]");
  if (c->max_events * kLayers * (int64_t)c->phi_bins >= (1ll << 31) - 1)
    return fail(PT_ERR_INVALID, "max_events * 10 * phi_bins must be < 2^31 - 1");
  if (c->reserved != 0) return fail(PT_ERR_INVALID, "reserved must be 0");
  return PT_OK;
}

}  // namespace

struct pt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  pt_capacity cap{};
  Params P{};
  Buffers B{};
  Launch L{};
  int n_events = 0;
  int64_t n_hits = 0;
  bool loaded = false;
  bool fitted = false;     // the tracks of the loaded batch are fitted
  bool vtx_ready = false;  // pt_find_vertices ran on the loaded batch
  std::vector<int64_t> hit_off;
  // pinned staging
  int32_t* h_off = nullptr;
  BatchHeader* h_hdr = nullptr;
  unsigned long long* h_cnt = nullptr;
  cudaEvent_t staged = nullptr;
  cudaGraphExec_t graph = nullptr;
  // validation staging, allocated on first use
  char* val = nullptr;
  size_t val_bytes = 0;
  // learned gate
  GateWeights* gate = nullptr;  // device, inside the workspace
  bool gate_on = false;
  bool fishbone_on = false;
  // the ntuplet search and the link exports follow a keep mask (gate and/or fishbone)
  bool masked() const { return gate_on || fishbone_on; }
  // whether the stage path's last link stage ran masked: the stage-path ntuplet search
  // follows the links as that stage left them (plain: each link records its target's
  // list head; masked: the keep mask and flags)
  bool links_masked = false;
  // raw input: module table and scratch (allocated on first use)
  pt_module* modules = nullptr;
  int n_modules = 0;
  char* raw_mem = nullptr;
  RawBuffers R{};
  // broken-line refit scratch: two track lists and the pass counters (first use)
  char* bl_mem = nullptr;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

pt_status last_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PT_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return PT_OK;
}

pt_status check_status(pt_ctx* c);

// Reads the device counters (synchronises the stream) and turns status bits into errors.
pt_status sync_counters(pt_ctx* c) {
  PT_CUDA(cudaMemcpyAsync(c->h_cnt, c->B.cnt, CNT_N * 8, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

// Status bits of the host copy of the counters -> error.
pt_status check_status(pt_ctx* c) {
  const unsigned long long st = c->h_cnt[CNT_STATUS];
  if (st & ST_DEBUG)
    return fail(PT_ERR_INTERNAL, "debug build: device bounds check %llu failed",
                c->h_cnt[CNT_DEBUG_SITE]);
  if (st & ST_LAYER) return fail(PT_ERR_INVALID, "input contains a layer code > 9");
  const unsigned long long raw = c->h_cnt[CNT_RAW_STATUS];
  if (raw & RAW_INVALID)
    return fail(PT_ERR_INVALID, "raw input: a module index, pixel or adc outside the module "
                                "table or range, or pixels of a module out of order or repeated");
  if (raw & RAW_RUN_CAPACITY)
    return fail(PT_ERR_CAPACITY, "raw input: more than 1024 digis on one module of an event");
  if (raw & RAW_CLUSTER_CAPACITY)
    return fail(PT_ERR_CAPACITY, "raw input: a cluster of more than 128 pixels");
  if (raw & RAW_HIT_CAPACITY)
    return fail(PT_ERR_CAPACITY, "raw input: %llu hits, more than max_hits = %lld",
                c->h_cnt[CNT_RAW_HITS], (long long)c->cap.max_hits);
  if (st & ST_VTX)
    return fail(PT_ERR_CAPACITY, "an event has more than 16384 tracks for vertex finding");
  if (st & ST_GATE_TIMEOUT)
    return fail(PT_ERR_TIMEOUT, "a bounded wait of the gate's tensor-core kernel expired");
  if (st & ST_CELLS)
    return fail(PT_ERR_CAPACITY,
                "max_cells = %lld is too small: about %llu cell slots needed (cells plus "
                "allocation slack)",
                (long long)c->cap.max_cells, c->h_cnt[CNT_CELLS]);
  if (st & ST_LINKS)
    return fail(PT_ERR_CAPACITY,
                "max_links = %lld is too small: at least %llu link slots needed",
                (long long)c->cap.max_links, c->h_cnt[CNT_LINKS]);
  if (st & ST_NT)
    return fail(PT_ERR_CAPACITY,
                "max_ntuplets = %lld is too small: at least %llu ntuplets needed",
                (long long)c->cap.max_ntuplets, c->h_cnt[CNT_NT]);
  return PT_OK;
}

pt_status stage_inputs(pt_ctx* c, int n_events, const int64_t* off, const float* x,
                       const float* y, const float* z, const uint8_t* layer, int on_device) {
  if (n_events < 1) return fail(PT_ERR_INVALID, "n_events must be >= 1");
  if (n_events > c->cap.max_events)
    return fail(PT_ERR_CAPACITY, "max_events = %lld is too small: %d events given",
                (long long)c->cap.max_events, n_events);
  if (!off) return fail(PT_ERR_INVALID, "hit_offsets is NULL");
  if (off[0] != 0) return fail(PT_ERR_INVALID, "hit_offsets[0] must be 0");
  for (int e = 0; e < n_events; ++e)
    if (off[e + 1] < off[e]) return fail(PT_ERR_INVALID, "hit_offsets must be non-decreasing");
  const int64_t n = off[n_events];
  if (n > c->cap.max_hits)
    return fail(PT_ERR_CAPACITY, "max_hits = %lld is too small: %lld hits given",
                (long long)c->cap.max_hits, (long long)n);
  if (n > 0 && (!x || !y || !z || !layer)) return fail(PT_ERR_INVALID, "hit array is NULL");
  if (!on_device)
    for (int64_t i = 0; i < n; ++i)
      if (layer[i] >= kLayers)
        return fail(PT_ERR_INVALID, "layer code %d > 9 at hit %lld", (int)layer[i], (long long)i);
  // the pinned staging of the previous call must have been consumed
  PT_CUDA(cudaEventSynchronize(c->staged));
  PT_CUDA(cudaMemsetAsync(&c->B.cnt[CNT_RAW_STATUS], 0, 8, c->stream));
  for (int e = 0; e <= n_events; ++e) c->h_off[e] = (int32_t)off[e];
  c->h_hdr->n_events = n_events;
  c->h_hdr->n_hits = (int32_t)n;
  PT_CUDA(cudaMemcpyAsync(c->B.hit_off, c->h_off, (n_events + 1) * 4, cudaMemcpyHostToDevice,
                          c->stream));
  PT_CUDA(cudaMemcpyAsync(c->B.hdr, c->h_hdr, sizeof(BatchHeader), cudaMemcpyHostToDevice,
                          c->stream));
  if (n > 0) {
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PT_CUDA(cudaMemcpyAsync(c->B.in_x, x, n * 4, k, c->stream));
    PT_CUDA(cudaMemcpyAsync(c->B.in_y, y, n * 4, k, c->stream));
    PT_CUDA(cudaMemcpyAsync(c->B.in_z, z, n * 4, k, c->stream));
    PT_CUDA(cudaMemcpyAsync(c->B.in_layer, layer, n, k, c->stream));
  }
  PT_CUDA(cudaEventRecord(c->staged, c->stream));
  c->n_events = n_events;
  c->n_hits = n;
  c->hit_off.assign(off, off + n_events + 1);
  c->loaded = true;
  c->fitted = false;
  c->vtx_ready = false;
  return PT_OK;
}

void enqueue_pipeline(pt_ctx* c, cudaStream_t s) {
  Launch L = c->L;
  L.tr = nullptr;  // a captured graph records no timing events
  launch_clear(c->B, c->P, L, s);
  launch_bin_hits(c->B, c->P, L, s);
  launch_doublets(c->B, c->P, L, s);
  launch_connect(c->B, c->P, L, s, c->gate_on);
  if (c->gate_on) launch_gate(c->B, c->P, L, c->gate, s);
  if (c->fishbone_on) launch_fishbone(c->B, c->P, L, s, c->gate_on);
  launch_ntuplets(c->B, c->P, L, s, c->masked());
  launch_fit(c->B, c->P, L, s);
  launch_export_ntuplets(c->B, L, s);
}

pt_status ensure_graph(pt_ctx* c) {
  if (c->graph) return PT_OK;
  cudaStream_t cs;
  PT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_pipeline(c, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return fail(PT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  }
  return PT_OK;
}

pt_status need_loaded(pt_ctx* c) {
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!c->loaded) return fail(PT_ERR_INVALID, "no hits loaded");
  return PT_OK;
}

pt_status val_staging(pt_ctx* c, size_t bytes) {
  if (bytes <= c->val_bytes) return PT_OK;
  if (c->val) cudaFree(c->val);
  c->val = nullptr;
  c->val_bytes = 0;
  PT_CUDA(cudaMalloc(&c->val, bytes));
  c->val_bytes = bytes;
  return PT_OK;
}

pt_status copy_out(pt_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
  if (!bytes || !dst) return PT_OK;
  PT_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream));
  return PT_OK;
}

}  // namespace

namespace ptca {
void set_last_error(const char* msg) { g_err = msg; }

cudaStream_t ctx_stream(pt_ctx* c) { return c->stream; }

pt_status ctx_counters_async(pt_ctx* c, cudaEvent_t done) {
  DeviceGuard guard(c->device);
  PT_CUDA(cudaMemcpyAsync(c->h_cnt, c->B.cnt, CNT_N * 8, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaEventRecord(done, c->stream));
  return PT_OK;
}

pt_status ctx_read_counters(pt_ctx* c, int64_t* n_ntuplets) {
  PT_TRY(check_status(c));
  *n_ntuplets = (int64_t)c->h_cnt[CNT_SV];
  return PT_OK;
}

pt_status ctx_results_async(pt_ctx* c, int64_t S, int32_t* hits, uint8_t* nhits,
                            pt_track* tracks, int64_t* event_offsets, cudaEvent_t done) {
  DeviceGuard guard(c->device);
  PT_TRY(copy_out(c, hits, c->B.exp_hits, (size_t)S * kMaxHits * 4, 0));
  PT_TRY(copy_out(c, nhits, c->B.exp_n, (size_t)S, 0));
  PT_TRY(copy_out(c, tracks, c->B.tracks, (size_t)S * sizeof(pt_track), 0));
  PT_TRY(copy_out(c, event_offsets, c->B.ev_nt_off, (size_t)(c->n_events + 1) * 8, 0));
  PT_CUDA(cudaEventRecord(done, c->stream));
  return PT_OK;
}
}  // namespace ptca

extern "C" {

const char* pt_last_error(void) { return g_err.c_str(); }

pt_status pt_workspace_size(const pt_capacity* cap, size_t* bytes) {
  g_err.clear();
  PT_TRY(check_capacity(cap));
  if (!bytes) return fail(PT_ERR_INVALID, "bytes is NULL");
  *bytes = layout(*cap, nullptr, nullptr);
  return PT_OK;
}

pt_status pt_create(const pt_geometry* geom, const pt_cuts* cuts, const pt_capacity* cap,
                    int device, void* workspace, size_t workspace_bytes, void* stream,
                    pt_ctx** out) {
  g_err.clear();
  if (!out) return fail(PT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!geom || !cuts) return fail(PT_ERR_INVALID, "geometry or cuts is NULL");
  PT_TRY(check_capacity(cap));
  int ndev = 0;
  PT_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(PT_ERR_INVALID, "device %d not present", device);
  DeviceGuard guard(device);
  const size_t need = layout(*cap, nullptr, nullptr);
  if (workspace) {
    if (workspace_bytes < need)
      return fail(PT_ERR_CAPACITY, "workspace of %zu bytes is too small: %zu needed",
                  workspace_bytes, need);
    if ((uintptr_t)workspace % kAlign)
      return fail(PT_ERR_INVALID, "workspace must be %zu-byte aligned", kAlign);
  }
  pt_ctx* c = new pt_ctx();
  c->device = device;
  c->cap = *cap;
  c->P.cuts = *cuts;
  c->P.pairs = default_pair_table();
  c->P.wait_cycles = 1ll << 31;
  c->P.bfield = geom->bfield_T;
  c->P.phi_bins = cap->phi_bins;
  c->P.max_events = cap->max_events;
  c->P.max_hits = cap->max_hits;
  c->P.max_cells = cap->max_cells;
  c->P.max_links = cap->max_links;
  c->P.max_ntuplets = cap->max_ntuplets;
  auto bail = [&](pt_status st) {
    pt_destroy(c);
    return st;
  };
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "cannot query the multiprocessor count"));
  c->L.sms = sms;
  c->L.grid = sms * 4;
  c->L.sgrid = sms * 5;
  if (workspace) {
    c->ws = (char*)workspace;
    c->ws_bytes = workspace_bytes;
  } else {
    if (cudaMalloc(&c->ws, need) != cudaSuccess) {
      cudaGetLastError();
      c->ws = nullptr;
      return bail(fail(PT_ERR_NOMEM, "cudaMalloc of %zu workspace bytes failed", need));
    }
    c->ws_bytes = need;
    c->own_ws = true;
  }
  layout(*cap, c->ws, &c->B, &c->gate);
  if (cudaMallocHost(&c->h_off, (cap->max_events + 1) * 4) != cudaSuccess ||
      cudaMallocHost(&c->h_hdr, sizeof(BatchHeader)) != cudaSuccess ||
      cudaMallocHost(&c->h_cnt, CNT_N * 8) != cudaSuccess)
    return bail(fail(PT_ERR_NOMEM, "pinned host allocation failed"));
  if (cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "cudaEventCreate failed"));
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&c->stream) != cudaSuccess)
      return bail(fail(PT_ERR_CUDA, "cudaStreamCreate failed"));
    c->own_stream = true;
  }
  if (cudaMemsetAsync(c->B.cnt, 0, CNT_N * 8, c->stream) != cudaSuccess)
    return bail(fail(PT_ERR_CUDA, "cudaMemsetAsync failed"));
  *out = c;
  return PT_OK;
}

pt_status pt_destroy(pt_ctx* c) {
  if (!c) return PT_OK;
  DeviceGuard guard(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->val) cudaFree(c->val);
  if (c->modules) cudaFree(c->modules);
  if (c->raw_mem) cudaFree(c->raw_mem);
  if (c->bl_mem) cudaFree(c->bl_mem);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->h_off) cudaFreeHost(c->h_off);
  if (c->h_hdr) cudaFreeHost(c->h_hdr);
  if (c->h_cnt) cudaFreeHost(c->h_cnt);
  if (c->staged) cudaEventDestroy(c->staged);
  delete c->L.tr;
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return PT_OK;
}

pt_status pt_set_tracing(pt_ctx* c, int on) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (on && !c->L.tr) c->L.tr = new Tracer();
  if (!on) {
    delete c->L.tr;
    c->L.tr = nullptr;
  }
  return PT_OK;
}

pt_status pt_get_trace(pt_ctx* c, pt_kernel_time* out, int cap, int* n) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!c->L.tr) return fail(PT_ERR_INVALID, "tracing is off (pt_set_tracing)");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  Tracer* t = c->L.tr;
  t->collect();
  const int m = (int)t->totals.size();
  if (n) *n = m;
  if (cap < m) return fail(PT_ERR_CAPACITY, "output capacity %d < %d kernels", cap, m);
  for (int i = 0; i < m; ++i) {
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, t->totals[i].first.c_str(), sizeof(out[i].name) - 1);
    out[i].total_ms = t->totals[i].second.first;
    out[i].launches = t->totals[i].second.second;
  }
  t->totals.clear();
  return PT_OK;
}

pt_status pt_set_stream(pt_ctx* c, void* stream) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->own_stream = false;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    PT_CUDA(cudaStreamCreate(&c->stream));
    c->own_stream = true;
  }
  return PT_OK;
}

pt_status pt_load_batch(pt_ctx* c, int n_events, const int64_t* hit_offsets, const float* x,
                        const float* y, const float* z, const uint8_t* layer, int on_device) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  DeviceGuard guard(c->device);
  PT_TRY(stage_inputs(c, n_events, hit_offsets, x, y, z, layer, on_device));
  launch_clear(c->B, c->P, c->L, c->stream);
  launch_bin_hits(c->B, c->P, c->L, c->stream);
  return last_launch();
}

pt_status pt_load_hits(pt_ctx* c, int64_t n, const float* x, const float* y, const float* z,
                       const uint8_t* layer, int on_device) {
  if (n < 0) return fail(PT_ERR_INVALID, "n must be >= 0");
  const int64_t off[2] = {0, n};
  return pt_load_batch(c, 1, off, x, y, z, layer, on_device);
}

#define STAGE_BODY(launch, counter, outp)                \
  g_err.clear();                                         \
  PT_TRY(need_loaded(c));                                \
  DeviceGuard guard(c->device);                          \
  launch;                                                \
  PT_TRY(last_launch());                                 \
  if (outp) {                                            \
    PT_TRY(sync_counters(c));                            \
    *(outp) = (int64_t)c->h_cnt[counter];                \
  }                                                      \
  return PT_OK;

// A stage call may run again on the same loaded batch: the counters it accumulates (and
// the ntuplet stage's per-hit tallies) start from zero each time.  The whole-batch graph
// has these cleared once by launch_clear.
int64_t loaded_hits(const pt_ctx* c) { return c->n_hits >= 0 ? c->n_hits : c->cap.max_hits; }

void reset_counters(pt_ctx* c, std::initializer_list<int> which) {
  for (int k : which) cudaMemsetAsync(&c->B.cnt[k], 0, sizeof(unsigned long long), c->stream);
}

pt_status pt_build_doublets(pt_ctx* c, int64_t* n_cells) {
  STAGE_BODY((reset_counters(c, {CNT_CELLS, CNT_CELLS_USED}),
              launch_doublets(c->B, c->P, c->L, c->stream)),
             CNT_CELLS_USED, n_cells)
}

pt_status pt_connect_cells(pt_ctx* c, int64_t* n_links) {
  if (c) c->links_masked = c->masked();
  if (c && c->masked()) {
    STAGE_BODY((reset_counters(c, {CNT_LINKS, CNT_LINKS_USED, CNT_GATE_KEPT}),
                launch_connect(c->B, c->P, c->L, c->stream, c->gate_on),
                c->gate_on ? launch_gate(c->B, c->P, c->L, c->gate, c->stream) : (void)0,
                c->fishbone_on ? launch_fishbone(c->B, c->P, c->L, c->stream, c->gate_on)
                               : (void)0),
               CNT_GATE_KEPT, n_links)
  }
  STAGE_BODY((reset_counters(c, {CNT_LINKS, CNT_LINKS_USED, CNT_GATE_KEPT}),
              launch_connect(c->B, c->P, c->L, c->stream)),
             CNT_LINKS_USED, n_links)
}

pt_status pt_find_ntuplets(pt_ctx* c, int64_t* n_ntuplets) {
  STAGE_BODY((reset_counters(c, {CNT_NT, CNT_SCAN_NT, CNT_SV}),
              cudaMemsetAsync(c->B.bucket_cnt, 0, (size_t)(loaded_hits(c) + 1) * 4, c->stream),
              cudaMemsetAsync(c->B.used, 0, (size_t)loaded_hits(c), c->stream),
              launch_ntuplets(c->B, c->P, c->L, c->stream, c->links_masked)),
             CNT_SV, n_ntuplets)
}

pt_status pt_fit_tracks(pt_ctx* c, int64_t* n_tracks) {
  STAGE_BODY((launch_fit(c->B, c->P, c->L, c->stream), c->fitted = true), CNT_SV, n_tracks)
}

pt_status pt_refit_broken_line(pt_ctx* c, float x0_barrel, float x0_disk, int64_t* n_tracks) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  if (!(x0_barrel > 0.0f && x0_barrel <= 1.0f) || !(x0_disk > 0.0f && x0_disk <= 1.0f))
    return fail(PT_ERR_INVALID, "material must be in (0, 1] radiation lengths");
  if (!c->fitted) return fail(PT_ERR_INVALID, "pt_fit_tracks has not run on this batch");
  DeviceGuard guard(c->device);
  const size_t list_bytes = (size_t)c->cap.max_ntuplets * 2 * sizeof(uint32_t);
  if (!c->bl_mem)
    PT_CUDA(cudaMalloc(&c->bl_mem, list_bytes + kRefitCounters * sizeof(unsigned long long)));
  PT_CUDA(launch_refit_broken_line(c->B, c->P, x0_barrel, x0_disk, (uint32_t*)c->bl_mem,
                                   (unsigned long long*)(c->bl_mem + list_bytes), c->L,
                                   c->stream));
  PT_TRY(last_launch());
  c->vtx_ready = false;
  if (n_tracks) {
    PT_TRY(sync_counters(c));
    *n_tracks = (int64_t)c->h_cnt[CNT_SV];
  }
  return PT_OK;
}

pt_status pt_get_ntuplets(pt_ctx* c, int32_t* hits, uint8_t* nhits, int64_t* event_offsets,
                          int64_t cap, int64_t* n, int on_device) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  launch_export_ntuplets(c->B, c->L, c->stream);
  PT_TRY(last_launch());
  PT_TRY(sync_counters(c));
  const int64_t S = (int64_t)c->h_cnt[CNT_SV];
  if (n) *n = S;
  if (cap < S)
    return fail(PT_ERR_CAPACITY, "output capacity %lld is too small: %lld ntuplets",
                (long long)cap, (long long)S);
  PT_TRY(copy_out(c, hits, c->B.exp_hits, (size_t)S * kMaxHits * 4, on_device));
  PT_TRY(copy_out(c, nhits, c->B.exp_n, (size_t)S, on_device));
  PT_TRY(copy_out(c, event_offsets, c->B.ev_nt_off, (size_t)(c->n_events + 1) * 8, on_device));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return PT_OK;
}

pt_status pt_get_tracks(pt_ctx* c, pt_track* tracks, int64_t cap, int64_t* n, int on_device) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t S = (int64_t)c->h_cnt[CNT_SV];
  if (n) *n = S;
  if (cap < S)
    return fail(PT_ERR_CAPACITY, "output capacity %lld is too small: %lld tracks",
                (long long)cap, (long long)S);
  PT_TRY(copy_out(c, tracks, c->B.tracks, (size_t)S * sizeof(pt_track), on_device));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return PT_OK;
}

pt_status pt_set_modules(pt_ctx* c, const pt_module* m, int n) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!m || n < 1 || n >= (1 << 24)) return fail(PT_ERR_INVALID, "need 1 <= n < 2^24 modules");
  for (int i = 0; i < n; ++i) {
    const pt_module& d = m[i];
    if (d.layer < 0 || d.layer >= kLayers || (d.kind != 0 && d.kind != 1) || d.ncol < 1 ||
        d.ncol > 4096 || d.nrow < 1 || d.nrow > 4096 || !std::isfinite(d.rz) ||
        !std::isfinite(d.phi0) || !std::isfinite(d.dphi_col) || !std::isfinite(d.v0) ||
        !std::isfinite(d.dv_row))
      return fail(PT_ERR_INVALID, "module %d is not valid", i);
  }
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->modules) cudaFree(c->modules);
  c->modules = nullptr;
  c->n_modules = 0;
  PT_CUDA(cudaMalloc(&c->modules, (size_t)n * sizeof(pt_module)));
  PT_CUDA(cudaMemcpy(c->modules, m, (size_t)n * sizeof(pt_module), cudaMemcpyHostToDevice));
  c->n_modules = n;
  return PT_OK;
}

pt_status pt_load_raw(pt_ctx* c, int n_events, const int64_t* off, const uint64_t* digis,
                      int on_device, int64_t* n_hits) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!c->modules) return fail(PT_ERR_INVALID, "no module table (pt_set_modules)");
  if (n_events < 1 || n_events > c->cap.max_events)
    return fail(PT_ERR_INVALID, "n_events must be in [1, max_events]");
  if (!off) return fail(PT_ERR_INVALID, "digi_offsets is NULL");
  if (off[0] != 0) return fail(PT_ERR_INVALID, "digi_offsets[0] must be 0");
  for (int e = 0; e < n_events; ++e)
    if (off[e + 1] < off[e]) return fail(PT_ERR_INVALID, "digi_offsets must be non-decreasing");
  const int64_t n = off[n_events];
  const int64_t max_digis = 8 * c->cap.max_hits;
  if (n > max_digis)
    return fail(PT_ERR_CAPACITY, "%lld digis, more than 8 x max_hits = %lld", (long long)n,
                (long long)max_digis);
  if (n > 0 && !digis) return fail(PT_ERR_INVALID, "digis is NULL");
  DeviceGuard guard(c->device);
  if (!c->raw_mem) {  // scratch for max_digis digis, carved like the workspace
    const size_t D = (size_t)max_digis, E = (size_t)c->cap.max_events;
    const size_t parts[] = {(E + 1) * 8, D * 8, (D + 1) * 4, (D + 1) * 4, (D + 1) * 4,
                            (D + 1) * 4, (D + 1) * 4, D * 16};
    size_t bytes = 0;
    for (size_t p : parts) bytes += (p + kAlign - 1) / kAlign * kAlign;
    PT_CUDA(cudaMalloc(&c->raw_mem, bytes));
    char* q = c->raw_mem;
    auto take = [&](size_t b) {
      char* r = q;
      q += (b + kAlign - 1) / kAlign * kAlign;
      return r;
    };
    c->R.digi_off = (int64_t*)take(parts[0]);
    c->R.words = (uint64_t*)take(parts[1]);
    c->R.flag = (uint32_t*)take(parts[2]);
    c->R.run_scan = (uint32_t*)take(parts[3]);
    c->R.run_first = (uint32_t*)take(parts[4]);
    c->R.run_nh = (uint32_t*)take(parts[5]);
    c->R.run_hoff = (uint32_t*)take(parts[6]);
    c->R.stage = (float4*)take(parts[7]);
    c->R.big_runs = c->R.flag;
  }
  c->R.n_events = n_events;
  c->R.scan_part = c->B.scan_part;
  c->R.cnt = c->B.cnt;
  PT_CUDA(cudaStreamSynchronize(c->stream));  // the previous batch no longer needs its inputs
  PT_CUDA(cudaMemcpyAsync(c->R.digi_off, off, (size_t)(n_events + 1) * 8, cudaMemcpyHostToDevice,
                          c->stream));
  if (n > 0)
    PT_CUDA(cudaMemcpyAsync(c->R.words, digis, (size_t)n * 8,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            c->stream));
  PT_CUDA(cudaMemsetAsync(&c->B.cnt[CNT_RAW_STATUS], 0, 8, c->stream));
  PT_CUDA(launch_raw(c->R, c->B, c->modules, c->n_modules, c->cap.max_hits, c->L, c->stream));
  launch_clear(c->B, c->P, c->L, c->stream);
  launch_bin_hits(c->B, c->P, c->L, c->stream);
  PT_TRY(last_launch());
  PT_CUDA(cudaStreamSynchronize(c->stream));  // the host offsets and digis may be reused
  c->n_events = n_events;
  c->n_hits = -1;
  c->hit_off.clear();
  c->loaded = true;
  c->fitted = false;
  c->vtx_ready = false;
  if (n_hits) {
    PT_TRY(sync_counters(c));
    *n_hits = (int64_t)c->h_cnt[CNT_RAW_HITS];
  }
  return PT_OK;
}

pt_status pt_get_hits(pt_ctx* c, float* x, float* y, float* z, uint8_t* layer,
                      int64_t* event_offsets, int64_t cap, int64_t* n) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  BatchHeader hdr{};
  PT_CUDA(cudaMemcpyAsync(&hdr, c->B.hdr, sizeof(hdr), cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t N = hdr.n_hits;
  if (n) *n = N;
  if (cap < N)
    return fail(PT_ERR_CAPACITY, "output capacity %lld is too small: %lld hits", (long long)cap,
                (long long)N);
  PT_TRY(copy_out(c, x, c->B.in_x, (size_t)N * 4, 0));
  PT_TRY(copy_out(c, y, c->B.in_y, (size_t)N * 4, 0));
  PT_TRY(copy_out(c, z, c->B.in_z, (size_t)N * 4, 0));
  PT_TRY(copy_out(c, layer, c->B.in_layer, (size_t)N, 0));
  std::vector<int32_t> off32((size_t)c->n_events + 1);
  PT_CUDA(cudaMemcpyAsync(off32.data(), c->B.hit_off, off32.size() * 4, cudaMemcpyDeviceToHost,
                          c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (event_offsets)
    for (size_t e = 0; e < off32.size(); ++e) event_offsets[e] = off32[e];
  return PT_OK;
}

pt_status pt_find_vertices(pt_ctx* c, int min_hits, float dz, int64_t* n_vertices) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  if (min_hits < 3 || min_hits > kMaxHits) return fail(PT_ERR_INVALID, "min_hits must be in [3, 6]");
  if (!(dz > 0.0f) || !std::isfinite(dz)) return fail(PT_ERR_INVALID, "dz must be finite and > 0");
  DeviceGuard guard(c->device);
  if (!c->fitted) return fail(PT_ERR_INVALID, "pt_fit_tracks has not run on this batch");
  PT_CUDA(launch_vertices(c->B, c->n_events, min_hits, dz, (uint64_t)c->cap.max_ntuplets, c->L,
                          c->stream));
  c->vtx_ready = true;
  if (n_vertices) {
    PT_TRY(sync_counters(c));
    *n_vertices = (int64_t)c->h_cnt[CNT_VTX];
  }
  return PT_OK;
}

pt_status pt_get_vertices(pt_ctx* c, pt_vertex* vertices, int64_t* event_offsets,
                          int32_t* track_vertex, int64_t cap, int64_t* n, int on_device) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  if (!c->vtx_ready) return fail(PT_ERR_INVALID, "pt_find_vertices has not run on this batch");
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t V = (int64_t)c->h_cnt[CNT_VTX];
  const int64_t S = (int64_t)c->h_cnt[CNT_SV];
  if (n) *n = V;
  if (cap < V)
    return fail(PT_ERR_CAPACITY, "output capacity %lld is too small: %lld vertices",
                (long long)cap, (long long)V);
  PT_TRY(copy_out(c, vertices, c->B.vtx, (size_t)V * sizeof(pt_vertex), on_device));
  PT_TRY(copy_out(c, event_offsets, c->B.ev_vtx_off, (size_t)(c->n_events + 1) * 8, on_device));
  PT_TRY(copy_out(c, track_vertex, c->B.trk_vtx, (size_t)S * 4, on_device));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return PT_OK;
}

pt_status pt_get_cells(pt_ctx* c, int32_t* inner, int32_t* outer, int32_t* event, int64_t cap,
                       int64_t* n) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t C = (int64_t)c->h_cnt[CNT_CELLS_USED];
  int64_t slots = (int64_t)c->h_cnt[CNT_CELLS];
  if (slots > c->cap.max_cells) slots = c->cap.max_cells;
  if (n) *n = C;
  if (cap < C) return fail(PT_ERR_CAPACITY, "output capacity %lld < %lld cells", (long long)cap,
                           (long long)C);
  if (C == 0) return PT_OK;
  PT_TRY(val_staging(c, (size_t)slots * 12));
  launch_export_cells(c->B, c->P, c->L, (int32_t*)c->val, c->stream);
  PT_TRY(last_launch());
  std::vector<int32_t> tmp((size_t)slots * 3);
  PT_CUDA(cudaMemcpyAsync(tmp.data(), c->val, (size_t)slots * 12, cudaMemcpyDeviceToHost,
                          c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  int64_t k = 0;
  for (int64_t i = 0; i < slots && k < C; ++i) {
    if (tmp[i * 3 + 2] < 0) continue;  // allocation hole
    if (inner) inner[k] = tmp[i * 3];
    if (outer) outer[k] = tmp[i * 3 + 1];
    if (event) event[k] = tmp[i * 3 + 2];
    ++k;
  }
  return PT_OK;
}

pt_status pt_get_links(pt_ctx* c, int32_t* h0, int32_t* h1, int32_t* h2, float* q,
                       int32_t* event, int64_t cap, int64_t* n) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t Lk = c->masked() ? (int64_t)c->h_cnt[CNT_GATE_KEPT] : (int64_t)c->h_cnt[CNT_LINKS_USED];
  int64_t slots = (int64_t)c->h_cnt[CNT_LINKS];
  if (slots > c->cap.max_links) slots = c->cap.max_links;
  if (n) *n = Lk;
  if (cap < Lk) return fail(PT_ERR_CAPACITY, "output capacity %lld < %lld links", (long long)cap,
                            (long long)Lk);
  if (Lk == 0) return PT_OK;
  PT_TRY(val_staging(c, (size_t)slots * 20));
  int32_t* o4 = (int32_t*)c->val;
  float* oq = (float*)(c->val + (size_t)slots * 16);
  PT_CUDA(cudaMemsetAsync(o4, 0xff, (size_t)slots * 16, c->stream));
  launch_export_links(c->B, c->P, c->L, o4, oq, c->stream, c->masked());
  PT_TRY(last_launch());
  std::vector<int32_t> tmp((size_t)slots * 4);
  std::vector<float> tq((size_t)slots);
  PT_CUDA(cudaMemcpyAsync(tmp.data(), o4, (size_t)slots * 16, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaMemcpyAsync(tq.data(), oq, (size_t)slots * 4, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  int64_t k = 0;
  for (int64_t i = 0; i < slots && k < Lk; ++i) {
    if (tmp[i * 4 + 3] < 0) continue;  // allocation hole
    if (h0) h0[k] = tmp[i * 4];
    if (h1) h1[k] = tmp[i * 4 + 1];
    if (h2) h2[k] = tmp[i * 4 + 2];
    if (event) event[k] = tmp[i * 4 + 3];
    if (q) q[k] = tq[i];
    ++k;
  }
  return PT_OK;
}

pt_status pt_get_candidates(pt_ctx* c, int32_t* hits, uint8_t* nhits, float* q, int32_t* event,
                            int64_t cap, int64_t* n) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t T = (int64_t)c->h_cnt[CNT_SCAN_NT];
  if (n) *n = T;
  if (cap < T) return fail(PT_ERR_CAPACITY, "output capacity %lld < %lld candidates",
                           (long long)cap, (long long)T);
  launch_export_candidates(c->B, c->L, c->stream);
  PT_TRY(last_launch());
  PT_TRY(copy_out(c, hits, c->B.exp_hits, (size_t)T * kMaxHits * 4, 0));
  PT_TRY(copy_out(c, nhits, c->B.exp_n, (size_t)T, 0));
  PT_TRY(copy_out(c, q, c->B.exp_q, (size_t)T * 4, 0));
  PT_TRY(copy_out(c, event, c->B.exp_ev, (size_t)T * 4, 0));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return PT_OK;
}

pt_status pt_set_gate(pt_ctx* c, const float* w, float tau) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (!w) {
    c->gate_on = false;
    return PT_OK;
  }
  for (int i = 0; i < kGateParams; ++i)
    if (!std::isfinite(w[i])) return fail(PT_ERR_INVALID, "gate parameter %d is not finite", i);
  if (!std::isfinite(tau)) return fail(PT_ERR_INVALID, "tau is not finite");
  GateWeights h{};
  const float* W1 = w;
  const float* b1 = W1 + kGateHidden * kGateFeat;
  const float* W2 = b1 + kGateHidden;
  const float* b2 = W2 + kGateHidden * kGateHidden;
  const float* w3 = b2 + kGateHidden;
  const float b3 = w3[kGateHidden];
  // bf16 (round to nearest even) in the core-matrix operand layout: element (row, k) of an
  // R x K operand at ((row/8) * (K/8) + k/8) * 64 + (row%8) * 8 + k%8 (16-bit units)
  auto bf16 = [](float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
  };
  auto cm = [](int row, int k, int K) {
    return (size_t)((row >> 3) * (K / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
  };
  for (int n = 0; n < kGateHidden; ++n) {
    for (int k = 0; k < kGateK1; ++k)
      h.w1[cm(n, k, kGateK1)] = k < kGateFeat ? bf16(W1[n * kGateFeat + k]) : (uint16_t)0;
    for (int k = 0; k < kGateHidden; ++k) h.w2[cm(n, k, kGateHidden)] = bf16(W2[n * kGateHidden + k]);
    h.b1[n] = b1[n];
    h.b2[n] = b2[n];
    h.w3[n] = w3[n];
  }
  h.b3 = b3;
  h.tau = tau;
  PT_CUDA(gate_prepare());
  PT_CUDA(cudaMemcpy(c->gate, &h, sizeof(h), cudaMemcpyHostToDevice));
  c->gate_on = true;
  return PT_OK;
}

int pt_debug_build(void) {
#ifdef PT_DEBUG
  return 1;
#else
  return 0;
#endif
}

pt_status pt_debug_inject(pt_ctx* c, int site) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!pt_debug_build()) return fail(PT_ERR_INVALID, "not the debug build");
  if (site < 1 || site > DBG_FB_RECORD) return fail(PT_ERR_INVALID, "site out of range");
  DeviceGuard guard(c->device);
  PT_CUDA(launch_debug_inject(c->B, (unsigned)site, c->stream));
  return PT_OK;
}

pt_status pt_set_fishbone(pt_ctx* c, int on) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (on != 0 && on != 1) return fail(PT_ERR_INVALID, "on must be 0 or 1");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->fishbone_on = on == 1;
  return PT_OK;
}

pt_status pt_get_link_features(pt_ctx* c, float* feat, int32_t* h0, int32_t* h1, int32_t* h2,
                               int32_t* event, float* score, int64_t cap, int64_t* n) {
  g_err.clear();
  PT_TRY(need_loaded(c));
  DeviceGuard guard(c->device);
  PT_TRY(sync_counters(c));
  const int64_t Lk = c->masked() ? (int64_t)c->h_cnt[CNT_GATE_KEPT] : (int64_t)c->h_cnt[CNT_LINKS_USED];
  int64_t slots = (int64_t)c->h_cnt[CNT_LINKS];
  if (slots > c->cap.max_links) slots = c->cap.max_links;
  if (n) *n = Lk;
  if (cap < Lk) return fail(PT_ERR_CAPACITY, "output capacity %lld < %lld links", (long long)cap,
                            (long long)Lk);
  if (Lk == 0) return PT_OK;
  PT_TRY(val_staging(c, (size_t)slots * (16 + 4 + 48)));
  int32_t* o4 = (int32_t*)c->val;
  float* oq = (float*)(c->val + (size_t)slots * 16);
  float* of = (float*)(c->val + (size_t)slots * 20);
  PT_CUDA(cudaMemsetAsync(o4, 0xff, (size_t)slots * 16, c->stream));
  launch_export_links(c->B, c->P, c->L, o4, oq, c->stream, c->masked());
  launch_export_link_features(c->B, c->P, c->L, c->masked(), of, c->stream);
  PT_TRY(last_launch());
  std::vector<int32_t> t4((size_t)slots * 4);
  std::vector<float> tf((size_t)slots * 12), ts((size_t)slots);
  PT_CUDA(cudaMemcpyAsync(t4.data(), o4, (size_t)slots * 16, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaMemcpyAsync(tf.data(), of, (size_t)slots * 48, cudaMemcpyDeviceToHost, c->stream));
  if (c->gate_on)
    PT_CUDA(cudaMemcpyAsync(ts.data(), c->B.gate_score, (size_t)slots * 4, cudaMemcpyDeviceToHost,
                            c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  int64_t k = 0;
  for (int64_t i = 0; i < slots && k < Lk; ++i) {
    if (t4[i * 4 + 3] < 0) continue;  // hole or removed link
    if (h0) h0[k] = t4[i * 4];
    if (h1) h1[k] = t4[i * 4 + 1];
    if (h2) h2[k] = t4[i * 4 + 2];
    if (event) event[k] = t4[i * 4 + 3];
    if (feat) std::memcpy(feat + k * 12, &tf[i * 12], 48);
    if (score) score[k] = c->gate_on ? ts[i] : std::nanf("");
    ++k;
  }
  return PT_OK;
}

pt_status pt_gate_score(pt_ctx* c, const float* feat, int64_t n, float* out) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!c->gate_on) return fail(PT_ERR_INVALID, "no gate set (pt_set_gate)");
  if (n < 0 || n > c->cap.max_links)
    return fail(PT_ERR_CAPACITY, "n must be in [0, max_links = %lld]", (long long)c->cap.max_links);
  if (n == 0) return PT_OK;
  if (!feat || !out) return fail(PT_ERR_INVALID, "feat and out must not be NULL");
  DeviceGuard guard(c->device);
  // a status word of its own, so that neither the loaded batch's status nor an earlier
  // scoring call's leaks into the answer
  PT_CUDA(cudaMemsetAsync(&c->B.cnt[CNT_SCORE_STATUS], 0, 8, c->stream));
  launch_gate_score(c->gate, feat, n, out, c->B.gate_x, &c->B.cnt[CNT_SCORE_STATUS], c->L.sms,
                    c->P.wait_cycles, c->stream);
  PT_TRY(last_launch());
  PT_CUDA(cudaMemcpyAsync(c->h_cnt, c->B.cnt, CNT_N * 8, cudaMemcpyDeviceToHost, c->stream));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->h_cnt[CNT_SCORE_STATUS] & ST_GATE_TIMEOUT)
    return fail(PT_ERR_TIMEOUT, "a bounded wait of the gate's tensor-core kernel expired");
  return PT_OK;
}

pt_status pt_gate_loss_grad(const float* w, const float* x, const float* y, int64_t n,
                            float* grad, float* loss, void* stream) {
  g_err.clear();
  if (!w || !grad || !loss || (n > 0 && (!x || !y)) || n < 0)
    return fail(PT_ERR_INVALID, "bad argument");
  int dev = 0, sms = 0;
  PT_CUDA(cudaGetDevice(&dev));
  PT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PT_CUDA(launch_gate_grad(w, x, y, n, grad, loss, sms, (cudaStream_t)stream));
  return PT_OK;
}

pt_status pt_gate_adam(float* w, float* m, float* v, const float* grad, int64_t n, float lr,
                       float beta1, float beta2, float eps, int step, void* stream) {
  g_err.clear();
  if (!w || !m || !v || !grad || n < 0 || step < 1) return fail(PT_ERR_INVALID, "bad argument");
  PT_CUDA(launch_gate_adam(w, m, v, grad, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
  return PT_OK;
}

pt_status pt_set_launch(pt_ctx* c, int blocks_per_sm, int search_blocks_per_sm) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (blocks_per_sm < 1 || blocks_per_sm > 32 || search_blocks_per_sm < 1 ||
      search_blocks_per_sm > 32)
    return fail(PT_ERR_INVALID, "blocks per multiprocessor must be in [1, 32]");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->L.grid = c->L.sms * blocks_per_sm;
  c->L.sgrid = c->L.sms * search_blocks_per_sm;
  return PT_OK;
}

pt_status pt_set_wait_limit(pt_ctx* c, int64_t cycles) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (cycles < 1) return fail(PT_ERR_INVALID, "the wait limit must be >= 1 cycle");
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->P.wait_cycles = (long long)cycles;
  return PT_OK;
}

pt_status pt_set_layer_pairs(pt_ctx* c, int n_pairs, const int32_t* inner, const int32_t* outer) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  PairTable t;
  if (n_pairs == 0) {
    t = default_pair_table();
  } else if (!make_pair_table(n_pairs, inner, outer, &t)) {
    return fail(PT_ERR_INVALID,
                "invalid layer-pair table: need 1..%d distinct pairs of layer codes 0..9 with "
                "inner != outer, at most %d outer and %d inner layers per layer, no cycle and "
                "no chain of more than %d pairs",
                kMaxPairs, kMaxOuter, kMaxInner, kMaxHits - 1);
  }
  DeviceGuard guard(c->device);
  PT_CUDA(cudaStreamSynchronize(c->stream));
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->P.pairs = t;
  return PT_OK;
}

pt_status pt_autotune(const pt_geometry* geom, const pt_cuts* cuts, const pt_capacity* cap,
                      int device, int n_events, const int64_t* hit_offsets, const float* x,
                      const float* y, const float* z, const uint8_t* layer,
                      const int32_t* phi_bins, int n_phi, const int32_t* blocks_per_sm,
                      int n_bps, const int32_t* search_blocks_per_sm, int n_sbps, int reps,
                      int32_t* best, float* results) {
  g_err.clear();
  if (!cap || !phi_bins || !blocks_per_sm || !search_blocks_per_sm || n_phi < 1 || n_bps < 1 ||
      n_sbps < 1 || reps < 1 || !best)
    return fail(PT_ERR_INVALID, "bad autotune arguments");
  DeviceGuard guard(device);
  float best_ms = 0.0f;
  bool have = false;
  for (int i = 0; i < n_phi; ++i) {
    pt_capacity c = *cap;
    c.phi_bins = phi_bins[i];
    pt_ctx* ctx = nullptr;
    PT_TRY(pt_create(geom, cuts, &c, device, nullptr, 0, nullptr, &ctx));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pt_status st = stage_inputs(ctx, n_events, hit_offsets, x, y, z, layer, 0);
    for (int j = 0; j < n_bps * n_sbps && st == PT_OK; ++j) {
      const int jb = j / n_sbps, js = j % n_sbps;
      st = pt_set_launch(ctx, blocks_per_sm[jb], search_blocks_per_sm[js]);
      if (st == PT_OK) st = ensure_graph(ctx);
      std::vector<float> t;
      for (int r = 0; r <= reps && st == PT_OK; ++r) {  // run 0 is the warm-up
        cudaEventRecord(e0, ctx->stream);
        if (cudaGraphLaunch(ctx->graph, ctx->stream) != cudaSuccess)
          st = fail(PT_ERR_CUDA, "graph launch failed");
        cudaEventRecord(e1, ctx->stream);
        if (st == PT_OK) st = sync_counters(ctx);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) t.push_back(ms);
      }
      if (st != PT_OK) break;
      std::sort(t.begin(), t.end());
      const float med = t[t.size() / 2];
      if (results) results[(int64_t)i * n_bps * n_sbps + j] = med;
      if (!have || med < best_ms) {
        have = true;
        best_ms = med;
        best[0] = phi_bins[i];
        best[1] = blocks_per_sm[jb];
        best[2] = search_blocks_per_sm[js];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pt_destroy(ctx);
    if (st != PT_OK) return st;
  }
  return PT_OK;
}

pt_status pt_enqueue_batch(pt_ctx* c, int n_events, const int64_t* hit_offsets, const float* x,
                           const float* y, const float* z, const uint8_t* layer, int on_device) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  DeviceGuard guard(c->device);
  PT_TRY(stage_inputs(c, n_events, hit_offsets, x, y, z, layer, on_device));
  PT_TRY(ensure_graph(c));
  PT_CUDA(cudaGraphLaunch(c->graph, c->stream));
  c->fitted = true;
  c->links_masked = c->masked();  // the graph's link stage ran in the current form
  return PT_OK;
}

pt_status pt_reconstruct_batch(pt_ctx* c, int n_events, const int64_t* hit_offsets,
                               const float* x, const float* y, const float* z,
                               const uint8_t* layer, int on_device, int32_t* hits_out,
                               uint8_t* nhits_out, pt_track* tracks_out, int64_t* event_offsets,
                               int64_t cap, int64_t* n, int out_on_device) {
  g_err.clear();
  if (!c) return fail(PT_ERR_INVALID, "context is NULL");
  if (!event_offsets) return fail(PT_ERR_INVALID, "event_offsets is NULL");
  DeviceGuard guard(c->device);
  PT_TRY(stage_inputs(c, n_events, hit_offsets, x, y, z, layer, on_device));
  PT_TRY(ensure_graph(c));
  PT_CUDA(cudaGraphLaunch(c->graph, c->stream));
  c->fitted = true;
  c->links_masked = c->masked();  // the graph's link stage ran in the current form
  PT_TRY(sync_counters(c));
  const int64_t S = (int64_t)c->h_cnt[CNT_SV];
  if (n) *n = S;
  if (cap < S)
    return fail(PT_ERR_CAPACITY, "output capacity %lld is too small: %lld ntuplets",
                (long long)cap, (long long)S);
  PT_TRY(copy_out(c, hits_out, c->B.exp_hits, (size_t)S * kMaxHits * 4, out_on_device));
  PT_TRY(copy_out(c, nhits_out, c->B.exp_n, (size_t)S, out_on_device));
  PT_TRY(copy_out(c, tracks_out, c->B.tracks, (size_t)S * sizeof(pt_track), out_on_device));
  PT_TRY(copy_out(c, event_offsets, c->B.ev_nt_off, (size_t)(n_events + 1) * 8, out_on_device));
  PT_CUDA(cudaStreamSynchronize(c->stream));
  return PT_OK;
}

}  // extern "C"
