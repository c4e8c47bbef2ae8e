// Internal declarations of the GB300 pixel-track CA library: device buffer layout,
// exact float32 cut predicates and the host-side launchers of every kernel.
//
// Every kernel is a fixed-grid, grid-stride kernel that reads its work size from
// device memory (batch header or a device counter).  No stage needs a host round
// trip, so the whole chain of a batch can be replayed from one captured CUDA graph
// whatever the batch's hit, cell or link counts are.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt_ca.h"

namespace ptca {

constexpr int kLayers = 10;
constexpr int kMaxHits = 6;                // longest chain of the layer graph
constexpr int kMaxCellsPerNt = kMaxHits - 1;
constexpr int kMaxOuter = 6;               // outer layers paired with one inner layer
constexpr int kMaxInner = 6;               // inner layers paired with one outer layer
constexpr int kMaxPairs = 64;              // layer pairs of one table
constexpr int kStage = 256;                // staged doublets per (hit, outer layer)
constexpr int kLocalLinks = 8;             // links of one cell kept in registers
constexpr int kRankBits = 29;              // duplicate-cleaning key: rank field width

// device counters (unsigned long long)
enum : int {
  CNT_CELLS = 0,
  CNT_LINKS = 1,
  CNT_NT = 2,
  CNT_STATUS = 3,
  CNT_SCAN_BINS = 4,  // sizes for the device-wide scans
  CNT_SCAN_HITS = 5,
  CNT_SCAN_NT = 6,
  CNT_GATE_KEPT = 7,
  CNT_SV = 8,         // cleaned ntuplets
  CNT_SCORE_STATUS = 9,  // status bits of the standalone gate scoring (pt_gate_score)
  CNT_CELLS_USED = 10,  // cells written (CNT_CELLS counts reserved slots incl. holes)
  CNT_LINKS_USED = 11,  // links written (CNT_LINKS counts reserved slots incl. holes)
  CNT_DBL_WORK = 12,    // doublet search: next chunk of 32 sorted hits
  CNT_SCAN_EV = 13,     // events (size of the scan over per-event vertex counts)
  CNT_VTX = 14,         // vertices of the batch
  CNT_RAW_STATUS = 15,  // raw input: status bits (RAW_*), not reset by the chain
  CNT_RAW_DIGIS = 16,   // raw input: digis of the batch (size of the run-flag scan)
  CNT_RAW_RUNS = 17,    // raw input: module runs (size of the hit-count scan)
  CNT_RAW_HITS = 18,    // raw input: hits made from the digis
  CNT_RAW_BIG = 19,     // raw input: long module runs listed for the block-per-run launch
  CNT_LNK_WORK = 20,    // link search: next chunk of 32 sorted middle hits
  CNT_DEBUG_SITE = 22,  // debug build: the first failing bounds check (DebugSite)
  CNT_N = 24
};
// raw-input status bits (cnt[CNT_RAW_STATUS])
enum : unsigned long long {
  RAW_INVALID = 1ull,           // bad module, pixel, adc or pixel order
  RAW_RUN_CAPACITY = 2ull,      // more than 1024 digis of one module in one event
  RAW_CLUSTER_CAPACITY = 4ull,  // a cluster of more than 128 pixels
  RAW_HIT_CAPACITY = 8ull,      // more hits than max_hits
};
// status bits
enum : unsigned long long {
  ST_CELLS = 1ull,
  ST_LINKS = 2ull,
  ST_NT = 4ull,
  ST_LAYER = 8ull,
  ST_GATE_TIMEOUT = 16ull,  // a bounded wait in the gate kernel expired
  ST_VTX = 32ull,           // an event has more tracks for vertexing than a block sorts
  ST_DEBUG = 64ull,         // a bounds check of the debug build failed (cnt[CNT_DEBUG_SITE])
};

// Sites of the debug build's bounds checks (the first one that fails is recorded).
enum DebugSite : unsigned {
  DBG_BIN_SCATTER = 1,   // sorted position of a hit < hits
  DBG_DBL_WINDOW = 2,    // a doublet window inside the sorted hits
  DBG_DBL_CELL = 3,      // a cell slot < max_cells
  DBG_CON_WINDOW = 4,    // a forward window inside the sorted hits
  DBG_CON_INCOMING = 5,  // an incoming cell id < cell slots
  DBG_CON_BUCKET = 6,    // a bucket range inside the staged piece
  DBG_CON_QUEUE = 7,     // queued pairs <= queue size
  DBG_CON_LINK = 8,      // a link slot < max_links
  DBG_TGT_SEGMENT = 9,   // a target's incoming segment inside the cell slots
  DBG_NT_LINKS = 10,     // a cell's link run inside the link slots
  DBG_NT_CELL = 11,      // a link target < cell slots
  DBG_FIT_HITS = 12,     // 3..6 hits per fitted ntuplet
  DBG_FB_RECORD = 13,    // a fishbone record position < max_links
};

// Gate parameters on the device: W1 and W2 as bf16 in the tensor-core operand layout,
// biases and the last layer in float32.
constexpr int kGateFeat = 12;
constexpr int kGateK1 = 16;   // layer-1 K padded to the MMA K
constexpr int kGateHidden = 64;
constexpr int kGateParams = 5057;
struct GateWeights {
  uint16_t w1[kGateHidden * kGateK1];      // core-matrix layout, see gate.cu
  uint16_t w2[kGateHidden * kGateHidden];  // core-matrix layout
  float b1[kGateHidden];
  float b2[kGateHidden];
  float w3[kGateHidden];
  float b3;
  float tau;
};

struct BatchHeader {
  int32_t n_events;
  int32_t n_hits;
};

// The layer-pair table of a context, as the kernels read it (a kernel argument):
// outer[L][k], k < n_outer[L], are the outer layers paired with inner layer L, inner[L][k],
// k < n_inner[L], the inner layers paired with outer layer L (a hit's incoming segments
// are numbered by these slots), slot[L][Li] = k with inner[L][k] == Li (-1 if none), and
// max_inner = the largest n_inner (the number of incoming segments stored per hit).
struct PairTable {
  int8_t outer[kLayers][kMaxOuter];
  int8_t n_outer[kLayers];
  int8_t inner[kLayers][kMaxInner];
  int8_t n_inner[kLayers];
  int8_t slot[kLayers][kLayers];
  int8_t max_inner;
};

// Builds the table of n (inner, outer) pairs, in the given order; false if a pair is out
// of range, repeated or pairs a layer with itself, if a layer gets more than kMaxOuter
// outer or kMaxInner inner layers, or if the layer graph has a cycle or a path of more
// than kMaxHits - 1 pairs.
bool make_pair_table(int n, const int32_t* inner, const int32_t* outer, PairTable* t);
// The chain's 13 pairs: barrel 0-1, 1-2, 2-3, and per side the three inner barrel
// layers and the disk chain into the first disk (0/1/2-4, 4-5, 5-6; 0/1/2-7, 7-8, 8-9).
PairTable default_pair_table();

struct Params {
  pt_cuts cuts;
  PairTable pairs;
  long long wait_cycles;  // limit of the bounded device-side waits (SM clock cycles)
  float bfield;
  int32_t phi_bins;
  int64_t max_events, max_hits, max_cells, max_links, max_ntuplets;
};

// Device buffers carved out of one workspace block (see layout() in runtime.cu).
struct Buffers {
  BatchHeader* hdr;
  unsigned long long* cnt;   // [CNT_N]
  // inputs, batch order
  float* in_x;
  float* in_y;
  float* in_z;
  uint8_t* in_layer;
  int32_t* hit_off;          // [max_events + 1]
  uint32_t* in_bin;          // [max_hits] global bin of input hit (or ~0)
  uint32_t* in_rank;         // [max_hits] rank within the bin
  // hits sorted by (event, layer, phi bin)
  float4* hit4;              // [max_hits] (x, y, z, r)
  uint32_t* perm;            // [max_hits] sorted -> input (batch) index
  uint32_t* hbin;            // [max_hits] global bin of sorted hit
  uint32_t* bin_cnt;         // [max_events*10*B + 1]
  uint32_t* bin_start;       // [max_events*10*B + 1]
  uint32_t* layer_rmax;      // [max_events*10] float bits of max r per event layer
  float* layer_asin;         // [max_events*10] asin(kmax r_max / 2) per event layer,
                             //   +inf when kmax r_max / 2 >= 0.7
  uint32_t* layer_rmin;      // [max_events*10] float bits of min r per event layer (+inf
                             //   for an empty layer)
  float* layer_asin_lo;      // [max_events*10] asin(kmax r_min / 2) (0 where that is >= 0.7
                             //   or the layer is empty)
  uint32_t* layer_zmin;      // [max_events*10] order keys (float_order_key) of min and max
  uint32_t* layer_zmax;      //   z per event layer (~0 and 0 for an empty layer)
  // incoming segments: per sorted (outer) hit and inner-layer slot, the cells ending on
  // the hit from that layer, cells [x, x + y), ordered by inner hit; the table's
  // max_inner slots per hit, all written
  uint2* seg;                // [max_hits*kMaxInner]
  // cells
  uint32_t* cell_in;         // [max_cells] sorted hit index
  uint32_t* cell_out;        // [max_cells]
  uint8_t* has_in;           // [max_cells] an accepted link ends on the cell
  uint8_t* has_out;          // [max_cells] an accepted link starts from the cell
  uint8_t* fb_kill;          // [max_cells] removed by the fishbone step (zeroed for every
                             //   cell when the step runs)
  uint32_t* fb_cnt;          // [max_hits + 1] fishbone: active cells per outer hit
  uint32_t* fb_start;        // [max_hits + 1]   and their first position in fb_list
  float4* fb_rec;            // [max_links * 2] active cells grouped by outer hit: vector to
                             //   the hit and |.|^2; cell, inner hit's input index, layer, sensor
  uint32_t* cell_head;       // [max_cells] the cell's latest out-link slot, the head of
                             //   its out-link list (valid where it has links)
  unsigned long long* best;  // [max_cells] duplicate-cleaning key (cells on ntuplets)
  // links
  uint32_t* link_dst;        // [max_links]
  uint32_t* link_next;       // [max_links] the source's next out-link slot (kHole: last)
  uint2* link_walk;          // [max_links] plain form: the target cell's out-link list head
                             //   (kHole: a leaf) and its outer hit (sorted index), written
                             //   with the target so that the ntuplet walk reads each step
                             //   from the link alone
  float* link_q;             // [max_links]
  // ntuplets before cleaning
  int32_t* nt_hits;          // [max_ntuplets*6] batch input index, -1 pad
  uint32_t* nt_cells;        // [max_ntuplets*5]
  uint8_t* nt_n;             // [max_ntuplets]
  float* nt_q;               // [max_ntuplets]
  uint32_t* nt_rank;         // [max_ntuplets] rank within its first-hit bucket, then (after
                             //   the canonical sort) its sorted position
  // canonical order
  uint32_t* bucket_cnt;      // [max_hits + 1]
  uint32_t* bucket_start;    // [max_hits + 1]
  uint32_t* ord;             // [max_ntuplets] sorted position -> ntuplet
  uint32_t* alive;           // [max_ntuplets]
  uint32_t* alive_scan;      // [max_ntuplets + 1]
  uint8_t* used;             // [max_hits]
  uint32_t* sv;              // [max_ntuplets] survivor -> sorted position
  int64_t* ev_nt_off;        // [max_events + 1]
  pt_track* tracks;          // [max_ntuplets]
  // primary vertices (pt_find_vertices)
  pt_vertex* vtx_stage;      // [max_ntuplets / 2 + 1] event e's vertices from floor(t0 / 2)
  pt_vertex* vtx;            // [max_ntuplets / 2 + 1] the batch's vertices, events in order
  int32_t* trk_vtx;          // [max_ntuplets] vertex of each track, -1 for none
  uint32_t* ev_nv;           // [max_events + 1] vertices per event
  uint32_t* ev_v_scan;       // [max_events + 1] exclusive scan of ev_nv
  int64_t* ev_vtx_off;       // [max_events + 1] the same as int64
  // learned gate (valid when enabled)
  uint16_t* gate_x;          // [max_links*16] bf16 features per link slot (12 used)
  float* gate_score;         // [max_links] logit per link slot
  uint8_t* gate_keep;        // [max_links] 1 where the link passes the gate
  uint32_t* link_src;        // [max_links] source cell of each link slot, kHole for unused
                             //   slots
  int32_t* exp_hits;         // [max_ntuplets*6] export staging (event-local indices)
  uint8_t* exp_n;            // [max_ntuplets]
  float* exp_q;              // [max_ntuplets]
  int32_t* exp_ev;           // [max_ntuplets]
  uint32_t* scan_part;       // [kScanBlocks + 1]
};

constexpr int kScanBlocks = 256;

// Raw-input scratch (allocated on the first pt_load_raw): the digis and the per-digi /
// per-run arrays of the clustering; max_digis entries (+1 for the scans).
struct RawBuffers {
  int n_events = 0;
  int64_t* digi_off = nullptr;   // [max_events + 1] event e owns digis [off[e], off[e+1])
  uint64_t* words = nullptr;     // [max_digis] packed digis
  uint32_t* flag = nullptr;      // [max_digis + 1] 1 where a module run starts
  uint32_t* run_scan = nullptr;  // [max_digis + 1] runs starting before each digi
  uint32_t* run_first = nullptr; // [max_digis + 1] first digi of each run (+ end)
  uint32_t* run_nh = nullptr;    // [max_digis + 1] hits of each run
  uint32_t* run_hoff = nullptr;  // [max_digis + 1] first hit of each run (+ total)
  float4* stage = nullptr;       // [max_digis] hits (x, y, z, layer bits) at digi positions
  uint32_t* big_runs = nullptr;  // aliases flag (free once the runs are numbered): long runs
  uint32_t* scan_part = nullptr; // the context's scan partials
  unsigned long long* cnt = nullptr;  // the context's counters
};

// Optional per-kernel timing of the stage calls (pt_set_tracing): CUDA events on the
// launching stream around every kernel; never active while the whole-batch graph is
// captured.  Defined in runtime.cu.
struct Tracer;
size_t trace_begin(Tracer* t, cudaStream_t s);
void trace_end(Tracer* t, const char* name, size_t i0, cudaStream_t s);
#define PT_TRACE(l, s, name, ...)                                  \
  do {                                                             \
    const size_t pt_t0_ = (l).tr ? trace_begin((l).tr, (s)) : 0;   \
    __VA_ARGS__;                                                   \
    if ((l).tr) trace_end((l).tr, (name), pt_t0_, (s));            \
  } while (0)

struct Launch {
  int sms;                // multiprocessors
  int grid;               // generic persistent grid (blocks of 256 threads)
  int sgrid;              // grid of the doublet search (warp per hit)
  Tracer* tr = nullptr;   // per-kernel timing, when enabled
};

// Sets the calling thread's pt_last_error() message.
void set_last_error(const char* msg);

// Requests a server has completed since it was created (for the router's balancing).
int64_t server_finished(pt_server* s);

// Asynchronous pieces of a batch for the request server (runtime.cu): read-back of the
// counters, status check of that copy, and copies of the cleaned ntuplets, tracks and
// per-event offsets into host memory, each completion recorded on `done`.
cudaStream_t ctx_stream(pt_ctx* c);
pt_status ctx_counters_async(pt_ctx* c, cudaEvent_t done);
pt_status ctx_read_counters(pt_ctx* c, int64_t* n_ntuplets);
pt_status ctx_results_async(pt_ctx* c, int64_t S, int32_t* hits, uint8_t* nhits,
                            pt_track* tracks, int64_t* event_offsets, cudaEvent_t done);

// ------------------------------------------------------------------ launchers
void launch_clear(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s);
void launch_bin_hits(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s);
void launch_doublets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s);
// gated = true: the link search also writes each link's gate features and source cell,
// and leaves the in/out flags to the gate (launch_gate)
void launch_connect(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                    bool gated = false);
// Fishbone step and the link filter after it (keep mask and link flags of the ntuplet
// search); gated: the gate's keep mask is the starting point.
void launch_fishbone(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                     bool gated);
// Debug build: records a failure of bounds check `site` as a failing check does.
cudaError_t launch_debug_inject(const Buffers& b, unsigned site, cudaStream_t s);
void launch_ntuplets(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s,
                     bool gated = false);
void launch_fit(const Buffers& b, const Params& p, const Launch& l, cudaStream_t s);
// raw digis -> hits in the chain's input arrays, per-event offsets and header
cudaError_t launch_raw(const RawBuffers& r, const Buffers& b, const pt_module* mods, int n_mod,
                       int64_t cap_hits, const Launch& l, cudaStream_t s);
// primary vertices of the fitted tracks of n_events events (tracks with >= min_hits
// hits, groups cut at z0 steps > dz)
cudaError_t launch_vertices(const Buffers& b, int n_events, int32_t min_hits, float dz,
                            uint64_t cap_nt, const Launch& l, cudaStream_t s);
// scan of n+1 entries: out[i] = sum(in[0..i)), n = *n_dev
void launch_scan(const uint32_t* in, uint32_t* out, const unsigned long long* n_dev,
                 uint32_t* part, cudaStream_t s);
// learned gate: features, tensor-core MLP and link pruning (enabled contexts only);
// gate_prepare() sets the MLP kernel's shared-memory attribute (call before capture)
cudaError_t gate_prepare();
void launch_gate(const Buffers& b, const Params& p, const Launch& l, const GateWeights* w,
                 cudaStream_t s);
// scores of n feature rows (float32 [n][12], device) with the gate's MLP -> out [n]
void launch_gate_score(const GateWeights* w, const float* feat, int64_t n, float* out,
                       uint16_t* xbuf, unsigned long long* status, int sms, long long wait_cycles,
                       cudaStream_t s);
// float32 features of the current links (gated: kept only) -> out [slots][12]
void launch_export_link_features(const Buffers& b, const Params& p, const Launch& l, bool gated,
                                 float* out, cudaStream_t s);
// gate training: mean BCE loss and its gradient (zeroed first); Adam step
cudaError_t launch_gate_grad(const float* w, const float* X, const float* y, int64_t n,
                             float* grad, float* loss, int sms, cudaStream_t s);
cudaError_t launch_gate_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr,
                             float b1, float b2, float eps, int step, cudaStream_t s);
// exports with event-local input indices
void launch_export_ntuplets(const Buffers& b, const Launch& l, cudaStream_t s);
void launch_export_candidates(const Buffers& b, const Launch& l, cudaStream_t s);
// cells -> out3 [n][3] (inner, outer, event); links -> out4 [n][4] (h0, h1, h2, event), q
void launch_export_cells(const Buffers& b, const Params& p, const Launch& l, int32_t* out3,
                         cudaStream_t s);
void launch_export_links(const Buffers& b, const Params& p, const Launch& l, int32_t* out4,
                         float* outq, cudaStream_t s, bool gated = false);

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
constexpr unsigned kFull = 0xffffffffu;

// Correctly rounded float32 operations that the compiler never contracts into FMA.
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// Order-preserving map of a float to an unsigned key (for atomicMin / atomicMax), and
// back.
__device__ __forceinline__ uint32_t float_order_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Whether a layer whose hits lie in the r-z box [rlo, rhi] x [zlo, zhi] can hold a
// partner of the hit (r, z), outward (larger r) or inward, that passes D2 and D3.  Both
// cuts bound the r-z slope s of the cell: |s| <= cotmax, and the line's z at r = 0,
// which is z - r s from either hit, within +-z0max.  Seen from the hit, the slopes of
// the box's points with a positive radial step fill the interval between its corners'
// slopes; the layer is ruled out only when that interval lies wholly beyond the allowed
// one, compared in multiplied form with margins (1e-3 on slopes, 1e-3 cm on z) far above
// float32 rounding.  Boxes reaching to the hit's radius or inside it are kept (D0
// decides them).
__device__ __forceinline__ bool rz_box_reachable(const pt_cuts& c, float r, float z, float rlo,
                                                 float rhi, float zlo, float zhi, bool outward) {
  float d0, d1, e0, e1;  // radial steps and z steps (towards the partner) over the box
  if (outward) {
    d0 = fmaxf(rlo - r, 0.0f), d1 = rhi - r, e0 = zlo - z, e1 = zhi - z;
  } else {
    d0 = fmaxf(r - rhi, 0.0f), d1 = r - rlo, e0 = z - zhi, e1 = z - zlo;
  }
  if (!(d1 > 0.0f) || !(r > 0.0f)) return true;
  const float lo = fmaxf((z - c.z0max) / r, -c.cotmax);
  const float hi = fminf((z + c.z0max) / r, c.cotmax);
  const float slo = lo - 1e-3f * (1.0f + fabsf(lo)), shi = hi + 1e-3f * (1.0f + fabsf(hi));
  e0 -= 1e-3f;
  e1 += 1e-3f;
  // largest slope of the box below slo, or its smallest above shi
  const bool below = e1 >= 0.0f ? e1 < slo * d0 : e1 < slo * d1;
  const bool above = e0 <= 0.0f ? e0 > shi * d0 : e0 > shi * d1;
  return !(below || above);
}

// Doublet cuts D0..D4 on (x, y, z, r) of the inner and outer hit, in the library's
// fixed evaluation order (see pt_cuts in pt_ca.h).
__device__ __forceinline__ bool doublet_pass(const pt_cuts& c, float4 hi, float4 ho) {
  const float dx = fsub(ho.x, hi.x), dy = fsub(ho.y, hi.y);
  const float dr = fsub(ho.w, hi.w), dz = fsub(ho.z, hi.z);
  if (!(dr > 0.0f)) return false;
  if (!(fadd(fmul(hi.x, ho.x), fmul(hi.y, ho.y)) > 0.0f)) return false;
  if (!(fabsf(fsub(fmul(hi.z, dr), fmul(hi.w, dz))) <= fmul(c.z0max, dr))) return false;
  if (!(fabsf(dz) <= fmul(c.cotmax, dr))) return false;
  const float l2 = fmul(fabsf(fsub(fmul(hi.x, ho.y), fmul(hi.y, ho.x))), 2.0f);
  const float r2 = fmul(c.kmax, fmul(fmul(hi.w, ho.w), fsqrt(fadd(fmul(dx, dx), fmul(dy, dy)))));
  return l2 <= r2;
}

// r-z alignment C1 only (cheap first test of a link).
__device__ __forceinline__ bool link_c1(const pt_cuts& c, float4 p0, float4 p1, float4 p2) {
  const float lc1 = fabsf(fsub(fmul(fsub(p1.z, p0.z), fsub(p2.w, p0.w)),
                               fmul(fsub(p2.z, p0.z), fsub(p1.w, p0.w))));
  const float rc1 = fadd(fmul(c.rz0, fsub(p2.w, p0.w)), fmul(c.rz1, fabsf(fsub(p2.z, p0.z))));
  return lc1 <= rc1;
}

// Curvature C2 and beam-spot distance C3 of the circle through three hits; q gets the
// distance (link quality) when both pass.
__device__ __forceinline__ bool link_c23(const pt_cuts& c, float4 p0, bool first_on_b0, float4 p1,
                                         float4 p2, float& q) {
  const float ax = fsub(p1.x, p0.x), ay = fsub(p1.y, p0.y);
  const float bx = fsub(p2.x, p0.x), by = fsub(p2.y, p0.y);
  const float cx = fsub(p2.x, p1.x), cy = fsub(p2.y, p1.y);
  const float a2 = fadd(fmul(ax, ax), fmul(ay, ay));
  const float b2 = fadd(fmul(bx, bx), fmul(by, by));
  const float cr = fsub(fmul(ax, by), fmul(ay, bx));
  const float lc2 = fmul(fabsf(cr), 2.0f);
  const float rc2 =
      fmul(c.kmax, fmul(fmul(fsqrt(a2), fsqrt(b2)), fsqrt(fadd(fmul(cx, cx), fmul(cy, cy)))));
  if (!(lc2 <= rc2)) return false;
  const float D = fmul(cr, 2.0f);
  const float ux = fsub(fmul(by, a2), fmul(ay, b2));
  const float uy = fsub(fmul(ax, b2), fmul(bx, a2));
  const float num = fadd(fmul(fadd(fmul(p0.x, p0.x), fmul(p0.y, p0.y)), D),
                         fmul(fadd(fmul(p0.x, ux), fmul(p0.y, uy)), 2.0f));
  const float px = fadd(fmul(p0.x, D), ux);
  const float py = fadd(fmul(p0.y, D), uy);
  const float den =
      fadd(fsqrt(fadd(fmul(px, px), fmul(py, py))), fsqrt(fadd(fmul(ux, ux), fmul(uy, uy))));
  const float dcamax = first_on_b0 ? c.dca_b0 : c.dca_other;
  const float l3 = fabsf(num);
  if (!(l3 <= fmul(dcamax, den))) return false;
  q = fdiv(l3, den);
  return true;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Bounds checks of the debug build (compiled with -DPT_DEBUG, libptca_debug.so): a
// failing check sets the status bit ST_DEBUG and records the first failing site, and the
// access it guards is skipped, so that the kernel reports the fault instead of making
// it.  In the normal build every check is the constant true and costs nothing.
#ifdef PT_DEBUG
__device__ __noinline__ inline void debug_fail(unsigned long long* cnt, unsigned site) {
  atomicOr(&cnt[CNT_STATUS], ST_DEBUG);
  atomicCAS(&cnt[CNT_DEBUG_SITE], 0ull, (unsigned long long)site);
}
#define PT_CHECK(cnt, cond, site) ((cond) ? true : (::ptca::debug_fail((cnt), (site)), false))
#else
#define PT_CHECK(cnt, cond, site) true
#endif

// Learned-gate features of link (h0 -> h1 -> h2) from the hit coordinates (x, y, z, r)
// and layers: C1, C2, C3 cut ratios, t_a/cotmax, 10 (t_b - t_a), r0/16, r1/16, r2/16,
// (z0 - r0 t_a)/z0max, layer0/9, layer1/9, layer2/9.
__device__ __forceinline__ void gate_link_features(const pt_cuts& c, float4 p0, float4 p1,
                                                   float4 p2, int L0, int L1, int L2,
                                                   float (&f)[12]) {
  const float lc1 = fabsf((p1.z - p0.z) * (p2.w - p0.w) - (p2.z - p0.z) * (p1.w - p0.w));
  const float rc1 = c.rz0 * (p2.w - p0.w) + c.rz1 * fabsf(p2.z - p0.z);
  const float ax = p1.x - p0.x, ay = p1.y - p0.y, bx = p2.x - p0.x, by = p2.y - p0.y;
  const float cx = p2.x - p1.x, cy = p2.y - p1.y;
  const float a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
  const float cr = ax * by - ay * bx;
  const float kap = 2.0f * fabsf(cr) / (sqrtf(a2) * sqrtf(b2) * sqrtf(cx * cx + cy * cy));
  const float D = 2.0f * cr;
  const float ux = by * a2 - ay * b2, uy = ax * b2 - bx * a2;
  const float num = (p0.x * p0.x + p0.y * p0.y) * D + 2.0f * (p0.x * ux + p0.y * uy);
  const float px = p0.x * D + ux, py = p0.y * D + uy;
  const float den = sqrtf(px * px + py * py) + sqrtf(ux * ux + uy * uy);
  const float dmax = L0 == 0 ? c.dca_b0 : c.dca_other;
  const float ta = (p1.z - p0.z) / (p1.w - p0.w);
  const float tb = (p2.z - p1.z) / (p2.w - p1.w);
  f[0] = lc1 / rc1;
  f[1] = kap / c.kmax;
  f[2] = fabsf(num) / den / dmax;
  f[3] = ta / c.cotmax;
  f[4] = 10.0f * (tb - ta);
  f[5] = p0.w * (1.0f / 16.0f);
  f[6] = p1.w * (1.0f / 16.0f);
  f[7] = p2.w * (1.0f / 16.0f);
  f[8] = (p0.z - p0.w * ta) / c.z0max;
  f[9] = L0 * (1.0f / 9.0f);
  f[10] = L1 * (1.0f / 9.0f);
  f[11] = L2 * (1.0f / 9.0f);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
  return lo | (hi << 16);
}

// Writes the 12 features as one bf16 row of 16 (4 zeros) = 32 bytes.
__device__ __forceinline__ void store_gate_row(uint16_t* row, const float (&f)[12]) {
  uint4 lo, hi;
  lo.x = pack_bf16x2(f[0], f[1]);
  lo.y = pack_bf16x2(f[2], f[3]);
  lo.z = pack_bf16x2(f[4], f[5]);
  lo.w = pack_bf16x2(f[6], f[7]);
  hi.x = pack_bf16x2(f[8], f[9]);
  hi.y = pack_bf16x2(f[10], f[11]);
  hi.z = 0;
  hi.w = 0;
  ((uint4*)row)[0] = lo;
  ((uint4*)row)[1] = hi;
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

constexpr uint32_t kHole = 0xffffffffu;  // marks a reserved but unused slot

// Per-warp bump allocator over a global counter.  The first chunk is exactly the first
// request (a warp that makes one request wastes nothing); later chunks double from
// kChunkMin up to kChunkMax, so a busy warp takes a global atomic about once per
// kChunkMax slots instead of once per request.  The unused tail of a chunk becomes a
// hole that the owner marks.  All members are warp-uniform.
struct WarpChunk {
  unsigned long long next = 0, end = 0;
  uint32_t size = 0;
};
constexpr uint32_t kChunkMin = 32;
constexpr uint32_t kChunkMax = 2048;

// Reserves n contiguous slots; returns the first.  The caller marks [old next, old end)
// as a hole when a new chunk is taken (reported through *hole_lo / *hole_hi).
__device__ __forceinline__ unsigned long long chunk_take(WarpChunk& ch, unsigned long long* counter,
                                                         uint32_t n, unsigned long long* hole_lo,
                                                         unsigned long long* hole_hi) {
  *hole_lo = *hole_hi = 0;
  if (ch.next + n > ch.end) {
    *hole_lo = ch.next;
    *hole_hi = ch.end;
    const uint32_t want = ch.size == 0 ? n : (n > ch.size ? n : ch.size);
    ch.size = ch.size == 0 ? (n > kChunkMin ? n : kChunkMin) : min(2 * ch.size, kChunkMax);
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0) base = atomicAdd(counter, (unsigned long long)want);
    base = __shfl_sync(0xffffffffu, base, 0);
    ch.next = base;
    ch.end = base + want;
  }
  const unsigned long long r = ch.next;
  ch.next += n;
  return r;
}

// Event owning batch hit g: largest e with off[e] <= g (empty events are skipped).
__device__ __forceinline__ int find_event(const int32_t* off, int n_events, int g) {
  int lo = 0, hi = n_events - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#endif

}  // namespace ptca
