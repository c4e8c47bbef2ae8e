/*
 * pt_ca.h -- C ABI of the GB300 pixel-track cellular automaton.
 *
 * The library implements, on one GPU, the pattern-recognition chain that the paper
 * serves as its rule-based tracking workload (Sec. 2.2.1, Fig. 2): hits on adjacent
 * detector layers are paired into doublets ("cells"), cells that share a hit are
 * linked by a cellular automaton into triplets, hit chains ("ntuplets") that may be
 * tracks are extracted and cleaned of duplicates, and a fit gives the track
 * parameters.  Detector constants are loaded once when a context is created and
 * intermediates stay on the device (Sec. 2.2.1 and Sec. 3); several requests can be
 * in flight on one GPU (Sec. 3, Sec. 4.2).
 *
 * Conventions for every function:
 *   - Return a pt_status; never throw, never abort.  On failure, pt_last_error()
 *     returns a message for the calling thread (valid until that thread's next call).
 *   - Input buffers are borrowed for the duration of the call only; output buffers are
 *     owned by the caller.  `on_device` = 1 means the pointer is a device pointer on
 *     the context's device, 0 means host memory (pinned host memory is faster).
 *   - Hit indices in outputs are the caller's input indices within the event (0-based),
 *     listed from the innermost to the outermost hit, padded with -1 to 6 entries.
 *   - Ntuplets of an event are returned in canonical order: hit tuple ascending
 *     (signed comparison, so a tuple sorts before its longer extensions).
 *   - Capacities are never exceeded silently: the call returns PT_ERR_CAPACITY and
 *     pt_last_error() names the capacity and the size that was needed.
 *   - A context is used by one host thread at a time; contexts are independent.
 *   - All GPU work of a context is issued on its stream, in call order.
 *
 * Layer codes: 0..3 barrel layers (inner to outer), 4..6 disks at +z (|z|
 * increasing), 7..9 disks at -z.  Allowed layer pairs (inner, outer):
 *   (0,1) (1,2) (2,3) (0,4) (1,4) (2,4) (4,5) (5,6) (0,7) (1,7) (2,7) (7,8) (8,9).
 * Units: cm, GeV, tesla.  The beam spot is the z axis (x = y = 0).
 */
#ifndef PT_CA_H
#define PT_CA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PT_OK = 0,
  PT_ERR_INVALID = 1,   /* bad argument: NULL pointer, negative size, layer code > 9 ... */
  PT_ERR_CAPACITY = 2,  /* a capacity of the context is too small for this input */
  PT_ERR_CUDA = 3,      /* a CUDA runtime call failed; message has the CUDA error string */
  PT_ERR_TIMEOUT = 4,   /* a bounded wait expired (pt_poll) */
  PT_ERR_NOT_READY = 5, /* result not ready yet (pt_poll with timeout 0) */
  PT_ERR_NOMEM = 6,     /* device or host allocation failed, or the budget is exhausted */
  PT_ERR_INTERNAL = 7   /* debug build only: a device-side bounds check failed (a library
                         * fault, reported instead of made; the message names the check) */
} pt_status;

typedef struct pt_ctx pt_ctx;

/* Cut constants (float32).  Every cut is evaluated in float32 with correctly rounded
 * + - * / sqrt only, in a fixed order, without fused multiply-add:
 *   doublet (inner i, outer o; dx = xo-xi, dy = yo-yi, dr = ro-ri, dz = zo-zi):
 *     D0 dr > 0;  D1 xi*xo + yi*yo > 0;
 *     D2 |xi*yo - yi*xo| * 2 <= kmax * ((ri*ro) * sqrt(dx*dx + dy*dy));
 *     D3 |zi*dr - ri*dz| <= z0max * dr;   D4 |dz| <= cotmax * dr.
 *   link of cells (h0,h1) -> (h1,h2):
 *     C1 |(z1-z0)*(r2-r0) - (z2-z0)*(r1-r0)| <= rz0*(r2-r0) + rz1*|z2-z0|;
 *     C2 curvature of the circle through the three hits <= kmax;
 *     C3 distance of closest approach of that circle to the z axis <= dca_b0 when h0
 *        is on layer 0, else dca_other (division-free form; the quotient is the link
 *        quality q). */
typedef struct {
  float kmax;      /* 1/cm */
  float z0max;     /* cm */
  float cotmax;
  float rz0;       /* cm */
  float rz1;
  float dca_b0;    /* cm */
  float dca_other; /* cm */
} pt_cuts;

typedef struct {
  float bfield_T;  /* solenoid field along +z, used for pT = 0.299792458 B / (100 |kappa|) */
} pt_geometry;

typedef struct {
  int64_t max_events;   /* events per batch */
  int64_t max_hits;     /* hits per batch (all events together) */
  int64_t max_cells;    /* doublets per batch */
  int64_t max_links;    /* accepted cell links per batch */
  int64_t max_ntuplets; /* ntuplets before duplicate cleaning, per batch */
  int32_t phi_bins;     /* azimuthal bins per layer, 16..4096 */
  int32_t reserved;     /* must be 0 */
} pt_capacity;

/* One fitted track.  kappa > 0: counter-clockwise seen from +z moving outwards;
 * phi0: direction of motion at the point of closest approach to the z axis, which is
 * d0 * (sin phi0, -cos phi0); z0 and cot_theta: z = z0 + cot_theta * s along the
 * transverse arc length s from that point; chi2 with 10 um (r-phi) and 20 um (z)
 * errors; charge = -sign(kappa). */
typedef struct {
  float kappa, phi0, d0, cot_theta, z0, pt, chi2_circle, chi2_line;
  int8_t charge;
  uint8_t nhits;
  uint8_t pad[2];
} pt_track;

/* One detector module of the pixel readout (pt_set_modules).  A pixel (row, col) of
 * the module covers azimuths phi0 + [col, col + 1) dphi_col and, along v (z on a barrel
 * module, r on a disk module), v0 + [row, row + 1) dv_row. */
typedef struct {
  int32_t layer;     /* layer code 0..9 */
  int32_t kind;      /* 0: barrel (at radius rz, rows along z); 1: disk (at z = rz, rows along r) */
  float rz;          /* barrel radius or disk z (cm) */
  float phi0;        /* azimuth of column 0's lower edge (rad) */
  float dphi_col;    /* azimuth per column (rad) */
  float v0;          /* z (barrel) or r (disk) of row 0's lower edge (cm) */
  float dv_row;      /* cm per row */
  int32_t ncol;      /* columns, 1..4096 */
  int32_t nrow;      /* rows, 1..4096 */
} pt_module;

/* One primary vertex (pt_find_vertices): z (cm), the sum of its tracks' pT^2 (GeV^2),
 * its number of tracks and its event in the batch. */
typedef struct {
  float z;
  float sum_pt2;
  int32_t n_tracks;
  int32_t event;
} pt_vertex;

/* ------------------------------------------------------------------ lifecycle */

/* Device bytes needed for a context of the given capacity (the workspace that
 * pt_create borrows when the caller supplies one).  Sec. 2.2.1: intermediates are kept
 * on the device, so all per-batch state lives in this one block. */
pt_status pt_workspace_size(const pt_capacity* cap, size_t* bytes);

/* Create a context on `device` (Sec. 3: detector constants are loaded once at start).
 * Capacity limits: max_hits < 2^29, max_cells and max_links < 2^32 - 1, max_ntuplets
 * < 2^29, phi_bins in [16, 4096], max_events * 10 * phi_bins < 2^31 - 1, reserved 0;
 * anything else is PT_ERR_INVALID.
 * workspace: device memory of >= pt_workspace_size bytes, 256-byte aligned, owned by
 *            the caller and borrowed until pt_destroy; NULL lets the library allocate.
 * stream:    a cudaStream_t owned by the caller, or NULL to create a private stream.
 * All three structs are copied.  On failure *out is NULL. */
pt_status pt_create(const pt_geometry* geom, const pt_cuts* cuts, const pt_capacity* cap,
                    int device, void* workspace, size_t workspace_bytes, void* stream,
                    pt_ctx** out);

/* Destroy a context; waits for its stream, frees what the library allocated. NULL ok. */
pt_status pt_destroy(pt_ctx* ctx);

/* Replace the stream of a context (caller-owned cudaStream_t, or NULL for private). */
pt_status pt_set_stream(pt_ctx* ctx, void* stream);

/* ------------------------------------------------------------ stage calls (Fig. 2) */

/* Load one event of n hits (x, y, z float32, layer uint8) and sort it into per-layer
 * azimuthal bins on the device.  Equivalent to pt_load_batch with one event. */
pt_status pt_load_hits(pt_ctx* ctx, int64_t n, const float* x, const float* y, const float* z,
                       const uint8_t* layer, int on_device);

/* Load a batch of events.  hit_offsets: host array [n_events + 1], offsets[0] = 0,
 * non-decreasing; event e owns hits [offsets[e], offsets[e+1]) of the x/y/z/layer
 * arrays.  Errors: PT_ERR_INVALID for bad offsets or a layer code > 9 (checked on the
 * device; reported by the next call that synchronises), PT_ERR_CAPACITY. */
pt_status pt_load_batch(pt_ctx* ctx, int n_events, const int64_t* hit_offsets, const float* x,
                        const float* y, const float* z, const uint8_t* layer, int on_device);

/* Detector module table of the pixel readout, used by pt_load_raw (Sec. 2.2.1, Fig. 2:
 * the fixed description of the detector's layers and module numbering sits on the GPU
 * before any event arrives).  modules[i] describes module index i; n in [1, 2^24).  The table
 * is copied into a device buffer that the context allocates and keeps.  PT_ERR_INVALID
 * for a layer code > 9, a kind other than 0/1, ncol or nrow outside [1, 4096] or a
 * non-finite float. */
pt_status pt_set_modules(pt_ctx* ctx, const pt_module* modules, int n);

/* Load a batch of raw pixel events (Sec. 2.2.1, Fig. 2: the compressed raw data are
 * unpacked on the GPU into digis, and neighbouring digis of one layer are clustered into
 * hits; the paper fixes no format).  digis: one 64-bit word per read-out pixel,
 * module << 40 | row << 28 | col << 16 | adc (adc <= 4095), event e owning
 * [digi_offsets[e], digi_offsets[e+1]) (host array [n_events + 1]); within an event the
 * digis come grouped by module and, within a module, in (row, col) order, each pixel
 * once.  Digis of one module whose pixels touch at an edge or a corner form a cluster;
 * each cluster gives one hit at its adc-weighted mean pixel centre on the module's
 * surface, with the module's layer.  Hits come module run by module run in input order,
 * and within a module in order of their cluster's first pixel.  The hits replace the
 * context's inputs as pt_load_batch's would and are binned for the chain.  The first
 * call allocates the raw-input scratch (8 x max_hits digis).  n_hits: NULL to stay
 * asynchronous, else the call synchronises and stores the number of hits.  Errors:
 * PT_ERR_INVALID (no module table, bad offsets, a module index, pixel or adc outside
 * the table or the range, pixels out of order or repeated); PT_ERR_CAPACITY (more than
 * 8 x max_hits digis, more hits than max_hits, more than 1024 digis on one module of an
 * event, a cluster of more than 128 pixels). */
pt_status pt_load_raw(pt_ctx* ctx, int n_events, const int64_t* digi_offsets,
                      const uint64_t* digis, int on_device, int64_t* n_hits);

/* The hits of the loaded batch as the chain sees them (pt_load_batch's inputs, or the
 * hits pt_load_raw made): x, y, z [cap] float32, layer [cap] uint8 (any may be NULL),
 * event_offsets [n_events + 1] int64 (may be NULL).  *n = number of hits;
 * PT_ERR_CAPACITY if cap < *n (nothing written).  Host buffers; synchronises. */
pt_status pt_get_hits(pt_ctx* ctx, float* x, float* y, float* z, uint8_t* layer,
                      int64_t* event_offsets, int64_t cap, int64_t* n);

/* Doublets of the loaded batch (Sec. 2.2.1, Fig. 2: hits in adjacent layers are
 * paired).  n_cells: NULL to stay asynchronous; else the call synchronises the stream
 * and stores the number of cells (and reports capacity errors). */
pt_status pt_build_doublets(pt_ctx* ctx, int64_t* n_cells);

/* Cellular-automaton links of cells that share a hit (Sec. 2.2.1: doublets are paired
 * to triplets).  n_links as above. */
pt_status pt_connect_cells(pt_ctx* ctx, int64_t* n_links);

/* Ntuplets: every path of linked cells from a cell without an incoming link to a cell
 * without an outgoing link, 3..6 hits (Sec. 2.2.1: the chain selects candidate sets of
 * hits), then duplicate cleaning and canonical ordering.  n_ntuplets
 * receives the number of cleaned ntuplets.  The links are taken as the last
 * pt_connect_cells left them: with the gate's and fishbone step's keep mask if either was
 * on then, whatever pt_set_gate or pt_set_fishbone were called with since. */
pt_status pt_find_ntuplets(pt_ctx* ctx, int64_t* n_ntuplets);

/* Circle + line fit of every cleaned ntuplet (Sec. 2.2.1: a fit determines the track
 * parameters).  n_tracks as above. */
pt_status pt_fit_tracks(pt_ctx* ctx, int64_t* n_tracks);

/* Broken-line refit of the fitted tracks, in place (Sec. 2.2.1: a fit determines the
 * track parameters; broken lines after V. Blobel, NIM A566 (2006) 14).  Each track's
 * circle + line fit is the reference; its offsets at the hits, one curvature
 * correction and the multiple-scattering kinks at the interior hits (Highland variances
 * for x0_barrel / x0_disk radiation lengths per layer at normal incidence, with 10 um
 * r-phi and 20 um z / r hit errors) are solved by linear least squares in float64, and
 * the parameters at the closest approach replace the track's; chi2_circle and
 * chi2_line become the two planes' broken-line chi2 (measurements plus kinks).  A
 * track whose reference is not finite, has |kappa| < 1e-7 /cm or whose hits are not
 * strictly ordered along the reference circle keeps its fit.  Run after pt_fit_tracks
 * (or a batch graph) on the same batch; pt_find_vertices must run again afterwards to
 * use the refitted tracks.  n_tracks as above.  Errors: PT_ERR_INVALID for no fitted
 * batch or material outside (0, 1]. */
pt_status pt_refit_broken_line(pt_ctx* ctx, float x0_barrel, float x0_disk, int64_t* n_tracks);

/* -------------------------------------------------------------------- results */

/* Cleaned ntuplets of the batch, events in order, canonical order within an event.
 * hits: [cap][6] int32 input indices within the event, -1 padded; nhits: [cap]
 * (either may be NULL); event_offsets: [n_events + 1] int64 (may be NULL), the
 * ntuplets of event e are [event_offsets[e], event_offsets[e+1]).  *n = total count.
 * PT_ERR_CAPACITY if cap < total (nothing written).  Synchronises the stream. */
pt_status pt_get_ntuplets(pt_ctx* ctx, int32_t* hits, uint8_t* nhits, int64_t* event_offsets,
                          int64_t cap, int64_t* n, int on_device);

/* Fitted tracks, one per cleaned ntuplet, same order.  Synchronises the stream. */
pt_status pt_get_tracks(pt_ctx* ctx, pt_track* tracks, int64_t cap, int64_t* n, int on_device);

/* Primary vertices of the fitted tracks (Sec. 2.2.1: vertex reconstruction is the last
 * of the chain's sub-algorithms, and Fig. 2 has the chain hand back both tracks and
 * vertices; the paper gives no algorithm).  Per event: the tracks with at least
 * min_hits hits (3..6; 4 keeps quadruplets and longer) and a finite z0 are ordered by
 * z0 (ties: canonical track order) and the list is cut wherever the float32 step to
 * the next z0 exceeds dz (cm, > 0; a step of exactly dz does not cut); every group of
 * two or more tracks is a vertex with z = mean z0.  Run after pt_fit_tracks on the same
 * batch.  n_vertices: NULL to stay asynchronous, else the call synchronises and stores
 * the number of vertices.  Errors: PT_ERR_INVALID for bad arguments or no fitted batch;
 * PT_ERR_CAPACITY when an event has more than 16384 such tracks. */
pt_status pt_find_vertices(pt_ctx* ctx, int min_hits, float dz, int64_t* n_vertices);

/* Vertices of the last pt_find_vertices, events in order, z ascending within an
 * event.  vertices: [cap] (may be NULL); event_offsets: [n_events + 1] int64 (may be
 * NULL), the vertices of event e are [event_offsets[e], event_offsets[e+1]);
 * track_vertex: [n_tracks] int32 (may be NULL), the vertex (index into the batch's
 * vertex list) of each fitted track in pt_get_tracks order, -1 for none.  *n = total
 * count; PT_ERR_CAPACITY if cap < *n (nothing written).  Synchronises the stream. */
pt_status pt_get_vertices(pt_ctx* ctx, pt_vertex* vertices, int64_t* event_offsets,
                          int32_t* track_vertex, int64_t cap, int64_t* n, int on_device);

/* Intermediate products, for validation.  Cells as (inner, outer) input-index pairs;
 * links as (h0, h1, h2) input-index triples with their quality q; ntuplets before
 * cleaning as [6] hit tuples with hit count and q.  Event e's entries carry the event
 * index in `event` (NULL allowed).  Order is unspecified.  Synchronise the stream. */
pt_status pt_get_cells(pt_ctx* ctx, int32_t* inner, int32_t* outer, int32_t* event, int64_t cap,
                       int64_t* n);
pt_status pt_get_links(pt_ctx* ctx, int32_t* h0, int32_t* h1, int32_t* h2, float* q,
                       int32_t* event, int64_t cap, int64_t* n);
pt_status pt_get_candidates(pt_ctx* ctx, int32_t* hits, uint8_t* nhits, float* q, int32_t* event,
                            int64_t cap, int64_t* n);

/* ------------------------------------------------------------- learned gate */

/* Learned link gate: an MLP 12 -> 64 -> 64 -> 1 (ReLU) scores every accepted cell link
 * from 12 geometric features and links scoring below tau are removed before the ntuplet
 * search; the exact cuts stay in force.  It is the library's analogue of the paper's
 * edge-filtering MLP (Sec. 2.2.2: an MLP scores graph edges, a fixed threshold drops
 * clearly fake ones).  Features of link (h0, h1, h2): C1, C2, C3 cut ratios,
 * t_a/cotmax, 10 (t_b - t_a), r0/16, r1/16, r2/16, (z0 - r0 t_a)/z0max, layer0/9,
 * layer1/9, layer2/9 (t = dz/dr of a cell).  Inference runs on the tensor cores with
 * bf16 weights, features and hidden activations and float32 accumulation.
 *
 * w: host array of 5057 float32 parameters, row-major W1[64][12], b1[64], W2[64][64],
 * b2[64], w3[64], b3; W1 and W2 are rounded to bf16 (nearest even) on upload, the rest
 * stays float32.  tau: threshold on the score (logit).  w == NULL switches the gate off.
 * Synchronises the stream; the next pt_reconstruct_batch re-captures its graph. */
pt_status pt_set_gate(pt_ctx* ctx, const float* w, float tau);

/* Current links with their float32 features [n][12], hits (event-local input indices),
 * event and gate score (NaN when the gate is off); host outputs, any may be NULL.  With
 * the gate on only the kept links are listed.  Synchronises the stream. */
pt_status pt_get_link_features(pt_ctx* ctx, float* feat, int32_t* h0, int32_t* h1, int32_t* h2,
                               int32_t* event, float* score, int64_t cap, int64_t* n);

/* Scores of n feature rows with the context's gate (tensor-core path): feat device
 * float32 [n][12], out device float32 [n]; n <= max_links.  Synchronises the stream. */
pt_status pt_gate_score(pt_ctx* ctx, const float* feat, int64_t n, float* out);

/* Training (Sec. 2.2.2 models are trained; here the gate is trained on the GPU): mean
 * binary cross-entropy of sigmoid(score) against labels y in {0, 1} and its gradient
 * with respect to the 5057 float32 parameters w.  All pointers are device pointers on
 * the current device: w [5057], x [n][12], y [n], grad [5057] (overwritten), loss [1]
 * (overwritten).  Asynchronous on `stream` (NULL: default stream). */
pt_status pt_gate_loss_grad(const float* w, const float* x, const float* y, int64_t n,
                            float* grad, float* loss, void* stream);

/* One Adam step (bias-corrected, step >= 1) on n float32 parameters: device pointers w,
 * first and second moment m and v (updated in place) and grad.  Asynchronous. */
pt_status pt_gate_adam(float* w, float* m, float* v, const float* grad, int64_t n, float lr,
                       float beta1, float beta2, float eps, int step, void* stream);

/* ------------------------------------------------------------- whole batch */

/* Load, doublets, links, ntuplets, fit and copy-out of a batch in one call; the GPU
 * stages run as one CUDA graph (captured on first use).  in_on_device applies to
 * x/y/z/layer, out_on_device to the outputs.  Outputs as in pt_get_ntuplets /
 * pt_get_tracks (hits, nhits, tracks may be NULL); event_offsets [n_events+1] required.
 * Synchronises the stream. */
pt_status pt_reconstruct_batch(pt_ctx* ctx, int n_events, const int64_t* hit_offsets,
                               const float* x, const float* y, const float* z,
                               const uint8_t* layer, int in_on_device, int32_t* hits_out,
                               uint8_t* nhits_out, pt_track* tracks_out,
                               int64_t* event_offsets, int64_t cap, int64_t* n,
                               int out_on_device);

/* Load a batch and enqueue all GPU stages (doublets, links, ntuplets, fit, export) as
 * one CUDA graph on the context's stream, without synchronising: results stay on the
 * device until a getter (pt_get_ntuplets, pt_get_tracks, ...) is called.  Input
 * validation errors are returned immediately; capacity errors by the next getter. */
pt_status pt_enqueue_batch(pt_ctx* ctx, int n_events, const int64_t* hit_offsets,
                           const float* x, const float* y, const float* z, const uint8_t* layer,
                           int on_device);

/* Doublets of one event without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory -- code whose
 * process hands all device memory to another allocator (a framework's caching pool
 * that has reserved the GPU), or real-time loops that must not allocate after start-up
 * -- and so cannot create a context.  Its scratch is a fixed array of about 2.4 MB
 * compiled into the library, which every GPU that loads the library keeps until the
 * process exits.
 *   n <= 65536 hits, else PT_ERR_CAPACITY with no GPU work.  x, y, z (float32) and
 *   layer (uint8): device pointers on the current device.  inner/outer: device arrays
 *   of cap int32 entries receiving each accepted doublet as input hit indices (inner,
 *   outer), in no particular order; the set equals the cells of pt_build_doublets with
 *   the same cuts.  *n_out (host) receives the number of doublets; if it exceeds cap the
 *   call returns PT_ERR_CAPACITY and only cap of them were written (which ones is
 *   unspecified).  A layer code > 9 gives PT_ERR_INVALID.
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * Every call looks up the scratch array's device address on the current device (the
 * first lookup on a device loads the library's device code there; later ones allocate
 * nothing), so the address stays right if the device's context is reset and made
 * again; make the first call on a device before any stream capture.  All calls share the one array and each call clears what it reads as zero:
 * calls whose GPU work overlaps (other threads, other streams) race and must not be
 * issued concurrently.  No cudaMalloc, cudaFree or other allocating call is made. */
pt_status pt_find_doublets_noalloc(const pt_cuts* cuts, int64_t n, const float* x,
                                   const float* y, const float* z, const uint8_t* layer,
                                   int32_t* inner, int32_t* outer, int64_t cap, int64_t* n_out,
                                   void* stream);

/* ------------------------------------------------------------------ tracing */

/* Total device time of one kernel (or of one prefix-sum helper, "scan") over the
 * launches traced since the last pt_get_trace. */
typedef struct {
  char name[48];     /* kernel name, NUL terminated */
  double total_ms;   /* sum of CUDA-event durations */
  int64_t launches;  /* number of traced launches */
} pt_kernel_time;

/* Per-kernel timing of the stage calls (on = 1) or none (on = 0, the default): every
 * kernel launched by pt_load_*, pt_build_doublets, pt_connect_cells, pt_find_ntuplets,
 * pt_fit_tracks and the getters is bracketed by CUDA events on the context's stream.
 * The whole-batch graph (pt_reconstruct_batch, pt_enqueue_batch) is never traced.
 * Synchronises the stream; switching off discards what was not read. */
pt_status pt_set_tracing(pt_ctx* ctx, int on);

/* Synchronises the stream and returns the per-kernel totals since the last call, in
 * the order the kernels first ran; *n receives their number.  PT_ERR_INVALID when
 * tracing is off, PT_ERR_CAPACITY when cap < *n (the totals are kept). */
pt_status pt_get_trace(pt_ctx* ctx, pt_kernel_time* out, int cap, int* n);

/* ------------------------------------------------------------------ tuning */

/* Launch sizes of the persistent grid-stride kernels, in blocks per multiprocessor
 * (each 1..32): blocks_per_sm for the 256-thread bookkeeping kernels (clear, binning,
 * scans, ntuplet walk, dedup, fit, export; default 4) and search_blocks_per_sm for the
 * warp-per-hit doublet search (default 5, its residency limit); the link search always
 * runs 4 blocks of 8 warps per multiprocessor, its residency limit.  Any value gives
 * the same results.  Synchronises the stream; the next whole-batch call
 * re-captures its graph. */
pt_status pt_set_launch(pt_ctx* ctx, int blocks_per_sm, int search_blocks_per_sm);

/* Layer pairs on which doublets are made (Sec. 2.2.1 and Fig. 2: hits of adjacent layers
 * are paired; the paper lists no pairs).  A context starts with the chain's 13 pairs:
 * barrel 0-1, 1-2, 2-3 and, per side, 0/1/2-4, 4-5, 5-6 and 0/1/2-7, 7-8, 8-9 (layer
 * codes as in pt_load_hits).  inner[i], outer[i] (host arrays of n_pairs int32) replace
 * them, e.g. with skip-layer pairs added so that a track that missed a layer still gives
 * a chain; n_pairs = 0 restores the default.  Every other step of the chain is unchanged
 * (the same cuts on every pair, maximal chains of 3..6 hits, the same cleaning).
 * PT_ERR_INVALID unless 1 <= n_pairs <= 64, every code is 0..9, inner != outer, no pair
 * repeats, no layer has more than 6 outer or 6 inner layers, and the pairs form no cycle
 * and no chain of more than 5 pairs (an ntuplet holds 6 hits).  Synchronises the stream;
 * the next whole-batch call re-captures its graph. */
pt_status pt_set_layer_pairs(pt_ctx* ctx, int n_pairs, const int32_t* inner, const int32_t* outer);

/* Fishbone duplicate removal, off by default.  The paper does not describe this step;
 * this is the library's reading of the overlap cleaning of the Patatrack chain
 * (Sec. 2.2.1 names the chain's steps).  A track crossing two overlapping sensors of
 * one layer leaves two hits there, and its cells from both to the next hit point the
 * same way.  After the links (and the learned gate, when set), cells with at least one
 * outgoing link that end on the same hit are compared two by two when their inner hits
 * lie on different layers or on different sensors of one layer (r, barrel layers 0..3,
 * or |z|, disks, more than 0.1 cm apart, as float32 r = sqrt(x x + y y) and |z|; the
 * stand-in for a sensor identity, which the hit input does not carry): with u, v the
 * float32 vectors from each cell's inner hit to the common outer hit, a pair is aligned when
 * u.v > 0 and (u.v)^2 >= 0.99999 |u|^2 |v|^2 (evaluated as
 * ((ux vx + uy vy) + uz vz)^2 >= 0.99999 (|u|^2 |v|^2), each |.|^2 as (x x + y y) + z z,
 * correctly rounded, no FMA).  Of an aligned pair on the same inner layer the shorter
 * cell loses, on different inner layers the longer one; at equal lengths the cell whose
 * inner hit has the larger input index loses.  Every cell that loses to some aligned
 * partner is removed with all its links before the ntuplet search; the link counts and
 * link exports then list the remaining links.  on: 0 off, 1 on; PT_ERR_INVALID
 * otherwise.  Synchronises the stream; the next whole-batch call re-captures its
 * graph. */
pt_status pt_set_fishbone(pt_ctx* ctx, int on);

/* 1 when this library is the debug build (libptca_debug.so, compiled with PT_DEBUG):
 * its kernels check the indexes of their main array accesses against the sizes they
 * hold, and a failing check sets a status bit and skips the access; the next call that
 * reads the device counters then returns PT_ERR_INTERNAL naming the first failing
 * check.  0 for the normal build, whose kernels carry no checks.  Touches no GPU. */
int pt_debug_build(void);

/* Debug build only: records a failure of bounds check `site` (1..13) on the context's
 * stream the way a failing check does, touching no array, so that the reporting path can
 * be tested: the next call that reads the device counters returns PT_ERR_INTERNAL
 * naming the site, until the next pt_load_hits / pt_load_batch clears the status.
 * PT_ERR_INVALID in the normal build, for a NULL context or a site out of range. */
pt_status pt_debug_inject(pt_ctx* ctx, int site);

/* Limit, in SM clock cycles (>= 1; default 2^31, about 1 s at 2 GHz), of the context's
 * bounded device-side waits: the learned gate's waits for its tensor-core results
 * (pt_connect_cells in the gated form, pt_gate_score, the whole-batch graph).  A wait that
 * runs out ends the kernel's work with a status bit, which the next synchronising call
 * reports as PT_ERR_TIMEOUT; the context stays usable.  The paper has no counterpart:
 * this bounds how long a kernel of the library can hold a GPU (a small limit is also how
 * the timeout path is tested).  When a wait gives up, the kernel still lets the matrix
 * multiplication in flight finish (waiting up to the default limit) before it frees
 * its tensor memory.  Synchronises the stream; the next whole-batch call re-captures
 * its graph. */
pt_status pt_set_wait_limit(pt_ctx* ctx, int64_t cycles);

/* Autotuner for the batched chain.  For every candidate azimuthal bin count
 * phi_bins[i] (context capacity otherwise as `cap`) it creates a context on `device`,
 * copies the caller's sample batch (HOST arrays, pt_load_batch layout) to it once, and
 * for every pair (blocks_per_sm[jb], search_blocks_per_sm[js]) of pt_set_launch sizes
 * launches the whole chain (the pt_enqueue_batch graph, plain form) once to warm up
 * and `reps` more times, timing each launch with CUDA events on the context's stream.  best[3] receives the
 * combination with the smallest median (phi_bins, blocks_per_sm, search_blocks_per_sm);
 * results (optional, n_phi * n_bps * n_sbps floats, index (i * n_bps + jb) * n_sbps + js)
 * each median in ms.  Every combination gives the same ntuplets: the binning and the
 * launch sizes only change how the work is spread.  Errors: PT_ERR_INVALID for empty
 * candidate lists or reps < 1, and any error of pt_create or of the batch itself. */
pt_status pt_autotune(const pt_geometry* geom, const pt_cuts* cuts, const pt_capacity* cap,
                      int device, int n_events, const int64_t* hit_offsets, const float* x,
                      const float* y, const float* z, const uint8_t* layer,
                      const int32_t* phi_bins, int n_phi, const int32_t* blocks_per_sm,
                      int n_bps, const int32_t* search_blocks_per_sm, int n_sbps, int reps,
                      int32_t* best, float* results);

/* ------------------------------------------------------------------ serving */

/* In-process request server: the as-a-service pattern of the paper (Sec. 1 Fig. 1 and
 * Sec. 3: clients send events, the server batches requests, runs them on the GPU and
 * returns the results; several requests are in flight at once, Sec. 3.2/4.2), without
 * network or inference server.  Continuous batching: the device budget is split into
 * max_slots slots (contexts with their own stream and workspace); a dispatcher thread
 * fills every free slot with the longest prefix of the FIFO of submitted events that
 * fits it (event count, hits, estimated cells ~ 1.6e-3 * hits^2), runs the whole chain
 * for it as one CUDA graph, and returns each event's ntuplets and tracks to its ticket.
 * Slots run concurrently; a batch that overflows its slot is re-run event by event.
 * Results are identical to running each event alone.  All functions are thread-safe. */
typedef struct pt_server pt_server;

/* device_budget_bytes: device memory the server may use for its workspaces (each slot
 * gets budget / max_slots); PT_ERR_NOMEM if one PU200-sized event does not fit a slot. */
pt_status pt_server_create(const pt_geometry* geom, const pt_cuts* cuts, int device,
                           size_t device_budget_bytes, int max_slots, pt_server** out);

/* Learned gate for all slots (pt_set_gate semantics); waits until no batch runs. */
pt_status pt_server_set_gate(pt_server* s, const float* w, float tau);

/* Queue one event (host arrays, copied before returning; never waits for the GPU).
 * PT_ERR_CAPACITY if the event cannot fit a slot, PT_ERR_INVALID for bad input. */
pt_status pt_submit(pt_server* s, int64_t n, const float* x, const float* y, const float* z,
                    const uint8_t* layer, uint64_t* ticket);

/* Result of a ticket: waits up to timeout_us (0: no wait -> PT_ERR_NOT_READY; < 0:
 * wait indefinitely; else PT_ERR_TIMEOUT when it expires).  On success the ticket is
 * released and hits [cap][6] / nhits [cap] / tracks [cap] (host, any may be NULL)
 * receive the event's cleaned ntuplets (canonical order) and tracks; *n their number.
 * PT_ERR_CAPACITY (ticket kept, *n set) if cap is too small. */
pt_status pt_poll(pt_server* s, uint64_t ticket, int64_t timeout_us, int32_t* hits,
                  uint8_t* nhits, pt_track* tracks, int64_t cap, int64_t* n);

/* Submit-to-ready latency percentiles (ms) and sustained events/s (completed events over
 * the time from the first submit to the last completion) since creation or reset. */
pt_status pt_server_stats(pt_server* s, double* p50_ms, double* p99_ms, double* events_per_s,
                          int64_t* n_done);

/* Batching counters since the server started or since pt_server_reset_stats: batches
 * launched, batches whose cells overflowed their slot (the cell estimate of the
 * admission was short) and were split, and the events those splits ran again alone
 * (each such event pays for two launches).  Any pointer may be NULL.  The paper has no
 * counterpart; it explains slow requests in the latency tail. */
pt_status pt_server_counters(pt_server* server, int64_t* batches, int64_t* split_batches,
                             int64_t* requeued_events);

/* Router over several server instances (Sec. 3.2, Sec. 4.2: the inference server
 * balances requests over several instances of the model, on one GPU or on several).
 * Instance i is a pt_server on devices[i] (host array of n_instances device ordinals,
 * 1..255 instances) with its own dispatcher thread, budget_per_instance bytes and
 * slots_per_instance slots.  A submission goes to the instance with the fewest requests
 * submitted and not yet completed on the device; the returned ticket names the
 * instance.  Submit and poll behave as pt_submit and pt_poll; the gate, statistics and
 * reset apply to every instance (p50: the instances' medians weighted by their
 * requests; p99: the largest instance p99; events_per_s: the sum; per_instance_done
 * (NULL or n_instances int64) receives each instance's completed requests).
 * Thread-safe. */
typedef struct pt_router pt_router;
pt_status pt_router_create(const pt_geometry* geom, const pt_cuts* cuts, const int* devices,
                           int n_instances, size_t budget_per_instance, int slots_per_instance,
                           pt_router** out);
pt_status pt_router_set_gate(pt_router* router, const float* w, float tau);
pt_status pt_router_submit(pt_router* router, int64_t n, const float* x, const float* y,
                           const float* z, const uint8_t* layer, uint64_t* ticket);
pt_status pt_router_poll(pt_router* router, uint64_t ticket, int64_t timeout_us, int32_t* hits,
                         uint8_t* nhits, pt_track* tracks, int64_t cap, int64_t* n);
pt_status pt_router_stats(pt_router* router, double* p50_ms, double* p99_ms,
                          double* events_per_s, int64_t* n_done, int64_t* per_instance_done);
pt_status pt_router_reset_stats(pt_router* router);
pt_status pt_router_destroy(pt_router* router);
pt_status pt_server_reset_stats(pt_server* s);

/* Stop accepting work, finish what is queued, free everything.  NULL ok. */
pt_status pt_server_destroy(pt_server* s);

/* Message for the last failed call on this thread ("" if none). */
const char* pt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PT_CA_H */
