// Broken-line refit of the fitted tracks (declared apart from the chain's internal
// header: the refit is an optional stage after the circle + line fit).
#pragma once

#include "ptca_internal.cuh"

namespace ptca {

// Passes of the broken-line refit over the cleaned tracks (b.tracks[0, cnt[CNT_SV]),
// replaced in place); x0_barrel and x0_disk are the layers' material in radiation
// lengths at normal incidence (> 0).  Scratch: list holds 2 x max_ntuplets track
// indices and counters kRefitCounters values.
constexpr int kRefitCounters = 4;
cudaError_t launch_refit_broken_line(const Buffers& b, const Params& p, float x0_barrel,
                                     float x0_disk, uint32_t* list, unsigned long long* counters,
                                     const Launch& l, cudaStream_t s);

}  // namespace ptca
