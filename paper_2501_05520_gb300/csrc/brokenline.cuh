// Broken-line refit of the fitted tracks (declared apart from the chain's internal
// header: the refit is an optional stage after the circle + line fit).
#pragma once

#include "ptca_internal.cuh"

namespace ptca {

// Replaces b.tracks[0, cnt[CNT_SV]) by their broken-line refits; x0_barrel and
// x0_disk are the layers' material in radiation lengths at normal incidence (> 0).
void launch_refit_broken_line(const Buffers& b, const Params& p, float x0_barrel, float x0_disk,
                              const Launch& l, cudaStream_t s);

}  // namespace ptca
