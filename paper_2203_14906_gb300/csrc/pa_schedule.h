// pa_schedule.h -- host-path chunk schedules (host logic, not part of the
// public ABI beyond pa_pipe_time / pa_pipe_schedule).
#pragma once

#include <stdint.h>

#include <vector>

#include "pa_hodmas.h"

namespace pa {

// Makespan (us) of a chunk schedule under the host-path pipeline model, and
// the best schedule of the searched family (chunks of at most cap frames).
double pipe_makespan(const pa_pipe_model& m, const int32_t* chunks, int n);
std::vector<int32_t> pipe_search(const pa_pipe_model& m, int n_frames, int cap);

}  // namespace pa
