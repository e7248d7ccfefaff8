// gmg_hw.h -- properties of the current device that size persistent grids.
#pragma once

namespace gmg {

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount),
// queried once per device and cached; 1 if the query fails.
int sm_count();

}  // namespace gmg
