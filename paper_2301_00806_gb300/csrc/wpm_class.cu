// wpm_class.cu -- one kernel size class of the search, selected by -DWPM_CLASS_ID=k at
// compile time (the build compiles this file once per class, in parallel).
#include "wpm_classes.h"
#include "wpm_search.cuh"

#ifndef WPM_CLASS_ID
#error "compile with -DWPM_CLASS_ID=<k>"
#endif

namespace wpm {

#define X(id, mw, nw)                                                                       \
  cudaError_t class_launch_##id(bool expand, const PassArgs &a, int grid, int n_items,     \
                                int tpb, cudaStream_t s) {                                 \
    if (tpb == 64) return launch_t<mw, nw, 64>(expand, a, grid, n_items, s);               \
    if (tpb == 128) return launch_t<mw, nw, 128>(expand, a, grid, n_items, s);             \
    return launch_t<mw, nw, 256>(expand, a, grid, n_items, s);                             \
  }                                                                                         \
  int class_occupancy_##id(int tpb) {                                                       \
    if (tpb == 64) return occupancy_t<mw, nw, 64>();                                        \
    if (tpb == 128) return occupancy_t<mw, nw, 128>();                                      \
    return occupancy_t<mw, nw, 256>();                                                      \
  }
WPM_ONE_CLASS(X, WPM_CLASS_ID)
#undef X

}  // namespace wpm
