// wpm_class.cu -- one kernel size class of the search, selected by -DWPM_CLASS_ID=k at
// compile time (the build compiles this file once per class, in parallel).
#include "wpm_classes.h"
#include "wpm_search.cuh"

#ifndef WPM_CLASS_ID
#error "compile with -DWPM_CLASS_ID=<k>"
#endif

namespace wpm {

#define X(id, mw, nw)                                                                       \
  cudaError_t class_launch_##id(int mode, const PassArgs &a, int grid, int n_items, int tpb, \
                                size_t smem, cudaStream_t s) {                             \
    return launch_t<mw, nw>(mode, a, grid, n_items, tpb, smem, s);                         \
  }                                                                                         \
  int class_occupancy_##id(int tpb, size_t smem) { return occupancy_t<mw, nw>(tpb, smem); } \
  static_assert(Cls<mw, nw>::SMW == ((nw + 2 * mw + 1) & ~1) + 4 * kMaxAffine,            \
                "state_words() in wpm_kernels.cu must match Cls::SMW");
WPM_ONE_CLASS(X, WPM_CLASS_ID)
#undef X

}  // namespace wpm
