// wpm_class.cu -- one kernel size class of the search kernels (per-thread and per-warp),
// selected by -DWPM_CLASS_ID=k at compile time (the build compiles this file once per class,
// in parallel).
#include "wpm_classes.h"
#include "wpm_tsearch.cuh"
#include "wpm_wsearch.cuh"

#ifndef WPM_CLASS_ID
#error "compile with -DWPM_CLASS_ID=<k>"
#endif

namespace wpm {

#define X(id, mw, nw)                                                                       \
  cudaError_t class_launch_##id(int mode, const PassArgs &a, int grid, int n_items, int tpb, \
                                size_t smem, cudaStream_t s) {                             \
    if (mode != 2) return wlaunch_t<mw, nw>(mode, a, grid, n_items, tpb, smem, s);          \
    if (tpb == 128 && a.rows == 1) return tlaunch_t<mw, nw, 128, 1>(a, grid, smem, s);      \
    if (tpb == 128 && a.rows == 2) return tlaunch_t<mw, nw, 128, 2>(a, grid, smem, s);      \
    if (tpb == 128 && a.rows == 3) return tlaunch_t<mw, nw, 128, 3>(a, grid, smem, s);      \
    if (tpb == 64) return tlaunch_t<mw, nw, 64>(a, grid, smem, s);                          \
    if (tpb == 128) return tlaunch_t<mw, nw, 128>(a, grid, smem, s);                        \
    return tlaunch_t<mw, nw, 256>(a, grid, smem, s);                                        \
  }                                                                                         \
  int class_occupancy_##id(int mode, int tpb, size_t smem) {                                \
    if (mode != 2) return woccupancy_t<mw, nw>(tpb, smem);                                  \
    if (tpb == 64) return toccupancy_t<mw, nw, 64>(smem);                                   \
    if (tpb == 128) return toccupancy_t<mw, nw, 128>(smem);                                 \
    return toccupancy_t<mw, nw, 256>(smem);                                                 \
  }                                                                                         \
  static_assert(WCls<mw, nw>::SMW == ((nw + 2 * mw + 1) & ~1) + 4 * kMaxAffine,           \
                "state_words() in wpm_kernels.cu must match WCls::SMW");                   \
  static_assert(ts::TCls<mw, nw, 64>::SMW == nw + 2 * mw + (nw <= 96 ? 0 : (nw + 31) / 32), \
                "tstate_words() in wpm_kernels.cu must match TCls::SMW");
WPM_ONE_CLASS(X, WPM_CLASS_ID)
#undef X

}  // namespace wpm
