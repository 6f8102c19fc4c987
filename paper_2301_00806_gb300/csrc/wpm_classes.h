// wpm_classes.h -- the kernel size classes: compile-time maxima of the u32 words of a
// facet bitset (mw) and of the packed 2-bit ridge counters (nw). Picard number 4 needs,
// per n: n<=3 (1,2), n<=5 (3,8), 6 (5,15), 7 (7,27), 8 (10,45), 9 (14,72), 10 (20,112),
// 11 (27,168); the last class holds the library limits (M <= 2048, N <= 4096).
#pragma once

#define WPM_CLASSES(X) \
  X(0, 1, 2)           \
  X(1, 3, 8)           \
  X(2, 5, 16)          \
  X(3, 7, 28)          \
  X(4, 10, 48)         \
  X(5, 14, 72)         \
  X(6, 20, 112)        \
  X(7, 27, 168)        \
  X(8, 64, 256)

#define WPM_N_CLASSES 9

// Expand X for class `k` only.
#define WPM_ONE_CLASS(X, k) WPM_ONE_CLASS_(X, k)
#define WPM_ONE_CLASS_(X, k) WPM_CLASS_##k(X)
#define WPM_CLASS_0(X) X(0, 1, 2)
#define WPM_CLASS_1(X) X(1, 3, 8)
#define WPM_CLASS_2(X) X(2, 5, 16)
#define WPM_CLASS_3(X) X(3, 7, 28)
#define WPM_CLASS_4(X) X(4, 10, 48)
#define WPM_CLASS_5(X) X(5, 14, 72)
#define WPM_CLASS_6(X) X(6, 20, 112)
#define WPM_CLASS_7(X) X(7, 27, 168)
#define WPM_CLASS_8(X) X(8, 64, 256)

namespace wpm {
struct PassArgs;
// mode 0: warp expansion, 1: warp depth-first pass, 2: thread depth-first pass
#define X(id, mw, nw)                                                                       \
  cudaError_t class_launch_##id(int mode, const PassArgs &a, int grid, int n_items, int tpb, \
                                size_t smem, cudaStream_t s);                              \
  int class_occupancy_##id(int mode, int tpb, size_t smem);
WPM_CLASSES(X)
#undef X
}  // namespace wpm
