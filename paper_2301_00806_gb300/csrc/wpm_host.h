// wpm_host.h -- host-side helpers shared by the runtime (wpm_runtime.cpp) and the serving
// engine (wpm_engine.cpp) of libwpm: error reporting, device/pinned buffers, and the copied,
// checked form of a caller's instance. Not part of the public ABI.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_internal.h"

namespace wpm {

// Record the calling thread's last error (printf-style) and return `code`.
int fail(int code, const char *fmt, ...);

#define CUDA_TRY(x)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess)                                                            \
      return ::wpm::fail(WPM_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_));  \
  } while (0)

#define WPM_TRY(x)                \
  do {                            \
    int r_ = (x);                 \
    if (r_ != WPM_OK) return r_;  \
  } while (0)

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap && p) return WPM_OK;
    release();
    size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(WPM_ERR_NOMEM, "cudaMalloc(%zu bytes) failed", want);
    }
    cap = want;
    return WPM_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

struct PinBuf {
  void *p = nullptr;
  size_t cap = 0;
  int ensure(size_t bytes) {
    if (bytes <= cap && p) return WPM_OK;
    release();
    size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    if (cudaMallocHost(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return fail(WPM_ERR_NOMEM, "cudaMallocHost(%zu bytes) failed", want);
    }
    cap = want;
    return WPM_OK;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// An instance as the caller gave it, copied and checked.
struct HostInst {
  int kind = 0, n = 0, m = 0;
  uint32_t cols[kMaxVertices] = {0};
  std::vector<uint16_t> given;
  int cap_req = -1, base_req = 0, n_facets_req = -1, n_aff = 0, post = 0;
  std::vector<uint64_t> fin, fout;
  std::vector<int32_t> c0, coef;
};

int copy_conditions(const wpm_conditions *c, HostInst &h);
int copy_map(const uint32_t *cols, int kind, int n, int m, HostInst &h);
int copy_facet_list(const uint16_t *facets, int M, int n, int m, HostInst &h);

}  // namespace wpm
