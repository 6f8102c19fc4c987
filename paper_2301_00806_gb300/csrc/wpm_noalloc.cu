// wpm_noalloc.cu -- wpm_candidate_facets_static: the candidate-facet computation with no
// device or host allocation, for callers that must not allocate.
//
// Some callers cannot let a library call cudaMalloc: a service that reserves its device
// memory once at start-up and must never grow it under load (an allocation can fail, or wait
// on other users of the GPU), or a host framework whose allocator owns all device memory.
// This entry point runs the same setup kernel as wpm_candidate_facets, but its scratch (the
// instance descriptor, the rank prefix sums and the incidence rows the kernel builds) lives
// in one file-scope __device__ array below, and its host side uses only stack variables.
//
// The call copies its result back to the host and synchronises its stream before it returns.
//
// Every GPU that loads the library holds that array (kStaticScratchBytes) until the process
// exits. All calls share it and it keeps the last call's contents; the kernel writes every
// word it later reads, so nothing has to be cleared between calls. Calls whose work overlaps
// on the GPU (two host threads, or two streams without ordering between them) race on the
// array: callers must serialise them.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_internal.h"

namespace wpm {

// Room for one instance's descriptor and setup tables. A map needs, rounded up to 256 bytes
// per table, 38 bytes per facet rank and 36 per ridge rank: about 38 C(m,n) + 36 C(m,n-1)
// bytes plus 1.5 KB. 512 KiB covers every Picard-4 map (the largest, n = 11 on 15 vertices,
// needs about 170 KB) and, for example, n = 6 on 16 vertices (about 463 KB, 12,376 ranks);
// n = 7 on 16 vertices (about 725 KB) is rejected.
constexpr size_t kStaticScratchBytes = 512u * 1024u;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, looked up once with that device current.
constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_static_mu;

static size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

static long long binom_s(int a, int b) {
  if (b < 0 || b > a) return 0;
  long long r = 1;
  for (int i = 0; i < b; i++) r = r * (a - i) / (i + 1);
  return r;
}

}  // namespace wpm

using namespace wpm;

extern "C" int wpm_candidate_facets_static(const uint32_t *lambda_cols, int kind, int n, int m,
                                           uint16_t *facets_out, int cap, void *cuda_stream) {
  std::lock_guard<std::mutex> g(g_static_mu);
  clear_last_error();
  if (kind != WPM_LAMBDA_PRIMAL && kind != WPM_LAMBDA_DUAL)
    return set_last_error(WPM_ERR_INPUT, "kind is neither primal nor dual");
  if (n < 2 || m <= n || m > WPM_MAX_VERTICES)
    return set_last_error(WPM_ERR_INPUT, "need 2 <= n < m <= 16");
  if (!lambda_cols) return set_last_error(WPM_ERR_INPUT, "lambda_cols is NULL");
  const int bits = kind == WPM_LAMBDA_PRIMAL ? n : m - n;
  for (int i = 0; i < m; i++) {
    if (bits < 32 && (lambda_cols[i] >> bits))
      return set_last_error(WPM_ERR_INPUT, "a column has bits above the map's target space");
    if (kind == WPM_LAMBDA_DUAL) {
      if (lambda_cols[i] == 0) return set_last_error(WPM_ERR_INPUT, "a dual row is zero");
      for (int j = 0; j < i; j++)
        if (lambda_cols[i] == lambda_cols[j])
          return set_last_error(WPM_ERR_INPUT, "two dual rows repeat");
    }
  }

  // scratch layout: descriptor, facets, rank prefix sums, facet rows, ridge rows
  const size_t nsub = (size_t)binom_s(m, n), nrsub = (size_t)binom_s(m, n - 1);
  const size_t o_desc = 0;
  const size_t o_facets = o_desc + round256(sizeof(InstDesc));
  const size_t o_fprefix = o_facets + round256(2 * nsub);
  const size_t o_rprefix = o_fprefix + round256(4 * (nsub + 1));
  const size_t o_frw = o_rprefix + round256(4 * (nrsub + 1));
  const size_t o_prw = o_frw + round256(32 * nsub);
  const size_t need = o_prw + round256(32 * nrsub);
  if (need > kStaticScratchBytes)
    return set_last_error(WPM_ERR_LIMIT,
                          "this map needs more device scratch than the fixed static array "
                          "holds (C(m,n) + C(m,n-1) too large); use wpm_candidate_facets");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(WPM_ERR_LIMIT, "device index too large");
  if (!g_scratch_addr[dev]) {  // once per device, with that device current
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_addr[dev] = ptr;
  }
  char *base = static_cast<char *>(g_scratch_addr[dev]);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  InstDesc d;  // host copy on the stack
  memset(&d, 0, sizeof(d));
  d.kind = kind;
  d.n = n;
  d.m = m;
  d.mode = WPM_MODE_COUNT;
  for (int v = 0; v < m; v++) d.cols[v] = lambda_cols[v];
  d.cap_req = WPM_CAP_NONE;
  d.n_facets_req = -1;
  d.nsub = (int)nsub;
  d.nrsub = (int)nrsub;
  d.facets = reinterpret_cast<uint16_t *>(base + o_facets);
  d.fprefix = reinterpret_cast<int32_t *>(base + o_fprefix);
  d.rprefix = reinterpret_cast<int32_t *>(base + o_rprefix);
  d.frw = reinterpret_cast<uint16_t *>(base + o_frw);
  d.prw = reinterpret_cast<uint16_t *>(base + o_prw);
  InstDesc *dd = reinterpret_cast<InstDesc *>(base + o_desc);

  e = cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_setup(dd, 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&d, dd, sizeof(d), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
  if (d.err & kErrLimit) return set_last_error(WPM_ERR_LIMIT, "M or N above the library limits");
  if (d.M == 0)
    return set_last_error(WPM_ERR_INPUT, "the map has too small a rank (no candidate facet)");
  if (d.M > cap) return set_last_error(WPM_ERR_CAPACITY, "facets_out holds fewer than M entries");
  if (!facets_out) return set_last_error(WPM_ERR_INPUT, "facets_out is NULL");
  e = cudaMemcpyAsync(facets_out, base + o_facets, 2 * (size_t)d.M, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
  return d.M;
}
