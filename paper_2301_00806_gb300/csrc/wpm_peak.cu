// wpm_peak.cu -- integer throughput of the GPU, measured, for the roofline of the search
// kernels (which are bound by integer and logic instructions, not by memory).
//
// Each thread runs kChains independent dependency chains, so every scheduler always has
// ready instructions; the instructions are written as PTX so that the compiler can neither
// fold a chain into a closed form nor drop it. Two streams: logic and add (one lop3 and one
// add per chain per step, the mix of the search's counter and bitset updates) and popc.
// The grid is a multiple of the SM count (four 512-thread blocks per SM). Timed with CUDA
// events around one launch after a warm-up launch.
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_internal.h"

namespace wpm {

constexpr int kChains = 8;

__global__ void __launch_bounds__(512) int_peak_kernel(uint32_t *sink, int iters, int op,
                                                       uint32_t seed) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) a[c] = seed ^ (t * 2654435761u + c);
  const uint32_t b = seed * 40503u + t, d = ~seed ^ (t << 7);
  if (op == 0) {
    for (int i = 0; i < iters; i++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));
        asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(b));
      }
    }
  } else {
    for (int i = 0; i < iters; i++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        uint32_t p;
        asm volatile("popc.b32 %0, %1;" : "=r"(p) : "r"(a[c]));
        asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[c]) : "r"(p));
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) x ^= a[c];
  if (x == 0x9E3779B9u) sink[t & 1023] = x;  // keeps the chains alive; almost never stored
}

}  // namespace wpm

using namespace wpm;

extern "C" int wpm_int_peak(int op, int iters, double *ops_per_sec, double *ms_out) {
  clear_last_error();
  if ((op != 0 && op != 1) || iters <= 0 || !ops_per_sec)
    return set_last_error(WPM_ERR_INPUT, "op must be 0 or 1, iters > 0, ops_per_sec non-NULL");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
  const int blocks = 4 * sms, threads = 512;
  uint32_t *sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  e = cudaMalloc(&sink, 4096);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    int_peak_kernel<<<blocks, threads, 0, s>>>(sink, iters / 4 + 1, op, 12345u);  // warm-up
    cudaEventRecord(e0, s);
    int_peak_kernel<<<blocks, threads, 0, s>>>(sink, iters, op, 67890u);
    cudaEventRecord(e1, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return set_last_error(WPM_ERR_CUDA, cudaGetErrorString(e));
  // two instructions per chain per step (lop3 + add, or popc + xor)
  const double ops = 2.0 * kChains * (double)iters * blocks * threads;
  *ops_per_sec = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return WPM_OK;
}
