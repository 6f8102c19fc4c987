// wpm_sweep.cu -- the GF(2) cycle-space sweep of libwpm (Section 2.1, Algorithm 2.2's
// kernel enumeration), an alternative to the canonical search for maps whose incidence
// matrix has a small kernel.
//
// Every WPM K satisfies A K = 0 over Z2 (each ridge lies in 0 or 2 facets of K), so K is a
// GF(2) combination of a basis of ker A. The sweep builds such a basis per map on the GPU
// (Gaussian elimination of A over GF(2) in shared memory, one block per map), then walks
// all 2^s combinations in Gray-code order: each thread takes a chunk of consecutive codes,
// builds the first combination, and from there flips one basis vector per step (the one
// at the lowest set bit of the step index), updating the ridge degrees of the facets it
// toggles. A combination is a WPM (Proposition 2.1) when no ridge has degree 4 (degrees
// are even inside the kernel); it is emitted when the properties hold as well. The emitted
// masks go through the same per-map sort as the search's, so lists are identical.
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {

// Rows of A over GF(2) (one per ridge, M bits) in shared memory; pivot columns and the
// resulting basis of ker A (kSweepW words per vector) in global memory.
__global__ void __launch_bounds__(256) kernel_basis_kernel(const InstDesc *insts, const int32_t *ids,
                                                           uint64_t *basis, int32_t *dims) {
  extern __shared__ uint64_t rows[];  // [N][kSweepW]
  __shared__ int piv_row;
  __shared__ int pivcol[kSweepMaxM];
  const InstDesc &I = insts[ids[blockIdx.x]];
  const int M = I.M, N = I.N, n = I.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int w = tid; w < N * kSweepW; w += nt) rows[w] = 0;
  __syncthreads();
  for (int j = tid; j < M; j += nt) {
    const uint16_t *fr = I.frw + (size_t)j * I.fstride;
    for (int k = 0; k < n; k++) {
      const int r = fr[k];
      atomicOr((unsigned long long *)&rows[r * kSweepW + (j >> 6)], 1ull << (j & 63));
    }
  }
  __syncthreads();
  // reduced row echelon form: for each column, a pivot row below the rank, swapped up,
  // cleared from every other row
  int rank = 0;
  for (int c = 0; c < M; c++) {
    if (tid == 0) piv_row = N;
    __syncthreads();
    const int w = c >> 6;
    const uint64_t bit = 1ull << (c & 63);
    for (int i = rank + tid; i < N; i += nt)
      if (rows[i * kSweepW + w] & bit) atomicMin(&piv_row, i);
    __syncthreads();
    const int p = piv_row;
    __syncthreads();       // every thread has read p before thread 0 resets it
    if (p == N) continue;  // a free column (uniform: every thread read the same p)
    if (p != rank && tid < kSweepW) {
      const uint64_t a = rows[p * kSweepW + tid];
      rows[p * kSweepW + tid] = rows[rank * kSweepW + tid];
      rows[rank * kSweepW + tid] = a;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
      if (i != rank && (rows[i * kSweepW + w] & bit)) {
        for (int x = 0; x < kSweepW; x++) rows[i * kSweepW + x] ^= rows[rank * kSweepW + x];
      }
    }
    if (tid == 0) pivcol[rank] = c;
    __syncthreads();
    rank++;
  }
  // one basis vector per free column f: bit f, and bit pivcol[i] for each pivot row i whose
  // row has bit f (so that A x = 0)
  uint64_t *B = basis + (size_t)blockIdx.x * kSweepMaxS * kSweepW;
  const int s = M - rank;
  if (tid == 0) dims[blockIdx.x] = s;
  if (s > kSweepMaxS) return;
  __syncthreads();
  if (tid == 0) {
    int j = 0, pi = 0;
    for (int f = 0; f < M; f++) {
      if (pi < rank && pivcol[pi] == f) {
        pi++;
        continue;
      }
      uint64_t v[kSweepW] = {};
      v[f >> 6] |= 1ull << (f & 63);
      for (int i = 0; i < rank; i++)
        if (rows[i * kSweepW + (f >> 6)] & (1ull << (f & 63)))
          v[pivcol[i] >> 6] |= 1ull << (pivcol[i] & 63);
      for (int x = 0; x < kSweepW; x++) B[j * kSweepW + x] = v[x];
      j++;
    }
  }
}

cudaError_t launch_kernel_basis(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                                int max_n_ridges, uint64_t *basis, int32_t *dims,
                                cudaStream_t s) {
  if (n_ids <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_n_ridges * kSweepW * 8;
  cudaError_t e = cudaFuncSetAttribute(kernel_basis_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel_basis_kernel<<<n_ids, 256, smem, s>>>(d_inst, d_ids, basis, dims);
  return cudaGetLastError();
}

// Ridge degrees of one thread: byte r of thread t at [r * TPB + t] (distinct banks per warp
// for any mix of ridges, four threads per bank word).
constexpr int kSweepTPB = 64;

__device__ __forceinline__ bool props_ok(const InstDesc &I, const uint64_t *K, int size) {
  if (I.cap >= 0 && size > I.cap) return false;
  if (I.base_req && (I.base_idx < 0 || !((K[I.base_idx >> 6] >> (I.base_idx & 63)) & 1ull)))
    return false;
  for (int w = 0; w < I.ow; w++) {
    if (I.fin && (K[w] & I.fin[w]) != I.fin[w]) return false;
    if (I.fout && (K[w] & I.fout[w])) return false;
  }
  for (int e = 0; e < I.n_aff; e++) {
    long long g = I.aff_c0[e];
    for (int w = 0; w < I.ow; w++) {
      uint64_t x = K[w];
      while (x) {
        const int j = w * 64 + __ffsll((long long)x) - 1;
        x &= x - 1;
        g += I.aff_coef[e * I.M + j];
      }
    }
    if (g <= 0) return false;
  }
  return true;
}

// chunks: exclusive prefix over the maps of their chunk counts (2^(s - clog) each, at least
// one); chunk c of map j covers Gray-code steps [c * 2^clog, (c + 1) * 2^clog) within 2^s.
__global__ void __launch_bounds__(kSweepTPB) sweep_kernel(const InstDesc *insts, const int32_t *ids,
                                                        int n_ids, const uint64_t *basis,
                                                        const int32_t *dims, const int32_t *clogs,
                                                        const unsigned long long *chunks,
                                                        const OutDesc *outs,
                                                        unsigned long long *ctr) {
  extern __shared__ uint8_t deg[];  // [N_max * kSweepTPB]
  const unsigned long long g = (unsigned long long)blockIdx.x * kSweepTPB + threadIdx.x;
  if (g >= chunks[n_ids]) return;
  // the map of this chunk: the last j with chunks[j] <= g
  int lo = 0, hi = n_ids - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunks[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  const int j = lo, id = ids[j];
  const InstDesc &I = insts[id];
  const int s = dims[j], clog = clogs[j], n = I.n, N = I.N;
  const uint64_t *B = basis + (size_t)j * kSweepMaxS * kSweepW;
  const unsigned long long first = (g - chunks[j]) << clog;
  const unsigned long long steps = 1ull << clog;
  uint8_t *d = deg + threadIdx.x;
  for (int r = 0; r < N; r++) d[r * kSweepTPB] = 0;
  // the combination of code gray(first)
  uint64_t K[kSweepW] = {};
  const unsigned long long code = first ^ (first >> 1);
  for (int b = 0; b < s; b++)
    if ((code >> b) & 1ull)
      for (int x = 0; x < kSweepW; x++) K[x] ^= B[b * kSweepW + x];
  int size = 0, bad = 0;
  for (int w = 0; w < kSweepW; w++) {
    uint64_t x = K[w];
    size += __popcll(x);
    while (x) {
      const int f = w * 64 + __ffsll((long long)x) - 1;
      x &= x - 1;
      const uint16_t *fr = I.frw + (size_t)f * I.fstride;
      for (int k = 0; k < n; k++) d[fr[k] * kSweepTPB]++;
    }
  }
  for (int r = 0; r < N; r++) bad += d[r * kSweepTPB] >= 4;
  unsigned long long count = 0;
  for (unsigned long long t = 0; t < steps; t++) {
    if (t > 0) {  // step first + t flips basis vector ctz(first + t)
      const int b = __ffsll((long long)(first + t)) - 1;
      for (int w = 0; w < kSweepW; w++) {
        uint64_t x = B[b * kSweepW + w];
        while (x) {
          const int f = w * 64 + __ffsll((long long)x) - 1;
          x &= x - 1;
          const bool in = (K[w] >> (f & 63)) & 1ull;
          K[w] ^= 1ull << (f & 63);
          size += in ? -1 : 1;
          const uint16_t *fr = I.frw + (size_t)f * I.fstride;
          for (int k = 0; k < n; k++) {
            uint8_t &v = d[fr[k] * kSweepTPB];
            if (in) {
              bad -= v == 4;
              v--;
            } else {
              v++;
              bad += v == 4;
            }
          }
        }
      }
    }
    if (bad || !props_ok(I, K, size)) continue;
    count++;
    if (I.mode == 0) {  // list mode: reserve a slot, write the mask
      const OutDesc &o = outs[id];
      const unsigned long long slot = atomicAdd(&ctr[kCtrN * id + kCtrFill], 1ull);
      if (slot < o.cap)
        for (int w = 0; w < I.ow; w++) o.out[slot * I.ow + w] = K[w];
    }
  }
  if (count) atomicAdd(&ctr[kCtrN * id + kCtrCount], count);
  atomicAdd(&ctr[kCtrN * id + kCtrNodes], steps);
  (void)s;
}

cudaError_t launch_sweep(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                         const uint64_t *basis, const int32_t *dims, const int32_t *clogs,
                         const unsigned long long *chunks, unsigned long long total_chunks,
                         int max_n_ridges, const OutDesc *outs, unsigned long long *ctr,
                         cudaStream_t s) {
  if (n_ids <= 0 || total_chunks == 0) return cudaSuccess;
  const size_t smem = (size_t)max_n_ridges * kSweepTPB;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned long long grid = (total_chunks + kSweepTPB - 1) / kSweepTPB;
  sweep_kernel<<<(unsigned)grid, kSweepTPB, smem, s>>>(d_inst, d_ids, n_ids, basis, dims, clogs,
                                                       chunks, outs, ctr);
  return cudaGetLastError();
}

}  // namespace wpm
