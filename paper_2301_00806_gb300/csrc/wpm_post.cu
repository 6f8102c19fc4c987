// wpm_post.cu -- the post-filters of Algorithm 4.4 (lines 8-12) on the found WPMs.
//
// For a WPM K on the vertex set [m]:
//   Pic(K) = (vertices used by K) - n, and line 9 discards Pic(K) < 4: K is kept when its
//   facets cover all m vertices (m = n + 4);
//   the seedness condition (Proposition 3.1): no edge {v, w} of K lies, for every minimal
//   non-face S of K, in S or outside S entirely (v in S <=> w in S).
// One warp per mask, in shared memory: the faces of K as a bitmap over all 2^m vertex
// subsets (32 subsets per word), built by marking the facets and closing downward one
// vertex at a time; the minimal non-faces (non-faces all of whose one-smaller subsets are
// faces); for each vertex v the set of vertices w that some minimal non-face separates from
// v; then every edge of K is checked. A second kernel compacts each list in order.
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_internal.h"

namespace wpm {

namespace {

constexpr int kPostWarps = 8;
constexpr int kPostWords = (1 << kPostMaxM) / 32;
constexpr unsigned kAll = 0xFFFFFFFFu;
// Within a word of 32 subsets (subset index p in bits 0..4): the positions whose bit i is set.
__constant__ uint32_t kHi[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};

}  // namespace

__global__ void __launch_bounds__(kPostWarps * 32)
    post_filter_kernel(const InstDesc *insts, const OutDesc *outs, const int32_t *sid, int ns,
                       const unsigned long long *seg, unsigned long long total, uint8_t *keep) {
  __shared__ uint32_t face_all[kPostWarps][kPostWords];
  __shared__ uint32_t split_all[kPostWarps][16];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *face = face_all[wid];
  uint32_t *split = split_all[wid];
  for (unsigned long long g = (unsigned long long)blockIdx.x * kPostWarps + wid; g < total;
       g += (unsigned long long)gridDim.x * kPostWarps) {
    int lo = 0, hi = ns - 1;  // the instance of mask g: the last j with seg[j] <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const int id = sid[lo];
    const InstDesc &I = insts[id];
    if (!I.post) {
      if (lane == 0) keep[g] = 1;
      continue;
    }
    const uint64_t *K = outs[id].out + (g - seg[lo]) * (unsigned long long)I.ow;
    const int m = I.m;
    const uint32_t all_v = (1u << m) - 1u;
    const int nwords = m >= 5 ? 1 << (m - 5) : 1;
    const uint32_t valid0 = m >= 5 ? kAll : ((1u << (1 << m)) - 1u);  // subsets in word 0
    for (int w = lane; w < nwords; w += 32) face[w] = 0;
    if (lane < 16) split[lane] = 0;
    __syncwarp();
    // the facets of K: their vertex masks marked as faces, and the vertices they cover
    uint32_t used = 0;
    for (int w = 0; w < I.ow; w++) {
      const uint64_t x = K[w];
      for (int b = lane; b < 64; b += 32) {
        if ((x >> b) & 1ull) {
          const uint32_t F = I.facets[w * 64 + b];
          used |= F;
          atomicOr(&face[F >> 5], 1u << (F & 31));
        }
      }
    }
    used = __reduce_or_sync(kAll, used);
    bool ok = !((I.post & WPM_POST_PIC) && used != all_v);
    if (ok && (I.post & WPM_POST_SEED)) {
      __syncwarp();
      // downward closure: every subset of a facet is a face
      for (int i = 0; i < m; i++) {
        if (i < 5) {
          const uint32_t hm = kHi[i];
          const int sh = 1 << i;
          for (int w = lane; w < nwords; w += 32) {
            const uint32_t x = face[w];
            face[w] = x | ((x & hm) >> sh);
          }
        } else {
          // words with bit b of their index pass their faces to the word without it (the
          // targets are never sources in this round)
          const int b = 1 << (i - 5);
          for (int w = lane; w < nwords; w += 32)
            if (w & b) face[w ^ b] |= face[w];
        }
        __syncwarp();
      }
      // minimal non-faces S (every S minus one vertex is a face), and the vertex pairs they
      // separate: bit w of split[v] when some minimal non-face holds exactly one of v, w
      for (int w = lane; w < nwords; w += 32) {
        const uint32_t x = face[w];
        uint32_t mnf = ~x & (w == 0 ? (valid0 & ~1u) : kAll);
        for (int i = 0; i < m; i++) {
          if (i < 5) {
            const uint32_t hm = kHi[i];
            mnf &= ((x << (1 << i)) & hm) | ~hm;
          } else {
            const int b = 1 << (i - 5);
            if (w & b) mnf &= face[w ^ b];
          }
        }
        while (mnf) {
          const int p = __ffs(mnf) - 1;
          mnf &= mnf - 1;
          const uint32_t S = ((uint32_t)w << 5) | (uint32_t)p;
          for (int v = 0; v < m; v++)
            atomicOr(&split[v], ((S >> v) & 1u) ? (~S & all_v) : S);
        }
      }
      __syncwarp();
      // an edge {v, w} that no minimal non-face separates breaks the seedness condition
      bool seed = true;
      if (lane < m) {
        for (int w2 = lane + 1; w2 < m; w2++) {
          const uint32_t S = (1u << lane) | (1u << w2);
          const bool edge = (face[S >> 5] >> (S & 31)) & 1u;
          if (edge && !((split[lane] >> w2) & 1u)) seed = false;
        }
      }
      ok = __all_sync(kAll, seed);
    }
    if (lane == 0) keep[g] = ok ? 1 : 0;
    __syncwarp();
  }
}

cudaError_t launch_post_filter(const InstDesc *d_inst, const OutDesc *outs, const int32_t *sid,
                               int ns, const unsigned long long *seg, unsigned long long total,
                               uint8_t *keep, cudaStream_t s) {
  if (ns <= 0 || total == 0) return cudaSuccess;
  unsigned long long blocks = (total + kPostWarps - 1) / kPostWarps;
  if (blocks > 4096ull * 152) blocks = 4096ull * 152;
  post_filter_kernel<<<(unsigned)blocks, kPostWarps * 32, 0, s>>>(d_inst, outs, sid, ns, seg,
                                                                  total, keep);
  return cudaGetLastError();
}

// One block per instance: the kept masks, in order, into out2 (by a block-wide prefix sum of
// the keep flags, one tile of 256 at a time), then back into out; the count and fill
// counters become the kept number.
__global__ void __launch_bounds__(256)
    post_compact_kernel(const InstDesc *insts, const OutDesc *outs, const int32_t *sid,
                        const unsigned long long *seg, const uint8_t *keep,
                        unsigned long long *ctr) {
  __shared__ unsigned warp_tot[8];
  __shared__ unsigned long long base;
  const int j = blockIdx.x, id = sid[j];
  const InstDesc &I = insts[id];
  if (!I.post) return;
  const OutDesc &o = outs[id];
  const unsigned long long b = seg[j], e = seg[j + 1];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ow = I.ow;
  if (tid == 0) base = 0;
  __syncthreads();
  for (unsigned long long t0 = b; t0 < e; t0 += 256) {
    const unsigned long long idx = t0 + tid;
    const bool f = idx < e && keep[idx];
    const unsigned bal = __ballot_sync(kAll, f);
    if (lane == 0) warp_tot[wid] = __popc(bal);
    __syncthreads();
    unsigned before = 0, tile = 0;
    for (int k = 0; k < 8; k++) {
      if (k < wid) before += warp_tot[k];
      tile += warp_tot[k];
    }
    const unsigned long long pos = base + before + __popc(bal & ((1u << lane) - 1u));
    if (f)
      for (int w = 0; w < ow; w++) o.out2[pos * ow + w] = o.out[(idx - b) * ow + w];
    __syncthreads();
    if (tid == 0) base += tile;
    __syncthreads();
  }
  const unsigned long long kept = base;
  for (unsigned long long k = tid; k < kept * (unsigned long long)ow; k += 256) o.out[k] = o.out2[k];
  if (tid == 0) {
    ctr[kCtrN * id + kCtrCount] = kept;
    ctr[kCtrN * id + kCtrFill] = kept;
  }
}

cudaError_t launch_post_compact(const InstDesc *d_inst, const OutDesc *outs, const int32_t *sid,
                                int ns, const unsigned long long *seg, const uint8_t *keep,
                                unsigned long long *ctr, cudaStream_t s) {
  if (ns <= 0) return cudaSuccess;
  post_compact_kernel<<<ns, 256, 0, s>>>(d_inst, outs, sid, seg, keep, ctr);
  return cudaGetLastError();
}

}  // namespace wpm
