// wpm_kernels.cu -- sm_103a kernels of libwpm: weak pseudo-manifold enumeration
// (Choi, Jang, Vallee, arXiv 2301.00806).
//
//   setup_kernel   one block per instance: candidate facets (Section 3.1 / Proposition
//                  4.2), ridges with parents and the ridge-facet incidence tables (Section
//                  2.1), the resolved properties (Section 4.2 bound, base facet).
//   roots_kernel   one root work item per instance (forced-in facets + base facet in,
//                  forced-out facets out).
//   expand_kernel  breadth-first: every child of every item becomes an item in HBM.
//   dfs_kernel     depth-first: one search per thread over its item, with a node budget
//                  per pass; on exhaustion the unexplored siblings of every open level go
//                  back to the ring as items. (expand_kernel and dfs_kernel live in
//                  wpm_search.cuh and are instantiated per size class by wpm_class.cu.)
//   sort_kernel    one merge pass of a per-instance merge sort of the output masks.
//
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_classes.h"
#include "wpm_internal.h"

namespace wpm {

// ------------------------------------------------------------------------------------
// Setup: candidate facets, ridges, incidence (one block per instance).
// ------------------------------------------------------------------------------------

// Binomials C[a][b] for a, b <= 16.
__device__ __forceinline__ void fill_binom(int (*C)[17]) {
  for (int i = threadIdx.x; i < 17 * 17; i += blockDim.x) {
    int a = i / 17, b = i % 17;
    long long v = 1;
    if (b > a) v = 0;
    else for (int k = 0; k < b; k++) v = v * (a - k) / (k + 1);
    C[a][b] = (int)v;
  }
}

// The R-th k-subset of [m] in lexicographic order of sorted tuples (combinatorial
// number system, smallest element first).
__device__ __forceinline__ uint32_t unrank(int R, int m, int k, const int (*C)[17]) {
  uint32_t mask = 0;
  int v = 0;
  for (int i = 0; i < k; i++) {
    for (; v < m; v++) {
      int cnt = C[m - 1 - v][k - 1 - i];
      if (R < cnt) { mask |= 1u << v; v++; break; }
      R -= cnt;
    }
  }
  return mask;
}

// Lexicographic rank of a k-subset of [m] (inverse of unrank).
__device__ __forceinline__ int rank_of(uint32_t mask, int m, int k, const int (*C)[17]) {
  int R = 0, i = 0, prev = -1;
  for (int v = 0; v < m; v++) {
    if (!((mask >> v) & 1u)) continue;
    for (int u = prev + 1; u < v; u++) R += C[m - 1 - u][k - 1 - i];
    prev = v;
    i++;
  }
  return R;
}

// Is the given set of vectors (up to 16 bits each) linearly independent over Z2? Each
// vector is reduced against a basis kept one slot per leading bit.
__device__ __forceinline__ bool independent(const uint32_t *cols, uint32_t which, int m) {
  uint32_t basis[16];
#pragma unroll
  for (int b = 0; b < 16; b++) basis[b] = 0;
  for (int v = 0; v < m; v++) {
    if (!((which >> v) & 1u)) continue;
    uint32_t x = cols[v] & 0xFFFFu;
    bool placed = false;
#pragma unroll
    for (int b = 15; b >= 0; b--) {
      if (!placed && ((x >> b) & 1u)) {
        if (basis[b] == 0) { basis[b] = x; placed = true; }
        else x ^= basis[b];
      }
    }
    if (!placed) return false;  // reduced to zero: dependent
  }
  return true;
}

// Exclusive scan of arr[0..L) in place by one block; arr[L] = total; returns total.
__device__ int block_scan(int32_t *arr, int L, int *tmp) {
  const int T = blockDim.x, t = threadIdx.x;
  const int chunk = (L + T - 1) / T;
  const int lo = min(L, t * chunk), hi = min(L, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; i++) s += arr[i];
  tmp[t] = s;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int i = 0; i < T; i++) { int v = tmp[i]; tmp[i] = acc; acc += v; }
    tmp[T] = acc;
  }
  __syncthreads();
  int acc = tmp[t];
  for (int i = lo; i < hi; i++) { int v = arr[i]; arr[i] = acc; acc += v; }
  const int total = tmp[T];
  __syncthreads();
  if (t == 0) arr[L] = total;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(256) setup_kernel(InstDesc *insts, const int32_t *ids) {
  __shared__ int C[17][17];
  __shared__ int tmp[257];
  __shared__ long long red[256];
  __shared__ uint32_t given[2048];  // kind 2: membership bitmap over all 2^16 vertex masks
  InstDesc &I = insts[ids ? ids[blockIdx.x] : (int)blockIdx.x];
  fill_binom(C);
  if (I.kind == 2) {
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) given[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < I.n_given; i += blockDim.x) {
      const uint32_t f = I.given[i];
      atomicOr(&given[f >> 5], 1u << (f & 31));
    }
  }
  __syncthreads();
  const int n = I.n, m = I.m, nsub = I.nsub, nrsub = I.nrsub;
  const int t = threadIdx.x, T = blockDim.x;
  uint32_t cols[kMaxVertices];
  for (int v = 0; v < kMaxVertices; v++) cols[v] = I.cols[v];
  const uint32_t all = (1u << m) - 1u;
  const int fstride = n <= 8 ? 8 : 16;           // u16 entries per facet row
  const int pstride = m - n + 1 <= 8 ? 8 : 16;   // u16 entries per ridge row

  // (a1) candidate facets: lambda(sigma) a basis (primal) or the complement's dual rows a
  // basis (dual, Proposition 4.2).
  for (int R = t; R < nsub; R += T) {
    uint32_t s = unrank(R, m, n, C);
    bool ok;
    if (I.kind == 0) ok = independent(cols, s, m);
    else if (I.kind == 1) ok = independent(cols, all & ~s, m);
    else ok = (given[s >> 5] >> (s & 31)) & 1u;
    I.fprefix[R] = ok ? 1 : 0;
  }
  __syncthreads();
  const int M = block_scan(I.fprefix, nsub, tmp);
  for (int R = t; R < nsub; R += T)
    if (I.fprefix[R + 1] != I.fprefix[R]) I.facets[I.fprefix[R]] = (uint16_t)unrank(R, m, n, C);

  // (a2) ridges: (n-1)-subsets with at least one candidate parent, lexicographic order.
  for (int R = t; R < nrsub; R += T) {
    uint32_t r = unrank(R, m, n - 1, C);
    int has = 0;
    for (int v = 0; v < m && !has; v++) {
      if ((r >> v) & 1u) continue;
      int F = rank_of(r | (1u << v), m, n, C);
      has = I.fprefix[F + 1] - I.fprefix[F];
    }
    I.rprefix[R] = has;
  }
  __syncthreads();
  const int N = block_scan(I.rprefix, nrsub, tmp);
  // the parents row of each ridge, ascending facet index: adding a larger vertex to the
  // same ridge gives a lexicographically larger facet
  for (int R = t; R < nrsub; R += T) {
    if (I.rprefix[R + 1] == I.rprefix[R]) continue;
    uint32_t r = unrank(R, m, n - 1, C);
    uint16_t *row = I.prw + pstride * (size_t)I.rprefix[R];
    int k = 0;
    for (int v = 0; v < m; v++) {
      if ((r >> v) & 1u) continue;
      int F = rank_of(r | (1u << v), m, n, C);
      if (I.fprefix[F + 1] != I.fprefix[F]) row[k++] = (uint16_t)I.fprefix[F];
    }
    for (; k < pstride; k++) row[k] = 0xFFFFu;
  }
  // the ridges row of each facet
  for (int j = t; j < M; j += T) {
    uint32_t f = I.facets[j];
    uint16_t *row = I.frw + fstride * (size_t)j;
    int k = 0;
    for (int v = 0; v < m; v++) {
      if (!((f >> v) & 1u)) continue;
      int R = rank_of(f & ~(1u << v), m, n - 1, C);
      row[k++] = (uint16_t)I.rprefix[R];
    }
    for (; k < fstride; k++) row[k] = 0;
  }

  // (a3) properties: sum of the positive coefficients of each affine property
  for (int a = 0; a < I.n_aff; a++) {
    long long s = 0;
    if (M == I.n_facets_req)
      for (int j = t; j < M; j += T) { int c = I.aff_coef[a * M + j]; if (c > 0) s += c; }
    red[t] = s;
    __syncthreads();
    if (t == 0) {
      long long acc = 0;
      for (int i = 0; i < T; i++) acc += red[i];
      I.aff_bound0[a] = (long long)I.aff_c0[a] + acc;
    }
    __syncthreads();
  }
  if (t == 0) {
    int err = 0;
    if (M > kMaxFacets || N > kMaxRidges) err |= kErrLimit;
    if ((I.has_fin || I.has_fout || I.n_aff > 0) && I.n_facets_req != M) err |= kErrMaskSize;
    int cap = I.cap_req;
    if (cap == -2) {
      if (m != n + 4) { err |= kErrCapNeedsPic4; cap = -1; }
      else cap = C[n + 4 - (n + 1) / 2][4] + C[n + 3 - n / 2][4];
    }
    I.M = M;
    I.N = N;
    I.cap = cap;
    I.base_idx = (I.fprefix[1] != I.fprefix[0]) ? 0 : -1;  // {0..n-1} has rank 0
    I.mw = (M + 31) / 32;
    I.nw = (N + 15) / 16;
    I.ow = M > 0 ? (M + 63) / 64 : 1;
    I.fstride = fstride;
    I.pstride = pstride;
    I.err = err;
  }
}

cudaError_t launch_setup(InstDesc *d_inst, int n_inst, cudaStream_t s) {
  if (n_inst <= 0) return cudaSuccess;
  setup_kernel<<<n_inst, 256, 0, s>>>(d_inst, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_setup_ids(InstDesc *d_inst, const int32_t *d_ids, int n_ids, cudaStream_t s) {
  if (n_ids <= 0) return cudaSuccess;
  setup_kernel<<<n_ids, 256, 0, s>>>(d_inst, d_ids);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Roots: one fresh item per instance.
// ------------------------------------------------------------------------------------

__global__ void roots_kernel(const InstDesc *insts, int n_ids, const int32_t *ids,
                             unsigned long long *ctr, uint32_t *ring,
                             unsigned long long ring_cap, int item_words, int cls_mw,
                             QueueCtl *q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ids) return;
  const int id = ids[i];
  const InstDesc &I = insts[id];
  if (I.err) return;
  if (I.base_req && I.base_idx < 0) {  // the base facet is no candidate: no outputs
    atomicAdd(&ctr[kCtrN * id + kCtrProbes], 1ull);
    return;
  }
  const unsigned long long slot = atomicAdd(&q->tail, 1ull);
  if (slot - q->head_start >= ring_cap) { atomicOr(&q->err, 1ull); return; }
  uint32_t *it = ring + (slot % ring_cap) * (unsigned long long)item_words;
  it[0] = (uint32_t)id;
  it[1] = kItemFresh;
  it[2] = 0;
  it[3] = 0;
  for (int w = 0; w < cls_mw; w++) {
    uint32_t in = 0, out = 0;
    if (w < I.mw) {
      if (I.fin) in = (uint32_t)(I.fin[w >> 1] >> ((w & 1) * 32));
      if (I.fout) out = (uint32_t)(I.fout[w >> 1] >> ((w & 1) * 32));
      if (I.base_req && w == 0) in |= 1u;
    }
    it[kItemHeader + w] = in;
    it[kItemHeader + cls_mw + w] = out;
  }
  atomicAdd(&ctr[kCtrN * id + kCtrLive], 1ull);
}

cudaError_t launch_roots(const InstDesc *d_inst, int n_ids, const int32_t *d_ids,
                         unsigned long long *ctr, uint32_t *ring, unsigned long long ring_cap,
                         int item_words, int cls_mw, QueueCtl *q, cudaStream_t s) {
  if (n_ids <= 0) return cudaSuccess;
  roots_kernel<<<(n_ids + 127) / 128, 128, 0, s>>>(d_inst, n_ids, d_ids, ctr, ring, ring_cap,
                                                  item_words, cls_mw, q);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Device-driven pass loop (a CUDA graph with a conditional while node runs prep, the
// depth-first pass and check until check clears the condition).
// ------------------------------------------------------------------------------------

// The items left by the last pass become this pass's: [head, tail). Per-warp passes may
// have overshot head past the old tail (their tickets past it are void).
__global__ void pass_prep_kernel(QueueCtl *q, int thread_mode) {
  unsigned long long head = q->head;
  if (!thread_mode && head > q->limit) head = q->limit;
  if (head > q->tail) head = q->tail;
  q->head = head;
  q->head_start = head;
  q->limit = q->tail;
  q->idle = q->nodes = q->parked = q->waiting = q->exited = q->full = 0;
  q->epoch++;
  q->passes++;
}

// Another pass while items are left or searches parked work, no error was raised, and the
// loop has not run max_passes times (then error 8).
__global__ void pass_check_kernel(QueueCtl *q, int thread_mode, cudaGraphConditionalHandle h,
                                  unsigned long long max_passes) {
  unsigned long long head = q->head;
  if (!thread_mode && head > q->limit) head = q->limit;
  bool more = q->err == 0 && (q->tail > head || q->parked > 0);
  if (more && q->passes >= max_passes) {
    q->err |= 8ull;
    more = false;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// After a level of the graph-driven expansion: its children, [limit, tail), are the next
// level's items. Another level while no error was raised and the new level has items, fewer
// than `target`, whose children fit in the ring (at most max_children each) -- the rule of the
// host-driven loop -- and fewer than max_levels levels have run (a bound only: stopping early
// leaves a smaller frontier, never a different result).
__global__ void expand_check_kernel(QueueCtl *q, cudaGraphConditionalHandle h,
                                    unsigned long long target, unsigned long long max_children,
                                    unsigned long long ring_cap, unsigned long long max_levels) {
  const unsigned long long live = q->tail - q->limit;
  q->head_start = q->limit;
  q->limit = q->tail;
  q->head = q->tail;
  q->passes++;
  const bool more = q->err == 0 && live > 0 && live < target &&
                    live * max_children + live <= ring_cap && q->passes < max_levels;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

cudaError_t launch_expand_check(QueueCtl *q, cudaGraphConditionalHandle h,
                                unsigned long long target, unsigned long long max_children,
                                unsigned long long ring_cap, unsigned long long max_levels,
                                cudaStream_t s) {
  expand_check_kernel<<<1, 1, 0, s>>>(q, h, target, max_children, ring_cap, max_levels);
  return cudaGetLastError();
}

cudaError_t launch_pass_prep(QueueCtl *q, int thread_mode, cudaStream_t s) {
  pass_prep_kernel<<<1, 1, 0, s>>>(q, thread_mode);
  return cudaGetLastError();
}

cudaError_t launch_pass_check(QueueCtl *q, int thread_mode, cudaGraphConditionalHandle h,
                              unsigned long long max_passes, cudaStream_t s) {
  pass_check_kernel<<<1, 1, 0, s>>>(q, thread_mode, h, max_passes);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Size classes and launchers (the search kernels are instantiated in wpm_class.cu).
// ------------------------------------------------------------------------------------

static const SizeClass kClasses[] = {
#define X(k, mw, nw) {mw, nw},
    WPM_CLASSES(X)
#undef X
};

int n_size_classes() { return (int)(sizeof(kClasses) / sizeof(kClasses[0])); }
SizeClass size_class(int k) { return kClasses[k]; }
int pick_size_class(int mw, int nw) {
  for (int k = 0; k < n_size_classes(); k++)
    if (kClasses[k].mw >= mw && kClasses[k].nw >= nw) return k;
  return -1;
}
int item_words_for(int k) { return kItemHeader + 2 * kClasses[k].mw + kClasses[k].nw; }
int state_words(int k) {  // must equal Cls<mw, nw>::SMW of wpm_search.cuh
  return ((kClasses[k].nw + 2 * kClasses[k].mw + 1) & ~1) + 4 * kMaxAffine;
}

int tstate_words(int k) {  // must equal ts::TCls<mw, nw, *>::SMW of wpm_tsearch.cuh
  const int nw = kClasses[k].nw, mw = kClasses[k].mw;
  return nw + 2 * mw + (nw <= 96 ? 0 : (nw + 31) / 32);
}

size_t dfs_smem_bytes(int k, int search, int tpb, int max_depth) {
  if (search == kSearchThread) return (size_t)tpb * tstate_words(k) * 4u;
  return (size_t)(tpb / 32) * (size_t)(state_words(k) + 2 * max_depth) * 4u;
}

static cudaError_t dispatch(int k, int mode, const PassArgs &a, int grid, int n_items, int tpb,
                            size_t smem, cudaStream_t s) {
  switch (k) {
#define X(id, mw, nw) \
  case id:            \
    return class_launch_##id(mode, a, grid, n_items, tpb, smem, s);
    WPM_CLASSES(X)
#undef X
    default:
      return cudaErrorInvalidValue;
  }
}

int dfs_max_blocks_per_sm(int k, int search, int tpb, int max_depth) {
  const size_t smem = dfs_smem_bytes(k, search, tpb, max_depth);
  const int mode = search == kSearchThread ? 2 : 1;
  switch (k) {
#define X(id, mw, nw) \
  case id:            \
    return class_occupancy_##id(mode, tpb, smem);
    WPM_CLASSES(X)
#undef X
    default:
      return 0;
  }
}

cudaError_t launch_expand(int k, const PassArgs &a, int n_items, int tpb, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const int wpb = tpb / 32;
  const size_t smem = (size_t)wpb * state_words(k) * 4u;
  return dispatch(k, 0, a, (n_items + wpb - 1) / wpb, n_items, tpb, smem, s);
}

cudaError_t launch_expand_queued(int k, const PassArgs &a, int blocks, cudaStream_t s) {
  const size_t smem = (size_t)8 * state_words(k) * 4u;
  return dispatch(k, 0, a, blocks, -1, 256, smem, s);
}

cudaError_t launch_dfs(int k, int search, const PassArgs &a, int blocks, int tpb, cudaStream_t s) {
  return dispatch(k, search == kSearchThread ? 2 : 1, a, blocks, 0, tpb,
                  dfs_smem_bytes(k, search, tpb, a.max_depth), s);
}

// ------------------------------------------------------------------------------------
// Output sort: one merge pass over every instance's masks (runs of length `run` are
// merged pairwise). Each element finds its place by a binary search in the other run;
// ties are impossible within an instance (the masks are distinct) but are ordered
// stably anyway (run A before run B).
// ------------------------------------------------------------------------------------

__device__ __forceinline__ int cmp_mask(const uint64_t *a, const uint64_t *b, int ow) {
  for (int w = ow - 1; w >= 0; w--) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}

__global__ void sort_kernel(const InstDesc *insts, const OutDesc *outs, const int32_t *ids,
                            int n_ids, const unsigned long long *seg, unsigned long long total,
                            unsigned long long run, int parity) {
  const unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int lo = 0, hi = n_ids;  // segment: seg[s] <= e < seg[s + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (seg[mid] <= e) lo = mid; else hi = mid;
  }
  const int id = ids[lo];
  const int ow = insts[id].ow;
  const OutDesc &O = outs[id];
  const uint64_t *src = parity ? O.out2 : O.out;
  uint64_t *dst = parity ? O.out : O.out2;
  const unsigned long long len = seg[lo + 1] - seg[lo];
  const unsigned long long i = e - seg[lo];
  const unsigned long long b = (i / (2 * run)) * (2 * run);
  const uint64_t *key = src + i * ow;
  unsigned long long pos;
  if (i < b + run) {
    // in run A: count the elements of B below key
    unsigned long long l = min(b + run, len), h = min(b + 2 * run, len);
    const unsigned long long b0 = l;
    while (l < h) {
      const unsigned long long mid = (l + h) >> 1;
      if (cmp_mask(src + mid * ow, key, ow) < 0) l = mid + 1; else h = mid;
    }
    pos = (i - b) + (l - b0);
  } else {
    // in run B: count the elements of A not above key
    unsigned long long l = b, h = b + run;
    while (l < h) {
      const unsigned long long mid = (l + h) >> 1;
      if (cmp_mask(src + mid * ow, key, ow) <= 0) l = mid + 1; else h = mid;
    }
    pos = (i - b - run) + (l - b);
  }
  uint64_t *d = dst + (b + pos) * ow;
  for (int w = 0; w < ow; w++) d[w] = key[w];
}

cudaError_t launch_sort_pass(const InstDesc *d_inst, const OutDesc *d_outs, const int32_t *d_ids,
                             int n_ids, const unsigned long long *d_seg, unsigned long long total,
                             unsigned long long run, int parity, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  const int tpb = 256;
  const unsigned long long grid = (total + tpb - 1) / tpb;
  sort_kernel<<<(unsigned)grid, tpb, 0, s>>>(d_inst, d_outs, d_ids, n_ids, d_seg, total, run,
                                             parity);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Segmented copy of the sorted outputs (into a staging buffer or the callers' buffers).
// ------------------------------------------------------------------------------------

__global__ void segment_copy_kernel(const CopySeg *segs, int n_segs,
                                    const unsigned long long *prefix, unsigned long long total) {
  for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < total;
       e += (unsigned long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_segs;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= e) lo = mid; else hi = mid;
    }
    segs[lo].dst[e - prefix[lo]] = segs[lo].src[e - prefix[lo]];
  }
}

cudaError_t launch_segment_copy(const CopySeg *d_segs, int n_segs, const unsigned long long *d_prefix,
                                unsigned long long total_words, cudaStream_t s) {
  if (total_words == 0 || n_segs == 0) return cudaSuccess;
  unsigned long long grid = (total_words + 255) / 256;
  if (grid > 65535ull * 8) grid = 65535ull * 8;
  segment_copy_kernel<<<(unsigned)grid, 256, 0, s>>>(d_segs, n_segs, d_prefix, total_words);
  return cudaGetLastError();
}

}  // namespace wpm
