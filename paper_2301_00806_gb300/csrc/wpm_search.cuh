// wpm_search.cuh -- the depth-first search of libwpm (included by wpm_class.cu, which is
// compiled once per kernel size class).
//
// The search is the ridge-driven branch-and-prune of the canonical tree: at a node the
// lowest-index ridge of degree 1 is completed by one of its undecided parents (the other
// parents are excluded); a node without degree-1 ridges is a WPM by Proposition 2.1 and is
// emitted when every property holds, then extended by a new lowest facet. A child that
// would raise a ridge to degree 3, exceed the facet cap, or make an affine property
// unreachable is rejected (a probe).
//
// Per-thread state lives in shared memory, word w of thread t at [w * TPB + t]: every
// dynamically indexed access of a warp then hits 32 distinct banks.
//   cnt[NW]  ridge degrees, 2 bits per ridge, 16 ridges per word (values 0, 1, 2)
//   inb[MW]  In, one bit per candidate facet
//   outb[MW] Out (explicit exclusions; bits >= M are set so they are never free)
//   summ[SW] one bit per cnt word that holds a degree-1 ridge (in a register if NW <= 64)
// Facets below `floor` that are not in In are excluded too (the "new lowest facet" rule of
// the seed branch), so a seed child needs no Out writes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {

// ------------------------------------------------------------------------------------
// The search state of one thread.
// ------------------------------------------------------------------------------------

template <int MW_, int NW_, int TPB_>
struct Cls {
  static constexpr int MW = MW_, NW = NW_, TPB = TPB_;
  static constexpr int SW = (NW + 31) / 32;
  static constexpr bool kSummReg = NW <= 64;
  static constexpr int SMW = NW + 2 * MW + (kSummReg ? 0 : SW);
  static constexpr int IW = kItemHeader + 2 * MW + NW;
};

// Stack entries (32 bits).
//   ridge level: bit 31 = 0 | r << 19 | cur << 15 | U       U: undecided parent slots of r
//                (15 bits), cur: slot of the child being explored (15 = none yet)
//   seed level:  bit 31 = 1 | node_floor << 12 | start      start: lowest facet not yet
//                tried as a new lowest facet
__device__ __forceinline__ uint32_t mk_ridge(int r, uint32_t U) {
  return ((uint32_t)r << 19) | (15u << 15) | U;
}
__device__ __forceinline__ uint32_t mk_seed(int nf, int start) {
  return 0x80000000u | ((uint32_t)nf << 12) | (uint32_t)start;
}

template <class K>
struct Search {
  uint32_t *sm;
  uint64_t summ;
  // instance
  const InstDesc *I;
  const OutDesc *od;
  unsigned long long *ctr;
  int inst, n, M, mw, nw, ow, cap, n_aff, list_mode;
  const uint16_t *fr;
  const int32_t *poff;
  const uint16_t *pidx;
  // node
  int size, floor_;
  long long s_in[kMaxAffine], neg_in[kMaxAffine];
  // statistics of the current item
  unsigned long long nodes, probes, count;

  __device__ __forceinline__ uint32_t &cnt(int w) { return sm[w * K::TPB]; }
  __device__ __forceinline__ uint32_t &inb(int w) { return sm[(K::NW + w) * K::TPB]; }
  __device__ __forceinline__ uint32_t &outb(int w) { return sm[(K::NW + K::MW + w) * K::TPB]; }
  __device__ __forceinline__ uint32_t &summw(int s) {
    return sm[(K::NW + 2 * K::MW + s) * K::TPB];
  }

  __device__ __forceinline__ void set_summ(int w, uint32_t v) {
    const uint32_t has = (v & ~(v >> 1) & 0x55555555u) != 0u;
    if (K::kSummReg) {
      summ = (summ & ~(1ull << w)) | ((uint64_t)has << w);
    } else {
      uint32_t &s = summw(w >> 5);
      s = (s & ~(1u << (w & 31))) | (has << (w & 31));
    }
  }

  __device__ __forceinline__ void bind(const InstDesc *insts, const OutDesc *outs,
                                       unsigned long long *ctr_, int id) {
    inst = id;
    I = insts + id;
    od = outs + id;
    ctr = ctr_;
    n = I->n; M = I->M; mw = I->mw; nw = I->nw; ow = I->ow; cap = I->cap;
    n_aff = I->n_aff; list_mode = I->mode == 0;
    fr = I->fr; poff = I->poff; pidx = I->pidx;
  }

  // No ridge of facet p has degree 2 (adding p keeps every degree <= 2).
  __device__ __forceinline__ bool fits(int p) {
    const uint16_t *f = fr + p * n;
    for (int k = 0; k < n; k++) {
      const int r = f[k];
      if ((cnt(r >> 4) >> ((r & 15) * 2)) & 2u) return false;
    }
    return true;
  }

  __device__ __forceinline__ bool child_ok(int p) {
    if (cap >= 0 && size >= cap) return false;
    for (int a = 0; a < n_aff; a++) {
      const long long c = I->aff_coef[a * M + p];
      if (I->aff_bound0[a] + neg_in[a] + (c < 0 ? c : 0) <= 0) return false;
    }
    return fits(p);
  }

  __device__ __forceinline__ void add(int p) {
    const uint16_t *f = fr + p * n;
    for (int k = 0; k < n; k++) {
      const int r = f[k], w = r >> 4;
      const uint32_t v = cnt(w) + (1u << ((r & 15) * 2));
      cnt(w) = v;
      set_summ(w, v);
    }
    inb(p >> 5) |= 1u << (p & 31);
    size++;
    for (int a = 0; a < n_aff; a++) {
      const long long c = I->aff_coef[a * M + p];
      s_in[a] += c;
      if (c < 0) neg_in[a] += c;
    }
  }

  __device__ __forceinline__ void remove(int p) {
    const uint16_t *f = fr + p * n;
    for (int k = 0; k < n; k++) {
      const int r = f[k], w = r >> 4;
      const uint32_t v = cnt(w) - (1u << ((r & 15) * 2));
      cnt(w) = v;
      set_summ(w, v);
    }
    inb(p >> 5) &= ~(1u << (p & 31));
    size--;
    for (int a = 0; a < n_aff; a++) {
      const long long c = I->aff_coef[a * M + p];
      s_in[a] -= c;
      if (c < 0) neg_in[a] -= c;
    }
  }

  // Lowest-index ridge of degree 1, or -1 (then In is a WPM).
  __device__ __forceinline__ int select_ridge() {
    int w = -1;
    if (K::kSummReg) {
      if (summ) w = __ffsll((long long)summ) - 1;
    } else {
      const int sw = (nw + 31) >> 5;
      for (int s = 0; s < sw; s++) {
        const uint32_t x = summw(s);
        if (x) { w = s * 32 + __ffs(x) - 1; break; }
      }
    }
    if (w < 0) return -1;
    const uint32_t v = cnt(w);
    const uint32_t d1 = v & ~(v >> 1) & 0x55555555u;
    return w * 16 + ((__ffs(d1) - 1) >> 1);
  }

  __device__ __forceinline__ bool decided(int q) {
    return q < floor_ || (((inb(q >> 5) | outb(q >> 5)) >> (q & 31)) & 1u);
  }

  __device__ __forceinline__ uint32_t undecided_parents(int r) {
    const int b = poff[r], e = poff[r + 1];
    uint32_t U = 0;
    for (int s = 0; s < e - b; s++)
      if (!decided(pidx[b + s])) U |= 1u << s;
    return U;
  }

  // Smallest facet g >= start in neither In nor Out, or -1.
  __device__ __forceinline__ int next_free(int start) {
    if (start >= M) return -1;
    int w = start >> 5;
    uint32_t x = ~(inb(w) | outb(w)) & (0xFFFFFFFFu << (start & 31));
    while (!x) {
      if (++w >= mw) return -1;
      x = ~(inb(w) | outb(w));
    }
    const int g = w * 32 + __ffs(x) - 1;
    return g < M ? g : -1;
  }

  __device__ __forceinline__ void emit() {
    for (int a = 0; a < n_aff; a++)
      if ((long long)I->aff_c0[a] + s_in[a] <= 0) return;
    count++;
    if (list_mode) {
      const unsigned long long slot = atomicAdd(&ctr[kCtrN * inst + kCtrFill], 1ull);
      if (slot < od->cap) {
        uint64_t *dst = od->out + slot * (unsigned long long)ow;
        for (int w = 0; w < ow; w++) {
          const uint32_t lo = (2 * w < mw) ? inb(2 * w) : 0u;
          const uint32_t hi = (2 * w + 1 < mw) ? inb(2 * w + 1) : 0u;
          dst[w] = (uint64_t)lo | ((uint64_t)hi << 32);
        }
      }
    }
  }

  // Branching of the node the state now holds: a ridge level, or (closure) a seed level
  // after emitting In when `emit_ok`.
  __device__ __forceinline__ uint32_t examine(bool emit_ok) {
    const int r = select_ridge();
    if (r >= 0) return mk_ridge(r, undecided_parents(r));
    if (emit_ok) emit();
    return mk_seed(floor_, floor_);
  }

  // Try the next child of `top`. 0: no child left; 1: rejected (probe); 2: applied.
  __device__ __forceinline__ int advance(uint32_t &top) {
    if (!(top >> 31)) {
      const uint32_t U = top & 0x7FFFu;
      const int cur = (top >> 15) & 15, r = top >> 19;
      const int from = (cur == 15) ? 0 : cur + 1;
      const uint32_t rem = (U >> from) << from;
      if (!rem) return 0;
      const int k = __ffs(rem) - 1;
      top = (top & ~(15u << 15)) | ((uint32_t)k << 15);
      const int base = poff[r];
      const int p = pidx[base + k];
      if (!child_ok(p)) return 1;
      add(p);
      uint32_t others = U & ~(1u << k);
      while (others) {
        const int s = __ffs(others) - 1;
        others &= others - 1;
        const int q = pidx[base + s];
        outb(q >> 5) |= 1u << (q & 31);
      }
      return 2;
    }
    const int start = top & 0xFFF;
    const int g = next_free(start);
    if (g < 0) return 0;
    top = (top & ~0xFFFu) | (uint32_t)(g + 1);
    if (!child_ok(g)) return 1;
    add(g);
    floor_ = g;
    return 2;
  }

  // Undo the child currently applied under entry e.
  __device__ __forceinline__ void retreat(uint32_t e) {
    if (!(e >> 31)) {
      const uint32_t U = e & 0x7FFFu;
      const int k = (e >> 15) & 15, r = e >> 19;
      const int base = poff[r];
      remove(pidx[base + k]);
      uint32_t others = U & ~(1u << k);
      while (others) {
        const int s = __ffs(others) - 1;
        others &= others - 1;
        const int q = pidx[base + s];
        outb(q >> 5) &= ~(1u << (q & 31));
      }
    } else {
      remove((int)(e & 0xFFF) - 1);
      floor_ = (e >> 12) & 0xFFF;
    }
  }

  // Does entry e still have a child to try?
  __device__ __forceinline__ bool has_more(uint32_t e) {
    if (!(e >> 31)) {
      const int cur = (e >> 15) & 15;
      const int from = (cur == 15) ? 0 : cur + 1;
      return ((e & 0x7FFFu) >> from) != 0;
    }
    return next_free(e & 0xFFF) >= 0;
  }

  // Write the node the state holds, restricted to the children entry e has not tried,
  // as an open item.
  __device__ void write_item(const PassArgs &a, uint32_t e) {
    const unsigned long long slot = atomicAdd(&a.q->tail, 1ull);
    if (slot - a.q->head_start >= a.ring_cap) { atomicOr(&a.q->err, 1ull); return; }
    uint32_t *it = a.ring + (slot % a.ring_cap) * (unsigned long long)K::IW;
    const bool seed = e >> 31;
    const int fl = seed ? (int)(e & 0xFFF) : floor_;
    it[0] = (uint32_t)inst;
    it[1] = kItemOpen | ((uint32_t)fl << 16);
    it[2] = (uint32_t)size;
    it[3] = 0;
    for (int w = 0; w < mw; w++) it[kItemHeader + w] = inb(w);
    for (int w = 0; w < mw; w++) it[kItemHeader + K::MW + w] = outb(w);
    if (!seed) {  // the tried parents of the ridge join Out
      const int cur = (e >> 15) & 15;
      if (cur != 15) {
        uint32_t tried = (e & 0x7FFFu) & ((2u << cur) - 1u);
        const int base = poff[e >> 19];
        while (tried) {
          const int s = __ffs(tried) - 1;
          tried &= tried - 1;
          const int q = pidx[base + s];
          it[kItemHeader + K::MW + (q >> 5)] |= 1u << (q & 31);
        }
      }
    }
    for (int w = 0; w < nw; w++) it[kItemHeader + 2 * K::MW + w] = cnt(w);
    atomicAdd(&ctr[kCtrN * inst + kCtrLive], 1ull);
  }

  // Load an item. Returns false when a fresh root fails its checks.
  __device__ bool load(const uint32_t *it, bool &fresh) {
    const uint32_t fl = it[1];
    fresh = fl & kItemFresh;
    floor_ = fl >> 16;
    nodes = probes = count = 0;
    for (int w = 0; w < mw; w++) {
      inb(w) = it[kItemHeader + w];
      outb(w) = it[kItemHeader + K::MW + w];
    }
    if (M & 31) outb(mw - 1) |= 0xFFFFFFFFu << (M & 31);
    if (!K::kSummReg) {
      const int sw = (nw + 31) >> 5;
      for (int s = 0; s < sw; s++) summw(s) = 0;
    }
    summ = 0;
    bool ok = true;
    if (fresh) {
      for (int w = 0; w < nw; w++) cnt(w) = 0;
      size = 0;
      for (int w = 0; w < mw; w++) {
        if (inb(w) & outb(w)) ok = false;
        uint32_t x = inb(w);
        while (x) {
          const int j = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          if (!fits(j)) ok = false;
          const uint16_t *f = fr + j * n;
          for (int k = 0; k < n; k++) {
            const int r = f[k];
            cnt(r >> 4) += 1u << ((r & 15) * 2);
          }
          size++;
        }
      }
      if (cap >= 0 && size > cap) ok = false;
    } else {
      size = (int)it[2];
      for (int w = 0; w < nw; w++) cnt(w) = it[kItemHeader + 2 * K::MW + w];
    }
    for (int w = 0; w < nw; w++) set_summ(w, cnt(w));
    for (int a = 0; a < n_aff; a++) {
      s_in[a] = 0;
      neg_in[a] = 0;
      for (int w = 0; w < mw; w++) {
        uint32_t x = inb(w);
        while (x) {
          const int j = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          const long long c = I->aff_coef[a * M + j];
          s_in[a] += c;
          if (c < 0) neg_in[a] += c;
        }
      }
      if (fresh && I->aff_bound0[a] + neg_in[a] <= 0) ok = false;
    }
    return ok;
  }

  __device__ __forceinline__ void flush() {
    if (count) atomicAdd(&ctr[kCtrN * inst + kCtrCount], count);
    if (nodes) atomicAdd(&ctr[kCtrN * inst + kCtrNodes], nodes);
    if (probes) atomicAdd(&ctr[kCtrN * inst + kCtrProbes], probes);
    atomicAdd(&ctr[kCtrN * inst + kCtrLive], (unsigned long long)-1ll);
    nodes = probes = count = 0;
  }
};

// ------------------------------------------------------------------------------------
// Breadth-first expansion: each item's children become items.
// ------------------------------------------------------------------------------------

template <class K>
__global__ void __launch_bounds__(K::TPB) expand_kernel(PassArgs a, int n_items) {
  extern __shared__ uint32_t smem[];
  const int i = blockIdx.x * K::TPB + threadIdx.x;
  if (i >= n_items) return;
  Search<K> S;
  S.sm = smem + threadIdx.x;
  const unsigned long long idx = a.q->head_start + (unsigned long long)i;
  const uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
  S.bind(a.inst, a.outs, a.ctr, (int)it[0]);
  bool fresh;
  if (!S.load(it, fresh)) {
    S.probes++;
    S.flush();
    return;
  }
  if (fresh) S.nodes++;
  uint32_t e = S.examine(fresh);
  for (;;) {
    const int rc = S.advance(e);
    if (rc == 0) break;
    if (rc == 1) { S.probes++; continue; }
    S.nodes++;
    const uint32_t child = S.examine(true);
    if (S.has_more(child)) S.write_item(a, child);
    S.retreat(e);
  }
  S.flush();
}

// ------------------------------------------------------------------------------------
// Depth-first passes.
// ------------------------------------------------------------------------------------

template <class K>
__global__ void __launch_bounds__(K::TPB) dfs_kernel(PassArgs a) {
  extern __shared__ uint32_t smem[];
  Search<K> S;
  S.sm = smem + threadIdx.x;
  const int gtid = blockIdx.x * K::TPB + threadIdx.x;
  uint32_t *stk = a.stack + gtid;
  const int stride = a.n_threads;
  const int lane = threadIdx.x & 31;
  int depth = 0;
  uint32_t top = 0;
  long long pass_nodes = 0;
  bool active = true;
  while (__any_sync(0xFFFFFFFFu, active)) {
    if (!active) continue;
    if (depth == 0) {
      if (pass_nodes >= a.budget) {  // this thread's share of the pass is done
        active = false;
        continue;
      }
      // take the next item (warp-aggregated ticket)
      const unsigned mask = __activemask();
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&a.q->head, (unsigned long long)__popc(mask));
      base = __shfl_sync(mask, base, leader);
      const unsigned long long idx = base + __popc(mask & ((1u << lane) - 1u));
      if (idx >= a.q->limit) {
        active = false;  // tickets past the limit are returned by the host
        continue;
      }
      const uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
      S.bind(a.inst, a.outs, a.ctr, (int)it[0]);
      bool fresh;
      if (!S.load(it, fresh)) {
        S.probes++;
        S.flush();
        continue;
      }
      if (fresh) { S.nodes++; pass_nodes++; }
      top = S.examine(fresh);
      depth = 1;
      continue;
    }
    if (pass_nodes >= a.budget &&
        (*(volatile unsigned long long *)&a.q->tail - a.q->head_start) < a.dump_limit) {
      // budget spent: every open level's untried children go back to the ring
      for (int L = depth; L >= 1; L--) {
        const uint32_t e = (L == depth) ? top : stk[(L - 1) * stride];
        if (S.has_more(e)) S.write_item(a, e);
        if (L > 1) S.retreat(stk[(L - 2) * stride]);
      }
      depth = 0;
      S.flush();
      active = false;
      continue;
    }
    const int rc = S.advance(top);
    if (rc == 0) {
      depth--;
      if (depth > 0) {
        top = stk[(depth - 1) * stride];
        S.retreat(top);
      } else {
        S.flush();
      }
    } else if (rc == 1) {
      S.probes++;
    } else {
      S.nodes++;
      pass_nodes++;
      const uint32_t child = S.examine(true);
      if (depth >= a.max_depth) {  // cannot happen when max_depth covers the facet cap
        atomicOr(&a.q->err, 2ull);
        S.retreat(top);
        continue;
      }
      stk[(depth - 1) * stride] = top;
      top = child;
      depth++;
    }
  }
}


template <int MW, int NW, int TPB>
static cudaError_t launch_t(bool expand, const PassArgs &a, int grid, int n_items, cudaStream_t s) {
  using K = Cls<MW, NW, TPB>;
  const size_t smem = (size_t)K::SMW * 4u * TPB;
  if (expand) {
    auto fn = expand_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, TPB, smem, s>>>(a, n_items);
  } else {
    auto fn = dfs_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, TPB, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <int MW, int NW, int TPB>
static int occupancy_t() {
  using K = Cls<MW, NW, TPB>;
  const size_t smem = (size_t)K::SMW * 4u * TPB;
  auto fn = dfs_kernel<K>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, TPB, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

}  // namespace wpm
