// wpm_wsearch.cuh -- the warp-per-search kernels of libwpm (included by wpm_class.cu, which is
// compiled once per kernel size class). Used for the breadth-first expansion always, and for
// the depth-first passes of large instances, whose per-thread state would not fit enough
// searches per SM (wpm_tsearch.cuh has the per-thread search).
//
// One search per warp. The 32 lanes share one search state in shared memory and work
// together on each node: every candidate child of a node is checked at once (one lane per
// parent of the branching ridge, or per free facet of a 32-facet window), and a child's n
// ridge counters are updated by n lanes with shared-memory atomics. All control flow is
// warp-uniform, so the lanes never diverge between search paths.
//
// The search is the ridge-driven branch-and-prune of the canonical tree: at a node the
// lowest-index ridge of degree 1 is completed by one of its undecided parents (the other
// undecided parents are excluded); a node without degree-1 ridges is a WPM by Proposition
// 2.1 and is emitted when every property holds, then extended by a new lowest facet. A
// child that would raise a ridge to degree 3, exceed the facet cap, or make an affine
// property unreachable is rejected (a probe). A node's children are all checked when the
// node is expanded, so its probes are counted then; a node returned to the work ring
// therefore carries only children that have not been counted.
//
// Per-warp shared memory (u32 words):
//   cnt[NW]  ridge degrees, 2 bits per ridge, 16 ridges per word (values 0, 1, 2)
//   inb[MW]  In, one bit per candidate facet
//   outb[MW] Out (explicit exclusions; bits >= M are set so they are never free)
//   aff      per affine property: sum of its coefficients over In, and of the negative ones
//   stack    max_depth 64-bit entries
// Facets below `floor` that are not in In are excluded too (the "new lowest facet" rule of
// the seed branch), so a seed child needs no Out writes.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int MW_, int NW_>
struct WCls {
  static constexpr int MW = MW_, NW = NW_;
  static constexpr int AFF = (NW + 2 * MW + 1) & ~1;  // affine sums (8-byte aligned)
  static constexpr int SMW = AFF + 4 * kMaxAffine;    // state words per warp (even)
  static constexpr int IW = kItemHeader + 2 * MW + NW;
};

// Stack entries (64 bits).
//   ridge level (bit 63 = 0): r [0,12) | U [12,27) | A [27,42) | cur [42,46)
//     U: undecided parent slots of r; A: the slots whose child passed its checks;
//     cur: slot of the child being explored (15 = none yet)
//   seed level (bit 63 = 1): node_floor [0,12) | base [12,24) | acc [24,56) | cur [56,61)
//     | has_cur (61) | valid (62)
//     the window of candidates [base, base + 32): acc = accepted positions not yet
//     explored (valid when `valid`), cur = position of the child being explored
typedef unsigned long long Entry;
__device__ __forceinline__ Entry mk_ridge(int r, uint32_t U, uint32_t A) {
  return (Entry)r | ((Entry)U << 12) | ((Entry)A << 27) | (15ull << 42);
}
__device__ __forceinline__ Entry mk_seed(int nf) {
  return (1ull << 63) | (Entry)nf | ((Entry)nf << 12);
}
__device__ __forceinline__ bool is_seed(Entry e) { return e >> 63; }
__device__ __forceinline__ int e_r(Entry e) { return (int)(e & 0xFFF); }
__device__ __forceinline__ uint32_t e_U(Entry e) { return (uint32_t)(e >> 12) & 0x7FFFu; }
__device__ __forceinline__ uint32_t e_A(Entry e) { return (uint32_t)(e >> 27) & 0x7FFFu; }
__device__ __forceinline__ int e_cur(Entry e) { return (int)(e >> 42) & 15; }
__device__ __forceinline__ int s_floor(Entry e) { return (int)(e & 0xFFF); }
__device__ __forceinline__ int s_base(Entry e) { return (int)(e >> 12) & 0xFFF; }
__device__ __forceinline__ uint32_t s_acc(Entry e) { return (uint32_t)(e >> 24); }
__device__ __forceinline__ int s_cur(Entry e) { return (int)(e >> 56) & 31; }
__device__ __forceinline__ bool s_has_cur(Entry e) { return (e >> 61) & 1; }
__device__ __forceinline__ bool s_valid(Entry e) { return (e >> 62) & 1; }
__device__ __forceinline__ Entry mk_seed_full(int nf, int base, uint32_t acc, int cur, bool has_cur,
                                              bool valid) {
  return (1ull << 63) | (Entry)nf | ((Entry)base << 12) | ((Entry)acc << 24) |
         ((Entry)cur << 56) | ((Entry)has_cur << 61) | ((Entry)valid << 62);
}

template <class K>
struct WSearch {
  uint32_t *st;   // this warp's state words
  Entry *stk;     // this warp's stack
  int lane;
  // instance (uniform)
  const InstDesc *I;
  const OutDesc *od;
  unsigned long long *ctr;
  int inst, n, M, mw, nw, ow, cap, n_aff, list_mode, fstride, pstride;
  const uint16_t *fr;  // facet rows (fstride entries: its n ridges)
  const uint16_t *pr;  // ridge rows (pstride entries: its parents, 0xFFFF padded)
  // node (uniform)
  int size, floor_;
  // lane s: parent slot s of the top entry's ridge (0xFFFF if none)
  int tq;
  // statistics of the current item (uniform)
  unsigned long long nodes, probes, count;
  // the loaded item's flags and seed window
  uint32_t item_flags, item_acc;
  int item_base;

  __device__ __forceinline__ uint32_t *cnt() { return st; }
  __device__ __forceinline__ uint32_t *inb() { return st + K::NW; }
  __device__ __forceinline__ uint32_t *outb() { return st + K::NW + K::MW; }
  // s_in(e): sum of property e's coefficients over In; neg_in(e): of its negative ones
  __device__ __forceinline__ long long &s_in(int e) {
    return reinterpret_cast<long long *>(st + K::AFF)[e];
  }
  __device__ __forceinline__ long long &neg_in(int e) {
    return reinterpret_cast<long long *>(st + K::AFF)[kMaxAffine + e];
  }

  __device__ __forceinline__ void bind(const InstDesc *insts, const OutDesc *outs,
                                       unsigned long long *ctr_, int id) {
    inst = id;
    I = insts + id;
    od = outs + id;
    ctr = ctr_;
    n = I->n; M = I->M; mw = I->mw; nw = I->nw; ow = I->ow; cap = I->cap;
    n_aff = I->n_aff; list_mode = I->mode == 0;
    fstride = I->fstride; pstride = I->pstride;
    fr = I->frw; pr = I->prw;
  }

  __device__ __forceinline__ bool is_free(int f) {
    return !(((inb()[f >> 5] | outb()[f >> 5]) >> (f & 31)) & 1u);
  }
  __device__ __forceinline__ bool decided(int q) { return q < floor_ || !is_free(q); }

  // Lane-private check of candidate facet p: the cap, the affine bounds, and no ridge of p
  // at degree 2.
  __device__ __forceinline__ bool child_ok(int p) {
    if (cap >= 0 && size >= cap) return false;
    for (int e = 0; e < n_aff; e++) {
      const long long c = I->aff_coef[e * M + p];
      if (I->aff_bound0[e] + neg_in(e) + (c < 0 ? c : 0) <= 0) return false;
    }
    return fits(p);
  }

  // Add (sign = +1) or remove (-1) facet p; every lane takes part.
  __device__ __forceinline__ void apply(int p, int sign) {
    if (lane < n) {
      const int r = fr[(size_t)p * fstride + lane];
      const uint32_t inc = 1u << ((r & 15) * 2);
      atomicAdd(&cnt()[r >> 4], sign > 0 ? inc : (uint32_t)(0u - inc));
    }
    if (lane == 0) {
      if (sign > 0) inb()[p >> 5] |= 1u << (p & 31);
      else inb()[p >> 5] &= ~(1u << (p & 31));
    }
    size += sign;
    if (n_aff > 0) {
      __syncwarp();
      if (lane < n_aff) {
        const long long c = I->aff_coef[lane * M + p];
        s_in(lane) += sign * c;
        if (c < 0) neg_in(lane) += sign * c;
      }
    }
    __syncwarp();
  }

  // Lowest-index ridge of degree 1, or -1 (then In is a WPM).
  __device__ __forceinline__ int select_ridge() {
    int best = INT_MAX;
    for (int w = lane; w < nw; w += 32) {
      const uint32_t v = cnt()[w];
      const uint32_t d1 = v & ~(v >> 1) & 0x55555555u;
      if (d1 && best == INT_MAX) best = w * 16 + ((__ffs(d1) - 1) >> 1);
    }
    best = __reduce_min_sync(kFull, best);
    return best == INT_MAX ? -1 : best;
  }

  // Smallest facet g >= start in neither In nor Out, or -1.
  __device__ __forceinline__ int next_free(int start) {
    if (start >= M) return -1;
    const int w0 = start >> 5;
    for (int w = w0 + lane;; w += 32) {
      uint32_t x = 0;
      if (w < mw) {
        x = ~(inb()[w] | outb()[w]);
        if (w == w0) x &= 0xFFFFFFFFu << (start & 31);
      }
      const unsigned hit = __ballot_sync(kFull, x != 0);
      if (hit) {
        const int src = __ffs(hit) - 1;
        const uint32_t xv = __shfl_sync(kFull, x, src);
        const int wv = __shfl_sync(kFull, w, src);
        const int g = wv * 32 + __ffs(xv) - 1;
        return g < M ? g : -1;
      }
      if (__all_sync(kFull, w >= mw)) return -1;
    }
  }

  // A new node was just created: count it and, when it is a WPM, emit it. Returns the
  // node's lowest degree-1 ridge (-1 for a WPM).
  __device__ __forceinline__ int created(bool emit_ok) {
    nodes++;
    const int r = select_ridge();
    if (emit_ok && r < 0) emit();
    return r;
  }

  __device__ __forceinline__ void emit() {
    for (int e = 0; e < n_aff; e++)
      if ((long long)I->aff_c0[e] + s_in(e) <= 0) return;
    count++;
    if (list_mode) {
      unsigned long long slot = 0;
      if (lane == 0) slot = atomicAdd(&ctr[kCtrN * inst + kCtrFill], 1ull);
      slot = __shfl_sync(kFull, slot, 0);
      if (slot < od->cap) {
        uint64_t *dst = od->out + slot * (unsigned long long)ow;
        if (lane < ow) {
          const uint32_t lo = (2 * lane < mw) ? inb()[2 * lane] : 0u;
          const uint32_t hi = (2 * lane + 1 < mw) ? inb()[2 * lane + 1] : 0u;
          dst[lane] = (uint64_t)lo | ((uint64_t)hi << 32);
        }
      }
    }
  }

  // Expand the node the state holds, whose lowest degree-1 ridge is r (-1: a WPM): its
  // branching entry, with every candidate child of a ridge level checked now (the rejected
  // ones counted as probes); lanes' q receive the parents of its ridge. A seed level's
  // windows are checked lazily by next_child().
  __device__ __forceinline__ Entry expand_at(int r, int &q_out) {
    if (r < 0) {
      q_out = 0xFFFF;
      return mk_seed(floor_);
    }
    const int q = lane < pstride ? (int)pr[(size_t)r * pstride + lane] : 0xFFFF;
    const bool und = q != 0xFFFF && !decided(q);
    const bool ok = und && child_ok(q);
    const uint32_t U = __ballot_sync(kFull, und) & 0x7FFFu;
    const uint32_t A = __ballot_sync(kFull, ok) & 0x7FFFu;
    probes += __popc(U) - __popc(A);
    q_out = q;
    return mk_ridge(r, U, A);
  }

  // Check the window of candidates starting at the first free facet >= from. Returns the
  // accepted positions (and the window's base in `base`), or base = -1 when no free facet
  // is left.
  __device__ __forceinline__ uint32_t check_window(int from, int &base) {
    base = next_free(from);
    if (base < 0) return 0;
    const int f = base + lane;
    const bool fr_ = f < M && is_free(f);
    const bool ok = fr_ && child_ok(f);
    const uint32_t acc = __ballot_sync(kFull, ok);
    probes += __popc(__ballot_sync(kFull, fr_)) - __popc(acc);
    return acc;
  }

  // Apply the next accepted child of `top`. Returns false when none is left.
  __device__ __forceinline__ bool next_child(Entry &top) {
    if (!is_seed(top)) {
      const uint32_t A = e_A(top);
      const int cur = e_cur(top);
      const uint32_t rem = cur == 15 ? A : (A & ~((2u << cur) - 1u));
      if (!rem) return false;
      const int k = __ffs(rem) - 1;
      top = (top & ~(15ull << 42)) | ((Entry)k << 42);
      const int p = __shfl_sync(kFull, tq, k);
      apply(p, +1);
      const uint32_t others = e_U(top) & ~(1u << k);
      if ((others >> lane) & 1u) atomicOr(&outb()[tq >> 5], 1u << (tq & 31));
      __syncwarp();
      return true;
    }
    int base = s_base(top);
    uint32_t acc = s_acc(top);
    bool valid = s_valid(top);
    for (;;) {
      if (!valid) {
        acc = check_window(base, base);
        if (base < 0) return false;
        valid = true;
      }
      if (acc) break;
      base += 32;
      valid = false;
    }
    const int k = __ffs(acc) - 1;
    acc &= acc - 1;
    top = mk_seed_full(s_floor(top), base, acc, k, true, true);
    const int p = base + k;
    apply(p, +1);
    floor_ = p;
    return true;
  }

  // Undo the child currently applied under entry e (lanes' tq must hold e's parents row
  // when e is a ridge level).
  __device__ __forceinline__ void retreat(Entry e) {
    if (!is_seed(e)) {
      const int k = e_cur(e);
      const int p = __shfl_sync(kFull, tq, k);
      apply(p, -1);
      const uint32_t others = e_U(e) & ~(1u << k);
      if ((others >> lane) & 1u) atomicAnd(&outb()[tq >> 5], ~(1u << (tq & 31)));
      __syncwarp();
    } else {
      apply(s_base(e) + s_cur(e), -1);
      floor_ = s_floor(e);
    }
  }

  __device__ __forceinline__ void load_tq(Entry e) {
    if (!is_seed(e)) tq = lane < pstride ? (int)pr[(size_t)e_r(e) * pstride + lane] : 0xFFFF;
  }

  // Write the state as an item (flags, floor fl, seed window base/acc); lane-private xq
  // (>= 0) adds one facet to the item's Out.
  __device__ void write_item(const PassArgs &a, uint32_t flags, int fl, int base, uint32_t acc,
                             int xq) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(&a.q->tail, 1ull);
    slot = __shfl_sync(kFull, slot, 0);
    if (slot - a.q->head_start >= a.ring_cap) {
      if (lane == 0) atomicOr(&a.q->err, 1ull);
      return;
    }
    uint32_t *it = a.ring + (slot % a.ring_cap) * (unsigned long long)K::IW;
    if (lane == 0) {
      it[0] = (uint32_t)inst;
      it[1] = flags | ((uint32_t)fl << 16);
      it[2] = (uint32_t)size | ((uint32_t)base << 16);
      it[3] = acc;
      atomicAdd(&ctr[kCtrN * inst + kCtrLive], 1ull);
    }
    for (int w = lane; w < mw; w += 32) {
      it[kItemHeader + w] = inb()[w];
      it[kItemHeader + K::MW + w] = outb()[w];
    }
    for (int w = lane; w < nw; w += 32) it[kItemHeader + 2 * K::MW + w] = cnt()[w];
    __syncwarp();
    if (xq >= 0) atomicOr(&it[kItemHeader + K::MW + (xq >> 5)], 1u << (xq & 31));
  }

  // Write the node the state holds, restricted to the children of entry e that have not
  // been counted yet. A ridge level's counted parents join Out (every child of the ridge
  // excludes them anyway); a seed level carries its window instead, so that the facets it
  // rejected are checked again, and counted, deeper in the tree.
  __device__ void write_remaining(const PassArgs &a, Entry e) {
    if (!is_seed(e)) {
      const uint32_t A = e_A(e);
      const int cur = e_cur(e);
      const uint32_t rem = cur == 15 ? A : (A & ~((2u << cur) - 1u));
      if (!rem) return;
      const uint32_t counted = e_U(e) & ~rem;
      write_item(a, kItemOpen, floor_, 0, 0, ((counted >> lane) & 1u) ? tq : -1);
      return;
    }
    const int base = s_base(e);
    if (s_valid(e) && s_acc(e)) {
      write_item(a, kItemOpen | kItemSeed | kItemSeedValid, floor_, base, s_acc(e), -1);
      return;
    }
    const int nb = s_valid(e) ? base + 32 : base;
    if (next_free(nb) < 0) return;
    write_item(a, kItemOpen | kItemSeed, floor_, nb, 0, -1);
  }

  // Degree check alone: no ridge of facet p has degree 2.
  __device__ __forceinline__ bool fits(int p) {
    const uint4 *row = reinterpret_cast<const uint4 *>(fr + (size_t)p * fstride);
    const uint4 a = __ldg(row);
    const uint4 b = fstride > 8 ? __ldg(row + 1) : make_uint4(0, 0, 0, 0);
    uint32_t bad = 0;
#define WPM_FIT(k, word)                                   \
    if ((k) < n) {                                         \
      const int r = ((word) >> (((k) & 1) * 16)) & 0xFFFF; \
      bad |= cnt()[r >> 4] >> ((r & 15) * 2);              \
    }
    WPM_FIT(0, a.x) WPM_FIT(1, a.x) WPM_FIT(2, a.y) WPM_FIT(3, a.y)
    WPM_FIT(4, a.z) WPM_FIT(5, a.z) WPM_FIT(6, a.w) WPM_FIT(7, a.w)
    if (n > 8) {
      WPM_FIT(8, b.x) WPM_FIT(9, b.x) WPM_FIT(10, b.y) WPM_FIT(11, b.y)
      WPM_FIT(12, b.z) WPM_FIT(13, b.z) WPM_FIT(14, b.w) WPM_FIT(15, b.w)
    }
#undef WPM_FIT
    return !(bad & 2u);
  }

  // Load an item into the state. Returns false when a fresh root fails its checks.
  __device__ bool load(const uint32_t *it, bool &fresh) {
    const uint32_t fl = it[1];
    fresh = fl & kItemFresh;
    floor_ = fl >> 16;
    item_flags = fl & 0xFFFFu;
    item_base = (int)(it[2] >> 16);
    item_acc = it[3];
    nodes = probes = count = 0;
    for (int w = lane; w < mw; w += 32) {
      inb()[w] = it[kItemHeader + w];
      uint32_t o = it[kItemHeader + K::MW + w];
      if (w == mw - 1 && (M & 31)) o |= 0xFFFFFFFFu << (M & 31);
      outb()[w] = o;
    }
    bool ok = true;
    if (fresh) {
      for (int w = lane; w < nw; w += 32) cnt()[w] = 0;
      __syncwarp();
      size = 0;
      for (int w = 0; w < mw; w++) {
        uint32_t x = inb()[w];
        if (x & outb()[w]) ok = false;
        while (x) {
          const int j = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          if (!fits(j)) ok = false;
          __syncwarp();
          if (lane < n) {
            const int r = fr[(size_t)j * fstride + lane];
            atomicAdd(&cnt()[r >> 4], 1u << ((r & 15) * 2));
          }
          __syncwarp();
          size++;
        }
      }
      if (cap >= 0 && size > cap) ok = false;
    } else {
      size = (int)(it[2] & 0xFFFFu);
      for (int w = lane; w < nw; w += 32) cnt()[w] = it[kItemHeader + 2 * K::MW + w];
    }
    __syncwarp();
    for (int e = 0; e < n_aff; e++) {
      long long si = 0, ni = 0;
      for (int w = lane; w < mw; w += 32) {
        uint32_t x = inb()[w];
        while (x) {
          const int j = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          const long long c = I->aff_coef[e * M + j];
          si += c;
          if (c < 0) ni += c;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        si += __shfl_xor_sync(kFull, si, o);
        ni += __shfl_xor_sync(kFull, ni, o);
      }
      if (lane == 0) {
        s_in(e) = si;
        neg_in(e) = ni;
      }
      if (fresh && I->aff_bound0[e] + ni <= 0) ok = false;
    }
    __syncwarp();
    return ok;
  }

  // The entry to continue a loaded item with (after load() returned true).
  __device__ __forceinline__ Entry resume(bool fresh) {
    if (item_flags & kItemSeed)
      return mk_seed_full(floor_, item_base, item_acc, 0, false, item_flags & kItemSeedValid);
    const int r = fresh ? created(true) : select_ridge();
    return expand_at(r, tq);
  }

  __device__ __forceinline__ void flush() {
    if (lane == 0) {
      if (count) atomicAdd(&ctr[kCtrN * inst + kCtrCount], count);
      if (nodes) atomicAdd(&ctr[kCtrN * inst + kCtrNodes], nodes);
      if (probes) atomicAdd(&ctr[kCtrN * inst + kCtrProbes], probes);
      atomicAdd(&ctr[kCtrN * inst + kCtrLive], (unsigned long long)-1ll);
    }
    nodes = probes = count = 0;
  }
};

// ------------------------------------------------------------------------------------
// Breadth-first expansion: each item's accepted children become items (one warp per item).
// ------------------------------------------------------------------------------------

// n_items >= 0: items [head_start, head_start + n_items), one warp each. n_items < 0: the
// items [head_start, limit) of the queue, the warps of a fixed grid striding over them (a level
// of the expansion loop that runs on the device).
template <class K>
__global__ void __launch_bounds__(256) wexpand_kernel(PassArgs a, int n_items) {
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  const unsigned long long wpb = blockDim.x >> 5;
  const unsigned long long n =
      n_items >= 0 ? (unsigned long long)n_items : a.q->limit - a.q->head_start;
  const unsigned long long stride = n_items >= 0 ? n : (unsigned long long)gridDim.x * wpb;
  WSearch<K> S;
  S.lane = threadIdx.x & 31;
  S.st = smem + wib * K::SMW;
  S.stk = nullptr;
  // whole warps take an item or leave together
  for (unsigned long long i = blockIdx.x * wpb + wib; i < n; i += stride) {
    const unsigned long long idx = a.q->head_start + i;
    uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
    if ((it[1] & 0xFFFFu) == kItemEmpty) continue;
    S.bind(a.inst, a.outs, a.ctr, (int)it[0]);
    bool fresh;
    if (S.load(it, fresh)) {
      Entry e = S.resume(fresh);
      while (S.next_child(e)) {
        S.created(true);
        S.write_item(a, kItemOpen, S.floor_, 0, 0, -1);  // unexpanded: its children are uncounted
        S.retreat(e);
      }
    } else {
      S.probes++;
    }
    S.flush();
    if (a.clear_expanded) {  // every lane has read the item: its slot is now empty
      __syncwarp();
      if (S.lane == 0) it[1] = kItemEmpty;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// Depth-first passes (one search per warp).
// ------------------------------------------------------------------------------------

template <class K>
__global__ void __launch_bounds__(256) wdfs_kernel(PassArgs a) {
  extern __shared__ uint32_t smem[];
  const int wib = threadIdx.x >> 5;
  WSearch<K> S;
  S.lane = threadIdx.x & 31;
  uint32_t *mine = smem + wib * (K::SMW + 2 * a.max_depth);
  S.st = mine;
  S.stk = reinterpret_cast<Entry *>(mine + K::SMW);
  int depth = 0;
  Entry top = 0;
  long long pass_nodes = 0;
  for (;;) {
    if (depth == 0) {
      if (pass_nodes >= a.budget) break;
      unsigned long long idx = 0;
      if (S.lane == 0) idx = atomicAdd(&a.q->head, 1ull);
      idx = __shfl_sync(kFull, idx, 0);
      if (idx >= a.q->limit) break;  // tickets past the limit are returned by the host
      const uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
      if ((it[1] & 0xFFFFu) == kItemEmpty) continue;
      S.bind(a.inst, a.outs, a.ctr, (int)it[0]);
      bool fresh;
      if (!S.load(it, fresh)) {
        S.probes++;
        S.flush();
        continue;
      }
      if (fresh) pass_nodes++;
      top = S.resume(fresh);
      depth = 1;
      continue;
    }
    const bool spent = pass_nodes >= a.budget ||
                       ((pass_nodes & 63) == 63 &&
                        *(volatile unsigned long long *)&a.q->idle >= a.idle_limit);
    if (spent &&
        (*(volatile unsigned long long *)&a.q->tail - a.q->head_start) < a.dump_limit) {
      // every open level's uncounted children go back to the ring
      Entry e = top;
      for (int L = depth; L >= 1; L--) {
        S.write_remaining(a, e);
        if (L > 1) {
          e = S.stk[L - 2];
          S.load_tq(e);
          S.retreat(e);
        }
      }
      depth = 0;
      S.flush();
      break;
    }
    if (S.next_child(top)) {
      const int r = S.created(true);
      pass_nodes++;
      if (depth >= a.max_depth) {  // cannot happen when max_depth covers the facet cap
        if (S.lane == 0) atomicOr(&a.q->err, 2ull);
        S.retreat(top);
        continue;
      }
      if (S.lane == 0) S.stk[depth - 1] = top;
      __syncwarp();
      top = S.expand_at(r, S.tq);
      depth++;
    } else {
      depth--;
      if (depth > 0) {
        top = S.stk[depth - 1];
        S.load_tq(top);
        S.retreat(top);
      } else {
        S.flush();
      }
    }
  }
  if (S.lane == 0) {
    atomicAdd(&a.q->idle, 1ull);
    atomicAdd(&a.q->nodes, (unsigned long long)pass_nodes);
  }
}

template <int MW, int NW>
static cudaError_t wlaunch_t(int mode, const PassArgs &a, int grid, int n_items, int tpb,
                             size_t smem, cudaStream_t s) {
  using K = WCls<MW, NW>;
  if (mode == 0) {
    auto fn = wexpand_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, tpb, smem, s>>>(a, n_items);
  } else {
    auto fn = wdfs_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, tpb, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <int MW, int NW>
static int woccupancy_t(int tpb, size_t smem) {
  auto fn = wdfs_kernel<WCls<MW, NW>>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, tpb, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

}  // namespace wpm
