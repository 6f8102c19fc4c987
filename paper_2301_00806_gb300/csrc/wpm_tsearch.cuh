// wpm_tsearch.cuh -- the per-thread depth-first search of libwpm (included by wpm_class.cu,
// compiled once per kernel size class).
//
// Each thread runs its own search. A loop iteration is one step of it: try the next
// candidate child of the top level (check it; on success add it, count the node and
// examine the child), or, when the level has no candidate left, pop it and undo its parent's
// child. The step is written so that the threads of a warp stay on one path: every loop
// over a facet's ridges or a ridge's parents is unrolled to its maximum and predicated, with
// no early exit, so threads that try and threads that pop split the warp only in two.
//
// The search is the ridge-driven branch-and-prune of the canonical tree (see
// wpm_wsearch.cuh); here a child is counted (node or probe) when it is tried, and a level
// returned to the work ring carries only its untried children: a ridge level's tried parents
// join Out, a seed level's floor moves past its tried facets.
//
// Per-thread state lives in shared memory, word w of thread t at [w * TPB + t], so every
// dynamically indexed access of a warp hits 32 distinct banks:
//   cnt[NW]  ridge degrees, 2 bits per ridge, 16 ridges per word (values 0, 1, 2)
//   inb[MW]  In; outb[MW] Out (bits >= M set)
//   summ[SW] one bit per cnt word that holds a degree-1 ridge (a register when NW <= 64)
// The stack is in global memory, entry L of thread t at [L * n_threads + t].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {
namespace ts {

template <int MW_, int NW_, int TPB_>
struct TCls {
  static constexpr int MW = MW_, NW = NW_, TPB = TPB_;
  static constexpr int SW = (NW + 31) / 32;
  static constexpr bool kSummReg = NW <= 64;
  static constexpr int SMW = NW + 2 * MW + (kSummReg ? 0 : SW);
  static constexpr int IW = kItemHeader + 2 * MW + NW;
};

constexpr unsigned kFull = 0xFFFFFFFFu;

// Stack entries (32 bits).
//   ridge level: bit 31 = 0 | r << 19 | cur << 15 | U       U: undecided parent slots of r
//                (15 bits), cur: slot of the child tried last (15 = none yet)
//   seed level:  bit 31 = 1 | node_floor << 12 | start      start: lowest facet not yet
//                tried as a new lowest facet
__device__ __forceinline__ uint32_t mk_ridge(int r, uint32_t U) {
  return ((uint32_t)r << 19) | (15u << 15) | U;
}
__device__ __forceinline__ uint32_t mk_seed(int nf, int start) {
  return 0x80000000u | ((uint32_t)nf << 12) | (uint32_t)start;
}

// Entry k (0..15) of a 32-byte row of u16 held as two uint4 (value selects only).
__device__ __forceinline__ int row_at(const uint4 &a, const uint4 &b, int k) {
  const bool lo = k < 8;
  const uint32_t x = lo ? a.x : b.x, y = lo ? a.y : b.y, z = lo ? a.z : b.z, w = lo ? a.w : b.w;
  const int c = (k >> 1) & 3;
  const uint32_t v = c == 0 ? x : (c == 1 ? y : (c == 2 ? z : w));
  return (int)((v >> ((k & 1) * 16)) & 0xFFFFu);
}

template <class K>
struct TSearch {
  uint32_t *sm;
  uint64_t summ;
  // instance
  const InstDesc *I;
  const OutDesc *od;
  unsigned long long *ctr;
  int inst, n, M, mw, nw, ow, cap, n_aff, list_mode, fstride, pstride;
  const uint16_t *fr;
  const uint16_t *pr;
  long long *aff;  // this thread's affine sums (global scratch): s_in[e], neg_in[e]
  // node
  int size, floor_;
  uint4 tp0, tp1;  // parents row of the top entry (ridge levels)
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
    fstride = I->fstride; pstride = I->pstride;
    fr = I->frw; pr = I->prw;
  }

  __device__ __forceinline__ void facet_row(int p, uint4 &a, uint4 &b) {
    const uint4 *row = reinterpret_cast<const uint4 *>(fr + (size_t)p * fstride);
    a = __ldg(row);
    b = fstride > 8 ? __ldg(row + 1) : make_uint4(0, 0, 0, 0);
  }
  __device__ __forceinline__ void ridge_row(int r, uint4 &a, uint4 &b) {
    const uint4 *row = reinterpret_cast<const uint4 *>(pr + (size_t)r * pstride);
    a = __ldg(row);
    b = pstride > 8 ? __ldg(row + 1) : make_uint4(kFull, kFull, kFull, kFull);
  }

  // No ridge of the facet (row a, b) has degree 2; every lookup is issued, none exits early.
  __device__ __forceinline__ bool fits(const uint4 &a, const uint4 &b) {
    uint32_t bad = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      if (k < n) {
        const int r = row_at(a, b, k);
        bad |= cnt(r >> 4) >> ((r & 15) * 2);
      }
    }
    if (n > 8) {
#pragma unroll
      for (int k = 8; k < 16; k++) {
        if (k < n) {
          const int r = row_at(a, b, k);
          bad |= cnt(r >> 4) >> ((r & 15) * 2);
        }
      }
    }
    return !(bad & 2u);
  }

  __device__ __forceinline__ bool child_ok(int p, const uint4 &a, const uint4 &b) {
    bool ok = !(cap >= 0 && size >= cap);
    for (int e = 0; e < n_aff; e++) {
      const long long c = I->aff_coef[e * M + p];
      if (I->aff_bound0[e] + aff[kMaxAffine + e] + (c < 0 ? c : 0) <= 0) ok = false;
    }
    return ok && fits(a, b);
  }

  // Add (sign = 1) or remove (sign = -1) facet p, whose row is (a, b).
  __device__ __forceinline__ void apply(int p, const uint4 &a, const uint4 &b, int sign) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
      if (k < n) {
        const int r = row_at(a, b, k), w = r >> 4;
        const uint32_t v = cnt(w) + (uint32_t)sign * (1u << ((r & 15) * 2));
        cnt(w) = v;
        set_summ(w, v);
      }
    }
    if (n > 8) {
#pragma unroll
      for (int k = 8; k < 16; k++) {
        if (k < n) {
          const int r = row_at(a, b, k), w = r >> 4;
          const uint32_t v = cnt(w) + (uint32_t)sign * (1u << ((r & 15) * 2));
          cnt(w) = v;
          set_summ(w, v);
        }
      }
    }
    if (sign > 0) inb(p >> 5) |= 1u << (p & 31);
    else inb(p >> 5) &= ~(1u << (p & 31));
    size += sign;
    for (int e = 0; e < n_aff; e++) {
      const long long c = I->aff_coef[e * M + p];
      aff[e] += sign * c;
      if (c < 0) aff[kMaxAffine + e] += sign * c;
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

  // Set (on) or clear Out bits of the parents in mask `m` of the row (a, b).
  __device__ __forceinline__ void out_bits(uint32_t m, const uint4 &a, const uint4 &b, bool on) {
    while (m) {
      const int s = __ffs(m) - 1;
      m &= m - 1;
      const int q = row_at(a, b, s);
      const uint32_t bit = 1u << (q & 31);
      const uint32_t v = outb(q >> 5);
      outb(q >> 5) = on ? (v | bit) : (v & ~bit);
    }
  }

  // Smallest facet g >= start in neither In nor Out, or -1.
  __device__ __forceinline__ int next_free(int start) {
    if (start >= M) return -1;
    int w = start >> 5;
    uint32_t x = ~(inb(w) | outb(w)) & (kFull << (start & 31));
    while (!x) {
      if (++w >= mw) return -1;
      x = ~(inb(w) | outb(w));
    }
    const int g = w * 32 + __ffs(x) - 1;
    return g < M ? g : -1;
  }

  __device__ void emit() {
    for (int e = 0; e < n_aff; e++)
      if ((long long)I->aff_c0[e] + aff[e] <= 0) return;
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

  // Branching of the node the state holds: a ridge level (its parents row to na, nb), or
  // (a WPM) a seed level after emitting In when `emit_ok`.
  __device__ __forceinline__ uint32_t examine(bool emit_ok, uint4 &na, uint4 &nb) {
    const int r = select_ridge();
    if (r >= 0) {
      ridge_row(r, na, nb);
      uint32_t U = 0;
#pragma unroll
      for (int s = 0; s < 8; s++) {
        const int q = row_at(na, nb, s);
        if (q != 0xFFFF && !decided(q)) U |= 1u << s;
      }
      if (pstride > 8) {
#pragma unroll
        for (int s = 8; s < 15; s++) {
          const int q = row_at(na, nb, s);
          if (q != 0xFFFF && !decided(q)) U |= 1u << s;
        }
      }
      return mk_ridge(r, U);
    }
    if (emit_ok) emit();
    return mk_seed(floor_, floor_);
  }

  // Undo the child applied under entry e (tp0/tp1 hold e's row for a ridge level).
  __device__ __forceinline__ void retreat(uint32_t e) {
    uint4 fa, fb;
    if (!(e >> 31)) {
      const int k = (e >> 15) & 15;
      const int p = row_at(tp0, tp1, k);
      facet_row(p, fa, fb);
      apply(p, fa, fb, -1);
      out_bits((e & 0x7FFFu) & ~(1u << k), tp0, tp1, false);
    } else {
      const int p = (int)(e & 0xFFF) - 1;
      facet_row(p, fa, fb);
      apply(p, fa, fb, -1);
      floor_ = (e >> 12) & 0xFFF;
    }
  }

  __device__ __forceinline__ void use_entry(uint32_t e) {
    if (!(e >> 31)) ridge_row(e >> 19, tp0, tp1);
  }

  __device__ __forceinline__ bool has_more(uint32_t e) {
    if (!(e >> 31)) {
      const int cur = (e >> 15) & 15;
      const int from = (cur == 15) ? 0 : cur + 1;
      return ((e & 0x7FFFu) >> from) != 0;
    }
    return next_free(e & 0xFFF) >= 0;
  }

  // Write the node the state holds, restricted to the untried children of entry e (tp0/tp1
  // hold e's row for a ridge level), as an open item in the reserved ring slot `slot`.
  __device__ void write_item(const PassArgs &a, unsigned long long slot, uint32_t e) {
    uint32_t *it = a.ring + (slot % a.ring_cap) * (unsigned long long)K::IW;
    const bool seed = e >> 31;
    it[0] = (uint32_t)inst;
    it[1] = kItemOpen | ((uint32_t)(seed ? (int)(e & 0xFFF) : floor_) << 16);
    it[2] = (uint32_t)size;
    it[3] = 0;
    for (int w = 0; w < mw; w++) it[kItemHeader + w] = inb(w);
    for (int w = 0; w < mw; w++) it[kItemHeader + K::MW + w] = outb(w);
    if (!seed) {
      const int cur = (e >> 15) & 15;
      if (cur != 15) {
        uint32_t tried = (e & 0x7FFFu) & ((2u << cur) - 1u);
        while (tried) {
          const int s = __ffs(tried) - 1;
          tried &= tried - 1;
          const int q = row_at(tp0, tp1, s);
          it[kItemHeader + K::MW + (q >> 5)] |= 1u << (q & 31);
        }
      }
    }
    for (int w = 0; w < nw; w++) it[kItemHeader + 2 * K::MW + w] = cnt(w);
    atomicAdd(&ctr[kCtrN * inst + kCtrLive], 1ull);
  }

  __device__ void write_empty(const PassArgs &a, unsigned long long slot) {
    uint32_t *it = a.ring + (slot % a.ring_cap) * (unsigned long long)K::IW;
    it[0] = 0;
    it[1] = kItemEmpty;
  }

  // Load an item. Returns false when a fresh root fails its checks.
  __device__ bool load(const uint32_t *it, bool &fresh) {
    const uint32_t fl = it[1];
    fresh = fl & kItemFresh;
    floor_ = (fl & kItemSeed) ? (int)(it[2] >> 16) : (int)(fl >> 16);
    nodes = probes = count = 0;
    for (int w = 0; w < mw; w++) {
      inb(w) = it[kItemHeader + w];
      outb(w) = it[kItemHeader + K::MW + w];
    }
    if (M & 31) outb(mw - 1) |= kFull << (M & 31);
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
          uint4 fa, fb;
          facet_row(j, fa, fb);
          if (!fits(fa, fb)) ok = false;
#pragma unroll
          for (int k = 0; k < 16; k++) {
            if (k < n) {
              const int r = row_at(fa, fb, k);
              cnt(r >> 4) += 1u << ((r & 15) * 2);
            }
          }
          size++;
        }
      }
      if (cap >= 0 && size > cap) ok = false;
    } else {
      size = (int)(it[2] & 0xFFFFu);
      for (int w = 0; w < nw; w++) cnt(w) = it[kItemHeader + 2 * K::MW + w];
    }
    for (int w = 0; w < nw; w++) set_summ(w, cnt(w));
    for (int e = 0; e < n_aff; e++) {
      long long si = 0, ni = 0;
      for (int w = 0; w < mw; w++) {
        uint32_t x = inb(w);
        while (x) {
          const int j = w * 32 + __ffs(x) - 1;
          x &= x - 1;
          const long long c = I->aff_coef[e * M + j];
          si += c;
          if (c < 0) ni += c;
        }
      }
      aff[e] = si;
      aff[kMaxAffine + e] = ni;
      if (fresh && I->aff_bound0[e] + ni <= 0) ok = false;
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

template <class K>
__global__ void __launch_bounds__(K::TPB) tdfs_kernel(PassArgs a) {
  extern __shared__ uint32_t smem[];
  TSearch<K> S;
  S.sm = smem + threadIdx.x;
  const int gtid = blockIdx.x * K::TPB + threadIdx.x;
  uint32_t *stk = a.stack + gtid;
  const int stride = a.n_threads;
  S.aff = a.aff_scratch + (size_t)gtid * 2 * kMaxAffine;
  const int lane = threadIdx.x & 31;
  int depth = 0;
  uint32_t top = 0;
  long long pass_nodes = 0;
  bool active = true, stop = false;
  unsigned long long t_iters = 0, t_step = 0, t_fetch = 0, t_dump = 0, t_stopped = 0;
  while (__any_sync(kFull, active)) {
    if (a.trace) {
      const unsigned act = __ballot_sync(kFull, active && !stop);
      const unsigned fetch = __ballot_sync(kFull, active && !stop && depth == 0);
      t_iters++;
      t_stopped += 32 - __popc(act);
      t_fetch += __popc(fetch);
      t_step += __popc(act & ~fetch);  // includes returning work (counted again below)
    }
    if (stop) {
      // one update per warp for the threads that stopped this iteration
      const unsigned m = __activemask();
      const unsigned done = __reduce_add_sync(m, (unsigned)pass_nodes);
      if (lane == __ffs(m) - 1) {
        atomicAdd(&a.q->idle, (unsigned long long)__popc(m));
        atomicAdd(&a.q->nodes, (unsigned long long)done);
      }
      stop = false;
      active = false;
      continue;
    }
    if (!active) continue;
    if (depth == 0) {
      if (pass_nodes >= a.budget) {
        stop = true;
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
        stop = true;  // tickets past the limit are returned by the host
        continue;
      }
      const uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
      if ((it[1] & 0xFFFFu) == kItemEmpty) continue;
      S.bind(a.inst, a.outs, a.ctr, (int)it[0]);
      bool fresh;
      if (!S.load(it, fresh)) {
        S.probes++;
        S.flush();
        continue;
      }
      if (fresh) {
        S.nodes++;
        pass_nodes++;
      }
      top = S.examine(fresh, S.tp0, S.tp1);
      depth = 1;
      continue;
    }
    const bool spent = pass_nodes >= a.budget ||
                       ((pass_nodes & 63) == 63 &&
                        *(volatile unsigned long long *)&a.q->idle >= a.idle_limit);
    // return work: reserve one ring slot per open level (a bounded compare-and-swap on the
    // tail that never passes unconsumed items); without room the search simply goes on
    unsigned long long base = ~0ull;
    if (spent) {
      unsigned long long t = *(volatile unsigned long long *)&a.q->tail;
      for (int tries = 0; tries < 64; tries++) {
        if (t + depth - a.q->head_start > a.ring_cap) break;
        const unsigned long long old = atomicCAS(&a.q->tail, t, t + depth);
        if (old == t) {
          base = t;
          break;
        }
        t = old;
      }
    }
    if (base != ~0ull) {
      // every open level's untried children go back to the ring
      if (a.trace) t_dump++;
      uint32_t e = top;
      for (int L = depth; L >= 1; L--) {
        const unsigned long long slot = base + (depth - L);
        if (S.has_more(e)) S.write_item(a, slot, e);
        else S.write_empty(a, slot);
        if (L > 1) {
          e = stk[(L - 2) * stride];
          S.use_entry(e);
          S.retreat(e);
        }
      }
      depth = 0;
      S.flush();
      stop = true;
      continue;
    }
    // One step. Either the top level has a candidate child left (try it: on success add it
    // and push), or the level is done (pop, and remove its parent's child). Both branches
    // meet in one update of the counters and of Out, so the warp's threads diverge only
    // in choosing the facet and in examining a pushed child.
    int p = -1;
    if (!(top >> 31)) {
      const uint32_t U = top & 0x7FFFu;
      const int cur = (top >> 15) & 15;
      const int from = (cur == 15) ? 0 : cur + 1;
      const uint32_t rem = (U >> from) << from;
      if (rem) {
        const int k = __ffs(rem) - 1;
        top = (top & ~(15u << 15)) | ((uint32_t)k << 15);
        p = row_at(S.tp0, S.tp1, k);
      }
    } else {
      p = S.next_free(top & 0xFFF);
      if (p >= 0) top = (top & ~0xFFFu) | (uint32_t)(p + 1);
    }
    const bool trying = p >= 0;
    if (!trying) {
      depth--;
      if (depth == 0) {
        S.flush();
        continue;
      }
      top = stk[(depth - 1) * stride];
      S.use_entry(top);
      // the child of `top` that is applied: slot cur of its ridge, or facet start - 1
      p = (top >> 31) ? (int)(top & 0xFFF) - 1 : row_at(S.tp0, S.tp1, (top >> 15) & 15);
    }
    uint4 fa, fb;
    S.facet_row(p, fa, fb);
    if (trying && !S.child_ok(p, fa, fb)) {
      S.probes++;
      continue;
    }
    const int sign = trying ? 1 : -1;
    S.apply(p, fa, fb, sign);
    if (!(top >> 31)) {
      const int k = (top >> 15) & 15;
      S.out_bits((top & 0x7FFFu) & ~(1u << k), S.tp0, S.tp1, trying);
    } else {
      S.floor_ = trying ? p : (int)((top >> 12) & 0xFFF);
    }
    if (!trying) continue;
    S.nodes++;
    pass_nodes++;
    uint4 na, nb;
    const uint32_t child = S.examine(true, na, nb);
    if (depth >= a.max_depth) {  // cannot happen when max_depth covers the facet cap
      atomicOr(&a.q->err, 2ull);
      S.retreat(top);
      continue;
    }
    stk[(depth - 1) * stride] = top;
    top = child;
    S.tp0 = na;
    S.tp1 = nb;
    depth++;
  }
  if (a.trace) {
    const unsigned long long dumps = __reduce_add_sync(kFull, (unsigned)t_dump);
    if (lane == 0) {
      atomicAdd(&a.q->iters, t_iters);
      atomicAdd(&a.q->lanes_step, t_step);
      atomicAdd(&a.q->lanes_fetch, t_fetch);
      atomicAdd(&a.q->lanes_dump, dumps);
      atomicAdd(&a.q->lanes_stopped, t_stopped);
    }
  }
}

}  // namespace ts

template <int MW, int NW, int TPB>
static cudaError_t tlaunch_t(const PassArgs &a, int grid, size_t smem, cudaStream_t s) {
  auto fn = ts::tdfs_kernel<ts::TCls<MW, NW, TPB>>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, TPB, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MW, int NW, int TPB>
static int toccupancy_t(size_t smem) {
  auto fn = ts::tdfs_kernel<ts::TCls<MW, NW, TPB>>;
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
