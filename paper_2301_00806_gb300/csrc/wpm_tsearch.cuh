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
// Work moves between searches inside a pass: while searches wait for items and the ring
// holds fewer items than are waiting, a busy search gives its shallowest open levels (the
// largest untried subtrees) to the ring and goes on with the rest; items written during the
// pass carry a ready flag, so a waiting search takes them at once. A pass ends when every
// search waits or has left and no item is left, or, for a search, when its node budget or
// time is spent or the ring has no room: it then gives a few shallowest levels while the ring
// is short of items and parks the rest of its work in its own park record (node state, top
// entry, depth; the stack stays in place), to resume it at the start of the next pass.
// Giving and parking never change which nodes are searched, so counts do not depend on where
// work is split.
//
// Per-thread state lives in shared memory, word w of thread t at [w * TPB + t], so every
// dynamically indexed access of a warp hits 32 distinct banks:
//   cnt[NW]  ridge degrees, 2 bits per ridge, 16 ridges per word (values 0, 1, 2)
//   inb[MW]  In; outb[MW] Out (bits >= M set)
//   summ[SW] one bit per cnt word that holds a degree-1 ridge (three registers, s0..s2,
//            when NW <= 96)
// The stack is in global memory, entry L of thread t at [L * n_threads + t].
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {
namespace ts {

// ROWS: 0 for any instance; otherwise every instance of the launch has ridges of at most 5
// parents (m - n <= 4, Picard number 4 or less) and facet rows of at most 8 ridges (1: n <=
// 8, the second halves of the rows are never read), 9 ridges (3: n <= 9) or 12 ridges (2:
// n <= 12). The variants need fewer registers and run no predicated loop iterations that
// no instance uses.
template <int MW_, int NW_, int TPB_, int ROWS_ = 0>
struct TCls {
  static constexpr int MW = MW_, NW = NW_, TPB = TPB_;
  static constexpr bool kSmall = ROWS_ == 1;         // rows of 8
  static constexpr bool kFewParents = ROWS_ != 0;    // at most 5 parents (rows of 8)
  static constexpr int kMaxRidges = ROWS_ == 1 ? 8 : (ROWS_ == 3 ? 9 : (ROWS_ == 2 ? 12 : 16));
  static constexpr int SW = (NW + 31) / 32;
  static constexpr bool kSummReg = NW <= 96;  // the summary in up to three registers
  static constexpr int SMW = NW + 2 * MW + (kSummReg ? 0 : SW);
  static constexpr int IW = kItemHeader + 2 * MW + NW;
};

constexpr unsigned kFull = 0xFFFFFFFFu;

// word with bit `pos` replaced by the low bit of `bit`
__device__ __forceinline__ uint32_t bfi1(uint32_t word, uint32_t bit, uint32_t pos) {
  uint32_t r;
  asm("bfi.b32 %0, %1, %2, %3, 1;" : "=r"(r) : "r"(bit), "r"(word), "r"(pos));
  return r;
}

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
  uint32_t s0, s1, s2;  // the summary when it is in registers: bit w % 32 of s[w / 32]
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
  uint32_t epoch;  // the pass's ready-flag stamp

  __device__ __forceinline__ uint32_t &cnt(int w) { return sm[w * K::TPB]; }
  __device__ __forceinline__ uint32_t &inb(int w) { return sm[(K::NW + w) * K::TPB]; }
  __device__ __forceinline__ uint32_t &outb(int w) { return sm[(K::NW + K::MW + w) * K::TPB]; }
  __device__ __forceinline__ uint32_t &summw(int s) {
    return sm[(K::NW + 2 * K::MW + s) * K::TPB];
  }

  __device__ __forceinline__ void set_summ(int w, uint32_t v) {
    const uint32_t has = (v & ~(v >> 1) & 0x55555555u) != 0u;
    if (K::kSummReg) {
      const uint32_t pos = (uint32_t)w & 31u;
      if (K::NW <= 32 || w < 32) s0 = bfi1(s0, has, pos);
      else if (K::NW <= 64 || w < 64) s1 = bfi1(s1, has, pos);
      else s2 = bfi1(s2, has, pos);
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
    b = (!K::kSmall && fstride > 8) ? __ldg(row + 1) : make_uint4(0, 0, 0, 0);
  }
  __device__ __forceinline__ void ridge_row(int r, uint4 &a, uint4 &b) {
    const uint4 *row = reinterpret_cast<const uint4 *>(pr + (size_t)r * pstride);
    a = __ldg(row);
    b = (!K::kFewParents && pstride > 8) ? __ldg(row + 1) : make_uint4(kFull, kFull, kFull, kFull);
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
    if (!K::kSmall && n > 8) {
#pragma unroll
      for (int k = 8; k < K::kMaxRidges; k++) {
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
    {
      const uint32_t sb = (uint32_t)__cvta_generic_to_shared(sm);
#pragma unroll
      for (int k = 0; k < 8; k++) {
        if (k < n) {
          const int r = row_at(a, b, k), w = r >> 4;
          const uint32_t d = (uint32_t)sign << ((r & 15) * 2);
          uint32_t old;
          asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(sb + (uint32_t)w * (K::TPB * 4u)), "r"(d) : "memory");
          set_summ(w, old + d);
        }
      }
    }
    if (!K::kSmall && n > 8) {
#pragma unroll
      for (int k = 8; k < K::kMaxRidges; k++) {
        if (k < n) {
          const int r = row_at(a, b, k), w = r >> 4;
          const uint32_t v = cnt(w) + (uint32_t)sign * (1u << ((r & 15) * 2));
          cnt(w) = v;
          set_summ(w, v);
        }
      }
    }
    if (sign > 0) atomicOr(&inb(p >> 5), 1u << (p & 31));
    else atomicAnd(&inb(p >> 5), ~(1u << (p & 31)));
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
      if (s0) w = __ffs(s0) - 1;
      else if (K::NW > 32 && s1) w = 32 + __ffs(s1) - 1;
      else if (K::NW > 64 && s2) w = 64 + __ffs(s2) - 1;
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
    if (K::kFewParents) {
#pragma unroll
      for (int s = 0; s < 5; s++) {
        if ((m >> s) & 1u) {
          const int q = row_at(a, b, s);
          const uint32_t bit = 1u << (q & 31);
          const uint32_t ad = (uint32_t)__cvta_generic_to_shared(&outb(q >> 5));
          if (on) asm volatile("red.shared.or.b32 [%0], %1;" :: "r"(ad), "r"(bit) : "memory");
          else asm volatile("red.shared.and.b32 [%0], %1;" :: "r"(ad), "r"(~bit) : "memory");
        }
      }
      return;
    }
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
      for (int s = 0; s < (K::kFewParents ? 5 : 8); s++) {
        const int q = row_at(na, nb, s);
        if (q != 0xFFFF && !decided(q)) U |= 1u << s;
      }
      if (!K::kFewParents && pstride > 8) {
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
    publish(a, slot);
  }

  __device__ void write_empty(const PassArgs &a, unsigned long long slot) {
    uint32_t *it = a.ring + (slot % a.ring_cap) * (unsigned long long)K::IW;
    it[0] = 0;
    it[1] = kItemEmpty;
    publish(a, slot);
  }

  // The item in `slot` is complete: make its words visible, then raise its ready flag.
  __device__ __forceinline__ void publish(const PassArgs &a, unsigned long long slot) {
    __threadfence();
    *(volatile uint32_t *)&a.ready[slot % a.ring_cap] = epoch;
  }

  // Load an item. Returns false when a fresh root fails its checks.
  __device__ bool load(const uint32_t *it, bool &fresh) {
    const uint32_t fl = __ldcg(it + 1);
    fresh = fl & kItemFresh;
    floor_ = (fl & kItemSeed) ? (int)(__ldcg(it + 2) >> 16) : (int)(fl >> 16);
    nodes = probes = count = 0;
    for (int w = 0; w < mw; w++) {
      inb(w) = __ldcg(it + kItemHeader + w);
      outb(w) = __ldcg(it + kItemHeader + K::MW + w);
    }
    if (M & 31) outb(mw - 1) |= kFull << (M & 31);
    if (!K::kSummReg) {
      const int sw = (nw + 31) >> 5;
      for (int s = 0; s < sw; s++) summw(s) = 0;
    }
    s0 = s1 = s2 = 0;
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
      size = (int)(__ldcg(it + 2) & 0xFFFFu);
      for (int w = 0; w < nw; w++) cnt(w) = __ldcg(it + kItemHeader + 2 * K::MW + w);
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

  // Counters of the item so far; the item stays live.
  __device__ __forceinline__ void flush_stats() {
    if (count) atomicAdd(&ctr[kCtrN * inst + kCtrCount], count);
    if (nodes) atomicAdd(&ctr[kCtrN * inst + kCtrNodes], nodes);
    if (probes) atomicAdd(&ctr[kCtrN * inst + kCtrProbes], probes);
    nodes = probes = count = 0;
  }

  // The item is finished: its counters, and one live item less.
  __device__ __forceinline__ void flush() {
    flush_stats();
    atomicAdd(&ctr[kCtrN * inst + kCtrLive], (unsigned long long)-1ll);
  }

  // Save the whole search (the node it holds and its position: top entry, depth, base) in
  // the park record `rec` (word w at rec[w * st]); the stack stays where it is.
  __device__ void park_save(uint32_t *rec, int st, uint32_t top, int depth, int base) {
    uint32_t *it = rec + (size_t)kParkHeader * st;
    rec[st] = top;
    rec[2 * (size_t)st] = (uint32_t)depth | ((uint32_t)base << 16);
    rec[3 * (size_t)st] = 0;
    it[0] = (uint32_t)inst;
    it[(size_t)st] = (uint32_t)floor_;
    it[2 * (size_t)st] = (uint32_t)size;
    for (int w = 0; w < mw; w++) it[(size_t)(kItemHeader + w) * st] = inb(w);
    for (int w = 0; w < mw; w++) it[(size_t)(kItemHeader + K::MW + w) * st] = outb(w);
    for (int w = 0; w < nw; w++) it[(size_t)(kItemHeader + 2 * K::MW + w) * st] = cnt(w);
    rec[0] = 1u;
  }

  // Restore a search saved by park_save (after bind() to the instance in its item word 0).
  __device__ void park_restore(const uint32_t *rec, int st, uint32_t &top, int &depth,
                               int &base) {
    const uint32_t *it = rec + (size_t)kParkHeader * st;
    top = rec[st];
    const uint32_t d = rec[2 * (size_t)st];
    depth = (int)(d & 0xFFFFu);
    base = (int)(d >> 16);
    floor_ = (int)it[(size_t)st];
    size = (int)it[2 * (size_t)st];
    nodes = probes = count = 0;
    for (int w = 0; w < mw; w++) inb(w) = it[(size_t)(kItemHeader + w) * st];
    for (int w = 0; w < mw; w++) outb(w) = it[(size_t)(kItemHeader + K::MW + w) * st];
    if (!K::kSummReg) {
      const int sw = (nw + 31) >> 5;
      for (int s = 0; s < sw; s++) summw(s) = 0;
    }
    s0 = s1 = s2 = 0;
    for (int w = 0; w < nw; w++) {
      cnt(w) = it[(size_t)(kItemHeader + 2 * K::MW + w) * st];
      set_summ(w, cnt(w));
    }
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
    }
    use_entry(top);
  }
};

__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// PassArgs::idle_polls bounds the steps of a waiting search before it leaves the pass (a
// step takes on the order of a microsecond), PassArgs::ready_polls the polls of a ready flag
// before the item is reported lost (error 4, and the search goes on). Both only bound waits
// that end by themselves in a correct run; a search that leaves early only lowers the
// parallelism of the rest of the pass.

template <class K>
__global__ void __maxnreg__(96) tdfs_kernel(PassArgs a) {
  extern __shared__ uint32_t smem[];
  TSearch<K> S;
  S.sm = smem + threadIdx.x;
  const int gtid = blockIdx.x * K::TPB + threadIdx.x;
  uint32_t *stk = a.stack + gtid;
  const int stride = a.n_threads;
  S.aff = a.aff_scratch + (size_t)gtid * 2 * kMaxAffine;
  const int lane = threadIdx.x & 31;
  QueueCtl *q = a.q;
  const unsigned long long t_end = a.time_left_ns ? global_ns() + a.time_left_ns : ~0ull;
  // items there when the pass began (complete); later ones carry a ready flag
  const unsigned long long limit = q->limit;
  S.epoch = (uint32_t)q->epoch;
  const uint32_t want_stamp = S.epoch ^ a.ready_xor;
  const int max_ready = a.ready_polls > 0 ? a.ready_polls : kDefaultReadyPolls;
  const int max_idle = a.idle_polls > 0 ? a.idle_polls : kDefaultIdlePolls;
  // Levels 1..depth of the stack are open (entry L at stk[(L - 1) * stride], the top one in
  // `top`); levels 1..base were given away, so the item is finished when the search pops
  // back to level base.
  int depth = 0, base = 0;
  uint32_t top = 0;
  long long pass_nodes = 0, next_check = 511, next_give = 0;
  // stop: leave the pass this iteration; counted: the leaving search adds itself to
  // q->exited (a waiting search is already counted in q->waiting)
  bool active = true, stop = false, counted = false, waiting = false;
  int polls = 0;
  uint32_t *rec = a.park + gtid;
  if (rec[0]) {  // resume the search parked here at the end of the last pass
    S.bind(a.inst, a.outs, a.ctr, (int)rec[(size_t)kParkHeader * stride]);
    S.park_restore(rec, stride, top, depth, base);
    rec[0] = 0;
  }
  unsigned long long t_iters = 0, t_step = 0, t_fetch = 0, t_dump = 0, t_stopped = 0;
  while (__any_sync(kFull, active)) {
    // lanes of this warp that hold work (a warp with none backs off while it polls)
    const unsigned busy = __ballot_sync(kFull, active && !stop && depth > 0);
    if (a.trace) {
      const unsigned act = __ballot_sync(kFull, active && !stop);
      t_iters++;
      t_stopped += 32 - __popc(act);
      t_fetch += __popc(act & ~busy);
      t_step += __popc(busy);  // includes giving work away (counted again below)
    }
    if (stop) {
      // one update per warp for the searches that leave the pass this iteration
      const unsigned m = __activemask();
      const unsigned done = __reduce_add_sync(m, (unsigned)pass_nodes);
      const unsigned add = __ballot_sync(m, counted);
      if (lane == __ffs(m) - 1) {
        if (add) atomicAdd(&q->exited, (unsigned long long)__popc(add));
        atomicAdd(&q->nodes, (unsigned long long)done);
      }
      stop = false;
      active = false;
      continue;
    }
    if (!active) continue;
    if (depth == 0) {
      // ---- looking for an item
      if (pass_nodes >= a.budget || global_ns() >= t_end) {
        if (waiting) atomicAdd(&q->waiting, (unsigned long long)-1ll);
        waiting = false;
        stop = true;
        counted = true;
        continue;
      }
      if (waiting && busy && (++polls & 31)) continue;  // poll every 32nd step beside busy lanes
      // take tickets for the lanes here (warp-aggregated; never past the tail). Waiting
      // lanes stop being counted as waiting before the take, so a search that sees every
      // search waiting or gone and no item left knows that no more items can come.
      const unsigned mask = __activemask();
      const int leader = __ffs(mask) - 1;
      const unsigned n_wait = __popc(__ballot_sync(mask, waiting));
      unsigned long long h0 = 0, got = 0;
      if (lane == leader) {
        // the waiting lanes here leave the count before any take; the lanes left without
        // an item join it again after
        const unsigned want = __popc(mask);
        unsigned long long h = vload(&q->head), t = vload(&q->tail);
        bool left = false;
        if (t >= h + (unsigned long long)a.n_threads) {
          // at least one item per search: even if every other search takes a ticket
          // meanwhile, these stay below the tail, so a plain add is safe
          if (n_wait) atomicAdd(&q->waiting, (unsigned long long)-(long long)n_wait);
          left = true;
          h = atomicAdd(&q->head, (unsigned long long)want);
          got = want;
        } else {
          // few items: take at most what is there (one compare-and-swap; on a lost race
          // the lanes try again at their next poll)
          got = t > h ? t - h : 0;
          if (got > want) got = want;
          if (got) {
            if (n_wait) atomicAdd(&q->waiting, (unsigned long long)-(long long)n_wait);
            left = true;
            if (atomicCAS(&q->head, h, h + got) != h) got = 0;
          }
        }
        const unsigned long long join = (want - (unsigned)got) - (left ? 0u : n_wait);
        if (join) atomicAdd(&q->waiting, join);
        h0 = h;
      }
      h0 = __shfl_sync(mask, h0, leader);
      got = __shfl_sync(mask, got, leader);
      const unsigned rank = __popc(mask & ((1u << lane) - 1u));
      const bool mine = rank < got;
      if (!mine) {
        if (!waiting) polls = 0;
        waiting = true;
        // every search waits or has left and no item is left: the pass is over
        const unsigned long long hh = vload(&q->head), tt = vload(&q->tail);
        if (hh >= tt &&
            vload(&q->waiting) + vload(&q->exited) >= (unsigned long long)a.n_threads) {
          stop = true;  // stays counted as waiting
          counted = false;
          continue;
        }
        if (++polls >= max_idle || (vload(&q->full) && vload(&q->head) >= vload(&q->tail))) {
          atomicAdd(&q->waiting, (unsigned long long)-1ll);
          waiting = false;
          stop = true;
          counted = true;
          continue;
        }
        if (!busy) __nanosleep(64);
        continue;
      }
      waiting = false;
      const unsigned long long idx = h0 + rank;
      if (idx >= limit) {  // written during this pass: wait until it is complete
        const uint32_t *rf = a.ready + idx % a.ring_cap;
        int spins = 0;
        while (*(const volatile uint32_t *)rf != want_stamp && ++spins < max_ready)
          __nanosleep(32);
        if (spins >= max_ready) {
          atomicOr(&q->err, 4ull);
          continue;
        }
        __threadfence();
      }
      const uint32_t *it = a.ring + (idx % a.ring_cap) * (unsigned long long)K::IW;
      if ((__ldcg(it + 1) & 0xFFFFu) == kItemEmpty) continue;
      S.bind(a.inst, a.outs, a.ctr, (int)__ldcg(it));
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
      base = 0;
      continue;
    }
    // ---- every 512 nodes: end of the pass (budget, time, full ring), or hand-over
    if (pass_nodes >= next_check) {
      next_check = pass_nodes + 512;
      const bool end = pass_nodes >= a.budget || vload(&q->full) || global_ns() >= t_end;
      const unsigned long long t = vload(&q->tail), h = vload(&q->head);
      const unsigned long long items = t > h ? t - h : 0;
      int give = 0;
      if (end) {
        // leaving: give the shallowest levels while the ring is short of items
        if (items < a.hungry) give = min(a.feed, depth - base);
      } else {
        // searches are waiting and the ring cannot serve them all: give the shallowest
        // levels (the largest untried subtrees), keep the rest; at most once every
        // donate_every nodes (a hand-over walks the whole stack)
        if (pass_nodes >= next_give) {
          const unsigned long long w = vload(&q->waiting);
          if (w > items) {
            give = min(a.donate, depth - base - 1);
            next_give = pass_nodes + a.donate_every;
          }
        }
      }
      // reserve one ring slot per given level (a bounded compare-and-swap on the tail that
      // never passes items of this pass); without room nothing is given and the pass ends
      unsigned long long slot0 = ~0ull;
      if (give > 0) {
        unsigned long long tt = t;
        for (int tries = 0; tries < 64; tries++) {
          if (tt + give - a.q->head_start > a.ring_cap) {
            atomicExch(&q->full, 1ull);
            break;
          }
          const unsigned long long old = atomicCAS(&q->tail, tt, tt + give);
          if (old == tt) {
            slot0 = tt;
            break;
          }
          tt = old;
        }
        if (slot0 == ~0ull) give = 0;
      }
      if (end || give > 0) {
        const bool all = end && give == depth - base;
        // the deepest node is saved before the walk up: for good when leaving, else to
        // come back to
        if (!all) S.park_save(rec, stride, top, depth, end ? base + give : base);
        if (give > 0) {
          if (a.trace) t_dump++;
          // walk the state up from the deepest level; levels base+1 .. base+give go to the
          // ring, deepest first, each with its untried children
          const int lo = base + 1, hi = base + give;
          uint32_t e = top;
          for (int L = depth; L >= lo; L--) {
            if (L <= hi) {
              const unsigned long long slot = slot0 + (hi - L);
              if (S.has_more(e)) S.write_item(a, slot, e);
              else S.write_empty(a, slot);
            }
            if (L > lo) {
              e = stk[(L - 2) * stride];
              S.use_entry(e);
              S.retreat(e);
            }
          }
        }
        if (end) {
          if (all) {
            S.flush();
          } else {
            S.flush_stats();
            atomicAdd(&q->parked, 1ull);
          }
          depth = 0;
          base = 0;
          stop = true;
          counted = true;
          continue;
        }
        // back to the deepest node; the given levels are no longer this search's
        S.flush_stats();
        int b;
        S.park_restore(rec, stride, top, depth, b);
        rec[0] = 0;
        base = b + give;
      }
    }
    // One step. Either the top level has a candidate child left (try it: on success add it
    // and push), or the level is done (pop, and remove its parent's child), or a seed level
    // moves on to its next word. The step is one code path in four segments (choose, pop,
    // facet row + degree test + update, examine + push); the lanes that entered it meet
    // again at every segment boundary (__syncwarp), so each segment runs once for the warp
    // with whichever lanes need it, instead of once per divergent group (measured: 1.35x on
    // the batched workload). Passing over a rejected candidate inside the step was measured
    // slower: each extra table read then stalls the whole warp.
    const unsigned smask = __activemask();
    int p = -1;
    bool skip = false;
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
      // one word of the undecided facets at or above start per step
      const int start = (int)(top & 0xFFF);
      if (start < S.M) {
        const int w = start >> 5;
        const uint32_t x = ~(S.inb(w) | S.outb(w)) & (kFull << (start & 31));
        if (x) {
          p = w * 32 + __ffs(x) - 1;
          top = (top & ~0xFFFu) | (uint32_t)(p + 1);
        } else {
          const int nxt = min((w + 1) * 32, S.M);
          top = (top & ~0xFFFu) | (uint32_t)nxt;
          skip = nxt < S.M;
        }
      }
    }
    __syncwarp(smask);
    const bool trying = p >= 0;
    const bool popping = !trying && !skip;
    if (popping) {
      depth--;
      if (depth == base) {
        depth = 0;
        base = 0;
        S.flush();
      } else {
        top = stk[(depth - 1) * stride];
        S.use_entry(top);
        // the child of `top` that is applied: slot cur of its ridge, or facet start - 1
        p = (top >> 31) ? (int)(top & 0xFFF) - 1 : row_at(S.tp0, S.tp1, (top >> 15) & 15);
      }
    }
    __syncwarp(smask);
    bool acc = false;
    if (p >= 0) {
      uint4 fa, fb;
      S.facet_row(p, fa, fb);
      const bool ok = !trying || S.child_ok(p, fa, fb);
      if (!ok) S.probes++;
      if (ok) {
        S.apply(p, fa, fb, trying ? 1 : -1);
        if (!(top >> 31)) {
          const int k = (top >> 15) & 15;
          S.out_bits((top & 0x7FFFu) & ~(1u << k), S.tp0, S.tp1, trying);
        } else {
          S.floor_ = trying ? p : (int)((top >> 12) & 0xFFF);
        }
        acc = trying;
      }
    }
    __syncwarp(smask);
    if (acc) {
      S.nodes++;
      pass_nodes++;
      uint4 na, nb;
      const uint32_t child = S.examine(true, na, nb);
      if (depth >= a.max_depth) {  // cannot happen when max_depth covers the facet cap
        atomicOr(&a.q->err, 2ull);
        S.retreat(top);
      } else {
        stk[(depth - 1) * stride] = top;
        top = child;
        S.tp0 = na;
        S.tp1 = nb;
        depth++;
      }
    }
    __syncwarp(smask);
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

template <int MW, int NW, int TPB, int ROWS = 0>
static cudaError_t tlaunch_t(const PassArgs &a, int grid, size_t smem, cudaStream_t s) {
  auto fn = ts::tdfs_kernel<ts::TCls<MW, NW, TPB, ROWS>>;
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
