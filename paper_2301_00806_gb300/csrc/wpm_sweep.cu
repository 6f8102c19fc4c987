// wpm_sweep.cu -- the GF(2) cycle-space sweep of libwpm (Section 2.1, the kernel enumeration
// of Algorithm 2.2, with Section 2.1's convenient basis and Section 4.4's fixed coordinates),
// an alternative to the canonical search for maps whose incidence matrix has a small kernel.
//
// Every WPM K satisfies A K = 0 over Z2 (each ridge lies in 0 or 2 facets of K), so K is a
// GF(2) combination of a basis of ker A. Three kernels, one block per map for the first two:
//   basis_kernel       Gaussian elimination of A over GF(2) (rows in an L2-resident scratch
//                      of the workspace), one basis vector per free column;
//   convenient_kernel  the generators' final form. Rows of facets that must be in K (forced
//                      in, and the base facet when required) and rows of facets that must not
//                      be (forced out) come first in a column echelon form: a generator led
//                      by a forced-in row is fixed to 1, one led by a forced-out row to 0,
//                      and the others are zero on every forced row (Section 4.4). Among those
//                      free generators, Z blocks are formed ridge by ridge (Section 2.1):
//                      ridges with pairwise disjoint parents, the largest rank of the free
//                      generators restricted to the parents first; column elimination makes
//                      a block the identity on pivot rows of the ridge's parents and every
//                      other generator zero there, so K has |S xor c| facets on those rows
//                      (S the block generators chosen, c the fixed part there) and a WPM needs
//                      at most 2: 1 + k + C(k,2) choices for a block of k. The map's shape
//                      (fixed part plus block centres, block sizes, free generators) is kept;
//   sweep_kernel       every combination: the block digits as an odometer (each choice within
//                      Hamming distance 2 of the block's centre), the single free generators
//                      as a Gray code; each thread walks a chunk of consecutive combinations
//                      (64 to 4096 of them, so that a run has up to some 1M chunks),
//                      toggling generators and updating the ridge degrees of the facets they
//                      flip. Inside ker A every degree is even, so a combination is a WPM
//                      (Proposition 2.1) when no ridge reaches 4; it is emitted when the
//                      properties hold too. The masks go through the same per-map sort as
//                      the search's, so lists are identical.
// With engine 2 the convenient kernel keeps the plain basis: no fixed coordinates, no blocks,
// all 2^s combinations in Gray order (the forced facets are then checked per combination).
#include <cstdint>
#include <cuda_runtime.h>

#include "wpm_internal.h"

namespace wpm {

// ---------------------------------------------------------------------------------------
// basis of ker A
// ---------------------------------------------------------------------------------------

// rows: [n_ids][max_n][kSweepW] scratch; basis: [n_ids][kSweepMaxS][kSweepW]
__global__ void __launch_bounds__(512) basis_kernel(const InstDesc *insts, const int32_t *ids,
                                                    uint64_t *rows_all, int max_n,
                                                    uint64_t *basis, int32_t *dims) {
  __shared__ int piv_row;
  __shared__ int pivcol[kSweepMaxM];
  const InstDesc &I = insts[ids[blockIdx.x]];
  const int M = I.M, N = I.N, n = I.n, ow = (M + 63) >> 6;
  const int tid = threadIdx.x, nt = blockDim.x;
  uint64_t *rows = rows_all + (size_t)blockIdx.x * max_n * kSweepW;
  for (int i = tid; i < N * kSweepW; i += nt) rows[i] = 0;
  __syncthreads();
  for (int j = tid; j < M; j += nt) {
    const uint16_t *fr = I.frw + (size_t)j * I.fstride;
    for (int k = 0; k < n; k++)
      atomicOr((unsigned long long *)&rows[fr[k] * kSweepW + (j >> 6)], 1ull << (j & 63));
  }
  __syncthreads();
  // reduced row echelon form: for each column a pivot row at or below the rank, swapped up
  // and cleared from every other row
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
    if (p == N) continue;  // a free column (every thread read the same p)
    if (p != rank && tid < ow) {
      const uint64_t a = rows[p * kSweepW + tid];
      rows[p * kSweepW + tid] = rows[rank * kSweepW + tid];
      rows[rank * kSweepW + tid] = a;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt)
      if (i != rank && (rows[i * kSweepW + w] & bit))
        for (int x = w; x < ow; x++) rows[i * kSweepW + x] ^= rows[rank * kSweepW + x];
    if (tid == 0) pivcol[rank] = c;
    __syncthreads();
    rank++;
  }
  // one basis vector per free column f: bit f, and bit pivcol[i] for each pivot row i that
  // has bit f (so that A x = 0); vector t belongs to the t-th free column
  uint64_t *B = basis + (size_t)blockIdx.x * kSweepMaxS * kSweepW;
  const int s = M - rank;
  if (tid == 0) dims[blockIdx.x] = s;
  if (s > kSweepMaxS) return;
  for (int t = tid; t < s; t += nt) {
    // the t-th free column: walk the pivot list (pivcol is ascending)
    int f = 0, pi = 0, seen = -1;
    for (f = 0; f < M; f++) {
      if (pi < rank && pivcol[pi] == f) {
        pi++;
        continue;
      }
      if (++seen == t) break;
    }
    if (f >= M) continue;  // cannot happen: there are s free columns
    uint64_t v[kSweepW];
    for (int x = 0; x < kSweepW; x++) v[x] = 0;
    v[f >> 6] |= 1ull << (f & 63);
    for (int i = 0; i < rank; i++)
      if (rows[i * kSweepW + (f >> 6)] & (1ull << (f & 63)))
        v[pivcol[i] >> 6] |= 1ull << (pivcol[i] & 63);
    for (int x = 0; x < kSweepW; x++) B[t * kSweepW + x] = v[x];
  }
}

// ---------------------------------------------------------------------------------------
// the convenient basis
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ bool gbit(const uint64_t *g, int j) { return (g[j >> 6] >> (j & 63)) & 1ull; }

// Rank of the generators list[0..cnt) restricted to the rows rr[0..np): each one, as an
// np-bit vector, reduced by the independent ones kept so far (each kept vector owns its
// lowest bit, which no other kept vector has).
__device__ int restricted_rank(const uint64_t (*G)[kSweepW], const int *list, int cnt,
                               const int *rr, int np) {
  uint32_t kept[16];
  int k = 0;
  for (int u = 0; u < cnt && k < np; u++) {
    uint32_t x = 0;
    for (int a = 0; a < np; a++) x |= (uint32_t)gbit(G[list[u]], rr[a]) << a;
    for (int e = 0; e < k; e++)
      if (x & kept[e] & (~kept[e] + 1u)) x ^= kept[e];
    if (x) {
      for (int e = 0; e < k; e++)
        if (kept[e] & x & (~x + 1u)) kept[e] ^= x;
      kept[k++] = x;
    }
  }
  return k;
}

// mode 1: fixed coordinates and blocks; mode 2: the plain basis. gens: [n_ids][kSweepMaxS]
// [kSweepW], block generators first (block by block), then the single generators.
__global__ void __launch_bounds__(256) convenient_kernel(const InstDesc *insts, const int32_t *ids,
                                                         const uint64_t *basis,
                                                         const int32_t *dims, int mode,
                                                         uint64_t *gens, SweepShape *shapes) {
  __shared__ uint64_t G[kSweepMaxS][kSweepW];
  __shared__ uint64_t F[kSweepW];
  __shared__ int list[kSweepMaxS];          // unblocked free generators
  __shared__ int blk_gen[kSweepMaxS], blk_row[kSweepMaxS];
  __shared__ int8_t blk_k[kSweepMaxBlocks];
  __shared__ uint8_t used[kSweepMaxM];
  __shared__ int sh_t, sh_best, n_list, n_bg, n_blk, s_i, s_j, feasible;
  const int b = blockIdx.x;
  const InstDesc &I = insts[ids[b]];
  const int M = I.M, ow = (M + 63) >> 6;
  const int tid = threadIdx.x, nt = blockDim.x;
  SweepShape &sh = shapes[b];
  const int s = dims[b];
  if (s > kSweepMaxS) {
    if (tid == 0) {
      sh.s = s;
      sh.feasible = 0;
      sh.n_blocks = sh.n_single = sh.n_gen = 0;
    }
    return;
  }
  const uint64_t *B = basis + (size_t)b * kSweepMaxS * kSweepW;
  for (int i = tid; i < s * kSweepW; i += nt) G[i / kSweepW][i % kSweepW] = B[i];
  for (int j = tid; j < M; j += nt) used[j] = 0;
  if (tid == 0) {
    s_i = s_j = 0;
    feasible = !(I.base_req && I.base_idx < 0);
    n_bg = n_blk = 0;
  }
  __syncthreads();
  if (mode == 1) {
    // fixed coordinates: rows of I (forced in, the base facet), then of J (forced out)
    for (int pass = 0; pass < 2; pass++) {
      for (int j = 0; j < M; j++) {
        const bool in_i = (I.fin && gbit(I.fin, j)) || (I.base_req && j == I.base_idx);
        const bool in_j = I.fout && gbit(I.fout, j);
        if (pass == 0 ? !in_i : (!in_j || in_i)) continue;  // uniform over the block
        if (tid == 0) {
          sh_t = -1;
          for (int u = s_j; u < s; u++)
            if (gbit(G[u], j)) { sh_t = u; break; }
        }
        __syncthreads();
        const int t = sh_t, piv = s_j;
        __syncthreads();
        if (t < 0) continue;
        if (t != piv && tid < kSweepW) {
          const uint64_t x = G[t][tid];
          G[t][tid] = G[piv][tid];
          G[piv][tid] = x;
        }
        __syncthreads();
        for (int u = tid; u < s; u += nt)
          if (u != piv && gbit(G[u], j))
            for (int x = 0; x < kSweepW; x++) G[u][x] ^= G[piv][x];
        __syncthreads();
        if (tid == 0) {
          if (pass == 0) s_i++;
          s_j++;
        }
        __syncthreads();
      }
    }
    if (tid < kSweepW) {
      uint64_t f = 0;
      for (int u = 0; u < s_i; u++) f ^= G[u][tid];
      F[tid] = f;
    }
    __syncthreads();
    for (int j = tid; j < M; j += nt) {
      const bool in_i = (I.fin && gbit(I.fin, j)) || (I.base_req && j == I.base_idx);
      const bool in_j = I.fout && gbit(I.fout, j);
      if ((in_i && in_j) || (in_i && !gbit(F, j)) || (in_j && gbit(F, j))) feasible = 0;
    }
    if (tid == 0) {
      n_list = 0;
      for (int u = s_j; u < s; u++) list[n_list++] = u;
    }
    __syncthreads();
    // Z blocks over ridges with pairwise disjoint parents, the largest rank first (the
    // lowest ridge index on ties), while a block of two or more remains
    for (;;) {
      if (tid == 0) sh_best = -1;
      __syncthreads();
      int best_key = -1;
      for (int r = tid; r < I.N; r += nt) {
        const uint16_t *pr = I.prw + (size_t)r * I.pstride;
        int rr[16], np = 0;
        bool clash = false;
        for (int a = 0; a < I.pstride; a++) {
          const int q = pr[a];
          if (q == 0xFFFF) break;
          clash |= used[q] != 0;
          rr[np++] = q;
        }
        if (clash || np < 3) continue;
        const int k = restricted_rank(G, list, n_list, rr, np);
        if (k < 2) continue;
        const int key = (k << 16) | (0xFFFF - r);
        best_key = max(best_key, key);
      }
      atomicMax(&sh_best, best_key);
      __syncthreads();
      const int key = sh_best;
      __syncthreads();
      if (key < 0) break;
      const int r = 0xFFFF - (key & 0xFFFF);
      const uint16_t *pr = I.prw + (size_t)r * I.pstride;
      const int g0 = n_bg;
      for (int a = 0; a < I.pstride; a++) {
        const int q = pr[a];
        if (q == 0xFFFF) break;
        if (tid == 0) {
          sh_t = -1;
          for (int u = 0; u < n_list; u++)
            if (gbit(G[list[u]], q)) { sh_t = u; break; }
        }
        __syncthreads();
        const int pick = sh_t;
        __syncthreads();
        if (pick < 0) continue;
        const int t = list[pick];
        // clear row q in every other free generator: the unblocked ones and the blocks'
        for (int u = tid; u < n_list; u += nt)
          if (u != pick && gbit(G[list[u]], q))
            for (int x = 0; x < kSweepW; x++) G[list[u]][x] ^= G[t][x];
        for (int e = tid; e < n_bg; e += nt)
          if (gbit(G[blk_gen[e]], q))
            for (int x = 0; x < kSweepW; x++) G[blk_gen[e]][x] ^= G[t][x];
        __syncthreads();
        if (tid == 0) {
          blk_gen[n_bg] = t;
          blk_row[n_bg] = q;
          n_bg++;
          list[pick] = list[--n_list];
        }
        __syncthreads();
      }
      for (int a = tid; a < I.pstride; a += nt)
        if (pr[a] != 0xFFFF) used[pr[a]] = 1;
      if (tid == 0) blk_k[n_blk++] = (int8_t)(n_bg - g0);
      __syncthreads();
    }
  } else if (tid == 0) {  // the plain basis: every combination is visited and checked
    n_list = 0;
    for (int u = 0; u < s; u++) list[n_list++] = u;
    for (int x = 0; x < kSweepW; x++) F[x] = 0;
    feasible = 1;
  }
  __syncthreads();
  // output: the base (F plus each block's centre combination), then the generators
  uint64_t *out = gens + (size_t)b * kSweepMaxS * kSweepW;
  if (tid < kSweepW) {
    uint64_t f = F[tid];
    for (int e = 0; e < n_bg; e++)
      if (gbit(F, blk_row[e])) f ^= G[blk_gen[e]][tid];
    sh.base[tid] = f;
  }
  for (int i = tid; i < (n_bg + n_list) * kSweepW; i += nt) {
    const int e = i / kSweepW, x = i % kSweepW;
    out[i] = G[e < n_bg ? blk_gen[e] : list[e - n_bg]][x];
  }
  for (int l = tid; l < kSweepMaxBlocks; l += nt) sh.block_k[l] = l < n_blk ? blk_k[l] : 0;
  if (tid == 0) {
    sh.s = s;
    sh.feasible = feasible;
    sh.n_blocks = n_blk;
    sh.n_single = n_list;
    sh.n_gen = n_bg + n_list;
  }
  (void)ow;
}

// ---------------------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------------------

constexpr int kSweepTPB = 64;

// The choice a of a block of k generators, relative to its centre: 0 none, 1..k one
// generator, then the pairs (i, j), i < j, in lexicographic order.
__device__ __forceinline__ uint32_t choice_set(int a, int k) {
  if (a == 0) return 0;
  if (a <= k) return 1u << (a - 1);
  int idx = a - k - 1;
  for (int i = 0; i < k; i++) {
    const int cnt = k - 1 - i;
    if (idx < cnt) return (1u << i) | (1u << (i + 1 + idx));
    idx -= cnt;
  }
  return 0;
}

__device__ __forceinline__ int choices(int k) { return 1 + k + k * (k - 1) / 2; }

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

struct SweepThread {
  const InstDesc *I;
  uint8_t *d;  // this thread's ridge degrees, ridge r at d[r * kSweepTPB]
  uint64_t K[kSweepW];
  int size, bad, ow;

  // Flip every facet of generator g, keeping the degrees and the count of ridges at 4.
  __device__ __forceinline__ void toggle(const uint64_t *g) {
    const int n = I->n;
    for (int w = 0; w < ow; w++) {
      uint64_t x = g[w];
      while (x) {
        const int f = w * 64 + __ffsll((long long)x) - 1;
        x &= x - 1;
        const bool in = (K[w] >> (f & 63)) & 1ull;
        K[w] ^= 1ull << (f & 63);
        size += in ? -1 : 1;
        const uint16_t *fr = I->frw + (size_t)f * I->fstride;
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
};

// chunks: exclusive prefix over the maps of their chunk counts; chunk c of map j covers the
// combinations [c * L, min((c + 1) * L, total_j)), L = chunk.
__global__ void __launch_bounds__(kSweepTPB) sweep_kernel(const InstDesc *insts, const int32_t *ids,
                                                        int n_ids, const uint64_t *gens,
                                                        const SweepShape *shapes,
                                                        const unsigned long long *totals,
                                                        const unsigned long long *chunks,
                                                        unsigned long long chunk,
                                                        const OutDesc *outs,
                                                        unsigned long long *ctr) {
  extern __shared__ uint8_t deg[];  // [N_max * kSweepTPB]
  const unsigned long long g = (unsigned long long)blockIdx.x * kSweepTPB + threadIdx.x;
  if (g >= chunks[n_ids]) return;
  int lo = 0, hi = n_ids - 1;  // the map of this chunk: the last j with chunks[j] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (chunks[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  const int j = lo, id = ids[j];
  const InstDesc &I = insts[id];
  const SweepShape &sh = shapes[j];
  const uint64_t *G = gens + (size_t)j * kSweepMaxS * kSweepW;
  const int nb = sh.n_blocks, ns = sh.n_single, N = I.N;
  const uint64_t *S = G + (size_t)(sh.n_gen - ns) * kSweepW;  // the single generators
  const unsigned long long t0 = (g - chunks[j]) * chunk;
  const unsigned long long t1 = min(t0 + chunk, totals[j]);
  SweepThread T;
  T.I = &I;
  T.d = deg + threadIdx.x;
  T.ow = I.ow;
  for (int r = 0; r < N; r++) T.d[r * kSweepTPB] = 0;
  for (int x = 0; x < kSweepW; x++) T.K[x] = 0;
  T.size = 0;
  T.bad = 0;
  // the combination t0 from scratch: the base, each block's choice, the singles' Gray code
  uint64_t K0[kSweepW];
  for (int x = 0; x < kSweepW; x++) K0[x] = sh.base[x];
  int bk[kSweepMaxBlocks], digit[kSweepMaxBlocks];
  for (int l = 0; l < nb; l++) bk[l] = sh.block_k[l];
  const unsigned long long inner_mask = ns >= 64 ? ~0ull : (1ull << ns) - 1ull;
  unsigned long long o = ns >= 64 ? 0 : (t0 >> ns);
  int gb = 0;  // first generator of the block
  for (int l = 0; l < nb; l++) {
    const int k = bk[l], R = choices(k);
    digit[l] = (int)(o % (unsigned long long)R);
    o /= (unsigned long long)R;
    const uint32_t set = choice_set(digit[l], k);
    for (int e = 0; e < k; e++)
      if ((set >> e) & 1u)
        for (int x = 0; x < kSweepW; x++) K0[x] ^= G[(gb + e) * kSweepW + x];
    gb += k;
  }
  const unsigned long long i0 = t0 & inner_mask, code = i0 ^ (i0 >> 1);
  for (int e = 0; e < ns; e++)
    if ((code >> e) & 1ull)
      for (int x = 0; x < kSweepW; x++) K0[x] ^= S[e * kSweepW + x];
  T.toggle(K0);  // from the empty set: every facet of K0 added
  // the lowest block digit, which moves at every odometer step, stays in registers
  const int k0 = nb > 0 ? bk[0] : 0, R0 = choices(k0);
  int d0 = nb > 0 ? digit[0] : 0;
  uint32_t set0 = choice_set(d0, k0);
  unsigned long long count = 0;
  for (unsigned long long t = t0; t < t1; t++) {
    if (t > t0) {
      const unsigned long long i = t & inner_mask;
      if (i != 0) {
        T.toggle(S + (size_t)(__ffsll((long long)i) - 1) * kSweepW);  // Gray step
      } else {
        // the singles return to none (the Gray code's last word has only the top one), and
        // the block odometer advances
        if (ns > 0) T.toggle(S + (size_t)(ns - 1) * kSweepW);
        if (nb > 0) {
          const int a2 = d0 + 1;
          const uint32_t nset = a2 < R0 ? choice_set(a2, k0) : 0u;
          const uint32_t diff = set0 ^ nset;
          for (int e = 0; e < k0; e++)
            if ((diff >> e) & 1u) T.toggle(G + (size_t)e * kSweepW);
          set0 = nset;
          d0 = a2 < R0 ? a2 : 0;
          if (a2 == R0) {  // block 0 wrapped: the carry moves on (rarely far)
            int gl = k0;
            for (int l = 1; l < nb; l++) {
              const int k = bk[l], R = choices(k);
              const int a = digit[l], b2 = a + 1 == R ? 0 : a + 1;
              const uint32_t dl = choice_set(a, k) ^ choice_set(b2, k);
              for (int e = 0; e < k; e++)
                if ((dl >> e) & 1u) T.toggle(G + (size_t)(gl + e) * kSweepW);
              digit[l] = b2;
              gl += k;
              if (b2 != 0) break;  // no carry
            }
          }
        }
      }
    }
    if (T.bad || !props_ok(I, T.K, T.size)) continue;
    count++;
    if (I.mode == 0) {  // list mode: reserve a slot, write the mask
      const OutDesc &od = outs[id];
      const unsigned long long slot = atomicAdd(&ctr[kCtrN * id + kCtrFill], 1ull);
      if (slot < od.cap)
        for (int w = 0; w < I.ow; w++) od.out[slot * I.ow + w] = T.K[w];
    }
  }
  if (count) atomicAdd(&ctr[kCtrN * id + kCtrCount], count);
  atomicAdd(&ctr[kCtrN * id + kCtrNodes], t1 - t0);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

cudaError_t launch_kernel_basis(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                                int max_n_ridges, uint64_t *rows_scratch, uint64_t *basis,
                                int32_t *dims, cudaStream_t s) {
  if (n_ids <= 0) return cudaSuccess;
  basis_kernel<<<n_ids, 512, 0, s>>>(d_inst, d_ids, rows_scratch, max_n_ridges, basis, dims);
  return cudaGetLastError();
}

cudaError_t launch_convenient(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                              const uint64_t *basis, const int32_t *dims, int mode,
                              uint64_t *gens, SweepShape *shapes, cudaStream_t s) {
  if (n_ids <= 0) return cudaSuccess;
  convenient_kernel<<<n_ids, 256, 0, s>>>(d_inst, d_ids, basis, dims, mode, gens, shapes);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                         const uint64_t *gens, const SweepShape *shapes,
                         const unsigned long long *totals, const unsigned long long *chunks,
                         unsigned long long total_chunks, unsigned long long chunk,
                         int max_n_ridges, const OutDesc *outs, unsigned long long *ctr,
                         cudaStream_t s) {
  if (n_ids <= 0 || total_chunks == 0) return cudaSuccess;
  const size_t smem = (size_t)max_n_ridges * kSweepTPB;
  cudaError_t e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned long long grid = (total_chunks + kSweepTPB - 1) / kSweepTPB;
  sweep_kernel<<<(unsigned)grid, kSweepTPB, smem, s>>>(d_inst, d_ids, n_ids, gens, shapes, totals,
                                                       chunks, chunk, outs, ctr);
  return cudaGetLastError();
}

}  // namespace wpm
