// wpm_internal.h -- device data layout shared by the kernels (wpm_kernels.cu) and the host
// runtime (wpm_runtime.cpp) of libwpm. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wpm {

constexpr int kMaxVertices = 16;
constexpr int kMaxFacets = 2048;
constexpr int kMaxRidges = 4096;
constexpr int kMaxAffine = 4;
constexpr int kItemHeader = 4;  // u32 words before In / Out / counters in a work item

// Per-instance error bits written by the device (InstDesc::err).
enum : uint32_t {
  kErrLimit = 1u,        // M or N above the library limits
  kErrMaskSize = 2u,     // condition masks built for another M
  kErrCapNeedsPic4 = 4u, // WPM_CAP_UBT asked for with m != n + 4
  kErrNoBase = 8u,       // (not an error: base facet missing means no outputs)
};

// Work items: u32 words [inst, flags | floor << 16, size | base << 16, acc], then In[MW],
// Out[MW], cnt[NW]. Flags (word 1, low 16 bits):
enum : uint32_t {
  kItemEmpty = 0u,      // a reserved slot left unused: readers skip it
  kItemFresh = 1u,      // a root: counters not built, not yet counted as a node
  kItemOpen = 2u,       // a counted (and, if a WPM, already emitted) node whose children
                        // have not been counted: the receiver expands it
  kItemSeed = 4u,       // a WPM node part-way through its new-lowest-facet children: they
                        // continue from the window at `base` (facets below are done)
  kItemSeedValid = 8u,  // ... whose window is already checked: `acc` holds its accepted
                        // positions not yet explored
};

// Per-instance counters (ctr[8 * inst + k]).
enum { kCtrCount = 0, kCtrNodes = 1, kCtrProbes = 2, kCtrFill = 3, kCtrLive = 4, kCtrN = 8 };

// One instance, as the device sees it. The host fills the "in" part and the arena
// pointers; the setup kernel fills the "derived" part.
struct InstDesc {
  // in
  int32_t kind, n, m, mode;  // kind: 0 primal map, 1 dual map, 2 explicit facet list
  uint32_t cols[kMaxVertices];
  int32_t cap_req;      // -1 none, -2 the Section 4.2 bound, >= 0 explicit
  int32_t base_req;     // require facet {0..n-1}
  int32_t n_facets_req; // M the condition masks were built for (-1: no masks)
  int32_t n_aff;
  int32_t nsub, nrsub;  // C(m, n), C(m, n-1): lex ranks of facets / ridges
  int32_t has_fin, has_fout;
  // arena (device pointers), sized by nsub / nrsub
  uint16_t *facets;     // [nsub] candidate vertex masks, compacted (first M valid)
  int32_t *fprefix;     // [nsub + 1] exclusive scan of the candidate flag over facet ranks
  int32_t *rprefix;     // [nrsub + 1] exclusive scan of the has-a-parent flag over ridge ranks
  uint16_t *frw;        // [nsub * fstride] row j: the n ridge indices of facet j
  uint16_t *prw;        // [nrsub * pstride] row r: the parents of ridge r, ascending facet
                        // index, padded with 0xFFFF (at most m - n + 1 <= 15 parents)
  int32_t fstride;      // 8 when n <= 8, else 16
  int32_t pstride;      // 8 when m - n + 1 <= 8, else 16
  const uint64_t *fin;  // [ceil(M/64)] forced-in mask or null
  const uint64_t *fout; // [ceil(M/64)] forced-out mask or null
  const int32_t *aff_c0;   // [n_aff]
  const int32_t *aff_coef; // [n_aff * M]
  const uint16_t *given;   // kind 2: the caller's facet list (n_given vertex masks)
  int32_t n_given, pad0;
  // derived (setup kernel)
  int32_t post;         // WPM_POST_* flags (applied to the sorted list)
  int32_t pad1;
  int32_t M, N, cap, base_idx;
  int32_t mw, nw, ow, err;
  int64_t aff_bound0[kMaxAffine];  // c0 + sum of the positive coefficients
};

// Output regions of one instance (list mode): `out` and its ping-pong twin `out2` for the
// merge sort, each `cap` masks of InstDesc::ow words.
struct OutDesc {
  uint64_t *out;
  uint64_t *out2;
  unsigned long long cap;
  unsigned long long pad;
};

// Work ring control (device). The counters that many searches update at once (head, tail,
// waiting) each have a 128-byte line of their own, away from the fields that searches only
// read while a pass runs (limit, head_start, full).
struct QueueCtl {
  alignas(128) unsigned long long head;  // next item to take (per-warp passes may overshoot
                                         // limit; per-thread passes never pass the tail)
  alignas(128) unsigned long long tail;  // next free slot
  alignas(128) unsigned long long waiting;  // per-thread passes: searches waiting for an item
  alignas(128) unsigned long long limit;    // items there when the pass began: [head_start, limit)
  unsigned long long head_start;
  unsigned long long full;        // per-thread passes: the ring had no room for given work (the
                                  // pass then ends early)
  unsigned long long epoch;       // per-thread passes: the pass's ready-flag stamp (1, 2, ...)
  unsigned long long passes;      // depth-first passes run by a graph-driven loop
  alignas(128) unsigned long long err;  // nonzero: 1 ring overflow, 2 stack overflow, 4 an
                                        // item not published within the bounded wait
  unsigned long long idle;        // per-warp passes: searches of this pass that have stopped
  unsigned long long nodes;       // nodes searched in this pass (tracing)
  unsigned long long parked;      // searches that parked their work at the end of this pass
  unsigned long long exited;      // per-thread passes: searches that have left the pass
  // tracing of per-thread passes (PassArgs::trace): warp loop iterations, and the lanes
  // that in them took a search step, fetched an item, returned work, or had stopped
  unsigned long long iters, lanes_step, lanes_fetch, lanes_dump, lanes_stopped;
};

struct PassArgs {
  const InstDesc *inst;
  const OutDesc *outs;
  unsigned long long *ctr;  // [8 * n_inst]
  uint32_t *ring;           // ring_cap items of item_words u32
  unsigned long long ring_cap;
  int item_words;
  QueueCtl *q;
  int max_depth;            // stack entries per search
  int n_threads;            // threads of a per-thread launch (stride of `stack`)
  uint32_t *stack;          // per-thread search: [max_depth * n_threads]
  long long *aff_scratch;   // per-thread search: [n_threads * 2 * kMaxAffine]
  long long budget;         // nodes per search per pass (dfs)
  int trace;                // nonzero: count loop iterations and lane activity
  int clear_expanded;       // breadth-first expansion: mark each expanded item's slot empty
                            // (items behind it in the ring are still to be taken)
  unsigned long long idle_limit;  // once this many searches of a pass have stopped, the
                                  // others return their remaining work and stop too
  unsigned long long dump_limit;  // a search returns work to the ring only while fewer
                                  // than this many items are in it (so that every search
                                  // dumping max_depth items at once still fits)
  // Parking (per-thread searches). A pass ends for a search once it has spent its budget or
  // once idle_limit searches of the pass have run out of items. The search then returns its
  // shallowest open levels to the ring (`feed` of them while the ring holds fewer than
  // `hungry` items, else `donate` of them when others are idle, else none) and parks the
  // rest: it saves its node and stack position in its park record and resumes there in the
  // next pass. Only the levels given away become ring items, so the ring stays small and a
  // search never runs on alone for want of room.
  uint32_t *park;                 // [(kParkHeader + item_words) * n_threads], word w of
                                  // thread t at [w * n_threads + t]; word 0 of each thread
                                  // zeroed before the first pass
  unsigned long long hungry;
  int donate;
  int feed;
  // In-pass hand-over (per-thread searches): an item written during a pass is published by
  // storing the pass's epoch (QueueCtl::epoch) in ready[slot] after its words; a search that
  // takes a ticket at or past `limit` waits (bounded) for that before reading it. Epochs only
  // grow over the life of the buffer, so stale flags never match.
  uint32_t *ready;                // [ring_cap]
  int rows;                       // per-thread passes, 128 threads: when every instance has
                                  // at most 5 parents per ridge, 1 for n <= 8, 3 for n <= 9,
                                  // 2 for n <= 12 (specialised kernels); else 0
  int donate_every;               // nodes a search searches between two hand-overs
  unsigned long long time_left_ns;  // > 0: searches leave the pass (parking their work) this
                                    // long after it started
  int ready_polls;                // polls of a ready flag before the item is reported lost
                                  // (0: kDefaultReadyPolls)
  int idle_polls;                 // fruitless steps before a waiting search leaves the pass
                                  // (0: kDefaultIdlePolls)
  uint32_t ready_xor;             // test hook: readers wait for epoch ^ ready_xor (0 in use)
  int pad2;
};

// Defaults of PassArgs::ready_polls / idle_polls.
constexpr int kDefaultReadyPolls = 1 << 22;
constexpr int kDefaultIdlePolls = 1 << 14;

// Park record header words (before the item words of the parked node).
constexpr int kParkHeader = 4;  // valid, top entry, depth | base << 16, unused

// GF(2) cycle-space sweep (wpm_sweep.cu): maps with M <= kSweepMaxM candidate facets and
// N <= kSweepMaxN ridges whose kernel has dimension s <= kSweepMaxS.
constexpr int kSweepW = 14;         // u64 words of a facet set
constexpr int kSweepMaxM = 64 * kSweepW;
constexpr int kSweepMaxN = 3200;    // ridge degrees of 64 threads in shared memory
constexpr int kSweepMaxS = 64;
constexpr int kSweepMaxBlocks = 32;  // Z blocks of two or more generators: at most s / 2
constexpr unsigned long long kSweepChunkMax = 4096;  // combinations per sweep thread, at most

// Shape of a map's generators after Section 4.4's fixed coordinates and Section 2.1's Z
// blocks: the sweep visits base + (at most two generators of each block) + (any of the
// single generators); gens holds the block generators block by block, then the singles.
struct SweepShape {
  int32_t s;         // dim ker A
  int32_t feasible;  // the fixed coordinates satisfy every forced row
  int32_t n_blocks, n_single, n_gen, pad[3];
  int8_t block_k[kSweepMaxBlocks];
  uint64_t base[kSweepW];  // the fixed part plus each block's centre combination
};

// Basis of ker A over GF(2) for maps ids[0..n_ids): rows_scratch holds n_ids x max_n_ridges
// x kSweepW words; basis[j] receives kSweepMaxS vectors of kSweepW words, dims[j] the
// dimension (vectors stored only when it is <= kSweepMaxS).
cudaError_t launch_kernel_basis(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                                int max_n_ridges, uint64_t *rows_scratch, uint64_t *basis,
                                int32_t *dims, cudaStream_t s);
// The generators' final form (mode 1: fixed coordinates and Z blocks; mode 2: the plain
// basis, every generator single): gens[j] (kSweepMaxS x kSweepW words) and shapes[j].
cudaError_t launch_convenient(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                              const uint64_t *basis, const int32_t *dims, int mode,
                              uint64_t *gens, SweepShape *shapes, cudaStream_t s);
// Every combination of each map (totals[j] of them) in chunks of `chunk` consecutive ones (a
// thread each); chunks is the exclusive prefix of the maps' chunk counts (n_ids + 1 entries,
// the last = total_chunks).
cudaError_t launch_sweep(const InstDesc *d_inst, const int32_t *d_ids, int n_ids,
                         const uint64_t *gens, const SweepShape *shapes,
                         const unsigned long long *totals, const unsigned long long *chunks,
                         unsigned long long total_chunks, unsigned long long chunk,
                         int max_n_ridges, const OutDesc *outs, unsigned long long *ctr,
                         cudaStream_t s);

// Post-filters of Algorithm 4.4 (wpm_post.cu) over the sorted lists of the instances
// sid[0..ns) (masks [seg[j], seg[j+1]) of the flat order): keep[g] = 1 for each mask g that
// passes its instance's WPM_POST_* flags (1 for instances without flags); then each flagged
// instance's list is compacted in order and its count and fill counters set to the kept
// number. Maps with m <= kPostMaxM.
constexpr int kPostMaxM = 15;
cudaError_t launch_post_filter(const InstDesc *d_inst, const OutDesc *outs, const int32_t *sid,
                               int ns, const unsigned long long *seg, unsigned long long total,
                               uint8_t *keep, cudaStream_t s);
cudaError_t launch_post_compact(const InstDesc *d_inst, const OutDesc *outs, const int32_t *sid,
                                int ns, const unsigned long long *seg, const uint8_t *keep,
                                unsigned long long *ctr, cudaStream_t s);

// PassArgs::rows for a launch whose largest n is max_n and whose largest parent count of a
// ridge is at most max_parents (m - n + 1 bounds it; 5 for Picard number 4).
inline int rows_variant(int max_n, int max_parents) {
  if (max_parents > 5) return 0;
  return max_n <= 8 ? 1 : (max_n <= 9 ? 3 : (max_n <= 12 ? 2 : 0));
}

// Launchers (wpm_kernels.cu). All return cudaError_t of the launch.
// One-thread kernels of a graph-driven pass loop: prep makes the items left by the last pass
// this pass's and clears the pass counters; check sets the loop's condition h.
cudaError_t launch_pass_prep(QueueCtl *q, int thread_mode, cudaStream_t s);
cudaError_t launch_pass_check(QueueCtl *q, int thread_mode, cudaGraphConditionalHandle h,
                              unsigned long long max_passes, cudaStream_t s);
// One-thread kernel after each level of a graph-driven breadth-first expansion: the level's
// children become the next level's items, and h is set while another level is wanted.
cudaError_t launch_expand_check(QueueCtl *q, cudaGraphConditionalHandle h,
                                unsigned long long target, unsigned long long max_children,
                                unsigned long long ring_cap, unsigned long long max_levels,
                                cudaStream_t s);
cudaError_t launch_setup(InstDesc *d_inst, int n_inst, cudaStream_t s);
// The setup kernel over the instances d_inst[d_ids[0..n_ids)] only.
cudaError_t launch_setup_ids(InstDesc *d_inst, const int32_t *d_ids, int n_ids, cudaStream_t s);
cudaError_t launch_roots(const InstDesc *d_inst, int n_ids, const int32_t *d_ids,
                         unsigned long long *ctr, uint32_t *ring, unsigned long long ring_cap,
                         int item_words, int cls_mw, QueueCtl *q, cudaStream_t s);

// A kernel size class: compile-time maxima of the u32 words of a facet bitset (mw) and
// of the packed 2-bit ridge counters (nw).
struct SizeClass { int mw, nw; };
int n_size_classes();
SizeClass size_class(int k);
int pick_size_class(int mw, int nw);  // smallest class that holds both, or -1
int item_words_for(int k);            // kItemHeader + 2 * mw + nw of class k
int state_words(int k);               // shared u32 words of one warp search's state
int tstate_words(int k);              // shared u32 words of one thread search's state

// Search modes of the depth-first passes.
enum { kSearchThread = 1, kSearchWarp = 2 };

// Breadth-first expansion: one warp per item; tpb a multiple of 32 (at most 256).
cudaError_t launch_expand(int k, const PassArgs &a, int n_items, int tpb, cudaStream_t s);
// The same over the queue's items [head_start, limit), read on the device, by the warps of a
// grid of `blocks` blocks of 256 threads (a level of the graph-driven expansion loop).
cudaError_t launch_expand_queued(int k, const PassArgs &a, int blocks, cudaStream_t s);
// Depth-first pass in the given search mode (tpb 64, 128 or 256).
cudaError_t launch_dfs(int k, int search, const PassArgs &a, int blocks, int tpb, cudaStream_t s);
size_t dfs_smem_bytes(int k, int search, int tpb, int max_depth);
int dfs_max_blocks_per_sm(int k, int search, int tpb, int max_depth);

// One merge pass over the masks of instances d_ids[0..n_ids): instance d_ids[s] holds
// d_seg[s+1] - d_seg[s] masks; parity 0 merges out -> out2, 1 merges out2 -> out.
cudaError_t launch_sort_pass(const InstDesc *d_inst, const OutDesc *d_outs, const int32_t *d_ids,
                             int n_ids, const unsigned long long *d_seg, unsigned long long total,
                             unsigned long long run, int parity, cudaStream_t s);

// Record the calling thread's last error (wpm_last_error) and return `code`.
int set_last_error(int code, const char *msg);
// Forget the calling thread's last error (every entry point does this first).
void clear_last_error();

// Copy segment s: prefix[s+1] - prefix[s] words from src to dst (device pointers).
struct CopySeg {
  const uint64_t *src;
  uint64_t *dst;
};
cudaError_t launch_segment_copy(const CopySeg *d_segs, int n_segs, const unsigned long long *d_prefix,
                                unsigned long long total_words, cudaStream_t s);

}  // namespace wpm
