// wpm_engine.cpp -- the serving engine of libwpm: continuous batching of enumeration jobs.
//
// An engine keeps one work ring resident on the device and a fixed number of job slots.
// Each step (wpm_engine_step):
//   1. admits queued jobs in arrival order while a slot is free and the job's output
//      region fits in the engine's output memory (admission by device memory);
//   2. builds the new jobs' candidate facets and incidence tables (setup kernel over their
//      slots) and puts their roots in the ring, next to the items of jobs already running;
//   3. runs one search pass: every search resumes the work it parked at the end of the last
//      pass or takes items from the ring, whatever job they belong to, until it has spent
//      its node budget; then it parks what is left (or, while the ring is short of items,
//      returns it there), so a pass is bounded in time and the ring stays small;
//   4. retires the jobs none of whose items are left (their per-slot live counter is zero):
//      sorts their lists on the GPU, copies them to the host and frees slot and memory.
// A job therefore overlaps on the GPU with whatever else is resident, and its result is the
// one wpm_enumerate gives (the same kernels, the same canonical tree).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_host.h"
#include "wpm_internal.h"

namespace wpm {

namespace {

long long binom_e(int a, int b) {
  if (b < 0 || b > a) return 0;
  long long r = 1;
  for (int i = 0; i < b; i++) r = r * (a - i) / (i + 1);
  return r;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes of one instance's setup tables (facets, rank prefix sums, incidence rows).
size_t table_bytes(int n, int m) {
  const size_t nsub = binom_e(m, n), nrsub = binom_e(m, n - 1);
  return a256(2 * nsub) + a256(4 * (nsub + 1)) + a256(4 * (nrsub + 1)) + a256(32 * nsub) +
         a256(32 * nrsub);
}

// Class of the largest Picard-4 instance with facet size max_n (see wpm_classes.h).
int class_for_n(int max_n) {
  if (max_n <= 3) return 0;
  if (max_n <= 5) return 1;
  if (max_n <= 11) return max_n - 4;
  return 8;
}

constexpr size_t kCondSlotBytes = 2 * 32 * 8 + kMaxAffine * 4 * (1 + kMaxFacets);

struct Job {
  uint64_t id = 0;
  HostInst hi;
  int mode = WPM_MODE_COUNT;
  uint64_t out_cap = 0;
  int slot = -1;
  int status = WPM_OK;
  int done = 0;
  uint64_t count = 0, nodes = 0, probes = 0;
  int M = 0, N = 0, ow = 1;
  size_t pool_off = 0, pool_bytes = 0;
  uint64_t *masks = nullptr;  // count * ow words (list mode): a block of the engine's host cache
  size_t masks_block = 0;     // that block's size class in bytes (0: no block)
};

// Finished jobs' sorted lists wait in page-locked host blocks until wpm_engine_result copies
// them out: copies into page-locked memory run at the link's full rate, several times faster
// than into pageable memory, and the blocks are reused from job to job (power-of-two size
// classes from 64 KiB; at most kHostCacheBytes kept free) so that page locking, which costs
// milliseconds per call, is paid only while the cache warms up. A block that cannot be locked
// falls back to ordinary memory.
constexpr size_t kHostCacheBytes = 4ull << 30;

struct HostCache {
  std::map<size_t, std::vector<void *>> spare;  // size class -> blocks not in use
  std::map<void *, bool> locked;               // every block handed out or free: page-locked?
  size_t free_bytes = 0;
  static size_t size_class(size_t bytes) {
    size_t c = 64 * 1024;
    while (c < bytes) c *= 2;
    return c;
  }
  void *take(size_t bytes, size_t &cls) {
    cls = size_class(bytes);
    auto it = spare.find(cls);
    if (it != spare.end() && !it->second.empty()) {
      void *p = it->second.back();
      it->second.pop_back();
      free_bytes -= cls;
      return p;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, cls, cudaHostAllocDefault) == cudaSuccess) {
      locked[p] = true;
      return p;
    }
    cudaGetLastError();
    p = malloc(cls);
    if (p) locked[p] = false;
    return p;
  }
  void drop(void *p) {
    auto it = locked.find(p);
    if (it == locked.end()) return;
    if (it->second) cudaFreeHost(p);
    else free(p);
    locked.erase(it);
  }
  void give(void *p, size_t cls) {
    if (!p) return;
    if (free_bytes + cls > kHostCacheBytes) {
      drop(p);
      return;
    }
    spare[cls].push_back(p);
    free_bytes += cls;
  }
  void release_all() {
    std::vector<void *> all;
    for (auto &kv : locked) all.push_back(kv.first);
    for (void *p : all) drop(p);
    spare.clear();
    free_bytes = 0;
  }
};

}  // namespace
}  // namespace wpm

using namespace wpm;

struct wpm_engine {
  int device = 0, sms = 0;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  int k = 0, search = kSearchThread, tpb = 128, blocks = 0, n_searches = 0, max_depth = 0, iw = 0;
  int max_jobs = 0, max_n = 0;
  long long budget = 4096;
  int slice_ms = 0;  // > 0: passes also end after this many milliseconds; 0: by load; < 0: none
  size_t slot_bytes = 0;
  unsigned long long ring_cap = 0, dump_limit = 0, idle_limit = 1, hungry = 1;
  unsigned long long parked = 0;  // searches holding parked work after the last pass
  unsigned long long pass_nodes = 0;
  DevBuf inst, outd, ctr, tables, cond, ring, ready, stack, aff, q, ids, seg, pool, park;
  uint32_t epoch = 0;
  PinBuf h_inst, h_outd, h_ctr, h_q, h_ids, h_seg, h_cond;
  HostCache host_lists;
  size_t pool_bytes = 0;
  std::map<size_t, size_t> free_blocks;  // output pool: offset -> bytes
  std::deque<Job *> pending;
  std::vector<Job *> slots;
  std::map<uint64_t, Job *> jobs;
  std::deque<uint64_t> finished;
  uint64_t next_id = 1;
  unsigned long long head = 0, tail = 0;

  bool pool_alloc(size_t bytes, size_t &off) {
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second < bytes) continue;
      off = it->first;
      const size_t rest = it->second - bytes;
      free_blocks.erase(it);
      if (rest) free_blocks[off + bytes] = rest;
      return true;
    }
    return false;
  }
  void pool_free(size_t off, size_t bytes) {
    if (!bytes) return;
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
};

namespace {

void finish(wpm_engine *e, Job *j, int status) {
  j->status = status;
  j->done = 1;
  if (j->slot >= 0) e->slots[j->slot] = nullptr;
  j->slot = -1;
  e->pool_free(j->pool_off, j->pool_bytes);
  j->pool_bytes = 0;
  e->finished.push_back(j->id);
}

int admit(wpm_engine *e) {
  std::vector<int32_t> fresh;
  for (int sl = 0; sl < e->max_jobs && !e->pending.empty(); sl++) {
    if (e->slots[sl]) continue;
    Job *j = e->pending.front();
    const HostInst &h = j->hi;
    if (table_bytes(h.n, h.m) > e->slot_bytes || h.n > e->max_n) {
      e->pending.pop_front();
      finish(e, j, fail(WPM_ERR_LIMIT, "job %llu: larger than the engine's max_n",
                        (unsigned long long)j->id));
      sl--;
      continue;
    }
    if (j->mode == WPM_MODE_LIST) {
      const size_t words = (binom_e(h.m, h.n) + 63) / 64;  // ceil(M/64) is at most this
      j->pool_bytes = a256(2 * 8 * words * std::max<uint64_t>(j->out_cap, 1));
      if (!e->pool_alloc(j->pool_bytes, j->pool_off)) {
        j->pool_bytes = 0;
        break;  // the oldest job waits until memory frees up
      }
    }
    e->pending.pop_front();
    j->slot = sl;
    e->slots[sl] = j;
    fresh.push_back(sl);
  }
  if (fresh.empty()) return WPM_OK;

  InstDesc *hd = e->h_inst.as<InstDesc>();
  char *tb = e->tables.as<char>(), *cb = e->cond.as<char>(), *hc = e->h_cond.as<char>();
  for (int sl : fresh) {
    Job *j = e->slots[sl];
    const HostInst &h = j->hi;
    InstDesc &d = hd[sl];
    memset(&d, 0, sizeof(d));
    d.kind = h.kind; d.n = h.n; d.m = h.m; d.mode = j->mode;
    for (int v = 0; v < kMaxVertices; v++) d.cols[v] = h.cols[v];
    d.cap_req = h.cap_req; d.base_req = h.base_req; d.n_facets_req = h.n_facets_req;
    d.n_aff = h.n_aff;
    d.nsub = (int)binom_e(h.m, h.n);
    d.nrsub = (int)binom_e(h.m, h.n - 1);
    d.has_fin = !h.fin.empty();
    d.has_fout = !h.fout.empty();
    char *t = tb + (size_t)sl * e->slot_bytes;
    auto take = [&](size_t bytes) { char *p = t; t += a256(bytes); return p; };
    d.facets = (uint16_t *)take(2 * (size_t)d.nsub);
    d.fprefix = (int32_t *)take(4 * ((size_t)d.nsub + 1));
    d.rprefix = (int32_t *)take(4 * ((size_t)d.nrsub + 1));
    d.frw = (uint16_t *)take(32 * (size_t)d.nsub);
    d.prw = (uint16_t *)take(32 * (size_t)d.nrsub);
    const size_t co = (size_t)sl * kCondSlotBytes;
    size_t c = 0;
    auto put = [&](const void *src, size_t bytes) -> const void * {
      if (!bytes) return nullptr;
      memcpy(hc + co + c, src, bytes);
      const void *p = cb + co + c;
      c += (bytes + 15) & ~(size_t)15;
      return p;
    };
    d.fin = (const uint64_t *)put(h.fin.data(), 8 * h.fin.size());
    d.fout = (const uint64_t *)put(h.fout.data(), 8 * h.fout.size());
    d.aff_c0 = (const int32_t *)put(h.c0.data(), 4 * h.c0.size());
    d.aff_coef = (const int32_t *)put(h.coef.data(), 4 * h.coef.size());
    if (c) CUDA_TRY(cudaMemcpyAsync(cb + co, hc + co, c, cudaMemcpyHostToDevice, e->s));
    CUDA_TRY(cudaMemcpyAsync(e->inst.as<InstDesc>() + sl, &d, sizeof(InstDesc),
                             cudaMemcpyHostToDevice, e->s));
  }
  int32_t *hid = e->h_ids.as<int32_t>();
  for (size_t i = 0; i < fresh.size(); i++) hid[i] = fresh[i];
  CUDA_TRY(cudaMemcpyAsync(e->ids.p, hid, 4 * fresh.size(), cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(launch_setup_ids(e->inst.as<InstDesc>(), e->ids.as<int32_t>(), (int)fresh.size(), e->s));
  for (int sl : fresh)
    CUDA_TRY(cudaMemcpyAsync(hd + sl, e->inst.as<InstDesc>() + sl, sizeof(InstDesc),
                             cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));

  OutDesc *ho = e->h_outd.as<OutDesc>();
  const SizeClass cls = size_class(e->k);
  std::vector<int32_t> roots;
  for (int sl : fresh) {
    Job *j = e->slots[sl];
    const InstDesc &d = hd[sl];
    j->M = d.M; j->N = d.N; j->ow = d.ow;
    int st = WPM_OK;
    if (d.err & kErrLimit) st = fail(WPM_ERR_LIMIT, "job: M or N above the library limits");
    else if (d.err & kErrMaskSize) st = fail(WPM_ERR_INPUT, "job: conditions built for another M");
    else if (d.err & kErrCapNeedsPic4) st = fail(WPM_ERR_INPUT, "job: WPM_CAP_UBT needs m = n + 4");
    else if (d.kind != 2 && d.M == 0) st = fail(WPM_ERR_INPUT, "job: the map's rank is too small");
    else if (d.mw > cls.mw || d.nw > cls.nw)
      st = fail(WPM_ERR_LIMIT, "job: larger than the engine's kernel size class");
    else if ((d.cap >= 0 ? std::min(d.cap, d.M) : d.M) + 2 > e->max_depth)
      st = fail(WPM_ERR_LIMIT, "job: deeper than the engine's search stack");
    if (st != WPM_OK) {
      finish(e, j, st);
      continue;
    }
    OutDesc &o = ho[sl];
    memset(&o, 0, sizeof(o));
    if (j->mode == WPM_MODE_LIST) {
      char *base = e->pool.as<char>() + j->pool_off;
      o.out = (uint64_t *)base;
      o.out2 = (uint64_t *)(base + j->pool_bytes / 2);
      o.cap = j->out_cap;
    }
    CUDA_TRY(cudaMemcpyAsync(e->outd.as<OutDesc>() + sl, &o, sizeof(OutDesc),
                             cudaMemcpyHostToDevice, e->s));
    CUDA_TRY(cudaMemsetAsync(e->ctr.as<unsigned long long>() + kCtrN * sl, 0, 8 * kCtrN, e->s));
    roots.push_back(sl);
  }
  if (roots.empty()) return WPM_OK;
  for (size_t i = 0; i < roots.size(); i++) hid[i] = roots[i];
  CUDA_TRY(cudaMemcpyAsync(e->ids.p, hid, 4 * roots.size(), cudaMemcpyHostToDevice, e->s));
  QueueCtl *hq = e->h_q.as<QueueCtl>();
  memset(hq, 0, sizeof(QueueCtl));
  hq->head = e->head;
  hq->tail = e->tail;
  hq->limit = e->tail;
  hq->head_start = e->head;
  CUDA_TRY(cudaMemcpyAsync(e->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(launch_roots(e->inst.as<InstDesc>(), (int)roots.size(), e->ids.as<int32_t>(),
                        e->ctr.as<unsigned long long>(), e->ring.as<uint32_t>(), e->ring_cap,
                        e->iw, cls.mw, e->q.as<QueueCtl>(), e->s));
  CUDA_TRY(cudaMemcpyAsync(hq, e->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  if (hq->err) return fail(WPM_ERR_NOMEM, "engine work ring overflow");
  const unsigned long long roots_at = e->tail;
  e->tail = hq->tail;

  // One breadth-first level over the new roots: a new job enters its first pass as its root's
  // children (up to M items, one per lowest facet), taken by as many searches at once, instead
  // of as one item that spreads only as fast as searches hand work over. The roots' slots are
  // marked empty. A root has at most M children, so the ring has room when this holds:
  unsigned long long children = 0;
  for (int sl : roots) children += (unsigned long long)e->slots[sl]->M + 1;
  if (e->tail - e->head + children > e->ring_cap) return WPM_OK;  // left as roots
  PassArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.inst = e->inst.as<InstDesc>();
  pa.outs = e->outd.as<OutDesc>();
  pa.ctr = e->ctr.as<unsigned long long>();
  pa.ring = e->ring.as<uint32_t>();
  pa.ring_cap = e->ring_cap;
  pa.item_words = e->iw;
  pa.q = e->q.as<QueueCtl>();
  pa.max_depth = e->max_depth;
  pa.clear_expanded = 1;
  memset(hq, 0, sizeof(QueueCtl));
  hq->head = e->head;
  hq->tail = e->tail;
  hq->limit = e->tail;
  hq->head_start = roots_at;  // the items expanded: [roots_at, roots_at + roots)
  CUDA_TRY(cudaMemcpyAsync(e->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(launch_expand(e->k, pa, (int)roots.size(), 256, e->s));
  CUDA_TRY(cudaMemcpyAsync(hq, e->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  if (hq->err) return fail(WPM_ERR_NOMEM, "engine work ring overflow");
  e->tail = hq->tail;
  return WPM_OK;
}

int pass(wpm_engine *e) {
  e->pass_nodes = 0;
  if (e->tail <= e->head && e->parked == 0) return WPM_OK;
  PassArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.inst = e->inst.as<InstDesc>();
  pa.outs = e->outd.as<OutDesc>();
  pa.ctr = e->ctr.as<unsigned long long>();
  pa.ring = e->ring.as<uint32_t>();
  pa.ring_cap = e->ring_cap;
  pa.item_words = e->iw;
  pa.q = e->q.as<QueueCtl>();
  pa.max_depth = e->max_depth;
  pa.n_threads = e->blocks * e->tpb;
  pa.stack = e->stack.as<uint32_t>();
  pa.aff_scratch = e->aff.as<long long>();
  pa.budget = e->budget;
  // the slice by load: when fewer than half the searches parked work at the end of the last
  // pass the GPU has room, and 50 ms slices admit and retire jobs sooner; under load 100 ms
  // slices park and resume the searches half as often (measured on the serving stream:
  // 60 jobs/s p50 0.41 s with 50 ms, 0.49 s with 100 ms; 200 jobs/s 6.3e9 and 6.5e9 nodes/s)
  const int slice = e->slice_ms > 0 ? e->slice_ms
                    : e->slice_ms < 0 ? 0
                                      : (2 * e->parked < (unsigned long long)e->n_searches ? 50 : 100);
  pa.time_left_ns = (unsigned long long)slice * 1000000ull;
  pa.idle_limit = e->idle_limit;
  pa.dump_limit = e->dump_limit;
  {  // the row variant the resident jobs allow (m - n + 1 bounds a ridge's parents)
    int max_n = 0, max_par = 0;
    for (Job *j : e->slots) {
      if (!j) continue;
      max_n = std::max(max_n, j->hi.n);
      max_par = std::max(max_par, j->hi.m - j->hi.n + 1);
    }
    pa.rows = e->tpb == 128 ? rows_variant(max_n, max_par) : 0;
  }
  pa.park = e->park.as<uint32_t>();
  pa.ready = e->ready.as<uint32_t>();

  pa.hungry = e->hungry;
  pa.feed = 8;
  pa.donate = 4;
  pa.donate_every = 2048;
  QueueCtl *hq = e->h_q.as<QueueCtl>();
  memset(hq, 0, sizeof(QueueCtl));
  hq->head = e->head;
  hq->tail = e->tail;
  hq->limit = e->tail;
  hq->head_start = e->head;
  hq->epoch = ++e->epoch;
  CUDA_TRY(cudaMemcpyAsync(e->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, e->s));
  CUDA_TRY(launch_dfs(e->k, e->search, pa, e->blocks, e->tpb, e->s));
  CUDA_TRY(cudaMemcpyAsync(hq, e->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  if (hq->err & 1ull) return fail(WPM_ERR_NOMEM, "engine work ring overflow");
  if (hq->err & 2ull) return fail(WPM_ERR_LIMIT, "engine search stack overflow");
  if (hq->err & 4ull)
    return fail(WPM_ERR_TIMEOUT, "engine: a work item was not published within the bounded wait");
  e->head = std::min(hq->head, hq->tail);  // items written during the pass are taken too
  e->tail = hq->tail;
  e->parked = hq->parked;
  e->pass_nodes = hq->nodes;
  return WPM_OK;
}

int retire(wpm_engine *e) {
  std::vector<int> active;
  for (int sl = 0; sl < e->max_jobs; sl++)
    if (e->slots[sl]) active.push_back(sl);
  if (active.empty()) return WPM_OK;
  unsigned long long *hc = e->h_ctr.as<unsigned long long>();
  CUDA_TRY(cudaMemcpyAsync(hc, e->ctr.p, 8ull * kCtrN * e->max_jobs, cudaMemcpyDeviceToHost, e->s));
  CUDA_TRY(cudaStreamSynchronize(e->s));
  std::vector<Job *> done, to_sort;
  std::vector<unsigned long long> seg(1, 0);
  unsigned long long max_len = 0;
  for (int sl : active) {
    const unsigned long long *c = hc + kCtrN * sl;
    if (c[kCtrLive] != 0) continue;
    Job *j = e->slots[sl];
    j->count = c[kCtrCount];
    j->nodes = c[kCtrNodes];
    j->probes = c[kCtrProbes];
    done.push_back(j);
    if (j->mode == WPM_MODE_LIST && j->count > 0 && j->count <= j->out_cap) {
      to_sort.push_back(j);
      seg.push_back(seg.back() + j->count);
      max_len = std::max<unsigned long long>(max_len, j->count);
    }
  }
  if (!to_sort.empty()) {
    const int ns = (int)to_sort.size();
    WPM_TRY(e->seg.ensure(8ull * (ns + 1)));
    WPM_TRY(e->h_seg.ensure(8ull * (ns + 1) + 4ull * ns));
    unsigned long long *hs = e->h_seg.as<unsigned long long>();
    int32_t *hid = (int32_t *)(hs + ns + 1);
    for (int i = 0; i <= ns; i++) hs[i] = seg[i];
    for (int i = 0; i < ns; i++) hid[i] = to_sort[i]->slot;
    CUDA_TRY(cudaMemcpyAsync(e->seg.p, hs, 8ull * (ns + 1), cudaMemcpyHostToDevice, e->s));
    CUDA_TRY(cudaMemcpyAsync(e->ids.p, hid, 4ull * ns, cudaMemcpyHostToDevice, e->s));
    int parity = 0;
    for (unsigned long long run = 1; run < max_len; run *= 2) {
      CUDA_TRY(launch_sort_pass(e->inst.as<InstDesc>(), e->outd.as<OutDesc>(), e->ids.as<int32_t>(),
                                ns, e->seg.as<unsigned long long>(), seg.back(), run, parity, e->s));
      parity ^= 1;
    }
    if (parity)
      CUDA_TRY(launch_sort_pass(e->inst.as<InstDesc>(), e->outd.as<OutDesc>(), e->ids.as<int32_t>(),
                                ns, e->seg.as<unsigned long long>(), seg.back(), 1ull << 62, 1, e->s));
    for (Job *j : to_sort) {
      const size_t bytes = 8 * j->count * j->ow;
      j->masks = (uint64_t *)e->host_lists.take(bytes, j->masks_block);
      if (!j->masks) return fail(WPM_ERR_NOMEM, "no host memory for a job's list (%zu bytes)", bytes);
      CUDA_TRY(cudaMemcpyAsync(j->masks, e->pool.as<char>() + j->pool_off, bytes,
                               cudaMemcpyDeviceToHost, e->s));
    }
    CUDA_TRY(cudaStreamSynchronize(e->s));
  }
  for (Job *j : done) {
    const bool over = j->mode == WPM_MODE_LIST && j->count > j->out_cap;
    finish(e, j, over ? fail(WPM_ERR_CAPACITY, "job: more masks than its capacity") : WPM_OK);
  }
  return WPM_OK;
}

}  // namespace

extern "C" {

int wpm_engine_create(const wpm_engine_config *cfg, void *cuda_stream, wpm_engine **out) {
  if (!out) return fail(WPM_ERR_INPUT, "out is NULL");
  *out = nullptr;
  wpm_engine *e = new wpm_engine();
  const int64_t mem = cfg && cfg->memory_bytes > 0 ? cfg->memory_bytes : (8ll << 30);
  e->max_jobs = cfg && cfg->max_jobs > 0 ? cfg->max_jobs : 1024;
  e->max_n = cfg && cfg->max_n > 0 ? std::min(cfg->max_n, 12) : 11;
  e->budget = cfg && cfg->budget > 0 ? cfg->budget : (1 << 20);
  e->slice_ms = cfg ? cfg->slice_ms : 0;
  auto bail = [&](int code) {
    wpm_engine_destroy(e);
    return code;
  };
  if (cudaGetDevice(&e->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device) != cudaSuccess)
    return bail(fail(WPM_ERR_CUDA, "no CUDA device"));
  if (cuda_stream) {
    e->s = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(WPM_ERR_CUDA, "cudaStreamCreate failed"));
    e->own_stream = true;
  }
  e->k = class_for_n(e->max_n);
  // per-thread searches, which can park their work between passes
  e->search = kSearchThread;
  e->tpb = 128;
  // deepest search: the upper-bound cap of the largest Picard-4 instance (jobs that could go
  // deeper, e.g. uncapped large ones, are refused at admission)
  const int mx = e->max_n;
  e->max_depth = (int)(binom_e(mx + 4 - (mx + 1) / 2, 4) + binom_e(mx + 3 - mx / 2, 4)) + 2;
  e->slot_bytes = 0;
  for (int n = 2; n <= mx; n++) e->slot_bytes = std::max(e->slot_bytes, table_bytes(n, n + 4));
  int occ = dfs_max_blocks_per_sm(e->k, e->search, e->tpb, e->max_depth);
  while (occ == 0 && e->tpb > 64) {
    e->tpb /= 2;
    occ = dfs_max_blocks_per_sm(e->k, e->search, e->tpb, e->max_depth);
  }
  if (occ == 0) return bail(fail(WPM_ERR_LIMIT, "engine size class does not fit"));
  e->blocks = e->sms * occ;
  const int n_threads = e->blocks * e->tpb;
  e->n_searches = e->search == kSearchThread ? n_threads : n_threads / 32;
  e->iw = item_words_for(e->k);
  const unsigned long long room = (unsigned long long)e->n_searches * e->max_depth;
  e->ring_cap = (e->search == kSearchThread ? 64ull * e->n_searches : 2 * room) +
                (unsigned long long)e->max_jobs;
  e->dump_limit = e->ring_cap > room ? e->ring_cap - room : 0;
  e->idle_limit = std::max<unsigned long long>(1, (unsigned long long)e->n_searches / 5);
  e->hungry = (unsigned long long)e->n_searches;
  e->pool_bytes = (size_t)mem;
  e->slots.assign(e->max_jobs, nullptr);
  int rc = WPM_OK;
  if ((rc = e->inst.ensure(sizeof(InstDesc) * e->max_jobs)) ||
      (rc = e->outd.ensure(sizeof(OutDesc) * e->max_jobs)) ||
      (rc = e->ctr.ensure(8ull * kCtrN * e->max_jobs)) ||
      (rc = e->tables.ensure(e->slot_bytes * e->max_jobs)) ||
      (rc = e->cond.ensure(kCondSlotBytes * e->max_jobs)) ||
      (rc = e->ring.ensure(e->ring_cap * e->iw * 4ull)) ||
      (rc = e->ready.ensure(e->ring_cap * 4ull)) ||
      (rc = e->q.ensure(sizeof(QueueCtl))) || (rc = e->ids.ensure(4ull * e->max_jobs)) ||
      (rc = e->pool.ensure(e->pool_bytes)) ||
      (rc = e->h_inst.ensure(sizeof(InstDesc) * e->max_jobs)) ||
      (rc = e->h_outd.ensure(sizeof(OutDesc) * e->max_jobs)) ||
      (rc = e->h_ctr.ensure(8ull * kCtrN * e->max_jobs)) || (rc = e->h_q.ensure(sizeof(QueueCtl))) ||
      (rc = e->h_ids.ensure(4ull * e->max_jobs)) ||
      (rc = e->h_cond.ensure(kCondSlotBytes * e->max_jobs)))
    return bail(rc);
  if (e->search == kSearchThread) {
    if ((rc = e->stack.ensure((size_t)n_threads * e->max_depth * 4ull)) ||
        (rc = e->aff.ensure((size_t)n_threads * 2 * kMaxAffine * 8ull)) ||
        (rc = e->park.ensure((size_t)n_threads * (kParkHeader + e->iw) * 4ull)))
      return bail(rc);
    if (cudaMemsetAsync(e->park.p, 0, e->park.cap, e->s) != cudaSuccess ||
        cudaMemsetAsync(e->ready.p, 0, e->ready.cap, e->s) != cudaSuccess ||
        cudaStreamSynchronize(e->s) != cudaSuccess)
      return bail(fail(WPM_ERR_CUDA, "cudaMemset of the park records failed"));
  }
  e->free_blocks[0] = e->pool.cap;
  *out = e;
  return WPM_OK;
}

int wpm_engine_submit(wpm_engine *e, const wpm_instance *inst, int mode, uint64_t out_capacity,
                      uint64_t *job_id) {
  if (!e || !inst || !job_id) return fail(WPM_ERR_INPUT, "NULL argument");
  if (mode != WPM_MODE_LIST && mode != WPM_MODE_COUNT) return fail(WPM_ERR_INPUT, "bad mode");
  Job *j = new Job();
  int rc = copy_map(inst->lambda_cols, inst->kind, inst->n, inst->m, j->hi);
  if (rc == WPM_OK) rc = copy_conditions(inst->cond, j->hi);
  if (rc == WPM_OK && j->hi.post)
    rc = fail(WPM_ERR_INPUT, "engine: post filters are applied by wpm_enumerate_batch only");
  if (rc == WPM_OK && mode == WPM_MODE_LIST) {
    // a job whose output region exceeds the engine's whole output memory could never be
    // admitted (and would hold up every job behind it): refuse it now
    const size_t words = (binom_e(j->hi.m, j->hi.n) + 63) / 64;
    const size_t bytes = a256(2 * 8 * words * std::max<uint64_t>(out_capacity, 1));
    if (bytes > e->pool_bytes)
      rc = fail(WPM_ERR_NOMEM, "engine: the job's output region (%zu bytes) exceeds the "
                "engine's output memory (%zu bytes)", bytes, e->pool_bytes);
  }
  if (rc != WPM_OK) {
    delete j;
    return rc;
  }
  j->id = e->next_id++;
  j->mode = mode;
  j->out_cap = out_capacity;
  e->jobs[j->id] = j;
  e->pending.push_back(j);
  *job_id = j->id;
  return WPM_OK;
}

int wpm_engine_step(wpm_engine *e, int *n_active) {
  if (!e) return fail(WPM_ERR_INPUT, "engine is NULL");
  static const bool trace = getenv("WPM_TRACE") != nullptr;
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const unsigned long long items0 = e->tail - e->head;
  int rc = admit(e);
  const auto t1 = clk::now();
  const unsigned long long items1 = e->tail - e->head;
  if (rc == WPM_OK) rc = pass(e);
  const auto t2 = clk::now();
  if (rc == WPM_OK) rc = retire(e);
  const auto t3 = clk::now();
  if (trace) {
    auto ms = [](clk::duration d) { return std::chrono::duration<double, std::milli>(d).count(); };
    int a = 0;
    for (Job *j : e->slots) a += j != nullptr;
    fprintf(stderr, "[wpm engine] items %llu -> %llu -> %llu; admit %.3f ms, pass %.3f ms, "
            "retire %.3f ms; active %d, pending %zu; parked %llu, nodes %llu\n", items0, items1,
            e->tail - e->head, ms(t1 - t0), ms(t2 - t1), ms(t3 - t2), a, e->pending.size(),
            e->parked, e->pass_nodes);
  }
  if (n_active) {
    int a = 0;
    for (Job *j : e->slots) a += j != nullptr;
    *n_active = a;
  }
  return rc;
}

int wpm_engine_poll(wpm_engine *e, uint64_t *job_ids, int cap) {
  if (!e) return fail(WPM_ERR_INPUT, "engine is NULL");
  int k = 0;
  while (k < cap && !e->finished.empty()) {
    job_ids[k++] = e->finished.front();
    e->finished.pop_front();
  }
  return k;
}

int wpm_engine_result(wpm_engine *e, uint64_t job_id, wpm_output *out) {
  if (!e || !out) return fail(WPM_ERR_INPUT, "NULL argument");
  auto it = e->jobs.find(job_id);
  if (it == e->jobs.end() || !it->second->done) return fail(WPM_ERR_INPUT, "no finished job %llu",
                                                            (unsigned long long)job_id);
  Job *j = it->second;
  out->count = j->count;
  out->found = j->count;  // the engine applies no post-filters
  out->nodes = j->nodes;
  out->probes = j->probes;
  out->words_per_mask = j->ow;
  out->M = j->M;
  out->N = j->N;
  out->status = j->status;
  int rc = j->status;
  if (rc == WPM_OK && j->mode == WPM_MODE_LIST) {
    if (out->capacity < j->count || (j->count && !out->masks)) {
      rc = fail(WPM_ERR_CAPACITY, "result buffer holds fewer than %llu masks",
                (unsigned long long)j->count);
      return rc;  // the result stays available for another call
    }
    if (j->count) memcpy(out->masks, j->masks, 8 * j->count * j->ow);
  }
  e->host_lists.give(j->masks, j->masks_block);
  e->jobs.erase(it);
  delete j;
  return rc;
}

void wpm_engine_destroy(wpm_engine *e) {
  if (!e) return;
  if (e->s) cudaStreamSynchronize(e->s);
  for (auto &kv : e->jobs) delete kv.second;
  e->host_lists.release_all();
  for (DevBuf *b : {&e->inst, &e->outd, &e->ctr, &e->tables, &e->cond, &e->ring, &e->ready,
                    &e->stack, &e->aff, &e->q, &e->ids, &e->seg, &e->pool, &e->park})
    b->release();
  for (PinBuf *b : {&e->h_inst, &e->h_outd, &e->h_ctr, &e->h_q, &e->h_ids, &e->h_seg, &e->h_cond})
    b->release();
  if (e->own_stream) cudaStreamDestroy(e->s);
  delete e;
}

}  // extern "C"
