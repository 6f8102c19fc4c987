// wpm_runtime.cpp -- host runtime and C ABI of libwpm (weak pseudo-manifold enumeration,
// Choi, Jang, Vallee, arXiv 2301.00806).
//
// The host validates arguments, lays out device memory, launches the kernels of
// wpm_kernels.cu and moves results. It performs none of the enumeration's arithmetic:
// candidate facets, ridges, incidence, the search and the output sort all run on the GPU.
//
// One run (any entry point) is:
//   upload the instances  ->  setup_kernel (facets, ridges, incidence, properties)
//   ->  roots_kernel  ->  breadth-first expand passes until the frontier is wide enough
//   ->  depth-first passes until the work ring is empty  ->  per-instance merge sort
//   ->  copy-out.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "wpm.h"
#include "wpm_host.h"
#include "wpm_internal.h"

namespace wpm {

static thread_local std::string t_err;
static thread_local wpm_run_stats t_stats;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }

void clear_last_error() { t_err.clear(); }

// Host outputs leave the device in chunks of at most this many words (256 MB) through two
// page-locked halves of the workspace's staging buffer.
constexpr size_t kStageChunk = 32u << 20;

// Device buffers reused across calls on one device.
// The depth-first pass loop as an instantiated CUDA graph: a conditional while node whose
// body is prep, the pass and check. Kept while the pass's arguments stay the same.
struct PassGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  PassArgs pa;
  int k = -1, search = 0, blocks = 0, tpb = 0;
  bool unsupported = false;  // conditional nodes are not available: use the host loop
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    k = -1;
  }
};

// The breadth-first expansion loop as an instantiated CUDA graph: a conditional while node
// whose body is one level (the expansion over the queued items, then its check). Kept while
// its arguments stay the same.
struct ExpandGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  PassArgs pa;
  int k = -1, blocks = 0;
  unsigned long long target = 0, max_children = 0, ring_cap = 0, max_levels = 0;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    k = -1;
  }
};

struct Workspace {
  int device = -1;
  int sms = 0;
  cudaStream_t own = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_stage[2] = {nullptr, nullptr};  // the two halves of h_stage filled
  PassGraph pg;
  ExpandGraph eg;
  DevBuf inst, outd, ctr, arena, cond, ids, q, ring, ready, stack, aff, park, out, seg, segs, stage,
      sweep, keep;
  PinBuf h_inst, h_outd, h_q, h_ctr, h_cond, h_ids, h_seg, h_segs, h_stage, h_sweep;
  void release() {
    pg.reset();
    eg.reset();
    if (pg.capture) cudaStreamDestroy(pg.capture);
    pg.capture = nullptr;
    for (DevBuf *b : {&inst, &outd, &ctr, &arena, &cond, &ids, &q, &ring, &ready, &stack, &aff, &park, &out, &seg,
                      &segs, &stage, &sweep, &keep})
      b->release();
    for (PinBuf *b : {&h_inst, &h_outd, &h_q, &h_ctr, &h_cond, &h_ids, &h_seg, &h_segs, &h_stage,
                      &h_sweep})
      b->release();
    for (cudaEvent_t &e : ev_stage) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
  }
};

static std::mutex g_mu;
static std::map<int, Workspace *> g_ws;

static int get_workspace(Workspace **out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  auto it = g_ws.find(dev);
  if (it != g_ws.end()) {
    *out = it->second;
    return WPM_OK;
  }
  Workspace *w = new Workspace();
  w->device = dev;
  CUDA_TRY(cudaDeviceGetAttribute(&w->sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaStreamCreateWithFlags(&w->own, cudaStreamNonBlocking));
  g_ws[dev] = w;
  *out = w;
  return WPM_OK;
}

static long long binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  long long r = 1;
  for (int i = 0; i < b; i++) r = r * (a - i) / (i + 1);
  return r;
}

int copy_conditions(const wpm_conditions *c, HostInst &h) {
  if (!c) return WPM_OK;
  if (c->ubt_cap < -2) return fail(WPM_ERR_INPUT, "ubt_cap %d is not a cap", c->ubt_cap);
  h.cap_req = c->ubt_cap;
  h.base_req = c->require_base_facet ? 1 : 0;
  if (c->post_filter & ~(WPM_POST_PIC | WPM_POST_SEED))
    return fail(WPM_ERR_INPUT, "unknown post_filter flags 0x%x", c->post_filter);
  h.post = c->post_filter;
  if (c->n_affine < 0 || c->n_affine > WPM_MAX_AFFINE)
    return fail(WPM_ERR_INPUT, "n_affine %d outside 0..%d", c->n_affine, WPM_MAX_AFFINE);
  const bool masks = c->forced_in || c->forced_out || c->n_affine > 0;
  if (!masks) return WPM_OK;
  if (c->n_facets <= 0 || c->n_facets > WPM_MAX_FACETS)
    return fail(WPM_ERR_INPUT, "n_facets %d: masks and coefficients need the instance's M",
                c->n_facets);
  const int M = c->n_facets, W = (M + 63) / 64;
  h.n_facets_req = M;
  auto take = [&](const uint64_t *src, std::vector<uint64_t> &dst) {
    if (!src) return;
    dst.assign(src, src + W);
    if (M % 64) dst[W - 1] &= (1ull << (M % 64)) - 1ull;  // bits >= M are not facets
  };
  take(c->forced_in, h.fin);
  take(c->forced_out, h.fout);
  if (c->n_affine > 0) {
    if (!c->affine_c0 || !c->affine_coef) return fail(WPM_ERR_INPUT, "affine arrays are NULL");
    h.n_aff = c->n_affine;
    h.c0.assign(c->affine_c0, c->affine_c0 + h.n_aff);
    h.coef.assign(c->affine_coef, c->affine_coef + (size_t)h.n_aff * M);
    for (int32_t v : h.coef)
      if (v > (1 << 20) || v < -(1 << 20)) return fail(WPM_ERR_INPUT, "|coefficient| > 2^20");
  }
  return WPM_OK;
}

int copy_map(const uint32_t *cols, int kind, int n, int m, HostInst &h) {
  if (kind != WPM_LAMBDA_PRIMAL && kind != WPM_LAMBDA_DUAL)
    return fail(WPM_ERR_INPUT, "kind %d is neither primal nor dual", kind);
  if (n < 2 || m <= n || m > WPM_MAX_VERTICES)
    return fail(WPM_ERR_INPUT, "need 2 <= n < m <= 16 (n=%d, m=%d)", n, m);
  if (!cols) return fail(WPM_ERR_INPUT, "lambda_cols is NULL");
  h.kind = kind;
  h.n = n;
  h.m = m;
  const int bits = kind == WPM_LAMBDA_PRIMAL ? n : m - n;
  for (int i = 0; i < m; i++) {
    if (bits < 32 && (cols[i] >> bits))
      return fail(WPM_ERR_INPUT, "column %d has bits above Z2^%d", i, bits);
    h.cols[i] = cols[i];
  }
  if (kind == WPM_LAMBDA_DUAL) {  // an injective DCM: nonzero, pairwise distinct rows
    for (int i = 0; i < m; i++) {
      if (cols[i] == 0) return fail(WPM_ERR_INPUT, "dual row %d is zero", i);
      for (int j = 0; j < i; j++)
        if (cols[i] == cols[j]) return fail(WPM_ERR_INPUT, "dual rows %d and %d repeat", j, i);
    }
  }
  return WPM_OK;
}

int copy_facet_list(const uint16_t *facets, int M, int n, int m, HostInst &h) {
  if (n < 2 || m <= n || m > WPM_MAX_VERTICES)
    return fail(WPM_ERR_INPUT, "need 2 <= n < m <= 16 (n=%d, m=%d)", n, m);
  if (M < 0 || M > WPM_MAX_FACETS) return fail(WPM_ERR_LIMIT, "M=%d outside 0..%d", M, WPM_MAX_FACETS);
  if (M > 0 && !facets) return fail(WPM_ERR_INPUT, "facets is NULL");
  h.kind = 2;
  h.n = n;
  h.m = m;
  h.given.assign(facets, facets + M);
  for (int j = 0; j < M; j++)
    if (__builtin_popcount(h.given[j]) != n || (h.given[j] >> m))
      return fail(WPM_ERR_INPUT, "facet %d is not an %d-subset of [%d]", j, n, m);
  std::vector<uint16_t> s = h.given;
  std::sort(s.begin(), s.end());
  if (std::adjacent_find(s.begin(), s.end()) != s.end())
    return fail(WPM_ERR_INPUT, "repeated facet in the list");
  return WPM_OK;
}

// Per-instance outcome of a run.
struct InstResult {
  int status = WPM_OK;
  unsigned long long count = 0, nodes = 0, probes = 0;
  unsigned long long found = 0;  // count before the post-filters
  int M = 0, N = 0, ow = 1;
};

struct RunOptions {
  int mode = WPM_MODE_COUNT;
  int tpb = 0;
  long long budget = 0;
  long long frontier_target = 0;
  long long ring_items = 0;
  int idle_percent = 0;
  int search = 0;
  int time_limit_ms = 0;
  int feed_levels = 0;
  int donate_levels = 0;
  int donate_every = 0;
  int graph = 0;  // < 0: host-driven pass loop
  int engine = 0;  // 1: GF(2) cycle-space sweep over the convenient basis; 2: plain sweep
  int sweep_max_s = 0;
  long long hungry_items = 0;
  int ready_polls = 0;
  int idle_polls = 0;
  int test_unpublished = 0;
  long long stage_chunk = 0;
  bool profile = false;
  bool setup_only = false;  // stop after the setup kernel (candidate facets)
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Account a host <-> device copy of the current run: (dst, src, bytes) as passed to the copy.
static void count_copy(const void *, const void *, size_t bytes, cudaMemcpyKind kind) {
  if (kind == cudaMemcpyHostToDevice) t_stats.h2d_bytes += bytes;
  else if (kind == cudaMemcpyDeviceToHost) t_stats.d2h_bytes += bytes;
}

// Most passes a graph-driven loop runs before it stops with error 8.
constexpr unsigned long long kMaxGraphPasses = 1ull << 20;

// Launch the depth-first pass loop as a CUDA graph on `s` (building it first unless the last
// one has the same arguments). Returns cudaErrorNotSupported when conditional graph nodes
// are not available (the caller then runs the host loop).
static cudaError_t launch_pass_graph(Workspace *W, const PassArgs &pa, int k, int search,
                                     int blocks, int tpb, cudaStream_t s) {
  PassGraph &G = W->pg;
  if (G.unsupported) return cudaErrorNotSupported;
  const bool same = G.exec && G.k == k && G.search == search && G.blocks == blocks &&
                    G.tpb == tpb && memcmp(&G.pa, &pa, sizeof(PassArgs)) == 0;
  if (!same) {
    G.reset();
    if (!G.capture) {
      cudaError_t e = cudaStreamCreateWithFlags(&G.capture, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGraphCreate(&G.graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      G.reset();
      G.unsupported = true;
      return cudaErrorNotSupported;
    }
    // (the parameter union has no default constructor in C++: zeroed storage instead)
    alignas(cudaGraphNodeParams) unsigned char cp_bytes[sizeof(cudaGraphNodeParams)];
    memset(cp_bytes, 0, sizeof(cp_bytes));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_bytes);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
      cudaGetLastError();
      G.reset();
      G.unsupported = true;
      return cudaErrorNotSupported;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int thread_mode = search == kSearchThread;
    e = cudaStreamBeginCaptureToGraph(G.capture, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      G.reset();
      return e;
    }
    cudaError_t e1 = launch_pass_prep(pa.q, thread_mode, G.capture);
    cudaError_t e2 = launch_dfs(k, search, pa, blocks, tpb, G.capture);
    cudaError_t e3 = launch_pass_check(pa.q, thread_mode, h, kMaxGraphPasses, G.capture);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(G.capture, &captured);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e != cudaSuccess) {
      G.reset();
      return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e));
    }
    e = cudaGraphInstantiate(&G.exec, G.graph, 0);
    if (e != cudaSuccess) {
      G.reset();
      return e;
    }
    G.pa = pa;
    G.k = k;
    G.search = search;
    G.blocks = blocks;
    G.tpb = tpb;
  }
  return cudaGraphLaunch(G.exec, s);
}

// Launch the breadth-first expansion loop as one graph (built on first use and kept while the
// arguments stay the same). The queue holds the first level's items as [head_start, limit);
// levels run until expand_check_kernel's rule stops them. cudaErrorNotSupported when this
// CUDA has no conditional nodes (the caller then loops on the host).
static cudaError_t launch_expand_graph(Workspace *W, const PassArgs &pa, int k, int blocks,
                                       unsigned long long target,
                                       unsigned long long max_children,
                                       unsigned long long ring_cap,
                                       unsigned long long max_levels, cudaStream_t s) {
  ExpandGraph &G = W->eg;
  if (W->pg.unsupported) return cudaErrorNotSupported;
  const bool same = G.exec && G.k == k && G.blocks == blocks && G.target == target &&
                    G.max_children == max_children && G.ring_cap == ring_cap &&
                    G.max_levels == max_levels && memcmp(&G.pa, &pa, sizeof(PassArgs)) == 0;
  if (!same) {
    G.reset();
    PassGraph &P = W->pg;  // its capture stream is shared
    if (!P.capture) {
      cudaError_t e = cudaStreamCreateWithFlags(&P.capture, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGraphCreate(&G.graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault) !=
        cudaSuccess) {
      cudaGetLastError();
      G.reset();
      return cudaErrorNotSupported;
    }
    alignas(cudaGraphNodeParams) unsigned char cp_bytes[sizeof(cudaGraphNodeParams)];
    memset(cp_bytes, 0, sizeof(cp_bytes));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_bytes);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
      cudaGetLastError();
      G.reset();
      return cudaErrorNotSupported;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(P.capture, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      G.reset();
      return e;
    }
    cudaError_t e1 = launch_expand_queued(k, pa, blocks, P.capture);
    cudaError_t e2 = launch_expand_check(pa.q, h, target, max_children, ring_cap, max_levels,
                                         P.capture);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(P.capture, &captured);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
      G.reset();
      return e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e);
    }
    e = cudaGraphInstantiate(&G.exec, G.graph, 0);
    if (e != cudaSuccess) {
      G.reset();
      return e;
    }
    G.pa = pa;
    G.k = k;
    G.blocks = blocks;
    G.target = target;
    G.max_children = max_children;
    G.ring_cap = ring_cap;
    G.max_levels = max_levels;
  }
  return cudaGraphLaunch(G.exec, s);
}

// The GF(2) cycle-space sweep over the valid instances (their ids are in W->ids): a kernel
// basis per map, then every element of the kernel in Gray-code order (wpm_sweep.cu). Counts
// and list-mode masks land in the same counters and output regions as the search's.
static int run_sweep(Workspace *W, const InstDesc *hd, const std::vector<int32_t> &valid,
                     int engine, int max_log2, cudaStream_t s) {
  const int nv = (int)valid.size();
  max_log2 = max_log2 > 0 ? std::min(max_log2, 48) : 30;
  int max_n_ridges = 1;
  for (int i : valid) {
    if (hd[i].M > kSweepMaxM || hd[i].N > kSweepMaxN)
      return fail(WPM_ERR_LIMIT, "sweep: instance %d has M=%d, N=%d (the sweep takes M <= %d, "
                  "N <= %d)", i, hd[i].M, hd[i].N, kSweepMaxM, kSweepMaxN);
    max_n_ridges = std::max(max_n_ridges, hd[i].N);
  }
  const size_t rows_bytes = align_up(8ull * nv * max_n_ridges * kSweepW);
  const size_t basis_bytes = align_up(8ull * nv * kSweepMaxS * kSweepW);
  const size_t shape_bytes = align_up(sizeof(SweepShape) * nv);
  const size_t dims_bytes = align_up(4ull * nv);
  const size_t u64_bytes = align_up(8ull * (nv + 1));
  // device: rows scratch, basis, generators, shapes, dims, totals, chunk prefix
  WPM_TRY(W->sweep.ensure(rows_bytes + 2 * basis_bytes + shape_bytes + dims_bytes +
                          2 * u64_bytes));
  WPM_TRY(W->h_sweep.ensure(shape_bytes + 2 * u64_bytes));
  char *db = W->sweep.as<char>();
  uint64_t *rows = (uint64_t *)db;
  uint64_t *basis = (uint64_t *)(db + rows_bytes);
  uint64_t *gens = (uint64_t *)(db + rows_bytes + basis_bytes);
  SweepShape *shapes = (SweepShape *)(db + rows_bytes + 2 * basis_bytes);
  int32_t *dims = (int32_t *)(db + rows_bytes + 2 * basis_bytes + shape_bytes);
  unsigned long long *totals =
      (unsigned long long *)(db + rows_bytes + 2 * basis_bytes + shape_bytes + dims_bytes);
  unsigned long long *chunks = totals + (u64_bytes / 8);
  char *hb = W->h_sweep.as<char>();
  SweepShape *hshape = (SweepShape *)hb;
  unsigned long long *htot = (unsigned long long *)(hb + shape_bytes);
  unsigned long long *hchunks = htot + (u64_bytes / 8);
  CUDA_TRY(launch_kernel_basis(W->inst.as<InstDesc>(), W->ids.as<int32_t>(), nv, max_n_ridges,
                               rows, basis, dims, s));
  CUDA_TRY(launch_convenient(W->inst.as<InstDesc>(), W->ids.as<int32_t>(), nv, basis, dims,
                             engine == 2 ? 2 : 1, gens, shapes, s));
  t_stats.kernel_launches += 2;
  CUDA_TRY(cudaMemcpyAsync(hshape, shapes, sizeof(SweepShape) * nv, cudaMemcpyDeviceToHost, s));
  count_copy(hshape, shapes, sizeof(SweepShape) * nv, cudaMemcpyDeviceToHost);
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int j = 0; j < nv; j++) htot[j] = 0;
  for (int j = 0; j < nv; j++) {
    const SweepShape &sh = hshape[j];
    if (sh.s > kSweepMaxS)
      return fail(WPM_ERR_LIMIT, "sweep: instance %d has a kernel of dimension %d (limit %d)",
                  valid[j], sh.s, kSweepMaxS);
    // combinations: each block's choices times 2^(single generators)
    double lg = sh.n_single;
    unsigned long long outer = 1;
    for (int l = 0; l < sh.n_blocks; l++) {
      const int k = sh.block_k[l];
      const unsigned long long c = 1ull + k + (unsigned long long)k * (k - 1) / 2;
      lg += std::log2((double)c);
      outer *= c;
    }
    if (lg > max_log2 + 1e-9)
      return fail(WPM_ERR_LIMIT, "sweep: instance %d needs 2^%.1f combinations (limit 2^%d)",
                  valid[j], lg, max_log2);
    htot[j] = sh.feasible ? (outer << sh.n_single) : 0;
  }
  // chunk length: up to about 1M chunks over the run (a thread each, so that every SM holds
  // many 64-thread blocks), 64 to 4096 combinations
  unsigned long long all = 0;
  for (int j = 0; j < nv; j++) all += htot[j];
  unsigned long long chunk = 64;
  while (chunk < kSweepChunkMax && chunk * (1ull << 20) < all) chunk *= 2;
  hchunks[0] = 0;
  for (int j = 0; j < nv; j++) hchunks[j + 1] = hchunks[j] + (htot[j] + chunk - 1) / chunk;
  CUDA_TRY(cudaMemcpyAsync(totals, htot, 2 * u64_bytes, cudaMemcpyHostToDevice, s));
  count_copy(totals, htot, 2 * u64_bytes, cudaMemcpyHostToDevice);
  CUDA_TRY(launch_sweep(W->inst.as<InstDesc>(), W->ids.as<int32_t>(), nv, gens, shapes, totals,
                        chunks, hchunks[nv], chunk, max_n_ridges, W->outd.as<OutDesc>(),
                        W->ctr.as<unsigned long long>(), s));
  t_stats.kernel_launches++;
  return WPM_OK;
}

// The engine of every entry point: run the instances `hi` on stream `s`.
// outs[i] (optional) provides list-mode buffers; res[i] receives the outcome.
static int run(Workspace *W, std::vector<HostInst> &hi, const RunOptions &opt, cudaStream_t s,
               const wpm_output *outs, std::vector<InstResult> &res, std::vector<uint16_t> *facets_out) {
  const int n_inst = (int)hi.size();
  res.assign(n_inst, InstResult());
  memset(&t_stats, 0, sizeof(t_stats));
  struct RunClock {  // run_ms on every way out
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    ~RunClock() {
      t_stats.run_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  } run_clock;
  if (n_inst == 0) return WPM_OK;

  // ---- device layout of the tables and of the caller's conditions --------------------
  size_t arena = 0, cond = 0;
  std::vector<size_t> a_off(n_inst), c_off(n_inst);
  for (int i = 0; i < n_inst; i++) {
    const HostInst &h = hi[i];
    const size_t nsub = binom(h.m, h.n), nrsub = binom(h.m, h.n - 1);
    a_off[i] = arena;
    arena += align_up(2 * nsub) + align_up(4 * (nsub + 1)) + align_up(4 * (nrsub + 1)) +
             align_up(32 * nsub) + align_up(32 * nrsub);
    c_off[i] = cond;
    cond += align_up(8 * h.fin.size()) + align_up(8 * h.fout.size()) + align_up(4 * h.c0.size()) +
            align_up(4 * h.coef.size()) + align_up(2 * h.given.size());
  }
  WPM_TRY(W->arena.ensure(arena));
  WPM_TRY(W->cond.ensure(cond + 256));
  WPM_TRY(W->h_cond.ensure(cond + 256));
  WPM_TRY(W->inst.ensure(sizeof(InstDesc) * n_inst));
  WPM_TRY(W->h_inst.ensure(sizeof(InstDesc) * n_inst));
  InstDesc *hd = W->h_inst.as<InstDesc>();
  char *ab = W->arena.as<char>(), *cb = W->cond.as<char>(), *hc = W->h_cond.as<char>();
  for (int i = 0; i < n_inst; i++) {
    const HostInst &h = hi[i];
    InstDesc &d = hd[i];
    memset(&d, 0, sizeof(d));
    d.kind = h.kind;
    d.n = h.n;
    d.m = h.m;
    d.mode = opt.mode;
    for (int v = 0; v < kMaxVertices; v++) d.cols[v] = h.cols[v];
    d.cap_req = h.cap_req;
    d.base_req = h.base_req;
    d.post = h.post;
    d.n_facets_req = h.n_facets_req;
    d.n_aff = h.n_aff;
    d.nsub = (int)binom(h.m, h.n);
    d.nrsub = (int)binom(h.m, h.n - 1);
    d.has_fin = !h.fin.empty();
    d.has_fout = !h.fout.empty();
    size_t o = a_off[i];
    auto take_a = [&](size_t bytes) { char *p = ab + o; o += align_up(bytes); return p; };
    d.facets = (uint16_t *)take_a(2 * (size_t)d.nsub);
    d.fprefix = (int32_t *)take_a(4 * ((size_t)d.nsub + 1));
    d.rprefix = (int32_t *)take_a(4 * ((size_t)d.nrsub + 1));
    d.frw = (uint16_t *)take_a(32 * (size_t)d.nsub);
    d.prw = (uint16_t *)take_a(32 * (size_t)d.nrsub);
    size_t c = c_off[i];
    auto take_c = [&](const void *src, size_t bytes) -> const void * {
      if (!bytes) return nullptr;
      memcpy(hc + c, src, bytes);
      const void *p = cb + c;
      c += align_up(bytes);
      return p;
    };
    d.fin = (const uint64_t *)take_c(h.fin.data(), 8 * h.fin.size());
    d.fout = (const uint64_t *)take_c(h.fout.data(), 8 * h.fout.size());
    d.aff_c0 = (const int32_t *)take_c(h.c0.data(), 4 * h.c0.size());
    d.aff_coef = (const int32_t *)take_c(h.coef.data(), 4 * h.coef.size());
    d.given = (const uint16_t *)take_c(h.given.data(), 2 * h.given.size());
    d.n_given = (int)h.given.size();
  }
  if (cond) CUDA_TRY(cudaMemcpyAsync(W->cond.p, W->h_cond.p, cond, cudaMemcpyHostToDevice, s));
  count_copy(W->cond.p, W->h_cond.p, cond, cudaMemcpyHostToDevice);
  CUDA_TRY(cudaMemcpyAsync(W->inst.p, hd, sizeof(InstDesc) * n_inst, cudaMemcpyHostToDevice, s));
  count_copy(W->inst.p, hd, sizeof(InstDesc) * n_inst, cudaMemcpyHostToDevice);
  CUDA_TRY(launch_setup(W->inst.as<InstDesc>(), n_inst, s));
  t_stats.kernel_launches++;
  CUDA_TRY(cudaMemcpyAsync(hd, W->inst.p, sizeof(InstDesc) * n_inst, cudaMemcpyDeviceToHost, s));
  count_copy(hd, W->inst.p, sizeof(InstDesc) * n_inst, cudaMemcpyDeviceToHost);
  CUDA_TRY(cudaStreamSynchronize(s));

  // ---- per-instance checks ----------------------------------------------------------
  std::vector<int32_t> valid;
  int mw_max = 1, nw_max = 1, max_depth = 2, max_children = 16;
  for (int i = 0; i < n_inst; i++) {
    const InstDesc &d = hd[i];
    InstResult &r = res[i];
    r.M = d.M;
    r.N = d.N;
    r.ow = d.ow;
    if (d.err & kErrLimit) {
      r.status = fail(WPM_ERR_LIMIT, "instance %d: M=%d or N=%d above the limits %d / %d", i, d.M,
                      d.N, kMaxFacets, kMaxRidges);
    } else if (d.err & kErrMaskSize) {
      r.status = fail(WPM_ERR_INPUT, "instance %d: conditions built for M=%d, the map has M=%d", i,
                      d.n_facets_req, d.M);
    } else if (d.err & kErrCapNeedsPic4) {
      r.status = fail(WPM_ERR_INPUT, "instance %d: WPM_CAP_UBT needs m = n + 4", i);
    } else if (d.post && opt.mode != WPM_MODE_LIST) {
      r.status = fail(WPM_ERR_INPUT, "instance %d: post filters need list mode", i);
    } else if (d.post && d.m > kPostMaxM) {
      r.status = fail(WPM_ERR_LIMIT, "instance %d: post filters take m <= %d", i, kPostMaxM);
    } else if (d.kind != 2 && d.M == 0) {
      r.status = fail(WPM_ERR_INPUT, "instance %d: the map has rank below %d (no candidate facet)",
                      i, d.kind == 0 ? d.n : d.m - d.n);
    }
    if (r.status != WPM_OK) continue;
    valid.push_back(i);
    mw_max = std::max(mw_max, d.mw);
    nw_max = std::max(nw_max, d.nw);
    const int depth = (d.cap >= 0 ? std::min(d.cap, d.M) : d.M) + 2;
    max_depth = std::max(max_depth, depth);
    max_children = std::max(max_children, d.M);
  }
  if (facets_out) {
    if (!valid.empty() && valid[0] == 0) {
      facets_out->resize(hd[0].M);
      if (hd[0].M)
        CUDA_TRY(cudaMemcpy(facets_out->data(), hd[0].facets, 2 * (size_t)hd[0].M,
                            cudaMemcpyDeviceToHost));
    }
    return WPM_OK;
  }
  if (opt.setup_only || valid.empty()) return WPM_OK;
  const int n_valid = (int)valid.size();

  // ---- size class and launch shape ------------------------------------------------
  const int k = pick_size_class(mw_max, nw_max);
  if (k < 0) return fail(WPM_ERR_LIMIT, "no kernel size class holds mw=%d nw=%d", mw_max, nw_max);
  // per-thread searches for batches of at least 16 maps of the size classes of n = 7..10;
  // per-warp searches for small maps, whose subtrees are too small to keep a thread each
  // busy, for n = 11, where a thread's state would leave too few searches per SM, and for a
  // few maps alone, which cannot keep some 80,000 per-thread searches fed (measured: the 7
  // IDCM orbits of n = 9 run 1.14 times faster per warp, the 3 of n = 10 1.4 times, the whole
  // n = 11 map 2.7 times; 16 maps of n = 10 run 1.3 times faster per thread)
  const int search = opt.search == kSearchThread || opt.search == kSearchWarp
                         ? opt.search
                         : (k >= 3 && k <= 6 && n_valid >= 16 ? kSearchThread : kSearchWarp);
  int tpb = opt.tpb > 0 ? opt.tpb : (search == kSearchThread ? 128 : 256);
  if (tpb != 64 && tpb != 128 && tpb != 256) tpb = 128;
  int occ = dfs_max_blocks_per_sm(k, search, tpb, max_depth);
  while (occ == 0 && tpb > 64) {
    tpb /= 2;
    occ = dfs_max_blocks_per_sm(k, search, tpb, max_depth);
  }
  if (occ == 0)
    return fail(WPM_ERR_LIMIT, "size class %d with depth %d does not fit in shared memory", k,
                max_depth);
  const int blocks = W->sms * occ;
  const int n_threads = blocks * tpb;
  const int n_searches = search == kSearchThread ? n_threads : n_threads / 32;
  const int iw = item_words_for(k);
  const long long budget = opt.budget > 0 ? opt.budget : (1ll << 40);
  const long long frontier_target =
      opt.frontier_target > 0 ? opt.frontier_target : 2LL * n_searches;
  // per-thread searches reserve their slots before returning work, so any ring size is
  // safe for them; per-warp searches need room for every search's levels at once
  const unsigned long long room_all = (unsigned long long)n_searches * max_depth;
  unsigned long long ring_cap =
      opt.ring_items > 0 ? (unsigned long long)opt.ring_items
                         : std::max<unsigned long long>(
                               search == kSearchThread ? std::min(2ull * room_all,
                                                                  64ull * n_searches)
                                                       : 2ull * room_all,
                               std::max(4ull * n_valid, 1ull << 16));
  ring_cap = std::max<unsigned long long>(ring_cap, (unsigned long long)n_valid + 1);
  const unsigned long long room = (unsigned long long)n_searches * max_depth;
  const unsigned long long dump_limit = ring_cap > room ? ring_cap - room : 0;

  // ---- buffers -------------------------------------------------------------------
  WPM_TRY(W->ctr.ensure(8ull * kCtrN * n_inst));
  WPM_TRY(W->h_ctr.ensure(8ull * kCtrN * n_inst));
  WPM_TRY(W->outd.ensure(sizeof(OutDesc) * n_inst));
  WPM_TRY(W->h_outd.ensure(sizeof(OutDesc) * n_inst));
  WPM_TRY(W->ids.ensure(4ull * n_inst + 4));
  WPM_TRY(W->h_ids.ensure(4ull * n_inst + 4));
  WPM_TRY(W->q.ensure(sizeof(QueueCtl)));
  WPM_TRY(W->h_q.ensure(sizeof(QueueCtl)));
  WPM_TRY(W->ring.ensure(ring_cap * iw * 4ull));
  if (search == kSearchThread) {
    WPM_TRY(W->stack.ensure((size_t)n_threads * max_depth * 4ull));
    WPM_TRY(W->aff.ensure((size_t)n_threads * 2 * kMaxAffine * 8ull));
    WPM_TRY(W->park.ensure((size_t)n_threads * (kParkHeader + iw) * 4ull));
    WPM_TRY(W->ready.ensure(ring_cap * 4ull));
    // no search is parked yet (word 0 of every park record); no ready flag is raised (the
    // passes of this run use epochs 1, 2, ...)
    CUDA_TRY(cudaMemsetAsync(W->park.p, 0, (size_t)n_threads * 4ull, s));
    CUDA_TRY(cudaMemsetAsync(W->ready.p, 0, ring_cap * 4ull, s));
  }
  const bool list = opt.mode == WPM_MODE_LIST;
  OutDesc *ho = W->h_outd.as<OutDesc>();
  memset(ho, 0, sizeof(OutDesc) * n_inst);
  if (list) {
    size_t total = 0;
    for (int i : valid) total += align_up(8ull * hd[i].ow * (outs ? outs[i].capacity : 0));
    WPM_TRY(W->out.ensure(2 * total + 256));
    char *ob = W->out.as<char>();
    size_t o = 0;
    for (int i : valid) {
      const unsigned long long cap = outs ? outs[i].capacity : 0;
      const size_t bytes = align_up(8ull * hd[i].ow * cap);
      ho[i].out = (uint64_t *)(ob + o);
      ho[i].out2 = (uint64_t *)(ob + total + o);
      ho[i].cap = cap;
      o += bytes;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(W->outd.p, ho, sizeof(OutDesc) * n_inst, cudaMemcpyHostToDevice, s));
  count_copy(W->outd.p, ho, sizeof(OutDesc) * n_inst, cudaMemcpyHostToDevice);
  CUDA_TRY(cudaMemsetAsync(W->ctr.p, 0, 8ull * kCtrN * n_inst, s));
  int32_t *hids = W->h_ids.as<int32_t>();
  for (int j = 0; j < n_valid; j++) hids[j] = valid[j];
  CUDA_TRY(cudaMemcpyAsync(W->ids.p, hids, 4ull * n_valid, cudaMemcpyHostToDevice, s));
  count_copy(W->ids.p, hids, 4ull * n_valid, cudaMemcpyHostToDevice);
  bool timed_out = false;
  if (opt.engine == 1 || opt.engine == 2) {
    WPM_TRY(run_sweep(W, hd, valid, opt.engine, opt.sweep_max_s, s));
    t_stats.search = 0;
  } else {
    QueueCtl *hq = W->h_q.as<QueueCtl>();
    memset(hq, 0, sizeof(QueueCtl));
    CUDA_TRY(cudaMemcpyAsync(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, s));
    count_copy(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice);
    t_stats.kernel_launches++;
    CUDA_TRY(launch_roots(W->inst.as<InstDesc>(), n_valid, W->ids.as<int32_t>(),
                          W->ctr.as<unsigned long long>(), W->ring.as<uint32_t>(), ring_cap, iw,
                          size_class(k).mw, W->q.as<QueueCtl>(), s));
    CUDA_TRY(cudaMemcpyAsync(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, s));
    count_copy(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost);
    CUDA_TRY(cudaStreamSynchronize(s));

    PassArgs pa;
    memset(&pa, 0, sizeof(pa));  // no parking: every field not set below is zero
    pa.inst = W->inst.as<InstDesc>();
    pa.outs = W->outd.as<OutDesc>();
    pa.ctr = W->ctr.as<unsigned long long>();
    pa.ring = W->ring.as<uint32_t>();
    pa.ring_cap = ring_cap;
    pa.item_words = iw;
    pa.q = W->q.as<QueueCtl>();
    pa.max_depth = max_depth;
    pa.n_threads = n_threads;
    pa.stack = search == kSearchThread ? W->stack.as<uint32_t>() : nullptr;
    pa.aff_scratch = search == kSearchThread ? W->aff.as<long long>() : nullptr;
    pa.budget = budget;
    pa.dump_limit = dump_limit;
    pa.park = search == kSearchThread ? W->park.as<uint32_t>() : nullptr;
    pa.ready = search == kSearchThread ? W->ready.as<uint32_t>() : nullptr;
  if (search == kSearchThread) {
    int max_n = 0, max_par = 0;  // m - n + 1 bounds a ridge's parents
    for (int i : valid) {
      max_n = std::max(max_n, hd[i].n);
      max_par = std::max(max_par, hd[i].m - hd[i].n + 1);
    }
    pa.rows = rows_variant(max_n, max_par);
  }
    pa.hungry = opt.hungry_items > 0 ? (unsigned long long)opt.hungry_items
                                      : (unsigned long long)n_searches;
    pa.feed = opt.feed_levels > 0 ? opt.feed_levels : (opt.feed_levels < 0 ? (1 << 20) : 8);
    pa.donate = opt.donate_levels > 0 ? opt.donate_levels : (opt.donate_levels < 0 ? 0 : 4);
    pa.donate_every = opt.donate_every > 0 ? opt.donate_every : 2048;
    pa.ready_polls = opt.ready_polls;
    pa.idle_polls = opt.idle_polls;
    pa.ready_xor = opt.test_unpublished ? 0x80000000u : 0u;
    const int idle_pct = (opt.idle_percent > 0 && opt.idle_percent <= 100) ? opt.idle_percent : 20;
    pa.idle_limit = std::max<unsigned long long>(1, (unsigned long long)n_searches * idle_pct / 100);
    const bool trace = getenv("WPM_TRACE") != nullptr;
    pa.trace = trace ? 1 : 0;
    if (trace)
      fprintf(stderr, "[wpm] %d instances, class %d (mw %d nw %d), %s search, %d blocks x %d "
              "threads, budget %lld, ring %llu items of %d words, max depth %d\n", n_valid, k,
              size_class(k).mw, size_class(k).nw, search == kSearchThread ? "thread" : "warp",
              blocks, tpb, budget, ring_cap, iw, max_depth);
    t_stats.search = search;
    t_stats.size_class = k;
    t_stats.searches = n_searches;
    const bool timed = trace || opt.profile;
    if (timed && !W->ev0) {
      CUDA_TRY(cudaEventCreate(&W->ev0));
      CUDA_TRY(cudaEventCreate(&W->ev1));
    }
    cudaEvent_t ev0 = W->ev0, ev1 = W->ev1;
    int pass_no = 0;

    // ---- breadth-first expansion, then depth-first passes -----------------------------
    const auto t_start = std::chrono::steady_clock::now();
    auto out_of_time = [&]() {
      if (opt.time_limit_ms <= 0) return false;
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                          std::chrono::steady_clock::now() - t_start).count();
      return ms >= opt.time_limit_ms;
    };
    timed_out = false;
    unsigned long long head = 0, tail = hq->tail;
    {
      // Without tracing the levels run on the device, as one graph launch: no host round
      // trip per level (small maps take a dozen levels before their frontier is wide enough
      // or their tree is done). The host loop below then finds nothing left to do.
      const unsigned long long live = tail - head;
      if (!trace && opt.graph >= 0 && live > 0 && (long long)live < frontier_target &&
          live * (unsigned long long)max_children + live <= ring_cap) {
        memset(hq, 0, sizeof(QueueCtl));
        hq->head = tail;
        hq->tail = tail;
        hq->limit = tail;
        hq->head_start = head;
        CUDA_TRY(cudaMemcpyAsync(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, s));
        count_copy(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice);
        if (timed) CUDA_TRY(cudaEventRecord(ev0, s));
        const cudaError_t ge = launch_expand_graph(
            W, pa, k, 4 * W->sms, (unsigned long long)frontier_target,
            (unsigned long long)max_children, ring_cap, (unsigned long long)max_depth + 2, s);
        if (ge == cudaSuccess) {
          if (timed) CUDA_TRY(cudaEventRecord(ev1, s));
          CUDA_TRY(cudaMemcpyAsync(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, s));
          count_copy(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost);
          CUDA_TRY(cudaStreamSynchronize(s));
          if (hq->err) return fail(WPM_ERR_NOMEM, "work ring overflow during expansion");
          t_stats.expand_passes += hq->passes;
          t_stats.kernel_launches += 2 * hq->passes;
          if (timed) {
            float ms = 0;
            CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
            t_stats.expand_ms += ms;
          }
          head = hq->head_start;
          tail = hq->tail;
        } else if (ge != cudaErrorNotSupported) {
          return fail(WPM_ERR_CUDA, "expansion graph: %s", cudaGetErrorString(ge));
        }
      }
    }
    for (;;) {
      const unsigned long long live = tail - head;
      if (live == 0 || (long long)live >= frontier_target) break;
      if (live * (unsigned long long)max_children + live > ring_cap) break;  // children must fit
      hq->head = tail;
      hq->tail = tail;
      hq->limit = tail;
      hq->head_start = head;
      hq->err = 0;
      hq->idle = 0;
      hq->nodes = 0;
      CUDA_TRY(cudaMemcpyAsync(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, s));
    count_copy(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice);
      if (timed) CUDA_TRY(cudaEventRecord(ev0, s));
      CUDA_TRY(launch_expand(k, pa, (int)live, 256, s));
      if (timed) CUDA_TRY(cudaEventRecord(ev1, s));
      t_stats.kernel_launches++;
      t_stats.expand_passes++;
      CUDA_TRY(cudaMemcpyAsync(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, s));
    count_copy(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost);
      CUDA_TRY(cudaStreamSynchronize(s));
      if (hq->err) return fail(WPM_ERR_NOMEM, "work ring overflow during expansion");
      float ms = 0;
      if (timed) {
        CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
        t_stats.expand_ms += ms;
      }
      if (trace) {
        fprintf(stderr, "[wpm] expand %d: %llu items -> %llu items, %.3f ms\n", pass_no++, live,
                hq->tail - tail, ms);
      }
      head = tail;
      tail = hq->tail;
    }
    unsigned long long parked = 0;  // searches that parked work in the last pass
    unsigned long long epoch = 0;   // ready-flag stamp of the last pass (the flags were zeroed)
    // Without tracing or a time limit the pass loop runs on the device: one graph launch, whose
    // conditional while node repeats prep, pass and check until no item or parked search is
    // left (no host round trip between passes).
    if (tail > head && !trace && opt.time_limit_ms <= 0 && opt.graph >= 0) {
      memset(hq, 0, sizeof(QueueCtl));
      hq->head = head;
      hq->tail = tail;
      hq->limit = tail;
      hq->head_start = head;
      CUDA_TRY(cudaMemcpyAsync(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, s));
      count_copy(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice);
      if (timed) CUDA_TRY(cudaEventRecord(ev0, s));
      const cudaError_t ge = launch_pass_graph(W, pa, k, search, blocks, tpb, s);
      if (ge == cudaSuccess) {
        if (timed) CUDA_TRY(cudaEventRecord(ev1, s));
        CUDA_TRY(cudaMemcpyAsync(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, s));
        count_copy(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost);
        CUDA_TRY(cudaStreamSynchronize(s));
        if (hq->err & 1ull) return fail(WPM_ERR_NOMEM, "work ring overflow (raise ring_items)");
        if (hq->err & 2ull) return fail(WPM_ERR_LIMIT, "search stack overflow");
        if (hq->err & 4ull)
          return fail(WPM_ERR_TIMEOUT, "a work item was not published within the bounded wait");
        if (hq->err & 8ull) return fail(WPM_ERR_CUDA, "pass loop did not finish");
        t_stats.dfs_passes += hq->passes;
        t_stats.kernel_launches += 3 * hq->passes;
        t_stats.graph_launches++;
        if (timed) {
          float ms = 0;
          CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
          t_stats.dfs_ms += ms;
        }
        head = tail = 0;  // all done
      } else if (ge != cudaErrorNotSupported) {
        return fail(WPM_ERR_CUDA, "pass graph: %s", cudaGetErrorString(ge));
      }
    }
    while (tail > head || parked > 0) {
      if (out_of_time()) {
        timed_out = true;
        break;
      }
      hq->head = head;
      hq->tail = tail;
      hq->limit = tail;
      hq->head_start = head;
      hq->err = 0;
      hq->idle = 0;
      hq->nodes = 0;
      hq->parked = 0;
      hq->iters = hq->lanes_step = hq->lanes_fetch = hq->lanes_dump = hq->lanes_stopped = 0;
      hq->waiting = hq->exited = hq->full = 0;
      hq->epoch = ++epoch;
      if (opt.time_limit_ms > 0) {  // a long pass ends by itself when the time is up
        const long long used = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now() - t_start).count();
        pa.time_left_ns = (unsigned long long)std::max<long long>(
            1, (long long)opt.time_limit_ms * 1000000ll - used);
      }
      CUDA_TRY(cudaMemcpyAsync(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice, s));
    count_copy(W->q.p, hq, sizeof(QueueCtl), cudaMemcpyHostToDevice);
      if (timed) CUDA_TRY(cudaEventRecord(ev0, s));
      CUDA_TRY(launch_dfs(k, search, pa, blocks, tpb, s));
      if (timed) CUDA_TRY(cudaEventRecord(ev1, s));
      t_stats.kernel_launches++;
      t_stats.dfs_passes++;
      CUDA_TRY(cudaMemcpyAsync(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost, s));
    count_copy(hq, W->q.p, sizeof(QueueCtl), cudaMemcpyDeviceToHost);
      CUDA_TRY(cudaStreamSynchronize(s));
      if (hq->err & 1ull) return fail(WPM_ERR_NOMEM, "work ring overflow (raise ring_items)");
      if (hq->err & 2ull) return fail(WPM_ERR_LIMIT, "search stack overflow");
      if (hq->err & 4ull)
        return fail(WPM_ERR_TIMEOUT, "a work item was not published within the bounded wait");
      // per-thread passes also take items written during the pass (their head never passes
      // the tail); per-warp passes take only items that were there when it began
      const unsigned long long taken_to =
          search == kSearchThread ? std::min(hq->head, hq->tail) : std::min(hq->head, tail);
      t_stats.items += taken_to - head;
      float ms = 0;
      if (timed) {
        CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
        t_stats.dfs_ms += ms;
      }
      if (trace) {
        fprintf(stderr, "[wpm] dfs %d: %llu items, %llu taken, %llu new, %llu parked, %llu nodes, "
                "%.3f ms", pass_no++, tail - head, taken_to - head, hq->tail - tail, hq->parked,
                hq->nodes, ms);
        if (hq->iters)
          fprintf(stderr, "; warp iterations %llu, lanes/iteration: step %.2f fetch %.3f stopped "
                  "%.2f; dumps %llu", hq->iters, (double)hq->lanes_step / hq->iters,
                  (double)hq->lanes_fetch / hq->iters, (double)hq->lanes_stopped / hq->iters,
                  hq->lanes_dump);
        fprintf(stderr, "\n");
      }
      head = taken_to;
      tail = hq->tail;
      parked = hq->parked;
    }
  }

  // ---- counters ----------------------------------------------------------------------
  unsigned long long *hc2 = W->h_ctr.as<unsigned long long>();
  CUDA_TRY(cudaMemcpyAsync(hc2, W->ctr.p, 8ull * kCtrN * n_inst, cudaMemcpyDeviceToHost, s));
  count_copy(hc2, W->ctr.p, 8ull * kCtrN * n_inst, cudaMemcpyDeviceToHost);
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> sorted_ids;
  std::vector<unsigned long long> seg(1, 0);
  unsigned long long max_len = 0;
  for (int i : valid) {
    InstResult &r = res[i];
    const unsigned long long *c = hc2 + kCtrN * i;
    r.count = c[kCtrCount];
    r.found = r.count;
    r.nodes = c[kCtrNodes];
    r.probes = c[kCtrProbes];
    if (timed_out && c[kCtrLive] != 0) {  // items of this instance are still in the ring
      r.status = fail(WPM_ERR_TIMEOUT, "instance %d: time limit reached (partial counts)", i);
      continue;
    }
    if (list) {
      const unsigned long long fill = c[kCtrFill];
      if (fill != r.count)  // every emission reserves one slot
        return fail(WPM_ERR_CUDA, "instance %d: %llu emitted, %llu slots", i, r.count, fill);
      if (fill > ho[i].cap) {
        r.status = fail(WPM_ERR_CAPACITY, "instance %d: %llu masks, capacity %llu", i, fill,
                        ho[i].cap);
      } else if (fill > 0) {
        sorted_ids.push_back(i);
        seg.push_back(seg.back() + fill);
        max_len = std::max(max_len, fill);
      }
    }
  }
  if (!list || sorted_ids.empty()) return WPM_OK;

  // ---- per-instance merge sort on the GPU -----------------------------------------------
  const int ns = (int)sorted_ids.size();
  WPM_TRY(W->seg.ensure(8ull * (ns + 1)));
  WPM_TRY(W->h_seg.ensure(8ull * (ns + 1) + 4ull * ns));
  WPM_TRY(W->ids.ensure(4ull * n_inst + 4ull * ns + 4));
  unsigned long long *hseg = W->h_seg.as<unsigned long long>();
  int32_t *hsid = (int32_t *)(hseg + ns + 1);
  for (int j = 0; j <= ns; j++) hseg[j] = seg[j];
  for (int j = 0; j < ns; j++) hsid[j] = sorted_ids[j];
  int32_t *d_sid = W->ids.as<int32_t>() + n_inst;
  CUDA_TRY(cudaMemcpyAsync(W->seg.p, hseg, 8ull * (ns + 1), cudaMemcpyHostToDevice, s));
  count_copy(W->seg.p, hseg, 8ull * (ns + 1), cudaMemcpyHostToDevice);
  CUDA_TRY(cudaMemcpyAsync(d_sid, hsid, 4ull * ns, cudaMemcpyHostToDevice, s));
  count_copy(d_sid, hsid, 4ull * ns, cudaMemcpyHostToDevice);
  const unsigned long long total = seg.back();
  int parity = 0;
  for (unsigned long long runlen = 1; runlen < max_len; runlen *= 2) {
    CUDA_TRY(launch_sort_pass(W->inst.as<InstDesc>(), W->outd.as<OutDesc>(), d_sid, ns,
                              W->seg.as<unsigned long long>(), total, runlen, parity, s));
    t_stats.kernel_launches++;
    t_stats.sort_passes++;
    parity ^= 1;
  }
  if (parity) {  // one copying pass brings the result back to `out`
    CUDA_TRY(launch_sort_pass(W->inst.as<InstDesc>(), W->outd.as<OutDesc>(), d_sid, ns,
                              W->seg.as<unsigned long long>(), total, 1ull << 62, 1, s));
    t_stats.kernel_launches++;
    t_stats.sort_passes++;
  }

  // ---- post-filters (Algorithm 4.4, lines 8-12) on the sorted lists ---------------------
  bool any_post = false;
  for (int i : sorted_ids) any_post |= hd[i].post != 0;
  if (any_post) {
    WPM_TRY(W->keep.ensure(total + 256));
    CUDA_TRY(launch_post_filter(W->inst.as<InstDesc>(), W->outd.as<OutDesc>(), d_sid, ns,
                                W->seg.as<unsigned long long>(), total, W->keep.as<uint8_t>(), s));
    CUDA_TRY(launch_post_compact(W->inst.as<InstDesc>(), W->outd.as<OutDesc>(), d_sid, ns,
                                 W->seg.as<unsigned long long>(), W->keep.as<uint8_t>(),
                                 W->ctr.as<unsigned long long>(), s));
    t_stats.kernel_launches += 2;
    CUDA_TRY(cudaMemcpyAsync(hc2, W->ctr.p, 8ull * kCtrN * n_inst, cudaMemcpyDeviceToHost, s));
    count_copy(hc2, W->ctr.p, 8ull * kCtrN * n_inst, cudaMemcpyDeviceToHost);
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int i : sorted_ids)
      if (hd[i].post) res[i].count = hc2[kCtrN * i + kCtrCount];
  }

  // ---- copy-out -------------------------------------------------------------------------
  const auto tc0 = std::chrono::steady_clock::now();
  std::vector<CopySeg> cs;
  std::vector<unsigned long long> cp(1, 0);
  std::vector<int> host_ids;
  for (int j = 0; j < ns; j++) {
    const int i = sorted_ids[j];
    if (outs[i].masks_on_device) continue;
    host_ids.push_back(i);
  }
  size_t stage_words = 0;
  for (int i : host_ids) stage_words += res[i].count * (unsigned long long)hd[i].ow;
  WPM_TRY(W->stage.ensure(8 * stage_words + 256));
  // the host side of the staging area: two chunks of at most kStageChunk words
  const size_t chunk = std::min<size_t>(opt.stage_chunk > 0 ? (size_t)opt.stage_chunk : kStageChunk,
                                        std::max<size_t>(stage_words, 1));
  WPM_TRY(W->h_stage.ensure(2 * 8 * chunk + 256));
  size_t sw = 0;
  for (int j = 0; j < ns; j++) {
    const int i = sorted_ids[j];
    const unsigned long long words = res[i].count * (unsigned long long)hd[i].ow;
    CopySeg c;
    c.src = ho[i].out;
    if (outs[i].masks_on_device) {
      c.dst = outs[i].masks;
    } else {
      c.dst = W->stage.as<uint64_t>() + sw;
      sw += words;
    }
    cs.push_back(c);
    cp.push_back(cp.back() + words);
  }
  WPM_TRY(W->segs.ensure(sizeof(CopySeg) * cs.size() + 8 * cp.size()));
  WPM_TRY(W->h_segs.ensure(sizeof(CopySeg) * cs.size() + 8 * cp.size()));
  memcpy(W->h_segs.p, cs.data(), sizeof(CopySeg) * cs.size());
  memcpy(W->h_segs.as<char>() + sizeof(CopySeg) * cs.size(), cp.data(), 8 * cp.size());
  CUDA_TRY(cudaMemcpyAsync(W->segs.p, W->h_segs.p, sizeof(CopySeg) * cs.size() + 8 * cp.size(),
                           cudaMemcpyHostToDevice, s));
  t_stats.kernel_launches++;
  CUDA_TRY(launch_segment_copy(W->segs.as<CopySeg>(), (int)cs.size(),
                               (const unsigned long long *)(W->segs.as<char>() +
                                                            sizeof(CopySeg) * cs.size()),
                               cp.back(), s));
  count_copy(W->h_stage.p, W->stage.p, 8 * sw, cudaMemcpyDeviceToHost);

  // staging -> the caller's host buffers, chunk by chunk through the two halves of h_stage:
  // the device-to-host copy of chunk c + 1 runs while host threads copy chunk c out (one
  // copy of the whole list into one large page-locked buffer ran several times slower than
  // copies of a few hundred MB into a buffer that is reused)
  std::vector<std::pair<size_t, int>> parts;  // (staging word offset, instance)
  size_t total_words = 0;
  for (int i : host_ids) {
    parts.emplace_back(total_words, i);
    total_words += res[i].count * (size_t)hd[i].ow;
  }
  // staging words [lo, hi), held in `src` from word `base` on
  auto copy_range = [&](size_t lo, size_t hi, const uint64_t *src, size_t base) {
    for (const auto &pi : parts) {
      const size_t a = pi.first, words = res[pi.second].count * (size_t)hd[pi.second].ow;
      const size_t x = std::max(a, lo), y = std::min(a + words, hi);
      if (x < y) memcpy(outs[pi.second].masks + (x - a), src + (x - base), 8 * (y - x));
    }
  };
  for (cudaEvent_t &e : W->ev_stage)
    if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const size_t n_chunks = (sw + chunk - 1) / chunk;
  auto half = [&](size_t c) { return W->h_stage.as<uint64_t>() + (c & 1) * chunk; };
  auto issue = [&](size_t c) -> cudaError_t {
    const size_t lo = c * chunk, len = std::min(chunk, sw - lo);
    cudaError_t e = cudaMemcpyAsync(half(c), W->stage.as<uint64_t>() + lo, 8 * len,
                                    cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? cudaEventRecord(W->ev_stage[c & 1], s) : e;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  double host_ms = 0;
  if (n_chunks) CUDA_TRY(issue(0));
  for (size_t c = 0; c < n_chunks; c++) {
    // the half that chunk c + 1 fills held chunk c - 1, copied out in the last iteration
    if (c + 1 < n_chunks) CUDA_TRY(issue(c + 1));
    CUDA_TRY(cudaEventSynchronize(W->ev_stage[c & 1]));
    const auto th0 = std::chrono::steady_clock::now();
    const size_t lo = c * chunk, hi = std::min(sw, lo + chunk);
    const uint64_t *src = half(c);
    const size_t n_thr = std::min<size_t>(std::min(16u, hw), 1 + (hi - lo) / (1u << 20));
    if (n_thr <= 1) {
      copy_range(lo, hi, src, lo);
    } else {
      std::vector<std::thread> th;
      const size_t per = (hi - lo + n_thr - 1) / n_thr;
      for (size_t t = 0; t < n_thr; t++)
        th.emplace_back(copy_range, lo + t * per, std::min(hi, lo + (t + 1) * per), src, lo);
      for (auto &t : th) t.join();
    }
    host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0)
                   .count();
  }
  CUDA_TRY(cudaStreamSynchronize(s));  // the device-side outputs too
  t_stats.copy_out_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count();
  t_stats.host_copy_ms = host_ms;
  return WPM_OK;
}

static void fill_output(const InstResult &r, wpm_output *o) {
  o->count = r.count;
  o->found = r.found;
  o->nodes = r.nodes;
  o->probes = r.probes;
  o->words_per_mask = r.ow;
  o->M = r.M;
  o->N = r.N;
  o->status = r.status;
}

static RunOptions options_from(const wpm_tuning *t, int mode) {
  RunOptions o;
  o.mode = mode;
  if (t) {
    o.tpb = t->threads_per_block;
    o.budget = t->budget;
    o.frontier_target = t->frontier_target;
    o.ring_items = t->ring_items;
    o.idle_percent = t->idle_percent;
    o.search = t->search;
    o.profile = t->profile != 0;
    o.time_limit_ms = t->time_limit_ms;
    o.feed_levels = t->feed_levels;
    o.donate_levels = t->donate_levels;
    o.donate_every = t->donate_every;
    o.graph = t->graph;
    o.engine = t->engine;
    o.sweep_max_s = t->sweep_max_s;
    o.hungry_items = t->hungry_items;
    o.ready_polls = t->ready_polls;
    o.idle_polls = t->idle_polls;
    o.test_unpublished = t->test_unpublished;
    o.stage_chunk = t->stage_chunk_words;
  }
  return o;
}

static int check_output(const wpm_output *out, int mode) {
  if (!out) return fail(WPM_ERR_INPUT, "out is NULL");
  if (mode != WPM_MODE_LIST && mode != WPM_MODE_COUNT)
    return fail(WPM_ERR_INPUT, "mode %d is neither list nor count", mode);
  if (mode == WPM_MODE_LIST && out->capacity > 0 && !out->masks)
    return fail(WPM_ERR_INPUT, "list mode with capacity but no buffer");
  return WPM_OK;
}

static int single(HostInst &h, wpm_output *out, int mode) {
  Workspace *W = nullptr;
  WPM_TRY(get_workspace(&W));
  std::vector<HostInst> v(1, h);
  std::vector<InstResult> res;
  const int rc = run(W, v, options_from(nullptr, mode), W->own, out, res, nullptr);
  if (rc != WPM_OK) return rc;
  fill_output(res[0], out);
  return res[0].status;
}

}  // namespace wpm

using namespace wpm;

// ---- autotuner ---------------------------------------------------------------------------
// Signature of a batch: smallest and largest n, whether any map is primal, and the size
// of the batch to a power of two (few maps and many maps want different searches).
static uint64_t batch_signature(const wpm_instance *inst, int count) {
  int lo = 99, hi = 0, primal = 0;
  for (int i = 0; i < count; i++) {
    lo = std::min(lo, (int)inst[i].n);
    hi = std::max(hi, (int)inst[i].n);
    primal |= inst[i].kind == WPM_LAMBDA_PRIMAL;
  }
  int size_log2 = 0;
  while ((1 << (size_log2 + 1)) <= count && size_log2 < 30) size_log2++;
  return ((uint64_t)size_log2 << 24) | ((uint64_t)lo << 16) | ((uint64_t)hi << 1) |
         (uint64_t)primal;
}

static std::map<uint64_t, wpm_tuning> g_tuned;  // guarded by g_mu

static bool tuned_for(const wpm_instance *inst, int count, wpm_tuning *out) {
  if (count <= 0 || !inst) return false;
  auto it = g_tuned.find(batch_signature(inst, count));
  if (it == g_tuned.end()) return false;
  *out = it->second;
  return true;
}

// The candidates: per-warp searches (two frontier sizes), per-thread searches with three
// hand-over chunks and a larger frontier.
constexpr int kTuneRounds = 2;

static std::vector<wpm_tuning> tune_candidates() {
  std::vector<wpm_tuning> c;
  auto add = [&](int search, int frontier, int donate, int every) {
    wpm_tuning t;
    memset(&t, 0, sizeof(t));
    t.search = search;
    t.frontier_target = frontier;
    t.donate_levels = donate;
    t.donate_every = every;
    c.push_back(t);
  };
  add(kSearchWarp, 0, 0, 0);
  add(kSearchWarp, 1 << 18, 0, 0);
  add(kSearchThread, 0, 4, 2048);
  add(kSearchThread, 0, 2, 512);
  add(kSearchThread, 0, 8, 8192);
  add(kSearchThread, 1 << 19, 4, 2048);
  return c;
}

extern "C" {

const char *wpm_last_error(void) { return t_err.c_str(); }

int wpm_last_run_stats(wpm_run_stats *out) {
  if (!out) return fail(WPM_ERR_INPUT, "out is NULL");
  *out = t_stats;
  return WPM_OK;
}

int wpm_version(void) { return 1; }

void wpm_release_workspace(void) {
  std::lock_guard<std::mutex> g(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  auto it = g_ws.find(dev);
  if (it == g_ws.end()) return;
  cudaStreamSynchronize(it->second->own);
  it->second->release();
  cudaStreamDestroy(it->second->own);
  delete it->second;
  g_ws.erase(it);
}

int wpm_candidate_facets(const uint32_t *lambda_cols, int kind, int n, int m, uint16_t *facets_out,
                         int cap) {
  std::lock_guard<std::mutex> g(g_mu);
  t_err.clear();
  HostInst h;
  WPM_TRY(copy_map(lambda_cols, kind, n, m, h));
  Workspace *W = nullptr;
  WPM_TRY(get_workspace(&W));
  std::vector<HostInst> v(1, h);
  std::vector<InstResult> res;
  std::vector<uint16_t> f;
  RunOptions o;
  o.setup_only = true;
  WPM_TRY(run(W, v, o, W->own, nullptr, res, &f));
  if (res[0].status != WPM_OK) return res[0].status;
  if ((int)f.size() > cap) return fail(WPM_ERR_CAPACITY, "%zu candidate facets, cap %d", f.size(), cap);
  if (!f.empty()) {
    if (!facets_out) return fail(WPM_ERR_INPUT, "facets_out is NULL");
    memcpy(facets_out, f.data(), 2 * f.size());
  }
  return (int)f.size();
}

int wpm_enumerate(const uint32_t *lambda_cols, int kind, int n, int m, const wpm_conditions *cond,
                  wpm_output *out, int mode) {
  std::lock_guard<std::mutex> g(g_mu);
  t_err.clear();
  WPM_TRY(check_output(out, mode));
  HostInst h;
  WPM_TRY(copy_map(lambda_cols, kind, n, m, h));
  WPM_TRY(copy_conditions(cond, h));
  return single(h, out, mode);
}

int wpm_enumerate_facets(const uint16_t *facets, int M, int n, int m, const wpm_conditions *cond,
                         wpm_output *out, int mode) {
  std::lock_guard<std::mutex> g(g_mu);
  t_err.clear();
  WPM_TRY(check_output(out, mode));
  HostInst h;
  WPM_TRY(copy_facet_list(facets, M, n, m, h));
  WPM_TRY(copy_conditions(cond, h));
  return single(h, out, mode);
}

int wpm_enumerate_batch(const wpm_instance *inst, int count, wpm_output *outs, int mode,
                        const wpm_tuning *tuning, void *cuda_stream) {
  std::lock_guard<std::mutex> g(g_mu);
  t_err.clear();
  if (count < 0 || (count > 0 && (!inst || !outs))) return fail(WPM_ERR_INPUT, "bad batch arrays");
  wpm_tuning tuned;
  if (!tuning && tuned_for(inst, count, &tuned)) tuning = &tuned;
  std::vector<HostInst> hi;
  std::vector<int> where;  // hi index -> caller index
  std::vector<int> status(count, WPM_OK);
  for (int i = 0; i < count; i++) {
    int rc = check_output(&outs[i], mode);
    HostInst h;
    if (rc == WPM_OK) rc = copy_map(inst[i].lambda_cols, inst[i].kind, inst[i].n, inst[i].m, h);
    if (rc == WPM_OK) rc = copy_conditions(inst[i].cond, h);
    status[i] = rc;
    if (rc == WPM_OK) {
      hi.push_back(std::move(h));
      where.push_back(i);
    }
  }
  Workspace *W = nullptr;
  WPM_TRY(get_workspace(&W));
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : W->own;
  std::vector<wpm_output> o2(hi.size());
  for (size_t j = 0; j < hi.size(); j++) o2[j] = outs[where[j]];
  std::vector<InstResult> res;
  const int rc = run(W, hi, options_from(tuning, mode), s, o2.data(), res, nullptr);
  if (rc != WPM_OK) {  // the run as a whole failed: no instance has a result
    for (size_t j = 0; j < hi.size(); j++) outs[where[j]].status = rc;
    return rc;
  }
  int first = WPM_OK;
  for (size_t j = 0; j < hi.size(); j++) {
    fill_output(res[j], &outs[where[j]]);
    status[where[j]] = res[j].status;
  }
  for (int i = 0; i < count; i++) {
    outs[i].status = status[i];
    if (status[i] != WPM_OK && first == WPM_OK) first = status[i];
  }
  return first;
}

int wpm_autotune(const wpm_instance *inst, int count, int sample, wpm_tuning *best,
                 double *best_ms, void *cuda_stream) {
  std::lock_guard<std::mutex> g(g_mu);
  t_err.clear();
  if (count <= 0 || !inst || !best) return fail(WPM_ERR_INPUT, "bad autotune arguments");
  if (sample <= 0) sample = 256;
  const int stride = std::max(1, count / sample);
  std::vector<HostInst> hi;
  for (int i = 0; i < count; i += stride) {
    HostInst h;
    if (copy_map(inst[i].lambda_cols, inst[i].kind, inst[i].n, inst[i].m, h) != WPM_OK ||
        copy_conditions(inst[i].cond, h) != WPM_OK)
      continue;
    hi.push_back(std::move(h));
  }
  if (hi.empty()) return fail(WPM_ERR_INPUT, "autotune: no valid instance in the sample");
  Workspace *W = nullptr;
  WPM_TRY(get_workspace(&W));
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : W->own;
  // every candidate is timed in kTuneRounds interleaved rounds and keeps its best time: the
  // per-thread candidates lie within a few percent of one another, about the noise of one run
  const std::vector<wpm_tuning> cands = tune_candidates();
  std::vector<double> t_best(cands.size(), 1e300);
  std::vector<InstResult> res;
  for (int round = 0; round < kTuneRounds; round++) {
    for (size_t ci = 0; ci < cands.size(); ci++) {
      std::vector<HostInst> h2 = hi;
      CUDA_TRY(cudaStreamSynchronize(s));
      const auto t0 = std::chrono::steady_clock::now();
      WPM_TRY(run(W, h2, options_from(&cands[ci], WPM_MODE_COUNT), s, nullptr, res, nullptr));
      CUDA_TRY(cudaStreamSynchronize(s));
      const double ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - t0).count();
      t_best[ci] = std::min(t_best[ci], ms);
    }
  }
  size_t wi = 0;
  for (size_t ci = 1; ci < cands.size(); ci++)
    if (t_best[ci] < t_best[wi]) wi = ci;
  const wpm_tuning win = cands[wi];
  const double best_t = t_best[wi];
  g_tuned[batch_signature(inst, count)] = win;
  *best = win;
  if (best_ms) *best_ms = best_t;
  return WPM_OK;
}

}  // extern "C"
