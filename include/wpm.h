/*
 * wpm.h -- C ABI of the GB300 weak pseudo-manifold enumeration library (libwpm.so).
 *
 * The library enumerates every weak pseudo-manifold (WPM) whose facets are drawn from
 * the candidate facets of a mod-2 characteristic map (Choi, Jang, Vallee, arXiv
 * 2301.00806). A pure complex K of dimension n-1 on [m] is a WPM when every ridge
 * ((n-1)-subset) lies in exactly 0 or 2 facets of K: the ridge-facet incidence matrix A
 * gives A K in {0, 2}^N (Section 2.1, Proposition 2.1). The output for a map lambda and a
 * set of properties G is
 *     { K subset of F(lambda) : A K in {0,2}^N and g(K) > 0 for every g in G }
 * returned as a count and, in list mode, as facet bitmasks.
 *
 * Every step after the inputs are copied to the GPU runs in CUDA kernels on the device:
 * candidate facets, ridges and incidence tables, the search, the output sort.
 *
 * Conventions shared by every entry point
 *   - Vertices are 0..m-1 (m <= 16). A facet is a uint16 vertex mask.
 *   - Candidate facets are numbered 0..M-1 in lexicographic order of their sorted vertex
 *     tuples. A facet set (an output K, a forced mask) is a bitmask of
 *     W = ceil(M/64) uint64 words: facet j is bit j%64 of word j/64.
 *   - Output masks are sorted ascending as multiword unsigned integers, word W-1 the most
 *     significant.
 *   - The empty complex satisfies Proposition 2.1; it is output when every property
 *     holds at K = 0.
 *   - Calls are serialised by a library-wide lock; the library allocates and caches its
 *     device workspace itself (it grows, and is freed by wpm_release_workspace or at
 *     exit).
 *   - Every function returns WPM_OK (0) or a negative WPM_ERR_* code; wpm_last_error()
 *     then describes the failure (thread-local string owned by the library).
 */
#ifndef WPM_H
#define WPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------------- */
#define WPM_OK            0
#define WPM_ERR_INPUT    -1  /* malformed argument (sizes, rank, repeated dual rows, ...)  */
#define WPM_ERR_CAPACITY -2  /* an output buffer is too small; wpm_output.count holds the
                                number of masks needed and nothing was written            */
#define WPM_ERR_CUDA     -3  /* a CUDA call failed                                        */
#define WPM_ERR_TIMEOUT  -4  /* a bounded device wait ran out                             */
#define WPM_ERR_NOMEM    -5  /* device or host allocation failed                          */
#define WPM_ERR_LIMIT    -6  /* the instance exceeds a library limit below                */

/* ---- limits ------------------------------------------------------------------------ */
#define WPM_MAX_VERTICES 16    /* m                                                       */
#define WPM_MAX_FACETS   2048  /* M, candidate facets per instance                        */
#define WPM_MAX_RIDGES   4096  /* N, ridges with at least one candidate parent            */
#define WPM_MAX_AFFINE   4     /* general affine properties per instance                  */

/* ---- map forms (Section 3.1) ------------------------------------------------------- */
#define WPM_LAMBDA_PRIMAL 0  /* lambda_cols[i] = lambda(i) in Z2^n, bit k = row k.
                                Candidates: n-subsets sigma with lambda(sigma) a basis of
                                Z2^n (the non-singularity condition).                     */
#define WPM_LAMBDA_DUAL   1  /* lambda_cols[i] = dual row lambda-bar(i) in Z2^(m-n).
                                Candidates: n-subsets whose complement indexes a basis of
                                Z2^(m-n) (linear Gale duality, Proposition 4.2). The rows
                                must be nonzero, distinct (an injective DCM) and of rank
                                m-n.                                                     */

/* ---- modes ------------------------------------------------------------------------- */
#define WPM_MODE_LIST  0  /* count and sorted masks */
#define WPM_MODE_COUNT 1  /* count only             */

/* ---- the upper-bound-theorem property (Section 4.2) -------------------------------- */
#define WPM_CAP_NONE -1  /* no bound on |K|                                               */
#define WPM_CAP_UBT  -2  /* |K| <= f_{n-1}(C^n(n+4)) = C(n+4-ceil(n/2),4)+C(n+3-floor(n/2),4),
                            the property g(K) = f - |K| + 1 > 0; requires m = n + 4       */

/*
 * Properties G (Section 2.1 "properties"; Section 4.2; Section 4.4). All pointers are
 * HOST pointers, read during the call only; NULL / 0 means absent.
 */
typedef struct {
    int32_t ubt_cap;            /* >= 0: |K| <= ubt_cap; WPM_CAP_NONE; WPM_CAP_UBT          */
    int32_t require_base_facet; /* nonzero: facet {0..n-1} must be in K (the normal form
                                   lambda = [I_n M] puts facet {1..n} in K, Section 3.1)    */
    int32_t n_facets;           /* M the masks / coefficient rows below were built for; it
                                   must equal the instance's M when any of them is given    */
    const uint64_t *forced_in;  /* ceil(M/64) words: facets that must be in K (Section 4.4,
                                   condition (1))                                           */
    const uint64_t *forced_out; /* ceil(M/64) words: facets that must not be in K (Section
                                   4.4, condition (2))                                      */
    int32_t n_affine;           /* <= WPM_MAX_AFFINE general properties
                                   g(K) = c0 + sum_j c_j k_j > 0                             */
    const int32_t *affine_c0;   /* [n_affine]                                               */
    const int32_t *affine_coef; /* [n_affine * M], row a = coefficients of property a;
                                   |c| <= 2^20                                              */
    int32_t post_filter;        /* WPM_POST_* flags: filters applied to the found WPMs
                                   (Algorithm 4.4, lines 8-12); list mode only, m <= 15      */
    int32_t reserved;
} wpm_conditions;

/* Post-filters (Algorithm 4.4): keep K only when it uses all m vertices, i.e. Pic(K) =
   m - n (line 9 discards Pic(K) < 4), and/or when it satisfies the seedness condition of
   Proposition 3.1 (line 10: no edge {v, w} of K lies, for every minimal non-face of K, in
   both or in neither). */
#define WPM_POST_PIC   1
#define WPM_POST_SEED  2

/*
 * Results of one instance. Fields marked "in" are set by the caller, "out" by the library.
 * In list mode the caller provides `masks` with room for `capacity` masks of
 * `words_per_mask` words; the pointer is a device pointer when masks_on_device is nonzero.
 * If the count exceeds `capacity` the call returns WPM_ERR_CAPACITY with `count` set to the
 * number needed, and the caller re-calls with a larger buffer.
 */
typedef struct {
    uint64_t count;          /* out: number of WPMs (including the empty one if output)   */
    uint64_t nodes;          /* out: search nodes of the canonical tree                   */
    uint64_t probes;         /* out: rejected children of the canonical tree              */
    uint64_t *masks;         /* in: output buffer (list mode), or NULL in count mode      */
    uint64_t capacity;       /* in: masks the buffer holds                                 */
    int32_t masks_on_device; /* in: nonzero when `masks` is a device pointer              */
    int32_t words_per_mask;  /* out: ceil(M/64) (at least 1)                               */
    int32_t M;               /* out: candidate facets                                      */
    int32_t N;               /* out: ridges                                                */
    int32_t status;          /* out: this instance's WPM_* code (batched calls)            */
    int32_t reserved;
    uint64_t found;          /* out: WPMs the search found, before any post-filter (equals
                                count when wpm_conditions.post_filter is 0)                 */
} wpm_output;

/* One instance of a batch. Pointers are host pointers, read during the call only. */
typedef struct {
    int32_t kind;                /* WPM_LAMBDA_PRIMAL or WPM_LAMBDA_DUAL                    */
    int32_t n;                   /* facet size (dimension + 1), 2..12                       */
    int32_t m;                   /* vertices, n < m <= 16                                   */
    int32_t reserved;
    const uint32_t *lambda_cols; /* m entries, see the map forms above                      */
    const wpm_conditions *cond;  /* NULL: no properties                                     */
} wpm_instance;

/*
 * Search tuning. Zero fields take the library's defaults (a tuned table keyed by the
 * instance size class). frontier_target: breadth-first frontier items to reach before
 * depth-first passes; budget: most search nodes per thread per depth-first pass;
 * threads_per_block: 64..512 (multiple of 32); ring_items: capacity of the device work
 * ring in items.
 */
typedef struct {
    int32_t frontier_target;
    int32_t budget;
    int32_t threads_per_block;
    int32_t idle_percent;   /* per-warp searches: a depth-first pass ends (busy searches
                               return their work to the ring) once this percentage of
                               searches is idle; 0 = 20                                    */
    int64_t ring_items;
    int32_t search;         /* 1: one search per thread, 2: one search per warp, 0: by size
                               (per thread for batches of 16 or more maps of the size
                               classes of n = 7..10)                                       */
    int32_t profile;        /* nonzero: time every depth-first pass with CUDA events on the
                               run's stream (see wpm_last_run_stats)                       */
    int32_t time_limit_ms;  /* > 0: launch no depth-first pass after this much wall time;
                               unfinished instances then report WPM_ERR_TIMEOUT with the
                               counts reached so far (no masks)                            */
    /* Per-thread searches hand work over inside a pass: while searches wait for items and
       the ring holds fewer items than are waiting, a busy search gives its donate_levels
       shallowest open levels (0 = 4, -1 = none) to the ring and goes on with the rest. A
       search that leaves a pass with work (budget or time spent, or no room in the ring)
       gives its feed_levels shallowest levels (0 = 8, -1 = all) while the ring holds fewer
       than hungry_items items (0 = one per search), and parks the rest until the next
       pass. donate_every: nodes a search searches between two hand-overs (0 = 2048).     */
    int32_t feed_levels;
    int64_t hungry_items;
    int32_t donate_levels;
    int32_t donate_every;
    int32_t graph;          /* 0: the breadth-first levels and the depth-first pass loop each
                               run as one CUDA graph launch (a conditional while node; the
                               pass loop not with a time limit, neither with tracing);
                               -1: the host launches each level and each pass             */
    int32_t engine;         /* 0: the canonical ridge-driven search. 1: the GF(2) cycle-space
                               sweep of Section 2.1 over its convenient basis: rows of forced
                               facets (and the base facet) fix coordinates of X as in Section
                               4.4, Z blocks over ridges with disjoint parents allow at most two
                               generators each, the other generators are swept freely. 2: the
                               plain sweep of all 2^s elements of ker_Z2 A in Gray-code order.
                               Both check Proposition 2.1 and the properties; maps with M <=
                               896, N <= 3200 and s <= 64, else WPM_ERR_LIMIT. Same counts and
                               lists as the search; `nodes` then counts the combinations
                               visited (|X| for engine 1, 2^s for engine 2), `probes` 0       */
    int32_t sweep_max_s;    /* largest log2 of the combinations a sweep may visit (0 = 30,
                               at most 48); beyond it WPM_ERR_LIMIT                           */
    /* Bounds of the per-thread passes' device waits (they only end waits that end by
       themselves in a correct run). ready_polls: polls of a work item's ready flag before the
       reader gives up; the kernel then returns and the run fails with WPM_ERR_TIMEOUT (0 =
       2^22, about half a second; a bound of a few polls can run out before a writer
       publishes, in a correct run too). idle_polls: fruitless steps after which a search waiting
       for work leaves the pass (0 = 2^14); leaving early never changes counts.           */
    int32_t ready_polls;
    int32_t idle_polls;
    int32_t test_unpublished; /* test hook, 0 in normal use: nonzero makes readers of items
                               written during a pass wait for a ready stamp that no writer
                               raises, so every such wait runs out (WPM_ERR_TIMEOUT)        */
    int32_t stage_chunk_words; /* host outputs leave the device in chunks of this many u64
                               words through two page-locked halves of a staging buffer, one
                               chunk's device-to-host copy overlapping the copy of the last one
                               into the caller's buffers (0 = 2^25, 256 MB)                  */
} wpm_tuning;

/* Statistics of the calling thread's last enumeration run. */
typedef struct {
    uint64_t kernel_launches;  /* kernels the run launched (setup, roots, passes, sort, copy)  */
    uint64_t expand_passes;    /* breadth-first passes                                         */
    uint64_t dfs_passes;       /* depth-first passes                                           */
    uint64_t sort_passes;      /* merge passes of the output sort                              */
    uint64_t items;            /* work items taken by the depth-first passes                   */
    double dfs_ms;             /* summed duration of the depth-first passes (profile only)     */
    double expand_ms;          /* summed duration of the expansion passes (profile only)      */
    int32_t search;            /* search mode used (1 thread, 2 warp)                          */
    int32_t size_class;        /* kernel size class                                            */
    int32_t searches;          /* concurrent searches of a depth-first pass                    */
    int32_t reserved;
    uint64_t h2d_bytes;        /* bytes copied host -> device by the run                       */
    uint64_t d2h_bytes;        /* bytes copied device -> host by the run                       */
    uint64_t graph_launches;   /* CUDA graph launches of the depth-first pass loop (run on the
                                  device by a conditional while node; the breadth-first levels'
                                  graph is counted in expand_passes alone)                     */
    double run_ms;             /* host time of the run, from the checked inputs to the results */
    double copy_out_ms;        /* host time of the copy-out: gather on the device, the copy to
                                  the page-locked staging buffer, the copies to host outputs   */
    double host_copy_ms;       /* the part of copy_out_ms spent copying from the staging buffer
                                  to the caller's host buffers                                 */
} wpm_run_stats;

int wpm_last_run_stats(wpm_run_stats *out);

/*
 * The candidate facets of a map (Section 3.1; Proposition 4.2), in lexicographic order,
 * computed on the GPU. lambda_cols: host, m entries. facets_out: host buffer of `cap`
 * entries. Returns M >= 0, or a negative code (WPM_ERR_CAPACITY if cap < M).
 */
int wpm_candidate_facets(const uint32_t *lambda_cols, int kind, int n, int m,
                         uint16_t *facets_out, int cap);

/*
 * Enumerate the WPMs of one map (Section 2.1 problem statement with the facets of
 * Proposition 4.2 and the properties of Section 4.2). Blocks until the result is in
 * `out`. mode: WPM_MODE_LIST or WPM_MODE_COUNT. cond may be NULL.
 */
int wpm_enumerate(const uint32_t *lambda_cols, int kind, int n, int m,
                  const wpm_conditions *cond, wpm_output *out, int mode);

/*
 * Enumerate the WPMs whose facets come from an arbitrary list (Section 2.1, the most
 * general input: a set of facets and properties). facets: host, M vertex masks of
 * popcount n on [m], distinct; they are renumbered in lexicographic order, so masks in
 * `cond` and in the output refer to that order.
 */
int wpm_enumerate_facets(const uint16_t *facets, int M, int n, int m,
                         const wpm_conditions *cond, wpm_output *out, int mode);

/*
 * Enumerate `count` instances in one batched run on the GPU: all candidate sets are
 * built by one launch, the search runs every instance's frontier together, and outputs
 * are sorted per instance. outs[i] receives instance i (its `status` field holds the
 * per-instance code; the return value is the first failure, or WPM_OK; when the run as a
 * whole fails -- a CUDA error, a ring overflow, a bounded device wait that ran out -- every
 * instance's status receives that code and no counts are valid). tuning may be NULL.
 * cuda_stream: a cudaStream_t to run on, or NULL for the library's own stream; the call
 * synchronises that stream before returning.
 */
int wpm_enumerate_batch(const wpm_instance *inst, int count, wpm_output *outs, int mode,
                        const wpm_tuning *tuning, void *cuda_stream);

/*
 * Autotuner of the batched run (the paper has no counterpart). Times a fixed set of
 * candidate tunings (search mode, i.e. one search per thread or per warp; breadth-first
 * frontier size; the hand-over chunk of per-thread searches: levels given and nodes between
 * hand-overs) on a sample of the batch, every k-th instance for about `sample` instances
 * (0: 256), in counting mode, each in two interleaved rounds keeping its best time, and
 * writes the fastest to *best. Counts do not depend on the
 * tuning, so the candidates differ only in time. The choice is also kept, for the rest of
 * the process, under the batch's signature (the smallest and largest n, whether any map is
 * primal, and the number of maps rounded down to a power of two): wpm_enumerate_batch with
 * tuning == NULL on a batch of the same signature uses it. best_ms (optional) receives the
 * winner's time on the sample, in milliseconds. Errors as wpm_enumerate_batch's; instances
 * that fail their own checks are left out.
 */
int wpm_autotune(const wpm_instance *inst, int count, int sample, wpm_tuning *best,
                 double *best_ms, void *cuda_stream);

/*
 * Isomorphism classes (Algorithm 4.4, line 14: one representative per class). Complex c,
 * for c = 0..count-1, has the facets facets[offsets[c] .. offsets[c+1]) (vertex masks on
 * [m], m <= 16; host pointers, offsets has count + 1 entries). Two complexes are in one class
 * when a relabeling of the vertices maps the facets of one onto the facets of the other.
 * class_of[c] receives the class of complex c, classes numbered 0.. in order of first
 * appearance; returns the number of classes, or a negative error code. Computed on the host
 * (several threads): a canonical form per complex, by colour refinement and
 * individualization, with subtrees that a found automorphism maps onto searched ones
 * skipped. Runs without a GPU.
 */
long wpm_iso_classes(int m, int count, const uint64_t *offsets, const uint16_t *facets,
                     int32_t *class_of);

/*
 * PL sphereness (Algorithm 4.4, line 16) by the criterion of Lemma 3.3: a weak
 * pseudo-manifold of Picard number at most 7 is a PL sphere exactly when the link of every
 * face, the empty face included, is a Z2-homology sphere. Complexes as in wpm_iso_classes
 * (every facet an n-subset of [m], m <= 15); is_sphere[c] receives 1 or 0; returns the number
 * of spheres, or a negative error code. Computed on the host (several threads): faces from a
 * bitmap of all vertex subsets, reduced Z2-Betti numbers of every link from GF(2) ranks of its
 * boundary maps. Runs without a GPU.
 */
long wpm_pl_spheres(int n, int m, int count, const uint64_t *offsets, const uint16_t *facets,
                    uint8_t *is_sphere);

/*
 * Link conditions of the n = 11 construction (Section 4.4, "Enumeration for n = 11",
 * conditions (1) and (2) on X). A complex K on [m] whose last vertex a = m - 1 has the link
 * L contains the cone {sigma + a : sigma a facet of L}; K is searched for with
 *   forced_in  = the cone facets sigma + a                              (condition (1)),
 *   forced_out = every other candidate facet of K's map through a      (condition (2)).
 * Inputs (host pointers, read during the call): n (facet size of K) and m (its vertices;
 * K's map is dual, of Picard number m - n); mu_rows[0..m-1): the dual rows of L's map on the
 * vertices 0..m-2 (nonzero, distinct vectors of Z2^(m-n)); apex_row: the dual row of a, or 0
 * for the one nonzero vector that mu does not take (the paper's case m = 15 = 2^4 - 1, where
 * mu fixes K's map); link_facets[0..link_count): L's facets as vertex masks, (n-1)-subsets of
 * [m-1]. Outputs (host, caller-owned): lambda_rows_out[0..m): K's dual map (mu, then the apex
 * row); forced_in and forced_out: `words` uint64 words each, over K's candidate facets in the
 * library's order (words beyond ceil(M/64) are zeroed). Returns M, the candidate facets of
 * K's map (the n_facets to pass in wpm_conditions with the masks), or WPM_ERR_INPUT (sizes,
 * zero or repeated rows, rank < m - n, apex_row 0 with mu missing other than one vector, a
 * link facet of the wrong size, through a, repeated, or whose cone facet is not a candidate,
 * i.e. L does not support mu), WPM_ERR_CAPACITY (words < ceil(M/64); nothing written),
 * WPM_ERR_LIMIT (M > WPM_MAX_FACETS). Computed on the host; runs without a GPU.
 */
int wpm_link_conditions(int n, int m, const uint32_t *mu_rows, uint32_t apex_row,
                        const uint16_t *link_facets, int link_count, uint32_t *lambda_rows_out,
                        uint64_t *forced_in, uint64_t *forced_out, int words);

/*
 * wpm_candidate_facets with no allocation (the paper has no counterpart: this serves callers
 * that must not allocate, e.g. a service that reserved its device memory at start-up, or a
 * host framework whose allocator owns the device). Same inputs and output as
 * wpm_candidate_facets (host pointers), run on `cuda_stream` (NULL: the default stream),
 * which the call synchronises before it returns. Its device scratch is one fixed 512 KiB
 * __device__ array of the library, present on every GPU that loads it; a map needs about
 * 38 C(m,n) + 36 C(m,n-1) bytes of it (n = 6 on 16 vertices fits, n = 7 on 16 does not), and
 * larger maps are rejected with WPM_ERR_LIMIT. The first call on a device looks up that
 * array's address (make it before any stream capture). Calls share the array: calls that
 * overlap on the GPU race.
 */
int wpm_candidate_facets_static(const uint32_t *lambda_cols, int kind, int n, int m,
                                uint16_t *facets_out, int cap, void *cuda_stream);

/* ---- serving engine (continuous batching) ------------------------------------------ */
/*
 * Serving (continuous batching). An engine keeps a device work ring resident and runs search
 * passes over every admitted job together (the per-map calls of Algorithm 4.4, Section 4.2,
 * served as independent requests). A job is admitted, in arrival order, when a
 * job slot is free and its output region (out_capacity masks, list mode) fits in the engine's
 * output memory; jobs submitted while others run join at the next step and share the GPU with
 * them. Results are identical to wpm_enumerate's. One engine is driven from one host thread.
 */
typedef struct wpm_engine wpm_engine;

typedef struct {
    int64_t memory_bytes;   /* device memory for job outputs; 0 = 8 GiB                   */
    int32_t max_jobs;       /* concurrent jobs (slots); 0 = 1024                          */
    int32_t budget;         /* most search nodes per search per step; 0 = 2^20            */
    int32_t max_n;          /* largest n admitted (sets the kernel size class and the
                               search depth, the upper-bound cap of n); 0 = 11             */
    int32_t slice_ms;       /* a step's search pass also ends this many milliseconds after it
                               began (every search parks at that time): it bounds how long a
                               queued job waits for admission, and passes that end together
                               leave no tail; 0 = by load (50 ms while fewer than half the
                               searches parked work at the end of the last pass, else 100 ms),
                               < 0 = the node budget alone                                  */
} wpm_engine_config;

/* Create an engine on the current device; stream may be NULL (the engine's own stream). */
int wpm_engine_create(const wpm_engine_config *cfg, void *cuda_stream, wpm_engine **out);
/* Queue a job (copied; pointers may be freed after the call). mode as above;
 * out_capacity: masks to reserve in list mode. job_id receives a handle. A list-mode job
 * whose output region (2 * 8 * ceil(C(m,n)/64) * out_capacity bytes) exceeds the engine's
 * memory_bytes is refused with WPM_ERR_NOMEM (it could never be admitted). */
int wpm_engine_submit(wpm_engine *e, const wpm_instance *inst, int mode,
                      uint64_t out_capacity, uint64_t *job_id);
/* Admit what fits, run one search pass over everything resident, retire finished jobs.
 * *n_active receives the jobs holding a slot afterwards. */
int wpm_engine_step(wpm_engine *e, int *n_active);
/* Finished jobs since the last poll: fills up to cap ids; returns how many. */
int wpm_engine_poll(wpm_engine *e, uint64_t *job_ids, int cap);
/* Copy a finished job's result into out (list mode: out->masks, a host buffer of
 * out->capacity masks) and forget the job. WPM_ERR_CAPACITY keeps the result for a retry with
 * a larger buffer; a job whose own out_capacity was too small reports WPM_ERR_CAPACITY with
 * its count. */
int wpm_engine_result(wpm_engine *e, uint64_t job_id, wpm_output *out);
void wpm_engine_destroy(wpm_engine *e);

/*
 * Integer throughput of the current GPU, measured (the paper has no counterpart: this is the
 * peak of the roofline that the search kernels, bound by integer and logic instructions, are
 * reported against). op 0: independent chains of lop3 and add instructions (the mix of the
 * search's bitset and counter updates); op 1: popc and xor. One launch of 4 blocks of 512
 * threads per SM, each thread running 8 independent chains for `iters` steps, timed with CUDA
 * events after a warm-up launch. *ops_per_sec receives the instructions per second over all
 * threads (each lop3, add, popc or xor counted once); *ms (optional) the launch's duration.
 * The call allocates a small device buffer and a stream of its own.
 */
int wpm_int_peak(int op, int iters, double *ops_per_sec, double *ms);

/* ---- misc -------------------------------------------------------------------------- */
const char *wpm_last_error(void);
int wpm_version(void);
/* Free the cached device workspace of the calling process. */
void wpm_release_workspace(void);

#ifdef __cplusplus
}
#endif
#endif /* WPM_H */
