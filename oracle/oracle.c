/*
 * oracle.c -- CPU oracle for enumerating weak pseudo-manifolds (Choi, Jang, Vallee,
 * arXiv 2301.00806).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, deliberately unoptimised statement of
 * what the GPU library computes. Only the tests, the smoke check and the bench's CPU
 * baseline may build, load or call it. The GPU library shares no code with it: not its
 * facet or ridge construction, its search, its bit layout or its sorting.
 *
 * What it computes (Section 2.1, Proposition 2.1): given candidate facets F_1..F_M
 * (n-subsets of [m]) and affine properties g, the set of all K subset of F with every
 * coordinate of A K in {0, 2} (A = ridge-facet incidence matrix) and g(K) > 0 for all g.
 *
 * Four independent routes to that set:
 *   orc_enumerate_brute   the definition itself: every one of the 2^M subsets, in Gray
 *                         order, checked by Proposition 2.1. M <= 40.
 *   orc_enumerate_sweep   Section 2.1: every WPM lies in ker_Z2 A; a basis of that kernel
 *                         is swept in Gray order and each combination K = BX is checked
 *                         by Proposition 2.1 over Z.
 *   orc_enumerate_dfs     the ridge-driven search (the canonical tree below), recursive,
 *                         with plain byte arrays. It also reports node and probe counts.
 *   orc_enumerate_sweep_fixed  the sweep with Section 4.4's initialization: forced-in /
 *                         forced-out facets fix part of X through a column echelon form
 *                         of the kernel basis; only the rest is swept.
 *   orc_enumerate_sweep_blocks  the sweep over Section 2.1's convenient basis: the same
 *                         fixed coordinates, then Z blocks over ridges with disjoint parents
 *                         (at most two generators of a block, within Hamming distance 2 of
 *                         the fixed part on its pivot rows), the other generators free.
 *                         orc_convenient_basis reports its shape and |X| (Table 1).
 *   orc_n2_cycle_sets     n = 2 only: a WPM of dimension 1 is a set of vertex-disjoint
 *                         cycles of the candidate graph; counted by graph search.
 *
 * And the post-filters of Algorithm 4.4 (lines 8-12) on an output K: orc_pic_seed (every
 * vertex used, so Pic(K) = 4, and the seedness condition of Proposition 3.1).
 *
 * The canonical tree (the GPU search reproduces it node for node):
 *   root: In = forced-in facets (plus facet {0..n-1} when the base facet is required),
 *         Out = forced-out facets; the root dies if the two meet or a check below fails.
 *   a node is a state (In, Out) that passed its checks. At a node:
 *     - if some ridge has degree 1, take the lowest-index such ridge r. For each parent
 *       p of r that is undecided (not in In, not in Out), in ascending index order, the
 *       child is In + {p}, Out + (the other undecided parents of r).
 *     - otherwise every ridge has degree 0 or 2 and In is a WPM (Proposition 2.1): it is
 *       emitted when every g(In) > 0. Then, for each undecided facet f in ascending order,
 *       the child is In + {f}, Out + (every undecided facet below f).
 *   checks on a child (a rejected child is a "probe", an accepted one a "node"):
 *     - adding the facet raises no ridge to degree 3;
 *     - |In| <= cap (the upper-bound-theorem condition g = f - |K| + 1 > 0, Section 4.2);
 *     - for each general affine g = c0 + sum c_j k_j: c0 + sum_{c_j>0} c_j
 *       + sum_{j in In, c_j<0} c_j > 0 (an upper bound of g over every K containing In).
 *   Node and probe counts are this tree's own quantities. The paper has no counterpart,
 *   so they are "parity unpinned" against the paper; only the output set is pinned.
 *
 * Orders: facets and ridges are listed in lexicographic order of their sorted vertex
 * tuples; output masks have facet j at bit j%64 of word j/64 and are sorted ascending as
 * multiword unsigned integers (the highest word compared first).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INPUT -1
#define ORC_ERR_CAPACITY -2
#define ORC_ERR_NOMEM -5

/* ---------------------------------------------------------------------------------- */
/* GF(2) linear algebra on small vectors.                                             */
/* ---------------------------------------------------------------------------------- */

/* Rank over Z2 of k vectors given as bit masks: Gaussian elimination, one pivot bit at a
 * time (the highest remaining bit of each kept vector). */
static int gf2_rank_small(const uint32_t *v, int k)
{
    uint32_t basis[32];
    int r = 0;
    for (int i = 0; i < k; i++) {
        uint32_t x = v[i];
        /* reduce x by the basis, pivoting on each basis vector's highest bit */
        for (int j = 0; j < r; j++) {
            int hb = 31 - __builtin_clz(basis[j]);
            if ((x >> hb) & 1u) x ^= basis[j];
        }
        if (x) {
            /* keep the basis in a form where every pivot bit appears in one vector only */
            int hb = 31 - __builtin_clz(x);
            for (int j = 0; j < r; j++)
                if ((basis[j] >> hb) & 1u) basis[j] ^= x;
            basis[r++] = x;
        }
    }
    return r;
}

/* ---------------------------------------------------------------------------------- */
/* Candidate facets (Section 3.1 non-singularity; Section 4.2, Proposition 4.2).      */
/* ---------------------------------------------------------------------------------- */

/* Advance c[0..k-1] (strictly increasing, values < m) to the next k-subset in
 * lexicographic order. Returns 0 when the last subset has been passed. */
static int next_combination(int *c, int k, int m)
{
    int i = k - 1;
    while (i >= 0 && c[i] == m - k + i) i--;
    if (i < 0) return 0;
    c[i]++;
    for (int j = i + 1; j < k; j++) c[j] = c[j - 1] + 1;
    return 1;
}

/*
 * The candidate facets of a mod-2 characteristic map, in lexicographic order.
 *  kind 0 (primal): cols[i] is lambda(i) in Z2^n. An n-subset sigma is a candidate when
 *                   {lambda(i) : i in sigma} is linearly independent, i.e. a basis of Z2^n
 *                   (the non-singularity condition, Section 3.1).
 *  kind 1 (dual):   cols[i] is the dual row lambda-bar(i) in Z2^(m-n). By linear Gale
 *                   duality (Proposition 4.2) sigma is a candidate when the rows indexed
 *                   by the complement [m] \ sigma form a basis of Z2^(m-n).
 * Writes vertex masks (bit i = vertex i) to facets[0..]; returns M, or a negative error.
 */
int orc_candidate_facets(int kind, int n, int m, const uint32_t *cols, uint16_t *facets, int cap)
{
    if (n < 1 || m < n || m > 16 || (kind != 0 && kind != 1)) return ORC_ERR_INPUT;
    int c[16];
    for (int i = 0; i < n; i++) c[i] = i;
    int M = 0;
    do {
        uint32_t v[16];
        int k = 0, need;
        int in_sigma[16] = {0};
        for (int i = 0; i < n; i++) in_sigma[c[i]] = 1;
        if (kind == 0) {
            for (int i = 0; i < n; i++) v[k++] = cols[c[i]];
            need = n;
        } else {
            for (int i = 0; i < m; i++)
                if (!in_sigma[i]) v[k++] = cols[i];
            need = m - n;
        }
        if (gf2_rank_small(v, k) == need) {
            if (M >= cap) return ORC_ERR_CAPACITY;
            uint16_t mask = 0;
            for (int i = 0; i < n; i++) mask |= (uint16_t)(1u << c[i]);
            facets[M++] = mask;
        }
    } while (next_combination(c, n, m));
    return M;
}

/* ---------------------------------------------------------------------------------- */
/* Ridges and the ridge-facet incidence (Section 2.1).                                */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    int n, M, N;
    uint16_t *ridge;   /* [N] vertex masks, lexicographic order                         */
    int *npar;         /* [N] number of parents P(r)                                     */
    int *par;          /* [N * M] parents of r, ascending (row r holds npar[r] entries)  */
    int *fr;           /* [M * n] the n ridges of each facet, by ridge index              */
} incidence_t;

static void incidence_free(incidence_t *I)
{
    free(I->ridge); free(I->npar); free(I->par); free(I->fr);
    memset(I, 0, sizeof(*I));
}

/* The ridges are every (n-1)-subset of [m] that lies in at least one candidate facet,
 * found by walking all (n-1)-subsets in lexicographic order and testing containment
 * against every facet. The parents of r are the facets that contain it. */
static int incidence_build(int n, int M, const uint16_t *facets, incidence_t *I)
{
    memset(I, 0, sizeof(*I));
    I->n = n; I->M = M;
    if (n < 2 || M < 0) return ORC_ERR_INPUT;
    uint16_t all = 0;
    for (int j = 0; j < M; j++) all |= facets[j];
    int m = 0;
    while (m < 16 && (all >> m)) m++;
    if (m < n) m = n;
    /* upper bound on the number of ridges: C(m, n-1) */
    long cap = 1;
    for (int i = 0; i < n - 1; i++) cap = cap * (m - i) / (i + 1);
    I->ridge = (uint16_t *)malloc(sizeof(uint16_t) * (cap ? cap : 1));
    I->npar = (int *)calloc(cap ? cap : 1, sizeof(int));
    I->par = (int *)malloc(sizeof(int) * (size_t)(cap ? cap : 1) * (M ? M : 1));
    I->fr = (int *)malloc(sizeof(int) * (size_t)(M ? M : 1) * n);
    if (!I->ridge || !I->npar || !I->par || !I->fr) { incidence_free(I); return ORC_ERR_NOMEM; }
    int c[16];
    for (int i = 0; i < n - 1; i++) c[i] = i;
    int N = 0;
    do {
        uint16_t r = 0;
        for (int i = 0; i < n - 1; i++) r |= (uint16_t)(1u << c[i]);
        int np = 0;
        for (int j = 0; j < M; j++)
            if ((facets[j] & r) == r) I->par[(size_t)N * M + np++] = j;
        if (np > 0) {
            I->ridge[N] = r;
            I->npar[N] = np;
            N++;
        }
    } while (n - 1 > 0 && next_combination(c, n - 1, m));
    I->N = N;
    for (int j = 0; j < M; j++) {
        int k = 0;
        for (int r = 0; r < N; r++)
            if ((facets[j] & I->ridge[r]) == I->ridge[r]) I->fr[j * n + k++] = r;
        if (k != n) { incidence_free(I); return ORC_ERR_INPUT; } /* facet of wrong size */
    }
    return ORC_OK;
}

/* Ridges (vertex masks, lexicographic order) and parent counts, for tests. */
int orc_ridges(int n, int M, const uint16_t *facets, uint16_t *ridges, int32_t *npar, int cap)
{
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    int N = I.N;
    if (N > cap) { incidence_free(&I); return ORC_ERR_CAPACITY; }
    for (int r = 0; r < N; r++) { ridges[r] = I.ridge[r]; npar[r] = I.npar[r]; }
    incidence_free(&I);
    return N;
}

/* dim ker_Z2 A = M - rank_Z2(A), A the N x M ridge-facet incidence matrix (Section 2.1).
 * Rank by Gaussian elimination over the rows of A stored as M-bit rows. */
static int gf2_kernel_basis(const incidence_t *I, uint64_t **basis_out, int *s_out)
{
    int M = I->M, N = I->N;
    int W = (M + 63) / 64;
    uint64_t *rows = (uint64_t *)calloc((size_t)(N ? N : 1) * W, sizeof(uint64_t));
    int *pivcol = (int *)malloc(sizeof(int) * (N ? N : 1));
    char *is_pivot = (char *)calloc(M ? M : 1, 1);
    if (!rows || !pivcol || !is_pivot) { free(rows); free(pivcol); free(is_pivot); return ORC_ERR_NOMEM; }
    for (int r = 0; r < N; r++)
        for (int k = 0; k < I->npar[r]; k++) {
            int j = I->par[(size_t)r * M + k];
            rows[(size_t)r * W + j / 64] |= 1ull << (j % 64);
        }
    /* reduced row echelon form */
    int rank = 0;
    for (int col = 0; col < M && rank < N; col++) {
        int sel = -1;
        for (int r = rank; r < N; r++)
            if ((rows[(size_t)r * W + col / 64] >> (col % 64)) & 1ull) { sel = r; break; }
        if (sel < 0) continue;
        if (sel != rank)
            for (int w = 0; w < W; w++) {
                uint64_t t = rows[(size_t)sel * W + w];
                rows[(size_t)sel * W + w] = rows[(size_t)rank * W + w];
                rows[(size_t)rank * W + w] = t;
            }
        for (int r = 0; r < N; r++)
            if (r != rank && ((rows[(size_t)r * W + col / 64] >> (col % 64)) & 1ull))
                for (int w = 0; w < W; w++) rows[(size_t)r * W + w] ^= rows[(size_t)rank * W + w];
        pivcol[rank] = col;
        is_pivot[col] = 1;
        rank++;
    }
    int s = M - rank;
    if (basis_out) {
        /* one kernel vector per free column f: x_f = 1, x_pivot(r) = row r's bit at f */
        uint64_t *B = (uint64_t *)calloc((size_t)(s ? s : 1) * W, sizeof(uint64_t));
        if (!B) { free(rows); free(pivcol); free(is_pivot); return ORC_ERR_NOMEM; }
        int t = 0;
        for (int f = 0; f < M; f++) {
            if (is_pivot[f]) continue;
            B[(size_t)t * W + f / 64] |= 1ull << (f % 64);
            for (int r = 0; r < rank; r++)
                if ((rows[(size_t)r * W + f / 64] >> (f % 64)) & 1ull)
                    B[(size_t)t * W + pivcol[r] / 64] |= 1ull << (pivcol[r] % 64);
            t++;
        }
        *basis_out = B;
    }
    free(rows); free(pivcol); free(is_pivot);
    *s_out = s;
    return ORC_OK;
}

int orc_kernel_dim(int n, int M, const uint16_t *facets)
{
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    int s = 0;
    rc = gf2_kernel_basis(&I, NULL, &s);
    incidence_free(&I);
    return rc ? rc : s;
}

/* ---------------------------------------------------------------------------------- */
/* Conditions (Section 2.1 properties; Section 4.2 upper bound; Section 4.4 forced).  */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    int32_t cap;                /* |K| <= cap; -1: none; -2: the Section 4.2 bound for n */
    int32_t base_facet;         /* nonzero: facet {0..n-1} must be in K (Section 3.1)     */
    const uint64_t *forced_in;  /* NULL or ceil(M/64) words: facets that must be in K     */
    const uint64_t *forced_out; /* NULL or ceil(M/64) words: facets that must not be in K */
    int32_t n_affine;           /* general properties g(K) = c0 + sum_j c_j k_j > 0      */
    const int32_t *c0;          /* [n_affine]                                             */
    const int32_t *coef;        /* [n_affine * M]                                         */
} orc_cond;

typedef struct {
    uint64_t count, nodes, probes;
} orc_stats;

static long binom(int a, int b)
{
    if (b < 0 || a < b) return 0;
    long r = 1;
    for (int i = 0; i < b; i++) r = r * (a - i) / (i + 1);
    return r;
}

/* f_{n-1}(C^n(n+4)) = C(n+4-ceil(n/2), 4) + C(n+3-floor(n/2), 4)  (Section 4.2). */
int orc_ubt_cap(int n)
{
    return (int)(binom(n + 4 - (n + 1) / 2, 4) + binom(n + 3 - n / 2, 4));
}

/* Resolve the cap: -2 means the Section 4.2 bound, which is stated for m = n + 4. */
static int resolve_cap(int cap, int n, int m)
{
    if (cap == -2) return (m == n + 4) ? orc_ubt_cap(n) : -3;
    return cap;
}

/* The base facet {0..n-1} as a candidate index, or -1 when it is not a candidate. */
static int base_facet_index(int n, int M, const uint16_t *facets)
{
    uint16_t b = (uint16_t)((1u << n) - 1u);
    for (int j = 0; j < M; j++)
        if (facets[j] == b) return j;
    return -1;
}

static int bit_of(const uint64_t *w, int j) { return (int)((w[j / 64] >> (j % 64)) & 1ull); }

/* Every g(K) > 0 for K given as a 0/1 array, computed from the definition. */
static int affine_ok(const orc_cond *c, int M, const char *inK)
{
    for (int a = 0; a < c->n_affine; a++) {
        long g = c->c0[a];
        for (int j = 0; j < M; j++)
            if (inK[j]) g += c->coef[(size_t)a * M + j];
        if (g <= 0) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------------------------------- */
/* Output collection.                                                                 */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    uint64_t *masks;   /* caller buffer, cap * W words, or NULL for counting only */
    uint64_t cap;
    uint64_t count;
    int W;
    int overflow;
} sink_t;

static void sink_emit(sink_t *s, int M, const char *inK)
{
    if (s->masks) {
        if (s->count < s->cap) {
            uint64_t *dst = s->masks + s->count * (uint64_t)s->W;
            memset(dst, 0, sizeof(uint64_t) * s->W);
            for (int j = 0; j < M; j++)
                if (inK[j]) dst[j / 64] |= 1ull << (j % 64);
        } else {
            s->overflow = 1;
        }
    }
    s->count++;
}

static int g_sort_W;
static int cmp_masks(const void *pa, const void *pb)
{
    const uint64_t *a = (const uint64_t *)pa, *b = (const uint64_t *)pb;
    for (int w = g_sort_W - 1; w >= 0; w--) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

static int sink_finish(sink_t *s)
{
    if (s->masks && !s->overflow) {
        g_sort_W = s->W;
        qsort(s->masks, s->count, sizeof(uint64_t) * s->W, cmp_masks);
    }
    return s->overflow ? ORC_ERR_CAPACITY : ORC_OK;
}

/* ---------------------------------------------------------------------------------- */
/* O3: the definition. Every subset K of the M candidates, visited in Gray-code order */
/* (one facet toggled per step), keeping the ridge degrees of A K up to date.         */
/* ---------------------------------------------------------------------------------- */

int orc_enumerate_brute(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                        uint64_t *masks, uint64_t cap_masks, orc_stats *st)
{
    if (M > 40) return ORC_ERR_INPUT;
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    int base = c->base_facet ? base_facet_index(n, M, facets) : -1;
    sink_t s = { masks, cap_masks, 0, (M + 63) / 64, 0 };
    int *deg = (int *)calloc(I.N ? I.N : 1, sizeof(int));
    char *inK = (char *)calloc(M ? M : 1, 1);
    int bad = 0;     /* ridges whose degree is not 0 or 2 */
    int size = 0;
    int fin_need = 0, fin_have = 0, fout_have = 0;
    for (int j = 0; j < M; j++) {
        int fi = (c->forced_in && bit_of(c->forced_in, j)) || j == base;
        fin_need += fi;
    }
    if (c->base_facet && base < 0) fin_need = -1; /* never satisfiable */
    uint64_t total = (M == 64) ? 0 : (1ull << M);
    for (uint64_t i = 0;; i++) {
        if (i > 0) {
            if (i == total) break;
            int j = __builtin_ctzll(i);
            int delta = inK[j] ? -1 : 1;
            inK[j] = (char)!inK[j];
            size += delta;
            if ((c->forced_in && bit_of(c->forced_in, j)) || j == base) fin_have += delta;
            if (c->forced_out && bit_of(c->forced_out, j)) fout_have += delta;
            for (int k = 0; k < n; k++) {
                int r = I.fr[j * n + k];
                int before_ok = (deg[r] == 0 || deg[r] == 2);
                deg[r] += delta;
                int after_ok = (deg[r] == 0 || deg[r] == 2);
                bad += before_ok - after_ok;
            }
        }
        if (bad == 0 && fin_have == fin_need && fout_have == 0 && (cap < 0 || size <= cap) &&
            affine_ok(c, M, inK))
            sink_emit(&s, M, inK);
    }
    free(deg); free(inK);
    incidence_free(&I);
    rc = sink_finish(&s);
    if (st) { st->count = s.count; st->nodes = 0; st->probes = 0; }
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* O2: Section 2.1. Sweep all 2^s elements K = BX of ker_Z2 A (Gray order over X) and */
/* keep those whose degrees A K over Z are all in {0, 2} (Proposition 2.1).           */
/* ---------------------------------------------------------------------------------- */

int orc_enumerate_sweep(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                        uint64_t *masks, uint64_t cap_masks, orc_stats *st, int max_s)
{
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    uint64_t *B = NULL;
    int s = 0;
    rc = gf2_kernel_basis(&I, &B, &s);
    if (rc) { incidence_free(&I); return rc; }
    if (s > max_s || s > 62) { free(B); incidence_free(&I); return ORC_ERR_INPUT; }
    int W = (M + 63) / 64;
    int base = c->base_facet ? base_facet_index(n, M, facets) : -1;
    sink_t snk = { masks, cap_masks, 0, W, 0 };
    int *deg = (int *)calloc(I.N ? I.N : 1, sizeof(int));
    char *inK = (char *)calloc(M ? M : 1, 1);
    int bad = 0;   /* ridges of degree not in {0, 2}: in the kernel, the degree-4 ones */
    int size = 0;
    for (uint64_t i = 0; i < (1ull << s); i++) {
        if (i > 0) {
            int t = __builtin_ctzll(i);
            for (int j = 0; j < M; j++) {
                if (!((B[(size_t)t * W + j / 64] >> (j % 64)) & 1ull)) continue;
                int delta = inK[j] ? -1 : 1;
                inK[j] = (char)!inK[j];
                size += delta;
                for (int k = 0; k < n; k++) {
                    int r = I.fr[j * n + k];
                    int before_ok = (deg[r] == 0 || deg[r] == 2);
                    deg[r] += delta;
                    int after_ok = (deg[r] == 0 || deg[r] == 2);
                    bad += before_ok - after_ok;
                }
            }
        }
        if (bad) continue;
        if (cap >= 0 && size > cap) continue;
        if (c->base_facet && (base < 0 || !inK[base])) continue;
        int ok = 1;
        for (int j = 0; j < M && ok; j++) {
            if (c->forced_in && bit_of(c->forced_in, j) && !inK[j]) ok = 0;
            if (c->forced_out && bit_of(c->forced_out, j) && inK[j]) ok = 0;
        }
        if (ok && affine_ok(c, M, inK)) sink_emit(&snk, M, inK);
    }
    free(deg); free(inK); free(B);
    incidence_free(&I);
    rc = sink_finish(&snk);
    if (st) { st->count = snk.count; st->nodes = 0; st->probes = 0; }
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* O2 with Section 4.4's initialization (Enumeration for n = 11, condition (X)). The   */
/* forced-in facets I and forced-out facets J fix part of X before the sweep: the      */
/* generators (the columns of B, here the kernel basis vectors) are brought to reduced */
/* column echelon form with the rows taken in the order I, J, the rest. The columns    */
/* whose leading row lies in I must have x_t = 1, those whose leading row lies in J    */
/* x_t = 0, and the other columns are zero on every row of I and J, so only they are   */
/* swept. If the fixed part already gives a row of I the value 0 or a row of J the     */
/* value 1, no K satisfies the conditions. nodes reports the combinations swept.       */
/* ---------------------------------------------------------------------------------- */

int orc_enumerate_sweep_fixed(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                              uint64_t *masks, uint64_t cap_masks, orc_stats *st, int max_free)
{
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    uint64_t *B = NULL;
    int s = 0;
    rc = gf2_kernel_basis(&I, &B, &s);
    if (rc) { incidence_free(&I); return rc; }
    int W = (M + 63) / 64;
    /* the row order: I, then J, then the rest */
    int *order = (int *)malloc(sizeof(int) * (M ? M : 1));
    int n_i = 0, n_j = 0, k = 0;
    for (int pass = 0; pass < 3; pass++)
        for (int j = 0; j < M; j++) {
            int in_i = c->forced_in && bit_of(c->forced_in, j);
            int in_j = !in_i && c->forced_out && bit_of(c->forced_out, j);
            int want = pass == 0 ? in_i : pass == 1 ? in_j : (!in_i && !in_j);
            if (!want) continue;
            order[k++] = j;
            n_i += pass == 0;
            n_j += pass == 1;
        }
    /* reduced column echelon form: one leading row per pivot column, in row order */
    int *lead = (int *)malloc(sizeof(int) * (s ? s : 1));
    int piv = 0;
    for (int q = 0; q < M && piv < s; q++) {
        int j = order[q];
        int t = -1;
        for (int u = piv; u < s; u++)
            if (bit_of(B + (size_t)u * W, j)) { t = u; break; }
        if (t < 0) continue;
        if (t != piv)
            for (int w = 0; w < W; w++) {
                uint64_t x = B[(size_t)t * W + w];
                B[(size_t)t * W + w] = B[(size_t)piv * W + w];
                B[(size_t)piv * W + w] = x;
            }
        for (int u = 0; u < s; u++)
            if (u != piv && bit_of(B + (size_t)u * W, j))
                for (int w = 0; w < W; w++) B[(size_t)u * W + w] ^= B[(size_t)piv * W + w];
        lead[piv++] = q;
    }
    int s_i = 0, s_j = 0;   /* pivot columns led by rows of I, and by rows of I or J */
    for (int t = 0; t < piv; t++) {
        if (lead[t] < n_i) s_i++;
        if (lead[t] < n_i + n_j) s_j++;
    }
    int n_free = s - s_j;
    if (n_free > max_free || n_free > 62) {
        free(order); free(lead); free(B); incidence_free(&I);
        return ORC_ERR_INPUT;
    }
    /* X fixed on its first s_J entries: x_t = 1 for t < s_I, 0 for s_I <= t < s_J */
    char *inK = (char *)calloc(M ? M : 1, 1);
    for (int t = 0; t < s_i; t++)
        for (int j = 0; j < M; j++)
            if (bit_of(B + (size_t)t * W, j)) inK[j] = (char)!inK[j];
    int feasible = 1;
    for (int q = 0; q < n_i + n_j; q++)
        if (inK[order[q]] != (q < n_i)) feasible = 0;
    int base = c->base_facet ? base_facet_index(n, M, facets) : -1;
    sink_t snk = { masks, cap_masks, 0, W, 0 };
    uint64_t swept = 0;
    if (feasible) {
        int *deg = (int *)calloc(I.N ? I.N : 1, sizeof(int));
        int bad = 0, size = 0;
        for (int j = 0; j < M; j++) {
            if (!inK[j]) continue;
            size++;
            for (int kk = 0; kk < n; kk++) deg[I.fr[j * n + kk]]++;
        }
        for (int r = 0; r < I.N; r++) bad += !(deg[r] == 0 || deg[r] == 2);
        for (uint64_t i = 0; i < (1ull << n_free); i++) {
            if (i > 0) {   /* Gray order over the free columns s_J .. s-1 */
                int t = s_j + __builtin_ctzll(i);
                for (int j = 0; j < M; j++) {
                    if (!bit_of(B + (size_t)t * W, j)) continue;
                    int delta = inK[j] ? -1 : 1;
                    inK[j] = (char)!inK[j];
                    size += delta;
                    for (int kk = 0; kk < n; kk++) {
                        int r = I.fr[j * n + kk];
                        int before_ok = (deg[r] == 0 || deg[r] == 2);
                        deg[r] += delta;
                        int after_ok = (deg[r] == 0 || deg[r] == 2);
                        bad += before_ok - after_ok;
                    }
                }
            }
            swept++;
            if (bad) continue;
            if (cap >= 0 && size > cap) continue;
            if (c->base_facet && (base < 0 || !inK[base])) continue;
            if (affine_ok(c, M, inK)) sink_emit(&snk, M, inK);
        }
        free(deg);
    }
    free(inK); free(order); free(lead); free(B);
    incidence_free(&I);
    rc = sink_finish(&snk);
    if (st) { st->count = snk.count; st->nodes = swept; st->probes = (uint64_t)n_free; }
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* O2 with Section 2.1's convenient basis (the Z blocks and the partition I_1..I_l).   */
/*                                                                                    */
/* Step 1, the generators: a basis of ker_Z2 A, as for the plain sweep.                 */
/* Step 2, the fixed coordinates (Section 4.4's initialization): the rows of facets     */
/*   that must be in K (forced in, and the base facet when it is required) come first,  */
/*   then the rows of facets that must not be in K, then the rest; the generators are    */
/*   brought to reduced column echelon form in that row order. A generator led by a     */
/*   forced-in row has x = 1, one led by a forced-out row x = 0; their sum F is a fixed */
/*   part of every K, and the other generators are zero on all forced rows.              */
/* Step 3, the blocks: repeatedly choose a ridge r whose parents P(r) meet the parents  */
/*   of no ridge chosen before, the one where the unblocked free generators restricted  */
/*   to the rows P(r) have the largest rank k (the lowest ridge index on ties), while    */
/*   k >= 2. Column elimination on those rows makes k of them the identity on k pivot    */
/*   rows of P(r) and the others zero on all of P(r); the pivot rows are then cleared in */
/*   the earlier blocks' generators by adding the new ones (which are zero on every      */
/*   earlier P(r), so the earlier blocks keep their form). The k generators form a part */
/*   I_l of the partition; every other free generator is a part of its own.             */
/* Step 4, the sets X_l: on a pivot row q of block l, K_q = F_q + x_q, since every other */
/*   generator is zero there. So K has |S delta c_l| facets among those rows, S the      */
/*   chosen generators of block l and c_l the pivot rows where F is 1, and a WPM needs   */
/*   at most 2 (the ridge r^l has degree at most 2): X_l ranges over the S within        */
/*   Hamming distance 2 of c_l, 1 + k + C(k, 2) choices instead of 2^k (with F = 0 these */
/*   are the combinations of at most two generators of the block, as in the paper). A    */
/*   single free generator takes both values.                                           */
/* Every K = F + B X with X in X_1 x ... x X_l is formed and checked by Proposition 2.1  */
/* and the properties. nodes reports the combinations visited, |X| = their product.     */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    int s, W, M;
    uint64_t *B;       /* [s * W] generators                                            */
    int s_i, s_j;      /* generators fixed to 1: [0, s_i); fixed to 0: [s_i, s_j)       */
    int feasible;      /* the fixed part satisfies every forced row                    */
    uint64_t *F;       /* [W] the fixed part of K                                       */
    int n_blocks;
    int *blk_start;    /* [n_blocks + 1] into blk_col / blk_row                          */
    int *blk_col;      /* generators of the blocks, block by block                       */
    int *blk_row;      /* the pivot row (facet) of each block generator                  */
    int *blk_ridge;    /* [n_blocks] the chosen ridge                                     */
    int n_single;
    int *single;       /* free generators outside every block                            */
} convenient_t;

static void convenient_free(convenient_t *C)
{
    free(C->B); free(C->F); free(C->blk_start); free(C->blk_col); free(C->blk_row);
    free(C->blk_ridge); free(C->single);
    memset(C, 0, sizeof(*C));
}

static void xor_col(uint64_t *dst, const uint64_t *src, int W)
{
    for (int w = 0; w < W; w++) dst[w] ^= src[w];
}

static int convenient_build(const incidence_t *I, int n, const uint16_t *facets,
                            const orc_cond *c, convenient_t *C)
{
    memset(C, 0, sizeof(*C));
    int M = I->M, N = I->N, W = (M + 63) / 64;
    C->M = M;
    C->W = W;
    int rc = gf2_kernel_basis(I, &C->B, &C->s);
    if (rc) return rc;
    int s = C->s;
    uint64_t *B = C->B;
    int base = c->base_facet ? base_facet_index(n, M, facets) : -1;
    /* step 2: the row order I, J, rest */
    char *kind = (char *)calloc(M ? M : 1, 1);   /* 1 forced in, 2 forced out, 3 both */
    for (int j = 0; j < M; j++) {
        if ((c->forced_in && bit_of(c->forced_in, j)) || j == base) kind[j] |= 1;
        if (c->forced_out && bit_of(c->forced_out, j)) kind[j] |= 2;
    }
    C->feasible = !(c->base_facet && base < 0);
    for (int j = 0; j < M; j++)
        if (kind[j] == 3) C->feasible = 0;
    int *order = (int *)malloc(sizeof(int) * (M ? M : 1));
    int n_i = 0, n_j = 0, q = 0;
    for (int pass = 1; pass <= 3; pass++)
        for (int j = 0; j < M; j++) {
            int k = kind[j] == 3 ? 1 : kind[j];
            if ((pass < 3 && k == pass) || (pass == 3 && k == 0)) {
                order[q++] = j;
                n_i += pass == 1;
                n_j += pass == 2;
            }
        }
    int piv = 0;
    int *lead = (int *)malloc(sizeof(int) * (s ? s : 1));
    for (int qq = 0; qq < n_i + n_j && piv < s; qq++) {
        int j = order[qq];
        int t = -1;
        for (int u = piv; u < s; u++)
            if (bit_of(B + (size_t)u * W, j)) { t = u; break; }
        if (t < 0) continue;
        if (t != piv)
            for (int w = 0; w < W; w++) {
                uint64_t x = B[(size_t)t * W + w];
                B[(size_t)t * W + w] = B[(size_t)piv * W + w];
                B[(size_t)piv * W + w] = x;
            }
        for (int u = 0; u < s; u++)
            if (u != piv && bit_of(B + (size_t)u * W, j)) xor_col(B + (size_t)u * W, B + (size_t)piv * W, W);
        lead[piv++] = qq;
    }
    C->s_i = C->s_j = 0;
    for (int t = 0; t < piv; t++) {
        if (lead[t] < n_i) C->s_i++;
        C->s_j++;
    }
    C->F = (uint64_t *)calloc(W, sizeof(uint64_t));
    for (int t = 0; t < C->s_i; t++) xor_col(C->F, B + (size_t)t * W, W);
    for (int qq = 0; qq < n_i + n_j; qq++)
        if (bit_of(C->F, order[qq]) != (qq < n_i)) C->feasible = 0;
    /* step 3: blocks among the free generators [s_j, s) */
    int n_free = s - C->s_j;
    int *unb = (int *)malloc(sizeof(int) * (n_free ? n_free : 1));   /* unblocked free */
    int n_unb = 0;
    for (int t = C->s_j; t < s; t++) unb[n_unb++] = t;
    char *used = (char *)calloc(M ? M : 1, 1);      /* parents of the chosen ridges       */
    C->blk_start = (int *)calloc((size_t)n_free + 2, sizeof(int));
    C->blk_col = (int *)malloc(sizeof(int) * (n_free ? n_free : 1));
    C->blk_row = (int *)malloc(sizeof(int) * (n_free ? n_free : 1));
    C->blk_ridge = (int *)malloc(sizeof(int) * (n_free ? n_free : 1));
    int n_bc = 0;
    for (;;) {
        int best = -1, best_k = 1;
        for (int r = 0; r < N; r++) {
            int np = I->npar[r], clash = 0;
            const int *P = I->par + (size_t)r * M;
            for (int a = 0; a < np; a++) clash |= used[P[a]];
            if (clash || np - 1 <= best_k) continue;   /* the rank is at most np - 1 */
            /* rank of the unblocked generators restricted to the rows P(r): each one, as an
               np-bit vector, is reduced by the independent ones kept so far */
            uint32_t kept[32];
            int k = 0;
            for (int u = 0; u < n_unb && k < np; u++) {
                uint32_t x = 0;
                for (int a = 0; a < np; a++) x |= (uint32_t)bit_of(B + (size_t)unb[u] * W, P[a]) << a;
                for (int e = 0; e < k; e++)
                    if (x & (kept[e] & (~kept[e] + 1u))) x ^= kept[e];
                if (x) {
                    for (int e = 0; e < k; e++)   /* keep every lowest bit owned by one vector */
                        if (kept[e] & (x & (~x + 1u))) kept[e] ^= x;
                    kept[k++] = x;
                }
            }
            if (k > best_k) { best_k = k; best = r; }
        }
        if (best < 0) break;
        int np = I->npar[best];
        const int *P = I->par + (size_t)best * M;
        int b0 = n_bc;
        for (int a = 0; a < np; a++) {
            int row = P[a];
            int pick = -1;
            for (int u = 0; u < n_unb; u++)
                if (bit_of(B + (size_t)unb[u] * W, row)) { pick = u; break; }
            if (pick < 0) continue;
            int t = unb[pick];
            unb[pick] = unb[--n_unb];
            /* clear this row in every other free generator: the unblocked ones, this block's
               and the earlier blocks' */
            for (int u = 0; u < n_unb; u++)
                if (bit_of(B + (size_t)unb[u] * W, row)) xor_col(B + (size_t)unb[u] * W, B + (size_t)t * W, W);
            for (int e = 0; e < n_bc; e++)
                if (bit_of(B + (size_t)C->blk_col[e] * W, row))
                    xor_col(B + (size_t)C->blk_col[e] * W, B + (size_t)t * W, W);
            C->blk_col[n_bc] = t;
            C->blk_row[n_bc] = row;
            n_bc++;
        }
        for (int a = 0; a < np; a++) used[P[a]] = 1;
        C->blk_ridge[C->n_blocks] = best;
        C->blk_start[C->n_blocks] = b0;
        C->n_blocks++;
        C->blk_start[C->n_blocks] = n_bc;
    }
    C->n_single = n_unb;
    C->single = unb;
    free(kind); free(order); free(lead); free(used);
    return ORC_OK;
}

/* Block sizes of the convenient basis and the size of X (Section 2.1; Table 1's |X|
 * rows). info receives: s, the generators fixed to 1, fixed to 0, feasible, the number of
 * blocks l, the single generators, then l block sizes. Returns the number of entries, or a
 * negative error code. *log2_x receives log2 |X| = sum log2(1 + k + C(k, 2)) + singles. */
int orc_convenient_basis(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                         int32_t *info, int info_cap, double *log2_x)
{
    (void)m;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    convenient_t C;
    rc = convenient_build(&I, n, facets, c, &C);
    if (rc) { incidence_free(&I); return rc; }
    int need = 6 + C.n_blocks;
    if (need > info_cap) { convenient_free(&C); incidence_free(&I); return ORC_ERR_CAPACITY; }
    info[0] = C.s; info[1] = C.s_i; info[2] = C.s_j - C.s_i; info[3] = C.feasible;
    info[4] = C.n_blocks; info[5] = C.n_single;
    double lx = C.n_single;
    for (int b = 0; b < C.n_blocks; b++) {
        int k = C.blk_start[b + 1] - C.blk_start[b];
        info[6 + b] = k;
        lx += log2(1.0 + k + k * (k - 1) / 2.0);
    }
    if (log2_x) *log2_x = lx;
    convenient_free(&C);
    incidence_free(&I);
    return need;
}

typedef struct {
    const incidence_t *I;
    const convenient_t *C;
    const orc_cond *c;
    int n, cap;
    uint64_t *K;        /* [W] the combination being formed */
    int *deg;
    char *inK;
    sink_t *snk;
    uint64_t visited;
} blocks_walk_t;

/* The leaf: K = F + the chosen generators, checked from the definition. */
static void blocks_leaf(blocks_walk_t *b)
{
    const incidence_t *I = b->I;
    int M = I->M, n = b->n;
    b->visited++;
    memset(b->deg, 0, sizeof(int) * (I->N ? I->N : 1));
    int size = 0;
    for (int j = 0; j < M; j++) {
        b->inK[j] = (char)bit_of(b->K, j);
        if (!b->inK[j]) continue;
        size++;
        for (int k = 0; k < n; k++) b->deg[I->fr[j * n + k]]++;
    }
    for (int r = 0; r < I->N; r++)
        if (b->deg[r] != 0 && b->deg[r] != 2) return;
    if (b->cap >= 0 && size > b->cap) return;
    const orc_cond *c = b->c;
    for (int j = 0; j < M; j++) {
        if (c->forced_in && bit_of(c->forced_in, j) && !b->inK[j]) return;
        if (c->forced_out && bit_of(c->forced_out, j) && b->inK[j]) return;
    }
    if (affine_ok(c, M, b->inK)) sink_emit(b->snk, M, b->inK);
}

static void blocks_singles(blocks_walk_t *b, int i)
{
    const convenient_t *C = b->C;
    if (i == C->n_single) { blocks_leaf(b); return; }
    const uint64_t *g = C->B + (size_t)C->single[i] * C->W;
    blocks_singles(b, i + 1);           /* x = 0 */
    xor_col(b->K, g, C->W);
    blocks_singles(b, i + 1);           /* x = 1 */
    xor_col(b->K, g, C->W);
}

/* Block l: every subset S of its generators within Hamming distance 2 of c_l. */
static void blocks_block(blocks_walk_t *b, int l)
{
    const convenient_t *C = b->C;
    if (l == C->n_blocks) { blocks_singles(b, 0); return; }
    int b0 = C->blk_start[l], k = C->blk_start[l + 1] - b0;
    uint32_t cl = 0;
    for (int e = 0; e < k; e++) cl |= (uint32_t)bit_of(C->F, C->blk_row[b0 + e]) << e;
    for (uint32_t S = 0; S < (1u << k); S++) {
        if (__builtin_popcount(S ^ cl) > 2) continue;
        for (int e = 0; e < k; e++)
            if ((S >> e) & 1u) xor_col(b->K, C->B + (size_t)C->blk_col[b0 + e] * C->W, C->W);
        blocks_block(b, l + 1);
        for (int e = 0; e < k; e++)
            if ((S >> e) & 1u) xor_col(b->K, C->B + (size_t)C->blk_col[b0 + e] * C->W, C->W);
    }
}

int orc_enumerate_sweep_blocks(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                               uint64_t *masks, uint64_t cap_masks, orc_stats *st,
                               double max_log2_x)
{
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    convenient_t C;
    rc = convenient_build(&I, n, facets, c, &C);
    if (rc) { incidence_free(&I); return rc; }
    double lx = C.n_single;
    for (int l = 0; l < C.n_blocks; l++) {
        int k = C.blk_start[l + 1] - C.blk_start[l];
        lx += log2(1.0 + k + k * (k - 1) / 2.0);
    }
    if (lx > max_log2_x) { convenient_free(&C); incidence_free(&I); return ORC_ERR_INPUT; }
    int W = C.W;
    sink_t snk = { masks, cap_masks, 0, W, 0 };
    blocks_walk_t b;
    memset(&b, 0, sizeof(b));
    b.I = &I; b.C = &C; b.c = c; b.n = n; b.cap = cap; b.snk = &snk;
    b.K = (uint64_t *)calloc(W, sizeof(uint64_t));
    b.deg = (int *)calloc(I.N ? I.N : 1, sizeof(int));
    b.inK = (char *)calloc(M ? M : 1, 1);
    if (C.feasible) {
        memcpy(b.K, C.F, sizeof(uint64_t) * W);
        blocks_block(&b, 0);
    }
    free(b.K); free(b.deg); free(b.inK);
    convenient_free(&C);
    incidence_free(&I);
    rc = sink_finish(&snk);
    if (st) { st->count = snk.count; st->nodes = b.visited; st->probes = 0; }
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* O1: the ridge-driven search, the canonical tree described at the top of the file.  */
/* ---------------------------------------------------------------------------------- */

enum { UNDECIDED = 0, IN = 1, OUT = 2 };

typedef struct {
    const incidence_t *I;
    const orc_cond *c;
    int cap;
    long *posall;          /* [n_affine]: sum of the positive coefficients            */
    long *negin;           /* [n_affine]: sum of the negative coefficients over In    */
    unsigned char *deg;    /* [N] ridge degrees (A K)_r                               */
    char *st;              /* [M] UNDECIDED / IN / OUT                                */
    char *inK;             /* [M] 1 when the facet is in In                           */
    int size;              /* |In|                                                    */
    sink_t *sink;
    uint64_t nodes, probes;
    uint64_t max_nodes;    /* 0: no limit; otherwise stop (and report) beyond this many nodes */
    int aborted;
} dfs_t;

/* Try to add facet p to In. Returns 1 and applies it when every check of the canonical
 * tree passes; returns 0 and changes nothing otherwise. */
static int dfs_add(dfs_t *d, int p)
{
    const incidence_t *I = d->I;
    int n = I->n, M = I->M;
    for (int k = 0; k < n; k++)
        if (d->deg[I->fr[p * n + k]] >= 2) return 0;          /* degree would reach 3 */
    if (d->cap >= 0 && d->size + 1 > d->cap) return 0;       /* upper bound on |K|   */
    for (int a = 0; a < d->c->n_affine; a++) {
        long cp = d->c->coef[(size_t)a * M + p];
        long bound = d->c->c0[a] + d->posall[a] + d->negin[a] + (cp < 0 ? cp : 0);
        if (bound <= 0) return 0;                             /* no completion has g > 0 */
    }
    for (int k = 0; k < n; k++) d->deg[I->fr[p * n + k]]++;
    for (int a = 0; a < d->c->n_affine; a++) {
        long cp = d->c->coef[(size_t)a * M + p];
        if (cp < 0) d->negin[a] += cp;
    }
    d->st[p] = IN;
    d->inK[p] = 1;
    d->size++;
    return 1;
}

static void dfs_remove(dfs_t *d, int p)
{
    const incidence_t *I = d->I;
    int n = I->n, M = I->M;
    for (int k = 0; k < n; k++) d->deg[I->fr[p * n + k]]--;
    for (int a = 0; a < d->c->n_affine; a++) {
        long cp = d->c->coef[(size_t)a * M + p];
        if (cp < 0) d->negin[a] -= cp;
    }
    d->st[p] = UNDECIDED;
    d->inK[p] = 0;
    d->size--;
}

static void dfs_visit(dfs_t *d)
{
    const incidence_t *I = d->I;
    int M = I->M, N = I->N;
    d->nodes++;
    if (d->max_nodes && d->nodes > d->max_nodes) { d->aborted = 1; return; }
    int r = -1;
    for (int i = 0; i < N; i++)
        if (d->deg[i] == 1) { r = i; break; }
    if (r >= 0) {
        /* ridge branch: exactly one more parent of r must join */
        int np = I->npar[r];
        const int *par = I->par + (size_t)r * M;
        int und[64], nu = 0;
        for (int k = 0; k < np; k++)
            if (d->st[par[k]] == UNDECIDED) und[nu++] = par[k];
        for (int a = 0; a < nu; a++) {
            int p = und[a];
            for (int b = 0; b < nu; b++)
                if (b != a) d->st[und[b]] = OUT;
            if (dfs_add(d, p)) {
                dfs_visit(d);
                dfs_remove(d, p);
            } else {
                d->probes++;
            }
            for (int b = 0; b < nu; b++)
                if (b != a) d->st[und[b]] = UNDECIDED;
            if (d->aborted) return;
        }
        return;
    }
    /* closure: In is a weak pseudo-manifold (Proposition 2.1) */
    if (affine_ok(d->c, M, d->inK)) sink_emit(d->sink, M, d->inK);
    int *und = (int *)malloc(sizeof(int) * (M ? M : 1));
    int nu = 0;
    for (int f = 0; f < M; f++)
        if (d->st[f] == UNDECIDED) und[nu++] = f;
    for (int a = 0; a < nu; a++) {
        int f = und[a];
        for (int b = 0; b < a; b++) d->st[und[b]] = OUT;
        if (dfs_add(d, f)) {
            dfs_visit(d);
            dfs_remove(d, f);
        } else {
            d->probes++;
        }
        for (int b = 0; b < a; b++) d->st[und[b]] = UNDECIDED;
        if (d->aborted) break;
    }
    free(und);
}

static int enumerate_dfs_budget(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                                uint64_t *masks, uint64_t cap_masks, orc_stats *st,
                                uint64_t max_nodes);

int orc_enumerate_dfs(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                      uint64_t *masks, uint64_t cap_masks, orc_stats *st)
{
    return enumerate_dfs_budget(n, m, M, facets, c, masks, cap_masks, st, 0);
}

/* As orc_enumerate_dfs, but give up (returning ORC_ERR_BUDGET) after max_nodes nodes. */
#define ORC_ERR_BUDGET -7
int orc_enumerate_dfs_budget(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                             orc_stats *st, uint64_t max_nodes)
{
    return enumerate_dfs_budget(n, m, M, facets, c, NULL, 0, st, max_nodes);
}

static int enumerate_dfs_budget(int n, int m, int M, const uint16_t *facets, const orc_cond *c,
                                uint64_t *masks, uint64_t cap_masks, orc_stats *st,
                                uint64_t max_nodes)
{
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    sink_t snk = { masks, cap_masks, 0, (M + 63) / 64, 0 };
    dfs_t d;
    memset(&d, 0, sizeof(d));
    d.I = &I; d.c = c; d.cap = cap; d.sink = &snk; d.max_nodes = max_nodes;
    int na = c->n_affine;
    d.posall = (long *)calloc(na ? na : 1, sizeof(long));
    d.negin = (long *)calloc(na ? na : 1, sizeof(long));
    d.deg = (unsigned char *)calloc(I.N ? I.N : 1, 1);
    d.st = (char *)calloc(M ? M : 1, 1);
    d.inK = (char *)calloc(M ? M : 1, 1);
    for (int a = 0; a < na; a++)
        for (int j = 0; j < M; j++) {
            long cj = c->coef[(size_t)a * M + j];
            if (cj > 0) d.posall[a] += cj;
        }
    /* the root: forced-in facets (and the base facet) in, forced-out facets out */
    int root_ok = 1;
    int base = c->base_facet ? base_facet_index(n, M, facets) : -1;
    if (c->base_facet && base < 0) root_ok = 0;
    for (int j = 0; j < M && root_ok; j++)
        if (c->forced_out && bit_of(c->forced_out, j)) {
            if ((c->forced_in && bit_of(c->forced_in, j)) || j == base) root_ok = 0;
            d.st[j] = OUT;
        }
    for (int j = 0; j < M && root_ok; j++)
        if ((c->forced_in && bit_of(c->forced_in, j)) || j == base)
            if (!dfs_add(&d, j)) root_ok = 0;
    if (root_ok)
        dfs_visit(&d);
    else
        d.probes++;
    free(d.posall); free(d.negin); free(d.deg); free(d.st); free(d.inK);
    incidence_free(&I);
    rc = sink_finish(&snk);
    if (st) { st->count = snk.count; st->nodes = d.nodes; st->probes = d.probes; }
    if (d.aborted) return ORC_ERR_BUDGET;
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* A seeded random walk down the canonical tree, used to pick subtrees of a large        */
/* instance as test inputs: from the root, `depth` times, list the children that pass     */
/* their checks and step into one drawn uniformly (splitmix64, Steele-Lea-Flood 2014);    */
/* at a node without children the walk starts again from the root with the generator     */
/* continuing. The node reached is returned as its In and Out masks (Out including the    */
/* facets excluded on the way), so that forced-in = In, forced-out = Out roots exactly    */
/* that subtree.                                                                          */
/* ---------------------------------------------------------------------------------- */

static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int orc_walk(int n, int m, int M, const uint16_t *facets, const orc_cond *c, uint64_t seed,
             int depth, uint64_t *in_mask, uint64_t *out_mask)
{
    int cap = resolve_cap(c->cap, n, m);
    if (cap == -3 || c->base_facet || c->forced_in || c->forced_out) return ORC_ERR_INPUT;
    incidence_t I;
    int rc = incidence_build(n, M, facets, &I);
    if (rc) return rc;
    dfs_t d;
    memset(&d, 0, sizeof(d));
    d.I = &I; d.c = c; d.cap = cap;
    int na = c->n_affine;
    d.posall = (long *)calloc(na ? na : 1, sizeof(long));
    d.negin = (long *)calloc(na ? na : 1, sizeof(long));
    d.deg = (unsigned char *)calloc(I.N ? I.N : 1, 1);
    d.st = (char *)calloc(M ? M : 1, 1);
    d.inK = (char *)calloc(M ? M : 1, 1);
    for (int a = 0; a < na; a++)
        for (int j = 0; j < M; j++)
            if (c->coef[(size_t)a * M + j] > 0) d.posall[a] += c->coef[(size_t)a * M + j];
    int *cand = (int *)malloc(sizeof(int) * (M ? M : 1));
    int *ok = (int *)malloc(sizeof(int) * (M ? M : 1));
    uint64_t rng = seed;
    int level = 0, attempts = 0;
    rc = ORC_OK;
    while (level < depth) {
        /* the children of the current node, as the canonical tree orders them */
        int r = -1;
        for (int i = 0; i < I.N; i++)
            if (d.deg[i] == 1) { r = i; break; }
        int nc = 0;
        if (r >= 0) {
            for (int k = 0; k < I.npar[r]; k++)
                if (d.st[I.par[(size_t)r * M + k]] == UNDECIDED) cand[nc++] = I.par[(size_t)r * M + k];
        } else {
            for (int f = 0; f < M; f++)
                if (d.st[f] == UNDECIDED) cand[nc++] = f;
        }
        int nok = 0;
        for (int a = 0; a < nc; a++)
            if (dfs_add(&d, cand[a])) { dfs_remove(&d, cand[a]); ok[nok++] = a; }
        if (nok == 0) {  /* dead end: start again from the root */
            if (++attempts > 10000) { rc = ORC_ERR_INPUT; break; }
            memset(d.deg, 0, I.N ? I.N : 1);
            memset(d.st, 0, M ? M : 1);
            memset(d.inK, 0, M ? M : 1);
            for (int a = 0; a < na; a++) d.negin[a] = 0;
            d.size = 0;
            level = 0;
            continue;
        }
        int a = ok[splitmix64_next(&rng) % (uint64_t)nok];
        int p = cand[a];
        if (r >= 0) {
            for (int b = 0; b < nc; b++)
                if (b != a) d.st[cand[b]] = OUT;
        } else {
            for (int b = 0; b < a; b++) d.st[cand[b]] = OUT;
        }
        dfs_add(&d, p);
        level++;
    }
    int W = (M + 63) / 64;
    for (int w = 0; w < W; w++) { in_mask[w] = 0; out_mask[w] = 0; }
    for (int j = 0; j < M; j++) {
        if (d.st[j] == IN) in_mask[j / 64] |= 1ull << (j % 64);
        if (d.st[j] == OUT) out_mask[j / 64] |= 1ull << (j % 64);
    }
    free(cand); free(ok);
    free(d.posall); free(d.negin); free(d.deg); free(d.st); free(d.inK);
    incidence_free(&I);
    return rc;
}

/* ---------------------------------------------------------------------------------- */
/* O4: n = 2. A pure 1-dimensional complex is a graph; it is a WPM exactly when every  */
/* vertex (ridge) has degree 0 or 2, i.e. it is a set of vertex-disjoint cycles.      */
/* Count those sets (with at most max_edges edges in total; -1 for no limit) by        */
/* listing every simple cycle of the candidate graph, then every family of pairwise   */
/* vertex-disjoint cycles.                                                             */
/* ---------------------------------------------------------------------------------- */

typedef struct { uint16_t verts; int len; } cycle_t;

static int adj_has(const uint16_t *adj, int a, int b) { return (adj[a] >> b) & 1; }

static void cycles_from(const uint16_t *adj, int s, int v, uint16_t used, int len, int second,
                        cycle_t *out, int *nout, int cap)
{
    for (int w = s + 1; w < 16; w++) {
        if (!adj_has(adj, v, w) || ((used >> w) & 1)) continue;
        cycles_from(adj, s, w, used | (uint16_t)(1u << w), len + 1, len == 1 ? w : second,
                    out, nout, cap);
    }
    /* close the path v -> s: a cycle needs 3+ vertices; keep one of its two directions
     * (the one whose second vertex is below its last vertex) */
    if (len >= 3 && adj_has(adj, v, s) && second < v) {
        if (*nout < cap) { out[*nout].verts = used; out[*nout].len = len; }
        (*nout)++;
    }
}

static long count_families(const cycle_t *cy, int nc, int from, uint16_t used, int edges,
                           int max_edges)
{
    long total = 1; /* the family chosen so far */
    for (int i = from; i < nc; i++) {
        if (cy[i].verts & used) continue;
        if (max_edges >= 0 && edges + cy[i].len > max_edges) continue;
        total += count_families(cy, nc, i + 1, used | cy[i].verts, edges + cy[i].len, max_edges);
    }
    return total;
}

/* edges: M vertex masks with two bits each. Returns the number of WPMs, or < 0. */
long orc_n2_cycle_sets(int M, const uint16_t *edges, int max_edges)
{
    uint16_t adj[16] = {0};
    for (int j = 0; j < M; j++) {
        if (__builtin_popcount(edges[j]) != 2) return ORC_ERR_INPUT;
        int a = __builtin_ctz(edges[j]);
        int b = 15 - __builtin_clz((unsigned)edges[j] << 16);
        adj[a] |= (uint16_t)(1u << b);
        adj[b] |= (uint16_t)(1u << a);
    }
    int cap = 1 << 16;
    cycle_t *cy = (cycle_t *)malloc(sizeof(cycle_t) * cap);
    int nc = 0;
    for (int s = 0; s < 16; s++)
        cycles_from(adj, s, s, (uint16_t)(1u << s), 1, -1, cy, &nc, cap);
    if (nc > cap) { free(cy); return ORC_ERR_CAPACITY; }
    long total = count_families(cy, nc, 0, 0, 0, max_edges);
    free(cy);
    return total;
}

/* Number of simple cycles of the candidate graph (n = 2), for tests. */
long orc_n2_cycle_count(int M, const uint16_t *edges)
{
    uint16_t adj[16] = {0};
    for (int j = 0; j < M; j++) {
        int a = __builtin_ctz(edges[j]);
        int b = 15 - __builtin_clz((unsigned)edges[j] << 16);
        adj[a] |= (uint16_t)(1u << b);
        adj[b] |= (uint16_t)(1u << a);
    }
    int cap = 1 << 16;
    cycle_t *cy = (cycle_t *)malloc(sizeof(cycle_t) * cap);
    int nc = 0;
    for (int s = 0; s < 16; s++)
        cycles_from(adj, s, s, (uint16_t)(1u << s), 1, -1, cy, &nc, cap);
    free(cy);
    return nc;
}

/* ---------------------------------------------------------------------------------- */
/* Algorithm 4.4, lines 8-12: the post-filters on each WPM K.                         */
/*   Pic(K) = (number of vertices of K) - n; K is discarded when Pic(K) < 4, i.e. when  */
/*   some vertex of [m] (m = n + 4) lies in no facet of K.                            */
/*   Seedness condition (Proposition 3.1): there is no face {v, w} of K such that every */
/*   minimal non-face of K contains both v and w or neither.                          */
/* Faces are the subsets of facets; a minimal non-face is a non-face all of whose     */
/* subsets with one vertex fewer are faces. Written out over all 2^m vertex subsets.  */
/* ---------------------------------------------------------------------------------- */

/* 1 when K (k facets given as vertex masks on [m]) uses every vertex and satisfies the
   seedness condition; 0 otherwise; -1 on bad input. */
int orc_pic_seed(int n, int m, int k, const uint16_t *kf)
{
    if (m < 1 || m > 16 || k < 0 || n < 1) return -1;
    uint32_t all = (m == 16) ? 0xFFFFu : ((1u << m) - 1u);
    uint32_t used = 0;
    for (int i = 0; i < k; i++) used |= kf[i];
    if (used != all) return 0;                      /* Pic(K) < 4 */
    uint32_t nsub = 1u << m;
    char *face = (char *)calloc(nsub, 1);
    if (!face) return -1;
    for (uint32_t S = 0; S < nsub; S++)
        for (int i = 0; i < k; i++)
            if ((S & ~(uint32_t)kf[i]) == 0) { face[S] = 1; break; }
    /* split[v][w] = 1 when some minimal non-face contains exactly one of v, w */
    char split[16][16];
    memset(split, 0, sizeof(split));
    for (uint32_t S = 1; S < nsub; S++) {
        if (face[S]) continue;
        int minimal = 1;
        for (int v = 0; v < m && minimal; v++)
            if (((S >> v) & 1u) && !face[S & ~(1u << v)]) minimal = 0;
        if (!minimal) continue;
        for (int v = 0; v < m; v++)
            for (int w = 0; w < m; w++)
                if ((((S >> v) & 1u) != 0) != (((S >> w) & 1u) != 0)) split[v][w] = 1;
    }
    int seed = 1;
    for (int v = 0; v < m && seed; v++)
        for (int w = v + 1; w < m && seed; w++)
            if (face[(1u << v) | (1u << w)] && !split[v][w]) seed = 0;
    free(face);
    return seed;
}

/* Apply orc_pic_seed to `count` output masks (W words each, facet j at bit j%64 of word
   j/64, facets[] the M candidate vertex masks): keep[i] = 1 for the kept ones. Returns the
   number kept, or -1 on bad input. */
long orc_filter_pic_seed(int n, int m, int M, const uint16_t *facets, const uint64_t *masks,
                         long count, int W, uint8_t *keep)
{
    uint16_t *kf = (uint16_t *)malloc(sizeof(uint16_t) * (M > 0 ? M : 1));
    if (!kf) return -1;
    long kept = 0;
    for (long i = 0; i < count; i++) {
        int k = 0;
        for (int j = 0; j < M; j++)
            if ((masks[i * W + j / 64] >> (j % 64)) & 1ull) kf[k++] = facets[j];
        int r = orc_pic_seed(n, m, k, kf);
        if (r < 0) { free(kf); return -1; }
        keep[i] = (uint8_t)r;
        kept += r;
    }
    free(kf);
    return kept;
}

/* ---------------------------------------------------------------------------------- */
/* Algorithm 4.4, line 14: one representative per isomorphism class. Two complexes are  */
/* isomorphic when a relabeling of the vertices maps the facets of one onto the facets  */
/* of the other. The canonical form of K is the smallest sorted list of relabeled facet */
/* masks over the leaves of a search that (1) colors the vertices by an invariant,      */
/* refined until stable (a vertex's new color: its color, then the sorted colors of the */
/* other vertices of each facet through it, those lists sorted), and (2) while some     */
/* color is shared, tries each vertex of the first shared color as a color of its own.  */
/* Every step uses invariants only, so isomorphic complexes get the same form.          */
/* ---------------------------------------------------------------------------------- */

typedef struct {
    int m, n, k;
    uint16_t f[512];
    uint16_t best[512];
    int have_best;
} canon_t;

/* one vertex's signature: its color, then the facets through it, each as the sorted colors
   of its other vertices, the facets sorted; written into sig (ints), returns the length */
static int vertex_signature(const canon_t *C, const int *col, int v, int *sig)
{
    int len = 0, nf = 0;
    int rows[512][16];
    sig[len++] = col[v];
    for (int i = 0; i < C->k; i++) {
        if (!((C->f[i] >> v) & 1u)) continue;
        int r = 0;
        for (int u = 0; u < C->m; u++)
            if (u != v && ((C->f[i] >> u) & 1u)) rows[nf][r++] = col[u];
        for (int a = 1; a < r; a++)              /* insertion sort of the row */
            for (int b = a; b > 0 && rows[nf][b - 1] > rows[nf][b]; b--) {
                int t = rows[nf][b]; rows[nf][b] = rows[nf][b - 1]; rows[nf][b - 1] = t;
            }
        for (int j = r; j < 16; j++) rows[nf][j] = -1;
        nf++;
    }
    for (int a = 1; a < nf; a++)                 /* sort the rows lexicographically */
        for (int b = a; b > 0 && memcmp(rows[b - 1], rows[b], sizeof(rows[0])) > 0; b--) {
            int t[16];
            memcpy(t, rows[b], sizeof(t)); memcpy(rows[b], rows[b - 1], sizeof(t));
            memcpy(rows[b - 1], t, sizeof(t));
        }
    sig[len++] = nf;
    for (int a = 0; a < nf; a++)
        for (int j = 0; j < 16; j++) sig[len++] = rows[a][j];
    return len;
}

static int cmp_sig(const int *a, int la, const int *b, int lb)
{
    int l = la < lb ? la : lb;
    for (int i = 0; i < l; i++)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return la == lb ? 0 : (la < lb ? -1 : 1);
}

/* refine col (ranks 0..) until the number of colors stops growing */
static void refine(const canon_t *C, int *col)
{
    static int sig[16][2 + 512 * 16];
    int len[16];
    for (;;) {
        int before = 0;
        for (int v = 0; v < C->m; v++) if (col[v] + 1 > before) before = col[v] + 1;
        for (int v = 0; v < C->m; v++) len[v] = vertex_signature(C, col, v, sig[v]);
        int idx[16], newcol[16];                /* vertices sorted by signature */
        for (int v = 0; v < C->m; v++) idx[v] = v;
        for (int a = 1; a < C->m; a++)
            for (int b = a; b > 0 && cmp_sig(sig[idx[b - 1]], len[idx[b - 1]],
                                             sig[idx[b]], len[idx[b]]) > 0; b--) {
                int t = idx[b]; idx[b] = idx[b - 1]; idx[b - 1] = t;
            }
        int rank = 0;                           /* equal signatures share a rank */
        for (int a = 0; a < C->m; a++) {
            if (a > 0 && cmp_sig(sig[idx[a - 1]], len[idx[a - 1]], sig[idx[a]], len[idx[a]]) != 0)
                rank++;
            newcol[idx[a]] = rank;
        }
        int after = 0;
        for (int v = 0; v < C->m; v++) if (newcol[v] + 1 > after) after = newcol[v] + 1;
        memcpy(col, newcol, sizeof(int) * C->m);
        if (after == before) return;
    }
}

static int cmp_u16(const void *a, const void *b)
{
    uint16_t x = *(const uint16_t *)a, y = *(const uint16_t *)b;
    return (x > y) - (x < y);
}

static void canon_search(canon_t *C, int *col)
{
    refine(C, col);
    int count[16] = {0};
    for (int v = 0; v < C->m; v++) count[col[v]]++;
    int target = -1;
    for (int c = 0; c < C->m; c++) if (count[c] > 1) { target = c; break; }
    if (target < 0) {                           /* discrete: vertex v gets label col[v] */
        uint16_t g[512];
        for (int i = 0; i < C->k; i++) {
            uint16_t x = 0;
            for (int v = 0; v < C->m; v++) if ((C->f[i] >> v) & 1u) x |= (uint16_t)(1u << col[v]);
            g[i] = x;
        }
        qsort(g, (size_t)C->k, sizeof(uint16_t), cmp_u16);
        int better = !C->have_best;
        for (int i = 0; i < C->k && !better; i++) {
            if (g[i] != C->best[i]) { better = g[i] < C->best[i]; break; }
        }
        if (better) { memcpy(C->best, g, sizeof(uint16_t) * (size_t)C->k); C->have_best = 1; }
        return;
    }
    for (int v = 0; v < C->m; v++) {
        if (col[v] != target) continue;
        int c2[16];                             /* v keeps the color, its cell mates move up */
        for (int u = 0; u < C->m; u++)
            c2[u] = col[u] > target ? col[u] + 1 : (col[u] == target && u != v ? target + 1 : col[u]);
        canon_search(C, c2);
    }
}

/* Canonical form of K (k facets as vertex masks on [m], m <= 16, k <= 512): the sorted
   relabeled facet masks in out[0..k). Returns 0, or -1 on bad input. */
int orc_canonical_form(int m, int k, const uint16_t *facets, uint16_t *out)
{
    if (m < 1 || m > 16 || k < 0 || k > 512) return -1;
    canon_t *C = (canon_t *)calloc(1, sizeof(canon_t));
    if (!C) return -1;
    C->m = m; C->k = k;
    memcpy(C->f, facets, sizeof(uint16_t) * (size_t)k);
    int col[16] = {0};
    canon_search(C, col);
    memcpy(out, C->best, sizeof(uint16_t) * (size_t)k);
    free(C);
    return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Algorithm 4.4, line 16: PL sphereness by the criterion of Lemma 3.3 (PL sphereness): */
/* a WPM of Picard number <= 7 is a PL sphere exactly when the link of every face,      */
/* the empty face included, is a Z2-homology sphere: its reduced Z2-homology is Z2 in   */
/* its top dimension and zero below. Faces and links are read off a bitmap of all 2^m   */
/* vertex subsets; reduced Betti numbers come from GF(2) ranks of boundary matrices.    */
/* ---------------------------------------------------------------------------------- */

/* GF(2) rank of nrows rows of W words (the rows are overwritten) */
static int gf2_rank_rows(uint64_t *rows, int nrows, int W)
{
    int rank = 0;
    for (int col = 0; col < W * 64 && rank < nrows; col++) {
        int w = col / 64;
        uint64_t bit = 1ull << (col % 64);
        int piv = -1;
        for (int r = rank; r < nrows; r++)
            if (rows[(size_t)r * W + w] & bit) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int x = 0; x < W; x++) {
                uint64_t t = rows[(size_t)piv * W + x];
                rows[(size_t)piv * W + x] = rows[(size_t)rank * W + x];
                rows[(size_t)rank * W + x] = t;
            }
        for (int r = 0; r < nrows; r++)
            if (r != rank && (rows[(size_t)r * W + w] & bit))
                for (int x = 0; x < W; x++) rows[(size_t)r * W + x] ^= rows[(size_t)rank * W + x];
        rank++;
    }
    return rank;
}

/* 1 when the link of sigma (a face; face[] the face bitmap of K over [m]) is a Z2-homology
   sphere of dimension d = dim K - |sigma| */
static int link_is_z2_sphere(const char *face, int m, uint32_t sigma, int d)
{
    uint32_t nsub = 1u << m;
    uint32_t rest = (nsub - 1u) & ~sigma;
    /* link faces by size: tau subset of rest with tau | sigma a face */
    int *idx = (int *)malloc(sizeof(int) * nsub);
    int cnt[18] = {0};
    uint32_t *list[18];
    for (int s = 0; s <= d + 1 && s < 18; s++) list[s] = (uint32_t *)malloc(sizeof(uint32_t) * nsub);
    for (uint32_t t = rest;; t = (t - 1) & rest) {
        if (face[t | sigma]) {
            int s = __builtin_popcount(t);
            if (s <= d + 1) { idx[t] = cnt[s]; list[s][cnt[s]++] = t; }
        }
        if (t == 0) break;
    }
    /* rank of the boundary from size s faces to size s-1 faces, s = 1..d+1 */
    int rk[19] = {0};
    for (int s = 1; s <= d + 1; s++) {
        int rows = cnt[s], cols = cnt[s - 1];
        if (!rows || !cols) continue;
        int W = (cols + 63) / 64;
        uint64_t *mat = (uint64_t *)calloc((size_t)rows * W, sizeof(uint64_t));
        for (int r = 0; r < rows; r++) {
            uint32_t t = list[s][r];
            for (int v = 0; v < m; v++)
                if ((t >> v) & 1u) {
                    int c = idx[t & ~(1u << v)];
                    mat[(size_t)r * W + c / 64] ^= 1ull << (c % 64);
                }
        }
        rk[s] = gf2_rank_rows(mat, rows, W);
        free(mat);
    }
    /* reduced Betti number in dimension i (faces of size i + 1): cnt - rank out - rank in */
    int ok = 1;
    for (int s = 0; s <= d + 1 && ok; s++) {
        int betti = cnt[s] - rk[s] - (s + 1 <= d + 1 ? rk[s + 1] : 0);
        int want = (s == d + 1) ? 1 : 0;
        if (betti != want) ok = 0;
    }
    for (int s = 0; s <= d + 1 && s < 18; s++) free(list[s]);
    free(idx);
    return ok;
}

/* 1 when K (k facets, vertex masks on [m], every facet of n vertices) satisfies Lemma 3.3's
   criterion; 0 otherwise; -1 on bad input. */
int orc_pl_sphere(int n, int m, int k, const uint16_t *kf)
{
    if (m < 1 || m > 15 || n < 1 || k < 0) return -1;
    uint32_t nsub = 1u << m;
    char *face = (char *)calloc(nsub, 1);
    if (!face) return -1;
    for (uint32_t S = 0; S < nsub; S++)
        for (int i = 0; i < k; i++)
            if ((S & ~(uint32_t)kf[i]) == 0) { face[S] = 1; break; }
    int ok = 1;
    for (uint32_t S = 0; S < nsub && ok; S++) {
        if (!face[S]) continue;
        int d = (n - 1) - __builtin_popcount(S);  /* dimension of the link of S */
        if (!link_is_z2_sphere(face, m, S, d)) ok = 0;
    }
    free(face);
    return ok;
}
