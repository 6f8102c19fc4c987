// wpm_link.cpp -- the link conditions of Section 4.4 ("Enumeration for n = 11"), on the host.
//
// A seed K of dimension 10 on 15 vertices has a vertex whose link has Picard number 4; call
// it the apex a = m - 1. Its link L is a 9-dimensional PL sphere on the other 14 vertices
// whose dual map mu is the restriction of K's map, and since mu is injective into the 15
// nonzero vectors of Z2^4, K's map is mu plus the one vector mu misses. Every K with
// Lk_K(a) = L contains the cone {sigma + a : sigma in L}, which gives conditions (1) and (2)
// on the facet vector of K: the cone facets are in K, every other candidate facet through a
// is not. This file turns (mu, L) into K's map and those two masks over K's candidate facets,
// which the search then takes as forced-in / forced-out properties.
#include <cstdint>
#include <cstring>
#include <vector>

#include "wpm.h"
#include "wpm_host.h"

namespace wpm {
namespace {

// GF(2) rank of k vectors of at most 16 bits
int rank_gf2(const uint32_t *v, int k) {
  uint32_t basis[32] = {0};  // basis[b]: the kept vector whose leading bit is b
  int r = 0;
  for (int i = 0; i < k; i++) {
    uint32_t x = v[i];
    for (int b = 31; b >= 0 && x; b--) {
      if (!((x >> b) & 1u)) continue;
      if (!basis[b]) {
        basis[b] = x;
        r++;
        x = 0;
      } else {
        x ^= basis[b];
      }
    }
  }
  return r;
}

}  // namespace
}  // namespace wpm

using namespace wpm;

extern "C" int wpm_link_conditions(int n, int m, const uint32_t *mu_rows, uint32_t apex_row,
                                   const uint16_t *link_facets, int link_count,
                                   uint32_t *lambda_rows_out, uint64_t *forced_in,
                                   uint64_t *forced_out, int words) {
  if (n < 2 || m <= n || m > WPM_MAX_VERTICES)
    return fail(WPM_ERR_INPUT, "wpm_link_conditions: need 2 <= n < m <= 16 (n=%d, m=%d)", n, m);
  if (!mu_rows || !lambda_rows_out || !forced_in || !forced_out || link_count < 0 ||
      (link_count > 0 && !link_facets))
    return fail(WPM_ERR_INPUT, "wpm_link_conditions: NULL pointer or negative link_count");
  const int p = m - n;
  const uint32_t top = 1u << p;
  // K's dual map: mu on 0..m-2, the apex row on m-1
  uint32_t lam[WPM_MAX_VERTICES];
  std::vector<char> taken(top, 0);
  for (int i = 0; i < m - 1; i++) {
    const uint32_t v = mu_rows[i];
    if (v == 0 || v >= top)
      return fail(WPM_ERR_INPUT, "wpm_link_conditions: mu row %d (%u) is not a nonzero vector "
                  "of Z2^%d", i, v, p);
    if (taken[v]) return fail(WPM_ERR_INPUT, "wpm_link_conditions: mu repeats the row %u", v);
    taken[v] = 1;
    lam[i] = v;
  }
  if (apex_row == 0) {
    int n_missing = 0;
    for (uint32_t v = 1; v < top; v++)
      if (!taken[v]) {
        n_missing++;
        apex_row = v;
      }
    if (n_missing != 1)
      return fail(WPM_ERR_INPUT, "wpm_link_conditions: apex_row 0 needs mu to miss exactly one "
                  "nonzero vector of Z2^%d (m = 2^%d - 1)", p, p);
  }
  if (apex_row >= top || taken[apex_row])
    return fail(WPM_ERR_INPUT, "wpm_link_conditions: apex row %u is not a new nonzero vector "
                "of Z2^%d", apex_row, p);
  lam[m - 1] = apex_row;
  if (rank_gf2(lam, m) != p)
    return fail(WPM_ERR_INPUT, "wpm_link_conditions: the dual rows have rank < %d", p);

  // K's candidate facets in lexicographic order of their sorted vertex tuples: the
  // n-subsets whose complement's p dual rows are a basis of Z2^p (Proposition 4.2)
  const uint32_t all = (1u << m) - 1u;
  std::vector<int32_t> index(1u << m, -1);
  int M = 0;
  int c[WPM_MAX_VERTICES];
  for (int i = 0; i < n; i++) c[i] = i;
  for (;;) {
    uint32_t s = 0;
    for (int i = 0; i < n; i++) s |= 1u << c[i];
    uint32_t rest[16];
    int k = 0;
    for (int v = 0; v < m; v++)
      if (((all & ~s) >> v) & 1u) rest[k++] = lam[v];
    if (rank_gf2(rest, k) == p) {
      if (M >= WPM_MAX_FACETS)
        return fail(WPM_ERR_LIMIT, "wpm_link_conditions: more than %d candidate facets",
                    WPM_MAX_FACETS);
      index[s] = M++;
    }
    int i = n - 1;
    while (i >= 0 && c[i] == m - n + i) i--;
    if (i < 0) break;
    c[i]++;
    for (int j = i + 1; j < n; j++) c[j] = c[j - 1] + 1;
  }
  const int W = M > 0 ? (M + 63) / 64 : 1;
  if (words < W)
    return fail(WPM_ERR_CAPACITY, "wpm_link_conditions: %d words per mask needed (M = %d), "
                "%d given", W, M, words);

  // condition (1): the cone facets; condition (2): the other candidates through the apex
  const uint32_t apex = 1u << (m - 1);
  std::vector<uint64_t> fin(W, 0), fout(W, 0);
  for (int i = 0; i < link_count; i++) {
    const uint32_t s = link_facets[i];
    if ((s & apex) || s >= apex || __builtin_popcount(s) != n - 1)
      return fail(WPM_ERR_INPUT, "wpm_link_conditions: link facet %d (0x%x) is not an "
                  "%d-subset of [%d]", i, s, n - 1, m - 1);
    const int j = index[s | apex];
    if (j < 0)
      return fail(WPM_ERR_INPUT, "wpm_link_conditions: link facet %d (0x%x) plus the apex is "
                  "not a candidate facet (the link does not support mu)", i, s);
    const uint64_t bit = 1ull << (j % 64);
    if (fin[j / 64] & bit)
      return fail(WPM_ERR_INPUT, "wpm_link_conditions: link facet %d (0x%x) is repeated", i, s);
    fin[j / 64] |= bit;
  }
  for (uint32_t s = 0; s <= all; s++) {
    if (!(s & apex) || index[s] < 0) continue;
    const int j = index[s];
    const uint64_t bit = 1ull << (j % 64);
    if (!(fin[j / 64] & bit)) fout[j / 64] |= bit;
  }
  std::memcpy(lambda_rows_out, lam, sizeof(uint32_t) * (size_t)m);
  for (int w = 0; w < words; w++) {
    forced_in[w] = w < W ? fin[w] : 0;
    forced_out[w] = w < W ? fout[w] : 0;
  }
  return M;
}
