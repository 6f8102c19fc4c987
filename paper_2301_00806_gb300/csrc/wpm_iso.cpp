// wpm_iso.cpp -- isomorphism classes of complexes (Algorithm 4.4, line 14), on the host.
//
// Two complexes on [m] are isomorphic when a relabeling of the vertices maps the facets of
// one onto the facets of the other. Each complex gets a canonical form: the smallest sorted
// list of relabeled facet masks over the leaves of a search that
//   - colours the vertices and refines the colours until their number stops growing: the
//     new colour of v mixes its colour with, over the facets through v, a mix of the
//     colours of the facet's other vertices (sums of mixed values, so no order enters);
//     colours are the ranks of these values;
//   - while a colour is shared, gives each vertex of the smallest shared colour, in turn, a
//     colour of its own and searches on.
// Every step depends on invariants only, so isomorphic complexes get equal forms; equal
// mixes of different data only merge colours, which widens the search without changing the
// form. Classes are numbered in order of first appearance.
//
// Automorphism pruning. Two leaves with equal relabeled facet lists give an automorphism g
// of K (one leaf's labeling followed by the inverse of the other's). If g fixes the vertices
// individualized above a node and maps an explored child u of that node to a child v, the
// subtrees of u and v have the same leaves up to g, so v is skipped; when a new automorphism
// shows that the child being searched is such a v, the search returns to that node at once.
// Pruning removes only subtrees whose leaves have all been seen, so forms are unchanged; it
// turns searches over highly symmetric complexes (joins, suspensions, wedges), whose
// automorphism groups have up to ~10^5 elements, from exponential into a few hundred leaves.
#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wpm.h"
#include "wpm_host.h"

namespace wpm {
namespace {

inline uint64_t mix64(uint64_t x) {  // a bijective 64-bit finaliser
  x ^= x >> 31;
  x *= 0x7fb5d329728ea185ull;
  x ^= x >> 27;
  x *= 0x81dadef4bc2dd44dull;
  x ^= x >> 33;
  return x;
}

struct FormHash {
  size_t operator()(const std::vector<uint16_t> &v) const {
    uint64_t h = 0x243f6a8885a308d3ull ^ v.size();
    for (uint16_t x : v) h = mix64(h ^ x);
    return (size_t)h;
  }
};

struct Canon {
  int m = 0;
  const uint16_t *f = nullptr;
  int k = 0;
  std::vector<uint16_t> best, leaf;
  bool have = false;

  // colours (ranks 0..) refined in place until their number is stable
  void refine(int *col) const {
    int ncol = 0;
    for (int v = 0; v < m; v++) ncol = std::max(ncol, col[v] + 1);
    for (;;) {
      uint64_t key[16];
      for (int v = 0; v < m; v++) key[v] = 0;
      for (int i = 0; i < k; i++) {
        const uint16_t F = f[i];
        uint64_t s = 0;  // the facet's colours, mixed and summed
        for (int u = 0; u < m; u++)
          if ((F >> u) & 1u) s += mix64(0x9e3779b97f4a7c15ull * (uint64_t)(col[u] + 1));
        for (int v = 0; v < m; v++) {
          if (!((F >> v) & 1u)) continue;
          const uint64_t others = s - mix64(0x9e3779b97f4a7c15ull * (uint64_t)(col[v] + 1));
          key[v] += mix64(others ^ 0x5851f42d4c957f2dull);
        }
      }
      // sort by (old colour, key); equal pairs share the new colour
      int idx[16];
      for (int v = 0; v < m; v++) idx[v] = v;
      std::sort(idx, idx + m, [&](int a, int b) {
        return col[a] != col[b] ? col[a] < col[b] : key[a] < key[b];
      });
      int nc[16], r = 0;
      for (int a = 0; a < m; a++) {
        if (a > 0 && (col[idx[a]] != col[idx[a - 1]] || key[idx[a]] != key[idx[a - 1]])) r++;
        nc[idx[a]] = r;
      }
      std::memcpy(col, nc, sizeof(int) * m);
      if (r + 1 == ncol) return;
      ncol = r + 1;
    }
  }

  // search state: path[d] = vertex individualized at depth d, done[d] = explored children
  // of the node at depth d (bit v), autos = automorphisms found, seen = leaf forms found
  int path[16] = {0};
  uint32_t done[17] = {0};
  std::vector<std::array<uint8_t, 16>> autos;
  std::unordered_map<std::vector<uint16_t>, std::array<uint8_t, 16>, FormHash> seen;
  static constexpr size_t kMaxAutos = 64, kMaxSeen = 4096;

  // 1 when v is in the orbit of a vertex of `set` under the group generated by the known
  // automorphisms that fix path[0..depth) pointwise
  bool orbit_hits(int v, uint32_t set, int depth) const {
    if (!set) return false;
    int parent[16];
    for (int u = 0; u < m; u++) parent[u] = u;
    auto find = [&](int x) {
      while (parent[x] != x) x = parent[x] = parent[parent[x]];
      return x;
    };
    for (const auto &g : autos) {
      bool fixes = true;
      for (int d = 0; d < depth && fixes; d++) fixes = g[path[d]] == path[d];
      if (!fixes) continue;
      for (int u = 0; u < m; u++) {
        const int a = find(u), b = find(g[u]);
        if (a != b) parent[a] = b;
      }
    }
    const int r = find(v);
    for (int u = 0; u < m; u++)
      if (((set >> u) & 1u) && find(u) == r) return true;
    return false;
  }

  // Searches the node at `depth`; returns -1, or the depth of an ancestor whose current
  // child turned out equivalent to an explored one (the search resumes there).
  int search(int *col, int depth) {
    refine(col);
    int cnt[16] = {0};
    for (int v = 0; v < m; v++) cnt[col[v]]++;
    int target = -1;
    for (int c = 0; c < m; c++)
      if (cnt[c] > 1) {
        target = c;
        break;
      }
    if (target < 0) {  // every vertex has its own colour: relabel v as col[v]
      leaf.resize(k);
      for (int i = 0; i < k; i++) {
        uint16_t x = 0;
        for (int v = 0; v < m; v++)
          if ((f[i] >> v) & 1u) x |= (uint16_t)(1u << col[v]);
        leaf[i] = x;
      }
      std::sort(leaf.begin(), leaf.end());
      if (!have || leaf < best) {
        best = leaf;
        have = true;
      }
      std::array<uint8_t, 16> lab{};
      for (int v = 0; v < m; v++) lab[v] = (uint8_t)col[v];
      auto it = seen.find(leaf);
      if (it == seen.end()) {
        if (seen.size() < kMaxSeen) seen.emplace(leaf, lab);
        return -1;
      }
      // equal forms: g = (the earlier leaf's labeling)^-1 o (this leaf's labeling)
      int inv[16];
      for (int v = 0; v < m; v++) inv[it->second[v]] = v;
      std::array<uint8_t, 16> g{};
      bool identity = true;
      for (int v = 0; v < m; v++) {
        g[v] = (uint8_t)inv[lab[v]];
        identity = identity && g[v] == v;
      }
      if (identity || autos.size() >= kMaxAutos) return -1;
      autos.push_back(g);
      for (int d = 0; d < depth; d++)
        if (orbit_hits(path[d], done[d], d)) return d;
      return -1;
    }
    done[depth] = 0;
    for (int v = 0; v < m; v++) {
      if (col[v] != target) continue;
      if (orbit_hits(v, done[depth], depth)) continue;
      int c2[16];
      for (int u = 0; u < m; u++)
        c2[u] = col[u] > target ? col[u] + 1 : (col[u] == target && u != v ? target + 1 : col[u]);
      path[depth] = v;
      const int r = search(c2, depth + 1);
      done[depth] |= 1u << v;
      if (r >= 0 && r < depth) return r;
    }
    return -1;
  }
};


}  // namespace
}  // namespace wpm

using namespace wpm;

extern "C" long wpm_iso_classes(int m, int count, const uint64_t *offsets,
                                const uint16_t *facets, int32_t *class_of) {
  if (m < 1 || m > WPM_MAX_VERTICES || count < 0 || (count > 0 && (!offsets || !facets || !class_of)))
    return fail(WPM_ERR_INPUT, "wpm_iso_classes: bad arguments");
  for (int c = 0; c < count; c++) {
    if (offsets[c + 1] < offsets[c])
      return fail(WPM_ERR_INPUT, "wpm_iso_classes: offsets decrease at %d", c);
    for (uint64_t i = offsets[c]; i < offsets[c + 1]; i++)
      if (m < 16 && (facets[i] >> m))
        return fail(WPM_ERR_INPUT, "wpm_iso_classes: complex %d has a vertex >= m", c);
  }
  std::vector<std::vector<uint16_t>> form(count);
  auto work = [&](int lo, int hi) {
    for (int c = lo; c < hi; c++) {
      Canon C;
      C.m = m;
      C.f = facets + offsets[c];
      C.k = (int)(offsets[c + 1] - offsets[c]);
      int col[16] = {0};
      C.search(col, 0);
      form[c] = std::move(C.best);
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int n_thr = (int)std::min<unsigned>(std::min(32u, hw), (unsigned)std::max(1, count / 64));
  if (n_thr <= 1) {
    work(0, count);
  } else {
    std::vector<std::thread> th;
    const int per = (count + n_thr - 1) / n_thr;
    for (int t = 0; t < n_thr; t++)
      th.emplace_back(work, t * per, std::min(count, (t + 1) * per));
    for (auto &t : th) t.join();
  }
  std::unordered_map<std::vector<uint16_t>, int32_t, FormHash> id;
  id.reserve((size_t)count);
  for (int c = 0; c < count; c++) {
    auto it = id.emplace(form[c], (int32_t)id.size()).first;
    class_of[c] = it->second;
  }
  return (long)id.size();
}
