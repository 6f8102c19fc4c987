// wpm_sphere.cpp -- PL sphereness of complexes (Algorithm 4.4, line 16), on the host.
//
// Lemma 3.3 (PL sphereness): a weak pseudo-manifold of Picard number at most 7 is a PL
// sphere exactly when the link of every face, the empty face included, is a Z2-homology
// sphere. For a complex K of dimension n - 1 on [m] (m <= 15): the faces of K are the
// vertex subsets inside some facet (a bitmap over all 2^m subsets); the link of a face s has
// the faces t, disjoint from s, with t + s a face, and dimension n - 1 - |s|. Its reduced
// Z2-Betti numbers are b_i = c_i - r_i - r_(i+1), with c_i its faces of dimension i (the
// empty face in dimension -1) and r_i the GF(2) rank of the boundary map from dimension i to
// dimension i - 1; a Z2-homology sphere of dimension d has b_d = 1 and every other b_i = 0.
// Ranks are computed by inserting each boundary row into a basis kept by leading bit.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "wpm.h"
#include "wpm_host.h"

namespace wpm {
namespace {

class Spheres {
 public:
  explicit Spheres(int m) : m_(m), nsub_(1u << m), face_(nsub_), pos_(nsub_) {}

  bool is_pl_sphere(int n, const uint16_t *f, int k) {
    std::fill(face_.begin(), face_.end(), 0);
    for (int i = 0; i < k; i++) {  // every subset of every facet
      const uint32_t F = f[i];
      for (uint32_t t = F;; t = (t - 1) & F) {
        face_[t] = 1;
        if (t == 0) break;
      }
    }
    for (uint32_t s = 0; s < nsub_; s++) {
      if (!face_[s]) continue;
      const int d = n - 1 - popc(s);
      if (!link_is_sphere(s, d)) return false;
    }
    return true;
  }

 private:
  static int popc(uint32_t x) { return __builtin_popcount(x); }

  // GF(2) rank of the boundary from the link faces of size sz to those of size sz - 1
  int boundary_rank(const std::vector<uint32_t> &hi, const std::vector<uint32_t> &lo) {
    if (hi.empty() || lo.empty()) return 0;
    const size_t W = (lo.size() + 63) / 64;
    for (size_t j = 0; j < lo.size(); j++) pos_[lo[j]] = (int32_t)j;
    basis_.clear();
    lead_.assign(lo.size(), -1);  // basis row whose leading column is j
    std::vector<uint64_t> row(W);
    int rank = 0;
    for (uint32_t t : hi) {
      std::fill(row.begin(), row.end(), 0);
      for (int v = 0; v < m_; v++)
        if ((t >> v) & 1u) {
          const int j = pos_[t & ~(1u << v)];
          row[j >> 6] ^= 1ull << (j & 63);
        }
      // reduce by the basis, leading (highest) column first
      for (int w = (int)W - 1; w >= 0; w--) {
        while (row[w]) {
          const int j = w * 64 + 63 - __builtin_clzll(row[w]);
          const int b = lead_[j];
          if (b < 0) {  // a new leading column: the row joins the basis
            lead_[j] = rank++;
            basis_.insert(basis_.end(), row.begin(), row.end());
            goto next_row;
          }
          const uint64_t *br = basis_.data() + (size_t)b * W;
          for (size_t x = 0; x <= (size_t)w; x++) row[x] ^= br[x];
        }
      }
    next_row:;
    }
    return rank;
  }

  bool link_is_sphere(uint32_t s, int d) {
    const uint32_t rest = (nsub_ - 1u) & ~s;
    for (auto &v : by_size_) v.clear();
    if ((int)by_size_.size() < d + 2) by_size_.resize(d + 2);
    for (uint32_t t = rest;; t = (t - 1) & rest) {
      if (face_[t | s]) {
        const int z = popc(t);
        if (z > d + 1) return false;  // a face above the link's dimension: not pure
        by_size_[z].push_back(t);
      }
      if (t == 0) break;
    }
    // b at size z (dimension z - 1): c - rank(size z -> z-1) - rank(size z+1 -> z)
    std::vector<int> r(d + 3, 0);
    for (int z = 1; z <= d + 1; z++) r[z] = boundary_rank(by_size_[z], by_size_[z - 1]);
    for (int z = 0; z <= d + 1; z++) {
      const int b = (int)by_size_[z].size() - r[z] - (z + 1 <= d + 1 ? r[z + 1] : 0);
      if (b != (z == d + 1 ? 1 : 0)) return false;
    }
    return true;
  }

  int m_;
  uint32_t nsub_;
  std::vector<uint8_t> face_;
  std::vector<int32_t> pos_;
  std::vector<std::vector<uint32_t>> by_size_;
  std::vector<uint64_t> basis_;
  std::vector<int> lead_;
};

}  // namespace
}  // namespace wpm

using namespace wpm;

extern "C" long wpm_pl_spheres(int n, int m, int count, const uint64_t *offsets,
                               const uint16_t *facets, uint8_t *is_sphere) {
  if (n < 1 || m < 1 || m > 15 || count < 0 ||
      (count > 0 && (!offsets || !facets || !is_sphere)))
    return fail(WPM_ERR_INPUT, "wpm_pl_spheres: bad arguments (m <= 15)");
  for (int c = 0; c < count; c++) {
    if (offsets[c + 1] < offsets[c])
      return fail(WPM_ERR_INPUT, "wpm_pl_spheres: offsets decrease at %d", c);
    for (uint64_t i = offsets[c]; i < offsets[c + 1]; i++)
      if ((facets[i] >> m) || __builtin_popcount(facets[i]) != n)
        return fail(WPM_ERR_INPUT, "wpm_pl_spheres: complex %d has a facet that is not an "
                    "n-subset of [m]", c);
  }
  auto work = [&](int lo, int hi) {
    Spheres S(m);
    for (int c = lo; c < hi; c++)
      is_sphere[c] = S.is_pl_sphere(n, facets + offsets[c], (int)(offsets[c + 1] - offsets[c]))
                         ? 1 : 0;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int n_thr = (int)std::min<unsigned>(std::min(32u, hw), (unsigned)std::max(1, count));
  if (n_thr <= 1) {
    work(0, count);
  } else {
    std::vector<std::thread> th;
    const int per = (count + n_thr - 1) / n_thr;
    for (int t = 0; t < n_thr; t++)
      th.emplace_back(work, std::min(count, t * per), std::min(count, (t + 1) * per));
    for (auto &t : th) t.join();
  }
  long spheres = 0;
  for (int c = 0; c < count; c++) spheres += is_sphere[c];
  return spheres;
}
