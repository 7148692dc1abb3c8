// Subdomain and coarse-agglomerate partitions (Sec. 3: T_H by agglomeration of fine elements) by
// recursive coordinate bisection of element area centroids.
#include <algorithm>
#include <numeric>
#include <utility>

#include "common.h"
#include "hostpool.h"
#include "plan.h"

namespace dgasm {

// Recursive coordinate bisection, level by level: every segment of a level (a range of elems with its part
// count k and first part number) is split independently (the longer side of its centroids' bounding box, the
// first floor(n floor(k/2) / k) elements in (coordinate, element id) order to the left), so the segments of a
// level run in parallel and the parts do not depend on the threads.
void rcb_parts(const MeshData& m, std::vector<int> elems, int k, std::vector<int>& part_of, int first_part) {
  struct Seg {
    size_t lo, hi;
    int k, first;
  };
  const double *cx = m.cx.data(), *cy = m.cy.data();
  std::vector<Seg> level{{0, elems.size(), k, first_part}}, next;
  while (!level.empty()) {
    next.assign(2 * level.size(), Seg{0, 0, 0, 0});
    parallel_for((int)level.size(), [&](int si) {
      const Seg g = level[si];
      if (g.k <= 1) {
        for (size_t i = g.lo; i < g.hi; ++i) part_of[elems[i]] = g.first;
        return;
      }
      double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
      for (size_t i = g.lo; i < g.hi; ++i) {
        const int e = elems[i];
        xmin = std::min(xmin, cx[e]); xmax = std::max(xmax, cx[e]);
        ymin = std::min(ymin, cy[e]); ymax = std::max(ymax, cy[e]);
      }
      const double* c = (xmax - xmin >= ymax - ymin) ? cx : cy;
      const int kl = g.k / 2;
      const size_t n = g.hi - g.lo;
      const size_t nl = (n * (size_t)kl) / (size_t)g.k;
      // the first nl elements in the (coordinate, element id) order: a strict total order, so selecting them
      // with nth_element gives exactly the set a full sort would (the keys sit side by side for the selection)
      if (nl > 0 && nl < n) {
        thread_local std::vector<std::pair<double, int>> keys;
        keys.resize(n);
        for (size_t i = 0; i < n; ++i) keys[i] = {c[elems[g.lo + i]], elems[g.lo + i]};
        std::nth_element(keys.begin(), keys.begin() + nl, keys.end());
        for (size_t i = 0; i < n; ++i) elems[g.lo + i] = keys[i].second;
      }
      next[2 * si] = Seg{g.lo, g.lo + nl, kl, g.first};
      next[2 * si + 1] = Seg{g.lo + nl, g.hi, g.k - kl, g.first + kl};
    });
    level.clear();
    for (const Seg& g : next)
      if (g.k > 0) level.push_back(g);
  }
}

int compute_partition(const MeshData& m, int nsub, int ncoarse, std::vector<int>& sub, std::vector<int>* agg) {
  int ne = m.ne;
  if (nsub < 1 || nsub > ne) return set_error(DGASM_EINVAL, "nsub=%d must lie in [1, %d]", nsub, ne);
  if (ncoarse < 0 || ncoarse > ne) return set_error(DGASM_EINVAL, "ncoarse=%d must lie in [0, %d]", ncoarse, ne);
  sub.assign(ne, 0);
  std::vector<int> all(ne);
  std::iota(all.begin(), all.end(), 0);
  rcb_parts(m, all, nsub, sub, 0);
  if (agg && ncoarse > 0) {
    agg->assign(ne, 0);
    if (ncoarse >= nsub) {
      std::vector<std::vector<int>> members(nsub);
      for (int e = 0; e < ne; ++e) members[sub[e]].push_back(e);
      for (int i = 0; i < nsub; ++i) {
        const int ci = (int)(((long long)(i + 1) * ncoarse) / nsub - ((long long)i * ncoarse) / nsub);
        if (ci < 1 || (size_t)ci > members[i].size())
          return set_error(DGASM_EINVAL, "subdomain %d cannot hold %d agglomerates", i, ci);
      }
      // subdomain i's agglomerates are numbered from floor(i ncoarse / nsub) on
      parallel_for(nsub, [&](int i) {
        const int first = (int)(((long long)i * ncoarse) / nsub);
        const int ci = (int)(((long long)(i + 1) * ncoarse) / nsub) - first;
        rcb_parts(m, members[i], ci, *agg, first);
      });
    } else {
      rcb_parts(m, all, ncoarse, *agg, 0);
    }
  }
  return DGASM_OK;
}

}  // namespace dgasm

extern "C" int dgasm_partition(dgasm_mesh_t h, int nsub, int ncoarse, int* sub_of_elem, int* agg_of_elem) {
  using namespace dgasm;
  clear_error();
  if (!h || !sub_of_elem) return set_error(DGASM_EINVAL, "dgasm_partition: NULL argument");
  if (ncoarse > 0 && !agg_of_elem) return set_error(DGASM_EINVAL, "dgasm_partition: agg_of_elem is NULL");
  std::vector<int> sub, agg;
  DG_TRY(compute_partition(h->m, nsub, ncoarse, sub, ncoarse > 0 ? &agg : nullptr));
  std::copy(sub.begin(), sub.end(), sub_of_elem);
  if (ncoarse > 0) std::copy(agg.begin(), agg.end(), agg_of_elem);
  return DGASM_OK;
}
