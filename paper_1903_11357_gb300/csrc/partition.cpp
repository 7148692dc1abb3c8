// Subdomain and coarse-agglomerate partitions (Sec. 3: T_H by agglomeration of fine elements) by
// recursive coordinate bisection of element area centroids.
#include <algorithm>
#include <numeric>
#include <utility>

#include "common.h"
#include "plan.h"

namespace dgasm {

static void rcb_rec(const double* cx, const double* cy, std::vector<int>& elems, size_t lo, size_t hi, int k,
                    std::vector<int>& part_of, int& next_part, std::vector<std::pair<double, int>>& keys) {
  if (k <= 1) {
    for (size_t i = lo; i < hi; ++i) part_of[elems[i]] = next_part;
    ++next_part;
    return;
  }
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (size_t i = lo; i < hi; ++i) {
    int e = elems[i];
    xmin = std::min(xmin, cx[e]); xmax = std::max(xmax, cx[e]);
    ymin = std::min(ymin, cy[e]); ymax = std::max(ymax, cy[e]);
  }
  const double* c = (xmax - xmin >= ymax - ymin) ? cx : cy;
  int kl = k / 2;
  size_t n = hi - lo;
  size_t nl = (n * (size_t)kl) / (size_t)k;
  // the first nl elements in the (coordinate, element id) order: a strict total order, so selecting them
  // with nth_element gives exactly the set a full sort would (the keys sit side by side for the selection)
  if (nl > 0 && nl < n) {
    keys.resize(n);
    for (size_t i = 0; i < n; ++i) keys[i] = {c[elems[lo + i]], elems[lo + i]};
    std::nth_element(keys.begin(), keys.begin() + nl, keys.end());
    for (size_t i = 0; i < n; ++i) elems[lo + i] = keys[i].second;
  }
  rcb_rec(cx, cy, elems, lo, lo + nl, kl, part_of, next_part, keys);
  rcb_rec(cx, cy, elems, lo + nl, hi, k - kl, part_of, next_part, keys);
}

void rcb_parts(const MeshData& m, std::vector<int> elems, int k, std::vector<int>& part_of, int first_part) {
  int next = first_part;
  std::vector<std::pair<double, int>> keys;
  rcb_rec(m.cx.data(), m.cy.data(), elems, 0, elems.size(), k, part_of, next, keys);
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
      int next = 0;
      for (int i = 0; i < nsub; ++i) {
        int ci = (int)(((long long)(i + 1) * ncoarse) / nsub - ((long long)i * ncoarse) / nsub);
        if (ci < 1 || (size_t)ci > members[i].size())
          return set_error(DGASM_EINVAL, "subdomain %d cannot hold %d agglomerates", i, ci);
        rcb_parts(m, members[i], ci, *agg, next);
        next += ci;
      }
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
