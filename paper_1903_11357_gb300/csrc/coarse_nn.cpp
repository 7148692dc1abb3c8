// R_0^T for a coarse mesh that is not an agglomeration of the fine mesh (Eq. R0T; the non-nested coarse
// spaces of Example 4).  R_0^T v_0 is the L2 projection of the piecewise polynomial v_0 onto V_h, so on a
// fine element kappa
//     R_0^T|_kappa = M_kappa^{-1} [N_kappa,j]_j,   N_kappa,j = int_{kappa cap D_j} phi psi_j^T,
// over every coarse element D_j that overlaps kappa.  The cells are convex (clipped Voronoi cells), so each
// piece kappa cap D_j is a convex polygon: Sutherland-Hodgman clipping of kappa against the half-planes of
// D_j's edges.  Pieces are integrated with the element rule (fan from the vertex average, Duffy-collapsed
// (p+2)-point Gauss rule per triangle: exact for the degree p + q <= 2p integrands); pieces smaller than
// 1e-12 |kappa| are dropped.  Candidates come from a uniform grid over the coarse cells' bounding boxes.
// Host C++ like the SIPG assembly; elements are split over threads and each element's pairs are computed
// by one thread in ascending coarse order, so the result does not depend on the thread count.
#include <algorithm>
#include <cmath>
#include <thread>

#include "basis.h"
#include "common.h"
#include "plan.h"

namespace dgasm {

namespace {

constexpr double MIN_REL_AREA = 1e-12;

struct Poly {
  std::vector<double> xy;   // 2 n
  int n() const { return (int)xy.size() / 2; }
};

Poly cell(const MeshData& m, int e) {
  Poly p;
  for (int k = m.ptr[e]; k < m.ptr[e + 1]; ++k) {
    p.xy.push_back(m.xy[2 * (size_t)m.vtx[k]]);
    p.xy.push_back(m.xy[2 * (size_t)m.vtx[k] + 1]);
  }
  return p;
}

double area(const Poly& p) {
  double s = 0.0;
  const int n = p.n();
  for (int k = 0; k < n; ++k) {
    const int l = (k + 1) % n;
    s += p.xy[2 * k] * p.xy[2 * l + 1] - p.xy[2 * l] * p.xy[2 * k + 1];
  }
  return 0.5 * s;
}

// the part of `s` left of every edge of the convex counter-clockwise polygon `c`
Poly clip(const Poly& s, const Poly& c) {
  Poly out = s, in;
  const int nc = c.n();
  for (int i = 0; i < nc && out.n() > 0; ++i) {
    const double ax = c.xy[2 * i], ay = c.xy[2 * i + 1];
    const double bx = c.xy[2 * ((i + 1) % nc)], by = c.xy[2 * ((i + 1) % nc) + 1];
    auto side = [&](double x, double y) { return (bx - ax) * (y - ay) - (by - ay) * (x - ax); };
    in = out;
    out.xy.clear();
    const int n = in.n();
    for (int k = 0; k < n; ++k) {
      const int j = (k + n - 1) % n;
      const double cx = in.xy[2 * k], cy = in.xy[2 * k + 1], px = in.xy[2 * j], py = in.xy[2 * j + 1];
      const double sc = side(cx, cy), sp = side(px, py);
      if (sc >= 0.0) {
        if (sp < 0.0) {
          const double t = sp / (sp - sc);
          out.xy.push_back(px + (cx - px) * t);
          out.xy.push_back(py + (cy - py) * t);
        }
        out.xy.push_back(cx);
        out.xy.push_back(cy);
      } else if (sp >= 0.0) {
        const double t = sp / (sp - sc);
        out.xy.push_back(px + (cx - px) * t);
        out.xy.push_back(py + (cy - py) * t);
      }
    }
  }
  return out;
}

// fan-of-triangles rule on a convex polygon
void poly_rule(const Poly& p, const std::vector<double>& t, const std::vector<double>& w, std::vector<double>& pts,
               std::vector<double>& wts) {
  const int n = p.n(), q = (int)t.size();
  double cx = 0, cy = 0;
  for (int k = 0; k < n; ++k) { cx += p.xy[2 * k]; cy += p.xy[2 * k + 1]; }
  cx /= n;
  cy /= n;
  pts.clear();
  wts.clear();
  for (int k = 0; k < n; ++k) {
    const int l = (k + 1) % n;
    const double e1x = p.xy[2 * k] - cx, e1y = p.xy[2 * k + 1] - cy;
    const double e2x = p.xy[2 * l] - p.xy[2 * k], e2y = p.xy[2 * l + 1] - p.xy[2 * k + 1];
    const double jac = std::fabs(e1x * e2y - e1y * e2x);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        const double u = t[i], v = t[j];
        pts.push_back(cx + u * e1x + u * v * e2x);
        pts.push_back(cy + u * e1y + u * v * e2y);
        wts.push_back(w[i] * w[j] * u * jac);
      }
  }
}

// the pairs of one fine element: coarse cells (ascending) and blocks [np][nq]
void element_pairs(const MeshData& f, int e, const MeshData& c, const std::vector<std::vector<int>>& bins, int G,
                   const double* gb, const Basis& Bp, const Basis& Bq, const std::vector<double>& gt,
                   const std::vector<double>& gw, std::vector<int>& cj, std::vector<double>& blk) {
  const int np = Bp.nb, nq = Bq.nb;
  const double* fb = &f.bbox[4 * (size_t)e];
  // candidates: coarse cells registered in the bins under this element's box, boxes overlapping
  auto bin = [&](double v, double lo, double hi) {
    int k = (int)std::floor((v - lo) / (hi - lo) * G);
    return std::min(std::max(k, 0), G - 1);
  };
  const int i0 = bin(fb[0], gb[0], gb[1]), i1 = bin(fb[1], gb[0], gb[1]);
  const int j0 = bin(fb[2], gb[2], gb[3]), j1 = bin(fb[3], gb[2], gb[3]);
  std::vector<int> cand;
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) cand.insert(cand.end(), bins[(size_t)j * G + i].begin(), bins[(size_t)j * G + i].end());
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  const Poly pe = cell(f, e);
  const double ae = area(pe);
  std::vector<double> pts, wts, v(np), u(nq), cf(np), cc(nq), wv(np);
  Bp.coefs(fb, cf.data());
  // M_kappa and its Cholesky factor
  poly_rule(pe, gt, gw, pts, wts);
  std::vector<double> M((size_t)np * np, 0.0);
  for (size_t k = 0; k < wts.size(); ++k) {
    Bp.values(fb, cf.data(), pts[2 * k], pts[2 * k + 1], v.data());
    double* __restrict Mp = M.data();
    const double* __restrict vp = v.data();
    const double wk = wts[k];
    for (int a = 0; a < np; ++a) {
      const double wa = wk * vp[a];
      for (int b = 0; b <= a; ++b) Mp[(size_t)a * np + b] += wa * vp[b];
    }
  }
  for (int j = 0; j < np; ++j) {   // in-place lower Cholesky
    double d = M[(size_t)j * np + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * np + k] * M[(size_t)j * np + k];
    d = std::sqrt(d);
    M[(size_t)j * np + j] = d;
    for (int i = j + 1; i < np; ++i) {
      double s = M[(size_t)i * np + j];
      for (int k = 0; k < j; ++k) s -= M[(size_t)i * np + k] * M[(size_t)j * np + k];
      M[(size_t)i * np + j] = s / d;
    }
  }
  std::vector<double> N((size_t)np * nq);
  for (int J : cand) {
    const double* cb = &c.bbox[4 * (size_t)J];
    if (!(cb[0] < fb[1] && cb[1] > fb[0] && cb[2] < fb[3] && cb[3] > fb[2])) continue;
    const Poly piece = clip(pe, cell(c, J));
    if (piece.n() < 3 || area(piece) <= MIN_REL_AREA * ae) continue;
    poly_rule(piece, gt, gw, pts, wts);
    std::fill(N.begin(), N.end(), 0.0);
    Bq.coefs(cb, cc.data());
    for (size_t k = 0; k < wts.size(); ++k) {
      Bp.values(fb, cf.data(), pts[2 * k], pts[2 * k + 1], v.data());
      Bq.values(cb, cc.data(), pts[2 * k], pts[2 * k + 1], u.data());
      double* __restrict Np = N.data();
      const double* __restrict up = u.data();
      const double wk = wts[k];
      for (int a = 0; a < np; ++a) {
        const double wa = wk * v[a];
        for (int b = 0; b < nq; ++b) Np[(size_t)a * nq + b] += wa * up[b];
      }
    }
    // M^{-1} N by the two triangular solves, column by column
    for (int b = 0; b < nq; ++b) {
      for (int a = 0; a < np; ++a) {
        double s = N[(size_t)a * nq + b];
        for (int k = 0; k < a; ++k) s -= M[(size_t)a * np + k] * N[(size_t)k * nq + b];
        N[(size_t)a * nq + b] = s / M[(size_t)a * np + a];
      }
      for (int a = np - 1; a >= 0; --a) {
        double s = N[(size_t)a * nq + b];
        for (int k = a + 1; k < np; ++k) s -= M[(size_t)k * np + a] * N[(size_t)k * nq + b];
        N[(size_t)a * nq + b] = s / M[(size_t)a * np + a];
      }
    }
    cj.push_back(J);
    blk.insert(blk.end(), N.begin(), N.end());
  }
}

}  // namespace

int nonnested_r0t(const MeshData& f, const std::vector<int>& perm, const MeshData& c, int p, int q, R0TPairs& out) {
  const int ne = f.ne, nc = c.ne;
  // the clipping needs convex (counter-clockwise) coarse cells: every turn left or straight
  for (int J = 0; J < nc; ++J) {
    const Poly cj = cell(c, J);
    const int n = cj.n();
    double scale = 0.0;
    for (int k = 0; k < n; ++k) scale = std::max(scale, std::fabs(cj.xy[2 * k]) + std::fabs(cj.xy[2 * k + 1]));
    for (int k = 0; k < n; ++k) {
      const int a = k, b = (k + 1) % n, d = (k + 2) % n;
      const double cr = (cj.xy[2 * b] - cj.xy[2 * a]) * (cj.xy[2 * d + 1] - cj.xy[2 * b + 1]) -
                        (cj.xy[2 * b + 1] - cj.xy[2 * a + 1]) * (cj.xy[2 * d] - cj.xy[2 * b]);
      if (cr < -1e-12 * scale * scale) return set_error(DGASM_EINVAL, "coarse cell %d is not convex", J);
    }
  }
  const Basis Bp(p), Bq(q);
  std::vector<double> gt, gw;
  gauss_legendre01(p + 2, gt, gw);
  // uniform grid over both meshes' boxes, each coarse cell in every bin its box touches
  double gb[4] = {1e300, -1e300, 1e300, -1e300};
  for (const MeshData* m : {&f, &c})
    for (int e = 0; e < m->ne; ++e) {
      gb[0] = std::min(gb[0], m->bbox[4 * (size_t)e]);
      gb[1] = std::max(gb[1], m->bbox[4 * (size_t)e + 1]);
      gb[2] = std::min(gb[2], m->bbox[4 * (size_t)e + 2]);
      gb[3] = std::max(gb[3], m->bbox[4 * (size_t)e + 3]);
    }
  const int G = std::max(1, (int)std::ceil(std::sqrt((double)nc)));
  std::vector<std::vector<int>> bins((size_t)G * G);
  auto bin = [&](double v, double lo, double hi) {
    int k = (int)std::floor((v - lo) / (hi - lo) * G);
    return std::min(std::max(k, 0), G - 1);
  };
  for (int J = 0; J < nc; ++J) {
    const double* b = &c.bbox[4 * (size_t)J];
    for (int j = bin(b[2], gb[2], gb[3]); j <= bin(b[3], gb[2], gb[3]); ++j)
      for (int i = bin(b[0], gb[0], gb[1]); i <= bin(b[1], gb[0], gb[1]); ++i) bins[(size_t)j * G + i].push_back(J);
  }
  // pairs per internal element, in parallel
  std::vector<std::vector<int>> cj(ne);
  std::vector<std::vector<double>> blk(ne);
  const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int i = (int)t; i < ne; i += (int)nt) element_pairs(f, perm[i], c, bins, G, gb, Bp, Bq, gt, gw, cj[i], blk[i]);
    });
  for (auto& x : th) x.join();
  out.ptr.assign(ne + 1, 0);
  out.col.clear();
  out.elem.clear();
  out.blocks.clear();
  for (int i = 0; i < ne; ++i) {
    if (cj[i].empty()) return set_error(DGASM_EINVAL, "fine element %d overlaps no coarse cell", perm[i]);
    out.col.insert(out.col.end(), cj[i].begin(), cj[i].end());
    out.elem.insert(out.elem.end(), cj[i].size(), i);
    out.blocks.insert(out.blocks.end(), blk[i].begin(), blk[i].end());
    out.ptr[i + 1] = (int)out.col.size();
  }
  // transpose: the pairs of each coarse cell, ascending
  out.tptr.assign(nc + 1, 0);
  for (int J : out.col) out.tptr[J + 1]++;
  for (int J = 0; J < nc; ++J) out.tptr[J + 1] += out.tptr[J];
  out.tpair.assign(out.col.size(), 0);
  std::vector<int> fill(out.tptr.begin(), out.tptr.end() - 1);
  for (int t = 0; t < (int)out.col.size(); ++t) out.tpair[fill[out.col[t]]++] = t;
  for (int J = 0; J < nc; ++J)
    if (out.tptr[J + 1] == out.tptr[J]) return set_error(DGASM_EINVAL, "coarse cell %d overlaps no fine element", J);
  return DGASM_OK;
}

}  // namespace dgasm

// Host query of the non-nested R_0^T blocks in the caller's element order (no device work)
extern "C" int dgasm_nonnested_prolongation(dgasm_mesh_t fine, dgasm_mesh_t coarse, int p, int q, int64_t* npair,
                                            int* ptr, int* col, double* blocks) {
  using namespace dgasm;
  clear_error();
  if (!fine || !coarse || !npair) return set_error(DGASM_EINVAL, "dgasm_nonnested_prolongation: NULL argument");
  if (p < 1 || p > 8 || q < 1 || q > p) return set_error(DGASM_EINVAL, "need 1 <= q <= p <= 8 (p=%d, q=%d)", p, q);
  std::vector<int> perm(fine->m.ne);
  for (int i = 0; i < fine->m.ne; ++i) perm[i] = i;
  R0TPairs out;
  DG_TRY(nonnested_r0t(fine->m, perm, coarse->m, p, q, out));
  *npair = (int64_t)out.col.size();
  if (ptr) std::copy(out.ptr.begin(), out.ptr.end(), ptr);
  if (col) std::copy(out.col.begin(), out.col.end(), col);
  if (blocks) std::copy(out.blocks.begin(), out.blocks.end(), blocks);
  return DGASM_OK;
}
