// R_0^T for a coarse mesh that is not an agglomeration of the fine mesh (Eq. R0T; the non-nested coarse
// spaces of Example 4).  R_0^T v_0 is the L2 projection of the piecewise polynomial v_0 onto V_h, so on a
// fine element kappa
//     R_0^T|_kappa = M_kappa^{-1} [N_kappa,j]_j,   N_kappa,j = int_{kappa cap D_j} phi psi_j^T,
// over every coarse element D_j that overlaps kappa.  The cells are convex (clipped Voronoi cells), so each
// piece kappa cap D_j is a convex polygon: Sutherland-Hodgman clipping of kappa against the half-planes of
// D_j's edges.  Integrals use a fan of triangles from the vertex average with a Duffy-collapsed m-point
// Gauss rule per triangle, exact for total degree 2m - 2: m = p + 1 for M_kappa (degree 2p) and
// m = ceil((p + q + 2) / 2) on the pieces (degree p + q); pieces smaller than 1e-12 |kappa| are dropped.  Candidates come from a uniform grid over the coarse cells' bounding boxes.
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

// C[a][b] = sum_k (w_k A[k][a]) B[k][b] for a < na and b < nb (A is [n][na], B is [n][nb], C is [na][nb]), each
// entry summed over k in ascending order.  lower: only b <= a is needed (entries above it may be written too).
// Columns go in blocks of 8 whose partial sums stay in registers; WA (na * n doubles) holds w_k A[k][a].
void weighted_products(int n, const double* w, const double* A, int na, const double* B, int nb, double* C, bool lower,
                       double* WA) {
  for (int k = 0; k < n; ++k)
    for (int a = 0; a < na; ++a) WA[(size_t)a * n + k] = w[k] * A[(size_t)k * na + a];
  for (int a = 0; a < na; ++a) {
    const double* wa = WA + (size_t)a * n;
    const int ncol = lower ? std::min(nb, a + 1) : nb;
    for (int b0 = 0; b0 < ncol; b0 += 8) {
      double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const int r = std::min(8, nb - b0);
      if (r == 8) {
        for (int k = 0; k < n; ++k) {
          const double* bk = B + (size_t)k * nb + b0;
          for (int j = 0; j < 8; ++j) s[j] += wa[k] * bk[j];
        }
      } else {
        for (int k = 0; k < n; ++k) {
          const double* bk = B + (size_t)k * nb + b0;
          for (int j = 0; j < r; ++j) s[j] += wa[k] * bk[j];
        }
      }
      for (int j = 0; j < r; ++j) C[(size_t)a * nb + b0 + j] = s[j];
    }
  }
}

// per-thread work arrays, reused from element to element
struct Scratch {
  std::vector<double> pts, wts, V, U, L, M, N, WA;
  std::vector<int> cand;
};

// the integration rules: m points per direction for M_kappa (degree 2p) and for the pieces (degree p + q)
struct Rules {
  std::vector<double> tM, wM, tN, wN;
};

// the pairs of one fine element: coarse cells (ascending) and blocks [np][nq]
void element_pairs(const MeshData& f, int e, const MeshData& c, const std::vector<std::vector<int>>& bins, int G,
                   const double* gb, const Basis& Bp, const Basis& Bq, const Rules& R, Scratch& W,
                   std::vector<int>& cj, std::vector<double>& blk) {
  const int np = Bp.nb, nq = Bq.nb;
  const double* fb = &f.bbox[4 * (size_t)e];
  // candidates: coarse cells registered in the bins under this element's box, boxes overlapping
  auto bin = [&](double v, double lo, double hi) {
    int k = (int)std::floor((v - lo) / (hi - lo) * G);
    return std::min(std::max(k, 0), G - 1);
  };
  const int i0 = bin(fb[0], gb[0], gb[1]), i1 = bin(fb[1], gb[0], gb[1]);
  const int j0 = bin(fb[2], gb[2], gb[3]), j1 = bin(fb[3], gb[2], gb[3]);
  std::vector<int>& cand = W.cand;
  cand.clear();
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) cand.insert(cand.end(), bins[(size_t)j * G + i].begin(), bins[(size_t)j * G + i].end());
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  const Poly pe = cell(f, e);
  const double ae = area(pe);
  double cf[64], cc[64];
  Bp.coefs(fb, cf);
  auto values = [&](const Basis& B, const double* box, const double* coef, std::vector<double>& out) {
    const int n = (int)W.wts.size();
    out.resize((size_t)n * B.nb);
    W.L.resize((size_t)2 * (B.p + 1) * n);
    B.values_at(box, coef, W.pts.data(), n, out.data(), W.L.data());
  };
  // M_kappa and its Cholesky factor
  poly_rule(pe, R.tM, R.wM, W.pts, W.wts);
  values(Bp, fb, cf, W.V);
  std::vector<double>& M = W.M;
  M.resize((size_t)np * np);
  W.WA.resize((size_t)np * W.wts.size());
  weighted_products((int)W.wts.size(), W.wts.data(), W.V.data(), np, W.V.data(), np, M.data(), true, W.WA.data());
  for (int j = 0; j < np; ++j) {   // in-place lower Cholesky of the lower triangle
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
  std::vector<double>& N = W.N;
  N.resize((size_t)np * nq);
  for (int J : cand) {
    const double* cb = &c.bbox[4 * (size_t)J];
    if (!(cb[0] < fb[1] && cb[1] > fb[0] && cb[2] < fb[3] && cb[3] > fb[2])) continue;
    const Poly piece = clip(pe, cell(c, J));
    if (piece.n() < 3 || area(piece) <= MIN_REL_AREA * ae) continue;
    poly_rule(piece, R.tN, R.wN, W.pts, W.wts);
    Bq.coefs(cb, cc);
    values(Bp, fb, cf, W.V);
    values(Bq, cb, cc, W.U);
    W.WA.resize((size_t)np * W.wts.size());
    weighted_products((int)W.wts.size(), W.wts.data(), W.V.data(), np, W.U.data(), nq, N.data(), false, W.WA.data());
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
  // an m-point collapsed rule integrates total degree 2m - 2 exactly
  Rules R;
  gauss_legendre01(p + 1, R.tM, R.wM);
  gauss_legendre01((p + q + 3) / 2, R.tN, R.wN);
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
      Scratch W;
      for (int i = (int)t; i < ne; i += (int)nt) element_pairs(f, perm[i], c, bins, G, gb, Bp, Bq, R, W, cj[i], blk[i]);
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
