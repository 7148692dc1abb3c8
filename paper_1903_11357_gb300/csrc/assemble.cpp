// SIPG assembly on the host (Sec. 2, Eq. Ah with the lifting of Eq. lifting, penalty of Eq. Sigma).
//
// The lifted form equals the weighted interior-penalty form because rho grad_h u is an admissible
// test field of the lifting (rho is constant per element), and with omega = rho^-/(rho^+ + rho^-)
// the weighted average {rho grad u}_omega equals <rho>/2 (grad u^+ + grad u^-), <.> the harmonic
// average.  Element integrals use a fan of triangles from the vertex average, each with a
// Duffy-collapsed (p+2)-point tensor Gauss rule (exact for the degree-2p integrands); faces use a
// (p+2)-point Gauss rule.  Each element's block row is computed by one thread, visiting its faces
// in ascending face order, so the result does not depend on the thread count.
#include <algorithm>
#include <cmath>
#include <memory>
#include <thread>

#include <cuda_runtime.h>

#include "basis.h"
#include "common.h"
#include "engine.h"

using namespace dgasm;

namespace {

// quadrature points/weights of polygon e: fan from the vertex average, Duffy rule per triangle
void polygon_points(const MeshData& m, int e, const std::vector<double>& t, const std::vector<double>& w,
                    std::vector<double>& pts, std::vector<double>& wts) {
  int b = m.ptr[e], n = m.ptr[e + 1] - b, q = (int)t.size();
  double cx = 0, cy = 0;
  for (int k = 0; k < n; ++k) { cx += m.xy[2 * (size_t)m.vtx[b + k]]; cy += m.xy[2 * (size_t)m.vtx[b + k] + 1]; }
  cx /= n; cy /= n;
  pts.clear(); wts.clear();
  for (int k = 0; k < n; ++k) {
    const double* B = &m.xy[2 * (size_t)m.vtx[b + k]];
    const double* C = &m.xy[2 * (size_t)m.vtx[b + (k + 1) % n]];
    double e1x = B[0] - cx, e1y = B[1] - cy, e2x = C[0] - B[0], e2y = C[1] - B[1];
    double jac = std::fabs(e1x * e2y - e1y * e2x);
    for (int i = 0; i < q; ++i)
      for (int j = 0; j < q; ++j) {
        double u = t[i], v = t[j];
        pts.push_back(cx + u * e1x + u * v * e2x);
        pts.push_back(cy + u * e1y + u * v * e2y);
        wts.push_back(w[i] * w[j] * u * jac);
      }
  }
}

void assemble_rows(const MeshData& m, const Basis& B, double c_sigma, const std::vector<int>& rowptr,
                   const std::vector<int>& col, std::vector<double>& vals, int e_begin, int e_end) {
  const int nb = B.nb, p = B.p, mq = p + 2;
  std::vector<double> t, w;
  gauss_legendre01(mq, t, w);
  std::vector<double> pts, wts;
  std::vector<double> v(nb), g(2 * nb), va(nb), ga(2 * nb), vb(nb), gb(2 * nb), dna(nb), dnb(nb);
  for (int e = e_begin; e < e_end; ++e) {
    const double* box = &m.bbox[4 * (size_t)e];
    int r0 = rowptr[e], r1 = rowptr[e + 1];
    auto block_of = [&](int c) -> double* {
      int k = (int)(std::lower_bound(col.begin() + r0, col.begin() + r1, c) - col.begin());
      return &vals[(size_t)k * nb * nb];
    };
    double* D = block_of(e);
    // element term rho_kappa int grad phi_a . grad phi_b
    polygon_points(m, e, t, w, pts, wts);
    for (size_t qp = 0; qp < wts.size(); ++qp) {
      B.eval(box, pts[2 * qp], pts[2 * qp + 1], v.data(), g.data());
      double wr = wts[qp] * m.rho[e];
      for (int a = 0; a < nb; ++a)
        for (int c = 0; c < nb; ++c)
          D[a * nb + c] += wr * (g[2 * a] * g[2 * c] + g[2 * a + 1] * g[2 * c + 1]);
    }
    // faces of e in ascending face order
    for (int fi = m.ef_ptr[e]; fi < m.ef_ptr[e + 1]; ++fi) {
      int f = m.ef_face[fi];
      int ep = m.f_ep[f], em = m.f_em[f];
      const double* P = &m.xy[2 * (size_t)m.f_va[f]];
      const double* Q = &m.xy[2 * (size_t)m.f_vb[f]];
      double dx = Q[0] - P[0], dy = Q[1] - P[1], len = std::hypot(dx, dy);
      double nx = dy / len, ny = -dx / len;  // outward normal of e_plus
      if (em < 0) {
        double sigma = c_sigma * m.rho[e] * p * p / m.diam[e];
        double rho = m.rho[e];
        for (int qp = 0; qp < mq; ++qp) {
          double x = P[0] + t[qp] * dx, y = P[1] + t[qp] * dy, wq = w[qp] * len;
          B.eval(box, x, y, v.data(), g.data());
          for (int a = 0; a < nb; ++a) dna[a] = g[2 * a] * nx + g[2 * a + 1] * ny;
          for (int a = 0; a < nb; ++a)
            for (int c = 0; c < nb; ++c)
              D[a * nb + c] += wq * (-rho * v[a] * dna[c] - rho * v[c] * dna[a] + sigma * v[a] * v[c]);
        }
        continue;
      }
      int other = (e == ep) ? em : ep;
      double sa = (e == ep) ? 1.0 : -1.0, sb = -sa;
      double rh = 2.0 * m.rho[ep] * m.rho[em] / (m.rho[ep] + m.rho[em]);
      double hh = 2.0 * m.diam[ep] * m.diam[em] / (m.diam[ep] + m.diam[em]);
      double sigma = c_sigma * rh * p * p / hh;
      const double* boxo = &m.bbox[4 * (size_t)other];
      double* O = block_of(other);
      for (int qp = 0; qp < mq; ++qp) {
        double x = P[0] + t[qp] * dx, y = P[1] + t[qp] * dy, wq = w[qp] * len;
        B.eval(box, x, y, va.data(), ga.data());
        B.eval(boxo, x, y, vb.data(), gb.data());
        for (int a = 0; a < nb; ++a) {
          dna[a] = ga[2 * a] * nx + ga[2 * a + 1] * ny;
          dnb[a] = gb[2 * a] * nx + gb[2 * a + 1] * ny;
        }
        // self block: test and trial on e (s_a s_a = 1)
        for (int a = 0; a < nb; ++a)
          for (int c = 0; c < nb; ++c)
            D[a * nb + c] += wq * (-0.5 * rh * sa * va[a] * dna[c] - 0.5 * rh * sa * va[c] * dna[a] + sigma * va[a] * va[c]);
        // cross block: test on e (s_a), trial on the neighbour (s_b)
        for (int a = 0; a < nb; ++a)
          for (int c = 0; c < nb; ++c)
            O[a * nb + c] += wq * (-0.5 * rh * sa * va[a] * dnb[c] - 0.5 * rh * sb * vb[c] * dna[a] + sigma * sa * sb * va[a] * vb[c]);
      }
    }
  }
}

}  // namespace

namespace {

// a fresh system with the block sparsity: each element and its face neighbours, ascending
dgasm_system_s* new_system(dgasm_mesh_t mh, int p, double c_sigma) {
  const MeshData& m = mh->m;
  auto* s = new (std::nothrow) dgasm_system_s();
  if (!s) return nullptr;
  s->mesh = mh;
  s->p = p;
  s->np = n_basis(p);
  s->np2s = (s->np * s->np + 1) & ~1;
  s->c_sigma = c_sigma;
  const int ne = m.ne;
  s->rowptr.assign(ne + 1, 0);
  std::vector<std::vector<int>> nbr(ne);
  for (int e = 0; e < ne; ++e) {
    nbr[e].push_back(e);
    for (int fi = m.ef_ptr[e]; fi < m.ef_ptr[e + 1]; ++fi) {
      int f = m.ef_face[fi];
      if (m.f_em[f] < 0) continue;
      nbr[e].push_back(m.f_ep[f] == e ? m.f_em[f] : m.f_ep[f]);
    }
    std::sort(nbr[e].begin(), nbr[e].end());
    nbr[e].erase(std::unique(nbr[e].begin(), nbr[e].end()), nbr[e].end());
    s->rowptr[e + 1] = s->rowptr[e] + (int)nbr[e].size();
  }
  s->col.resize(s->rowptr[ne]);
  for (int e = 0; e < ne; ++e) std::copy(nbr[e].begin(), nbr[e].end(), s->col.begin() + s->rowptr[e]);
  return s;
}

// load vector b_a = int f phi_a, (p+5)-point rule, callback on this thread in chunks
void assemble_rhs(const MeshData& m, const Basis& B, dgasm_rhs_fn f, void* user, dgasm_system_s* s) {
  const int ne = m.ne, nb = B.nb, p = B.p;
  s->b.assign((size_t)ne * nb, 0.0);
  s->has_b = true;
  std::vector<double> t, w, pts, wts, allp, fv, v(nb);
  gauss_legendre01(p + 5, t, w);
  const int chunk = 256;
  for (int c0 = 0; c0 < ne; c0 += chunk) {
    int c1 = std::min(ne, c0 + chunk);
    std::vector<size_t> off(1, 0);
    allp.clear();
    std::vector<double> allw;
    for (int e = c0; e < c1; ++e) {
      polygon_points(m, e, t, w, pts, wts);
      allp.insert(allp.end(), pts.begin(), pts.end());
      allw.insert(allw.end(), wts.begin(), wts.end());
      off.push_back(allw.size());
    }
    fv.assign(allw.size(), 0.0);
    f((int)allw.size(), allp.data(), fv.data(), user);
    for (int e = c0; e < c1; ++e) {
      double* be = &s->b[(size_t)e * nb];
      for (size_t qp = off[e - c0]; qp < off[e - c0 + 1]; ++qp) {
        B.eval(&m.bbox[4 * (size_t)e], allp[2 * qp], allp[2 * qp + 1], v.data(), nullptr);
        for (int a = 0; a < nb; ++a) be[a] += allw[qp] * fv[qp] * v[a];
      }
    }
  }
}

int check_args(const char* fn, dgasm_mesh_t mh, int p, double c_sigma, dgasm_system_t* out) {
  if (!out) return set_error(DGASM_EINVAL, "%s: out is NULL", fn);
  *out = nullptr;
  if (!mh) return set_error(DGASM_EINVAL, "%s: NULL mesh", fn);
  if (p < 1 || p > 8) return set_error(DGASM_EINVAL, "p=%d must lie in [1, 8]", p);
  if (!(c_sigma > 0.0)) return set_error(DGASM_EINVAL, "c_sigma must be positive");
  return DGASM_OK;
}

}  // namespace

extern "C" int dgasm_assemble(dgasm_mesh_t mh, int p, double c_sigma, dgasm_rhs_fn f, void* user,
                              dgasm_system_t* out) {
  clear_error();
  DG_TRY(check_args("dgasm_assemble", mh, p, c_sigma, out));
  const MeshData& m = mh->m;
  dgasm_system_s* s = new_system(mh, p, c_sigma);
  if (!s) return set_error(DGASM_ENOMEM, "host allocation failed");
  const int ne = m.ne, nb = s->np;
  s->vals.assign((size_t)s->rowptr[ne] * nb * nb, 0.0);
  Basis B(p);
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (ne < 256) nt = 1;
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nt; ++k) {
    int e0 = (int)((long long)ne * k / nt), e1 = (int)((long long)ne * (k + 1) / nt);
    th.emplace_back([&, e0, e1]() { assemble_rows(m, B, c_sigma, s->rowptr, s->col, s->vals, e0, e1); });
  }
  for (auto& x : th) x.join();
  if (f) assemble_rhs(m, B, f, user, s);
  *out = s;
  return DGASM_OK;
}

// The same system with the matrix assembled on the device, straight into the device block layout; the
// load vector (a host callback) stays on the host.  The host copy of the blocks is made on demand.
extern "C" int dgasm_assemble_device(dgasm_mesh_t mh, int p, double c_sigma, dgasm_rhs_fn f, void* user, void* stream,
                                     dgasm_system_t* out) {
  clear_error();
  DG_TRY(check_args("dgasm_assemble_device", mh, p, c_sigma, out));
  const MeshData& m = mh->m;
  std::unique_ptr<dgasm_system_s> s(new_system(mh, p, c_sigma));
  if (!s) return set_error(DGASM_ENOMEM, "host allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf rho, diam, efp, eff, fep, fem, fva, fvb, gt, gw;
  std::vector<double> t, w;
  gauss_legendre01(p + 2, t, w);
  DG_TRY(upload(s->d_rowptr, s->rowptr));
  DG_TRY(upload(s->d_col, s->col));
  DG_TRY(upload(s->d_xy, m.xy));
  DG_TRY(upload(s->d_pptr, m.ptr));
  DG_TRY(upload(s->d_pvtx, m.vtx));
  DG_TRY(upload(s->d_bbox, m.bbox));
  DG_TRY(upload(rho, m.rho));
  DG_TRY(upload(diam, m.diam));
  DG_TRY(upload(efp, m.ef_ptr));
  DG_TRY(upload(eff, m.ef_face));
  DG_TRY(upload(fep, m.f_ep));
  DG_TRY(upload(fem, m.f_em));
  DG_TRY(upload(fva, m.f_va));
  DG_TRY(upload(fvb, m.f_vb));
  DG_TRY(upload(gt, t));
  DG_TRY(upload(gw, w));
  DevBuf vals;
  DG_TRY(vals.alloc(sizeof(double) * (size_t)s->rowptr[m.ne] * s->np2s));
  DG_CUDA(cudaMemsetAsync(vals.ptr, 0, vals.bytes, st));
  AsmMesh A{m.ne, s->d_xy.as<double>(), s->d_pptr.as<int>(), s->d_pvtx.as<int>(), s->d_bbox.as<double>(),
            rho.as<double>(), diam.as<double>(), efp.as<int>(), eff.as<int>(), fep.as<int>(), fem.as<int>(),
            fva.as<int>(), fvb.as<int>()};
  DG_CUDA(launch_assemble(A, p, c_sigma, gt.as<double>(), gw.as<double>(), s->d_rowptr.as<int>(), s->d_col.as<int>(),
                          s->np2s, vals.as<double>(), st));
  if (f) assemble_rhs(m, Basis(p), f, user, s.get());   // overlaps the kernel
  DG_CUDA(cudaStreamSynchronize(st));
  s->d_vals = std::move(vals);
  DG_CUDA(cudaGetDevice(&s->dev));
  *out = s.release();
  return DGASM_OK;
}

extern "C" int dgasm_system_dofs(dgasm_system_t s, int64_t* ndof, int* np) {
  if (!s) return set_error(DGASM_EINVAL, "NULL system");
  if (ndof) *ndof = (int64_t)s->mesh->m.ne * s->np;
  if (np) *np = s->np;
  return DGASM_OK;
}

extern "C" int dgasm_system_rhs(dgasm_system_t s, double* b) {
  if (!s || !b) return set_error(DGASM_EINVAL, "NULL argument");
  if (!s->has_b) return set_error(DGASM_EINVAL, "system was assembled without a right-hand side");
  std::copy(s->b.begin(), s->b.end(), b);
  return DGASM_OK;
}

extern "C" int dgasm_system_blocks(dgasm_system_t s, int64_t* nnzb, int* rowptr, int* col, double* vals) {
  if (!s || !nnzb) return set_error(DGASM_EINVAL, "NULL argument");
  *nnzb = (int64_t)s->col.size();
  if (rowptr) std::copy(s->rowptr.begin(), s->rowptr.end(), rowptr);
  if (col) std::copy(s->col.begin(), s->col.end(), col);
  if (vals) {
    DG_TRY(s->ensure_host());
    std::copy(s->vals.begin(), s->vals.end(), vals);
  }
  return DGASM_OK;
}

extern "C" int dgasm_system_destroy(dgasm_system_t s) {
  delete s;
  return DGASM_OK;
}

// Device copies (blocks column-major with stride np2s, and the mesh geometry), made on first use so
// that assembly itself needs no GPU.
int dgasm_system_s::ensure_device() {
  std::lock_guard<std::mutex> lk(dev_mu);
  if (d_vals.ptr) return DGASM_OK;
  const MeshData& m = mesh->m;
  const int nb = np;
  std::vector<double> dv((size_t)rowptr[m.ne] * np2s, 0.0);
  for (size_t k = 0; k < (size_t)rowptr[m.ne]; ++k)
    for (int a = 0; a < nb; ++a)
      for (int c = 0; c < nb; ++c) dv[k * np2s + (size_t)c * nb + a] = vals[k * nb * nb + (size_t)a * nb + c];
  DG_TRY(upload(d_rowptr, rowptr));
  DG_TRY(upload(d_col, col));
  DG_TRY(upload(d_xy, m.xy));
  DG_TRY(upload(d_pptr, m.ptr));
  DG_TRY(upload(d_pvtx, m.vtx));
  DG_TRY(upload(d_bbox, m.bbox));
  DG_TRY(upload(d_vals, dv));
  DG_CUDA(cudaGetDevice(&dev));
  return DGASM_OK;
}

// Host copy of the blocks of a device-assembled system (row-major per block)
int dgasm_system_s::ensure_host() {
  std::lock_guard<std::mutex> lk(dev_mu);
  const size_t nnzb = col.size();
  if (vals.size() == nnzb * np * np) return DGASM_OK;
  std::vector<double> dv(nnzb * np2s);
  DG_CUDA(cudaMemcpy(dv.data(), d_vals.ptr, sizeof(double) * dv.size(), cudaMemcpyDeviceToHost));
  vals.assign(nnzb * np * np, 0.0);
  for (size_t k = 0; k < nnzb; ++k)
    for (int a = 0; a < np; ++a)
      for (int c = 0; c < np; ++c) vals[k * np * np + (size_t)a * np + c] = dv[k * np2s + (size_t)c * np + a];
  return DGASM_OK;
}
