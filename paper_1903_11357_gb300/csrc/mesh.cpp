// Polygonal mesh: validation, geometry (area, centroid, diameter, bounding box) and faces
// (Sec. 2: elements kappa, faces F_h = F_h^I u F_h^B, diameter h_kappa).
#include <algorithm>
#include <cmath>
#include <memory>
#include <unordered_map>

#include "common.h"

using namespace dgasm;

namespace {
inline uint64_t edge_key(int a, int b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }
}  // namespace

extern "C" int dgasm_mesh_create(int nv, const double* xy, int ne, const int* poly_ptr, const int* poly_vtx,
                                 const double* rho, dgasm_mesh_t* out) {
  clear_error();
  if (!out) return set_error(DGASM_EINVAL, "dgasm_mesh_create: out is NULL");
  *out = nullptr;
  if (nv < 3 || ne < 1 || !xy || !poly_ptr || !poly_vtx || !rho)
    return set_error(DGASM_EINVAL, "dgasm_mesh_create: empty mesh or NULL array");
  // owned until it is handed out, so an error return frees it only after its message is formatted
  std::unique_ptr<dgasm_mesh_s> h(new (std::nothrow) dgasm_mesh_s());
  if (!h) return set_error(DGASM_ENOMEM, "dgasm_mesh_create: host allocation failed");
  MeshData& m = h->m;
  m.nv = nv;
  m.ne = ne;
  m.xy.assign(xy, xy + 2 * (size_t)nv);
  if (poly_ptr[0] != 0) { return set_error(DGASM_EINVAL, "poly_ptr[0] must be 0"); }
  m.ptr.assign(poly_ptr, poly_ptr + ne + 1);
  for (int e = 0; e < ne; ++e) {
    if (m.ptr[e + 1] - m.ptr[e] < 3) { return set_error(DGASM_EINVAL, "element %d has fewer than 3 vertices", e); }
  }
  m.vtx.assign(poly_vtx, poly_vtx + m.ptr[ne]);
  for (size_t i = 0; i < m.vtx.size(); ++i)
    if (m.vtx[i] < 0 || m.vtx[i] >= nv) { return set_error(DGASM_EINVAL, "vertex id %d out of range", m.vtx[i]); }
  m.rho.assign(rho, rho + ne);
  m.area.resize(ne); m.cx.resize(ne); m.cy.resize(ne); m.diam.resize(ne); m.bbox.resize(4 * (size_t)ne);
  for (int e = 0; e < ne; ++e) {
    if (!(m.rho[e] > 0.0) || !std::isfinite(m.rho[e])) { return set_error(DGASM_EINVAL, "element %d: rho must be positive and finite", e); }
    int b = m.ptr[e], n = m.ptr[e + 1] - b;
    // shoelace, summed vertex by vertex from the first vertex
    double a2 = 0, sx = 0, sy = 0;
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300, dmax = 0;
    for (int k = 0; k < n; ++k) {
      const double* P = &m.xy[2 * (size_t)m.vtx[b + k]];
      const double* Q = &m.xy[2 * (size_t)m.vtx[b + (k + 1) % n]];
      double cr = P[0] * Q[1] - Q[0] * P[1];
      a2 += cr;
      sx += (P[0] + Q[0]) * cr;
      sy += (P[1] + Q[1]) * cr;
      x0 = std::min(x0, P[0]); x1 = std::max(x1, P[0]);
      y0 = std::min(y0, P[1]); y1 = std::max(y1, P[1]);
      for (int l = k + 1; l < n; ++l) {
        const double* R = &m.xy[2 * (size_t)m.vtx[b + l]];
        dmax = std::max(dmax, std::hypot(P[0] - R[0], P[1] - R[1]));
      }
    }
    if (!(a2 > 0.0)) { return set_error(DGASM_EINVAL, "element %d: non-positive signed area (clockwise or degenerate)", e); }
    m.area[e] = 0.5 * a2;
    m.cx[e] = sx / (3.0 * a2);
    m.cy[e] = sy / (3.0 * a2);
    m.diam[e] = dmax;
    m.bbox[4 * (size_t)e + 0] = x0; m.bbox[4 * (size_t)e + 1] = x1;
    m.bbox[4 * (size_t)e + 2] = y0; m.bbox[4 * (size_t)e + 3] = y1;
  }
  // faces from directed edges
  std::unordered_map<uint64_t, int> owner;
  owner.reserve(m.vtx.size() * 2);
  for (int e = 0; e < ne; ++e) {
    int b = m.ptr[e], n = m.ptr[e + 1] - b;
    for (int k = 0; k < n; ++k) {
      int va = m.vtx[b + k], vb = m.vtx[b + (k + 1) % n];
      if (va == vb) { return set_error(DGASM_EINVAL, "element %d: repeated consecutive vertex", e); }
      auto ins = owner.emplace(edge_key(va, vb), e);
      if (!ins.second) { return set_error(DGASM_EINVAL, "element %d: edge (%d,%d) used twice in the same direction", e, va, vb); }
    }
  }
  struct F { int ep, em, va, vb; };
  std::vector<F> faces;
  faces.reserve(owner.size());
  for (int e = 0; e < ne; ++e) {
    int b = m.ptr[e], n = m.ptr[e + 1] - b;
    for (int k = 0; k < n; ++k) {
      int va = m.vtx[b + k], vb = m.vtx[b + (k + 1) % n];
      auto it = owner.find(edge_key(vb, va));
      if (it == owner.end()) faces.push_back({e, -1, va, vb});
      else if (e < it->second) faces.push_back({e, it->second, va, vb});
    }
  }
  std::sort(faces.begin(), faces.end(), [](const F& a, const F& b) {
    if (a.ep != b.ep) return a.ep < b.ep;
    if (a.em != b.em) return a.em < b.em;
    if (a.va != b.va) return a.va < b.va;
    return a.vb < b.vb;
  });
  size_t nf = faces.size();
  m.f_ep.resize(nf); m.f_em.resize(nf); m.f_va.resize(nf); m.f_vb.resize(nf);
  std::vector<int> cnt(ne + 1, 0);
  for (size_t f = 0; f < nf; ++f) {
    m.f_ep[f] = faces[f].ep; m.f_em[f] = faces[f].em; m.f_va[f] = faces[f].va; m.f_vb[f] = faces[f].vb;
    if (faces[f].em < 0) ++m.nfb; else ++m.nfi;
    cnt[faces[f].ep + 1]++;
    if (faces[f].em >= 0) cnt[faces[f].em + 1]++;
  }
  m.ef_ptr.assign(ne + 1, 0);
  for (int e = 0; e < ne; ++e) m.ef_ptr[e + 1] = m.ef_ptr[e] + cnt[e + 1];
  m.ef_face.resize(m.ef_ptr[ne]);
  std::vector<int> fill(m.ef_ptr.begin(), m.ef_ptr.end() - 1);
  for (size_t f = 0; f < nf; ++f) {
    m.ef_face[fill[faces[f].ep]++] = (int)f;
    if (faces[f].em >= 0) m.ef_face[fill[faces[f].em]++] = (int)f;
  }
  *out = h.release();
  return DGASM_OK;
}

extern "C" int dgasm_mesh_info(dgasm_mesh_t h, int* ne, int* nfi, int* nfb) {
  if (!h) return set_error(DGASM_EINVAL, "dgasm_mesh_info: NULL mesh");
  if (ne) *ne = h->m.ne;
  if (nfi) *nfi = h->m.nfi;
  if (nfb) *nfb = h->m.nfb;
  return DGASM_OK;
}

extern "C" int dgasm_mesh_centroids(dgasm_mesh_t h, double* out) {
  if (!h || !out) return set_error(DGASM_EINVAL, "dgasm_mesh_centroids: NULL argument");
  for (int e = 0; e < h->m.ne; ++e) { out[2 * e] = h->m.cx[e]; out[2 * e + 1] = h->m.cy[e]; }
  return DGASM_OK;
}

extern "C" int dgasm_mesh_destroy(dgasm_mesh_t h) {
  delete h;
  return DGASM_OK;
}
