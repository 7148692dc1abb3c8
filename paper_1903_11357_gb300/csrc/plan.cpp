// Plan construction: element renumbering (subdomain by subdomain, reverse Cuthill-McKee inside),
// tile envelopes of the local Cholesky factors and their task lists.
//
// A Cholesky factor L of A_i has no entry left of the first nonzero of each row of A_i (fill stays
// inside the row envelope), so storing the tiles (I, F(I)) .. (I, I), with F(I) the first tile
// column touched by any row of tile row I, holds the exact dense factor.  Reverse Cuthill-McKee
// keeps the envelope narrow for the planar element graphs of a subdomain.
#include <algorithm>
#include <numeric>
#include <queue>
#include <thread>
#include <tuple>

#include "engine.h"
#include "hostpool.h"
#include "plan.h"

namespace dgasm {

void Envelope::build(const std::vector<std::vector<int>>& first_col, int sr_) {
  sr = sr_;
  const int SR = sr;
  nsub = (int)first_col.size();
  ndof.resize(nsub);
  sub_trow.assign(nsub + 1, 0);
  trow_F.clear();
  trow_ptr.clear();
  ntiles = 0;
  max_nbt = 0;
  std::vector<std::vector<int>> Fs(nsub);
  for (int s = 0; s < nsub; ++s) {
    int n = (int)first_col[s].size();
    ndof[s] = n;
    int nbt = (n + TILE - 1) / TILE;
    max_nbt = std::max(max_nbt, nbt);
    Fs[s].resize(nbt);
    for (int I = 0; I < nbt; ++I) {
      int F = I;
      for (int r = I * TILE; r < std::min(n, (I + 1) * TILE); ++r) F = std::min(F, first_col[s][r] / TILE);
      Fs[s][I] = F;
      trow_F.push_back(F);
      trow_ptr.push_back(ntiles);
      ntiles += I - F + 1;
    }
    sub_trow[s + 1] = sub_trow[s] + nbt;
  }
  // super-rows, their inverse blocks, the two solve streams and their runs
  sub_sr.assign(nsub + 1, 0);
  dinv_ptr.assign(1, 0);
  dinv_task.clear();
  fwd_ptr.assign(nsub + 1, 0);
  bwd_ptr.assign(nsub + 1, 0);
  fwd_src.clear();
  bwd_src.clear();
  fwd_run.clear();
  bwd_run.clear();
  fwd_src.reserve((size_t)ntiles + (size_t)ntiles / 2);
  bwd_src.reserve((size_t)ntiles + (size_t)ntiles / 2);
  for (int s = 0; s < nsub; ++s) {
    const int nbt = (int)Fs[s].size(), tr0 = sub_trow[s];
    const int nsr = (nbt + SR - 1) / SR;
    const int q0 = sub_sr[s];
    sub_sr[s + 1] = q0 + nsr;
    fwd_run.resize((size_t)(q0 + nsr) * SR * 2, 0);
    bwd_run.resize((size_t)(q0 + nsr) * SR * 2, 0);
    for (int q = 0; q < nsr; ++q) {
      const int I0 = q * SR, ntr = std::min(SR, nbt - I0);
      dinv_task.push_back(s);
      dinv_task.push_back(I0);
      dinv_task.push_back(ntr);
      dinv_ptr.push_back(dinv_ptr.back() + ntr * (ntr + 1) / 2);
    }
    // inverse-block tile (i, j), j <= i, of super-row q
    auto xtile = [&](int q, int i, int j) { return -(dinv_ptr[q0 + q] + i * (i + 1) / 2 + j + 1); };
    for (int q = 0; q < nsr; ++q) {
      const int I0 = q * SR, ntr = std::min(SR, nbt - I0);
      for (int o = 0; o < ntr; ++o) {   // run o: tile row I0+o left of the super-row, J ascending
        const int I = I0 + o, F = std::min(Fs[s][I], I0);
        for (int J = F; J < I0; ++J) fwd_src.push_back(trow_ptr[tr0 + I] + (J - Fs[s][I]));
        fwd_run[((size_t)(q0 + q) * SR + o) * 2] = F;
        fwd_run[((size_t)(q0 + q) * SR + o) * 2 + 1] = I0 - F;
      }
      for (int o = 0; o < ntr; ++o)
        for (int j = 0; j <= o; ++j) fwd_src.push_back(xtile(q, o, j));
    }
    for (int q = nsr - 1; q >= 0; --q) {
      const int I0 = q * SR, ntr = std::min(SR, nbt - I0), I1 = I0 + ntr;
      for (int o = 0; o < ntr; ++o) {   // run o: column J = I0+o below the super-row, I ascending
        const int J = I0 + o;
        int first = -1, last = -1;
        for (int I = I1; I < nbt; ++I)
          if (Fs[s][I] <= J) {
            if (first < 0) first = I;
            last = I;
          }
        if (first >= 0)
          for (int I = first; I <= last; ++I)
            bwd_src.push_back(Fs[s][I] <= J ? trow_ptr[tr0 + I] + (J - Fs[s][I]) : ZERO_TILE);
        bwd_run[((size_t)(q0 + q) * SR + o) * 2] = first >= 0 ? first : I1;
        bwd_run[((size_t)(q0 + q) * SR + o) * 2 + 1] = first >= 0 ? last - first + 1 : 0;
      }
      for (int o = 0; o < ntr; ++o)
        for (int i = o; i < ntr; ++i) bwd_src.push_back(xtile(q, i, o));
    }
    fwd_ptr[s + 1] = (long long)fwd_src.size();
    bwd_ptr[s + 1] = (long long)bwd_src.size();
  }
  ndinv = dinv_ptr.back();
  // Cholesky task lists by step K; the steps are independent, so each is built on its own (in parallel) and
  // the lists are then laid end to end in step order (panel indices in the tensor-core groups shifted to the
  // step's place), which gives the same arrays as building them one step after the other
  struct StepTasks {
    std::vector<int> diag, panel, tc, upd;
  };
  std::vector<StepTasks> steps(max_nbt);
  parallel_for(max_nbt, [&](int K) {
    StepTasks& T = steps[K];
    std::vector<int> S;
    for (int s = 0; s < nsub; ++s) {
      const int nbt = (int)Fs[s].size();
      if (K >= nbt) continue;
      T.diag.push_back(s);
      S.clear();
      for (int I = K + 1; I < nbt; ++I)
        if (Fs[s][I] <= K) S.push_back(I);
      const int pstart = (int)(T.panel.size() / 2), n = (int)S.size();   // within the step
      for (int I : S) { T.panel.push_back(s); T.panel.push_back(I); }
      for (int mb = 0; 4 * mb < n; ++mb) {
        const int bmax = std::min(n, 4 * mb + 4);   // column tiles J <= the block's last row tile
        for (int nb = 0; 8 * nb < bmax; ++nb) {
          T.tc.push_back(pstart);
          T.tc.push_back(n);
          T.tc.push_back(mb);
          T.tc.push_back(nb);
        }
      }
      for (size_t a = 0; a < S.size(); ++a)
        for (size_t b = 0; b <= a; ++b) {
          T.upd.push_back(s);
          T.upd.push_back(S[a]);
          T.upd.push_back(S[b]);
        }
    }
  });
  diag_off.assign(max_nbt + 1, 0);
  panel_off.assign(max_nbt + 1, 0);
  upd_off.assign(max_nbt + 1, 0);
  tc_off.assign(max_nbt + 1, 0);
  for (int K = 0; K < max_nbt; ++K) {
    diag_off[K + 1] = diag_off[K] + (int)steps[K].diag.size();
    panel_off[K + 1] = panel_off[K] + (int)(steps[K].panel.size() / 2);
    upd_off[K + 1] = upd_off[K] + (int)(steps[K].upd.size() / 3);
    tc_off[K + 1] = tc_off[K] + (int)(steps[K].tc.size() / 4);
  }
  diag_task.assign((size_t)diag_off[max_nbt], 0);
  panel_task.assign(2 * (size_t)panel_off[max_nbt], 0);
  upd_task.assign(3 * (size_t)upd_off[max_nbt], 0);
  tc_task.assign(4 * (size_t)tc_off[max_nbt], 0);
  parallel_for(max_nbt, [&](int K) {
    const StepTasks& T = steps[K];
    std::copy(T.diag.begin(), T.diag.end(), diag_task.begin() + diag_off[K]);
    std::copy(T.panel.begin(), T.panel.end(), panel_task.begin() + 2 * (size_t)panel_off[K]);
    std::copy(T.upd.begin(), T.upd.end(), upd_task.begin() + 3 * (size_t)upd_off[K]);
    int* tc = tc_task.data() + 4 * (size_t)tc_off[K];
    for (size_t i = 0; i < T.tc.size(); ++i) tc[i] = T.tc[i] + (i % 4 == 0 ? panel_off[K] : 0);
  });
}

namespace {

// Reverse Cuthill-McKee of the element graph restricted to `elems` (caller ids, ascending); returns the
// order.  `loc` is a scratch array over all elements (entries for `elems` are overwritten).
std::vector<int> rcm_order(const std::vector<int>& elems, const std::vector<int>& rowptr, const std::vector<int>& col,
                           const std::vector<int>& sub_of, int s, std::vector<int>& loc) {
  const int n = (int)elems.size();
  for (int i = 0; i < n; ++i) loc[elems[i]] = i;
  std::vector<int> aptr(n + 1, 0), adj;
  adj.reserve(8 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const int e = elems[i];
    for (int k = rowptr[e]; k < rowptr[e + 1]; ++k) {
      const int c = col[k];
      if (c != e && sub_of[c] == s) adj.push_back(loc[c]);
    }
    aptr[i + 1] = (int)adj.size();
  }
  auto deg = [&](int i) { return aptr[i + 1] - aptr[i]; };
  std::vector<int> order, level(n), visited(n, 0), result, nb;
  order.reserve(n);
  result.reserve(n);
  auto bfs = [&](int root) {
    order.clear();
    std::fill(level.begin(), level.end(), -1);
    order.push_back(root);
    level[root] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
      const int u = order[h];
      nb.clear();
      for (int k = aptr[u]; k < aptr[u + 1]; ++k)
        if (level[adj[k]] < 0) { level[adj[k]] = level[u] + 1; nb.push_back(adj[k]); }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg(a) != deg(b) ? deg(a) < deg(b) : a < b; });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  };
  for (int start = 0; start < n; ++start) {
    if (visited[start]) continue;
    // pseudo-peripheral root of this component (George-Liu iteration)
    int root = start;
    int best_depth = -1;
    for (int it = 0; it < 4; ++it) {
      bfs(root);
      const int depth = level[order.back()];
      if (depth <= best_depth) break;
      best_depth = depth;
      int cand = order.back();
      for (int u : order) if (level[u] == depth && deg(u) < deg(cand)) cand = u;
      root = cand;
    }
    bfs(root);
    for (int u : order) { visited[u] = 1; result.push_back(u); }
  }
  std::reverse(result.begin(), result.end());
  std::vector<int> out(n);
  for (int i = 0; i < n; ++i) out[i] = elems[result[i]];
  return out;
}

}  // namespace

int build_plan(const dgasm_system_s& sys, int nsub, int ncoarse, int q, const int* sub_in, const int* agg_in, int sr,
               Plan& P, const MeshData* coarse) {
  const MeshData& m = sys.mesh->m;
  const int ne = m.ne, np = sys.np;
  P.ne = ne;
  P.np = np;
  // partition
  if (sub_in) {
    P.sub_of.assign(sub_in, sub_in + ne);
    int mx = 0;
    for (int e = 0; e < ne; ++e) {
      if (P.sub_of[e] < 0) return set_error(DGASM_EINVAL, "sub_of_elem[%d] is negative", e);
      mx = std::max(mx, P.sub_of[e]);
    }
    nsub = mx + 1;
    std::vector<int> cnt(nsub, 0);
    for (int e = 0; e < ne; ++e) cnt[P.sub_of[e]]++;
    for (int s = 0; s < nsub; ++s) if (!cnt[s]) return set_error(DGASM_EINVAL, "subdomain %d is empty", s);
  } else {
    DG_TRY(compute_partition(m, nsub, 0, P.sub_of, nullptr));
  }
  P.nsub = nsub;
  P.q = q;
  P.nq = ncoarse > 0 || agg_in || coarse ? n_basis(q) : 0;
  P.nonnested = coarse != nullptr;
  P.agg_of.clear();
  if (coarse) {
    if (coarse->ne < 1) return set_error(DGASM_EINVAL, "the coarse mesh has no cells");
    P.nagg = coarse->ne;
  } else if (agg_in) {
    P.agg_of.assign(agg_in, agg_in + ne);
    int mx = 0;
    for (int e = 0; e < ne; ++e) {
      if (P.agg_of[e] < 0) return set_error(DGASM_EINVAL, "agg_of_elem[%d] is negative", e);
      mx = std::max(mx, P.agg_of[e]);
    }
    P.nagg = mx + 1;
  } else if (ncoarse > 0) {
    if (ncoarse > ne) return set_error(DGASM_EINVAL, "ncoarse=%d exceeds the element count", ncoarse);
    P.agg_of.assign(ne, 0);
    if (ncoarse >= nsub) {
      std::vector<std::vector<int>> members(nsub);
      for (int e = 0; e < ne; ++e) members[P.sub_of[e]].push_back(e);
      for (int i = 0; i < nsub; ++i) {
        const int ci = (int)(((long long)(i + 1) * ncoarse) / nsub - ((long long)i * ncoarse) / nsub);
        if (ci < 1 || (size_t)ci > members[i].size())
          return set_error(DGASM_EINVAL, "subdomain %d cannot hold %d agglomerates", i, ci);
      }
      // subdomain i's agglomerates are numbered from floor(i ncoarse / nsub) on
      parallel_for(nsub, [&](int i) {
        const int first = (int)(((long long)i * ncoarse) / nsub);
        rcb_parts(m, members[i], (int)(((long long)(i + 1) * ncoarse) / nsub) - first, P.agg_of, first);
      });
    } else {
      std::vector<int> all(ne);
      std::iota(all.begin(), all.end(), 0);
      rcb_parts(m, all, ncoarse, P.agg_of, 0);
    }
    P.nagg = ncoarse;
  } else {
    P.nagg = 0;
  }
  if (P.nagg > 0 && !P.nonnested) {
    std::vector<int> cnt(P.nagg, 0);
    for (int e = 0; e < ne; ++e) cnt[P.agg_of[e]]++;
    for (int j = 0; j < P.nagg; ++j) if (!cnt[j]) return set_error(DGASM_EINVAL, "agglomerate %d is empty", j);
  }
  // internal order: subdomain by subdomain, RCM inside
  std::vector<std::vector<int>> members(nsub);
  for (int e = 0; e < ne; ++e) members[P.sub_of[e]].push_back(e);
  // RCM of each subdomain, in parallel (subdomains are independent; results do not depend on threads)
  std::vector<std::vector<int>> ords(nsub);
  parallel_for(nsub, [&](int s) {
    thread_local std::vector<int> loc;   // rcm_order writes the entries it reads
    if ((int)loc.size() < ne) loc.resize(ne);
    ords[s] = rcm_order(members[s], sys.rowptr, sys.col, P.sub_of, s, loc);
  });
  P.perm.clear();
  P.perm.reserve(ne);
  P.sub_e0.assign(nsub + 1, 0);
  for (int s = 0; s < nsub; ++s) {
    P.perm.insert(P.perm.end(), ords[s].begin(), ords[s].end());
    P.sub_e0[s + 1] = (int)P.perm.size();
  }
  P.iperm.assign(ne, 0);
  for (int i = 0; i < ne; ++i) P.iperm[P.perm[i]] = i;
  // permuted CSR (columns ascending in internal ids; a row's columns are distinct, so insertion places each)
  P.rowptr.assign(ne + 1, 0);
  for (int i = 0; i < ne; ++i) P.rowptr[i + 1] = P.rowptr[i] + (sys.rowptr[P.perm[i] + 1] - sys.rowptr[P.perm[i]]);
  P.col.resize(P.rowptr[ne]);
  P.src_blk.resize(P.rowptr[ne]);
  {
    const int *srp = sys.rowptr.data(), *sc = sys.col.data(), *ip = P.iperm.data(), *rp = P.rowptr.data(),
              *pm = P.perm.data();
    int* pc = P.col.data();
    long long* ps = P.src_blk.data();
    constexpr int RB = 512;   // internal rows per task
    parallel_for((ne + RB - 1) / RB, [&](int b) {
      for (int i = b * RB; i < std::min(ne, (b + 1) * RB); ++i) {
        const int e = pm[i], base = rp[i];
        int n = 0;
        for (int k = srp[e]; k < srp[e + 1]; ++k, ++n) {
          const int c = ip[sc[k]];
          int j = n;
          for (; j > 0 && pc[base + j - 1] > c; --j) {
            pc[base + j] = pc[base + j - 1];
            ps[base + j] = ps[base + j - 1];
          }
          pc[base + j] = c;
          ps[base + j] = k;
        }
      }
    });
  }
  // envelopes: first column of each local dof row
  std::vector<std::vector<int>> fc(nsub);
  parallel_for(nsub, [&](int s) {
    int e0 = P.sub_e0[s], e1 = P.sub_e0[s + 1];
    fc[s].resize((size_t)(e1 - e0) * np);
    for (int i = e0; i < e1; ++i) {
      int first = i - e0;
      for (int k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
        int c = P.col[k];
        if (c >= e0 && c < e1) first = std::min(first, c - e0);
      }
      for (int a = 0; a < np; ++a) fc[s][(size_t)(i - e0) * np + a] = first * np;
    }
  });
  P.env.build(fc, sr);
  // groups and coarse data
  P.agg_int.assign(ne, -1);
  P.grp_ptr.assign(1, 0);
  P.grp_elems.clear();
  if (P.nagg > 0 && !P.nonnested) {
    std::vector<std::vector<int>> mem(P.nagg);
    for (int i = 0; i < ne; ++i) { P.agg_int[i] = P.agg_of[P.perm[i]]; mem[P.agg_int[i]].push_back(i); }
    for (int j = 0; j < P.nagg; ++j) {
      P.grp_elems.insert(P.grp_elems.end(), mem[j].begin(), mem[j].end());
      P.grp_ptr.push_back((int)P.grp_elems.size());
    }
    P.ngrp = P.nagg;
    P.agg_bbox.assign(4 * (size_t)P.nagg, 0.0);
    for (int j = 0; j < P.nagg; ++j) {
      P.agg_bbox[4 * j] = 1e300; P.agg_bbox[4 * j + 1] = -1e300;
      P.agg_bbox[4 * j + 2] = 1e300; P.agg_bbox[4 * j + 3] = -1e300;
    }
    for (int e = 0; e < ne; ++e) {
      int j = P.agg_of[e];
      const double* b = &m.bbox[4 * (size_t)e];
      P.agg_bbox[4 * j] = std::min(P.agg_bbox[4 * j], b[0]);
      P.agg_bbox[4 * j + 1] = std::max(P.agg_bbox[4 * j + 1], b[1]);
      P.agg_bbox[4 * j + 2] = std::min(P.agg_bbox[4 * j + 2], b[2]);
      P.agg_bbox[4 * j + 3] = std::max(P.agg_bbox[4 * j + 3], b[3]);
    }
  } else {
    const int G = 64;
    for (int i = 0; i < ne; i += G) {
      for (int k = i; k < std::min(ne, i + G); ++k) P.grp_elems.push_back(k);
      P.grp_ptr.push_back((int)P.grp_elems.size());
    }
    P.ngrp = (int)P.grp_ptr.size() - 1;
  }
  if (P.nagg > 0) {   // the coarse factor: one dense block
    int n0 = P.nagg * P.nq;
    std::vector<std::vector<int>> fc0(1, std::vector<int>(n0, 0));
    P.env0.build(fc0, super_row(DGASM_FP64));
  }
  return DGASM_OK;
}

// Consistency checks of an envelope against its own definitions (for tests; no device work):
//  * the tensor-core update groups of every step K cover exactly the plain update tasks (s, I, J), I >= J,
//    each block inside the panel and targets inside the envelope right of K;
//  * each subdomain's forward stream is, per super-row q and row o, the factor tiles (I0+o, J), J = F .. I0-1,
//    then the inverse-block tiles (o, j), j <= o; the backward stream, per super-row q descending and column
//    o, the tiles (I, I0+o) of the rows below from the first to the last that reach column I0+o (zero tiles
//    in between where a row does not), then the inverse-block tiles (i, o), i >= o; run tables match.
// Returns the number of violations; *checks counts what was compared.
long long check_envelope(const Envelope& E, long long* checks) {
  long long bad = 0, n = 0;
  const int SR = E.sr;
  for (int K = 0; K < E.max_nbt; ++K) {
    std::vector<std::tuple<int, int, int>> ref, got;
    for (int t = E.upd_off[K]; t < E.upd_off[K + 1]; ++t)
      ref.emplace_back(E.upd_task[3 * t], E.upd_task[3 * t + 1], E.upd_task[3 * t + 2]);
    for (int t = E.tc_off[K]; t < E.tc_off[K + 1]; ++t) {
      const int pstart = E.tc_task[4 * t], nn = E.tc_task[4 * t + 1], mb = E.tc_task[4 * t + 2], nb = E.tc_task[4 * t + 3];
      const int s = E.panel_task[2 * pstart];
      const int a0 = 4 * mb, na = std::min(4, nn - a0), b0 = 8 * nb, nbt = std::min(8, std::min(nn, a0 + 4) - b0);
      bad += (na <= 0 || nbt <= 0 || pstart < E.panel_off[K] || pstart + nn > E.panel_off[K + 1]);
      for (int w = 0; w < na; ++w)
        for (int u = 0; u < nbt && b0 + u <= a0 + w; ++u) {
          const int I = E.panel_task[2 * (pstart + a0 + w) + 1], J = E.panel_task[2 * (pstart + b0 + u) + 1];
          const int tr = E.sub_trow[s] + I;
          bad += (J < E.trow_F[tr] || J > I || J <= K || E.panel_task[2 * (pstart + b0 + u)] != s);
          got.emplace_back(s, I, J);
        }
    }
    std::sort(ref.begin(), ref.end());
    std::sort(got.begin(), got.end());
    bad += ref != got;
    n += (long long)ref.size();
  }
  for (int s = 0; s < E.nsub; ++s) {
    const int t0 = E.sub_trow[s], nbt = E.sub_trow[s + 1] - t0, nsr = (nbt + SR - 1) / SR, q0 = E.sub_sr[s];
    auto tile = [&](int I, int J) -> long long { return E.trow_ptr[t0 + I] + (J - E.trow_F[t0 + I]); };
    long long f = E.fwd_ptr[s];
    for (int q = 0; q < nsr; ++q) {
      const int I0 = q * SR, ntr = std::min(SR, nbt - I0);
      for (int o = 0; o < ntr; ++o) {
        const int I = I0 + o, F = std::min(E.trow_F[t0 + I], I0);
        bad += E.fwd_run[((size_t)(q0 + q) * SR + o) * 2] != F || E.fwd_run[((size_t)(q0 + q) * SR + o) * 2 + 1] != I0 - F;
        for (int J = F; J < I0; ++J, ++f, ++n) bad += E.fwd_src[f] != tile(I, J);
      }
      for (int o = 0; o < ntr; ++o)
        for (int j = 0; j <= o; ++j, ++f, ++n) bad += E.fwd_src[f] != -(E.dinv_ptr[q0 + q] + o * (o + 1) / 2 + j + 1);
    }
    bad += f != E.fwd_ptr[s + 1];
    long long b = E.bwd_ptr[s];
    for (int q = nsr - 1; q >= 0; --q) {
      const int I0 = q * SR, ntr = std::min(SR, nbt - I0), I1 = I0 + ntr;
      for (int o = 0; o < ntr; ++o) {
        const int J = I0 + o;
        int first = -1, last = -1;
        for (int I = I1; I < nbt; ++I)
          if (E.trow_F[t0 + I] <= J) { if (first < 0) first = I; last = I; }
        const int len = first >= 0 ? last - first + 1 : 0;
        bad += E.bwd_run[((size_t)(q0 + q) * SR + o) * 2 + 1] != len;
        for (int I = first; len > 0 && I <= last; ++I, ++b, ++n)
          bad += E.bwd_src[b] != (E.trow_F[t0 + I] <= J ? tile(I, J) : ZERO_TILE);
      }
      for (int o = 0; o < ntr; ++o)
        for (int i = o; i < ntr; ++i, ++b, ++n) bad += E.bwd_src[b] != -(E.dinv_ptr[q0 + q] + i * (i + 1) / 2 + o + 1);
    }
    bad += b != E.bwd_ptr[s + 1];
  }
  if (checks) *checks = n;
  return bad;
}

}  // namespace dgasm

extern "C" int dgasm_selftest_plan(dgasm_system_t s, int nsub, int64_t* violations, int64_t* checks) {
  using namespace dgasm;
  clear_error();
  if (!s || !violations || nsub < 1) return set_error(DGASM_EINVAL, "dgasm_selftest_plan: bad arguments");
  Plan P;
  DG_TRY(build_plan(*s, nsub, 0, 1, nullptr, nullptr, super_row(DGASM_FP64), P));
  long long n = 0;
  *violations = check_envelope(P.env, &n);
  if (checks) *checks = n;
  return DGASM_OK;
}
