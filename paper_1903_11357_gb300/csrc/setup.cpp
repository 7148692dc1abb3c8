// dgasm_setup: partition and ordering (host), then on the device the extraction of each A_i (Sec. 3),
// its tile Cholesky factorisation, the L2 prolongation R_0^T (Eq. R0T), A_0 = R_0 A R_0^T (Eq. A0) and
// the FP64 factor and inverse of A_0.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "hostpool.h"
#include "plan.h"
#include "profile.h"
#include "solver.h"

using namespace dgasm;

namespace dgasm {

namespace {

int fact_elem_bytes(int prec) { return prec == DGASM_FP64 ? 8 : 4; }
int store_elem_bytes(int prec) { return prec == DGASM_FP64 ? 8 : (prec == DGASM_BF16 ? 2 : 4); }

int upload_env(const Envelope& E, EnvBufs& D) {
  std::vector<int> ndof(E.ndof);
  DG_TRY(upload(D.ndof, ndof));
  DG_TRY(upload(D.sub_trow, E.sub_trow));
  DG_TRY(upload(D.trow_F, E.trow_F));
  DG_TRY(upload(D.trow_ptr, E.trow_ptr));
  DG_TRY(upload(D.diag_task, E.diag_task));
  DG_TRY(upload(D.panel_task, E.panel_task));
  DG_TRY(upload(D.upd_task, E.upd_task));
  DG_TRY(upload(D.tc_task, E.tc_task));
  DG_TRY(upload(D.bwd_src, E.bwd_src));
  DG_TRY(upload(D.fwd_src, E.fwd_src));
  DG_TRY(upload(D.fwd_ptr, E.fwd_ptr));
  DG_TRY(upload(D.bwd_ptr, E.bwd_ptr));
  DG_TRY(upload(D.dinv_task, E.dinv_task));
  DG_TRY(upload(D.dinv_ptr, E.dinv_ptr));
  DG_TRY(upload(D.sub_sr, E.sub_sr));
  DG_TRY(upload(D.fwd_run, E.fwd_run));
  DG_TRY(upload(D.bwd_run, E.bwd_run));
  D.dev.nsub = E.nsub;
  D.dev.ndof = D.ndof.as<int>();
  D.dev.sub_trow = D.sub_trow.as<int>();
  D.dev.trow_F = D.trow_F.as<int>();
  D.dev.trow_ptr = D.trow_ptr.as<long long>();
  return DGASM_OK;
}

// factor the tile pool Lr (row-major, factor precision) in place, step by step
int factor_env(int prec, const Envelope& E, EnvBufs& D, void* Lr, int* err, cudaStream_t st, EventPairs* ev,
               int* launches) {
  const int fp = prec == DGASM_FP64 ? 0 : 1;
  for (int K = 0; K < E.max_nbt; ++K) {
    int nd = E.diag_off[K + 1] - E.diag_off[K];
    int npn = E.panel_off[K + 1] - E.panel_off[K];
    int nu = E.upd_off[K + 1] - E.upd_off[K];
    int id = ev && nd ? ev->begin(PK_CHOL_DIAG, st) : -1;
    int rc = launch_chol_diag(fp, D.dev, Lr, K, D.diag_task.as<int>() + E.diag_off[K], nd, err, st);
    if (ev) ev->end(id, st);
    if (rc) return cuda_error(rc, "tile Cholesky diagonal step");
    id = ev && npn ? ev->begin(PK_CHOL_PANEL, st) : -1;
    rc = launch_chol_panel(fp, D.dev, Lr, K, D.panel_task.as<int>() + 2 * (size_t)E.panel_off[K], npn, st);
    if (ev) ev->end(id, st);
    if (rc) return cuda_error(rc, "tile Cholesky panel step");
    id = ev && nu ? ev->begin(PK_CHOL_UPDATE, st) : -1;
    if (prec == DGASM_TF32 || prec == DGASM_BF16)   // tensor cores (split TF32 or BF16 products, FP32 accumulation)
      rc = launch_chol_update_tc(D.dev, (float*)Lr, K, D.panel_task.as<int>(), D.tc_task.as<int>() + 4 * (size_t)E.tc_off[K],
                                 E.tc_off[K + 1] - E.tc_off[K], err, st, prec == DGASM_BF16 ? 1 : 0);
    else
      rc = launch_chol_update(fp, D.dev, Lr, K, D.upd_task.as<int>() + 3 * (size_t)E.upd_off[K], nu, st);
    if (ev) ev->end(id, st);
    if (rc) return cuda_error(rc, "tile Cholesky update step");
    *launches += (nd > 0) + (npn > 0) + (nu > 0);
  }
  return DGASM_OK;
}

// From the factored tile pool Lf (row-major, diagonal tiles inverted): the super-row inverse blocks,
// then the forward stream (column-major tiles) and the backward stream (row-major tiles) in the order
// the triangular solves consume them.  Asynchronous on st: Lf and the temporaries go to `keep`, released
// by the caller after the setup's final synchronisation.
int build_streams(int fprec, const Envelope& E, EnvBufs& D, DevBuf& Lf, DevBuf& Lc, DevBuf& Lr, cudaStream_t st,
                  int* nl, SetupTemps& keep) {
  const int fp = fprec == DGASM_FP64 ? 0 : 1;
  const size_t eb = fact_elem_bytes(fprec);
  const long long nf = (long long)E.fwd_src.size(), nb = (long long)E.bwd_src.size();
  const int nsr = (int)E.dinv_ptr.size() - 1;
  DevBuf X, Sf, Sb;
  DG_TRY(X.alloc((size_t)std::max<long long>(E.ndinv, 1) * TILE * TILE * eb));
  DG_CUDA(launch_dinv(fp, D.dev, Lf.ptr, D.dinv_task.as<int>(), D.dinv_ptr.as<long long>(), X.ptr, nsr, st));
  DG_TRY(Sf.alloc((size_t)nf * TILE * TILE * eb));
  DG_TRY(Sb.alloc((size_t)nb * TILE * TILE * eb));
  DG_CUDA(launch_stream_gather(fp, Lf.ptr, X.ptr, D.fwd_src.as<long long>(), Sf.ptr, nf, 1, st));
  DG_CUDA(launch_stream_gather(fp, Lf.ptr, X.ptr, D.bwd_src.as<long long>(), Sb.ptr, nb, 0, st));
  *nl += 3;
  if (fprec == DGASM_BF16) {
    DG_TRY(Lc.alloc((size_t)nf * TILE * TILE * 2));
    DG_TRY(Lr.alloc((size_t)nb * TILE * TILE * 2));
    DG_CUDA(launch_to_bf16(Sf.as<float>(), Lc.ptr, nf * TILE * TILE, st));
    DG_CUDA(launch_to_bf16(Sb.as<float>(), Lr.ptr, nb * TILE * TILE, st));
    *nl += 2;
    keep.add(std::move(Sf));
    keep.add(std::move(Sb));
  } else {
    Lc = std::move(Sf);
    Lr = std::move(Sb);
  }
  keep.add(std::move(X));
  keep.add(std::move(Lf));
  return DGASM_OK;
}

}  // namespace

}  // namespace dgasm

// ---- setup ---------------------------------------------------------------------------------------
namespace dgasm {

// Validation, streams and the host plan (partition, ordering, envelopes, task lists): no device work
// besides the one-time upload of the system matrix.
int prec_plan(dgasm_system_s* s, const dgasm_setup_opts* o, std::unique_ptr<dgasm_prec_s>& pc) {
  if (!s || !o) return set_error(DGASM_EINVAL, "dgasm_setup: NULL argument");
  if (o->precision < DGASM_FP64 || o->precision > DGASM_BF16) return set_error(DGASM_EINVAL, "unknown precision %d", o->precision);
  const bool coarse = o->ncoarse > 0 || o->agg_of_elem || o->coarse_mesh;
  if (coarse && (o->p_c < 1 || o->p_c > s->p)) return set_error(DGASM_EINVAL, "p_c=%d must lie in [1, p=%d]", o->p_c, s->p);
  const auto t_start = std::chrono::steady_clock::now();
  pc.reset(new (std::nothrow) dgasm_prec_s());
  if (!pc) return set_error(DGASM_ENOMEM, "host allocation failed");
  pc->t_start = t_start;
  pc->sys = s;
  pc->precision = o->precision;
  DG_TRY(s->ensure_device());
  DG_TRY(pc->init_streams(o->stream));
  Plan& P = pc->P;
  const MeshData* cm = o->coarse_mesh ? &o->coarse_mesh->m : nullptr;
  DG_TRY(build_plan(*s, o->nsub, o->ncoarse, coarse ? o->p_c : 1, o->sub_of_elem, o->agg_of_elem,
                    super_row(o->precision), P, cm));
  pc->n0 = P.nagg * P.nq;
  // non-nested coarse space: R_0^T blocks over the fine/coarse cell intersections (host, like the assembly)
  if (P.nonnested) DG_TRY(nonnested_r0t(s->mesh->m, P.perm, *cm, s->p, P.q, pc->nn));
  pc->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return DGASM_OK;
}

// Device bytes of a built preconditioner (peak during its setup) plus the Krylov state for nrhs
// right-hand sides and maxit recorded iterations.
size_t prec_estimate_bytes(const dgasm_prec_s& pc, int nrhs, int maxit) {
  const Plan& P = pc.P;
  const size_t ndof = (size_t)P.ne * P.np, t = (size_t)P.env.ntiles * TILE * TILE, n0 = pc.n0;
  size_t b = P.col.size() * (size_t)pc.sys->np2s * 8 + ndof * 8 + P.col.size() * 12 + (size_t)P.ne * 20;
  const size_t ns = P.env.fwd_src.size() + P.env.bwd_src.size();
  const size_t ts = ns * TILE * TILE, td = (size_t)P.env.ndinv * TILE * TILE;
  b += (t + td) * (pc.precision == DGASM_FP64 ? 8 : 4) + ts * (pc.precision == DGASM_FP64 ? 8 : 4) + ns * 8;
  b += (P.env.upd_task.size() + P.env.tc_task.size() + P.env.panel_task.size() + P.env.diag_task.size() +
        P.env.trow_F.size() * 3) * 4;
  b += pc.nn.blocks.size() * 8 + (pc.nn.ptr.size() + pc.nn.col.size() * 3 + pc.nn.tptr.size()) * 4;
  if (n0) b += ndof * P.nq * 8 + n0 * n0 * 8 * 3 + (size_t)P.env0.ntiles * TILE * TILE * 16 + P.col.size() * P.nq * P.nq * 8;
  const int epi = NTHREADS / P.np;
  b += 8 * ((size_t)6 * nrhs * ndof + 2 * nrhs * std::max<size_t>(n0, 1) + 2 * (size_t)nrhs * maxit +
            (size_t)nrhs * ((P.ne + epi - 1) / epi + P.ngrp + P.nsub + n0 / 8 + 1)) + 4096;
  return b;
}

// The coarse space (R_0^T, A_0 = R_0 A R_0^T, its factor and inverse) does not depend on the local factors:
// it is issued on the side stream and runs beside the local factorisation.  Nothing is freed and no stream is
// synchronised until all device work of the setup has been issued (a cudaFree waits for the whole device).
int prec_build(dgasm_prec_s* pc, SetupTemps* defer) {
  dgasm_system_s* s = pc->sys;
  Plan& P = pc->P;
  EventPairs* ev = profiling() ? &pc->setup_ev : nullptr;
  if (ev) ev->reset();
  int nl = 0;
  cudaStream_t st = pc->stream, cs = pc->side;
  const int ne = P.ne, np = P.np, np2s = s->np2s;
  SetupTemps keep;
  DevBuf Lf;  // factorisation pool (row-major)
  // on every return, the work issued on both streams finishes before keep and Lf are freed
  struct Drain {
    cudaStream_t a, b;
    ~Drain() { cudaStreamSynchronize(a); cudaStreamSynchronize(b); }
  } drain{st, cs};
  // plan arrays
  DG_TRY(upload(pc->perm, P.perm));
  DG_TRY(upload(pc->rowptr, P.rowptr));
  DG_TRY(upload(pc->col, P.col));
  DG_TRY(upload(pc->src_blk, P.src_blk));
  DG_TRY(upload(pc->sub_e0, P.sub_e0));
  DG_TRY(upload(pc->grp_ptr, P.grp_ptr));
  DG_TRY(upload(pc->grp_elems, P.grp_elems));
  DG_TRY(upload(pc->agg_int, P.agg_int));
  DG_TRY(upload_env(P.env, pc->env));
  std::vector<int> err0{0, -1, -1, 0, 0, -1, -1, 0};
  DG_TRY(upload(pc->err, err0));
  // permuted matrix and scaling
  const long long nnzb = (long long)P.col.size();
  DG_TRY(pc->vals.alloc(sizeof(double) * nnzb * np2s));
  DG_CUDA(launch_permute_blocks(s->d_vals.as<double>(), pc->src_blk.as<long long>(), pc->vals.as<double>(), nnzb, np2s, st));
  nl += 2;
  DG_TRY(pc->scale.alloc(sizeof(double) * (size_t)ne * np));
  DG_CUDA(launch_scale(pc->rowptr.as<int>(), pc->col.as<int>(), pc->vals.as<double>(), ne, np, np2s, pc->scale.as<double>(), st));
  DG_CUDA(cudaEventRecord(pc->ev_fork, st));   // the permuted matrix is ready for the coarse stream
  // local factors (stream st)
  pc->blocks = P.nsub == P.ne;
  const int fprec = pc->precision;
  if (pc->blocks) {
    // every subdomain is one element: explicit FP64 inverses of the diagonal blocks
    DG_TRY(pc->dinv.alloc(sizeof(double) * (size_t)ne * np * np));
    DG_CUDA(launch_bjac_inverse(pc->rowptr.as<int>(), pc->col.as<int>(), pc->vals.as<double>(), ne, np, np2s,
                                pc->dinv.as<double>(), pc->err.as<int>(), st));
    nl += 1;
  } else {
    const size_t ftiles = (size_t)P.env.ntiles * TILE * TILE;
    DG_TRY(Lf.alloc(ftiles * fact_elem_bytes(fprec)));
    DG_CUDA(cudaMemsetAsync(Lf.ptr, 0, Lf.bytes, st));
    DG_CUDA(launch_extract_rows(fprec == DGASM_FP64 ? 0 : 1, pc->env.dev, pc->sub_e0.as<int>(), pc->rowptr.as<int>(),
                                pc->col.as<int>(), pc->vals.as<double>(), np, np2s, pc->scale.as<double>(), Lf.ptr,
                                P.nsub, ne, st));
    nl += 1;
    DG_TRY(factor_env(fprec, P.env, pc->env, Lf.ptr, pc->err.as<int>(), st, ev, &nl));
  }
  // coarse space: R_0^T, A_0 = R_0 A R_0^T, FP64 factor and explicit inverse (stream cs)
  int* coarse_err = nullptr;   // error word of the coarse inverse's bounded waits
  if (pc->n0 > 0) {
    DG_CUDA(cudaStreamWaitEvent(cs, pc->ev_fork, 0));
    const int n0 = pc->n0, q = P.q, nq = P.nq, mq = (s->p + q + 2) / 2;
    std::vector<double> gt, gw;
    gauss_legendre01(mq, gt, gw);
    DevBuf d_gt, d_gw, d_aggbox;
    DG_TRY(upload(d_gt, gt));
    DG_TRY(upload(d_gw, gw));
    DG_TRY(upload(d_aggbox, P.agg_bbox));
    DevBuf A0;
    DG_TRY(A0.alloc(sizeof(double) * (size_t)n0 * n0));
    if (P.nonnested) {
      // R_0^T pairs from the plan; A_0 accumulated row block by row block on the device
      DG_TRY(upload(pc->r0t, pc->nn.blocks));
      DG_TRY(upload(pc->r0t_ptr, pc->nn.ptr));
      DG_TRY(upload(pc->r0t_col, pc->nn.col));
      DG_TRY(upload(pc->r0t_elem, pc->nn.elem));
      DG_TRY(upload(pc->rT_ptr, pc->nn.tptr));
      DG_TRY(upload(pc->rT_pair, pc->nn.tpair));
      DG_CUDA(cudaMemsetAsync(A0.ptr, 0, A0.bytes, cs));
      DG_CUDA(launch_galerkin_nn(pc->rowptr.as<int>(), pc->col.as<int>(), pc->vals.as<double>(), np, np2s, nq,
                                 pc->r0t_ptr.as<int>(), pc->r0t_col.as<int>(), pc->r0t_elem.as<int>(), pc->r0t.as<double>(),
                                 pc->rT_ptr.as<int>(), pc->rT_pair.as<int>(), P.nagg, n0, A0.as<double>(), cs));
    } else {
      DG_TRY(pc->r0t.alloc(sizeof(double) * (size_t)ne * np * nq));
      DG_CUDA(launch_r0t(pc->perm.as<int>(), s->d_bbox.as<double>(), pc->agg_int.as<int>(), d_aggbox.as<double>(), ne,
                         s->p, q, d_gt.as<double>(), d_gw.as<double>(), mq, pc->r0t.as<double>(), cs));
      DevBuf W;
      DG_TRY(W.alloc(sizeof(double) * P.col.size() * (size_t)nq * nq));
      DG_CUDA(launch_galerkin(pc->grp_ptr.as<int>(), pc->grp_elems.as<int>(), pc->agg_int.as<int>(), pc->rowptr.as<int>(),
                              pc->col.as<int>(), pc->vals.as<double>(), pc->r0t.as<double>(), ne, (long long)P.col.size(),
                              P.nagg, np, np2s, nq, W.as<double>(), A0.as<double>(), cs));
      keep.add(std::move(W));
    }
    DG_TRY(upload_env(P.env0, pc->env0));
    DevBuf scale0, Lr0, Lc0, Lb0;
    DG_TRY(scale0.alloc(sizeof(double) * n0));
    const size_t t0 = (size_t)P.env0.ntiles * TILE * TILE;
    DG_TRY(Lr0.alloc(sizeof(double) * t0));
    DG_CUDA(cudaMemsetAsync(Lr0.ptr, 0, Lr0.bytes, cs));
    DG_CUDA(launch_coarse_extract(A0.as<double>(), n0, scale0.as<double>(), pc->env0.dev, Lr0.as<double>(), cs));
    nl += 4;
    DG_TRY(factor_env(DGASM_FP64, P.env0, pc->env0, Lr0.ptr, pc->err.as<int>() + 4, cs, ev, &nl));
    DG_TRY(build_streams(DGASM_FP64, P.env0, pc->env0, Lr0, Lc0, Lb0, cs, &nl, keep));
    // A_0^{-1} = columns of the local-solve kernel applied to the identity
    DG_TRY(pc->A0inv.alloc(sizeof(double) * (size_t)n0 * n0));
    DG_TRY(pc->coarse_inverse(scale0, Lb0, Lc0, cs, keep, &coarse_err));
    nl += 3;
    for (DevBuf* b : {&d_gt, &d_gw, &d_aggbox, &A0, &scale0, &Lb0, &Lc0}) keep.add(std::move(*b));
    pc->nn = R0TPairs{};
  }
  if (!pc->blocks) {
    if (fprec == DGASM_TF32 || fprec == DGASM_BF16) {
      // breakdown of the tensor-core factorisation (a non-positive pivot): factorise again from A_i with the
      // FP32 CUDA-core updates
      int herr[3];
      DG_CUDA(cudaMemcpyAsync(herr, pc->err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, st));
      DG_CUDA(cudaStreamSynchronize(st));
      if (herr[0]) {
        const int err0[3] = {0, -1, -1};
        DG_CUDA(cudaMemcpyAsync(pc->err.ptr, err0, sizeof(err0), cudaMemcpyHostToDevice, st));
        DG_CUDA(cudaMemsetAsync(Lf.ptr, 0, Lf.bytes, st));
        DG_CUDA(launch_extract_rows(1, pc->env.dev, pc->sub_e0.as<int>(), pc->rowptr.as<int>(), pc->col.as<int>(),
                                    pc->vals.as<double>(), np, np2s, pc->scale.as<double>(), Lf.ptr, P.nsub, ne, st));
        DG_TRY(factor_env(DGASM_FP32, P.env, pc->env, Lf.ptr, pc->err.as<int>(), st, ev, &nl));
        pc->tc_fallback = 1;
        nl += 1;
      }
    }
    // super-row inverse blocks, then the forward (column-major) and backward (row-major) solve streams
    DG_TRY(build_streams(fprec, P.env, pc->env, Lf, pc->Lc, pc->Lr, st, &nl, keep));
  }
  if (pc->n0 > 0) {
    DG_CUDA(cudaEventRecord(pc->ev_join, cs));
    DG_CUDA(cudaStreamWaitEvent(st, pc->ev_join, 0));
  }
  // check factorisation errors
  int herr[8];
  int cerr = 0;
  DG_CUDA(cudaMemcpyAsync(herr, pc->err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, st));
  if (coarse_err) DG_CUDA(cudaMemcpyAsync(&cerr, coarse_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (herr[0]) return set_error(DGASM_ENOTSPD, "non-positive pivot in the Cholesky factor of subdomain %d at row %d", herr[1], herr[2]);
  if (herr[4]) return set_error(DGASM_ENOTSPD, "non-positive pivot in the Cholesky factor of the coarse operator A_0");
  if (herr[3]) return set_error(DGASM_ETIMEOUT, "a tensor-core trailing update did not complete within its wait limit");
  if (cerr) return set_error(DGASM_ECUDA, "a bounded wait in the coarse inverse gave up (error word set)");
  if (ev) ev->accumulate();
  pc->setup_launches = nl;
  pc->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - pc->t_start).count();
  if (defer) {   // every stream of this setup has finished: the buffers are idle, their release is the caller's
    for (auto& b : keep.bufs) defer->add(std::move(b));
    keep.bufs.clear();
    defer->add(std::move(Lf));
    defer->add(std::move(pc->src_blk));
  }
  pc->src_blk.reset();
  return DGASM_OK;
}

}  // namespace dgasm

extern "C" int dgasm_setup(dgasm_system_t s, const dgasm_setup_opts* o, dgasm_prec_t* out) {
  clear_error();
  if (!out) return set_error(DGASM_EINVAL, "dgasm_setup: out is NULL");
  *out = nullptr;
  std::unique_ptr<dgasm_prec_s> pc;
  DG_TRY(prec_plan(s, o, pc));
  DG_TRY(prec_build(pc.get()));
  *out = pc.release();
  return DGASM_OK;
}

extern "C" int dgasm_setup_batch(int n, const dgasm_system_t* systems, const dgasm_setup_opts* const* opts,
                                 dgasm_prec_t* out) {
  clear_error();
  if (n < 1 || !systems || !opts || !out) return set_error(DGASM_EINVAL, "dgasm_setup_batch: bad arguments");
  for (int i = 0; i < n; ++i) out[i] = nullptr;
  for (int i = 0; i < n; ++i)
    if (!systems[i] || !opts[i]) return set_error(DGASM_EINVAL, "dgasm_setup_batch: NULL entry %d", i);
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  std::vector<std::unique_ptr<dgasm_prec_s>> pcs(n);
  std::vector<SetupTemps> temps(n);   // released after the last setup has finished
  std::vector<int> rc(n, DGASM_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  std::atomic<bool> failed{false};
  // each worker takes the next problem: its host plan (loops run on the worker itself, nested in this job)
  // and its device work on the problem's own streams, so plans and device work of different problems overlap
  const int width = std::min(n, pool_width());
  parallel_for(width, [&](int) {
    if (cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return;
    }
    for (int i = next.fetch_add(1); i < n && !failed.load(); i = next.fetch_add(1)) {
      int r = prec_plan(systems[i], opts[i], pcs[i]);
      if (r == DGASM_OK) r = prec_build(pcs[i].get(), &temps[i]);
      if (r != DGASM_OK) {
        char buf[512];
        dgasm_last_error(buf, sizeof(buf));
        rc[i] = r;
        msg[i] = buf;
        pcs[i].reset();
        failed = true;
      }
    }
  });
  temps.clear();
  for (int i = 0; i < n; ++i)
    if (rc[i] != DGASM_OK) {
      pcs.clear();
      return set_error(rc[i], "dgasm_setup_batch: problem %d: %s", i, msg[i].c_str());
    }
  if (failed.load()) {
    pcs.clear();
    return set_error(DGASM_ECUDA, "dgasm_setup_batch: a worker thread could not select device %d", dev);
  }
  for (int i = 0; i < n; ++i) out[i] = pcs[i].release();
  return DGASM_OK;
}


// ---- dgasm_prec_s members ----------------------------------------------------------------------------
int dgasm_prec_s::init_streams(void* user_stream) {
  if (user_stream) {
    stream = (cudaStream_t)user_stream;
  } else {
    DG_CUDA(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
    stream = own_stream;
  }
  DG_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
  DG_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  DG_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  return DGASM_OK;
}

dgasm_prec_s::~dgasm_prec_s() {
  engine.reset();
  if (side) cudaStreamDestroy(side);
  if (own_stream) cudaStreamDestroy(own_stream);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
}

// asynchronous on st; its temporaries go to `keep`, and *err_word is the device word its bounded waits set
int dgasm_prec_s::coarse_inverse(DevBuf& scale0, DevBuf& Lr0, DevBuf& Lc0, cudaStream_t st, SetupTemps& keep, int** err_word) {
  const int n0 = this->n0;
  // a one-subdomain problem with n0 right-hand sides: the unit vectors
  DevBuf ident, sub_e0c, misc, probs, prefix;
  DG_TRY(ident.alloc(sizeof(double) * (size_t)n0 * n0));
  DG_CUDA(launch_identity(ident.as<double>(), n0, st));
  std::vector<int> se{0, 1};
  DG_TRY(upload(sub_e0c, se));
  const int chunks = (n0 + KC - 1) / KC;
  const size_t rz_off = (sizeof(int) * (n0 + 2) + 15) & ~(size_t)15;
  DG_TRY(misc.alloc(rz_off + sizeof(double) * (size_t)n0));
  DG_CUDA(cudaMemsetAsync(misc.ptr, 0, misc.bytes, st));
  ProbDev D;
  std::memset(&D, 0, sizeof(D));
  D.np = n0; D.ndof = n0; D.nsub = 1; D.k = n0; D.kc = KC; D.n_rhs_chunks = chunks; D.prec = DGASM_FP64;
  D.sub_e0 = sub_e0c.as<int>(); D.sub_trow = env0.sub_trow.as<int>(); D.trow_F = env0.trow_F.as<int>();
  D.trow_ptr = env0.trow_ptr.as<long long>(); D.fwd_ptr = env0.fwd_ptr.as<long long>();
  D.bwd_ptr = env0.bwd_ptr.as<long long>();
  D.sr = P.env0.sr;
  D.sub_sr = env0.sub_sr.as<int>(); D.fwd_run = env0.fwd_run.as<int>(); D.bwd_run = env0.bwd_run.as<int>();
  D.Lr = Lr0.ptr; D.Lc = Lc0.ptr; D.scale = scale0.as<double>();
  D.fwd_total = (long long)P.env0.fwd_src.size();
  D.bwd_total = (long long)P.env0.bwd_src.size();
  D.r = ident.as<double>(); D.z = A0inv.as<double>();
  D.done = (int*)misc.ptr;
  D.part_rz = (double*)((char*)misc.ptr + rz_off);
  std::vector<ProbDev> hp{D};
  DG_TRY(probs.alloc(sizeof(ProbDev)));
  DG_CUDA(cudaMemcpyAsync(probs.ptr, hp.data(), sizeof(ProbDev), cudaMemcpyHostToDevice, st));
  std::vector<int> pre{0, chunks};
  DG_TRY(prefix.alloc(sizeof(int) * 2));
  DG_CUDA(cudaMemcpyAsync(prefix.ptr, pre.data(), sizeof(int) * 2, cudaMemcpyHostToDevice, st));
  BatchDev B;
  std::memset(&B, 0, sizeof(B));
  B.probs = probs.as<ProbDev>();
  B.nprob = 1;
  B.err = (int*)misc.ptr + n0;
  const int slot = K_NKINDS + 2 * DGASM_FP64 + 1;
  B.prefix[slot] = prefix.as<int>();
  DG_CUDA(launch_local(B, slot, chunks, local_smem_bytes(DGASM_FP64, n0, KC), st));
  *err_word = B.err;
  for (DevBuf* b : {&ident, &sub_e0c, &misc, &probs, &prefix}) keep.add(std::move(*b));
  return DGASM_OK;
}

namespace dgasm {

// explicit inverses: at most this many dofs per subdomain and this many bytes in all
constexpr int DLI_MAX_N = 2048;
constexpr size_t DLI_MAX_BYTES = size_t(1) << 30;
constexpr int DLI_CB = 64;   // unit vectors per pass of the local-solve kernel

bool dli_candidate(const dgasm_prec_s& pc) {
  if (pc.blocks || pc.P.nsub < 1) return false;
  const size_t eb = pc.precision == DGASM_FP64 ? 8 : 4;
  size_t bytes = 0;
  for (int s = 0; s < pc.P.nsub; ++s) {
    const size_t n = (size_t)pc.P.env.ndof[s];
    if (n > (size_t)DLI_MAX_N) return false;
    bytes += n * n * eb;
  }
  return bytes <= DLI_MAX_BYTES;
}

// X_s = A_s^{-1} for every subdomain: the local-solve kernel (the sweeps with the envelope factors, in the
// factor precision) applied to DLI_CB unit vectors per subdomain at a time, each result column stored into X_s
int build_dli(dgasm_prec_s* pc) {
  if (pc->dli.ptr) return DGASM_OK;
  if (!dli_candidate(*pc)) return set_error(DGASM_EINVAL, "explicit local inverses: subdomains too large (at most %d "
                                                          "dofs each and %zu bytes in all)", DLI_MAX_N, DLI_MAX_BYTES);
  const Plan& P = pc->P;
  const int nsub = P.nsub, np = P.np;
  const long long ndof = (long long)P.ne * np;
  const bool fp64 = pc->precision == DGASM_FP64;
  const size_t eb = fp64 ? 8 : 4;
  cudaStream_t st = pc->stream;
  std::vector<long long> off(nsub + 1, 0);
  std::vector<int> items;
  int nmax = 0;
  for (int s = 0; s < nsub; ++s) {
    const int n = P.env.ndof[s];
    nmax = std::max(nmax, n);
    off[s + 1] = off[s] + (long long)n * n;
    for (int r0 = 0; r0 < n; r0 += DLI_ROWS) { items.push_back(s); items.push_back(r0); }
  }
  DevBuf X, offs, item, r, z, misc, probs, prefix;
  DG_TRY(X.alloc((size_t)off[nsub] * eb));
  DG_TRY(upload(offs, off));
  DG_TRY(upload(item, items));
  DG_TRY(r.alloc(sizeof(double) * (size_t)DLI_CB * ndof));
  DG_TRY(z.alloc(sizeof(double) * (size_t)DLI_CB * ndof));
  // done flags [DLI_CB], error word, partial (r, z) [nsub][DLI_CB]
  const size_t rz_off = (sizeof(int) * (DLI_CB + 2) + 15) & ~(size_t)15;
  DG_TRY(misc.alloc(rz_off + sizeof(double) * (size_t)nsub * DLI_CB));
  DG_CUDA(cudaMemsetAsync(misc.ptr, 0, misc.bytes, st));
  const int chunks = DLI_CB / KC;
  ProbDev D;
  std::memset(&D, 0, sizeof(D));
  D.ne = P.ne; D.np = np; D.np2s = pc->sys->np2s; D.ndof = (int)ndof; D.nsub = nsub; D.k = DLI_CB; D.kc = KC;
  D.n_rhs_chunks = chunks; D.prec = pc->precision;
  D.sub_e0 = pc->sub_e0.as<int>(); D.sub_trow = pc->env.sub_trow.as<int>(); D.trow_F = pc->env.trow_F.as<int>();
  D.trow_ptr = pc->env.trow_ptr.as<long long>(); D.fwd_ptr = pc->env.fwd_ptr.as<long long>();
  D.bwd_ptr = pc->env.bwd_ptr.as<long long>();
  D.sr = P.env.sr;
  D.sub_sr = pc->env.sub_sr.as<int>(); D.fwd_run = pc->env.fwd_run.as<int>(); D.bwd_run = pc->env.bwd_run.as<int>();
  D.Lr = pc->Lr.ptr; D.Lc = pc->Lc.ptr; D.scale = pc->scale.as<double>();
  D.fwd_total = (long long)P.env.fwd_src.size();
  D.bwd_total = (long long)P.env.bwd_src.size();
  D.r = r.as<double>(); D.z = z.as<double>();
  D.done = (int*)misc.ptr;
  D.part_rz = (double*)((char*)misc.ptr + rz_off);
  DG_TRY(probs.alloc(sizeof(ProbDev)));
  DG_CUDA(cudaMemcpyAsync(probs.ptr, &D, sizeof(ProbDev), cudaMemcpyHostToDevice, st));
  std::vector<int> pre{0, nsub * chunks};
  DG_TRY(upload(prefix, pre));
  BatchDev B;
  std::memset(&B, 0, sizeof(B));
  B.probs = probs.as<ProbDev>();
  B.nprob = 1;
  B.err = (int*)misc.ptr + DLI_CB;
  const int slot = K_NKINDS + 2 * pc->precision + 1;
  B.prefix[slot] = prefix.as<int>();
  for (int c0 = 0; c0 < nmax; c0 += DLI_CB) {
    DG_CUDA(cudaMemsetAsync(r.ptr, 0, r.bytes, st));
    DG_CUDA(launch_unit_block(pc->sub_e0.as<int>(), nsub, np, c0, DLI_CB, ndof, r.as<double>(), st));
    DG_CUDA(launch_local(B, slot, nsub * chunks, local_smem_bytes(pc->precision, nmax, KC), st));
    DG_CUDA(launch_dli_store(fp64 ? 1 : 0, pc->sub_e0.as<int>(), nsub, np, offs.as<long long>(), c0, DLI_CB, ndof,
                             z.as<double>(), X.ptr, nmax, st));
  }
  int herr = 0;
  DG_CUDA(cudaMemcpyAsync(&herr, B.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (herr) return set_error(DGASM_ECUDA, "a bounded wait while forming the explicit local inverses gave up");
  pc->dli = std::move(X);
  pc->dli_off = std::move(offs);
  pc->dli_item = std::move(item);
  pc->n_dli_items = (int)(items.size() / 2);
  pc->dli_nmax = nmax;
  return DGASM_OK;
}

}  // namespace dgasm

size_t dgasm_prec_s::footprint() const {
  size_t b = perm.bytes + rowptr.bytes + col.bytes + vals.bytes + sub_e0.bytes + scale.bytes + Lr.bytes + Lc.bytes +
             grp_ptr.bytes + grp_elems.bytes + agg_int.bytes + r0t.bytes + A0inv.bytes + err.bytes + dinv.bytes +
             r0t_ptr.bytes + r0t_col.bytes + r0t_elem.bytes + rT_ptr.bytes + rT_pair.bytes + dli.bytes + dli_off.bytes +
             dli_item.bytes;
  const EnvBufs* es[2] = {&env, &env0};
  for (const EnvBufs* e : es)
    b += e->ndof.bytes + e->sub_trow.bytes + e->trow_F.bytes + e->trow_ptr.bytes + e->diag_task.bytes +
         e->panel_task.bytes + e->upd_task.bytes + e->tc_task.bytes + e->bwd_src.bytes + e->fwd_src.bytes + e->fwd_ptr.bytes +
         e->bwd_ptr.bytes + e->dinv_task.bytes + e->dinv_ptr.bytes + e->sub_sr.bytes + e->fwd_run.bytes + e->bwd_run.bytes;
  return b;
}

extern "C" int dgasm_prec_partition(dgasm_prec_t pc, int* sub, int* agg) {
  if (!pc) return set_error(DGASM_EINVAL, "NULL preconditioner");
  if (sub) std::copy(pc->P.sub_of.begin(), pc->P.sub_of.end(), sub);
  if (agg && !pc->P.agg_of.empty()) std::copy(pc->P.agg_of.begin(), pc->P.agg_of.end(), agg);
  return DGASM_OK;
}

extern "C" int dgasm_prec_footprint(dgasm_prec_t pc, int64_t* bytes) {
  if (!pc || !bytes) return set_error(DGASM_EINVAL, "NULL argument");
  *bytes = (int64_t)pc->footprint();
  return DGASM_OK;
}

extern "C" int dgasm_prec_info(dgasm_prec_t pc, dgasm_prec_info_t* info) {
  if (!pc || !info) return set_error(DGASM_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  const Plan& P = pc->P;
  info->nsub = P.nsub;
  info->nagg = P.nagg;
  info->n0 = pc->n0;
  info->precision = pc->precision;
  info->local_dofs = (int64_t)P.ne * P.np;
  info->local_tiles = P.env.ntiles;
  info->stream_tiles = pc->blocks ? 0 : (int64_t)(P.env.fwd_src.size() + P.env.bwd_src.size());
  int64_t upd = (int64_t)P.env.upd_task.size() / 3, pan = (int64_t)P.env.panel_task.size() / 2, dg = (int64_t)P.env.diag_task.size();
  const int64_t t3 = (int64_t)TILE * TILE * TILE;
  info->factor_flops = upd * 2 * t3 + pan * t3 + dg * (t3 / 3 + t3 / 3);
  info->nnzb = (int64_t)P.col.size();
  info->plan_ms = pc->plan_ms;
  info->setup_ms = pc->setup_ms;
  info->setup_launches = pc->setup_launches;
  info->tc_fallback = pc->tc_fallback;
  return DGASM_OK;
}

extern "C" int dgasm_prec_destroy(dgasm_prec_t pc) {
  delete pc;
  return DGASM_OK;
}

// One trailing-update step on the tensor cores for a dense lower tile matrix (Sec. 3, local solvers: the
// update C_IJ -= L_I0 L_J0^T of step 0 of the tile Cholesky), for tests of the tcgen05 kernel.
namespace {
int selftest_tc(int n, const float* tiles, float* out, int bf16) {
  using namespace dgasm;
  clear_error();
  if (n < 1 || n > 64 || !tiles || !out) return set_error(DGASM_EINVAL, "dgasm_selftest_tc_update: need 1 <= n <= 64 and buffers");
  // one subdomain of n + 1 tile rows, every row reaching column 0: the envelope is the full lower triangle
  std::vector<std::vector<int>> first_col(1, std::vector<int>((size_t)(n + 1) * TILE, 0));
  Envelope E;
  E.build(first_col, 8);
  EnvBufs D;
  DG_TRY(upload_env(E, D));
  const size_t bytes = (size_t)E.ntiles * TILE * TILE * sizeof(float);
  DevBuf L, err;
  DG_TRY(L.alloc(bytes));
  DG_TRY(err.alloc(4 * sizeof(int)));
  DG_CUDA(cudaMemcpy(L.ptr, tiles, bytes, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemset(err.ptr, 0, 4 * sizeof(int)));
  int rc = launch_chol_update_tc(D.dev, L.as<float>(), 0, D.panel_task.as<int>(), D.tc_task.as<int>() + 4 * (size_t)E.tc_off[0],
                                 E.tc_off[1] - E.tc_off[0], err.as<int>(), nullptr, bf16);
  if (rc) return cuda_error(rc, "tensor-core update self-test launch");
  DG_CUDA(cudaDeviceSynchronize());
  int h[4];
  DG_CUDA(cudaMemcpy(h, err.ptr, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[3]) return set_error(DGASM_ETIMEOUT, "a tensor-core trailing update did not complete within its wait limit");
  DG_CUDA(cudaMemcpy(out, L.ptr, bytes, cudaMemcpyDeviceToHost));
  return DGASM_OK;
}
}  // namespace

extern "C" int dgasm_selftest_tc_update(int n, const float* tiles, float* out) { return selftest_tc(n, tiles, out, 0); }

extern "C" int dgasm_selftest_tc_update_bf16(int n, const float* tiles, float* out) { return selftest_tc(n, tiles, out, 1); }

