// Host orchestration: dgasm_setup (partition, device extraction and factorisation of the A_i, coarse
// space), dgasm_solve / dgasm_solve_batch (batched ASPCG under captured CUDA graphs, Sec. 7) and
// dgasm_prec_apply.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "plan.h"
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
  D.dev.nsub = E.nsub;
  D.dev.ndof = D.ndof.as<int>();
  D.dev.sub_trow = D.sub_trow.as<int>();
  D.dev.trow_F = D.trow_F.as<int>();
  D.dev.trow_ptr = D.trow_ptr.as<long long>();
  return DGASM_OK;
}

// factor the tile pool Lr (row-major, factor precision) in place, step by step
int factor_env(int prec, const Envelope& E, EnvBufs& D, void* Lr, int* err, cudaStream_t st) {
  for (int K = 0; K < E.max_nbt; ++K) {
    int nd = E.diag_off[K + 1] - E.diag_off[K];
    int npn = E.panel_off[K + 1] - E.panel_off[K];
    int nu = E.upd_off[K + 1] - E.upd_off[K];
    int rc = launch_chol_step(prec == DGASM_FP64 ? 0 : 1, D.dev, Lr, K, D.diag_task.as<int>() + E.diag_off[K], nd,
                              D.panel_task.as<int>() + 2 * (size_t)E.panel_off[K], npn,
                              D.upd_task.as<int>() + 3 * (size_t)E.upd_off[K], nu, err, st);
    if (rc) return cuda_error(rc, "tile Cholesky step");
  }
  return DGASM_OK;
}

}  // namespace

// ---- workspace of one problem for k right-hand sides ------------------------------------------
int Workspace::ensure(const dgasm_prec_s& pc, int k_, int maxit_) {
  if (k_ <= k && maxit_ <= maxit && buf.ptr) return DGASM_OK;
  k = std::max(k_, k);
  maxit = std::max(maxit_, maxit);
  const Plan& P = pc.P;
  const long long ndof = (long long)P.ne * P.np;
  const int n0 = pc.n0;
  const int epi = NTHREADS / P.np;
  n_chunk_items = (P.ne + epi - 1) / epi;
  n_coarse_items = n0 > 0 ? (n0 + 7) / 8 : 0;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  o_vec = take(sizeof(double) * 6 * k * ndof);
  o_coarse = take(sizeof(double) * 2 * k * std::max(n0, 1));
  o_scal = take(sizeof(double) * 5 * k);
  o_int = take(sizeof(int) * 3 * k);
  o_hist = take(sizeof(double) * 2 * (size_t)k * maxit);
  o_ppq = take(sizeof(double) * (size_t)n_chunk_items * k);
  o_prr = take(sizeof(double) * (size_t)P.ngrp * k);
  o_prz = take(sizeof(double) * (size_t)P.nsub * k);
  o_pc = take(sizeof(double) * (size_t)std::max(n_coarse_items, 1) * k);
  o_cnt = take(sizeof(unsigned) * C_NCOUNTERS);
  DG_TRY(buf.alloc(off));
  DG_CUDA(cudaMemset(buf.ptr, 0, off));
  return DGASM_OK;
}

void Workspace::fill(const dgasm_prec_s& pc, ProbDev& D, int kk, const double* b_user, double* x_user, int maxit_,
                     int fixed, double rtol) const {
  const Plan& P = pc.P;
  const long long ndof = (long long)P.ne * P.np;
  char* base = (char*)buf.ptr;
  std::memset(&D, 0, sizeof(D));
  D.ne = P.ne; D.np = P.np; D.np2s = pc.sys->np2s; D.nq = pc.n0 > 0 ? P.nq : 0; D.ndof = (int)ndof;
  D.nsub = P.nsub; D.ngrp = P.ngrp; D.n0 = pc.n0; D.k = kk; D.prec = pc.precision;
  D.epi = NTHREADS / P.np;
  D.n_chunk_items = n_chunk_items;
  D.n_coarse_items = n_coarse_items;
  D.kc = kk > 1 ? KC : 1;
  D.n_rhs_chunks = (kk + D.kc - 1) / D.kc;
  D.maxit = maxit_;
  D.fixed_iters = fixed;
  D.rtol = rtol;
  D.rowptr = pc.rowptr.as<int>(); D.col = pc.col.as<int>(); D.vals = pc.vals.as<double>(); D.perm = pc.perm.as<int>();
  D.sub_e0 = pc.sub_e0.as<int>(); D.sub_trow = pc.env.sub_trow.as<int>(); D.trow_F = pc.env.trow_F.as<int>();
  D.trow_ptr = pc.env.trow_ptr.as<long long>(); D.Lr = pc.Lr.ptr; D.Lc = pc.Lc.ptr; D.scale = pc.scale.as<double>();
  D.grp_ptr = pc.grp_ptr.as<int>(); D.grp_elems = pc.grp_elems.as<int>(); D.agg_int = pc.agg_int.as<int>();
  D.r0t = pc.r0t.as<double>(); D.A0inv = pc.A0inv.as<double>();
  D.b_user = b_user; D.x_user = x_user;
  double* v = (double*)(base + o_vec);
  D.b = v; D.x = v + k * ndof; D.r = v + 2 * k * ndof; D.p = v + 3 * k * ndof; D.q = v + 4 * k * ndof; D.z = v + 5 * k * ndof;
  double* c = (double*)(base + o_coarse);
  D.r0 = c; D.z0 = c + (size_t)k * std::max(pc.n0, 1);
  double* s = (double*)(base + o_scal);
  D.bnorm = s; D.gamma = s + k; D.alpha = s + 2 * k; D.relres = s + 3 * k; D.true_rr = s + 4 * k;
  int* iv = (int*)(base + o_int);
  D.done = iv; D.iters = iv + k; D.status = iv + 2 * k;
  double* h = (double*)(base + o_hist);
  D.alpha_hist = h; D.beta_hist = h + (size_t)k * maxit;
  D.maxit = std::min(maxit_, maxit);
  D.part_pq = (double*)(base + o_ppq); D.part_rr = (double*)(base + o_prr); D.part_rz = (double*)(base + o_prz);
  D.part_c = (double*)(base + o_pc); D.counters = (unsigned*)(base + o_cnt);
}

}  // namespace dgasm

// ---- setup ---------------------------------------------------------------------------------------
extern "C" int dgasm_setup(dgasm_system_t s, const dgasm_setup_opts* o, dgasm_prec_t* out) {
  clear_error();
  if (!out) return set_error(DGASM_EINVAL, "dgasm_setup: out is NULL");
  *out = nullptr;
  if (!s || !o) return set_error(DGASM_EINVAL, "dgasm_setup: NULL argument");
  if (o->precision < DGASM_FP64 || o->precision > DGASM_BF16) return set_error(DGASM_EINVAL, "unknown precision %d", o->precision);
  const bool coarse = o->ncoarse > 0 || o->agg_of_elem;
  if (coarse && (o->p_c < 1 || o->p_c > s->p)) return set_error(DGASM_EINVAL, "p_c=%d must lie in [1, p=%d]", o->p_c, s->p);
  std::unique_ptr<dgasm_prec_s> pc(new (std::nothrow) dgasm_prec_s());
  if (!pc) return set_error(DGASM_ENOMEM, "host allocation failed");
  pc->sys = s;
  pc->precision = o->precision;
  DG_TRY(s->ensure_device());
  DG_TRY(pc->init_streams(o->stream));
  Plan& P = pc->P;
  DG_TRY(build_plan(*s, o->nsub, o->ncoarse, coarse ? o->p_c : 1, o->sub_of_elem, o->agg_of_elem, P));
  pc->n0 = P.nagg * P.nq;
  cudaStream_t st = pc->stream;
  const int ne = P.ne, np = P.np, np2s = s->np2s;
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
  DG_TRY(pc->scale.alloc(sizeof(double) * (size_t)ne * np));
  DG_CUDA(launch_scale(pc->rowptr.as<int>(), pc->col.as<int>(), pc->vals.as<double>(), ne, np, np2s, pc->scale.as<double>(), st));
  // local factors
  const int fprec = pc->precision;
  const size_t ftiles = (size_t)P.env.ntiles * TILE * TILE;
  DevBuf Lf;  // factorisation pool (row-major)
  DG_TRY(Lf.alloc(ftiles * fact_elem_bytes(fprec)));
  DG_CUDA(cudaMemsetAsync(Lf.ptr, 0, Lf.bytes, st));
  DG_CUDA(launch_extract_rows(fprec == DGASM_FP64 ? 0 : 1, pc->env.dev, pc->sub_e0.as<int>(), pc->rowptr.as<int>(),
                              pc->col.as<int>(), pc->vals.as<double>(), np, np2s, pc->scale.as<double>(), Lf.ptr,
                              P.nsub, ne, st));
  DG_TRY(factor_env(fprec, P.env, pc->env, Lf.ptr, pc->err.as<int>(), st));
  if (fprec == DGASM_BF16) {
    DevBuf Lcf;
    DG_TRY(Lcf.alloc(ftiles * 4));
    DG_CUDA(launch_to_colmajor(1, Lf.ptr, Lcf.ptr, P.env.ntiles, st));
    DG_TRY(pc->Lr.alloc(ftiles * 2));
    DG_TRY(pc->Lc.alloc(ftiles * 2));
    DG_CUDA(launch_to_bf16(Lf.as<float>(), pc->Lr.ptr, (long long)ftiles, st));
    DG_CUDA(launch_to_bf16(Lcf.as<float>(), pc->Lc.ptr, (long long)ftiles, st));
    DG_CUDA(cudaStreamSynchronize(st));
  } else {
    DG_TRY(pc->Lc.alloc(ftiles * fact_elem_bytes(fprec)));
    DG_CUDA(launch_to_colmajor(fprec == DGASM_FP64 ? 0 : 1, Lf.ptr, pc->Lc.ptr, P.env.ntiles, st));
    pc->Lr = std::move(Lf);
  }
  // coarse space: R_0^T, A_0 = R_0 A R_0^T, FP64 factor and explicit inverse
  if (pc->n0 > 0) {
    const int n0 = pc->n0, q = P.q, nq = P.nq, mq = s->p + 2;
    std::vector<double> gt, gw;
    gauss_legendre01(mq, gt, gw);
    DevBuf d_gt, d_gw, d_aggbox;
    DG_TRY(upload(d_gt, gt));
    DG_TRY(upload(d_gw, gw));
    DG_TRY(upload(d_aggbox, P.agg_bbox));
    DG_TRY(pc->r0t.alloc(sizeof(double) * (size_t)ne * np * nq));
    DG_CUDA(launch_r0t(pc->perm.as<int>(), s->d_xy.as<double>(), s->d_pptr.as<int>(), s->d_pvtx.as<int>(),
                       s->d_bbox.as<double>(), pc->agg_int.as<int>(), d_aggbox.as<double>(), ne, s->p, q,
                       d_gt.as<double>(), d_gw.as<double>(), mq, pc->r0t.as<double>(), st));
    DevBuf A0;
    DG_TRY(A0.alloc(sizeof(double) * (size_t)n0 * n0));
    DG_CUDA(cudaMemsetAsync(A0.ptr, 0, A0.bytes, st));
    DG_CUDA(launch_galerkin(pc->grp_ptr.as<int>(), pc->grp_elems.as<int>(), pc->agg_int.as<int>(), pc->rowptr.as<int>(),
                            pc->col.as<int>(), pc->vals.as<double>(), pc->r0t.as<double>(), P.nagg, np, np2s, nq,
                            A0.as<double>(), st));
    DG_TRY(upload_env(P.env0, pc->env0));
    DevBuf scale0, Lr0, Lc0;
    DG_TRY(scale0.alloc(sizeof(double) * n0));
    const size_t t0 = (size_t)P.env0.ntiles * TILE * TILE;
    DG_TRY(Lr0.alloc(sizeof(double) * t0));
    DG_CUDA(cudaMemsetAsync(Lr0.ptr, 0, Lr0.bytes, st));
    DG_CUDA(launch_coarse_extract(A0.as<double>(), n0, scale0.as<double>(), pc->env0.dev, Lr0.as<double>(), st));
    DG_TRY(factor_env(DGASM_FP64, P.env0, pc->env0, Lr0.ptr, pc->err.as<int>() + 4, st));
    DG_TRY(Lc0.alloc(sizeof(double) * t0));
    DG_CUDA(launch_to_colmajor(0, Lr0.ptr, Lc0.ptr, P.env0.ntiles, st));
    // A_0^{-1} = columns of the local-solve kernel applied to the identity
    DG_TRY(pc->A0inv.alloc(sizeof(double) * (size_t)n0 * n0));
    DG_TRY(pc->coarse_inverse(scale0, Lr0, Lc0));
  }
  // check factorisation errors
  int herr[8];
  DG_CUDA(cudaMemcpyAsync(herr, pc->err.ptr, sizeof(herr), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (herr[0]) return set_error(DGASM_ENOTSPD, "non-positive pivot in the Cholesky factor of subdomain %d at row %d", herr[1], herr[2]);
  if (herr[4]) return set_error(DGASM_ENOTSPD, "non-positive pivot in the Cholesky factor of the coarse operator A_0");
  pc->src_blk.reset();
  *out = pc.release();
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
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (side) cudaStreamDestroy(side);
  if (own_stream) cudaStreamDestroy(own_stream);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
}

int dgasm_prec_s::coarse_inverse(DevBuf& scale0, DevBuf& Lr0, DevBuf& Lc0) {
  const int n0 = this->n0;
  cudaStream_t st = stream;
  // a one-subdomain problem with n0 right-hand sides: the unit vectors
  DevBuf ident, sub_e0c, misc, probs, prefix;
  DG_TRY(ident.alloc(sizeof(double) * (size_t)n0 * n0));
  DG_CUDA(launch_identity(ident.as<double>(), n0, st));
  std::vector<int> se{0, 1};
  DG_TRY(upload(sub_e0c, se));
  const int chunks = (n0 + KC - 1) / KC;
  DG_TRY(misc.alloc(sizeof(int) * n0 + sizeof(double) * (size_t)n0));
  DG_CUDA(cudaMemsetAsync(misc.ptr, 0, misc.bytes, st));
  ProbDev D;
  std::memset(&D, 0, sizeof(D));
  D.np = n0; D.ndof = n0; D.nsub = 1; D.k = n0; D.kc = KC; D.n_rhs_chunks = chunks; D.prec = DGASM_FP64;
  D.sub_e0 = sub_e0c.as<int>(); D.sub_trow = env0.sub_trow.as<int>(); D.trow_F = env0.trow_F.as<int>();
  D.trow_ptr = env0.trow_ptr.as<long long>(); D.Lr = Lr0.ptr; D.Lc = Lc0.ptr; D.scale = scale0.as<double>();
  D.r = ident.as<double>(); D.z = A0inv.as<double>();
  D.done = (int*)misc.ptr;
  D.part_rz = (double*)((char*)misc.ptr + sizeof(int) * n0);
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
  const int slot = K_NKINDS + 2 * DGASM_FP64 + 1;
  B.prefix[slot] = prefix.as<int>();
  DG_CUDA(launch_local(B, slot, chunks, local_smem_bytes(DGASM_FP64, n0, KC), st));
  DG_CUDA(cudaStreamSynchronize(st));
  return DGASM_OK;
}

size_t dgasm_prec_s::footprint() const {
  size_t b = perm.bytes + rowptr.bytes + col.bytes + vals.bytes + sub_e0.bytes + scale.bytes + Lr.bytes + Lc.bytes +
             grp_ptr.bytes + grp_elems.bytes + agg_int.bytes + r0t.bytes + A0inv.bytes + err.bytes;
  const EnvBufs* es[2] = {&env, &env0};
  for (const EnvBufs* e : es)
    b += e->ndof.bytes + e->sub_trow.bytes + e->trow_F.bytes + e->trow_ptr.bytes + e->diag_task.bytes +
         e->panel_task.bytes + e->upd_task.bytes;
  return b;
}

// ---- batched solve -------------------------------------------------------------------------------
namespace dgasm {

int run_batch(int nprob, dgasm_prec_s* const* pcs, const int* nrhs, const double* const* b, double* const* x,
              const dgasm_solve_opts* o, dgasm_stats* st, BatchState& S, bool apply_only) {
  if (nprob < 1) return set_error(DGASM_EINVAL, "empty batch");
  const double rtol = (o && o->rtol > 0) ? o->rtol : 1e-8;
  const int maxit = (o && o->maxit > 0) ? o->maxit : 10000;
  const int fixed = o ? std::max(o->fixed_iters, 0) : 0;
  const int hist = fixed > 0 ? std::max(fixed, 1) : maxit;
  cudaStream_t stream = pcs[0]->stream;
  if (o && o->stream) stream = (cudaStream_t)o->stream;
  cudaStream_t side = pcs[0]->side;
  int total_rhs = 0;
  for (int i = 0; i < nprob; ++i) {
    if (nrhs[i] < 1 || nrhs[i] > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs[i], KMAX);
    total_rhs += nrhs[i];
  }
  // workspaces and descriptors
  std::vector<ProbDev> hp(nprob);
  std::vector<int> pre((K_NKINDS + 8) * (nprob + 1), 0);
  auto P_ = [&](int kind, int i) -> int& { return pre[kind * (nprob + 1) + i]; };
  int max_smem[8] = {0};
  for (int i = 0; i < nprob; ++i) {
    dgasm_prec_s* pc = pcs[i];
    DG_TRY(pc->ws.ensure(*pc, nrhs[i], hist));
    pc->ws.fill(*pc, hp[i], nrhs[i], b[i], x[i], hist, fixed, rtol);
    const ProbDev& D = hp[i];
    for (int kind = 0; kind < K_NKINDS + 8; ++kind) P_(kind, i + 1) = P_(kind, i);
    P_(K_SPMV, i + 1) += D.n_chunk_items;
    P_(K_GRP, i + 1) += D.ngrp;
    P_(K_COARSE, i + 1) += D.nq > 0 ? D.n_coarse_items : 0;
    const int slot = K_NKINDS + 2 * D.prec + (D.kc > 1 ? 1 : 0);
    P_(slot, i + 1) += D.nsub * D.n_rhs_chunks;
    int maxn = 0;
    for (int sdx = 0; sdx < pc->P.nsub; ++sdx) maxn = std::max(maxn, pc->P.env.ndof[sdx]);
    max_smem[slot - K_NKINDS] = std::max(max_smem[slot - K_NKINDS], local_smem_bytes(D.prec, maxn, D.kc));
  }
  // device tables: [ProbDev x nprob][prefix][remaining]
  const size_t tb = sizeof(ProbDev) * nprob + sizeof(int) * pre.size() + 64;
  if (S.tables.bytes < tb) DG_TRY(S.tables.alloc(tb));
  char* tdev = (char*)S.tables.ptr;
  int* d_pre = (int*)(tdev + sizeof(ProbDev) * nprob);
  int* d_remaining = (int*)(tdev + ((sizeof(ProbDev) * nprob + sizeof(int) * pre.size() + 15) & ~(size_t)15));
  for (auto& D : hp) D.remaining = d_remaining;
  BatchDev B;
  std::memset(&B, 0, sizeof(B));
  B.probs = (const ProbDev*)tdev;
  B.nprob = nprob;
  for (int kind = 0; kind < K_NKINDS + 8; ++kind) B.prefix[kind] = d_pre + kind * (nprob + 1);
  DG_CUDA(cudaMemcpyAsync(tdev, hp.data(), sizeof(ProbDev) * nprob, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(d_pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(d_remaining, &total_rhs, sizeof(int), cudaMemcpyHostToDevice, stream));
  for (int i = 0; i < nprob; ++i) {
    const ProbDev& D = hp[i];
    DG_CUDA(cudaMemsetAsync(D.done, 0, sizeof(int) * 3 * pcs[i]->ws.k, stream));
    DG_CUDA(cudaMemsetAsync(D.counters, 0, sizeof(unsigned) * C_NCOUNTERS, stream));
  }
  const int tot_spmv = P_(K_SPMV, nprob), tot_grp = P_(K_GRP, nprob), tot_coarse = P_(K_COARSE, nprob);
  cudaEvent_t e0 = S.ev0, e1 = S.ev1;
  DG_CUDA(cudaEventRecord(e0, stream));
  S.launches = 0;
  // the preconditioner application z = B r, shared by the initial step and every iteration
  auto precond = [&](int mode) -> int {
    DG_CUDA(cudaEventRecord(pcs[0]->ev_fork, stream));
    DG_CUDA(cudaStreamWaitEvent(side, pcs[0]->ev_fork, 0));
    if (tot_coarse) { DG_CUDA(launch_coarse(B, tot_coarse, side)); ++S.launches; }
    DG_CUDA(cudaEventRecord(pcs[0]->ev_join, side));
    for (int slot = 0; slot < 8; ++slot) {
      const int tot = P_(K_NKINDS + slot, nprob);
      if (tot) { DG_CUDA(launch_local(B, K_NKINDS + slot, tot, max_smem[slot], stream)); ++S.launches; }
    }
    DG_CUDA(cudaStreamWaitEvent(stream, pcs[0]->ev_join, 0));
    DG_CUDA(launch_pupdate(B, tot_spmv, mode, stream));
    ++S.launches;
    return DGASM_OK;
  };
  DG_CUDA(launch_update(B, tot_grp, MODE_INIT, 0, stream));
  ++S.launches;
  DG_TRY(precond(MODE_INIT));
  if (apply_only) {
    DG_CUDA(launch_finish(B, tot_spmv, 1, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return DGASM_OK;
  }
  // iterations: CHUNK per captured graph, until every right-hand side is done
  const int CHUNK = 8;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  int per_iter_launches = 0;
  {
    int before = S.launches;
    for (int it = 0; it < CHUNK; ++it) {
      int rc1 = launch_spmv(B, tot_spmv, 0, stream);
      int rc2 = launch_update(B, tot_grp, MODE_ITER, 0, stream);
      S.launches += 2;
      int rc3 = precond(MODE_ITER);
      if (rc1 || rc2 || rc3 < 0) {
        cudaStreamEndCapture(stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        return rc3 < 0 ? rc3 : cuda_error(rc1 ? rc1 : rc2, "kernel launch during capture");
      }
    }
    per_iter_launches = (S.launches - before) / CHUNK;
    S.launches = before;
  }
  DG_CUDA(cudaStreamEndCapture(stream, &graph));
  int rc = (int)cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (rc) return cuda_error(rc, "cudaGraphInstantiate");
  int* h_rem = S.h_remaining;
  const int max_chunks = (std::max(fixed, maxit) + CHUNK - 1) / CHUNK + 1;
  int nchunks = 0;
  for (; nchunks < max_chunks; ++nchunks) {
    rc = (int)cudaGraphLaunch(exec, stream);
    if (rc) break;
    rc = (int)cudaMemcpyAsync(h_rem, d_remaining, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (rc) break;
    rc = (int)cudaStreamSynchronize(stream);
    if (rc) break;
    if (*h_rem <= 0) { ++nchunks; break; }
  }
  cudaGraphExecDestroy(exec);
  if (rc) return cuda_error(rc, "graph launch");
  S.launches += nchunks * CHUNK * per_iter_launches;
  // true residual and caller-order solution
  DG_CUDA(launch_spmv(B, tot_spmv, 1, stream));
  DG_CUDA(launch_finish(B, tot_spmv, 0, stream));
  S.launches += 2;
  DG_CUDA(cudaEventRecord(e1, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  S.ms = ms;
  // statistics
  int worst = DGASM_OK;
  int r = 0;
  for (int i = 0; i < nprob; ++i) {
    const ProbDev& D = hp[i];
    const int k = nrhs[i];
    const int wk = pcs[i]->ws.k;
    std::vector<double> sc(5 * (size_t)wk);
    std::vector<int> iv(3 * (size_t)wk);
    DG_CUDA(cudaMemcpy(sc.data(), D.bnorm, sizeof(double) * 5 * wk, cudaMemcpyDeviceToHost));
    DG_CUDA(cudaMemcpy(iv.data(), D.done, sizeof(int) * 3 * wk, cudaMemcpyDeviceToHost));
    for (int kk = 0; kk < k; ++kk, ++r) {
      const int done = iv[kk], iters = iv[wk + kk], status = iv[2 * wk + kk];
      dgasm_stats s;
      std::memset(&s, 0, sizeof(s));
      s.iters = iters;
      s.relres = sc[3 * (size_t)wk + kk];
      s.true_relres = sc[4 * (size_t)wk + kk];
      s.converged = fixed > 0 ? (s.relres <= rtol) : (done == 1);
      s.solve_ms = ms;
      s.lambda_min = s.lambda_max = s.kappa = NAN;
      const int nh = std::min(iters, D.maxit);
      if (nh >= 1) {
        std::vector<double> al(nh), be(std::max(nh - 1, 1));
        DG_CUDA(cudaMemcpy(al.data(), D.alpha_hist + (size_t)kk * D.maxit, sizeof(double) * nh, cudaMemcpyDeviceToHost));
        if (nh > 1)
          DG_CUDA(cudaMemcpy(be.data(), D.beta_hist + (size_t)kk * D.maxit, sizeof(double) * (nh - 1), cudaMemcpyDeviceToHost));
        double lo, hi;
        if (dgasm_lanczos(nh, al.data(), be.data(), &lo, &hi) == DGASM_OK) {
          s.lambda_min = lo;
          s.lambda_max = hi;
          s.kappa = hi / lo;
        }
        clear_error();
      }
      if (st) st[r] = s;
      if (status == DGASM_ENAN) worst = DGASM_ENAN;
      else if (done == 2 && worst == DGASM_OK) worst = DGASM_ENOCONV;
    }
  }
  if (worst == DGASM_ENAN) return set_error(DGASM_ENAN, "NaN/Inf in the right-hand side or a Krylov scalar (breakdown)");
  if (worst == DGASM_ENOCONV) return set_error(DGASM_ENOCONV, "maxit=%d reached before rtol=%g", maxit, rtol);
  return DGASM_OK;
}

BatchState::BatchState() {
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaMallocHost((void**)&h_remaining, sizeof(int));
}
BatchState::~BatchState() {
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (h_remaining) cudaFreeHost(h_remaining);
}

}  // namespace dgasm

// ---- C entry points --------------------------------------------------------------------------------
extern "C" int dgasm_solve(dgasm_prec_t pc, int nrhs, const double* b, double* x, const dgasm_solve_opts* o,
                           dgasm_stats* st) {
  clear_error();
  if (!pc || !b || !x) return set_error(DGASM_EINVAL, "dgasm_solve: NULL argument");
  if (o && o->x0_given) return set_error(DGASM_EINVAL, "dgasm_solve: an initial guess is not supported (x0_given)");
  std::lock_guard<std::mutex> lk(pc->mu);
  if (o && o->host_buffers) {
    const size_t n = (size_t)pc->P.ne * pc->P.np * nrhs;
    if (nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs, KMAX);
    if (pc->io.bytes < 2 * n * sizeof(double)) DG_TRY(pc->io.alloc(2 * n * sizeof(double)));
    cudaStream_t stream = o->stream ? (cudaStream_t)o->stream : pc->stream;
    double* db = pc->io.as<double>();
    double* dx = db + n;
    DG_CUDA(cudaMemcpyAsync(db, b, n * sizeof(double), cudaMemcpyHostToDevice, stream));
    dgasm_prec_s* arr[1] = {pc};
    const double* bb[1] = {db};
    double* xx[1] = {dx};
    int rc = run_batch(1, arr, &nrhs, bb, xx, o, st, pc->bstate, false);
    if (rc != DGASM_OK && rc != DGASM_ENOCONV) return rc;
    DG_CUDA(cudaMemcpyAsync(x, dx, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return rc;
  }
  dgasm_prec_s* arr[1] = {pc};
  const double* bb[1] = {b};
  double* xx[1] = {x};
  return run_batch(1, arr, &nrhs, bb, xx, o, st, pc->bstate, false);
}

extern "C" int dgasm_solve_batch(int nprob, const dgasm_prec_t* pcs, const int* nrhs, const double* const* b,
                                 double* const* x, const dgasm_solve_opts* o, dgasm_stats* st) {
  clear_error();
  if (nprob < 1 || !pcs || !nrhs || !b || !x) return set_error(DGASM_EINVAL, "dgasm_solve_batch: bad arguments");
  if (o && (o->x0_given || o->host_buffers))
    return set_error(DGASM_EINVAL, "dgasm_solve_batch: device buffers and zero initial guesses only");
  for (int i = 0; i < nprob; ++i) {
    if (!pcs[i] || !b[i] || !x[i]) return set_error(DGASM_EINVAL, "dgasm_solve_batch: NULL entry %d", i);
    for (int j = 0; j < i; ++j)
      if (pcs[j] == pcs[i]) return set_error(DGASM_EINVAL, "dgasm_solve_batch: preconditioner %d appears twice", i);
  }
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int i = 0; i < nprob; ++i) locks.emplace_back(pcs[i]->mu);
  static thread_local BatchState bs;
  return run_batch(nprob, pcs, nrhs, b, x, o, st, bs, false);
}

extern "C" int dgasm_prec_apply(dgasm_prec_t pc, int nrhs, const double* r, double* z, void* stream) {
  clear_error();
  if (!pc || !r || !z) return set_error(DGASM_EINVAL, "dgasm_prec_apply: NULL argument");
  std::lock_guard<std::mutex> lk(pc->mu);
  dgasm_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.stream = stream;
  o.maxit = 1;
  dgasm_prec_s* arr[1] = {pc};
  const double* bb[1] = {r};
  double* xx[1] = {z};
  // a zero right-hand side is finished by the initial step: clear z so it reads zero
  const size_t n = (size_t)pc->P.ne * pc->P.np * nrhs;
  cudaStream_t st = stream ? (cudaStream_t)stream : pc->stream;
  DG_CUDA(cudaMemsetAsync(z, 0, n * sizeof(double), st));
  DG_TRY(pc->ws.ensure(*pc, nrhs, 1));
  DG_CUDA(cudaMemsetAsync((char*)pc->ws.buf.ptr + pc->ws.o_vec, 0, sizeof(double) * 6 * pc->ws.k * (size_t)pc->P.ne * pc->P.np, st));
  return run_batch(1, arr, &nrhs, bb, xx, &o, nullptr, pc->bstate, true);
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

extern "C" int dgasm_prec_destroy(dgasm_prec_t pc) {
  delete pc;
  return DGASM_OK;
}

extern "C" int dgasm_system_spmv(dgasm_system_t s, const double* x, double* y, void* stream) {
  clear_error();
  if (!s || !x || !y) return set_error(DGASM_EINVAL, "dgasm_system_spmv: NULL argument");
  DG_TRY(s->ensure_device());
  DG_CUDA(launch_system_spmv(s->d_rowptr.as<int>(), s->d_col.as<int>(), s->d_vals.as<double>(), s->mesh->m.ne, s->np,
                             s->np2s, x, y, stream));
  DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return DGASM_OK;
}
