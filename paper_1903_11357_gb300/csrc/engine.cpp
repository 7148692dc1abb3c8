// Batched ASPCG driver (Sec. 7): prepares the descriptor tables of a batch of problems, runs the
// initial residual and preconditioner application, then PCG iterations as captured CUDA graphs of
// CHUNK iterations until every right-hand side meets its stop test, and finally the true residual.
// Also the C entry points dgasm_solve, dgasm_solve_batch, dgasm_prec_apply and dgasm_system_spmv.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "plan.h"
#include "profile.h"
#include "solver.h"

namespace dgasm {

// ---- workspace of one problem for k right-hand sides ------------------------------------------
int Workspace::ensure(const dgasm_prec_s& pc, int k_, int maxit_, cudaStream_t stream) {
  // partial (r, z) sums: one per subdomain, element chunk (element blocks) or explicit-inverse item
  const int need_rz = std::max(pc.P.nsub, std::max(pc.n_dli_items, (pc.P.ne + NTHREADS / pc.P.np - 1) / (NTHREADS / pc.P.np)));
  if (k_ <= k && maxit_ <= maxit && need_rz <= n_rz_cap && buf.ptr) return DGASM_OK;
  n_rz_cap = need_rz;
  k = std::max(k_, k);
  maxit = std::max(maxit_, maxit);
  const Plan& P = pc.P;
  const long long ndof = (long long)P.ne * P.np;
  const int n0 = pc.n0;
  const int epi = NTHREADS / P.np;
  n_chunk_items = (P.ne + epi - 1) / epi;
  const int epis = SPMV_THREADS / P.np;
  n_spmv_items = (P.ne + epis - 1) / epis;
  const int rows_per_item = COARSE_ROWS_PER_WARP * (NTHREADS / 32);
  n_coarse_items = n0 > 0 ? (n0 + rows_per_item - 1) / rows_per_item : 0;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  o_vec = take(sizeof(double) * 6 * k * ndof);
  o_coarse = take(sizeof(double) * 2 * k * std::max(n0, 1));
  o_scal = take(sizeof(double) * 6 * k);
  o_int = take(sizeof(int) * 3 * k);
  o_hist = take(sizeof(double) * 2 * (size_t)k * maxit);
  o_ppq = take(sizeof(double) * (size_t)n_spmv_items * k);
  o_prr = take(sizeof(double) * (size_t)P.ngrp * k);
  o_prz = take(sizeof(double) * (size_t)n_rz_cap * k);
  o_pc = take(sizeof(double) * (size_t)std::max(n_coarse_items, 1) * k);
  o_cnt = take(sizeof(unsigned) * C_NCOUNTERS);
  DG_TRY(buf.alloc(off));
  DG_CUDA(cudaMemsetAsync(buf.ptr, 0, off, stream));
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
  D.epi_spmv = SPMV_THREADS / P.np;
  D.n_spmv_items = n_spmv_items;
  D.n_coarse_items = n_coarse_items;
  D.kc = kk > 1 ? (pc.rhs_chunk[kk] ? pc.rhs_chunk[kk] : KC) : 1;
  D.n_rhs_chunks = (kk + D.kc - 1) / D.kc;
  D.fixed_iters = fixed;
  D.rtol = rtol;
  D.rowptr = pc.rowptr.as<int>(); D.col = pc.col.as<int>(); D.vals = pc.vals.as<double>(); D.perm = pc.perm.as<int>();
  D.sub_e0 = pc.sub_e0.as<int>(); D.sub_trow = pc.env.sub_trow.as<int>(); D.trow_F = pc.env.trow_F.as<int>();
  D.trow_ptr = pc.env.trow_ptr.as<long long>(); D.fwd_ptr = pc.env.fwd_ptr.as<long long>();
  D.bwd_ptr = pc.env.bwd_ptr.as<long long>();
  D.sr = pc.P.env.sr;
  D.dinv = pc.blocks ? pc.dinv.as<double>() : nullptr;
  const bool inv = !pc.blocks && pc.local_variant == LV_INVERSE;
  D.n_rz = pc.blocks ? n_chunk_items : inv ? pc.n_dli_items : P.nsub;
  D.dli = inv ? pc.dli.ptr : nullptr;
  D.dli_off = inv ? pc.dli_off.as<long long>() : nullptr;
  D.dli_item = inv ? pc.dli_item.as<int>() : nullptr;
  D.n_dli_items = inv ? pc.n_dli_items : 0;
  D.sub_sr = pc.env.sub_sr.as<int>(); D.fwd_run = pc.env.fwd_run.as<int>(); D.bwd_run = pc.env.bwd_run.as<int>();
  D.Lr = pc.Lr.ptr; D.Lc = pc.Lc.ptr; D.scale = pc.scale.as<double>();
  D.fwd_total = (long long)pc.P.env.fwd_src.size();
  D.bwd_total = (long long)pc.P.env.bwd_src.size();
  D.grp_ptr = pc.grp_ptr.as<int>(); D.grp_elems = pc.grp_elems.as<int>(); D.agg_int = pc.agg_int.as<int>();
  D.r0t = pc.r0t.as<double>(); D.A0inv = pc.A0inv.as<double>();
  D.nc = P.nagg;
  if (P.nonnested && pc.n0 > 0) {
    D.r0t_ptr = pc.r0t_ptr.as<int>(); D.r0t_col = pc.r0t_col.as<int>(); D.r0t_elem = pc.r0t_elem.as<int>();
    D.rT_ptr = pc.rT_ptr.as<int>(); D.rT_pair = pc.rT_pair.as<int>();
  }
  D.b_user = b_user; D.x_user = x_user;
  double* v = (double*)(base + o_vec);
  D.b = v; D.x = v + k * ndof; D.r = v + 2 * k * ndof; D.p = v + 3 * k * ndof; D.q = v + 4 * k * ndof; D.z = v + 5 * k * ndof;
  double* c = (double*)(base + o_coarse);
  D.r0 = c; D.z0 = c + (size_t)k * std::max(pc.n0, 1);
  double* s = (double*)(base + o_scal);
  D.bnorm = s; D.gamma = s + k; D.alpha = s + 2 * k; D.relres = s + 3 * k; D.true_rr = s + 4 * k; D.gamma1 = s + 5 * k;
  int* iv = (int*)(base + o_int);
  D.done = iv; D.iters = iv + k; D.status = iv + 2 * k;
  double* h = (double*)(base + o_hist);
  D.alpha_hist = h; D.beta_hist = h + (size_t)k * maxit;
  D.maxit = std::min(maxit_, maxit);
  D.part_pq = (double*)(base + o_ppq); D.part_rr = (double*)(base + o_prr); D.part_rz = (double*)(base + o_prz);
  D.part_c = (double*)(base + o_pc); D.counters = (unsigned*)(base + o_cnt);
}

// ---- engine ----------------------------------------------------------------------------------------
Engine::Engine() {
  cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  cudaMallocHost((void**)&h_remaining, 2 * sizeof(int));
}

Engine::~Engine() {
  if (exec) cudaGraphExecDestroy(exec);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (side) cudaStreamDestroy(side);
  if (h_remaining) cudaFreeHost(h_remaining);
}

int Engine::build(int n, dgasm_prec_s* const* pcs_, const int* nrhs_, const double* const* b, double* const* x,
                  const dgasm_solve_opts* const* os, cudaStream_t st, int remaining) {
  if (n < 1) return set_error(DGASM_EINVAL, "empty batch");
  if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
  nprob = n;
  stream = st;
  pcs.assign(pcs_, pcs_ + n);
  nrhs.assign(nrhs_, nrhs_ + n);
  total_rhs = 0;
  km = 1;
  for (int i = 0; i < n; ++i) {
    if (nrhs[i] < 1 || nrhs[i] > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs[i], KMAX);
    total_rhs += nrhs[i];
    if (nrhs[i] > 1) km = KMAX;
  }
  hp.assign(n, ProbDev{});
  pre.assign(K_NSLOTS * (n + 1), 0);
  auto P_ = [&](int kind, int i) -> int& { return pre[kind * (n + 1) + i]; };
  std::fill(max_smem, max_smem + 8, 0);
  for (int i = 0; i < n; ++i) {
    dgasm_prec_s* pc = pcs[i];
    const dgasm_solve_opts* o = os ? os[i] : nullptr;
    const double rtol = (o && o->rtol > 0) ? o->rtol : 1e-8;
    const int maxit = (o && o->maxit > 0) ? o->maxit : 10000;
    const int fixed = o ? std::max(o->fixed_iters, 0) : 0;
    const int hist = fixed > 0 ? fixed : maxit;
    DG_TRY(pc->ws.ensure(*pc, nrhs[i], hist, st));
    pc->ws.fill(*pc, hp[i], nrhs[i], b[i], x[i], hist, fixed, rtol);
    const ProbDev& D = hp[i];
    for (int kind = 0; kind < K_NSLOTS; ++kind) P_(kind, i + 1) = P_(kind, i);
    P_(K_SPMV, i + 1) += D.n_chunk_items;
    P_(K_SPMV_P + pc->sys->p - 1, i + 1) += D.n_spmv_items;
    P_(K_GRP, i + 1) += D.ngrp;
    P_(K_COARSE, i + 1) += D.nq > 0 ? D.n_coarse_items : 0;
    P_(K_RNN, i + 1) += D.r0t_ptr ? D.nc : 0;
    if (pc->blocks) {
      P_(K_BJAC, i + 1) += D.n_chunk_items;
    } else if (D.dli) {
      P_(K_DLI + (D.prec == DGASM_FP64 ? 0 : 1), i + 1) += D.n_dli_items;
    } else {
      const int slot = 2 * D.prec + (D.kc > 1 ? 1 : 0);
      P_(K_NKINDS + slot, i + 1) += D.nsub * D.n_rhs_chunks;
      int maxn = 0;
      for (int sdx = 0; sdx < pc->P.nsub; ++sdx) maxn = std::max(maxn, pc->P.env.ndof[sdx]);
      max_smem[slot] = std::max(max_smem[slot], local_smem_bytes(D.prec, maxn, D.kc));
    }
  }
  tot_spmv = P_(K_SPMV, n);
  tot_grp = P_(K_GRP, n);
  tot_coarse = P_(K_COARSE, n);
  tot_rnn = P_(K_RNN, n);
  const size_t o_pre = sizeof(ProbDev) * n;
  const size_t o_rem = (o_pre + sizeof(int) * pre.size() + 15) & ~(size_t)15;
  const size_t tb = o_rem + 16;
  if (tables.bytes < tb) DG_TRY(tables.alloc(tb));
  char* tdev = (char*)tables.ptr;
  d_remaining = (int*)(tdev + o_rem);
  d_err = d_remaining + 1;
  for (auto& D : hp) D.remaining = d_remaining;
  std::memset(&B, 0, sizeof(B));
  B.probs = (const ProbDev*)tdev;
  B.nprob = n;
  B.err = d_err;
  for (int kind = 0; kind < K_NSLOTS; ++kind) B.prefix[kind] = (const int*)(tdev + o_pre) + kind * (n + 1);
  const int rem = remaining < 0 ? total_rhs : remaining;
  DG_CUDA(cudaMemcpyAsync(tdev, hp.data(), sizeof(ProbDev) * n, cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaMemcpyAsync(tdev + o_pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, stream));
  h_remaining[0] = rem;
  h_remaining[1] = 0;
  DG_CUDA(cudaMemcpyAsync(d_remaining, h_remaining, 2 * sizeof(int), cudaMemcpyHostToDevice, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  return DGASM_OK;
}

int Engine::reset_state() {
  for (int i = 0; i < nprob; ++i) {
    const ProbDev& D = hp[i];
    DG_CUDA(cudaMemsetAsync(D.done, 0, sizeof(int) * 3 * pcs[i]->ws.k, stream));
    DG_CUDA(cudaMemsetAsync(D.counters, 0, sizeof(unsigned) * C_NCOUNTERS, stream));
  }
  return DGASM_OK;
}

namespace {
template <typename F>
int timed_launch(int kind, cudaStream_t s, EventPairs* ev, long long& launches, F&& launch) {
  const bool prof = ev && profiling();
  int id = prof ? ev->begin(kind, s) : -1;
  int rc = launch();
  if (prof) ev->end(id, s);
  ++launches;
  return rc;
}
}  // namespace

int Engine::spmv(int operand, EventPairs* ev) {
  const int n = nprob;
  for (int p = 1; p <= 8; ++p) {
    const int tot = pre[(K_SPMV_P + p - 1) * (n + 1) + n];
    if (tot) DG_CUDA(timed_launch(PK_SPMV, stream, ev, launches, [&] { return launch_spmv(B, p, tot, operand, km, stream); }));
  }
  return DGASM_OK;
}

int Engine::precond(int mode, EventPairs* ev, int wslot) {
  const int n = nprob;
  if (tot_rnn)   // non-nested coarse spaces: r_0 = R_0 r before the coarse solve forks off
    DG_CUDA(timed_launch(PK_UPDATE, stream, ev, launches, [&] { return launch_restrict_nn(B, tot_rnn, km, stream); }));
  DG_CUDA(cudaEventRecord(ev_fork, stream));
  DG_CUDA(cudaStreamWaitEvent(side, ev_fork, 0));
  if (tot_coarse) DG_CUDA(timed_launch(PK_COARSE, side, ev, launches, [&] { return launch_coarse(B, tot_coarse, km, side); }));
  DG_CUDA(cudaEventRecord(ev_join, side));
  for (int slot = 0; slot < 8; ++slot) {
    const int tot = pre[(K_NKINDS + slot) * (n + 1) + n];
    if (tot)
      DG_CUDA(timed_launch(PK_LOCAL, stream, ev, launches,
                           [&] { return launch_local(B, K_NKINDS + slot, tot, max_smem[slot], stream); }));
  }
  const int tot_bjac = pre[K_BJAC * (n + 1) + n];
  if (tot_bjac)
    DG_CUDA(timed_launch(PK_LOCAL, stream, ev, launches, [&] { return launch_bjac(B, tot_bjac, km, stream); }));
  for (int slot = K_DLI; slot <= K_DLI + 1; ++slot) {
    const int tot = pre[slot * (n + 1) + n];
    if (tot) DG_CUDA(timed_launch(PK_LOCAL, stream, ev, launches, [&] { return launch_dli(B, slot, tot, km, stream); }));
  }
  DG_CUDA(cudaStreamWaitEvent(stream, ev_join, 0));
  DG_CUDA(timed_launch(PK_PUPDATE, stream, ev, launches, [&] { return launch_pupdate(B, tot_spmv, mode, km, tot_rnn > 0, wslot, stream); }));
  return DGASM_OK;
}

int Engine::init(bool x0) {
  init_ev.reset();
  for (int i = 0; i < nprob; ++i) pcs[i]->ws.lanczos_len.assign(pcs[i]->ws.k, -1);
  if (!x0) {
    DG_CUDA(timed_launch(PK_UPDATE, stream, &init_ev, launches, [&] { return launch_update(B, tot_grp, MODE_INIT, km, 0, stream); }));
  } else {
    DG_CUDA(timed_launch(PK_UPDATE, stream, &init_ev, launches, [&] { return launch_update(B, tot_grp, MODE_INIT_X0, km, 0, stream); }));
    // a zero right-hand side has the solution 0 whatever the initial guess
    for (int i = 0; i < nprob; ++i) {
      const ProbDev& D = hp[i];
      const int wk = pcs[i]->ws.k;
      std::vector<double> bn(wk);
      DG_CUDA(cudaMemcpyAsync(bn.data(), D.bnorm, sizeof(double) * wk, cudaMemcpyDeviceToHost, stream));
      DG_CUDA(cudaStreamSynchronize(stream));
      for (int kk = 0; kk < nrhs[i]; ++kk)
        if (bn[kk] == 0.0) DG_CUDA(cudaMemsetAsync(D.x + (size_t)kk * D.ndof, 0, sizeof(double) * D.ndof, stream));
    }
    DG_TRY(spmv(1, &init_ev));
    DG_CUDA(timed_launch(PK_UPDATE, stream, &init_ev, launches, [&] { return launch_update(B, tot_grp, MODE_RESTART, km, 0, stream); }));
  }
  DG_TRY(precond(MODE_INIT, &init_ev, 0));
  return DGASM_OK;
}

int Engine::true_residual() { return spmv(1, &init_ev); }

int Engine::restart(int* count) {
  *count = 0;
  for (int i = 0; i < nprob; ++i) {
    const ProbDev& D = hp[i];
    if (D.fixed_iters > 0) continue;
    const int wk = pcs[i]->ws.k;
    std::vector<double> sc(5 * (size_t)wk);
    std::vector<int> iv(3 * (size_t)wk);
    DG_CUDA(cudaMemcpyAsync(sc.data(), D.bnorm, sizeof(double) * 5 * wk, cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaMemcpyAsync(iv.data(), D.done, sizeof(int) * 3 * wk, cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    bool any = false;
    for (int kk = 0; kk < nrhs[i]; ++kk) {
      const double true_rr = sc[4 * (size_t)wk + kk];
      if (iv[kk] == 1 && true_rr > D.rtol && iv[wk + kk] < D.maxit && std::isfinite(true_rr)) {
        std::vector<int>& ll = pcs[i]->ws.lanczos_len;
        if ((int)ll.size() < wk) ll.resize(wk, -1);
        if (ll[kk] < 0) ll[kk] = iv[wk + kk];
        iv[kk] = 0;
        any = true;
        ++*count;
      }
    }
    if (any) DG_CUDA(cudaMemcpyAsync(D.done, iv.data(), sizeof(int) * wk, cudaMemcpyHostToDevice, stream));
  }
  if (*count == 0) return DGASM_OK;
  h_remaining[0] = *count;
  h_remaining[1] = 0;
  DG_CUDA(cudaMemcpyAsync(d_remaining, h_remaining, 2 * sizeof(int), cudaMemcpyHostToDevice, stream));
  DG_CUDA(timed_launch(PK_UPDATE, stream, &init_ev, launches, [&] { return launch_update(B, tot_grp, MODE_RESTART, km, 0, stream); }));
  DG_TRY(precond(MODE_INIT, &init_ev, 0));
  return DGASM_OK;
}

int Engine::iterate(int max_iters, int* ran) {
  if (ran) *ran = 0;
  if (!exec) {
    graph_ev.reset();
    if (profiling()) graph_ev.reserve(CHUNK * 12);
    cudaGraph_t graph = nullptr;
    DG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    const long long before = launches;
    int rc = 0;
    // gamma alternates between two slots: the p update of iteration it reads slot it % 2 and writes the other,
    // the x/r update of iteration it reads slot it % 2 (CHUNK is even, and the initial p update writes slot 0)
    static_assert(CHUNK % 2 == 0, "the gamma slots must line up from one graph launch to the next");
    for (int it = 0; it < CHUNK && rc == 0; ++it) {
      const int gs = it & 1;
      rc = spmv(0, &graph_ev);
      if (!rc) rc = timed_launch(PK_UPDATE, stream, &graph_ev, launches, [&] { return launch_update(B, tot_grp, MODE_ITER, km, gs, stream); });
      if (!rc) {
        int r3 = precond(MODE_ITER, &graph_ev, gs ^ 1);
        if (r3 < 0) rc = r3;
      }
    }
    cudaError_t ce = cudaStreamEndCapture(stream, &graph);
    per_iter_launches = (int)((launches - before) / CHUNK);
    launches = before;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc < 0 ? rc : cuda_error(rc, "kernel launch during capture");
    }
    if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
    rc = (int)cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (rc) { exec = nullptr; return cuda_error(rc, "cudaGraphInstantiate"); }
  }
  const int max_chunks = (max_iters + CHUNK - 1) / CHUNK;
  for (int c = 0; c < max_chunks; ++c) {
    DG_CUDA(cudaGraphLaunch(exec, stream));
    DG_CUDA(cudaMemcpyAsync(h_remaining, d_remaining, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    launches += (long long)CHUNK * per_iter_launches;
    if (h_remaining[1]) return set_error(DGASM_ECUDA, "a bounded wait in the local-solve kernel gave up (error word set)");
    if (ran) *ran += CHUNK;
    if (profiling()) graph_ev.accumulate();
    if (*h_remaining <= 0) break;
  }
  return DGASM_OK;
}

int Engine::finish() {
  DG_CUDA(launch_finish(B, tot_spmv, 0, stream));
  ++launches;
  return DGASM_OK;
}

int Engine::apply_out() {
  DG_CUDA(launch_finish(B, tot_spmv, 1, stream));
  ++launches;
  return DGASM_OK;
}

int Engine::read_done(std::vector<int>& done, int* not_done_rhs) {
  done.assign(nprob, 0);
  int open_rhs = 0;
  int tmp[KMAX];
  for (int i = 0; i < nprob; ++i) {
    DG_CUDA(cudaMemcpyAsync(tmp, hp[i].done, sizeof(int) * nrhs[i], cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    int all = 1;
    for (int kk = 0; kk < nrhs[i]; ++kk) {
      all &= tmp[kk] != 0;
      open_rhs += tmp[kk] == 0;
    }
    done[i] = all;
  }
  if (not_done_rhs) *not_done_rhs = open_rhs;
  return DGASM_OK;
}

int Engine::collect(dgasm_stats* st, double ms, std::vector<int>* rcs) {
  int worst = DGASM_OK;
  int r = 0;
  if (rcs) rcs->assign(nprob, DGASM_OK);
  for (int i = 0; i < nprob; ++i) {
    const ProbDev& D = hp[i];
    const int fixed = D.fixed_iters;
    const double rtol = D.rtol;
    int prc = DGASM_OK;
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
      s.launches = (int)launches;
      s.lambda_min = s.lambda_max = s.kappa = NAN;
      int nh = std::min(iters, D.maxit);
      // after a residual replacement the coefficients of the first CG run give the Lanczos estimate
      const std::vector<int>& ll = pcs[i]->ws.lanczos_len;
      if (kk < (int)ll.size() && ll[kk] >= 0) nh = std::min(nh, ll[kk]);
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
      if (status == DGASM_ENAN) prc = DGASM_ENAN;
      else if (done == 2 && prc == DGASM_OK) prc = DGASM_ENOCONV;
    }
    if (rcs) (*rcs)[i] = prc;
    if (prc == DGASM_ENAN) worst = DGASM_ENAN;
    else if (prc == DGASM_ENOCONV && worst == DGASM_OK) worst = DGASM_ENOCONV;
  }
  if (worst == DGASM_ENAN) return set_error(DGASM_ENAN, "NaN/Inf in the right-hand side or a Krylov scalar (breakdown)");
  if (worst == DGASM_ENOCONV) return set_error(DGASM_ENOCONV, "the iteration limit was reached before the tolerance");
  return DGASM_OK;
}

constexpr int MAX_RESTARTS = 4;

// One complete solve of a batch: init, iterate until done, true residual (and residual replacement where
// it misses the tolerance), x out, statistics.
int solve_all(Engine& E, int n, dgasm_prec_s* const* pcs, const int* nrhs, const double* const* b, double* const* x,
              const dgasm_solve_opts* o, cudaStream_t stream, dgasm_stats* st) {
  const int maxit = (o && o->maxit > 0) ? o->maxit : 10000;
  const int fixed = o ? std::max(o->fixed_iters, 0) : 0;
  E.launches = 0;
  std::vector<const dgasm_solve_opts*> os(n, o);
  DG_TRY(E.build(n, pcs, nrhs, b, x, os.data(), stream, -1));
  DG_TRY(E.reset_state());
  DG_CUDA(cudaEventRecord(E.ev0, stream));
  DG_TRY(E.init(o && o->x0_given));
  int ran = 0;
  DG_TRY(E.iterate((fixed > 0 ? fixed : maxit) + Engine::CHUNK, &ran));
  DG_TRY(E.true_residual());
  // the recursion's residual can drift from b - A x by rounding: continue from the true residual until
  // both meet rtol (a few restarts at most)
  for (int round = 0; round < MAX_RESTARTS; ++round) {
    int nre = 0;
    DG_TRY(E.restart(&nre));
    if (nre == 0) break;
    DG_TRY(E.iterate(maxit + Engine::CHUNK, &ran));
    DG_TRY(E.true_residual());
  }
  DG_TRY(E.finish());
  DG_CUDA(cudaEventRecord(E.ev1, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  if (profiling()) E.init_ev.accumulate();
  float ms = 0.f;
  cudaEventElapsedTime(&ms, E.ev0, E.ev1);
  return E.collect(st, ms, nullptr);
}

}  // namespace dgasm

using namespace dgasm;

// ---- C entry points --------------------------------------------------------------------------------
namespace dgasm {

// z = B r with the engine of the preconditioner (internal: the caller holds pc->mu)
int apply_locked(dgasm_prec_s* pc, int nrhs, const double* r, double* z, cudaStream_t stream) {
  if (!pc->engine) pc->engine.reset(new (std::nothrow) Engine());
  if (!pc->engine) return set_error(DGASM_ENOMEM, "host allocation failed");
  dgasm_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.maxit = 1;
  dgasm_prec_s* arr[1] = {pc};
  const double* bb[1] = {r};
  double* xx[1] = {z};
  Engine& E = *pc->engine;
  const dgasm_solve_opts* os[1] = {&o};
  DG_TRY(E.build(1, arr, &nrhs, bb, xx, os, stream, -1));
  DG_TRY(E.reset_state());
  // a zero right-hand side is finished by the initial step, and p keeps its old contents: clear it
  DG_CUDA(cudaMemsetAsync(E.hp[0].p, 0, sizeof(double) * (size_t)pc->ws.k * pc->P.ne * pc->P.np, stream));
  DG_TRY(E.init());
  DG_TRY(E.apply_out());
  return DGASM_OK;
}

// The local-solve kernel can give each CTA pair 1 or KC right-hand sides.  KC reads each factor once for KC
// vectors; 1 gives KC times as many CTA pairs, which wins when there are few subdomains.  The choice is
// measured once per (preconditioner, k): one warm-up and two timed applications of b per candidate.  Both
// choices add the same products in the same order for every right-hand side, so the solution does not
// depend on the outcome (tested bitwise).
int tune_rhs_chunk(dgasm_prec_s* pc, int nrhs, const double* b, cudaStream_t stream) {
  if (nrhs <= 1 || pc->rhs_chunk[nrhs] != 0 || pc->blocks) return DGASM_OK;
  const size_t n = (size_t)pc->P.ne * pc->P.np * nrhs;
  DevBuf z;
  DG_TRY(z.alloc(n * sizeof(double)));
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  const int cand[2] = {KC, 1};
  float best = 0.f;
  int pick = KC, rc = DGASM_OK;
  for (int c = 0; c < 2 && rc == DGASM_OK; ++c) {
    pc->rhs_chunk[nrhs] = cand[c];
    rc = apply_locked(pc, nrhs, b, z.as<double>(), stream);
    if (rc) break;
    cudaEventRecord(e0, stream);
    for (int r = 0; r < 2 && rc == DGASM_OK; ++r) rc = apply_locked(pc, nrhs, b, z.as<double>(), stream);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_error((int)cudaGetLastError(), "right-hand-side chunk tuning");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c == 0 || ms < best) { best = ms; pick = cand[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pc->rhs_chunk[nrhs] = rc == DGASM_OK ? pick : 0;
  return rc;
}

// The local solves of a preconditioner whose subdomains are small enough can use explicit inverses (one
// dense matrix-vector product per subdomain) instead of the forward/backward sweeps.  The first solve
// measures both on b (one warm-up and two timed preconditioner applications each) and keeps the faster; the
// inverses are freed again if the sweeps win.  Both give the same solution up to rounding.
// The outcome is kept per shape (precision, n_p, subdomain count, largest subdomain in steps of 128 dofs,
// right-hand sides), so that a stream of similar problems measures once.
namespace {
std::mutex g_variant_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_variant;
}  // namespace

int tune_local_variant(dgasm_prec_s* pc, int nrhs, const double* b, cudaStream_t stream) {
  if (pc->blocks || pc->local_variant != LV_TUNE) return DGASM_OK;
  if (!dli_candidate(*pc)) {
    pc->local_variant = LV_SWEEPS;
    return DGASM_OK;
  }
  int nmax = 0;
  for (int s = 0; s < pc->P.nsub; ++s) nmax = std::max(nmax, pc->P.env.ndof[s]);
  const auto key = std::make_tuple(pc->precision, pc->P.np, pc->P.nsub, (nmax + 127) / 128, nrhs);
  {
    std::lock_guard<std::mutex> lk(g_variant_mu);
    auto it = g_variant.find(key);
    if (it != g_variant.end()) {
      if (it->second == LV_INVERSE) DG_TRY(build_dli(pc));
      pc->local_variant = it->second;
      return DGASM_OK;
    }
  }
  DG_TRY(build_dli(pc));
  const size_t n = (size_t)pc->P.ne * pc->P.np * nrhs;
  DevBuf z;
  DG_TRY(z.alloc(n * sizeof(double)));
  cudaEvent_t e0, e1;
  DG_CUDA(cudaEventCreate(&e0));
  DG_CUDA(cudaEventCreate(&e1));
  const int cand[2] = {LV_SWEEPS, LV_INVERSE};
  float best = 0.f;
  int pick = LV_SWEEPS, rc = DGASM_OK;
  for (int c = 0; c < 2 && rc == DGASM_OK; ++c) {
    pc->local_variant = cand[c];
    rc = apply_locked(pc, nrhs, b, z.as<double>(), stream);
    if (rc) break;
    cudaEventRecord(e0, stream);
    for (int r = 0; r < 2 && rc == DGASM_OK; ++r) rc = apply_locked(pc, nrhs, b, z.as<double>(), stream);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_error((int)cudaGetLastError(), "local-solve variant tuning");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c == 0 || ms < best) { best = ms; pick = cand[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pc->local_variant = rc == DGASM_OK ? pick : LV_TUNE;
  if (rc == DGASM_OK) {
    std::lock_guard<std::mutex> lk(g_variant_mu);
    g_variant[key] = pick;
  }
  if (pc->local_variant != LV_INVERSE) {
    pc->dli.reset();
    pc->dli_off.reset();
    pc->dli_item.reset();
    pc->n_dli_items = 0;
  }
  return rc;
}

}  // namespace dgasm

extern "C" int dgasm_prec_set_rhs_chunk(dgasm_prec_t pc, int nrhs, int kc) {
  clear_error();
  if (!pc || nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "dgasm_prec_set_rhs_chunk: bad arguments");
  if (kc != 0 && kc != 1 && kc != KC) return set_error(DGASM_EINVAL, "kc=%d must be 0 (tune), 1 or %d", kc, KC);
  std::lock_guard<std::mutex> lk(pc->mu);
  pc->rhs_chunk[nrhs] = kc;
  return DGASM_OK;
}

extern "C" int dgasm_prec_set_local_variant(dgasm_prec_t pc, int variant) {
  clear_error();
  if (!pc || variant < LV_TUNE || variant > LV_INVERSE)
    return set_error(DGASM_EINVAL, "dgasm_prec_set_local_variant: bad arguments");
  std::lock_guard<std::mutex> lk(pc->mu);
  if (pc->blocks) return variant == LV_INVERSE || variant == LV_TUNE ? DGASM_OK
                                                                    : set_error(DGASM_EINVAL, "element-block local solves have no sweeps");
  if (variant == LV_INVERSE) DG_TRY(build_dli(pc));
  pc->local_variant = variant;
  if (variant != LV_INVERSE) {
    pc->dli.reset();
    pc->dli_off.reset();
    pc->dli_item.reset();
    pc->n_dli_items = 0;
  }
  return DGASM_OK;
}

extern "C" int dgasm_prec_get_local_variant(dgasm_prec_t pc, int* variant) {
  clear_error();
  if (!pc || !variant) return set_error(DGASM_EINVAL, "dgasm_prec_get_local_variant: bad arguments");
  std::lock_guard<std::mutex> lk(pc->mu);
  *variant = pc->blocks ? LV_INVERSE : pc->local_variant;
  return DGASM_OK;
}

extern "C" int dgasm_prec_get_rhs_chunk(dgasm_prec_t pc, int nrhs, int* kc) {
  clear_error();
  if (!pc || !kc || nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "dgasm_prec_get_rhs_chunk: bad arguments");
  std::lock_guard<std::mutex> lk(pc->mu);
  *kc = nrhs == 1 ? 1 : pc->rhs_chunk[nrhs];
  return DGASM_OK;
}

extern "C" int dgasm_solve(dgasm_prec_t pc, int nrhs, const double* b, double* x, const dgasm_solve_opts* o,
                           dgasm_stats* st) {
  clear_error();
  if (!pc || !b || !x) return set_error(DGASM_EINVAL, "dgasm_solve: NULL argument");
  if (nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs, KMAX);
  std::lock_guard<std::mutex> lk(pc->mu);
  if (!pc->engine) pc->engine.reset(new (std::nothrow) Engine());
  if (!pc->engine) return set_error(DGASM_ENOMEM, "host allocation failed");
  cudaStream_t stream = (o && o->stream) ? (cudaStream_t)o->stream : pc->stream;
  dgasm_prec_s* arr[1] = {pc};
  if (o && o->host_buffers) {
    const size_t n = (size_t)pc->P.ne * pc->P.np * nrhs;
    if (pc->io.bytes < 2 * n * sizeof(double)) DG_TRY(pc->io.alloc(2 * n * sizeof(double)));
    double* db = pc->io.as<double>();
    double* dx = db + n;
    DG_CUDA(cudaMemcpyAsync(db, b, n * sizeof(double), cudaMemcpyHostToDevice, stream));
    if (o->x0_given) DG_CUDA(cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, stream));
    DG_TRY(tune_local_variant(pc, nrhs, db, stream));
    DG_TRY(tune_rhs_chunk(pc, nrhs, db, stream));
    const double* bb[1] = {db};
    double* xx[1] = {dx};
    int rc = solve_all(*pc->engine, 1, arr, &nrhs, bb, xx, o, stream, st);
    if (rc != DGASM_OK && rc != DGASM_ENOCONV) return rc;
    DG_CUDA(cudaMemcpyAsync(x, dx, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    DG_CUDA(cudaStreamSynchronize(stream));
    return rc;
  }
  DG_TRY(tune_local_variant(pc, nrhs, b, stream));
  DG_TRY(tune_rhs_chunk(pc, nrhs, b, stream));
  const double* bb[1] = {b};
  double* xx[1] = {x};
  return solve_all(*pc->engine, 1, arr, &nrhs, bb, xx, o, stream, st);
}

extern "C" int dgasm_solve_batch(int nprob, const dgasm_prec_t* pcs, const int* nrhs, const double* const* b,
                                 double* const* x, const dgasm_solve_opts* o, dgasm_stats* st) {
  clear_error();
  if (nprob < 1 || !pcs || !nrhs || !b || !x) return set_error(DGASM_EINVAL, "dgasm_solve_batch: bad arguments");
  if (o && o->host_buffers) return set_error(DGASM_EINVAL, "dgasm_solve_batch: device buffers only");
  for (int i = 0; i < nprob; ++i) {
    if (!pcs[i] || !b[i] || !x[i]) return set_error(DGASM_EINVAL, "dgasm_solve_batch: NULL entry %d", i);
    for (int j = 0; j < i; ++j)
      if (pcs[j] == pcs[i]) return set_error(DGASM_EINVAL, "dgasm_solve_batch: preconditioner %d appears twice", i);
  }
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int i = 0; i < nprob; ++i) locks.emplace_back(pcs[i]->mu);
  static thread_local std::unique_ptr<Engine> eng;
  if (!eng) eng.reset(new (std::nothrow) Engine());
  if (!eng) return set_error(DGASM_ENOMEM, "host allocation failed");
  cudaStream_t stream = (o && o->stream) ? (cudaStream_t)o->stream : pcs[0]->stream;
  for (int i = 0; i < nprob; ++i) DG_TRY(tune_local_variant(pcs[i], nrhs[i], b[i], stream));
  return solve_all(*eng, nprob, pcs, nrhs, b, x, o, stream, st);
}

extern "C" int dgasm_prec_apply(dgasm_prec_t pc, int nrhs, const double* r, double* z, void* stream_) {
  clear_error();
  if (!pc || !r || !z) return set_error(DGASM_EINVAL, "dgasm_prec_apply: NULL argument");
  if (nrhs < 1 || nrhs > KMAX) return set_error(DGASM_EINVAL, "nrhs=%d must lie in [1, %d]", nrhs, KMAX);
  std::lock_guard<std::mutex> lk(pc->mu);
  cudaStream_t stream = stream_ ? (cudaStream_t)stream_ : pc->stream;
  DG_TRY(apply_locked(pc, nrhs, r, z, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
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

extern "C" int dgasm_selftest_bounded_wait(double limit_ms, int* gave_up, double* elapsed_ms) {
  using namespace dgasm;
  clear_error();
  if (!gave_up || !(limit_ms > 0.0) || limit_ms > 1000.0)
    return set_error(DGASM_EINVAL, "dgasm_selftest_bounded_wait: need gave_up and 0 < limit_ms <= 1000");
  int dev = 0, khz = 0;
  DG_CUDA(cudaGetDevice(&dev));
  DG_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long limit = (long long)(limit_ms * (double)khz);   // cycles at the reported SM clock
  DevBuf err;
  DG_TRY(err.alloc(2 * sizeof(int)));
  DG_CUDA(cudaMemset(err.ptr, 0, 2 * sizeof(int)));
  cudaEvent_t a, b;
  DG_CUDA(cudaEventCreate(&a));
  DG_CUDA(cudaEventCreate(&b));
  cudaEventRecord(a, nullptr);
  int rc = launch_wait_selftest(err.as<int>(), limit, nullptr);
  cudaEventRecord(b, nullptr);
  cudaError_t se = cudaEventSynchronize(b);
  float ms = 0.f;
  if (rc == 0 && se == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return cuda_error(rc, "bounded-wait self-test launch");
  if (se != cudaSuccess) return cuda_error((int)se, "bounded-wait self-test");
  int h[2] = {0, 0};
  DG_CUDA(cudaMemcpy(h, err.ptr, sizeof(h), cudaMemcpyDeviceToHost));
  *gave_up = (h[0] == 1 && h[1] == 1) ? 1 : 0;
  if (elapsed_ms) *elapsed_ms = ms;
  return DGASM_OK;
}
