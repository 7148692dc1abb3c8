// Preconditioner handle and batched-solve state (host side).
#pragma once

#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "plan.h"

namespace dgasm {

struct EnvBufs {
  DevBuf ndof, sub_trow, trow_F, trow_ptr, diag_task, panel_task, upd_task;
  EnvDev dev{};
};

// Krylov state of one problem, carved from one device allocation; grows on demand.
struct Workspace {
  DevBuf buf;
  int k = 0, maxit = 0;
  int n_chunk_items = 0, n_coarse_items = 0;
  size_t o_vec = 0, o_coarse = 0, o_scal = 0, o_int = 0, o_hist = 0, o_ppq = 0, o_prr = 0, o_prz = 0, o_pc = 0, o_cnt = 0;
  int ensure(const dgasm_prec_s& pc, int k, int maxit);
  void fill(const dgasm_prec_s& pc, ProbDev& D, int k, const double* b_user, double* x_user, int maxit, int fixed,
            double rtol) const;
};

struct BatchState {
  DevBuf tables;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int* h_remaining = nullptr;
  int launches = 0;
  float ms = 0.f;
  BatchState();
  ~BatchState();
};

int run_batch(int nprob, dgasm_prec_s* const* pcs, const int* nrhs, const double* const* b, double* const* x,
              const dgasm_solve_opts* o, dgasm_stats* st, BatchState& S, bool apply_only);

}  // namespace dgasm

struct dgasm_prec_s {
  dgasm_system_s* sys = nullptr;
  dgasm::Plan P;
  int precision = DGASM_FP64;
  int n0 = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  dgasm::DevBuf perm, rowptr, col, vals, src_blk, sub_e0, scale, Lr, Lc, grp_ptr, grp_elems, agg_int, r0t, A0inv, err, io;
  dgasm::EnvBufs env, env0;
  dgasm::Workspace ws;
  dgasm::BatchState bstate;
  std::mutex mu;
  int init_streams(void* user_stream);
  int coarse_inverse(dgasm::DevBuf& scale0, dgasm::DevBuf& Lr0, dgasm::DevBuf& Lc0);
  size_t footprint() const;
  ~dgasm_prec_s();
};
