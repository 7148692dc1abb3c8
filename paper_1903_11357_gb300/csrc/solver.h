// Preconditioner handle and batched-solve state (host side).
#pragma once

#include <chrono>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "engine.h"
#include "plan.h"
#include "profile.h"

namespace dgasm {

// Device buffers of a setup whose work may still be in flight, released together after the setup's final
// synchronisation (freeing one earlier would wait for the whole device).
struct SetupTemps {
  std::vector<DevBuf> bufs;
  void add(DevBuf&& b) { bufs.push_back(std::move(b)); }
};

struct EnvBufs {
  DevBuf ndof, sub_trow, trow_F, trow_ptr, diag_task, panel_task, upd_task, tc_task, bwd_src, fwd_src, fwd_ptr, bwd_ptr,
      dinv_task, dinv_ptr, sub_sr, fwd_run, bwd_run;
  EnvDev dev{};
};

// Krylov state of one problem, carved from one device allocation; grows on demand.
struct Workspace {
  DevBuf buf;
  int k = 0, maxit = 0;
  int n_chunk_items = 0, n_spmv_items = 0, n_coarse_items = 0;
  int n_rz_cap = 0;   // partial (r, z) sums the buffer holds per right-hand side
  // per right-hand side: iterations of the first CG run when a residual replacement restarted it (-1:
  // none); kept with the problem, so it survives the engine being rebuilt for other batches
  std::vector<int> lanczos_len;
  size_t o_vec = 0, o_coarse = 0, o_scal = 0, o_int = 0, o_hist = 0, o_ppq = 0, o_prr = 0, o_prz = 0, o_pc = 0, o_cnt = 0;
  // (re)allocates for k right-hand sides and maxit recorded iterations; a new buffer is zeroed on `stream`, the
  // stream the caller's kernels then use (a plain cudaMemset would run on the legacy stream, unordered with
  // the library's non-blocking streams, and could land after the first kernels had written the state)
  int ensure(const dgasm_prec_s& pc, int k, int maxit, cudaStream_t stream);
  void fill(const dgasm_prec_s& pc, ProbDev& D, int k, const double* b_user, double* x_user, int maxit, int fixed,
            double rtol) const;
};

// A batch of problems prepared for the batched kernels: device descriptor tables, item prefix sums,
// a captured graph of CHUNK iterations, and the event pairs used when profiling.
struct Engine {
  static constexpr int CHUNK = 8;
  int nprob = 0;
  std::vector<dgasm_prec_s*> pcs;
  std::vector<int> nrhs;
  std::vector<ProbDev> hp;
  std::vector<int> pre;
  int max_smem[8] = {0};
  int tot_spmv = 0, tot_grp = 0, tot_coarse = 0, tot_rnn = 0;
  int total_rhs = 0;
  int km = 1;   // 1 when every problem has one right-hand side
  DevBuf tables;
  int* d_remaining = nullptr;
  int* d_err = nullptr;
  int* h_remaining = nullptr;
  BatchDev B{};
  cudaStream_t stream = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  int per_iter_launches = 0;
  long long launches = 0;
  EventPairs init_ev, graph_ev;
  Engine();
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;
  // Prepares the tables; `remaining` = right-hand sides not yet done (-1: all, for a fresh solve).
  int build(int n, dgasm_prec_s* const* pcs, const int* nrhs, const double* const* b, double* const* x,
            const dgasm_solve_opts* const* opts, cudaStream_t stream, int remaining);
  int reset_state();                 // clears done flags, counters and iteration counts
  int init(bool x0 = false);         // r = b (- A x0), z = B r, p = z, gamma = (r, z)
  // Residual replacement for right-hand sides whose recursive residual met rtol but whose true residual
  // (from the last true_residual()) did not: r = b - A x, z = B r, p = z; *count = how many restarted.
  int restart(int* count);
  int true_residual();               // q = A x and the true relative residual of every right-hand side
  int iterate(int max_iters, int* ran);  // CHUNK-iteration graphs until all done or max_iters
  int finish();                      // x in the caller's order
  int apply_out();                   // z = B r into the caller's buffer (preconditioner apply)
  // statistics of every right-hand side (problem order); per-problem return codes in rcs if given
  int collect(dgasm_stats* st, double ms, std::vector<int>* rcs);
  // per problem: 1 when all its right-hand sides are done; not_done_rhs counts the open ones
  int read_done(std::vector<int>& done, int* not_done_rhs);
 private:
  int precond(int mode, EventPairs* ev, int wslot);   // wslot: the gamma slot the p update writes
  int spmv(int operand, EventPairs* ev);
};

int solve_all(Engine& E, int n, dgasm_prec_s* const* pcs, const int* nrhs, const double* const* b, double* const* x,
              const dgasm_solve_opts* o, cudaStream_t stream, dgasm_stats* st);
int prec_plan(dgasm_system_s* s, const dgasm_setup_opts* o, std::unique_ptr<dgasm_prec_s>& pc);
size_t prec_estimate_bytes(const dgasm_prec_s& pc, int nrhs, int maxit);
// With `defer`, the setup's temporaries are handed to it after the final synchronisation instead of being
// freed (a free waits for the whole device, which would stall setups running beside this one).
int prec_build(dgasm_prec_s* pc, SetupTemps* defer = nullptr);
// times one preconditioner application of b with each right-hand-side chunking and keeps the faster
int tune_rhs_chunk(dgasm_prec_s* pc, int nrhs, const double* b, cudaStream_t stream);
// local-solve variants: 1 = forward/backward sweeps with the envelope factors, 2 = explicit inverses
enum LocalVariant { LV_TUNE = 0, LV_SWEEPS = 1, LV_INVERSE = 2 };
bool dli_candidate(const dgasm_prec_s& pc);   // explicit inverses small enough to form and keep
int build_dli(dgasm_prec_s* pc);              // forms them (once)
// times the local-solve variants on b (when the preconditioner is a candidate and not yet tuned) and keeps
// the faster; the caller holds pc->mu
int tune_local_variant(dgasm_prec_s* pc, int nrhs, const double* b, cudaStream_t stream);
// z = B r (the caller holds pc->mu)
int apply_locked(dgasm_prec_s* pc, int nrhs, const double* r, double* z, cudaStream_t stream);

}  // namespace dgasm

struct dgasm_prec_s {
  dgasm_system_s* sys = nullptr;
  dgasm::Plan P;
  int precision = DGASM_FP64;
  int n0 = 0;
  double plan_ms = 0, setup_ms = 0;
  std::chrono::steady_clock::time_point t_start;
  int setup_launches = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  dgasm::DevBuf perm, rowptr, col, vals, src_blk, sub_e0, scale, Lr, Lc, grp_ptr, grp_elems, agg_int, r0t, A0inv, err, io;
  dgasm::DevBuf r0t_ptr, r0t_col, r0t_elem, rT_ptr, rT_pair;   // non-nested coarse space: R_0^T pairs
  dgasm::R0TPairs nn;       // host copy of the pairs between the plan and the upload
  // right-hand sides per local-solve item for a solve of k right-hand sides: 0 = not chosen yet (the default
  // KC, tuned by the first dgasm_solve with k > 1), else 1 or KC
  int rhs_chunk[dgasm::KMAX + 1] = {0};
  bool blocks = false;      // every subdomain is one element: local solves with explicit block inverses
  int local_variant = dgasm::LV_TUNE;   // envelope problems: sweeps or explicit inverses (LocalVariant)
  dgasm::DevBuf dli, dli_off, dli_item;  // explicit inverses, their offsets and the item table
  int n_dli_items = 0, dli_nmax = 0;
  int tc_fallback = 0;      // 1: the tensor-core factorisation broke down and was redone with FP32 CUDA cores
  dgasm::DevBuf dinv;       // [ne][np][np] FP64, internal element order
  dgasm::EnvBufs env, env0;
  dgasm::Workspace ws;
  dgasm::EventPairs setup_ev;
  std::unique_ptr<dgasm::Engine> engine;  // reused by dgasm_solve
  std::mutex mu;
  int init_streams(void* user_stream);
  int coarse_inverse(dgasm::DevBuf& scale0, dgasm::DevBuf& Lr0, dgasm::DevBuf& Lc0, cudaStream_t st,
                     dgasm::SetupTemps& keep, int** err_word);
  size_t footprint() const;
  ~dgasm_prec_s();
};
