// Device-side descriptors of the batched PCG engine and the launch wrappers of its kernels.
// Shared by the CUDA translation units and the host orchestration; plain data only.
#pragma once

#include <cstdint>

#include "dgasm.h"

namespace dgasm {

constexpr int NTHREADS = 256;  // threads per CTA of the vector kernels
constexpr int SPMV_THREADS = 128;   // threads per CTA of the SpMV (finer items balance the SMs better)
constexpr int KMAX = 8;        // right-hand sides per problem
constexpr int KC = 4;          // right-hand sides per local-solve CTA
constexpr int SUPER_ROW_MAX = 8;   // tile rows per super-row of the local triangular solves, at most
// Super-row size by precision of the local factors.  Larger blocks trade more inverse-block tiles for
// fewer sequential reductions; on the 16384-cell p=3 workload 8 beat 4 for FP64 (328 vs 354 us per local
// solve) and FP32 (139 vs 158 us), and 16 gained FP32 only 3%.
constexpr int super_row(int /*prec*/) { return 8; }
constexpr long long ZERO_TILE = -(1LL << 62);   // solve-stream entry: a tile of zeros
constexpr int COARSE_ROWS_PER_WARP = 4;          // k_coarse: rows of A_0^{-1} per warp (32 per CTA)

enum Kind { K_SPMV = 0, K_GRP = 1, K_LOCAL = 2, K_COARSE = 3, K_NKINDS = 4 };
constexpr int K_SPMV_P = K_NKINDS + 8;   // per-degree SpMV prefix slots p = 1..8
constexpr int K_BJAC = K_SPMV_P + 8;     // element-block local solves (subdomains = elements)
constexpr int K_RNN = K_BJAC + 1;        // restriction r_0 = R_0 r of non-nested coarse spaces (one item per cell)
constexpr int K_DLI = K_RNN + 1;         // local solves with explicit inverses: K_DLI FP64, K_DLI + 1 FP32 storage
constexpr int K_NSLOTS = K_DLI + 2;
constexpr int DLI_ROWS = 32;             // rows of an explicit-inverse local-solve item
enum Counter { C_SPMV = 0, C_GRP = 1, C_PUPD = 2, C_NCOUNTERS = 4 };

// One problem (one preconditioner with k right-hand sides) of a batch.
struct ProbDev {
  int ne, np, np2s, nq, ndof, nsub, ngrp, n0, k, prec;
  int epi;            // elements per element-chunk item
  int n_chunk_items;  // element-chunk items (p update, output)
  int epi_spmv;       // elements per SpMV item
  int n_spmv_items;   // SpMV items
  int n_coarse_items; // coarse GEMV items (8 rows each)
  int kc;             // right-hand sides per local-solve item
  int n_rhs_chunks;   // ceil(k / kc)
  int maxit, fixed_iters;
  double rtol;
  // matrix, internal order, blocks column-major with stride np2s
  const int* rowptr;
  const int* col;
  const double* vals;
  const int* perm;    // internal element -> caller element
  // local factors
  const int* sub_e0;
  const int* sub_trow;
  const int* trow_F;
  const long long* trow_ptr;
  const long long* fwd_ptr;     // [nsub+1] each subdomain's range in the forward stream
  const long long* bwd_ptr;     // [nsub+1] and in the backward stream
  long long fwd_total, bwd_total;  // tiles in each stream (all subdomains)
  int sr;                       // tile rows per super-row of the local factors
  const double* dinv;           // subdomains = elements: [ne][np][np] inverses of the diagonal blocks, row-major
  int n_rz;                     // partial sums of (r, z): nsub (envelope solves), n_chunk_items (blocks) or
                                // n_dli_items (explicit inverses)
  // explicit subdomain inverses (local-solve variant for small subdomains): X_s = A_s^{-1} dense row-major at
  // dli_off[s] in dli (FP64, or FP32 for the lower-precision modes); items (subdomain, first row) in dli_item
  const void* dli;
  const long long* dli_off;
  const int* dli_item;
  int n_dli_items;
  const int* sub_sr;            // [nsub+1] first global super-row of each subdomain
  const int* fwd_run;           // [global super-row][sr][2]: coupling runs (first operand block, tiles)
  const int* bwd_run;
  const void* Lr;     // backward stream: row-major tiles in consumption order, as [2][bwd_total][16 x 32]
  const void* Lc;     // forward stream: column-major tiles in consumption order, as [2][fwd_total][16 x 32]
  const double* scale;
  // groups and coarse space
  const int* grp_ptr;
  const int* grp_elems;
  const int* agg_int; // agglomerate of each internal element
  const double* r0t;  // [ne][np][nq] R_0^T blocks, internal element order; non-nested: [npair][np][nq]
  // non-nested coarse space (r0t_ptr == nullptr for agglomerates): pairs (element, coarse cell) by element
  // (r0t_ptr [ne+1], r0t_col) and by coarse cell (rT_ptr [nc+1], rT_pair); r0t_elem = element of a pair
  const int* r0t_ptr;
  const int* r0t_col;
  const int* r0t_elem;
  const int* rT_ptr;
  const int* rT_pair;
  int nc;             // coarse cells (non-nested) or agglomerates
  const double* A0inv;// [n0][n0]
  // caller-order input/output, column-major ndof x k
  const double* b_user;
  double* x_user;
  // Krylov state [k][ndof], internal order
  double *b, *x, *r, *p, *q, *z;
  double *r0, *z0;    // [k][n0]
  // per right-hand side scalars
  double *bnorm, *gamma, *alpha, *relres, *true_rr;
  double* gamma1;     // second slot of gamma: the p update of an iteration reads one slot and writes the other
  int *done, *iters, *status;
  double *alpha_hist, *beta_hist;  // [k][maxit]
  // deterministic partial sums
  double *part_pq;    // [n_spmv_items][k]
  double *part_rr;    // [ngrp][k]
  double *part_rz;    // [nsub][k]
  double *part_c;     // [n_coarse_items][k]
  unsigned int* counters;  // [C_NCOUNTERS]
  int* remaining;     // right-hand sides still iterating, shared by the batch
};

struct BatchDev {
  const ProbDev* probs;
  int nprob;
  int* err;          // device error word: nonzero when a bounded wait in a kernel gave up
  const int* prefix[K_NSLOTS];  // item prefix per kind; K_NKINDS + 2*prec + (kc > 1) for local solves;
                                // K_SPMV_P + p - 1 for the SpMV of degree-p problems
};

// ---- solve kernels (kernels_solve.cu) ----
// k_update modes: INIT r = b, x = 0; ITER the CG update and stop test; RESTART r = b - q with q = A x
// from the SpMV (residual replacement, no iteration counted); INIT_X0 like INIT but x = the caller's
// initial guess (r = b - A x follows by SpMV + RESTART)
enum UpdateMode { MODE_INIT = 0, MODE_ITER = 1, MODE_RESTART = 2, MODE_INIT_X0 = 3 };
// km: 1 when every problem of the batch has one right-hand side, else KMAX
int launch_spmv(const BatchDev& B, int p, int total, int operand /*0: q = A p, 1: q = A x, true residual*/, int km,
                void* stream);
// gslot: the gamma slot (0 or 1) the ITER mode reads for alpha = gamma / (p, q)
int launch_update(const BatchDev& B, int total, int mode, int km, int gslot, void* stream);
int launch_local(const BatchDev& B, int slot, int total, int smem_bytes, void* stream);
int launch_coarse(const BatchDev& B, int total, int km, void* stream);
// element-block local solves z_e = inv(A_ee) r_e with the partial (r, z) per chunk item
// one CTA waits on an mbarrier nothing arrives on, bounded by `limit` cycles: err[0] = 1 (the wait gave
// up and set the error word), err[1] = 1 (the wait returned false)
int launch_wait_selftest(int* err, long long limit, void* stream);
int launch_bjac(const BatchDev& B, int total, int km, void* stream);
// explicit-inverse local solves (kernels_dli.cu): slot K_DLI (FP64 inverses) or K_DLI + 1 (FP32)
int launch_dli(const BatchDev& B, int slot, int total, int km, void* stream);
// r zero on entry: column kk of r ([cb][ndof]) becomes unit vector c0 + kk of every subdomain
int launch_unit_block(const int* sub_e0, int nsub, int np, int c0, int cb, long long ndof, double* r, void* stream);
// X_s[i][c0 + kk] = z[kk][d0_s + i] into the explicit inverses (FP64 if fp64, else FP32); nmax = largest n_s
int launch_dli_store(int fp64, const int* sub_e0, int nsub, int np, const long long* off, int c0, int cb,
                     long long ndof, const double* z, void* X, int nmax, void* stream);
// nonnested: some problem of the batch has a non-nested coarse space; wslot: the gamma slot this launch writes
// (the ITER mode reads the other one for beta)
int launch_pupdate(const BatchDev& B, int total, int mode, int km, int nonnested, int wslot, void* stream);
// r_0 = R_0 r for non-nested coarse spaces: one CTA per coarse cell (prefix slot K_RNN)
int launch_restrict_nn(const BatchDev& B, int total, int km, void* stream);
int launch_finish(const BatchDev& B, int total, int operand /*0: x, 1: p*/, void* stream);
// dynamic shared memory of a local-solve launch over subdomains of at most ndof_max dofs
int local_smem_bytes(int prec, int ndof_max, int kc);
int launch_system_spmv(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s,
                       const double* x, double* y, void* stream);

// ---- setup kernels (kernels_setup.cu) ----
struct EnvDev {
  int nsub;
  const int* ndof;        // [nsub]
  const int* sub_trow;
  const int* trow_F;
  const long long* trow_ptr;
};
int launch_permute_blocks(const double* src, const long long* src_blk, double* dst, long long nnzb, int np2s,
                          void* stream);
int launch_scale(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s, double* scale,
                 void* stream);
int launch_extract_rows(int prec, const EnvDev& E, const int* sub_e0, const int* rowptr, const int* col,
                        const double* vals, int np, int np2s, const double* scale, void* Lr, int nsub, int ne,
                        void* stream);
int launch_chol_diag(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, int* err, void* stream);
int launch_chol_panel(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, void* stream);
int launch_chol_update(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, void* stream);
// the trailing update of step K on the tensor cores (tcgen05, FP32 accumulation in tensor memory; bf16 = 0:
// kind::tf32 with operands split in two, 1: kind::f16 with BF16 operands split in three); tasks: n quadruples
// (pstart, n, mb, nb) of Envelope::tc_task, panel_task: all (s, I) pairs; err[3] (bounded wait on the MMA
// completion gave up) is set on timeout
int launch_chol_update_tc(const EnvDev& E, float* L, int K, const int* panel_task, const int* tasks, int n, int* err,
                          void* stream, int bf16);
int launch_to_colmajor(int prec, const void* Lr, void* Lc, long long ntiles, void* stream);
int launch_to_bf16(const float* src, void* dst, long long n, void* stream);
// dst tile t = src tile idx[t] (same element layout), for the backward-ordered copy of a factor
int launch_gather_tiles(int prec, const void* src, const long long* idx, void* dst, long long ntiles, void* stream);
// inverse blocks of the super-rows (task triples: subdomain, first tile row, tile rows)
int launch_dinv(int prec, const EnvDev& E, const void* L, const int* task, const long long* dinv_ptr, void* X, int nsr,
                void* stream);
// solve streams from factor tiles (src >= 0) and inverse-block tiles (src < 0)
int launch_stream_gather(int prec, const void* L, const void* X, const long long* src, void* dst, long long n,
                         int transpose, void* stream);
// subdomains = elements: inverses of the diagonal blocks [ne][np][np] (err as the Cholesky kernels)
int launch_bjac_inverse(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s, double* dinv,
                        int* err, void* stream);
int launch_r0t(const int* perm, const double* bbox, const int* agg_int, const double* agg_bbox, int ne, int p, int q,
               const double* gl_t, const double* gl_w, int mq, double* r0t, void* st);
// W: nnzb * nq * nq doubles of scratch
int launch_galerkin(const int* grp_ptr, const int* grp_elems, const int* agg_int, const int* rowptr,
                    const int* col, const double* vals, const double* r0t, int ne, long long nnzb, int nagg, int np,
                    int np2s, int nq, double* W, double* A0, void* stream);
// SIPG assembly on the device (kernels_assemble.cu): mesh arrays as in MeshData, on the device
struct AsmMesh {
  int ne;
  const double* xy;
  const int* ptr;
  const int* vtx;
  const double* bbox;
  const double* rho;
  const double* diam;
  const int* ef_ptr;
  const int* ef_face;
  const int* f_ep;
  const int* f_em;
  const int* f_va;
  const int* f_vb;
};
// vals: the device blocks (column-major, stride np2s), zero on entry; gt, gw: the (p+2)-point Gauss rule on [0, 1]
int launch_assemble(const AsmMesh& M, int p, double c_sigma, const double* gt, const double* gw, const int* rowptr,
                    const int* col, int np2s, double* vals, void* stream);
// A_0 = R_0 A R_0^T for a non-nested coarse space (pairs as in ProbDev); A0 [n0][n0] must be zero on entry
int launch_galerkin_nn(const int* rowptr, const int* col, const double* vals, int np, int np2s, int nq,
                       const int* r0t_ptr, const int* r0t_col, const int* r0t_elem, const double* r0t, const int* rT_ptr,
                       const int* rT_pair, int nc, int n0, double* A0, void* stream);
int launch_coarse_extract(const double* A0, int n0, double* scale0, const EnvDev& E0, double* Lr0, void* stream);
int launch_identity(double* I, int n, void* stream);

}  // namespace dgasm
