/*
 * dgasm: SIPG discretisation of -div(rho grad u) = f on polygonal meshes of a 2D domain, solved by
 * conjugate gradients preconditioned with the two-level non-overlapping additive Schwarz operator
 *     B = R_0^T A_0^{-1} R_0 + sum_i R_i^T A_i^{-1} R_i
 * of Antonietti, Houston, Pennesi and Suli (arXiv 1903.11357), on one GPU (sm_103a).
 *
 * Conventions
 *  - Every function returns an int: DGASM_OK (0), DGASM_PENDING (> 0, serving only) or a negative
 *    DGASM_E* code.  dgasm_last_error() returns the calling thread's last message.
 *  - Handles are opaque, owned by the caller, and released by the matching *_destroy (NULL is a
 *    no-op).  A system must outlive the preconditioners built from it; a mesh must outlive its
 *    systems.
 *  - Host arrays passed in are copied during the call; the caller keeps ownership.
 *  - Device pointers are borrowed for the duration of the call (dgasm_solve) or until dgasm_poll /
 *    dgasm_wait reports completion (dgasm_submit).
 *  - "stream" arguments are cudaStream_t values passed as void*; NULL means the library's own
 *    stream.  Calls are synchronous with respect to the host unless stated otherwise.
 *  - Indices are 0-based int32.  Dof a of element e (in the caller's element order) has global index
 *    e * n_p + a, with n_p = (p+1)(p+2)/2 and the basis order below.
 *  - The library allocates device memory with cudaMalloc unless dgasm_set_allocator installs hooks.
 *  - Distinct handles may be used from distinct threads concurrently; one handle is not thread-safe
 *    except a server, whose submit/poll/wait are.
 */
#ifndef DGASM_H
#define DGASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DGASM_OK = 0,
  DGASM_PENDING = 1,      /* request admitted or queued, not finished */
  DGASM_EINVAL = -1,      /* invalid argument or mesh topology; message names the index */
  DGASM_ENOMEM = -2,      /* device or host allocation failed */
  DGASM_ENOTSPD = -3,     /* a non-positive pivot in a local or coarse Cholesky factorisation */
  DGASM_ENOCONV = -4,     /* maxit reached before the stop test held; x holds the last iterate */
  DGASM_ENAN = -5,        /* NaN or Inf in the right-hand side or in a Krylov scalar */
  DGASM_ECUDA = -6,       /* a CUDA runtime call failed; message carries cudaGetErrorString */
  DGASM_ETIMEOUT = -7,    /* dgasm_wait deadline passed, or a request exceeded its time limit */
  DGASM_ETOOBIG = -8,     /* request footprint exceeds the server's whole memory budget */
  DGASM_ECANCELLED = -9,  /* request cancelled before it ran */
  DGASM_ENOTFOUND = -10   /* unknown ticket */
};

typedef enum {
  DGASM_FP64 = 0, /* local factors and solves in FP64 */
  DGASM_FP32 = 1, /* local factors and solves in FP32 (CUDA cores); outer loop FP64 */
  DGASM_TF32 = 2, /* local factor trailing updates on tensor cores (TF32 in, FP32 accumulate) */
  DGASM_BF16 = 3  /* local factor stored in BF16, FP32 accumulation; outer loop FP64 */
} dgasm_precision;

typedef struct dgasm_mesh_s* dgasm_mesh_t;
typedef struct dgasm_system_s* dgasm_system_t;
typedef struct dgasm_prec_s* dgasm_prec_t;
typedef struct dgasm_server_s* dgasm_server_t;

/* Right-hand side callback: f(xy[2i], xy[2i+1]) -> out[i] for i < n.  Called from the calling
 * thread only, with n up to a few thousand points per call. */
typedef void (*dgasm_rhs_fn)(int n, const double* xy, double* out, void* user);

/* Optional device allocator hooks (e.g. a framework's caching allocator). alloc returns NULL on
 * failure.  Passing NULL for both restores cudaMalloc/cudaFree.  Process-wide. */
typedef void* (*dgasm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*dgasm_free_fn)(void* ptr, void* stream, void* user);
int dgasm_set_allocator(dgasm_alloc_fn alloc, dgasm_free_fn free_, void* user);

/* Copies the calling thread's last error message (NUL-terminated, truncated to n) into buf.
 * Returns the code of that error (DGASM_OK if none). */
int dgasm_last_error(char* buf, size_t n);

/* ---- Mesh (Sec. 2: tessellation T_h of polygons kappa, diameter h_kappa, faces F_h^I, F_h^B;
 *      Remark 2.1: rho piecewise constant, rho_kappa > 0) ------------------------------------- */

/* nv vertices xy[2*nv] (x, y interleaved); ne polygons, polygon e has vertex ids
 * poly_vtx[poly_ptr[e] .. poly_ptr[e+1]) in counter-clockwise order; rho[ne] > 0.
 * Faces are derived from shared vertex pairs: an edge (a, b) whose reverse (b, a) belongs to
 * another polygon is an interior face, otherwise a boundary face (zero Dirichlet data).
 * Computes areas, area centroids, diameters h_kappa (largest vertex distance) and bounding boxes.
 * Errors: DGASM_EINVAL for fewer than 3 vertices, a vertex id out of range, non-positive signed
 * area (clockwise or degenerate polygon), rho <= 0 or non-finite, an edge used twice in the same
 * direction; the message names the element. */
int dgasm_mesh_create(int nv, const double* xy, int ne, const int* poly_ptr, const int* poly_vtx,
                      const double* rho, dgasm_mesh_t* out);
/* Counts: elements, interior faces, boundary faces. */
int dgasm_mesh_info(dgasm_mesh_t m, int* ne, int* nf_interior, int* nf_boundary);
/* Area centroids (2*ne doubles, x/y interleaved) as used by the partitioner. */
int dgasm_mesh_centroids(dgasm_mesh_t m, double* out_xy);
int dgasm_mesh_destroy(dgasm_mesh_t m);

/* ---- Partitions (Sec. 3: subdomains Omega_i, unions of elements; coarse agglomerates D_j) ------
 * Recursive coordinate bisection of the element area centroids: a set is cut along the longer side
 * of its centroid bounding box (x on ties) after sorting by (coordinate, element id); for k parts
 * the first floor(k/2) parts take floor(n floor(k/2) / k) elements; parts numbered depth-first,
 * lower side first.  Agglomerates: if ncoarse >= nsub, subdomain i is cut into
 * floor((i+1) ncoarse / nsub) - floor(i ncoarse / nsub) agglomerates (nested in the subdomains);
 * otherwise the whole mesh is cut into ncoarse agglomerates.  ncoarse = 0 leaves agg_of_elem
 * untouched.  Outputs are host arrays of ne ints.  Errors: DGASM_EINVAL if nsub < 1 or > ne or
 * ncoarse < 0 or > ne. */
int dgasm_partition(dgasm_mesh_t m, int nsub, int ncoarse, int* sub_of_elem, int* agg_of_elem);

/* ---- SIPG system (Sec. 2, Eq. Ah with the lifting of Eq. lifting, penalty of Eq. Sigma) ---------
 * Basis on element kappa with bounding box [x0,x1]x[y0,y1]: phi_ij = c_ij L_i(xi) L_j(eta),
 * xi = 2(x - xc)/wx, eta = 2(y - yc)/wy, i + j <= p, c_ij = sqrt((2i+1)(2j+1)/(wx wy)); ordered by
 * total degree ascending, then i descending.  The matrix is
 *   A[a,b] = rho_k int grad phi_a . grad phi_b
 *          + sum_F int_F ( -<rho>/2 s_a phi_a d_n phi_b - <rho>/2 s_b phi_b d_n phi_a
 *                          + sigma s_a s_b phi_a phi_b )
 * with <.> the harmonic average (rho_kappa and h_kappa themselves on boundary faces), s = +-1 the
 * side and sigma = c_sigma <rho> p^2 / <h>.  All integrals are exact up to rounding.  If f is not
 * NULL the load vector b_a = int f phi_a is assembled (Gauss rule of p+5 points per direction on
 * each triangle of the element's fan).  The block-sparse matrix is uploaded to the device and kept
 * by the system.  Errors: DGASM_EINVAL (p < 1 or p > 8, c_sigma <= 0), DGASM_ENOMEM, DGASM_ECUDA. */
int dgasm_assemble(dgasm_mesh_t m, int p, double c_sigma, dgasm_rhs_fn f, void* user,
                   dgasm_system_t* out);
/* The same system with the matrix assembled on the device (one CTA per element block row, the same terms,
 * rules and summation order as dgasm_assemble; entries agree up to the contraction of products into FMAs),
 * written straight into the device block layout on `stream` (cudaStream_t, NULL = default stream); the
 * load vector, a host callback, is assembled on the host while the kernel runs.  Synchronous.  The host copy
 * of the blocks (dgasm_system_blocks) is made on first request.  Errors as dgasm_assemble. */
int dgasm_assemble_device(dgasm_mesh_t m, int p, double c_sigma, dgasm_rhs_fn f, void* user, void* stream,
                          dgasm_system_t* out);
/* Number of dofs (ne * n_p) and n_p. */
int dgasm_system_dofs(dgasm_system_t s, int64_t* ndof, int* n_p);
/* Host copy of the load vector (ndof doubles); DGASM_EINVAL if no f was given. */
int dgasm_system_rhs(dgasm_system_t s, double* b);
/* Host copy of the block-sparse matrix in the caller's element order: block rows = elements,
 * rowptr[ne+1], col[nnzb], vals[nnzb * n_p * n_p] with block (e, col) stored row-major
 * (vals[k*n_p*n_p + a*n_p + b] = A[e*n_p + a, col*n_p + b]).  Pass NULL to query nnzb only. */
int dgasm_system_blocks(dgasm_system_t s, int64_t* nnzb, int* rowptr, int* col, double* vals);
/* y = A x on the device, caller's dof order; x, y device arrays of ndof doubles. */
int dgasm_system_spmv(dgasm_system_t s, const double* x, double* y, void* stream);
int dgasm_system_destroy(dgasm_system_t s);

/* y = A x and the energy product x^T A x, without any device allocation (the paper has no counterpart).
 * It serves callers that must not allocate device memory once they run: code whose device memory belongs
 * to another runtime's caching allocator, which a cudaMalloc would bypass and fragment, and real-time loops
 * whose memory is fixed at start-up.  x, y are device arrays of ndof doubles in the caller's dof order,
 * xAx a device pointer to one double; all three are the caller's and must not overlap (DGASM_EINVAL).
 * The per-block partial sums live in a fixed 512 KB (+256 B) __device__ array inside the library, held by
 * every GPU that loads it until the process exits, so a call handles at most 65536 thread blocks of 256
 * threads (65536 * floor(256 / n_p) elements, e.g. 1.6 million elements at p = 3); larger systems get
 * DGASM_ETOOBIG.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream capture.  The
 * array is shared by every call on a device and keeps the last call's contents (its counter is cleared at
 * the start of each call), so calls that overlap on the GPU (on different streams, or from different
 * threads) race: serialise them.  The matrix must already be on the device (dgasm_system_spmv or
 * dgasm_setup upload it on first use), and that device must be the current one; otherwise DGASM_EINVAL.
 * Asynchronous on the stream; y is bitwise identical to dgasm_system_spmv's. */
int dgasm_system_spmv_dot_noalloc(dgasm_system_t s, const double* x, double* y, double* xAx, void* stream);

/* Form of the FP32 and BF16 local-solve launches (no paper counterpart; a scheduling choice of this library,
 * process-wide): 0 (the default) runs each subdomain item on a cluster of two CTAs while all of a launch's
 * items fit on the GPU at once, and on one CTA per item beyond that; 1 one CTA wherever its shared memory holds
 * two ring slots next to the subdomain's vectors (else a pair); 2 always a pair.  Both forms add the same
 * products in the same order, so results do not depend on it (FP64 local solves always use pairs).  Takes
 * effect for solves and applications started after the call.  Errors: DGASM_EINVAL for another value. */
int dgasm_set_local_cta_form(int form);

/* FP64 FMA issue-rate probe (the paper has no counterpart; measurement support for the roofline of the FP64
 * kernels).  Runs one CTA of 512 threads per SM on the current device, each thread 8 independent FP64 FMA
 * chains, and reports *nsm (SM count), *fma_per_clk_per_sm (FMA per clock per SM, median SM, from the CTAs'
 * clock64 cycles) and *tflops (the GPU-wide FP64 FMA rate at the clock the launch ran at, from CUDA events).
 * Synchronous (default stream); allocates a few KB.  Errors: DGASM_EINVAL (NULL argument), DGASM_ECUDA. */
int dgasm_probe_fp64(int* nsm, double* fma_per_clk_per_sm, double* tflops);

/* ---- Failure detection self-test (no counterpart in the paper) --------------------------------------
 * Every wait inside the library's kernels (ring slots, the CTA pair's exchange) is bounded: past its limit
 * it sets the batch error word, stops waiting and lets the kernel return, and the host reports
 * DGASM_ECUDA ("a bounded wait ... gave up") with the context still usable.  This call runs that path on
 * purpose: one CTA waits on an mbarrier nothing arrives on, with a limit of limit_ms milliseconds (0 < limit_ms
 * <= 1000).  *gave_up = 1 when the wait expired and reported it (the expected outcome); *elapsed_ms is the
 * kernel's device time.  Returns DGASM_EINVAL for a limit out of range, DGASM_ECUDA on a CUDA error. */
int dgasm_selftest_bounded_wait(double limit_ms, int* gave_up, double* elapsed_ms);

/* ---- Tensor-core trailing update self-test ------------------------------------------------------------
 * The TF32 precision mode runs the trailing updates of the local tile Cholesky (Sec. 3, local solvers:
 * C_IJ -= L_IK L_JK^T) on the tensor cores with split TF32 operands.  This call runs that kernel once on a
 * caller-supplied dense lower tile matrix of n + 1 tile rows (1 <= n <= 64): `tiles` (host, FP32) holds the
 * (n+1)(n+2)/2 tiles row by row, tile (I, J), J <= I, at index I(I+1)/2 + J, each 32 x 32 row-major; the call
 * applies step K = 0, C_IJ -= L_I0 L_J0^T for 1 <= J <= I <= n, and writes the whole matrix to `out` (host,
 * same layout; tile row 0 is unchanged).  Synchronous.  DGASM_EINVAL for bad arguments, DGASM_ETIMEOUT if
 * the kernel's bounded wait on the MMA completion gave up, DGASM_ECUDA on a CUDA error. */
int dgasm_selftest_tc_update(int n, const float* tiles, float* out);
/* The same step with the BF16 mode's kernel: tcgen05.mma of kind::f16 on BF16 operands, each FP32 entry split
 * in three BF16 parts (hi, mid, lo) and six products accumulated in FP32 in tensor memory.  Arguments, layout
 * and errors as dgasm_selftest_tc_update. */
int dgasm_selftest_tc_update_bf16(int n, const float* tiles, float* out);

/* ---- Two-level Schwarz preconditioner (Sec. 3: local solvers, coarse solver, Eq. R0T, Eq. A0) --- */
typedef struct {
  int nsub;                 /* number of subdomains (1..ne); ignored if sub_of_elem is given */
  int ncoarse;              /* number of coarse agglomerates; 0 = one-level (no coarse space) */
  int p_c;                  /* coarse degree q, 1 <= q <= p (Sec. 3 requires q <= p) */
  const int* sub_of_elem;   /* optional host array [ne]: subdomain of each element */
  const int* agg_of_elem;   /* optional host array [ne]: agglomerate of each element */
  int precision;            /* dgasm_precision for the local factors and solves */
  void* stream;             /* cudaStream_t or NULL */
  dgasm_mesh_t coarse_mesh; /* optional: an independent polygonal mesh of the same domain whose (convex) cells
                               D_j carry the coarse space V_0 = P_q(D_j) (non-nested coarse space, Example 4;
                               a non-convex cell is rejected with DGASM_EINVAL);
                               ncoarse and agg_of_elem are then ignored.  Borrowed for the call (dgasm_setup)
                               or until the request finishes (dgasm_submit).  NULL = agglomerates. */
} dgasm_setup_opts;

/* Builds the partition (RCB as dgasm_partition, unless arrays are given), renumbers the elements
 * subdomain by subdomain (reverse Cuthill-McKee inside each), extracts each A_i (the principal
 * submatrix of A on Omega_i's dofs, Sec. 3), scales it to unit diagonal and factors it by tile
 * Cholesky (FP64/FP32/TF32/BF16 per precision); builds R_0^T|_kappa = M_kappa^{-1} N_kappa (Eq. R0T,
 * exact injection in the nested case, Remark 3.1), A_0 = R_0 A R_0^T (Eq. A0) and its FP64 Cholesky
 * factor and inverse.  With a coarse_mesh, R_0^T|_kappa = M_kappa^{-1} [int_{kappa cap D_j} phi psi_j^T]_j over
 * the coarse cells overlapping kappa (pieces by convex clipping, computed on the host like the assembly;
 * A_0 and everything after it on the device).  Errors: DGASM_EINVAL (bad options or arrays, a fine element
 * or coarse cell that overlaps nothing), DGASM_ENOTSPD (the message names the subdomain, or "coarse", and
 * the pivot row), DGASM_ENOMEM, DGASM_ECUDA. */
int dgasm_setup(dgasm_system_t s, const dgasm_setup_opts* o, dgasm_prec_t* out);
/* n preconditioners at once (a batch of independent problems; the paper sets up one): out[i] is what
 * dgasm_setup(systems[i], opts[i], &out[i]) would build, with the same plan and bitwise the same factors.  The
 * host plans run on the library's worker threads, several problems at a time, and each problem's device work
 * on its own streams (or on opts[i]->stream where one is given: problems that share a stream run their device
 * work in turn), so the setups of small problems, which leave most of the GPU idle, overlap.  The setups'
 * temporaries are released only after the last one has finished: the call's peak device memory is the sum of
 * every problem's setup peak.  All or nothing: on an error every preconditioner built so far is destroyed, out
 * is all NULL, and the code and message are those of the failing problem (the message names its index).
 * Errors as dgasm_setup, and DGASM_EINVAL for n < 1 or NULL arrays or entries. */
int dgasm_setup_batch(int n, const dgasm_system_t* systems, const dgasm_setup_opts* const* opts, dgasm_prec_t* out);
/* z = B r for nrhs vectors (device, caller's dof order, column-major ndof x nrhs). */
int dgasm_prec_apply(dgasm_prec_t pc, int nrhs, const double* r, double* z, void* stream);
/* Consistency self-check of the host plan dgasm_setup would build for nsub RCB subdomains (no device work): the
 * tensor-core trailing-update groups cover exactly the plain update tasks of every Cholesky step, and every
 * subdomain's forward and backward solve streams and run tables match their definitions from the tile envelope.
 * *violations = number of mismatches (0 expected); *checks = entries compared.  Errors: DGASM_EINVAL. */
int dgasm_selftest_plan(dgasm_system_t s, int nsub, int64_t* violations, int64_t* checks);
/* The R_0^T of a non-nested coarse mesh as dgasm_setup builds it (Eq. R0T over the clipped intersections of the
 * fine element kappa with the coarse cells D_j), on the host, in the caller's element order: *npair pairs
 * (kappa, j); ptr [ne+1] the pairs of each fine element, col [npair] their coarse cells (ascending), blocks
 * [npair][n_p][n_q] (row a = fine basis function, column c = coarse one) = M_kappa^{-1} int_{kappa cap D_j} phi_a
 * psi_c.  Call with NULL arrays to get *npair first.  1 <= q <= p <= 8.  Errors: DGASM_EINVAL (bad degrees, a
 * cell that overlaps nothing). */
int dgasm_nonnested_prolongation(dgasm_mesh_t fine, dgasm_mesh_t coarse, int p, int q, int64_t* npair, int* ptr,
                                 int* col, double* blocks);
/* Right-hand sides per local-solve work item for solves of nrhs right-hand sides (2 <= nrhs <= 8): 1 or 4.
 * With 4, a pair of SMs streams each local factor once for 4 vectors; with 1 there are 4 times as many work
 * items, which is faster when there are few subdomains.  0 (the default) lets the first dgasm_solve with that
 * nrhs measure both (one warm-up and two timed preconditioner applications each) and keep the faster; both
 * give bitwise the same solutions.  get returns the current choice (0 = not measured yet; 1 for nrhs = 1).
 * Errors: DGASM_EINVAL. */
int dgasm_prec_set_rhs_chunk(dgasm_prec_t pc, int nrhs, int kc);
int dgasm_prec_get_rhs_chunk(dgasm_prec_t pc, int nrhs, int* kc);
/* Local-solve variant (Sec. 3, local solvers z_i = A_i^{-1} r_i): 1 = forward and backward substitution with the
 * tile-envelope Cholesky factors (the sweeps); 2 = explicit inverses X_i = A_i^{-1}, formed once from those
 * factors (the sweeps applied to unit vectors, in the factor precision) and kept dense (FP64 in FP64 mode, FP32
 * otherwise), so that a local solve is one matrix-vector product per subdomain with no sequential dependency:
 * faster for small subdomains, whose sweeps are latency bound.  Only preconditioners whose subdomains have at
 * most 2048 dofs and whose inverses take at most 1 GiB can use 2 (DGASM_EINVAL otherwise; setting 2 forms the
 * inverses at once).  0 (the default) lets the first dgasm_solve / dgasm_solve_batch measure both (one warm-up
 * and two timed preconditioner applications each) and keep the faster; the outcome is reused for later
 * preconditioners of the same shape (precision, n_p, subdomain count, largest subdomain in steps of 128 dofs,
 * right-hand sides).  The two variants give the same solution up to rounding.  get returns the current choice
 * (0 = not measured yet; 2 when every subdomain is one element, whose block inverses are always explicit).
 * Errors: DGASM_EINVAL. */
int dgasm_prec_set_local_variant(dgasm_prec_t pc, int variant);
int dgasm_prec_get_local_variant(dgasm_prec_t pc, int* variant);
/* Partition actually used (host arrays [ne]); either pointer may be NULL; agg_of_elem is not written when
 * the coarse space lives on a coarse_mesh. */
int dgasm_prec_partition(dgasm_prec_t pc, int* sub_of_elem, int* agg_of_elem);
/* Bytes held on the device by the preconditioner (factors, coarse operator, permuted matrix). */
int dgasm_prec_footprint(dgasm_prec_t pc, int64_t* bytes);
/* Structure and cost of a preconditioner (for reporting and roofline accounting). */
typedef struct {
  int nsub;               /* subdomains N_H (Sec. 3) */
  int nagg;               /* coarse agglomerates N_H of T_H (0 if one-level) */
  int n0;                 /* coarse dofs nagg * (q+1)(q+2)/2 */
  int precision;          /* dgasm_precision of the local factors */
  int64_t local_dofs;     /* sum of the subdomain dof counts (= ndof) */
  int64_t local_tiles;    /* 32x32 tiles in the envelopes of all local factors (one copy) */
  int64_t stream_tiles;   /* 32x32 tiles read by one local solve, forward and backward sweep together:
                             envelope tiles outside the diagonal super-row blocks, the inverted super-row
                             blocks, and the few zero tiles that keep backward runs contiguous */
  int64_t factor_flops;   /* flops of the tile Cholesky of the local factors (tile-level count) */
  int64_t nnzb;           /* blocks of the block-sparse matrix */
  double plan_ms;         /* host part of dgasm_setup: partition, ordering, envelopes, task lists */
  double setup_ms;        /* wall time of dgasm_setup */
  int setup_launches;     /* kernels launched by dgasm_setup */
  int tc_fallback;        /* TF32 / BF16 modes: 1 if the tensor-core factorisation met a non-positive pivot and
                             the local factors were computed again with the FP32 CUDA-core updates */
} dgasm_prec_info_t;
int dgasm_prec_info(dgasm_prec_t pc, dgasm_prec_info_t* info);
int dgasm_prec_destroy(dgasm_prec_t pc);

/* ---- ASPCG solve (Sec. 7: PCG with P_ad from x0 = 0, stop when ||r||_2 / ||b||_2 < rtol) ---------
 * The stop test is taken on the recursive residual; the true residual b - A x is then recomputed in
 * FP64, and where it misses rtol the recursion restarts from it (residual replacement: r = b - A x,
 * p = B r; no iteration counted), at most 4 times and within maxit, so that a converged right-hand side
 * meets rtol in both senses. */
typedef struct {
  double rtol;          /* relative residual tolerance (Sec. 7 uses 1e-8); <= 0 means 1e-8 */
  int maxit;            /* iteration limit; <= 0 means 10000 */
  int fixed_iters;      /* > 0: run exactly this many iterations, no stop test */
  int x0_given;         /* 1: x holds the initial guess on entry (device or host, as b); 0: start from
                           zero (Sec. 7).  Not accepted by dgasm_submit. */
  int host_buffers;     /* 1: b and x are host pointers (copied in and out inside the call) */
  void* stream;         /* cudaStream_t or NULL */
} dgasm_solve_opts;

typedef struct {
  int iters;            /* PCG iterations (matrix-vector products after the initial residual) */
  int converged;        /* 1 if ||r_k|| / ||b|| <= rtol held (and, unless fixed_iters, ||b - A x|| too) */
  double relres;        /* recursive residual ||r_k|| / ||b|| */
  double true_relres;   /* ||b - A x_k|| / ||b||, recomputed in FP64 */
  double lambda_min;    /* Lanczos extreme-eigenvalue estimates of B A from the CG coefficients */
  double lambda_max;
  double kappa;         /* lambda_max / lambda_min: the estimate of K(P_ad) of Sec. 7 */
  double solve_ms;      /* device time of the solve */
  int launches;         /* kernels launched by the solve */
} dgasm_stats;

/* Solves A x = b for nrhs right-hand sides (column-major ndof x nrhs, caller's dof order), device
 * pointers unless opts->host_buffers.  st (nrhs entries) may be NULL.  The Lanczos estimate uses the
 * CG coefficients of the run up to its first convergence (before any residual replacement).  Returns DGASM_ENOCONV if a right-hand side hit maxit (x holds the
 * last iterate), DGASM_ENAN on a NaN/Inf in b or in a Krylov scalar, DGASM_EINVAL, DGASM_ECUDA. */
int dgasm_solve(dgasm_prec_t pc, int nrhs, const double* b, double* x, const dgasm_solve_opts* o,
                dgasm_stats* st);

/* Solves nprob independent problems in one set of batched launches: problem i uses pcs[i] with
 * nrhs[i] right-hand sides b[i] / x[i] (device pointers; x0_given allowed, host_buffers not).  Results are bitwise identical to
 * dgasm_solve of each problem alone.  st holds sum(nrhs) entries in problem order (may be NULL). */
int dgasm_solve_batch(int nprob, const dgasm_prec_t* pcs, const int* nrhs, const double* const* b,
                      double* const* x, const dgasm_solve_opts* o, dgasm_stats* st);

/* Convenience: Lanczos extremes of the tridiagonal built from k CG coefficients alpha[k], beta[k-1]
 * (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j), host only. */
int dgasm_lanczos(int k, const double* alpha, const double* beta, double* lambda_min, double* lambda_max);

/* ---- Kernel timing (CUDA events on the launching streams) --------------------------------------
 * Every launch of an enabled kind made by dgasm_setup / dgasm_solve is bracketed by CUDA events
 * (inside the captured graphs as event nodes) and its device time is accumulated.
 * Kinds: 0 SpMV, 1 x/r update + restriction, 2 local solves, 3 coarse solve, 4 p update,
 * 5 Cholesky diagonal tiles, 6 Cholesky panels, 7 Cholesky trailing updates.  Process-wide.
 * mask: bit k enables kind k (0xFF: all kinds, 0: off).  Timing fewer kinds adds fewer event nodes. */
int dgasm_profile_enable(int mask);
/* Accumulated time (ms) and launch count of one kind since the last reset (reset = 1 clears). */
int dgasm_profile_read(int kind, double* total_ms, int64_t* launches, int reset);

/* ---- Serving: continuous batching of solve requests ---------------------------------------------
 * A server owns a scheduler thread.  dgasm_submit enqueues a request (a system, setup options, nrhs
 * right-hand sides); the request is admitted when its device footprint (factors + coarse operator +
 * Krylov state for nrhs) fits in hbm_budget next to the admitted ones and one of max_slots slots is
 * free.  Admitted requests are set up, then advance together, one PCG iteration each per batched
 * round; finished requests retire between rounds and queued ones join.  b and x are device pointers
 * (ndof x nrhs, column-major) borrowed until completion; so is the system handle sys, which must not be
 * destroyed while one of its requests is queued or running. */
int dgasm_server_create(size_t hbm_budget, int max_slots, void* stream, dgasm_server_t* out);
int dgasm_submit(dgasm_server_t sv, dgasm_system_t sys, const dgasm_setup_opts* so, int nrhs,
                 const double* b, double* x, const dgasm_solve_opts* o, uint64_t* ticket);
/* DGASM_PENDING while queued or running; DGASM_OK or the request's error when finished (st gets the
 * statistics of each right-hand side, may be NULL); DGASM_ENOTFOUND for an unknown or already
 * collected ticket.  A finished ticket is released by the first poll that reports it. */
int dgasm_poll(dgasm_server_t sv, uint64_t ticket, dgasm_stats* st);
/* Blocks until the ticket finishes or timeout_ms passes (DGASM_ETIMEOUT, ticket stays valid). */
int dgasm_wait(dgasm_server_t sv, uint64_t ticket, int timeout_ms, dgasm_stats* st);
/* Cancels a queued (not yet admitted) request: DGASM_OK, or DGASM_PENDING if it already runs. */
int dgasm_cancel(dgasm_server_t sv, uint64_t ticket);
/* Server counters: requests done, rounds run, admission stalls, bytes in use. */
int dgasm_server_stats(dgasm_server_t sv, int64_t* done, int64_t* rounds, int64_t* stalls,
                       int64_t* bytes_in_use);
int dgasm_server_destroy(dgasm_server_t sv);

#ifdef __cplusplus
}
#endif
#endif /* DGASM_H */
