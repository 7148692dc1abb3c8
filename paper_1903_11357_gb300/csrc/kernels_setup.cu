// Device setup kernels: matrix permutation, Jacobi scaling, extraction of the subdomain matrices A_i
// (principal submatrices of A, Sec. 3) into tile envelopes, tile Cholesky factorisation with inverted
// diagonal tiles, the L2 prolongation R_0^T (Eq. R0T) and the Galerkin coarse operator A_0 (Eq. A0).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int T = 32;      // tile edge
constexpr int TT = T * T;

template <typename S> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

template <typename C> __device__ __forceinline__ C crsqrt(C x);
template <> __device__ __forceinline__ double crsqrt<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float crsqrt<float>(float x) { return rsqrtf(x); }

__device__ __forceinline__ long long tile_index(const EnvDev& E, int s, int I, int J) {
  int tr = E.sub_trow[s] + I;
  return E.trow_ptr[tr] + (J - E.trow_F[tr]);
}

__global__ void k_permute_blocks(const double* __restrict__ src, const long long* __restrict__ src_blk,
                                 double* __restrict__ dst, long long nnzb, int np2s) {
  long long total = nnzb * np2s;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    long long b = t / np2s;
    int o = (int)(t - b * np2s);
    dst[t] = src[src_blk[b] * np2s + o];
  }
}

// scale[i*np + a] = 1 / sqrt(A_ii[a][a]) from the diagonal block of internal row i
__global__ void k_scale(const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ vals,
                        int ne, int np, int np2s, double* __restrict__ scale) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ne * np; t += gridDim.x * blockDim.x) {
    int i = t / np, a = t - i * np;
    double d = -1.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) { d = vals[(long long)k * np2s + a * np + a]; break; }
    scale[t] = d > 0.0 ? 1.0 / sqrt(d) : __longlong_as_double(0x7ff8000000000000ULL);
  }
}

// one warp per internal element row: write the lower-triangle entries of the scaled A_i into the
// row-major tile pool; padding rows of the last tile row get a unit diagonal
template <typename S>
__global__ void k_extract(EnvDev E, const int* __restrict__ sub_e0, const int* __restrict__ rowptr,
                          const int* __restrict__ col, const double* __restrict__ vals, int np, int np2s,
                          const double* __restrict__ scale, S* __restrict__ Lr, int nsub) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int ne = sub_e0[nsub];
  if (warp >= ne) return;
  int i = warp;
  // subdomain of row i (binary search)
  int lo = 0, hi = nsub;
  while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (sub_e0[mid] <= i) lo = mid; else hi = mid; }
  int s = lo, e0 = sub_e0[s], e1 = sub_e0[s + 1];
  int n = (e1 - e0) * np;
  for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
    int c = col[k];
    if (c < e0 || c >= e1) continue;
    for (int t = lane; t < np * np; t += 32) {
      int a = t % np, b = t / np;  // column-major entry (a, b) at b*np + a
      int row = (i - e0) * np + a, cl = (c - e0) * np + b;
      if (row < cl) continue;
      double v = vals[(long long)k * np2s + t] * scale[(long long)i * np + a] * scale[(long long)c * np + b];
      long long ti = tile_index(E, s, row / T, cl / T);
      Lr[ti * TT + (row % T) * T + (cl % T)] = (S)v;
    }
  }
  // padding: the last element of the subdomain writes the unit diagonal of the padded rows
  if (i == e1 - 1) {
    int nbt = (n + T - 1) / T;
    for (int row = n + lane; row < nbt * T; row += 32) {
      long long ti = tile_index(E, s, nbt - 1, nbt - 1);
      Lr[ti * TT + (row % T) * T + (row % T)] = (S)1.0;
    }
  }
}

// Cholesky of the diagonal tile (K, K) and in-place replacement by inv(L_KK) (lower triangular)
template <typename S>
__global__ void __launch_bounds__(256) k_chol_diag(EnvDev E, S* __restrict__ L, int K, const int* __restrict__ tasks,
                                                   int* __restrict__ err) {
  using C = typename Compute<S>::type;
  __shared__ C a[T][T + 1];
  __shared__ C inv[T][T + 1];
  __shared__ C rdbuf[2];   // 1/sqrt(pivot) of step j in rdbuf[j & 1]
  __shared__ int bad;
  int s = tasks[blockIdx.x];
  long long ti = tile_index(E, s, K, K);
  S* tile = L + ti * TT;
  const int tid = threadIdx.x;
  for (int t = tid; t < TT; t += blockDim.x) {
    int r = t / T, c = t % T;
    a[r][c] = (r >= c) ? (C)tile[t] : (C)0;
    inv[r][c] = (r == c) ? (C)1 : (C)0;
  }
  __syncthreads();
  if (tid == 0) {
    bad = -1;
    C d = a[0][0];
    if (!(d > (C)0)) { bad = 0; d = (C)1; }
    rdbuf[0] = crsqrt<C>(d);
  }
  __syncthreads();
  // Right-looking Cholesky of the tile, and in the same sweep X = inv(L) by forward elimination of L X = I,
  // with one barrier per step.  Step j reads the pivot d = a_jj, column j of A and row j of X as the earlier
  // steps left them (not yet divided by sqrt(d)); with rd = 1/sqrt(d), l_rj = a_rj rd and x_jc = x~_jc rd, so
  //   a_rc -= u_r a_cj   (c > j, r >= c)      and      x_rc -= u_r x~_jc   (r > j, c <= j),    u_r = a_rj rd^2.
  // Nothing writes column j of A or row j of X during step j; row j - 1 of X is scaled by its rd in step j,
  // when nothing reads it any more (row T - 1 after the loop).  Eight threads share a row (u_r computed once
  // and shuffled); the thread that updates a_(j+1)(j+1) forms the next pivot's rd.  L itself is not stored: the
  // tile receives X = inv(L_KK), and only the pivots of A are read again.
  // The FP64 pipe spends its slots on a warp instruction whatever its active lanes, so work that a whole warp
  // (rows 4w .. 4w + 3) or a whole column group m of a warp would skip is branched around, not predicated.
  const int r = tid >> 3, sub = tid & 7, w = tid >> 5, rlo = 4 * w, rhi = 4 * w + 3;
  C rd_prev = (C)0;
  for (int j = 0; j < T; ++j) {
    const C rd = rdbuf[j & 1];
    if (j <= rhi + 1) {   // some row of this warp changes in step j (rows above j - 1 are final)
      const bool upd = rhi > j;   // a row of this warp lies below the pivot
      C u = (C)0;
      if (upd) {
        if (sub == 0) u = a[r][j] * (rd * rd);
        u = __shfl_sync(0xffffffffu, u, (tid & 31) & ~7);
      }
#pragma unroll
      for (int m = 0; m < T / 8; ++m) {
        const int c = sub + 8 * m;
        // column group m of this warp: entries (r, c) with c > j, r >= c exist; entries c <= j < r exist;
        // row j - 1 of X is in this warp
        if (upd && max(8 * m, j + 1) <= min(8 * m + 7, rhi)) {
          if (c > j && r >= c) {
            a[r][c] -= u * a[c][j];
            if (r == j + 1 && c == j + 1) {
              C d = a[r][c];
              if (!(d > (C)0)) { if (bad < 0) bad = j + 1; d = (C)1; }
              rdbuf[(j + 1) & 1] = crsqrt<C>(d);
            }
          }
        }
        if (upd && 8 * m <= j) {
          if (r > j && c <= j) inv[r][c] -= u * inv[j][c];
          else if (j > 0 && r == j - 1 && c <= r) inv[r][c] *= rd_prev;
        } else if (j > 0 && j - 1 >= rlo && j - 1 <= rhi && 8 * m <= j - 1) {
          if (r == j - 1 && c <= r) inv[r][c] *= rd_prev;
        }
      }
    }
    rd_prev = rd;
    __syncthreads();
  }
  for (int c = tid; c < T; c += blockDim.x) inv[T - 1][c] *= rd_prev;
  __syncthreads();
  for (int t = tid; t < TT; t += blockDim.x) tile[t] = (S)inv[t / T][t % T];
  if (tid == 0 && bad >= 0) {
    // record the first failure: subdomain and pivot row
    atomicCAS(&err[0], 0, 1);
    atomicCAS(&err[1], -1, s);
    atomicCAS(&err[2], -1, K * T + bad);
  }
}

// panel: L_IK = A_IK inv(L_KK)^T, entry (r, c) = sum_{m <= c} A_rm X_cm (X = inv(L_KK), lower triangular).
// Lane = row r; warp w computes columns w, w + 8, w + 16, w + 24, so the triangular loop length is the same
// across a warp (no idle lanes) and the four columns of a warp balance the warps' work.
template <typename S>
__global__ void __launch_bounds__(256) k_chol_panel(EnvDev E, S* __restrict__ L, int K, const int* __restrict__ tasks) {
  using C = typename Compute<S>::type;
  __shared__ C inv[T][T + 1];
  __shared__ C A[T][T + 1];
  int s = tasks[2 * blockIdx.x], I = tasks[2 * blockIdx.x + 1];
  const S* D = L + tile_index(E, s, K, K) * TT;
  S* P = L + tile_index(E, s, I, K) * TT;
  for (int t = threadIdx.x; t < TT; t += blockDim.x) {
    inv[t / T][t % T] = (C)D[t];
    A[t / T][t % T] = (C)P[t];
  }
  __syncthreads();
  const int r = threadIdx.x & 31, w = threadIdx.x >> 5;
  C acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = w + 8 * u;
    acc[u] = (C)0;
    for (int m = 0; m <= c; ++m) acc[u] += A[r][m] * inv[c][m];
  }
  __syncthreads();   // every warp is done reading A: stage the result there for a coalesced store
#pragma unroll
  for (int u = 0; u < 4; ++u) A[r][w + 8 * u] = acc[u];
  __syncthreads();
  for (int t = threadIdx.x; t < TT; t += blockDim.x) P[t] = (S)A[t / T][t % T];
}

// trailing update: A_IJ -= L_IK L_JK^T
template <typename S>
__global__ void __launch_bounds__(256) k_chol_update(EnvDev E, S* __restrict__ L, int K, const int* __restrict__ tasks) {
  using C = typename Compute<S>::type;
  __shared__ C X[T][T + 1];
  __shared__ C Y[T][T + 1];
  int s = tasks[3 * blockIdx.x], I = tasks[3 * blockIdx.x + 1], J = tasks[3 * blockIdx.x + 2];
  const S* Li = L + tile_index(E, s, I, K) * TT;
  const S* Lj = L + tile_index(E, s, J, K) * TT;
  S* Cij = L + tile_index(E, s, I, J) * TT;
  for (int t = threadIdx.x; t < TT; t += blockDim.x) {
    X[t / T][t % T] = (C)Li[t];
    Y[t / T][t % T] = (C)Lj[t];
  }
  __syncthreads();
  if (I == J) {
    // a diagonal target: only its lower triangle is read again, so its 528 entries r >= c (enumerated row by
    // row) are spread over the threads and whole warps go idle instead of predicated-off lanes
    constexpr int NLT = T * (T + 1) / 2;
    for (int e = threadIdx.x; e < NLT; e += blockDim.x) {
      int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
      if (r * (r + 1) / 2 > e) --r;
      if ((r + 1) * (r + 2) / 2 <= e) ++r;
      const int c = e - r * (r + 1) / 2;
      C acc = 0;
      for (int m = 0; m < T; ++m) acc += X[r][m] * Y[c][m];
      Cij[r * T + c] = (S)((C)Cij[r * T + c] - acc);
    }
    return;
  }
  // each thread owns 4 entries of one column c: rows r0, r0+8, r0+16, r0+24
  int c = threadIdx.x % T, r0 = threadIdx.x / T;
  C acc[4] = {0, 0, 0, 0};
  for (int m = 0; m < T; ++m) {
    C y = Y[c][m];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += X[r0 + 8 * u][m] * y;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int r = r0 + 8 * u;
    Cij[r * T + c] = (S)((C)Cij[r * T + c] - acc[u]);
  }
}

template <typename S>
__global__ void k_to_colmajor(const S* __restrict__ Lr, S* __restrict__ Lc, long long ntiles) {
  __shared__ S buf[T][T + 1];
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const S* src = Lr + t * TT;
    S* dst = Lc + t * TT;
    for (int u = threadIdx.x; u < TT; u += blockDim.x) buf[u / T][u % T] = src[u];
    __syncthreads();
    for (int u = threadIdx.x; u < TT; u += blockDim.x) dst[u] = buf[u % T][u / T];
    __syncthreads();
  }
}

template <typename S>
__global__ void k_gather_tiles(const S* __restrict__ src, const long long* __restrict__ idx, S* __restrict__ dst,
                               long long ntiles) {
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const S* a = src + idx[t] * TT;
    S* b = dst + t * TT;
    for (int u = threadIdx.x; u < TT; u += blockDim.x) b[u] = a[u];
  }
}

// Inverse of the lower-triangular diagonal block of one super-row (tile rows I0 .. I0+ntr-1), whose
// diagonal tiles already hold inv(L_ii):  X_ii = inv(L_ii),  X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj
// (block forward substitution; L_ik = 0 left of the envelope).  Tiles row-major, order (i, j), j <= i.
template <typename S>
__global__ void __launch_bounds__(256) k_dinv(EnvDev E, const S* __restrict__ L, const int* __restrict__ task,
                                              const long long* __restrict__ dinv_ptr, S* __restrict__ X) {
  using C = typename Compute<S>::type;
  __shared__ C a[T][T + 1];
  __shared__ C b[T][T + 1];
  __shared__ C w[T][T + 1];
  const int q = blockIdx.x, j = blockIdx.y;   // super-row, tile column of its inverse block
  const int s = task[3 * q], I0 = task[3 * q + 1], ntr = task[3 * q + 2];
  if (j >= ntr) return;
  const long long xb = dinv_ptr[q];
  auto xt = [&](int i, int jj) { return X + (xb + i * (i + 1) / 2 + jj) * TT; };
  const int tid = threadIdx.x, c = tid % T, r0 = tid / T;
  {
    // X_jj = inv(L_jj), which the diagonal factor tile already holds
    const S* src = L + tile_index(E, s, I0 + j, I0 + j) * TT;
    S* dst = xt(j, j);
    for (int t = tid; t < TT; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  // X_ij = -inv(L_ii) sum_{k=j}^{i-1} L_ik X_kj, i = j+1 .. ntr-1: column j depends only on itself
  for (int i = j + 1; i < ntr; ++i) {
    const int Fi = E.trow_F[E.sub_trow[s] + I0 + i];
    C acc[4] = {0, 0, 0, 0};
    for (int kk = j; kk < i; ++kk) {
      if (I0 + kk < Fi) continue;
      const S* A = L + tile_index(E, s, I0 + i, I0 + kk) * TT;
      const S* B = xt(kk, j);
      for (int t = tid; t < TT; t += blockDim.x) {
        a[t / T][t % T] = (C)A[t];
        b[t / T][t % T] = (C)B[t];
      }
      __syncthreads();
      for (int m = 0; m < T; ++m) {
        const C bv = b[m][c];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += a[r0 + 8 * u][m] * bv;
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) w[r0 + 8 * u][c] = acc[u];
    const S* D = L + tile_index(E, s, I0 + i, I0 + i) * TT;
    for (int t = tid; t < TT; t += blockDim.x) a[t / T][t % T] = (C)D[t];
    __syncthreads();
    S* dst = xt(i, j);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + 8 * u;
      C v = (C)0;
      for (int m = 0; m <= r; ++m) v += a[r][m] * w[m][c];
      dst[r * T + c] = (S)(-v);
    }
    __syncthreads();
  }
}

// stream tile p = factor tile src[p] (src[p] >= 0), a zero tile (ZERO_TILE) or inverse-block tile
// -src[p]-1, transposed if asked.  A line is a row of the stored tile (a column of the factor tile when
// transposed).  The stream is stored as two arrays of half tiles, lines 0-15 of every tile then lines
// 16-31, so that each CTA of a pair reads its half of a run of tiles with one contiguous copy; inside a
// half tile, lines 2w and 2w+1 are interleaved ([8][32][2]: pair w, position k, line), so that the warp
// that owns the pair reads both of its entries with one vector load.
template <typename S>
__global__ void k_stream_gather(const S* __restrict__ L, const S* __restrict__ X, const long long* __restrict__ src,
                                S* __restrict__ dst, long long n, int transpose) {
  constexpr int HT = TT / 2;
  __shared__ S buf[T][T + 1];
  for (long long p = blockIdx.x; p < n; p += gridDim.x) {
    const long long v = src[p];
    if (v == ZERO_TILE) {
      for (int u = threadIdx.x; u < TT; u += blockDim.x) buf[u / T][u % T] = (S)0;
    } else {
      const S* a = v >= 0 ? L + v * TT : X + (-v - 1) * TT;
      for (int u = threadIdx.x; u < TT; u += blockDim.x) buf[u / T][u % T] = a[u];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < TT; u += blockDim.x) {
      const int line = u / T, k = u % T;
      const int h = line / 16, w = (line % 16) / 2, b = line % 2;
      dst[(long long)h * n * HT + p * HT + (w * T + k) * 2 + b] = transpose ? buf[k][line] : buf[line][k];
    }
    __syncthreads();
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] = __float2bfloat16_rn(src[t]);
}

// ---- coarse transfer R_0^T|_kappa = M_kappa^{-1} N_kappa (Eq. R0T, nested agglomerates) ---------

__device__ void legendre_dev(int p, double t, double* L, double* dL) {
  L[0] = 1.0; dL[0] = 0.0;
  if (p >= 1) { L[1] = t; dL[1] = 1.0; }
  for (int k = 1; k < p; ++k) {
    L[k + 1] = ((2.0 * k + 1.0) * t * L[k] - k * L[k - 1]) / (k + 1.0);
    dL[k + 1] = dL[k - 1] + (2.0 * k + 1.0) * L[k];
  }
}

// Subdomains = elements (Sec. 7's setting): the inverse of each diagonal block A_ee, one warp per element,
// by Gauss-Jordan elimination without pivoting (A_ee is SPD, so every pivot is positive; a non-positive
// pivot is recorded like a failed Cholesky).  Output row-major [ne][np][np].
constexpr int BJAC_WARPS = 4;
__global__ void k_bjac_inverse(const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ vals, int ne, int np, int np2s, double* __restrict__ dinv,
                               int* __restrict__ err) {
  extern __shared__ double bsm[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * BJAC_WARPS + wid;
  if (e >= ne) return;
  const int ld = np + 1;
  double* A = bsm + (size_t)wid * (np * ld + np);   // [np][np + 1]
  double* f = A + np * ld;                          // [np]: column k before its elimination step
  // the diagonal block: the entry of row e whose column is e
  int kd = -1;
  for (int k = rowptr[e] + lane; k < rowptr[e + 1]; k += 32)
    if (col[k] == e) kd = k;
  for (int o = 16; o > 0; o >>= 1) kd = max(kd, __shfl_xor_sync(0xffffffffu, kd, o));
  const double* Bk = vals + (long long)kd * np2s;   // column-major: entry (r, c) at c * np + r
  for (int t = lane; t < np * np; t += 32) A[(t % np) * ld + t / np] = Bk[t];
  __syncwarp();
  int bad = -1;
  for (int k = 0; k < np; ++k) {
    double p = A[k * ld + k];
    if (!(p > 0.0)) {
      if (bad < 0) bad = k;
      p = 1.0;
    }
    const double rp = 1.0 / p;
    for (int i = lane; i < np; i += 32) f[i] = A[i * ld + k];
    __syncwarp();
    for (int j = lane; j < np; j += 32) A[k * ld + j] = (j == k ? 1.0 : A[k * ld + j]) * rp;
    __syncwarp();
    for (int t = lane; t < np * np; t += 32) {
      const int i = t / np, j = t % np;
      if (i == k) continue;
      A[i * ld + j] = (j == k ? 0.0 : A[i * ld + j]) - f[i] * A[k * ld + j];
    }
    __syncwarp();
  }
  double* out = dinv + (long long)e * np * np;
  for (int t = lane; t < np * np; t += 32) out[t] = A[(t / np) * ld + t % np];
  if (lane == 0 && (bad >= 0 || kd < 0)) {
    atomicCAS(&err[0], 0, 1);
    atomicCAS(&err[1], -1, e);
    atomicCAS(&err[2], -1, bad >= 0 ? bad : 0);
  }
}

// R_0^T|_kappa = M_kappa^{-1} N_kappa (Eq. R0T) for nested agglomerates: the coarse basis functions are
// polynomials of total degree q <= p, so (Remark 3.1) M^{-1} N holds the exact coefficients of their
// restrictions in the element's basis, whatever domain the two mass matrices are integrated on.  On the
// element's bounding box that basis is orthonormal (M = I), so R0T[a][c] = integral over the box of
// phi_a psi_c, exact with mq = ceil((p + q + 1) / 2) Gauss points per direction (degree <= p + q in each
// variable).  One thread per (element, a, c).
__global__ void k_r0t(const int* __restrict__ perm, const double* __restrict__ bbox, const int* __restrict__ agg_int,
                      const double* __restrict__ agg_bbox, int ne, int p, int q, const double* __restrict__ gl_t,
                      const double* __restrict__ gl_w, int mq, double* __restrict__ r0t) {
  const int np = (p + 1) * (p + 2) / 2, nq = (q + 1) * (q + 2) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ne * np * nq) return;
  const int i = (int)(t / (np * nq)), ent = (int)(t % (np * nq)), a = ent / nq, c = ent % nq;
  const double* box = bbox + 4LL * perm[i];
  const double* cbox = agg_bbox + 4LL * agg_int[i];
  // (i, j) degrees of basis function a (degree d, i from d down to 0) and of coarse function c
  auto degrees = [](int idx, int* di, int* dj) {
    int d = 0;
    while (idx > d) { idx -= d + 1; ++d; }
    *di = d - idx;
    *dj = idx;
  };
  int ai, aj, ci, cj;
  degrees(a, &ai, &aj);
  degrees(c, &ci, &cj);
  const double wx = box[1] - box[0], wy = box[3] - box[2];
  const double cwx = cbox[1] - cbox[0], cwy = cbox[3] - cbox[2];
  const double na = sqrt((2.0 * ai + 1.0) * (2.0 * aj + 1.0) / (wx * wy));
  const double nc = sqrt((2.0 * ci + 1.0) * (2.0 * cj + 1.0) / (cwx * cwy));
  double acc = 0.0;
  for (int iu = 0; iu < mq; ++iu) {
    const double x = box[0] + wx * gl_t[iu];
    double Lx[10], dLx[10], Cx[10], dCx[10];
    legendre_dev(p, 2.0 * gl_t[iu] - 1.0, Lx, dLx);
    legendre_dev(q, 2.0 * (x - 0.5 * (cbox[0] + cbox[1])) / cwx, Cx, dCx);
    for (int iv = 0; iv < mq; ++iv) {
      const double y = box[2] + wy * gl_t[iv];
      double Ly[10], dLy[10], Cy[10], dCy[10];
      legendre_dev(p, 2.0 * gl_t[iv] - 1.0, Ly, dLy);
      legendre_dev(q, 2.0 * (y - 0.5 * (cbox[2] + cbox[3])) / cwy, Cy, dCy);
      acc = fma(gl_w[iu] * gl_w[iv], (Lx[ai] * Ly[aj]) * (Cx[ci] * Cy[cj]), acc);
    }
  }
  r0t[t] = acc * na * nc * wx * wy;
}

// A_0 = R_0 A R_0^T (Eq. A0) in two passes.  Pass 1, one thread per (block k, a, c): the block's
// contribution W_k = R_e^T B_k R_c (n_q x n_q; e the block's row element, c its column element).
__global__ void k_galerkin_w(const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ vals, const double* __restrict__ r0t, int ne, long long nnzb,
                             int np, int np2s, int nq, double* __restrict__ W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb * nq * nq) return;
  const long long k = t / (nq * nq);
  const int a = (int)((t / nq) % nq), cc = (int)(t % nq);
  int lo = 0, hi = ne;   // row element: rowptr[e] <= k < rowptr[e + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (rowptr[mid] <= k) lo = mid; else hi = mid;
  }
  const double* Re = r0t + (long long)lo * np * nq;
  const double* Rc = r0t + (long long)col[k] * np * nq;
  const double* Bk = vals + k * np2s;   // column-major: entry (r, m) at m * np + r
  double acc = 0.0;
  for (int r = 0; r < np; ++r) {
    double tr = 0.0;
    for (int m = 0; m < np; ++m) tr = fma(Bk[m * np + r], Rc[m * nq + cc], tr);
    acc = fma(Re[r * nq + a], tr, acc);
  }
  W[t] = acc;
}

// Pass 2, one warp per agglomerate J: the blocks of J's elements are added in a fixed order into the
// warp's shared copy of row block J of A_0, which is then written out (only this warp writes those
// rows, so no atomics; the sum order is deterministic).
__global__ void k_galerkin_sum(const int* __restrict__ grp_ptr, const int* __restrict__ grp_elems,
                               const int* __restrict__ agg_int, const int* __restrict__ rowptr,
                               const int* __restrict__ col, const double* __restrict__ W, int nagg, int nq,
                               double* __restrict__ A0) {
  extern __shared__ double rowJ[];   // [nq][n0]
  const int J = blockIdx.x, lane = threadIdx.x;
  const int n0 = nagg * nq, nqq = nq * nq;
  for (int t = lane; t < nq * n0; t += 32) rowJ[t] = 0.0;
  __syncwarp();
  for (int g = grp_ptr[J]; g < grp_ptr[J + 1]; ++g) {
    const int e = grp_elems[g];
    for (int k = rowptr[e]; k < rowptr[e + 1]; ++k) {
      const int Jc = agg_int[col[k]];
      for (int t = lane; t < nqq; t += 32) rowJ[(t / nq) * n0 + Jc * nq + t % nq] += W[(long long)k * nqq + t];
      __syncwarp();
    }
  }
  for (int t = lane; t < nq * n0; t += 32) A0[(long long)(J * nq + t / n0) * n0 + t % n0] = rowJ[t];
}

// A_0 = R_0 A R_0^T (Eq. A0) for a non-nested coarse space: one CTA per coarse cell J owns the rows J*nq ..
// of A_0 and adds, for every pair t = (e, J), block (e, e') of A and pair t' = (e', J'), the product
// R_t^T A_ee' R_t' into columns J'*nq .. (W = A_ee' R_t' first, in shared memory).  Each entry is updated by
// one thread, in the loop order, so the sum is deterministic.
__global__ void __launch_bounds__(128) k_galerkin_nn(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                     const double* __restrict__ vals, int np, int np2s, int nq,
                                                     const int* __restrict__ r0t_ptr, const int* __restrict__ r0t_col,
                                                     const int* __restrict__ r0t_elem, const double* __restrict__ r0t,
                                                     const int* __restrict__ rT_ptr, const int* __restrict__ rT_pair,
                                                     int n0, double* __restrict__ A0) {
  extern __shared__ double Wsm[];   // [np][nq]
  const int J = blockIdx.x;
  for (int pr = rT_ptr[J]; pr < rT_ptr[J + 1]; ++pr) {
    const int t = rT_pair[pr], e = r0t_elem[t];
    const double* R = r0t + (long long)t * np * nq;
    for (int kb = rowptr[e]; kb < rowptr[e + 1]; ++kb) {
      const int e2 = col[kb];
      const double* Ab = vals + (long long)kb * np2s;   // column-major: (a, b) at b * np + a
      for (int t2 = r0t_ptr[e2]; t2 < r0t_ptr[e2 + 1]; ++t2) {
        const double* R2 = r0t + (long long)t2 * np * nq;
        const long long c0 = (long long)r0t_col[t2] * nq;
        __syncthreads();   // the previous W has been used
        for (int i = threadIdx.x; i < np * nq; i += blockDim.x) {
          const int a = i / nq, c2 = i % nq;
          double w = 0.0;
          for (int b = 0; b < np; ++b) w = fma(Ab[b * np + a], R2[b * nq + c2], w);
          Wsm[i] = w;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nq * nq; i += blockDim.x) {
          const int c = i / nq, c2 = i % nq;
          double v = 0.0;
          for (int a = 0; a < np; ++a) v = fma(R[a * nq + c], Wsm[a * nq + c2], v);
          A0[(long long)(J * nq + c) * n0 + c0 + c2] += v;
        }
      }
    }
  }
}

// symmetrise, scale to unit diagonal and write the lower triangle of A_0 into its (dense) tile envelope
__global__ void k_coarse_scale(const double* __restrict__ A0, int n0, double* __restrict__ scale0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  double d = A0[(long long)i * n0 + i];
  scale0[i] = d > 0.0 ? 1.0 / sqrt(d) : __longlong_as_double(0x7ff8000000000000ULL);
}

__global__ void k_coarse_extract(const double* __restrict__ A0, int n0, const double* __restrict__ scale0, EnvDev E,
                                 double* __restrict__ Lr) {
  int nbt = (n0 + T - 1) / T;
  long long total = (long long)nbt * T * nbt * T;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int row = (int)(t / (nbt * T)), cl = (int)(t % (nbt * T));
    if (row < cl) continue;
    double v;
    if (row < n0 && cl < n0)
      v = 0.5 * (A0[(long long)row * n0 + cl] + A0[(long long)cl * n0 + row]) * scale0[row] * scale0[cl];
    else
      v = (row == cl) ? 1.0 : 0.0;
    Lr[tile_index(E, 0, row / T, cl / T) * TT + (row % T) * T + (cl % T)] = v;
  }
}

__global__ void k_identity(double* __restrict__ I, int n) {
  long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    I[t] = (t / n == t % n) ? 1.0 : 0.0;
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_permute_blocks(const double* src, const long long* src_blk, double* dst, long long nnzb, int np2s, void* st) {
  k_permute_blocks<<<grid_for(nnzb * np2s, 256), 256, 0, (cudaStream_t)st>>>(src, src_blk, dst, nnzb, np2s);
  return (int)cudaGetLastError();
}

int launch_scale(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s, double* scale, void* st) {
  k_scale<<<grid_for((long long)ne * np, 256), 256, 0, (cudaStream_t)st>>>(rowptr, col, vals, ne, np, np2s, scale);
  return (int)cudaGetLastError();
}

int launch_extract_rows(int prec, const EnvDev& E, const int* sub_e0, const int* rowptr, const int* col,
                        const double* vals, int np, int np2s, const double* scale, void* Lr, int nsub, int ne, void* st) {
  int blocks = (ne * 32 + 255) / 256;
  if (prec == 0)
    k_extract<double><<<blocks, 256, 0, (cudaStream_t)st>>>(E, sub_e0, rowptr, col, vals, np, np2s, scale, (double*)Lr, nsub);
  else
    k_extract<float><<<blocks, 256, 0, (cudaStream_t)st>>>(E, sub_e0, rowptr, col, vals, np, np2s, scale, (float*)Lr, nsub);
  return (int)cudaGetLastError();
}

int launch_chol_diag(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, int* err, void* st) {
  if (!n) return 0;
  if (prec == 0) k_chol_diag<double><<<n, 256, 0, (cudaStream_t)st>>>(E, (double*)L, K, tasks, err);
  else k_chol_diag<float><<<n, 256, 0, (cudaStream_t)st>>>(E, (float*)L, K, tasks, err);
  return (int)cudaGetLastError();
}

int launch_chol_panel(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, void* st) {
  if (!n) return 0;
  if (prec == 0) k_chol_panel<double><<<n, 256, 0, (cudaStream_t)st>>>(E, (double*)L, K, tasks);
  else k_chol_panel<float><<<n, 256, 0, (cudaStream_t)st>>>(E, (float*)L, K, tasks);
  return (int)cudaGetLastError();
}

int launch_chol_update(int prec, const EnvDev& E, void* L, int K, const int* tasks, int n, void* st) {
  if (!n) return 0;
  if (prec == 0) k_chol_update<double><<<n, 256, 0, (cudaStream_t)st>>>(E, (double*)L, K, tasks);
  else k_chol_update<float><<<n, 256, 0, (cudaStream_t)st>>>(E, (float*)L, K, tasks);
  return (int)cudaGetLastError();
}

int launch_to_colmajor(int prec, const void* Lr, void* Lc, long long ntiles, void* st) {
  int g = (int)(ntiles < 152 * 16 ? ntiles : 152 * 16);
  if (g < 1) g = 1;
  if (prec == 0) k_to_colmajor<double><<<g, 256, 0, (cudaStream_t)st>>>((const double*)Lr, (double*)Lc, ntiles);
  else k_to_colmajor<float><<<g, 256, 0, (cudaStream_t)st>>>((const float*)Lr, (float*)Lc, ntiles);
  return (int)cudaGetLastError();
}

int launch_gather_tiles(int prec, const void* src, const long long* idx, void* dst, long long ntiles, void* st) {
  int g = (int)(ntiles < 152 * 16 ? ntiles : 152 * 16);
  if (g < 1) g = 1;
  if (prec == 0) k_gather_tiles<double><<<g, 256, 0, (cudaStream_t)st>>>((const double*)src, idx, (double*)dst, ntiles);
  else k_gather_tiles<float><<<g, 256, 0, (cudaStream_t)st>>>((const float*)src, idx, (float*)dst, ntiles);
  return (int)cudaGetLastError();
}

int launch_dinv(int prec, const EnvDev& E, const void* L, const int* task, const long long* dinv_ptr, void* X, int nsr,
                void* st) {
  if (nsr <= 0) return 0;
  const dim3 grid(nsr, SUPER_ROW_MAX);
  if (prec == 0) k_dinv<double><<<grid, 256, 0, (cudaStream_t)st>>>(E, (const double*)L, task, dinv_ptr, (double*)X);
  else k_dinv<float><<<grid, 256, 0, (cudaStream_t)st>>>(E, (const float*)L, task, dinv_ptr, (float*)X);
  return (int)cudaGetLastError();
}

int launch_stream_gather(int prec, const void* L, const void* X, const long long* src, void* dst, long long n,
                         int transpose, void* st) {
  int g = (int)(n < 152 * 16 ? n : 152 * 16);
  if (g < 1) g = 1;
  if (prec == 0)
    k_stream_gather<double><<<g, 256, 0, (cudaStream_t)st>>>((const double*)L, (const double*)X, src, (double*)dst, n,
                                                              transpose);
  else
    k_stream_gather<float><<<g, 256, 0, (cudaStream_t)st>>>((const float*)L, (const float*)X, src, (float*)dst, n,
                                                             transpose);
  return (int)cudaGetLastError();
}

int launch_to_bf16(const float* src, void* dst, long long n, void* st) {
  k_to_bf16<<<grid_for(n, 256), 256, 0, (cudaStream_t)st>>>(src, (__nv_bfloat16*)dst, n);
  return (int)cudaGetLastError();
}

int launch_bjac_inverse(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s, double* dinv,
                        int* err, void* st) {
  const size_t smem = sizeof(double) * (size_t)BJAC_WARPS * (np * (np + 1) + np);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bjac_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  k_bjac_inverse<<<(ne + BJAC_WARPS - 1) / BJAC_WARPS, 32 * BJAC_WARPS, smem, (cudaStream_t)st>>>(rowptr, col, vals, ne, np, np2s,
                                                                                              dinv, err);
  return (int)cudaGetLastError();
}

int launch_r0t(const int* perm, const double* bbox, const int* agg_int, const double* agg_bbox, int ne, int p, int q,
               const double* gl_t, const double* gl_w, int mq, double* r0t, void* st) {
  const int np = (p + 1) * (p + 2) / 2, nq = (q + 1) * (q + 2) / 2;
  const long long n = (long long)ne * np * nq;
  k_r0t<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)st>>>(perm, bbox, agg_int, agg_bbox, ne, p, q, gl_t, gl_w, mq, r0t);
  return (int)cudaGetLastError();
}

int launch_galerkin_nn(const int* rowptr, const int* col, const double* vals, int np, int np2s, int nq,
                       const int* r0t_ptr, const int* r0t_col, const int* r0t_elem, const double* r0t, const int* rT_ptr,
                       const int* rT_pair, int nc, int n0, double* A0, void* st) {
  if (nc <= 0) return 0;
  k_galerkin_nn<<<nc, 128, sizeof(double) * np * nq, (cudaStream_t)st>>>(rowptr, col, vals, np, np2s, nq, r0t_ptr, r0t_col,
                                                                        r0t_elem, r0t, rT_ptr, rT_pair, n0, A0);
  return (int)cudaGetLastError();
}

int launch_galerkin(const int* grp_ptr, const int* grp_elems, const int* agg_int, const int* rowptr, const int* col,
                    const double* vals, const double* r0t, int ne, long long nnzb, int nagg, int np, int np2s, int nq,
                    double* W, double* A0, void* st) {
  const long long n = nnzb * nq * nq;
  k_galerkin_w<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)st>>>(rowptr, col, vals, r0t, ne, nnzb, np, np2s, nq, W);
  const size_t smem = sizeof(double) * (size_t)nq * nagg * nq;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_galerkin_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  k_galerkin_sum<<<nagg, 32, smem, (cudaStream_t)st>>>(grp_ptr, grp_elems, agg_int, rowptr, col, W, nagg, nq, A0);
  return (int)cudaGetLastError();
}

int launch_coarse_extract(const double* A0, int n0, double* scale0, const EnvDev& E0, double* Lr0, void* st) {
  k_coarse_scale<<<(n0 + 255) / 256, 256, 0, (cudaStream_t)st>>>(A0, n0, scale0);
  int nbt = (n0 + T - 1) / T;
  k_coarse_extract<<<grid_for((long long)nbt * T * nbt * T, 256), 256, 0, (cudaStream_t)st>>>(A0, n0, scale0, E0, Lr0);
  return (int)cudaGetLastError();
}

int launch_identity(double* I, int n, void* st) {
  k_identity<<<grid_for((long long)n * n, 256), 256, 0, (cudaStream_t)st>>>(I, n);
  return (int)cudaGetLastError();
}

}  // namespace dgasm
