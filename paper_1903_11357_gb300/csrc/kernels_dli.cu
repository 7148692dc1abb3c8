// Local solves with explicit subdomain inverses (Sec. 3, local solvers: z_i = A_i^{-1} r_i), the variant for
// small subdomains.  The inverse X_i = A_i^{-1} of every subdomain is formed once at setup from its Cholesky
// factor (the local-solve kernel applied to blocks of unit vectors) and stored dense, row-major; a local solve
// is then one matrix-vector product per subdomain with no sequential dependency: one warp per row, rows split
// into items of DLI_ROWS rows, and the partial (r, z) of each item summed in a fixed order.  For subdomains of a
// few hundred dofs the forward/backward sweeps are latency bound (a handful of dependent super-row steps with
// reductions) while the product streams n_i^2 entries at full bandwidth from L2 or HBM.
#include <cuda_runtime.h>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int NWD = NTHREADS / 32;

__device__ __forceinline__ int find_prob(const int* __restrict__ prefix, int nprob, int item) {
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename C> __device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// unit vectors: column kk of the block is e_(c0 + kk) of every subdomain (r zero on entry)
__global__ void k_unit_block(const int* __restrict__ sub_e0, int nsub, int np, int c0, int cb, long long ndof,
                             double* __restrict__ r) {
  const int s = blockIdx.x;
  if (s >= nsub) return;
  const int e0 = sub_e0[s], n = (sub_e0[s + 1] - e0) * np;
  for (int kk = threadIdx.x; kk < cb; kk += blockDim.x)
    if (c0 + kk < n) r[kk * ndof + (long long)e0 * np + c0 + kk] = 1.0;
}

// X_s[i][c0 + kk] = z[kk][d0_s + i] (column c0 + kk of A_s^{-1}; X_s is symmetric, stored row-major)
template <typename S>
__global__ void k_dli_store(const int* __restrict__ sub_e0, int np, const long long* __restrict__ off, int c0, int cb,
                            long long ndof, const double* __restrict__ z, S* __restrict__ X) {
  const int s = blockIdx.y;
  const int e0 = sub_e0[s], n = (sub_e0[s + 1] - e0) * np;
  const long long d0 = (long long)e0 * np;
  for (int i = blockIdx.x * blockDim.y + threadIdx.y; i < n; i += gridDim.x * blockDim.y)
    for (int kk = threadIdx.x; kk < cb && c0 + kk < n; kk += blockDim.x)
      X[off[s] + (long long)i * n + c0 + kk] = (S)z[kk * ndof + d0 + i];
}

// z_s = X_s r_s for the rows of one item; C: accumulation type (double for FP64 inverses, float otherwise)
template <typename S, typename C, int KM>
__global__ void __launch_bounds__(NTHREADS) k_dli(BatchDev B, int slot) {
  __shared__ double red[NWD][KMAX];
  const int pi = find_prob(B.prefix[slot], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[slot][pi];
  const int k = P.k;
  const int s = P.dli_item[2 * item], row0 = P.dli_item[2 * item + 1];
  const int e0 = P.sub_e0[s], n = (P.sub_e0[s + 1] - e0) * P.np;
  const long long d0 = (long long)e0 * P.np;
  const S* X = reinterpret_cast<const S*>(P.dli) + P.dli_off[s];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool act[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) act[kk] = kk < k && P.done[kk] == 0;
  double prz[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) prz[kk] = 0.0;
  const int row1 = min(row0 + DLI_ROWS, n);
  for (int i = row0 + w; i < row1; i += NWD) {
    const S* Xi = X + (long long)i * n;
    C acc[KM];
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) acc[kk] = (C)0;
#pragma unroll 4
    for (int j = lane; j < n; j += 32) {
      const C xv = (C)__ldg(Xi + j);
#pragma unroll
      for (int kk = 0; kk < KM; ++kk)
        if (act[kk]) acc[kk] = fma(xv, (C)P.r[kk * (long long)P.ndof + d0 + j], acc[kk]);
    }
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (!act[kk]) continue;
      const double v = (double)warp_sum<C>(acc[kk]);
      const long long o = kk * (long long)P.ndof + d0 + i;
      if (lane == 0) P.z[o] = v;
      prz[kk] = fma(P.r[o], v, prz[kk]);   // the same in every lane
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) red[w][kk] = prz[kk];
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double sum = 0.0;
    for (int ww = 0; ww < NWD; ++ww) sum += red[ww][threadIdx.x];
    P.part_rz[(long long)item * k + threadIdx.x] = P.done[threadIdx.x] == 0 ? sum : 0.0;
  }
}

}  // namespace

int launch_unit_block(const int* sub_e0, int nsub, int np, int c0, int cb, long long ndof, double* r, void* st) {
  k_unit_block<<<nsub, 64, 0, (cudaStream_t)st>>>(sub_e0, nsub, np, c0, cb, ndof, r);
  return (int)cudaGetLastError();
}

int launch_dli_store(int fp64, const int* sub_e0, int nsub, int np, const long long* off, int c0, int cb,
                     long long ndof, const double* z, void* X, int nmax, void* st) {
  const dim3 block(32, 8), grid((unsigned)((nmax + 7) / 8), (unsigned)nsub);
  if (fp64) k_dli_store<double><<<grid, block, 0, (cudaStream_t)st>>>(sub_e0, np, off, c0, cb, ndof, z, (double*)X);
  else k_dli_store<float><<<grid, block, 0, (cudaStream_t)st>>>(sub_e0, np, off, c0, cb, ndof, z, (float*)X);
  return (int)cudaGetLastError();
}

// slot K_DLI: FP64 inverses, K_DLI + 1: FP32 inverses
int launch_dli(const BatchDev& B, int slot, int total, int km, void* st) {
  cudaStream_t s = (cudaStream_t)st;
  if (slot == K_DLI) {
    if (km == 1) k_dli<double, double, 1><<<total, NTHREADS, 0, s>>>(B, slot);
    else k_dli<double, double, KMAX><<<total, NTHREADS, 0, s>>>(B, slot);
  } else {
    if (km == 1) k_dli<float, float, 1><<<total, NTHREADS, 0, s>>>(B, slot);
    else k_dli<float, float, KMAX><<<total, NTHREADS, 0, s>>>(B, slot);
  }
  return (int)cudaGetLastError();
}

}  // namespace dgasm
