// Batched ASPCG kernels (Sec. 7): block-sparse SpMV q = A p, the fused x/r update with the coarse
// restriction r_0 = R_0 r, the local subdomain solves z_i = A_i^{-1} r_i by forward and backward
// substitution with tile-envelope Cholesky factors, the coarse solve z_0 = A_0^{-1} r_0 and the search
// direction update p = z + beta p with z = sum_i R_i^T z_i + R_0^T z_0 (Sec. 3, P_ad = B A).
//
// Every kernel works on a batch of problems: CTA b maps to (problem, item) through a per-kind prefix
// array.  Inner products are reduced deterministically: each CTA writes its partial sums, and the last
// CTA of the kernel for a problem (detected with a fenced atomic counter) adds them in item order, so
// results do not depend on scheduling or on the other problems of the batch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int T = 32;
constexpr int TT = T * T;
constexpr int NW = NTHREADS / 32;

__device__ __forceinline__ int find_prob(const int* __restrict__ prefix, int nprob, int item) {
  int lo = 0, hi = nprob;  // prefix[lo] <= item < prefix[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// deterministic CTA sum of k values per thread; result in out[0..k) (shared), all threads synced
__device__ void block_sum_k(const double* v, int k, double* red /*[NW][KMAX]*/, double* out) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    if (kk < k) {
      double s = warp_sum(v[kk]);
      if (lane == 0) red[w * KMAX + kk] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int ww = 0; ww < NW; ++ww) s += red[ww * KMAX + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// returns true in the last CTA of this kernel for problem P (all CTAs must call it exactly once)
__device__ bool last_block(unsigned int* counter, unsigned int n_items, int* flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    *flag_smem = (prev == n_items - 1);
    if (*flag_smem) *counter = 0u;
  }
  __syncthreads();
  bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// ---- SpMV: q = A p (operand 0, with partial (p, q)) or q = A x and (b - A x)^2 (operand 1) ------
__global__ void __launch_bounds__(NTHREADS) k_spmv(BatchDev B, int operand) {
  __shared__ double red[NW * KMAX];
  __shared__ double tot[KMAX];
  __shared__ int lastf;
  const int pi = find_prob(B.prefix[K_SPMV], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_SPMV][pi];
  const int k = P.k, np = P.np;
  bool act[KMAX];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    act[kk] = kk < k && (operand == 1 || P.done[kk] == 0);
    any |= act[kk];
  }
  double part[KMAX];
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) part[kk] = 0.0;
  if (any) {
    const int e_begin = item * P.epi;
    const int nel = min(P.epi, P.ne - e_begin);
    const int t = threadIdx.x;
    if (t < nel * np) {
      const int e = e_begin + t / np, r = t % np;
      const double* vec = operand == 0 ? P.p : P.x;
      double acc[KMAX];
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) acc[kk] = 0.0;
      for (int kb = P.rowptr[e]; kb < P.rowptr[e + 1]; ++kb) {
        const double* blk = P.vals + (long long)kb * P.np2s + r;
        const double* xc = vec + (long long)P.col[kb] * np;
        for (int c = 0; c < np; ++c) {
          double a = __ldg(blk + c * np);
#pragma unroll
          for (int kk = 0; kk < KMAX; ++kk)
            if (act[kk]) acc[kk] = fma(a, xc[(long long)kk * P.ndof + c], acc[kk]);
        }
      }
      const long long d = (long long)e * np + r;
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) {
        if (!act[kk]) continue;
        P.q[kk * (long long)P.ndof + d] = acc[kk];
        if (operand == 0) {
          part[kk] = P.p[kk * (long long)P.ndof + d] * acc[kk];
        } else {
          double rr = P.b[kk * (long long)P.ndof + d] - acc[kk];
          part[kk] = rr * rr;
        }
      }
    }
  }
  block_sum_k(part, k, red, tot);
  if (threadIdx.x < k) P.part_pq[(long long)item * k + threadIdx.x] = tot[threadIdx.x];
  if (!last_block(&P.counters[C_SPMV], P.n_chunk_items, &lastf)) return;
  if (threadIdx.x < k) {
    const int kk = threadIdx.x;
    if (!act[kk]) return;
    double s = 0.0;
    for (int i = 0; i < P.n_chunk_items; ++i) s += P.part_pq[(long long)i * k + kk];
    if (operand == 1) {
      P.true_rr[kk] = P.bnorm[kk] > 0.0 ? sqrt(s) / P.bnorm[kk] : 0.0;
      return;
    }
    double alpha = P.gamma[kk] / s;
    if (!(s > 0.0) || !finite_d(alpha)) {
      P.status[kk] = DGASM_ENAN;
      P.done[kk] = 3;
      atomicSub(P.remaining, 1);
      alpha = 0.0;
    }
    P.alpha[kk] = alpha;
  }
}

// ---- x/r update (or initial residual) with partial ||r||^2 and the coarse restriction ----------
__global__ void __launch_bounds__(NTHREADS) k_update(BatchDev B, int mode) {
  __shared__ double red[NW * KMAX];
  __shared__ double tot[KMAX];
  __shared__ int lastf;
  const int pi = find_prob(B.prefix[K_GRP], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int g = blockIdx.x - B.prefix[K_GRP][pi];
  const int k = P.k, np = P.np, nq = P.nq;
  bool act[KMAX];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  double alpha[KMAX];
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) alpha[kk] = (mode == MODE_ITER && act[kk]) ? P.alpha[kk] : 0.0;
  const int g0 = P.grp_ptr[g], g1 = P.grp_ptr[g + 1];
  const int nd = (g1 - g0) * np;
  double prr[KMAX];
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) prr[kk] = 0.0;
  // restriction accumulators: at most KMAX x 3 (q = 1) are kept per thread; larger nq loop below
  const bool restrict_ = nq > 0;
  for (int base = 0; base < nd && any; base += NTHREADS) {
    const int t = base + threadIdx.x;
    if (t >= nd) break;
    const int e = P.grp_elems[g0 + t / np], a = t % np;
    const long long d = (long long)e * np + a;
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk) {
      if (!act[kk]) continue;
      const long long o = kk * (long long)P.ndof + d;
      double rv;
      if (mode == MODE_INIT) {
        rv = P.b_user[kk * (long long)P.ndof + (long long)P.perm[e] * np + a];
        P.b[o] = rv;
        P.x[o] = 0.0;
      } else {
        P.x[o] = fma(alpha[kk], P.p[o], P.x[o]);
        rv = fma(-alpha[kk], P.q[o], P.r[o]);
      }
      P.r[o] = rv;
      prr[kk] = fma(rv, rv, prr[kk]);
    }
  }
  block_sum_k(prr, k, red, tot);
  if (threadIdx.x < k) P.part_rr[(long long)g * k + threadIdx.x] = tot[threadIdx.x];
  if (restrict_ && any) {
    // r_0[J*nq + c] = sum_{e in J} sum_a R0T_e[a][c] r_e[a], reduced per (c) in a fixed order
    for (int c = 0; c < nq; ++c) {
      double v[KMAX];
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) v[kk] = 0.0;
      for (int base = 0; base < nd; base += NTHREADS) {
        const int t = base + threadIdx.x;
        if (t >= nd) break;
        const int e = P.grp_elems[g0 + t / np], a = t % np;
        const double w = P.r0t[((long long)e * np + a) * nq + c];
#pragma unroll
        for (int kk = 0; kk < KMAX; ++kk)
          if (act[kk]) v[kk] = fma(w, P.r[kk * (long long)P.ndof + (long long)e * np + a], v[kk]);
      }
      block_sum_k(v, k, red, tot);
      if (threadIdx.x < k && act[threadIdx.x]) P.r0[(long long)threadIdx.x * P.n0 + g * nq + c] = tot[threadIdx.x];
    }
  }
  if (!last_block(&P.counters[C_GRP], P.ngrp, &lastf)) return;
  if (threadIdx.x < k) {
    const int kk = threadIdx.x;
    if (!act[kk]) return;
    double s = 0.0;
    for (int i = 0; i < P.ngrp; ++i) s += P.part_rr[(long long)i * k + kk];
    if (mode == MODE_INIT) {
      double bn = sqrt(s);
      P.bnorm[kk] = bn;
      P.relres[kk] = bn > 0.0 ? 1.0 : 0.0;
      P.iters[kk] = 0;
      if (!finite_d(bn)) {
        P.status[kk] = DGASM_ENAN;
        P.done[kk] = 3;
        atomicSub(P.remaining, 1);
      } else if (bn == 0.0) {
        P.done[kk] = 1;
        atomicSub(P.remaining, 1);
      }
      return;
    }
    const double rel = sqrt(s) / P.bnorm[kk];
    const int it = P.iters[kk] + 1;
    P.iters[kk] = it;
    P.relres[kk] = rel;
    if (it <= P.maxit) P.alpha_hist[(long long)kk * P.maxit + it - 1] = P.alpha[kk];
    int newdone = 0;
    if (!finite_d(rel)) { P.status[kk] = DGASM_ENAN; newdone = 3; }
    else if (P.fixed_iters > 0) { if (it >= P.fixed_iters) newdone = 1; }
    else if (rel <= P.rtol) newdone = 1;
    else if (it >= P.maxit) newdone = 2;
    if (newdone) {
      P.done[kk] = newdone;
      atomicSub(P.remaining, 1);
    }
  }
}

// ---- local solves z_i = A_i^{-1} r_i with the scaled tile-envelope factor -----------------------
template <typename S> __device__ __forceinline__ float to_f(S v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S, typename C> __device__ __forceinline__ C ld_c(const S* p);
template <> __device__ __forceinline__ double ld_c<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_c<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_c<__nv_bfloat16, float>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

template <typename S, typename C, int KCT>
__global__ void __launch_bounds__(NTHREADS) k_local(BatchDev B, int slot) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[NW * KMAX];
  __shared__ double tot[KMAX];
  const int* prefix = B.prefix[slot];
  const int pi = find_prob(prefix, B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int li = blockIdx.x - prefix[pi];
  const int s = li / P.n_rhs_chunks, ch = li % P.n_rhs_chunks;
  const int k0 = ch * KCT;
  const int kc = min(KCT, P.k - k0);
  bool act[KCT];
  bool any = false;
#pragma unroll
  for (int j = 0; j < KCT; ++j) {
    act[j] = j < kc && P.done[k0 + j] == 0;
    any |= act[j];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e0 = P.sub_e0[s];
  const int n = (P.sub_e0[s + 1] - e0) * P.np;
  const long long d0 = (long long)e0 * P.np;
  const int nbt = (n + T - 1) / T, npad = nbt * T;
  if (!any) return;
  C* y = reinterpret_cast<C*>(smem_raw);  // [KCT][npad]
  C* part = y + KCT * npad;                // [NW][KCT][T]
  C* tmp = part + NW * KCT * T;            // [KCT][T]
  for (int idx = threadIdx.x; idx < KCT * npad; idx += NTHREADS) {
    const int j = idx / npad, i = idx - j * npad;
    C v = (C)0;
    if (i < n && act[j]) v = (C)(P.scale[d0 + i] * P.r[(long long)(k0 + j) * P.ndof + d0 + i]);
    y[idx] = v;
  }
  __syncthreads();
  const int tr0 = P.sub_trow[s];
  const S* Lc = reinterpret_cast<const S*>(P.Lc);
  const S* Lr = reinterpret_cast<const S*>(P.Lr);
  // forward substitution: y_I <- inv(L_II) (y_I - sum_{J<I} L_IJ y_J), column-major tiles
  for (int I = 0; I < nbt; ++I) {
    const int F = P.trow_F[tr0 + I];
    const long long base = P.trow_ptr[tr0 + I];
    const int nt = I - F;
    C acc[KCT];
#pragma unroll
    for (int j = 0; j < KCT; ++j) acc[j] = (C)0;
    for (int jt = w; jt < nt; jt += NW) {
      const S* tile = Lc + (base + jt) * TT + lane;
      const C* yv = y + (F + jt) * T;
#pragma unroll 8
      for (int c = 0; c < T; ++c) {
        const C a = ld_c<S, C>(tile + c * T);
#pragma unroll
        for (int j = 0; j < KCT; ++j) acc[j] += a * yv[j * npad + c];
      }
    }
#pragma unroll
    for (int j = 0; j < KCT; ++j) part[(w * KCT + j) * T + lane] = acc[j];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int j = 0; j < KCT; ++j) {
        C v = y[j * npad + I * T + lane];
        for (int ww = 0; ww < NW; ++ww) v -= part[(ww * KCT + j) * T + lane];
        tmp[j * T + lane] = v;
      }
      __syncwarp();
      const S* D = Lc + (base + nt) * TT + lane;
      C o[KCT];
#pragma unroll
      for (int j = 0; j < KCT; ++j) o[j] = (C)0;
#pragma unroll 8
      for (int c = 0; c < T; ++c) {
        const C a = ld_c<S, C>(D + c * T);
#pragma unroll
        for (int j = 0; j < KCT; ++j) o[j] += a * tmp[j * T + c];
      }
#pragma unroll
      for (int j = 0; j < KCT; ++j) y[j * npad + I * T + lane] = o[j];
    }
    __syncthreads();
  }
  // backward substitution with L^T: x_J <- inv(L_JJ)^T y_J, then y_K -= L_JK^T x_J, row-major tiles
  for (int J = nbt - 1; J >= 0; --J) {
    const int F = P.trow_F[tr0 + J];
    const long long base = P.trow_ptr[tr0 + J];
    const int nt = J - F;
    if (w == 0) {
      const S* D = Lr + (base + nt) * TT + lane;
      C o[KCT];
#pragma unroll
      for (int j = 0; j < KCT; ++j) o[j] = (C)0;
#pragma unroll 8
      for (int r = 0; r < T; ++r) {
        const C a = ld_c<S, C>(D + r * T);
#pragma unroll
        for (int j = 0; j < KCT; ++j) o[j] += a * y[j * npad + J * T + r];
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < KCT; ++j) y[j * npad + J * T + lane] = o[j];
    }
    __syncthreads();
    for (int jt = w; jt < nt; jt += NW) {
      const S* tile = Lr + (base + jt) * TT + lane;
      const C* xv = y + J * T;
      C acc[KCT];
#pragma unroll
      for (int j = 0; j < KCT; ++j) acc[j] = (C)0;
#pragma unroll 8
      for (int r = 0; r < T; ++r) {
        const C a = ld_c<S, C>(tile + r * T);
#pragma unroll
        for (int j = 0; j < KCT; ++j) acc[j] += a * xv[j * npad + r];
      }
#pragma unroll
      for (int j = 0; j < KCT; ++j) y[j * npad + (F + jt) * T + lane] -= acc[j];
    }
    __syncthreads();
  }
  // z_i = D^{-1/2} y, partial (r, z) for this subdomain
  double prz[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) prz[j] = 0.0;
  for (int i = threadIdx.x; i < n; i += NTHREADS) {
    const double sc = P.scale[d0 + i];
#pragma unroll
    for (int j = 0; j < KCT; ++j) {
      if (!act[j]) continue;
      const long long o = (long long)(k0 + j) * P.ndof + d0 + i;
      const double zv = sc * (double)y[j * npad + i];
      P.z[o] = zv;
      prz[j] = fma(P.r[o], zv, prz[j]);
    }
  }
  block_sum_k(prz, KCT, red, tot);
  if (threadIdx.x < kc) P.part_rz[(long long)s * P.k + k0 + threadIdx.x] = act[threadIdx.x] ? tot[threadIdx.x] : 0.0;
}

// ---- coarse solve z_0 = A_0^{-1} r_0: one warp per row of the explicit inverse -------------------
__global__ void __launch_bounds__(NTHREADS) k_coarse(BatchDev B) {
  __shared__ double wpart[NW][KMAX];
  const int pi = find_prob(B.prefix[K_COARSE], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_COARSE][pi];
  const int k = P.k, n0 = P.n0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = item * NW + w;
  bool act[KMAX];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  if (!any) return;
  double acc[KMAX];
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) acc[kk] = 0.0;
  if (row < n0) {
    const double* Arow = P.A0inv + (long long)row * n0;
    for (int j = lane; j < n0; j += 32) {
      const double a = __ldg(Arow + j);
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk)
        if (act[kk]) acc[kk] = fma(a, P.r0[(long long)kk * n0 + j], acc[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    if (kk >= k) break;
    double v = warp_sum(acc[kk]);
    if (lane == 0) {
      double prod = 0.0;
      if (row < n0 && act[kk]) {
        P.z0[(long long)kk * n0 + row] = v;
        prod = v * P.r0[(long long)kk * n0 + row];
      }
      wpart[w][kk] = prod;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int ww = 0; ww < NW; ++ww) s += wpart[ww][threadIdx.x];
    P.part_c[(long long)item * k + threadIdx.x] = s;
  }
}

// ---- p = z + R_0^T z_0 + beta p, beta = (r, z)_new / (r, z)_old ----------------------------------
__global__ void __launch_bounds__(NTHREADS) k_pupdate(BatchDev B, int mode) {
  __shared__ double beta_s[KMAX];
  __shared__ double gnew_s[KMAX];
  __shared__ int lastf;
  const int pi = find_prob(B.prefix[K_SPMV], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_SPMV][pi];
  const int k = P.k, np = P.np, nq = P.nq;
  bool act[KMAX];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  if (threadIdx.x < k) {
    const int kk = threadIdx.x;
    double g = 0.0;
    if (act[kk]) {
      for (int s = 0; s < P.nsub; ++s) g += P.part_rz[(long long)s * k + kk];
      if (nq > 0)
        for (int i = 0; i < P.n_coarse_items; ++i) g += P.part_c[(long long)i * k + kk];
    }
    gnew_s[kk] = g;
    beta_s[kk] = (mode == MODE_INIT || !act[kk]) ? 0.0 : g / P.gamma[kk];
  }
  __syncthreads();
  if (any) {
    const int e_begin = item * P.epi;
    const int nel = min(P.epi, P.ne - e_begin);
    const int t = threadIdx.x;
    if (t < nel * np) {
      const int e = e_begin + t / np, a = t % np;
      const long long d = (long long)e * np + a;
      const int J = nq > 0 ? P.agg_int[e] : 0;
#pragma unroll
      for (int kk = 0; kk < KMAX; ++kk) {
        if (!act[kk]) continue;
        const long long o = kk * (long long)P.ndof + d;
        double zv = P.z[o];
        if (nq > 0) {
          const double* R = P.r0t + d * nq;
          const double* z0 = P.z0 + (long long)kk * P.n0 + J * nq;
          for (int c = 0; c < nq; ++c) zv = fma(R[c], z0[c], zv);
        }
        P.p[o] = (mode == MODE_INIT) ? zv : fma(beta_s[kk], P.p[o], zv);
      }
    }
  }
  if (!last_block(&P.counters[C_PUPD], P.n_chunk_items, &lastf)) return;
  if (threadIdx.x < k) {
    const int kk = threadIdx.x;
    if (!act[kk]) return;
    const double g = gnew_s[kk];
    if (mode == MODE_ITER) {
      const int it = P.iters[kk];
      if (it >= 1 && it <= P.maxit) P.beta_hist[(long long)kk * P.maxit + it - 1] = beta_s[kk];
    }
    P.gamma[kk] = g;
    if (!finite_d(g) || !(g > 0.0)) {
      P.status[kk] = DGASM_ENAN;
      P.done[kk] = 3;
      atomicSub(P.remaining, 1);
    }
  }
}

// ---- internal -> caller order for x (operand 0) or p (operand 1, used by the preconditioner apply)
__global__ void __launch_bounds__(NTHREADS) k_finish(BatchDev B, int operand) {
  const int pi = find_prob(B.prefix[K_SPMV], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_SPMV][pi];
  const int np = P.np;
  const int e_begin = item * P.epi;
  const int nel = min(P.epi, P.ne - e_begin);
  const int t = threadIdx.x;
  if (t >= nel * np) return;
  const int e = e_begin + t / np, a = t % np;
  const double* src = operand == 0 ? P.x : P.p;
  for (int kk = 0; kk < P.k; ++kk)
    P.x_user[kk * (long long)P.ndof + (long long)P.perm[e] * np + a] = src[kk * (long long)P.ndof + (long long)e * np + a];
}

// ---- y = A x in the caller's element order (system matrix), no reductions -----------------------
__global__ void k_system_spmv(const int* __restrict__ rowptr, const int* __restrict__ col,
                              const double* __restrict__ vals, int ne, int np, int np2s, const double* __restrict__ x,
                              double* __restrict__ y) {
  const int epi = NTHREADS / np;
  const int e_begin = blockIdx.x * epi;
  const int nel = min(epi, ne - e_begin);
  const int t = threadIdx.x;
  if (t >= nel * np) return;
  const int e = e_begin + t / np, r = t % np;
  double acc = 0.0;
  for (int kb = rowptr[e]; kb < rowptr[e + 1]; ++kb) {
    const double* blk = vals + (long long)kb * np2s + r;
    const double* xc = x + (long long)col[kb] * np;
    for (int c = 0; c < np; ++c) acc = fma(blk[c * np], xc[c], acc);
  }
  y[(long long)e * np + r] = acc;
}

// Opt in to the largest dynamic shared memory once per kernel instantiation (and device), before any
// stream capture: the first launch of each instantiation happens in the uncaptured initial step.
template <typename K>
int ensure_smem(K fn, int smem) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  if (smem <= 48 * 1024) return 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({(const void*)fn, dev})) return 0;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
  if (e != cudaSuccess) return (int)e;
  done.insert({(const void*)fn, dev});
  return 0;
}

template <typename S, typename C>
int launch_local_t(const BatchDev& B, int slot, int kcl, int total, int smem, cudaStream_t st) {
  if (kcl == 0) {
    auto fn = k_local<S, C, 1>;
    if (int e = ensure_smem(fn, smem)) return e;
    fn<<<total, NTHREADS, smem, st>>>(B, slot);
  } else {
    auto fn = k_local<S, C, KC>;
    if (int e = ensure_smem(fn, smem)) return e;
    fn<<<total, NTHREADS, smem, st>>>(B, slot);
  }
  return (int)cudaGetLastError();
}

}  // namespace

int local_smem_bytes(int prec, int ndof_max, int kc) {
  int npad = ((ndof_max + T - 1) / T) * T;
  int csize = prec == 0 ? 8 : 4;
  int kct = kc > 1 ? KC : 1;
  return csize * (kct * npad + NW * kct * T + kct * T);
}

int launch_spmv(const BatchDev& B, int total, int operand, void* st) {
  k_spmv<<<total, NTHREADS, 0, (cudaStream_t)st>>>(B, operand);
  return (int)cudaGetLastError();
}

int launch_update(const BatchDev& B, int total, int mode, int /*use_q*/, void* st) {
  k_update<<<total, NTHREADS, 0, (cudaStream_t)st>>>(B, mode);
  return (int)cudaGetLastError();
}

// slot = K_NKINDS + 2 * prec + (kc > 1)
int launch_local(const BatchDev& B, int slot, int total, int smem, void* st) {
  const int prec = (slot - K_NKINDS) / 2, kcl = (slot - K_NKINDS) % 2;
  cudaStream_t s = (cudaStream_t)st;
  switch (prec) {
    case DGASM_FP64: return launch_local_t<double, double>(B, slot, kcl, total, smem, s);
    case DGASM_FP32:
    case DGASM_TF32: return launch_local_t<float, float>(B, slot, kcl, total, smem, s);
    default: return launch_local_t<__nv_bfloat16, float>(B, slot, kcl, total, smem, s);
  }
}

int launch_coarse(const BatchDev& B, int total, void* st) {
  k_coarse<<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  return (int)cudaGetLastError();
}

int launch_pupdate(const BatchDev& B, int total, int mode, void* st) {
  k_pupdate<<<total, NTHREADS, 0, (cudaStream_t)st>>>(B, mode);
  return (int)cudaGetLastError();
}

int launch_finish(const BatchDev& B, int total, int operand, void* st) {
  k_finish<<<total, NTHREADS, 0, (cudaStream_t)st>>>(B, operand);
  return (int)cudaGetLastError();
}

int launch_system_spmv(const int* rowptr, const int* col, const double* vals, int ne, int np, int np2s, const double* x,
                       double* y, void* st) {
  const int epi = NTHREADS / np;
  k_system_spmv<<<(ne + epi - 1) / epi, NTHREADS, 0, (cudaStream_t)st>>>(rowptr, col, vals, ne, np, np2s, x, y);
  return (int)cudaGetLastError();
}

}  // namespace dgasm
