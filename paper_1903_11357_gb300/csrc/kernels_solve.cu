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

#include "engine.h"

namespace dgasm {

namespace {

constexpr int NW = NTHREADS / 32;
// the x / r update runs one CTA per element group (an agglomerate, about 64 elements); 512 threads per CTA
// measured slower than 256 (the kernel's time is its serial tail, not the pass over the group)
constexpr int UPD_THREADS = 256;
constexpr int UPD_NW = UPD_THREADS / 32;

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
template <int KM, int NWB = NW>
__device__ void block_sum_k(const double* v, int k, double* red /*[NWB][KMAX]*/, double* out) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    if (kk < k) {
      double s = warp_sum(v[kk]);
      if (lane == 0) red[w * KMAX + kk] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int ww = 0; ww < NWB; ++ww) s += red[ww * KMAX + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// the problem descriptor in shared memory: one coalesced copy per CTA, so the kernel's many field reads
// (and the pointer chains that start from them) do not each pay a global-memory round trip
static_assert(sizeof(ProbDev) % 8 == 0, "ProbDev is copied as 8-byte words");
__device__ __forceinline__ const ProbDev& stage_prob(const ProbDev* src, ProbDev* dst) {
  constexpr int W = (int)(sizeof(ProbDev) / 8);
  for (int i = threadIdx.x; i < W; i += blockDim.x)
    reinterpret_cast<long long*>(dst)[i] = reinterpret_cast<const long long*>(src)[i];
  __syncthreads();
  return *dst;
}

// sum of v[i * stride] for i < n by one warp, in a fixed order (lane-strided partial sums, then a fixed
// shuffle tree); every lane returns the total
__device__ __forceinline__ double warp_sum_strided(const double* v, int n, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += v[(long long)i * stride];
  return warp_sum(s);
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

// one thread per (element, row): q_e[r] = sum over the blocks of row e of B[r][c] x_col[c], with the
// block width NP known at compile time (fully unrolled, two accumulator chains per right-hand side)
template <int NP, int KM>
__device__ __forceinline__ void spmv_rows(const ProbDev& P, int item, int operand, const bool* act, double* part) {
  const int e_begin = item * P.epi_spmv;
  const int nel = min(P.epi_spmv, P.ne - e_begin);
  const int t = threadIdx.x;
  if (t >= nel * NP) return;
  const int e = e_begin + t / NP, r = t % NP;
  const double* vec = operand == 0 ? P.p : P.x;
  const int k = P.k;
  double acc[KM][2];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) acc[kk][0] = acc[kk][1] = 0.0;
  const int kb0 = P.rowptr[e], kb1 = P.rowptr[e + 1];
  for (int kb = kb0; kb < kb1; ++kb) {
    const double* blk = P.vals + (long long)kb * P.np2s + r;
    const double* xc = vec + (long long)__ldg(P.col + kb) * NP;
    double a[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) a[c] = __ldg(blk + c * NP);
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (kk >= k || !act[kk]) continue;
      const double* xk = xc + (long long)kk * P.ndof;
#pragma unroll
      for (int c = 0; c < NP; ++c) acc[kk][c & 1] = fma(a[c], xk[c], acc[kk][c & 1]);
    }
  }

  const long long d = (long long)e * NP + r;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    if (kk >= k || !act[kk]) continue;
    const double q = acc[kk][0] + acc[kk][1];
    P.q[kk * (long long)P.ndof + d] = q;
    if (operand == 0) {
      part[kk] = P.p[kk * (long long)P.ndof + d] * q;
    } else {
      const double rr = P.b[kk * (long long)P.ndof + d] - q;
      part[kk] = rr * rr;
    }
  }
}

// ---- SpMV: q = A p (operand 0, with partial (p, q)) or q = A x and (b - A x)^2 (operand 1) ------
template <int NP, int KM>
__global__ void __launch_bounds__(SPMV_THREADS) k_spmv(BatchDev B, int operand, int slot) {
  constexpr int SW = SPMV_THREADS / 32;
  __shared__ double red[SW * KMAX];
  __shared__ double tot[KMAX];
  __shared__ int lastf;
  __shared__ __align__(16) ProbDev Ps;
  const int pi = find_prob(B.prefix[slot], B.nprob, blockIdx.x);
  const ProbDev& P = stage_prob(B.probs + pi, &Ps);
  const int item = blockIdx.x - B.prefix[slot][pi];
  const int k = P.k;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && (operand == 1 || P.done[kk] == 0);
    any |= act[kk];
  }
  double part[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) part[kk] = 0.0;
  if (any) spmv_rows<NP, KM>(P, item, operand, act, part);
  block_sum_k<KM, SW>(part, k, red, tot);
  if (threadIdx.x < k) P.part_pq[(long long)item * k + threadIdx.x] = tot[threadIdx.x];
  // q = A p: the x/r update that follows sums the (p, q) partials itself (alpha in every CTA), so this
  // kernel ends without a last-CTA step
  if (operand == 0) return;
  if (!last_block(&P.counters[C_SPMV], P.n_spmv_items, &lastf)) return;
  for (int kk = threadIdx.x >> 5; kk < k; kk += SW) {
    if (!act[kk]) continue;
    const double s = warp_sum_strided(P.part_pq + kk, P.n_spmv_items, k);
    if ((threadIdx.x & 31) == 0) P.true_rr[kk] = P.bnorm[kk] > 0.0 ? sqrt(s) / P.bnorm[kk] : 0.0;
  }
}

// ---- x/r update (or initial residual) with partial ||r||^2 and the coarse restriction ----------
template <int KM>
__global__ void __launch_bounds__(UPD_THREADS) k_update(BatchDev B, int mode, int gslot) {
  __shared__ double red[UPD_NW * KMAX];
  __shared__ double tot[KMAX];
  __shared__ double alpha_s[KMAX];
  __shared__ int bad_s[KMAX];
  __shared__ double colbuf[4][UPD_THREADS];   // per-thread values of up to four sums at a time
  __shared__ int lastf;
  __shared__ __align__(16) ProbDev Ps;
  const int pi = find_prob(B.prefix[K_GRP], B.nprob, blockIdx.x);
  const ProbDev& P = stage_prob(B.probs + pi, &Ps);
  const int g = blockIdx.x - B.prefix[K_GRP][pi];
  const int k = P.k, np = P.np, nq = P.nq;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  // alpha = gamma / (p, q) from the SpMV's partial sums, formed identically in every CTA; a right-hand side
  // whose (p, q) is not positive or whose alpha is not finite is left alone here and failed by the last CTA
  double alpha[KM];
  bool bad[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    alpha[kk] = 0.0;
    bad[kk] = false;
  }
  // loads that do not depend on the sums below are issued before them
  const int g0 = P.grp_ptr[g], g1 = P.grp_ptr[g + 1];
  // FP64 instructions are scarce on this part (each warp instruction costs the pipe the same whatever its
  // active lanes), so one warp per right-hand side sums the (p, q) partials and one lane divides
  if (mode == MODE_ITER) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = P.n_spmv_items;
    for (int kk = wid; kk < k; kk += UPD_NW) {
      double sum = 0.0;
      for (int i0 = lane; i0 < n; i0 += 8 * 32) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + 32 * u;
          v[u] = i < n ? P.part_pq[(long long)i * k + kk] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) sum += v[u];
      }
      sum = warp_sum(sum);
      if (lane == 0) {
        const double a = (gslot ? P.gamma1 : P.gamma)[kk] / sum;
        const int b = !(sum > 0.0) || !finite_d(a);
        alpha_s[kk] = b ? 0.0 : a;
        bad_s[kk] = b;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (!act[kk]) continue;
      if (bad_s[kk]) {
        bad[kk] = true;
        act[kk] = false;
      } else {
        alpha[kk] = alpha_s[kk];
      }
    }
    any = false;
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) any |= act[kk];
  }
  const int nd = (g1 - g0) * np;
  // one pass: x/r update, ||r||^2 and, for q = 1 (nq = 3), the restriction r_0[J] = sum R0T^T r
  constexpr int NQ1 = 3;
  double prr[KM], pr0[KM][NQ1];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    prr[kk] = 0.0;
#pragma unroll
    for (int c = 0; c < NQ1; ++c) pr0[kk][c] = 0.0;
  }
  // non-nested coarse spaces restrict in their own kernel (an element meets several coarse cells)
  const bool restrict_ = nq > 0 && P.r0t_ptr == nullptr;
  const bool fused_r0 = restrict_ && nq == NQ1;
  if (mode == MODE_ITER) {
    // the CG update, H dofs per thread and pass (all index loads, then all data loads of the pass, issued
    // before the stores); each thread still accumulates its dofs t, t + UPD_THREADS, t + 2 UPD_THREADS, ...
    // in that order
    constexpr int H = KM == 1 ? 4 : 2;
    for (int t0 = threadIdx.x; t0 < nd && any; t0 += H * UPD_THREADS) {
      long long dv[H];
      bool ok[H];
      double w2[H][NQ1];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int t = t0 + h * UPD_THREADS;
        ok[h] = t < nd;
        dv[h] = P.grp_elems[g0 + (ok[h] ? t : t0) / np];
      }
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int tt = ok[h] ? t0 + h * UPD_THREADS : t0;
        dv[h] = dv[h] * np + tt % np;
#pragma unroll
        for (int c = 0; c < NQ1; ++c) w2[h][c] = fused_r0 ? P.r0t[dv[h] * NQ1 + c] : 0.0;
      }
#pragma unroll
      for (int kk = 0; kk < KM; ++kk) {
        if (!act[kk]) continue;
        double xv[H], pv[H], qv[H], rv0[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const long long o = kk * (long long)P.ndof + dv[h];
          xv[h] = P.x[o];
          pv[h] = P.p[o];
          qv[h] = P.q[o];
          rv0[h] = P.r[o];
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
          if (!ok[h]) continue;
          const long long o = kk * (long long)P.ndof + dv[h];
          P.x[o] = fma(alpha[kk], pv[h], xv[h]);
          const double rv = fma(-alpha[kk], qv[h], rv0[h]);
          P.r[o] = rv;
          prr[kk] = fma(rv, rv, prr[kk]);
#pragma unroll
          for (int c = 0; c < NQ1; ++c) pr0[kk][c] = fma(w2[h][c], rv, pr0[kk][c]);
        }
      }
    }
  }
  for (int base = 0; base < nd && any && mode != MODE_ITER; base += UPD_THREADS) {
    const int t = base + threadIdx.x;
    if (t >= nd) break;
    const int e = P.grp_elems[g0 + t / np], a = t % np;
    const long long d = (long long)e * np + a;
    double w[NQ1] = {0.0, 0.0, 0.0};
    if (fused_r0) {
#pragma unroll
      for (int c = 0; c < NQ1; ++c) w[c] = P.r0t[d * NQ1 + c];
    }
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (!act[kk]) continue;
      const long long o = kk * (long long)P.ndof + d;
      double rv;
      if (mode == MODE_INIT || mode == MODE_INIT_X0) {
        const long long u = kk * (long long)P.ndof + (long long)P.perm[e] * np + a;
        rv = P.b_user[u];
        P.b[o] = rv;
        P.x[o] = mode == MODE_INIT ? 0.0 : P.x_user[u];
      } else if (mode == MODE_RESTART) {
        rv = P.b[o] - P.q[o];
      } else {
        P.x[o] = fma(alpha[kk], P.p[o], P.x[o]);
        rv = fma(-alpha[kk], P.q[o], P.r[o]);
      }
      P.r[o] = rv;
      prr[kk] = fma(rv, rv, prr[kk]);
#pragma unroll
      for (int c = 0; c < NQ1; ++c) pr0[kk][c] = fma(w[c], rv, pr0[kk][c]);
    }
  }
  // CTA sums of ||r||^2 and the three restriction components: each thread's values go through shared
  // memory and one warp per sum adds them (lane-strided, then a fixed shuffle tree), four sums at a time
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = fused_r0 ? 1 + NQ1 : 1;
    const int nsum = k * nv;
    for (int c0 = 0; c0 < nsum; c0 += 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = c0 + j;
        if (cc >= nsum) break;
        const int kk = cc / nv, c = cc % nv;
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < KM; ++q)
          if (q == kk) v = c == 0 ? prr[q] : pr0[q][c == 1 ? 0 : (c == 2 ? 1 : 2)];
        colbuf[j][threadIdx.x] = v;
      }
      __syncthreads();
      if (wid < 4 && c0 + wid < nsum) {
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < UPD_THREADS / 32; ++i) v += colbuf[wid][lane + 32 * i];
        v = warp_sum(v);
        if (lane == 0) {
          const int cc = c0 + wid, kk = cc / nv, c = cc % nv;
          if (c == 0) P.part_rr[(long long)g * k + kk] = v;
          else if (act[kk]) P.r0[(long long)kk * P.n0 + g * nq + c - 1] = v;
        }
      }
      __syncthreads();
    }
  }
  if (restrict_ && !fused_r0 && any) {
    // general coarse degree: one reduction per coarse basis function
    for (int c = 0; c < nq; ++c) {
      double v[KM];
#pragma unroll
      for (int kk = 0; kk < KM; ++kk) v[kk] = 0.0;
      for (int base = 0; base < nd; base += UPD_THREADS) {
        const int t = base + threadIdx.x;
        if (t >= nd) break;
        const int e = P.grp_elems[g0 + t / np], a = t % np;
        const double wv = P.r0t[((long long)e * np + a) * nq + c];
#pragma unroll
        for (int kk = 0; kk < KM; ++kk)
          if (act[kk]) v[kk] = fma(wv, P.r[kk * (long long)P.ndof + (long long)e * np + a], v[kk]);
      }
      block_sum_k<KM, UPD_NW>(v, k, red, tot);
      if (threadIdx.x < k && act[threadIdx.x]) P.r0[(long long)threadIdx.x * P.n0 + g * nq + c] = tot[threadIdx.x];
    }
  }
  if (!last_block(&P.counters[C_GRP], P.ngrp, &lastf)) return;
  if ((threadIdx.x >> 5) < k) {
    const int kk = threadIdx.x >> 5;
    if (bad[kk]) {
      if ((threadIdx.x & 31) == 0) {
        P.alpha[kk] = 0.0;
        P.status[kk] = DGASM_ENAN;
        P.done[kk] = 3;
        atomicSub(P.remaining, 1);
      }
      return;
    }
    if (!act[kk]) return;
    const double s = warp_sum_strided(P.part_rr + kk, P.ngrp, k);
    if ((threadIdx.x & 31) != 0) return;
    if (mode == MODE_RESTART) {
      // residual replacement: the recursion continues from r = b - A x; no iteration is counted
      const double rel = sqrt(s) / P.bnorm[kk];
      P.relres[kk] = rel;
      if (!finite_d(rel)) {
        P.status[kk] = DGASM_ENAN;
        P.done[kk] = 3;
        atomicSub(P.remaining, 1);
      } else if (P.fixed_iters == 0 && rel <= P.rtol) {
        P.done[kk] = 1;
        atomicSub(P.remaining, 1);
      }
      return;
    }
    if (mode == MODE_INIT || mode == MODE_INIT_X0) {
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
    P.alpha[kk] = alpha[kk];
    if (it <= P.maxit) P.alpha_hist[(long long)kk * P.maxit + it - 1] = alpha[kk];
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

// ---- coarse solve z_0 = A_0^{-1} r_0: one warp per row of the explicit inverse -------------------
template <int KM>
__global__ void __launch_bounds__(NTHREADS) k_coarse(BatchDev B) {
  __shared__ double wpart[NW][KMAX];
  const int pi = find_prob(B.prefix[K_COARSE], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_COARSE][pi];
  const int k = P.k, n0 = P.n0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  if (!any) return;
  double prod[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) prod[kk] = 0.0;
  // COARSE_ROWS_PER_WARP rows per warp, so that the GEMV of a 768-row A_0^{-1} takes 24 CTAs: the SMs the
  // local-solve clusters leave free, instead of SMs a cluster then has to wait for
  for (int i = 0; i < COARSE_ROWS_PER_WARP; ++i) {
    const int row = (item * COARSE_ROWS_PER_WARP + i) * NW + w;
    double acc[KM];
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) acc[kk] = 0.0;
    if (row < n0) {
      const double* Arow = P.A0inv + (long long)row * n0;
      for (int j = lane; j < n0; j += 32) {
        const double a = __ldg(Arow + j);
#pragma unroll
        for (int kk = 0; kk < KM; ++kk)
          if (act[kk]) acc[kk] = fma(a, P.r0[(long long)kk * n0 + j], acc[kk]);
      }
    }
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (kk >= k) break;
      const double v = warp_sum(acc[kk]);
      if (lane == 0 && row < n0 && act[kk]) {
        P.z0[(long long)kk * n0 + row] = v;
        prod[kk] += v * P.r0[(long long)kk * n0 + row];
      }
    }
  }
#pragma unroll
  for (int kk = 0; kk < KM; ++kk)
    if (kk < k && lane == 0) wpart[w][kk] = prod[kk];
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int ww = 0; ww < NW; ++ww) s += wpart[ww][threadIdx.x];
    P.part_c[(long long)item * k + threadIdx.x] = s;
  }
}

// ---- element-block local solves (subdomains = elements, Sec. 7's setting): z_e = inv(A_ee) r_e with
// the inverses precomputed at setup; one thread per (element, row), partial (r, z) per chunk item --------
template <int KM>
__global__ void __launch_bounds__(NTHREADS) k_bjac(BatchDev B) {
  __shared__ double red[NW * KMAX];
  __shared__ double tot[KMAX];
  const int pi = find_prob(B.prefix[K_BJAC], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int item = blockIdx.x - B.prefix[K_BJAC][pi];
  const int k = P.k, np = P.np;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  double prz[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) prz[kk] = 0.0;
  const int e_begin = item * P.epi;
  const int nel = min(P.epi, P.ne - e_begin);
  const int t = threadIdx.x;
  if (any && t < nel * np) {
    const int e = e_begin + t / np, a = t % np;
    const double* Dr = P.dinv + ((long long)e * np + a) * np;   // row a of inv(A_ee)
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (!act[kk]) continue;
      const double* rv = P.r + kk * (long long)P.ndof + (long long)e * np;
      double z = 0.0;
      for (int c = 0; c < np; ++c) z = fma(Dr[c], rv[c], z);
      P.z[kk * (long long)P.ndof + (long long)e * np + a] = z;
      prz[kk] = rv[a] * z;
    }
  }
  block_sum_k<KM>(prz, k, red, tot);
  if (threadIdx.x < k) P.part_rz[(long long)item * k + threadIdx.x] = P.done[threadIdx.x] == 0 ? tot[threadIdx.x] : 0.0;
}

// ---- p = z + R_0^T z_0 + beta p, beta = (r, z)_new / (r, z)_old ----------------------------------
// NN: the batch holds a non-nested coarse space (prolongation over (element, coarse cell) pairs); the
// instantiation without it keeps the agglomerate path lean
template <int KM, bool NN>
__global__ void __launch_bounds__(NTHREADS) k_pupdate(BatchDev B, int mode, int wslot) {
  __shared__ double beta_s[KMAX];
  __shared__ double gnew_s[KMAX];
  __shared__ __align__(16) ProbDev Ps;
  const int pi = find_prob(B.prefix[K_SPMV], B.nprob, blockIdx.x);
  const ProbDev& P = stage_prob(B.probs + pi, &Ps);
  const int item = blockIdx.x - B.prefix[K_SPMV][pi];
  const int k = P.k, np = P.np, nq = P.nq;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  // the element's data first (none of it depends on beta): z, the old p and, for coarse degree 1 with
  // agglomerates, z + R_0^T z_0 itself
  constexpr int NQ1 = 3;
  const int e_begin = item * P.epi;
  const int nel = min(P.epi, P.ne - e_begin);
  const int t = threadIdx.x;
  const bool mine = any && t < nel * np;
  const bool nn = NN && nq > 0 && P.r0t_ptr != nullptr;
  const bool fast = !nn && nq == NQ1;
  const int e = e_begin + (mine ? t / np : 0), a = mine ? t % np : 0;
  const long long d = (long long)e * np + a;
  double zv[KM], pv[KM];
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    zv[kk] = pv[kk] = 0.0;
    if (mine && kk < k) {
      const long long o = kk * (long long)P.ndof + d;
      zv[kk] = P.z[o];
      pv[kk] = P.p[o];
    }
  }
  if (mine && fast) {
    const int J = P.agg_int[e];
    double R[NQ1];
#pragma unroll
    for (int c = 0; c < NQ1; ++c) R[c] = P.r0t[d * NQ1 + c];
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (kk >= k) break;
      const double* z0 = P.z0 + (long long)kk * P.n0 + J * NQ1;
#pragma unroll
      for (int c = 0; c < NQ1; ++c) zv[kk] = fma(R[c], z0[c], zv[kk]);
    }
  }
  if ((threadIdx.x >> 5) < k) {
    const int kk = threadIdx.x >> 5;
    double g = 0.0;
    if (act[kk]) {
      g = warp_sum_strided(P.part_rz + kk, P.n_rz, k);
      if (nq > 0) g += warp_sum_strided(P.part_c + kk, P.n_coarse_items, k);
    }
    if ((threadIdx.x & 31) == 0) {
      gnew_s[kk] = g;
      beta_s[kk] = (mode == MODE_INIT || !act[kk]) ? 0.0 : g / (wslot ? P.gamma : P.gamma1)[kk];
    }
  }
  __syncthreads();
  if (mine) {
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) {
      if (!act[kk]) continue;
      const long long o = kk * (long long)P.ndof + d;
      double z = zv[kk];
      if (nn) {
        // non-nested: every coarse cell that meets the element, in ascending order
        for (int u = P.r0t_ptr[e]; u < P.r0t_ptr[e + 1]; ++u) {
          const double* R = P.r0t + ((long long)u * np + a) * nq;
          const double* z0 = P.z0 + (long long)kk * P.n0 + (long long)P.r0t_col[u] * nq;
          for (int c = 0; c < nq; ++c) z = fma(R[c], z0[c], z);
        }
      } else if (nq > 0 && !fast) {
        const double* R = P.r0t + d * nq;
        const double* z0 = P.z0 + (long long)kk * P.n0 + P.agg_int[e] * nq;
        for (int c = 0; c < nq; ++c) z = fma(R[c], z0[c], z);
      }
      P.p[o] = (mode == MODE_INIT) ? z : fma(beta_s[kk], pv[kk], z);
    }
  }
  // the new gamma goes to the other slot, so no CTA of this launch can read it in place of the old one: the
  // first item records it (every item formed the same sum) and no last-CTA step is needed
  if (item != 0) return;
  if (threadIdx.x < k) {
    const int kk = threadIdx.x;
    if (!act[kk]) return;
    const double g = gnew_s[kk];
    if (mode == MODE_ITER) {
      const int it = P.iters[kk];
      if (it >= 1 && it <= P.maxit) P.beta_hist[(long long)kk * P.maxit + it - 1] = beta_s[kk];
    }
    (wslot ? P.gamma1 : P.gamma)[kk] = g;
    if (!finite_d(g) || !(g > 0.0)) {
      P.status[kk] = DGASM_ENAN;
      P.done[kk] = 3;
      atomicSub(P.remaining, 1);
    }
  }
}

// ---- r_0 = R_0 r for a non-nested coarse space: one CTA per coarse cell J, over the pairs (element, J) in
// ascending order; per coarse basis function c a deterministic block sum of R[pair][a][c] r[e a]
template <int KM>
__global__ void __launch_bounds__(NTHREADS) k_restrict_nn(BatchDev B) {
  __shared__ double red[NW * KMAX];
  __shared__ double tot[KMAX];
  const int pi = find_prob(B.prefix[K_RNN], B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int J = blockIdx.x - B.prefix[K_RNN][pi];
  const int k = P.k, np = P.np, nq = P.nq;
  bool act[KM];
  bool any = false;
#pragma unroll
  for (int kk = 0; kk < KM; ++kk) {
    act[kk] = kk < k && P.done[kk] == 0;
    any |= act[kk];
  }
  if (!any) return;
  const int t0 = P.rT_ptr[J], n = (P.rT_ptr[J + 1] - t0) * np;
  for (int c = 0; c < nq; ++c) {
    double v[KM];
#pragma unroll
    for (int kk = 0; kk < KM; ++kk) v[kk] = 0.0;
    for (int i = threadIdx.x; i < n; i += NTHREADS) {
      const int t = P.rT_pair[t0 + i / np], a = i % np;
      const double w = P.r0t[((long long)t * np + a) * nq + c];
      const long long d = (long long)P.r0t_elem[t] * np + a;
#pragma unroll
      for (int kk = 0; kk < KM; ++kk)
        if (act[kk]) v[kk] = fma(w, P.r[kk * (long long)P.ndof + d], v[kk]);
    }
    block_sum_k<KM>(v, k, red, tot);
    if (threadIdx.x < k && act[threadIdx.x]) P.r0[(long long)threadIdx.x * P.n0 + (long long)J * nq + c] = tot[threadIdx.x];
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

}  // namespace

// one launch per polynomial degree present in the batch: slot K_SPMV_P + p - 1 holds the item prefix of
// the problems of degree p
template <int KM>
int launch_spmv_k(const BatchDev& B, int p, int total, int operand, cudaStream_t s) {
  const int slot = K_SPMV_P + p - 1;
  switch (p) {
    case 1: k_spmv<3, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 2: k_spmv<6, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 3: k_spmv<10, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 4: k_spmv<15, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 5: k_spmv<21, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 6: k_spmv<28, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    case 7: k_spmv<36, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
    default: k_spmv<45, KM><<<total, SPMV_THREADS, 0, s>>>(B, operand, slot); break;
  }
  return (int)cudaGetLastError();
}

// one launch per polynomial degree present in the batch: slot K_SPMV_P + p - 1 holds the item prefix of
// the problems of degree p; km = 1 when every problem of the batch has one right-hand side
int launch_spmv(const BatchDev& B, int p, int total, int operand, int km, void* st) {
  return km == 1 ? launch_spmv_k<1>(B, p, total, operand, (cudaStream_t)st)
                 : launch_spmv_k<KMAX>(B, p, total, operand, (cudaStream_t)st);
}

int launch_update(const BatchDev& B, int total, int mode, int km, int gslot, void* st) {
  if (km == 1) k_update<1><<<total, UPD_THREADS, 0, (cudaStream_t)st>>>(B, mode, gslot);
  else k_update<KMAX><<<total, UPD_THREADS, 0, (cudaStream_t)st>>>(B, mode, gslot);
  return (int)cudaGetLastError();
}

int launch_coarse(const BatchDev& B, int total, int km, void* st) {
  if (km == 1) k_coarse<1><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  else k_coarse<KMAX><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  return (int)cudaGetLastError();
}

int launch_bjac(const BatchDev& B, int total, int km, void* st) {
  if (km == 1) k_bjac<1><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  else k_bjac<KMAX><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  return (int)cudaGetLastError();
}

int launch_pupdate(const BatchDev& B, int total, int mode, int km, int nonnested, int wslot, void* st) {
  cudaStream_t s = (cudaStream_t)st;
  if (nonnested) {
    if (km == 1) k_pupdate<1, true><<<total, NTHREADS, 0, s>>>(B, mode, wslot);
    else k_pupdate<KMAX, true><<<total, NTHREADS, 0, s>>>(B, mode, wslot);
  } else {
    if (km == 1) k_pupdate<1, false><<<total, NTHREADS, 0, s>>>(B, mode, wslot);
    else k_pupdate<KMAX, false><<<total, NTHREADS, 0, s>>>(B, mode, wslot);
  }
  return (int)cudaGetLastError();
}

int launch_restrict_nn(const BatchDev& B, int total, int km, void* st) {
  if (km == 1) k_restrict_nn<1><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
  else k_restrict_nn<KMAX><<<total, NTHREADS, 0, (cudaStream_t)st>>>(B);
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
