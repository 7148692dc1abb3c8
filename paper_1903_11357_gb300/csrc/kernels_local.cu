// Local subdomain solves z_i = R_i^T A_i^{-1} R_i r (Sec. 3, local solvers) with the scaled tile-envelope
// Cholesky factor A~_i = L L^T (A~_i = D^{-1/2} A_i D^{-1/2}): forward substitution with L, backward
// substitution with L^T, diagonal tiles stored as inv(L_II) so both become tile GEMVs.
//
// One CTA per (subdomain, right-hand-side chunk).  Warp 8 is a producer: one elected lane streams the
// factor tiles from HBM into a ring of shared-memory slots with bulk asynchronous copies (cp.async.bulk,
// completion counted on an mbarrier per slot).  Both copies of the factor are stored in the order the
// sweeps consume them (forward: rows of column-major tiles; backward: columns of row-major tiles), so
// the producer streams two contiguous ranges, 32 KB per copy (the cost of a bulk copy is mostly per
// operation, not per byte).
// Warps 0..7 consume every tile together: warp w owns the four tile columns 4w..4w+3 (the matching four
// entries of every solution block), so each warp only ever needs its own entries of y and the FP64
// work of a tile row is split evenly over the SM's four sub-partitions.  Both sweeps are written as
// dot products: forward y_I = inv(L_II) (r_I - sum_J L_IJ y_J) over the column-major copy of row I,
// backward x_J = inv(L_JJ)^T (y_J - sum_{I>J} L_IJ^T x_I) over the row-major copy of column J.  Each
// tile row costs two barriers: one after the off-diagonal partial sums, one after the diagonal product.
// Every mbarrier wait is bounded; on timeout the kernel records an error in the batch error word and
// stops waiting.
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
constexpr int SR = 4;                  // tile rows per super-row (matches the plan)
constexpr int NCW = 8;                 // consumer warps
constexpr int NCT = NCW * 32;          // consumer threads
constexpr int NTH = NCT + 32;          // + producer warp
constexpr long long WAIT_CYCLES = 4000000000LL;  // about two seconds at the GB300 clock

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and raises the abort flag and the error word) on timeout
__device__ bool mbar_wait(unsigned long long* bar, unsigned parity, volatile int* abort_flag, int* err) {
  if (*abort_flag) return false;
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NCT) : "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int find_prob(const int* __restrict__ prefix, int nprob, int item) {
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename C> __device__ __forceinline__ C shfl_xor_c(C v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <typename C> __device__ __forceinline__ C shfl_c(C v, int src) { return __shfl_sync(0xffffffffu, v, src); }

template <typename S, typename C> __device__ __forceinline__ C cvt(S v) { return (C)v; }
template <> __device__ __forceinline__ float cvt<__nv_bfloat16, float>(__nv_bfloat16 v) { return __bfloat162float(v); }

// acc[j][u] += tile[(c0+u)*T + lane] * v[j][c0+u] for the four tile lines u of this warp's chunk: four
// independent accumulation chains, so the four FMAs of a tile are in flight together
template <typename S, typename C, int KCT>
__device__ __forceinline__ void gemv4(const S* __restrict__ tile, const C* __restrict__ v, int vstride, C (*acc)[4]) {
  C t[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) t[u] = cvt<S, C>(tile[u * T]);
#pragma unroll
  for (int j = 0; j < KCT; ++j)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[j][u] = fma(t[u], v[j * vstride + u], acc[j][u]);
}

template <typename S, typename C, int KCT>
__global__ void __launch_bounds__(NTH) k_local(BatchDev B, int slot, int ring_off, int nstage, int ch) {
  constexpr int NCH = KCT == 1 ? 2 : 1;   // independent accumulation chains per coupling accumulator
  constexpr int DCH = KCT == 1 ? 2 : 1;   // and per diagonal-block accumulator
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[NCW + 1][KCT];
  __shared__ int abort_flag;
  const int* prefix = B.prefix[slot];
  const int pi = find_prob(prefix, B.nprob, blockIdx.x);
  const ProbDev& P = B.probs[pi];
  const int li = blockIdx.x - prefix[pi];
  const int s = li / P.n_rhs_chunks, kch = li % P.n_rhs_chunks;
  const int k0 = kch * KCT;
  const int kc = min(KCT, P.k - k0);
  bool act[KCT];
  bool any = false;
#pragma unroll
  for (int j = 0; j < KCT; ++j) {
    act[j] = j < kc && P.done[k0 + j] == 0;
    any |= act[j];
  }
  if (!any) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int e0 = P.sub_e0[s];
  const int n = (P.sub_e0[s + 1] - e0) * P.np;
  const long long d0 = (long long)e0 * P.np;
  const int nbt = (n + T - 1) / T, npad = nbt * T;
  const int nsr = (nbt + SR - 1) / SR;
  const int tr0 = P.sub_trow[s];
  const long long f0 = P.stream_ptr[s];
  const long long nstream = P.stream_ptr[s + 1] - f0;
  C* y = reinterpret_cast<C*>(smem);                  // [KCT][npad]
  C* part = y + KCT * npad;                            // [NCW][SR][KCT][T]
  C* dpart = part + NCW * SR * KCT * T;                // [NCW][SR][KCT][T]
  C* tvs = dpart + NCW * SR * KCT * T;                 // [NCW][SR * 4][KCT]
  int* Fs = reinterpret_cast<int*>(tvs + NCW * SR * 4 * KCT);   // tile-row F values
  S* ring = reinterpret_cast<S*>(smem + ring_off);     // [nstage][ch][TT]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(ring + (size_t)nstage * ch * TT);
  unsigned long long* empty = full + nstage;
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < nstage; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (w == NCW) {
    // ---- producer: the forward stream, then the backward stream, nstream tiles each, in chunks of ch
    // consecutive tiles (one bulk copy per chunk)
    if (lane == 0) {
      const S* Lc = reinterpret_cast<const S*>(P.Lc);
      const S* Lr = reinterpret_cast<const S*>(P.Lr);
      int sl = 0;
      unsigned round = 0;   // how many times the ring has wrapped
      bool ok = true;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        const S* base = (pass == 0 ? Lc : Lr) + f0 * TT;
        for (long long t = 0; t < nstream && ok; t += ch) {
          const int len = (int)min((long long)ch, nstream - t);
          if (round > 0 && !mbar_wait(empty + sl, (round - 1) & 1, &abort_flag, B.err)) { ok = false; break; }
          const unsigned bytes = (unsigned)(len * TT * sizeof(S));
          mbar_expect_tx(full + sl, bytes);
          bulk_g2s(ring + (size_t)sl * ch * TT, base + t * TT, bytes, full + sl);
          if (++sl == nstage) { sl = 0; ++round; }
        }
      }
    }
  } else {
    // ---- consumers: warp w owns tile columns (forward) / tile rows (backward) c0 .. c0+3 of every tile
    const int c0 = 4 * w;
    for (int i = tid; i < nbt; i += NCT) Fs[i] = P.trow_F[tr0 + i];
    for (int idx = tid; idx < KCT * npad; idx += NCT) {
      const int j = idx / npad, i = idx - j * npad;
      C v = (C)0;
      if (i < n && act[j]) v = (C)(P.scale[d0 + i] * P.r[(long long)(k0 + j) * P.ndof + d0 + i]);
      y[idx] = v;
    }
    consumer_sync();
    // stream cursor: ring slot, its phase parity, position in the chunk, chunk length
    int cs = 0, cpos = 0;
    unsigned cph = 0;
    long long taken = 0;
    int clen = (int)min((long long)ch, nstream);
    auto acquire = [&]() -> const S* {
      if (cpos == 0 && !mbar_wait(full + cs, cph, &abort_flag, B.err)) return nullptr;
      return ring + ((size_t)cs * ch + cpos) * TT;
    };
    auto release = [&]() {
      ++taken;
      if (++cpos == clen) {
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + cs);
        cpos = 0;
        if (++cs == nstage) { cs = 0; cph ^= 1u; }
        if (taken == nstream) taken = 0;   // the backward stream starts with a fresh chunk
        clen = (int)min((long long)ch, nstream - taken);
      }
    };
    // Lane l reduces block entry e = l >> 1 (tile row e >> 2 of the super-row, line c0 + (e & 3)) over
    // four warps' partials (half l & 1), then across the two halves: a fixed order on every warp.
    const int re = lane >> 1, rii = re >> 2, ru = re & 3, rh = lane & 1;
    auto reduce_entry = [&](const C* buf, int j) -> C {
      C v = buf[(((4 * rh) * SR + rii) * KCT + j) * T + c0 + ru];
#pragma unroll
      for (int ww = 1; ww < 4; ++ww) v += buf[(((4 * rh + ww) * SR + rii) * KCT + j) * T + c0 + ru];
      return v + shfl_xor_c(v, 1);
    };
    C* tw = tvs + w * SR * 4 * KCT;   // this warp's right-hand sides of the diagonal block product
    // one super-row (tile rows I0 .. I0+ntr-1): acc holds the coupling sums; t = y_S - sum over warps,
    // y_S = X t (forward) or X^T t (backward) with X the inverse of the diagonal block
    auto finish_super = [&](int I0, int ntr, C (*acc)[KCT][NCH], bool fwd) {
#pragma unroll
      for (int ii = 0; ii < SR; ++ii)
#pragma unroll
        for (int j = 0; j < KCT; ++j) {
          C v = (C)0;
#pragma unroll
          for (int h = 0; h < NCH; ++h) v += acc[ii][j][h];
          part[((w * SR + ii) * KCT + j) * T + lane] = ii < ntr ? v : (C)0;
        }
      consumer_sync();
#pragma unroll
      for (int j = 0; j < KCT; ++j) {
        const C tot = reduce_entry(part, j);
        const C t = rii < ntr ? y[j * npad + (I0 + rii) * T + c0 + ru] - tot : (C)0;
        if (rh == 0) tw[re * KCT + j] = t;
      }
      __syncwarp();
      C o[SR][KCT][DCH];
#pragma unroll
      for (int ii = 0; ii < SR; ++ii)
#pragma unroll
        for (int j = 0; j < KCT; ++j)
#pragma unroll
          for (int h = 0; h < DCH; ++h) o[ii][j][h] = (C)0;
#pragma unroll
      for (int i = 0; i < SR; ++i) {
        if (i >= ntr) break;
#pragma unroll
        for (int jj = 0; jj <= i; ++jj) {
          const S* tile = acquire();
          if (tile) {
            const S* tl = tile + c0 * T + lane;
            C tv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) tv[u] = cvt<S, C>(tl[u * T]);
            // forward: X_(i,jj) times block jj into output block i; backward: X_(i,jj)^T times block i
            // into output block jj
            const int src = fwd ? jj : i;
#pragma unroll
            for (int j = 0; j < KCT; ++j) {
              const C* vv = tw + (src * 4) * KCT + j;
              C& x = fwd ? o[i][j][jj % DCH] : o[jj][j][i % DCH];
              x = fma(tv[0], vv[0], x);
              x = fma(tv[1], vv[KCT], x);
              x = fma(tv[2], vv[2 * KCT], x);
              x = fma(tv[3], vv[3 * KCT], x);
            }
          }
          release();
        }
      }
#pragma unroll
      for (int ii = 0; ii < SR; ++ii)
#pragma unroll
        for (int j = 0; j < KCT; ++j) {
          C v = o[ii][j][0];
#pragma unroll
          for (int h = 1; h < DCH; ++h) v += o[ii][j][h];
          dpart[((w * SR + ii) * KCT + j) * T + lane] = v;
        }
      consumer_sync();
#pragma unroll
      for (int j = 0; j < KCT; ++j) {
        const C tot = reduce_entry(dpart, j);
        if (rh == 0 && rii < ntr) y[j * npad + (I0 + rii) * T + c0 + ru] = tot;
      }
      __syncwarp();
    };
    C acc[SR][KCT][NCH];
    auto zero_acc = [&]() {
#pragma unroll
      for (int ii = 0; ii < SR; ++ii)
#pragma unroll
        for (int j = 0; j < KCT; ++j)
#pragma unroll
          for (int h = 0; h < NCH; ++h) acc[ii][j][h] = (C)0;
    };
    // one coupling tile: a[j][0] += sum_u tile line (c0+u) * v[j][c0+u], then the chains rotate so the
    // next tile accumulates into the next chain (static register indices throughout)
    auto couple = [&](const S* tile, const C* v, C (&a)[KCT][NCH]) {
      const S* tl = tile + c0 * T + lane;
      C tv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) tv[u] = cvt<S, C>(tl[u * T]);
#pragma unroll
      for (int j = 0; j < KCT; ++j) {
        const C* vj = v + j * npad;
        C x = a[j][0];
        x = fma(tv[0], vj[0], x);
        x = fma(tv[1], vj[1], x);
        x = fma(tv[2], vj[2], x);
        x = fma(tv[3], vj[3], x);
#pragma unroll
        for (int h = 0; h + 1 < NCH; ++h) a[j][h] = a[j][h + 1];
        a[j][NCH - 1] = x;
      }
    };
    // forward substitution, super-row by super-row
    for (int q = 0; q < nsr; ++q) {
      const int I0 = q * SR, ntr = min(SR, nbt - I0);
      zero_acc();
#pragma unroll
      for (int ii = 0; ii < SR; ++ii) {
        if (ii >= ntr) break;
        for (int J = Fs[I0 + ii]; J < I0; ++J) {
          const S* tile = acquire();
          if (tile) couple(tile, y + J * T + c0, acc[ii]);
          release();
        }
      }
      finish_super(I0, ntr, acc, true);
    }
    // backward substitution with L^T, super-row by super-row from the last: the tile rows I after the
    // super-row that couple to its columns, each with its tiles (I, J), J ascending
    for (int q = nsr - 1; q >= 0; --q) {
      const int I0 = q * SR, ntr = min(SR, nbt - I0), I1 = I0 + ntr;
      const int Ilast = P.sr_ilast[P.sub_sr[s] + q];
      zero_acc();
      for (int I = I1; I <= Ilast; ++I) {
        const int FI = Fs[I];
        if (FI > I1 - 1) continue;
        const int jstart = FI > I0 ? FI - I0 : 0;
#pragma unroll
        for (int jj = 0; jj < SR; ++jj) {
          if (jj < jstart || jj >= ntr) continue;
          const S* tile = acquire();
          if (tile) couple(tile, y + I * T + c0, acc[jj]);
          release();
        }
      }
      finish_super(I0, ntr, acc, false);
    }
  }
  __syncthreads();
  // z_i = D^{-1/2} y, partial (r, z) for this subdomain (producer warp contributes zeros)
  double prz[KCT];
#pragma unroll
  for (int j = 0; j < KCT; ++j) prz[j] = 0.0;
  if (w < NCW) {
    for (int i = tid; i < n; i += NCT) {
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
  }
#pragma unroll
  for (int j = 0; j < KCT; ++j) {
    const double v = warp_sum(prz[j]);
    if (lane == 0) red[w][j] = v;
  }
  __syncthreads();
  if (tid < kc) {
    double sum = 0.0;
    for (int ww = 0; ww <= NCW; ++ww) sum += red[ww][tid];
    P.part_rz[(long long)s * P.k + k0 + tid] = act[tid] ? sum : 0.0;
  }
}

// shared memory: y, partial sums and F values, then a ring of nstage slots of ch tiles (32 KB per slot)
template <typename S, typename C>
int smem_layout(int ndof_max, int kct, int* ring_off, int* nstage, int* ch, int* total) {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int npad = ((ndof_max + T - 1) / T) * T;
  const int head = (int)sizeof(C) * (kct * npad + 2 * NCW * SR * kct * T + NCW * SR * 4 * kct) + 4 * (npad / T + 4);
  const int off = (head + 127) & ~127;
  const int budget = optin - 2048 - off;   // static shared memory and slack
  int c = (32 * 1024) / (int)(TT * sizeof(S));
  int ns = 0;
  for (; c >= 1; c /= 2) {
    ns = budget / (c * (int)(TT * sizeof(S)) + 16);
    if (ns >= 3) break;
  }
  if (c < 1) c = 1;
  if (ns > 32) ns = 32;
  if (ns < 2) return -1;
  *ring_off = off;
  *nstage = ns;
  *ch = c;
  *total = off + ns * c * (int)(TT * sizeof(S)) + ns * 16;
  return 0;
}

template <typename K>
int ensure_smem(K fn, int smem) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({(const void*)fn, dev})) return 0;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
  if (e != cudaSuccess) return (int)e;
  done.insert({(const void*)fn, dev});
  (void)smem;
  return 0;
}

template <typename S, typename C>
int launch_local_t(const BatchDev& B, int slot, int kcl, int total, int ndof_max, cudaStream_t st) {
  int ring_off, nstage, ch, smem;
  if (kcl == 0) {
    if (smem_layout<S, C>(ndof_max, 1, &ring_off, &nstage, &ch, &smem)) return (int)cudaErrorInvalidValue;
    auto fn = k_local<S, C, 1>;
    if (int e = ensure_smem(fn, smem)) return e;
    fn<<<total, NTH, smem, st>>>(B, slot, ring_off, nstage, ch);
  } else {
    if (smem_layout<S, C>(ndof_max, KC, &ring_off, &nstage, &ch, &smem)) return (int)cudaErrorInvalidValue;
    auto fn = k_local<S, C, KC>;
    if (int e = ensure_smem(fn, smem)) return e;
    fn<<<total, NTH, smem, st>>>(B, slot, ring_off, nstage, ch);
  }
  return (int)cudaGetLastError();
}

}  // namespace

// the launch is sized inside launch_local from ndof_max; this returns ndof_max itself so that callers
// can keep one number per launch slot
int local_smem_bytes(int /*prec*/, int ndof_max, int /*kc*/) { return ndof_max; }

// slot = K_NKINDS + 2 * prec + (kc > 1); `param` is the largest subdomain dof count of the launch
int launch_local(const BatchDev& B, int slot, int total, int param, void* stream) {
  const int prec = (slot - K_NKINDS) / 2, kcl = (slot - K_NKINDS) % 2;
  cudaStream_t s = (cudaStream_t)stream;
  switch (prec) {
    case DGASM_FP64: return launch_local_t<double, double>(B, slot, kcl, total, param, s);
    case DGASM_FP32:
    case DGASM_TF32: return launch_local_t<float, float>(B, slot, kcl, total, param, s);
    default: return launch_local_t<__nv_bfloat16, float>(B, slot, kcl, total, param, s);
  }
}

}  // namespace dgasm
