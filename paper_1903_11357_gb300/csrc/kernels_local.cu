// Local subdomain solves z_i = R_i^T A_i^{-1} R_i r (Sec. 3, local solvers) with the scaled tile-envelope
// Cholesky factor A~_i = L L^T (A~_i = D^{-1/2} A_i D^{-1/2}): forward substitution with L, backward
// substitution with L^T.
//
// The rows are processed in super-rows of SR = 8 tile rows (256 rows; the size is a per-precision choice
// of the plan and of this kernel).  The setup stores, in the order the
// sweeps consume them, the factor tiles that couple different super-rows and the explicit inverse X_q of
// each super-row's lower-triangular diagonal block, so a super-row costs tile GEMVs, one reduction, a
// product with X_q (or X_q^T) and one more reduction:
//   forward   y_q = X_q (r_q - sum_{J before q} L_qJ y_J)
//   backward  x_q = X_q^T (y_q - sum_{I after q} L_Iq^T x_I).
// The streams are cut into runs: consecutive tiles that add into one output block with consecutive
// operand blocks (the plan gives each coupling run's first operand block and length), so a warp keeps
// one pair of accumulators per run and walks the tiles of a run with plain pointer steps.
//
// A cluster of two CTAs (two SMs) works on one (subdomain, right-hand-side chunk).  Each stream is stored
// as two arrays of half tiles, lines 0-15 and lines 16-31 of every 32 x 32 tile (a line is a column of the
// column-major forward tiles, a row of the row-major backward tiles); CTA rank r streams half r.  In each
// CTA warp 8 is a producer: one elected lane copies runs of half tiles from HBM into a ring of shared-memory
// slots with bulk asynchronous copies (cp.async.bulk, 32 KB per slot, completion counted on an mbarrier per
// slot).  Warps 0..7 consume: warp w of rank r owns lines 16r + 2w and 16r + 2w + 1 of every tile (stored
// interleaved, one vector load per tile; lane = the other tile index), so the FP64 work is spread evenly
// over both SMs' sub-partitions and a warp only ever needs its own entries of each solution block.
//
// FP32 and BF16 launches have a second form for launches with more pairs than the GPU holds at once: one CTA
// of 16 consumer warps per item, whose slots carry the same runs of both halves (the half-0 tiles, then the
// half-1 tiles) and whose warps 8..15 take the lines of the pair's rank 1.  A block entry is then (sum of warps
// 0..7) + (sum of warps 8..15), the pair's (rank 0 sum) + (rank 1 sum), so both forms give the same bits.
//
// Reductions.  The warps' partial sums of a block entry are added in a fixed order inside each CTA; the
// entries the peer owns are sent to it with st.async, which counts its bytes on the peer's exchange
// mbarrier, and each entry's total is (rank 0 sum) + (rank 1 sum).  The result therefore does not depend
// on timing, on the batch a subdomain is launched in or on which SMs run it.  Every wait is bounded; on
// timeout the kernel records an error in the batch error word, stops waiting, and before returning waits
// (again bounded) for its own copies still in flight.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <set>
#include <utility>

#include "common.h"
#include "engine.h"

namespace dgasm {

namespace {

constexpr int T = 32;
constexpr int TT = T * T;
constexpr int HT = TT / 2;             // half tile: 16 lines of 32
constexpr int NCW_PAIR = 8;            // consumer warps of each CTA of a pair (a CTA alone has twice as many)
constexpr int LW = 2;                  // tile lines per consumer warp
constexpr long long WAIT_CYCLES = 4000000000LL;  // about two seconds at the GB300 clock

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and raises the abort flag and the error word) after `limit` cycles
__device__ bool mbar_wait(unsigned long long* bar, unsigned parity, volatile int* abort_flag, int* err,
                          long long limit = WAIT_CYCLES) {
  if (*abort_flag) return false;
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

// bounded wait that ignores the abort flag (used to let transfers in flight land before returning)
__device__ void mbar_drain(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > WAIT_CYCLES) return;
}

// wait for the peer's partial sums.  The peer sends them whatever happens to its own waits, so this
// wait ignores the abort flag and has a longer limit than the ring waits; if it still gives up, the
// exchange is marked dead and no later reduction arms or waits on the exchange barriers.
__device__ void xbar_wait(unsigned long long* bar, unsigned parity, volatile int* abort_flag, volatile int* xdead,
                          int* err) {
  if (*xdead) return;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*xdead) return;
    if (clock64() - t0 > 3 * WAIT_CYCLES) {
      *xdead = 1;
      *abort_flag = 1;
      atomicExch(err, 1);
      return;
    }
  }
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

// shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ unsigned mapa(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// store into the peer's shared memory; the store's bytes complete a transaction on the peer's barrier
__device__ __forceinline__ void st_async(unsigned addr, double v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void st_async(unsigned addr, float v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void st_cluster(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// all threads of both CTAs; orders every shared-memory access before it (release / acquire)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// named barrier 1 over the n consumer threads (the producer warp never joins it)
template <int N>
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }

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

// the two entries of a warp's line pair, stored next to each other in the solve streams
template <typename S> struct Pair;
template <> struct Pair<double> { using V = double2; };
template <> struct Pair<float> { using V = float2; };
template <> struct Pair<__nv_bfloat16> { using V = __nv_bfloat162; };

template <typename C>
__device__ __forceinline__ void ld_pair(const double2* p, C& a, C& b) {
  const double2 v = *p;
  a = (C)v.x;
  b = (C)v.y;
}
template <typename C>
__device__ __forceinline__ void ld_pair(const float2* p, C& a, C& b) {
  const float2 v = *p;
  a = (C)v.x;
  b = (C)v.y;
}
template <typename C>
__device__ __forceinline__ void ld_pair(const __nv_bfloat162* p, C& a, C& b) {
  const float2 v = __bfloat1622float2(*p);
  a = (C)v.x;
  b = (C)v.y;
}
// an operand pair (two consecutive entries, 2-element aligned)
__device__ __forceinline__ double2 ld_pair2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ float2 ld_pair2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// tiles per ring slot: 32 KB of half tiles (the cost of a bulk copy is mostly per operation)
template <typename S> __host__ __device__ constexpr int slot_tiles() { return (32 * 1024) / (int)(HT * sizeof(S)); }

// PAIR: a cluster of two CTAs per item, CTA rank h holding lines 16h .. 16h + 15 of every tile.  Otherwise one
// CTA of 16 consumer warps per item does the work of both: its warp 8h + w takes the lines of warp w of rank h,
// its ring slots hold the same tiles of both halves, and it adds the two halves' partial sums in the pair's
// order, so both forms give the same bits (the engine takes the one CTA form when a launch's pairs would not all
// be resident at once: it needs no exchange and half the SMs per item).
template <typename S, typename C, int KCT, bool PAIR>
__device__ __forceinline__ void local_body(const BatchDev& B, int slot, int ring_off, int nstage) {
  using VS = typename Pair<S>::V;
  constexpr int NCW = PAIR ? NCW_PAIR : 2 * NCW_PAIR;   // consumer warps
  constexpr int NCT = NCW * 32;
  constexpr int SR = 8;                   // tile rows per super-row: super_row() of every precision
  constexpr int YL = PAIR ? 16 : 32;      // lines of every tile this CTA holds (its half, or all)
  constexpr int NX = SR * 16 * KCT;       // entries exchanged per reduction (each direction, PAIR)
  constexpr int NE = SR * KCT * T;        // entries summed per reduction in each CTA
  constexpr bool TWO = sizeof(C) == 4;    // two accumulation chains (FP32: cover the FMA latency)
  constexpr int CH = slot_tiles<S>();     // tiles per ring slot and half
  constexpr int SLOT = (PAIR ? 1 : 2) * CH * HT;   // elements of a ring slot
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[NCW + 1][KCT];
  __shared__ double peer_rz[KCT];
  __shared__ int abort_flag, xdead;
  __shared__ __align__(8) unsigned long long xbar[2];   // the peer's partial sums have landed
  const unsigned rank = PAIR ? cluster_rank() : 0u, peer = rank ^ 1u;
  const int* prefix = B.prefix[slot];
  const int item = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int pi = find_prob(prefix, B.nprob, item);
  const ProbDev& P = B.probs[pi];
  const int li = item - prefix[pi];
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
  if (!any) return;   // both CTAs of a pair read the same flags and leave together
  if (P.sr != SR) {   // the plan was built for another super-row size: refuse
    if (threadIdx.x == 0) atomicExch(B.err, 2);
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int e0 = P.sub_e0[s];
  const int n = (P.sub_e0[s + 1] - e0) * P.np;
  const long long d0 = (long long)e0 * P.np;
  const int nbt = (n + T - 1) / T, npadh = nbt * YL;
  const int nsr = (nbt + SR - 1) / SR;
  const int sr0 = P.sub_sr[s];
  const long long ff0 = P.fwd_ptr[s], bb0 = P.bwd_ptr[s];
  C* y = reinterpret_cast<C*>(smem);                  // [KCT][nbt][YL]: the held lines of every block
  // per-warp partial sums [NCW][SR][KCT][T], one buffer for both reductions of a super-row: a reduction
  // reads it only before its internal barrier, which every warp passes before writing the next partials
  C* part = y + KCT * npadh;
  C* dpart = part;
  C* tvs = part + NCW * SR * KCT * T;                  // [NCW][SR][KCT][LW]
  C* xbuf = tvs + NCW * SR * KCT * LW;                 // [2][SR][KCT][16]: the peer's sums of own entries (PAIR)
  C* cpart = xbuf + (PAIR ? 2 * NX : 0);               // [SR][KCT][YL]: the sums of the held entries
  int* runs_s = reinterpret_cast<int*>(cpart + (PAIR ? NX : NE));   // [2][nsr][SR][2]: the coupling runs
  S* ring = reinterpret_cast<S*>(smem + ring_off);     // [nstage][SLOT]: per slot CH tiles of each held half
  unsigned long long* full = reinterpret_cast<unsigned long long*>(ring + (size_t)nstage * SLOT);
  unsigned long long* empty = full + nstage;
  if (tid == 0) {
    abort_flag = 0;
    xdead = 0;
    for (int i = 0; i < nstage; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, NCW);
    }
    mbar_init(&xbar[0], 1);
    mbar_init(&xbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if constexpr (PAIR) cluster_sync();   // the peer's barriers exist before any store reaches them

  if (w == NCW) {
    // ---- producer: half `rank` (PAIR) or both halves of the subdomain's forward stream, then of its backward
    // stream.  Each super-row's coupling section and inverse-block section is copied in runs of up to CH
    // tiles (one bulk copy per run and half), every section starting in a fresh slot.
    if (lane == 0) {
      int sl = 0;
      unsigned round = 0;   // how many times the ring has wrapped
      long long issued = 0;
      bool ok = true;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        const long long tot = pass == 0 ? P.fwd_total : P.bwd_total;
        const S* base = pass == 0 ? reinterpret_cast<const S*>(P.Lc) + (rank * P.fwd_total + ff0) * HT
                                  : reinterpret_cast<const S*>(P.Lr) + (rank * P.bwd_total + bb0) * HT;
        const int* rt = (pass == 0 ? P.fwd_run : P.bwd_run) + (size_t)sr0 * SR * 2;
        long long pos = 0;
        for (int qi = 0; qi < nsr && ok; ++qi) {
          const int q = pass == 0 ? qi : nsr - 1 - qi;
          const int ntr = min(SR, nbt - q * SR);
          int lc = 0;
          for (int o = 0; o < ntr; ++o) lc += rt[(q * SR + o) * 2 + 1];
          for (int sec = 0; sec < 2 && ok; ++sec) {
            const int len_sec = sec == 0 ? lc : ntr * (ntr + 1) / 2;
            for (int t = 0; t < len_sec; t += CH) {
              const int len = min(CH, len_sec - t);
              if (round > 0 && !mbar_wait(empty + sl, (round - 1) & 1, &abort_flag, B.err)) { ok = false; break; }
              const unsigned bytes = (unsigned)(len * HT * sizeof(S));
              mbar_expect_tx(full + sl, PAIR ? bytes : 2 * bytes);
              bulk_g2s(ring + (size_t)sl * SLOT, base + (pos + t) * HT, bytes, full + sl);
              if constexpr (!PAIR)   // the same tiles' second half, after the first half's CH tiles
                bulk_g2s(ring + (size_t)sl * SLOT + (size_t)CH * HT, base + (tot + pos + t) * HT, bytes, full + sl);
              ++issued;
              if (++sl == nstage) { sl = 0; ++round; }
            }
            pos += len_sec;
          }
        }
      }
      // let every copy issued land (they all have when the consumers finished normally)
      for (int i = 0; i < nstage && i < issued; ++i) {
        const long long fills = (issued - i + nstage - 1) / nstage;
        mbar_drain(full + i, (unsigned)((fills - 1) & 1));
      }
    }
  } else {
    // ---- consumers: warp w owns the lines l0, l0 + 1 of every tile
    const int lw = LW * w;               // line within this CTA's half
    const int l0 = 16 * (int)rank + lw;  // line within the tile
    for (int t = tid; t < nsr * SR * 2; t += NCT) {
      runs_s[t] = P.fwd_run[(size_t)sr0 * SR * 2 + t];
      runs_s[nsr * SR * 2 + t] = P.bwd_run[(size_t)sr0 * SR * 2 + t];
    }
    for (int idx = tid; idx < KCT * npadh; idx += NCT) {
      const int j = idx / npadh, m = idx - j * npadh;
      const int i = (m / YL) * T + 16 * (int)rank + (m % YL);
      C v = (C)0;
      if (i < n && act[j]) v = (C)(P.scale[d0 + i] * P.r[(long long)(k0 + j) * P.ndof + d0 + i]);
      y[idx] = v;
    }
    consumer_sync<NCT>();
    // Stream cursor: ring slot cs (phase parity cph), this warp's line pair of the current tile in it
    // (cur), tiles left in the slot's run of tiles (left_in), tiles of the current stream still to come
    // after this slot (rest).  A slot is waited for when the cursor enters it and handed back to the
    // producer when the cursor leaves it.
    int cs = 0, left_in = 0, rest = 0;
    unsigned cph = 0;
    const VS* cur = nullptr;
    // this warp's pair within a slot, in pairs: its half's region (one CTA), then its line pair in the half
    const size_t wofs = (PAIR ? 0 : (size_t)(w >> 3) * CH * (HT / 2)) + (size_t)(w & 7) * T + lane;
    auto enter_slot = [&]() {
      left_in = min(CH, rest);
      rest -= left_in;
      cur = reinterpret_cast<const VS*>(ring + (size_t)cs * SLOT) + wofs;
      if (left_in > 0 && !mbar_try(full + cs, cph)) mbar_wait(full + cs, cph, &abort_flag, B.err);
    };
    auto leave_slot = [&]() {
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + cs);
      if (++cs == nstage) { cs = 0; cph ^= 1u; }
      enter_slot();
    };
    auto start_section = [&](int len) {
      rest = len;
      enter_slot();
    };
    // One run: cnt consecutive stream tiles into one output block of this warp's lanes,
    //   res[j] = sum_k (line pair of tile k) . (operand pair k of right-hand side j),
    // operand pair k of rhs j at v + k * vstride + j * jstride.  FP32 tiles alternate between two
    // accumulators (restarting in each slot, so the grouping depends only on the plan).  After a
    // timed-out wait the data are stale; the error word is set and the result is discarded.
    auto run = [&](int cnt, const C* v, int vstride, int jstride, C (&res)[KCT]) {
      C a0[KCT], a1[KCT];
#pragma unroll
      for (int j = 0; j < KCT; ++j) a0[j] = a1[j] = (C)0;
      while (cnt > 0) {
        const int m = min(cnt, left_in);
        int t = 0;
        for (; t + 1 < m; t += 2) {
          C x0, x1, z0, z1;
          ld_pair(cur + t * (HT / 2), x0, x1);
          ld_pair(cur + (t + 1) * (HT / 2), z0, z1);
#pragma unroll
          for (int j = 0; j < KCT; ++j) {
            const auto o0 = ld_pair2(v + t * vstride + j * jstride);
            const auto o1 = ld_pair2(v + (t + 1) * vstride + j * jstride);
            C& b = TWO ? a1[j] : a0[j];
            a0[j] = fma(x0, o0.x, a0[j]);
            b = fma(z0, o1.x, b);
            a0[j] = fma(x1, o0.y, a0[j]);
            b = fma(z1, o1.y, b);
          }
        }
        if (t < m) {
          C x0, x1;
          ld_pair(cur + t * (HT / 2), x0, x1);
#pragma unroll
          for (int j = 0; j < KCT; ++j) {
            const auto o0 = ld_pair2(v + t * vstride + j * jstride);
            a0[j] = fma(x0, o0.x, a0[j]);
            a0[j] = fma(x1, o0.y, a0[j]);
          }
        }
        cur += m * (HT / 2);
        v += m * vstride;
        cnt -= m;
        left_in -= m;
        if (left_in == 0) leave_slot();
      }
#pragma unroll
      for (int j = 0; j < KCT; ++j) res[j] = TWO ? a0[j] + a1[j] : a0[j];
    };
    // Reduction number xcount of the partials in buf (written, followed by consumer_sync).  Thread t sums
    // the eight warps' partials of entries t, t + 256, ... in warp order; the sums of the peer's entries go
    // to the peer (st.async), those of own entries to cpart.  After a consumer_sync and the peer's signal
    // each warp forms (rank 0 sum) + (rank 1 sum) of its own entries and hands it to use(ii, j, u, total).
    // Reductions alternate between two exchange buffers and barriers; the peer cannot send reduction m + 2
    // before it has received reduction m + 1, which this CTA sends only after every warp has read the
    // buffer of reduction m, and thread 0 arms a barrier for reduction m + 2 only after waiting on m.
    unsigned xcount = 0;
    C* tw = tvs + w * SR * KCT * LW;   // this warp's own entries of t (the block product's input)
    auto reduce = [&](const C* buf, auto&& use) {
      if constexpr (!PAIR) {
        // as a pair would: each half's eight warps in warp order, then (half 0 sum) + (half 1 sum)
        for (int e = tid; e < NE; e += NCT) {
          const int c = e % T, j = (e / T) % KCT, ii = e / (T * KCT);
          const C* b = buf + (ii * KCT + j) * T + c;
          C v0 = b[0], v1 = b[8 * SR * KCT * T];
#pragma unroll
          for (int ww = 1; ww < 8; ++ww) {
            v0 += b[ww * SR * KCT * T];
            v1 += b[(8 + ww) * SR * KCT * T];
          }
          cpart[(ii * KCT + j) * T + c] = v0 + v1;
        }
        consumer_sync<NCT>();
        for (int e = lane; e < SR * LW * KCT; e += 32) {
          const int u = e % LW, ii = (e / LW) % SR, j = e / (LW * SR);
          use(ii, j, u, cpart[(ii * KCT + j) * T + lw + u]);
        }
        __syncwarp();
        return;
      }
      const unsigned xb = xcount & 1u, xph = (xcount >> 1) & 1u;
      ++xcount;
      if (tid == 0 && !xdead) mbar_expect_tx(&xbar[xb], (unsigned)(NX * sizeof(C)));
      const unsigned pbar = mapa(&xbar[xb], peer);
      const unsigned pbuf = mapa(xbuf + xb * NX, peer);
      for (int e = tid; e < NE; e += NCT) {
        const int c = e % T, j = (e / T) % KCT, ii = e / (T * KCT);
        const C* b = buf + (ii * KCT + j) * T + c;
        C v = b[0];
#pragma unroll
        for (int ww = 1; ww < NCW; ++ww) v += b[ww * SR * KCT * T];
        const int slot16 = (ii * KCT + j) * 16 + (c & 15);
        if ((c >> 4) == (int)rank) cpart[slot16] = v;
        else st_async(pbuf + (unsigned)(slot16 * sizeof(C)), v, pbar);
      }
      consumer_sync<NCT>();
      xbar_wait(&xbar[xb], xph, &abort_flag, &xdead, B.err);
      for (int e = lane; e < SR * LW * KCT; e += 32) {
        const int u = e % LW, ii = (e / LW) % SR, j = e / (LW * SR);
        const int slot16 = (ii * KCT + j) * 16 + lw + u;
        use(ii, j, u, cpart[slot16] + xbuf[xb * NX + slot16]);
      }
      __syncwarp();
    };
    // One super-row of a sweep: coupling runs, reduction to t = y_q - sum, block-inverse runs on t,
    // reduction to the new y_q.  runs: the plan's (first operand block, tiles) per output block.
    // The inverse-block section of a full super-row (ntr = SR): its SR(SR+1)/2 tiles start in a fresh slot,
    // so every tile sits at a static offset; fully unrolled, one accumulator per output block, a slot handed
    // back after every CH tiles.  Forward: out_i += X(i, j) t_j, tiles (i, j) row by row; backward:
    // out_o += X(i, o)^T t_i, tiles (i, o) column by column.
    auto inverse_block = [&](bool fwd, C (&out)[SR][KCT]) {
#pragma unroll
      for (int a = 0; a < SR; ++a)
#pragma unroll
        for (int j = 0; j < KCT; ++j) out[a][j] = (C)0;
      int u = 0;
      auto tile = [&](int dst, int src) {
        C x0, x1;
        ld_pair(cur + u * (HT / 2), x0, x1);
#pragma unroll
        for (int j = 0; j < KCT; ++j) {
          const auto o0 = ld_pair2(tw + (src * KCT + j) * LW);
          out[dst][j] = fma(x0, o0.x, out[dst][j]);
          out[dst][j] = fma(x1, o0.y, out[dst][j]);
        }
        if (++u == CH) {
          leave_slot();
          u = 0;
        }
      };
      if (fwd) {
#pragma unroll
        for (int a = 0; a < SR; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b) tile(a, b);
      } else {
#pragma unroll
        for (int a = 0; a < SR; ++a)
#pragma unroll
          for (int b = a; b < SR; ++b) tile(a, b);
      }
      if (u != 0) leave_slot();
    };
    auto sweep_step = [&](int q, const int* runs, bool fwd) {
      const int I0 = q * SR, ntr = min(SR, nbt - I0);
      int lc = 0;
      for (int o = 0; o < ntr; ++o) lc += runs[2 * o + 1];
      start_section(lc);
      for (int o = 0; o < SR; ++o) {
        C res[KCT];
        if (o < ntr) {
          const int op0 = runs[2 * o], cnt = runs[2 * o + 1];
          run(cnt, y + op0 * YL + lw, YL, npadh, res);
        } else {
#pragma unroll
          for (int j = 0; j < KCT; ++j) res[j] = (C)0;
        }
#pragma unroll
        for (int j = 0; j < KCT; ++j) part[((w * SR + o) * KCT + j) * T + lane] = res[j];
      }
      consumer_sync<NCT>();
      reduce(part, [&](int ii, int j, int u, C tot) {
        tw[(ii * KCT + j) * LW + u] = ii < ntr ? y[j * npadh + (I0 + ii) * YL + lw + u] - tot : (C)0;
      });
      start_section(ntr * (ntr + 1) / 2);
      if (ntr == SR) {
        C out[SR][KCT];
        inverse_block(fwd, out);
#pragma unroll
        for (int o = 0; o < SR; ++o)
#pragma unroll
          for (int j = 0; j < KCT; ++j) dpart[((w * SR + o) * KCT + j) * T + lane] = out[o][j];
      } else {
        // a partial last super-row: the same products run by run
        for (int o = 0; o < SR; ++o) {
          C res[KCT];
          if (o < ntr) {
            if (fwd) run(o + 1, tw, KCT * LW, LW, res);
            else run(ntr - o, tw + o * KCT * LW, KCT * LW, LW, res);
          } else {
#pragma unroll
            for (int j = 0; j < KCT; ++j) res[j] = (C)0;
          }
#pragma unroll
          for (int j = 0; j < KCT; ++j) dpart[((w * SR + o) * KCT + j) * T + lane] = res[j];
        }
      }
      consumer_sync<NCT>();
      reduce(dpart, [&](int ii, int j, int u, C tot) {
        if (ii < ntr) y[j * npadh + (I0 + ii) * YL + lw + u] = tot;
      });
    };
    for (int q = 0; q < nsr; ++q) sweep_step(q, runs_s + q * SR * 2, true);
    for (int q = nsr - 1; q >= 0; --q) sweep_step(q, runs_s + (nsr + q) * SR * 2, false);
  }
  __syncthreads();
  // z_i = D^{-1/2} y on own entries, partial (r, z) of each half (a pair: of each CTA; rank 1 hands its sums to
  // rank 0), and the item's partial = (half 0 sum) + (half 1 sum); one CTA groups the rows exactly as a pair
  const int h = PAIR ? (int)rank : (tid >> 8);    // the half whose rows this thread takes
  const int th = PAIR ? tid : (tid & 255);        // its thread index within that half
  double prz[KCT];
#pragma unroll
  for (int j = 0; j < KCT; ++j) prz[j] = 0.0;
  if (w < NCW) {
    for (int m = th; m < nbt * 16; m += NCW_PAIR * 32) {
      const int i = (m >> 4) * T + 16 * h + (m & 15);
      if (i >= n) continue;
      const double sc = P.scale[d0 + i];
#pragma unroll
      for (int j = 0; j < KCT; ++j) {
        if (!act[j]) continue;
        const long long o = (long long)(k0 + j) * P.ndof + d0 + i;
        const double zv = sc * (double)y[j * npadh + (PAIR ? m : i)];
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
  if constexpr (PAIR) {
    double csum = 0.0;
    if (tid < kc) {
      for (int ww = 0; ww <= NCW; ++ww) csum += red[ww][tid];
      if (rank == 1) st_cluster(mapa(&peer_rz[tid], 0), csum);
    }
    cluster_sync();   // also: no access to this CTA's shared memory from the peer after this point
    if (rank == 0 && tid < kc) P.part_rz[(long long)s * P.k + k0 + tid] = P.done[k0 + tid] == 0 ? csum + peer_rz[tid] : 0.0;
  } else if (tid < kc) {
    double c0 = 0.0, c1 = 0.0;
    for (int ww = 0; ww < NCW_PAIR; ++ww) {
      c0 += red[ww][tid];
      c1 += red[NCW_PAIR + ww][tid];
    }
    c0 += red[NCW][tid];   // the producer warp's zero, where a pair's CTAs add theirs
    c1 += red[NCW][tid];
    P.part_rz[(long long)s * P.k + k0 + tid] = P.done[k0 + tid] == 0 ? c0 + c1 : 0.0;
  }
}

template <typename S, typename C, int KCT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NCW_PAIR * 32 + 32, 1)
    k_local(BatchDev B, int slot, int ring_off, int nstage) {
  local_body<S, C, KCT, true>(B, slot, ring_off, nstage);
}

template <typename S, typename C, int KCT>
__global__ void __launch_bounds__(2 * NCW_PAIR * 32 + 32, 1) k_local1(BatchDev B, int slot, int ring_off, int nstage) {
  local_body<S, C, KCT, false>(B, slot, ring_off, nstage);
}

// shared memory: y, partial sums, exchange buffers and run tables, then a ring of nstage slots of 32 KB of
// half tiles
template <typename S, typename C>
int smem_layout(int ndof_max, int kct, bool pair, int* ring_off, int* nstage, int* total) {
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  constexpr int SR = 8;
  const int npad = ((ndof_max + T - 1) / T) * T;
  const int nsr_max = (npad / T + SR - 1) / SR;
  const int ncw = pair ? NCW_PAIR : 2 * NCW_PAIR;
  const int head = (int)sizeof(C) * (kct * npad / (pair ? 2 : 1) + ncw * SR * kct * T + ncw * SR * LW * kct +
                                     (pair ? 3 * SR * kct * 16 : SR * kct * T)) +
                   (int)sizeof(int) * 4 * nsr_max * SR;
  const int off = (head + 127) & ~127;
  const int budget = optin - 2048 - off;   // static shared memory and slack
  const int slot = (pair ? 1 : 2) * slot_tiles<S>() * (int)(HT * sizeof(S)) + 16;   // 32 KB of tiles per half + barriers
  int ns = budget / slot;
  if (ns > 32) ns = 32;
  if (ns < 2) return -1;   // the subdomains are too large for this kernel's shared memory
  *ring_off = off;
  *nstage = ns;
  *total = off + ns * slot;
  return 0;
}

template <typename K>
int ensure_smem(K fn) {
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
  return 0;
}

// one CTA pair per item, or one CTA per item (the same bits; chosen by the caller, and a pair wherever a CTA
// alone would not hold two ring slots next to its subdomain's vectors)
template <typename S, typename C, int KCT>
int launch_one(const BatchDev& B, int slot, int items, int ndof_max, bool pair, cudaStream_t st) {
  int ring_off, nstage, smem;
  if (!pair && smem_layout<S, C>(ndof_max, KCT, false, &ring_off, &nstage, &smem)) pair = true;
  if (pair && smem_layout<S, C>(ndof_max, KCT, true, &ring_off, &nstage, &smem)) return (int)cudaErrorInvalidValue;
  if (pair) {
    auto fn = k_local<S, C, KCT>;
    if (int e = ensure_smem(fn)) return e;
    fn<<<2 * items, NCW_PAIR * 32 + 32, smem, st>>>(B, slot, ring_off, nstage);
  } else {
    auto fn = k_local1<S, C, KCT>;
    if (int e = ensure_smem(fn)) return e;
    fn<<<items, 2 * NCW_PAIR * 32 + 32, smem, st>>>(B, slot, ring_off, nstage);
  }
  return (int)cudaGetLastError();
}

template <typename S, typename C>
int launch_local_t(const BatchDev& B, int slot, int kcl, int items, int ndof_max, bool pair, cudaStream_t st) {
  if constexpr (sizeof(C) == 8) pair = true;   // FP64 sweeps always take both SMs' FP64 pipes
  return kcl == 0 ? launch_one<S, C, 1>(B, slot, items, ndof_max, pair, st)
                  : launch_one<S, C, KC>(B, slot, items, ndof_max, pair, st);
}

std::atomic<int> g_cta_form{0};   // 0: by the rule below, 1: one CTA per item, 2: a CTA pair per item

// Self-test of the bounded wait every ring and exchange wait of k_local goes through: one CTA waits on an
// mbarrier that nothing arrives on, with a limit of `limit` cycles; the wait gives up, sets the error word
// and the kernel returns normally (no trap, no fault, the context stays usable).
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(&bar, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(&bar, 0, &abort_flag, err, limit);
    err[1] = ok ? 0 : 1;
    mbar_arrive(&bar);   // complete the phase so the barrier is left consistent
  }
}

}  // namespace

// the launch is sized inside launch_local from ndof_max; this returns ndof_max itself so that callers
// can keep one number per launch slot
int local_smem_bytes(int /*prec*/, int ndof_max, int /*kc*/) { return ndof_max; }

int launch_wait_selftest(int* err, long long limit, void* stream) {
  k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(err, limit);
  return (int)cudaGetLastError();
}

// slot = K_NKINDS + 2 * prec + (kc > 1); `param` is the largest subdomain dof count of the launch
// The FP32 and BF16 sweeps run as CTA pairs while all of a launch's pairs fit on the GPU at once (the lowest
// latency for one problem), and as one CTA per item beyond that (no exchange, half the SMs per item: more
// items in flight for batches); both forms give the same bits.
int launch_local(const BatchDev& B, int slot, int total, int param, void* stream) {
  const int prec = (slot - K_NKINDS) / 2, kcl = (slot - K_NKINDS) % 2;
  cudaStream_t s = (cudaStream_t)stream;
  bool pair = true;
  const int form = g_cta_form.load();
  if (form == 1) {
    pair = false;
  } else if (form == 0) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return (int)cudaGetLastError();
    pair = 2 * total <= nsm;
  }
  switch (prec) {
    case DGASM_FP64: return launch_local_t<double, double>(B, slot, kcl, total, param, true, s);
    case DGASM_FP32:
    case DGASM_TF32: return launch_local_t<float, float>(B, slot, kcl, total, param, pair, s);
    default: return launch_local_t<__nv_bfloat16, float>(B, slot, kcl, total, param, pair, s);
  }
}

}  // namespace dgasm

extern "C" int dgasm_set_local_cta_form(int form) {
  if (form < 0 || form > 2) return dgasm::set_error(DGASM_EINVAL, "dgasm_set_local_cta_form: form %d is not 0, 1 or 2", form);
  dgasm::g_cta_form.store(form);
  return DGASM_OK;
}
