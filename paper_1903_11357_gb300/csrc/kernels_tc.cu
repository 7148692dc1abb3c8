// Trailing update of the tile Cholesky factorisation of the subdomain matrices A_i (Sec. 3, local
// solvers: A_i is the principal submatrix of A on the subdomain's dofs) on the 5th-generation tensor cores,
// used by the TF32 precision mode (kind::tf32) and the BF16 precision mode (kind::f16 with BF16 operands).
//
// Step K of the right-looking tile Cholesky updates C_IJ -= L_IK L_JK^T for every pair I >= J of the tile
// rows S(s, K) below the diagonal tile that reach column K.  Per (subdomain, K) this is the lower triangle
// of the product P P^T of the panel P = [L_IK], I in S, a 32 |S| x 32 matrix.  A CTA takes a block of
// 4 row tiles (M = 128) against up to 8 column tiles (N <= 256) and forms it with tcgen05.mma of kind
// tf32 into tensor memory (128 lanes x N columns of FP32), then each of the 4 warps reads its 32 lanes
// (the rows of one row tile) back with tcgen05.ld and subtracts the tiles I >= J from the factor pool.
//
// TF32 keeps 10 mantissa bits.  Each FP32 operand is split as v = hi + lo with hi = tf32(v) and
// lo = tf32(v - hi), and the product is accumulated as lo*hi + hi*lo + hi*hi (the small terms first), which
// recovers close to FP32 accuracy from the TF32 tensor-core products ("split TF32", three MMAs per k-step),
// so the factor stays as accurate as the FP32 mode's and the subdomain Cholesky stays positive definite at
// the coefficient contrasts the method targets.
//
// BF16 keeps 8 mantissa bits, so the BF16 mode splits each FP32 operand three ways, v = hi + mid + lo with
// hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid), and accumulates the six products down to the
// order of FP32 rounding, lo*hi + hi*lo + mid*mid + mid*hi + hi*mid + hi*hi (six BF16 MMAs per K = 16 step):
// BF16 tensor-core products with FP32 accumulation in tensor memory at FP32-level accuracy.
//
// Operands are staged by the CTA's threads into shared memory in the canonical K-major layout without
// swizzling: core matrices of 8 rows x 16 bytes (4 TF32 or 8 BF16 entries), 128 contiguous bytes each; the core
// matrices of an 8-row group follow each other along K (leading-dimension offset 128 B) and row groups are
// 1024 B (TF32) or 512 B (BF16) apart (stride-dimension offset).  One thread issues the MMAs and commits them to an mbarrier; the
// wait on it is bounded, and on timeout the kernel sets the error word, skips its stores, waits once more
// (bounded) and frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <set>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int T = 32;
constexpr int TT = T * T;
constexpr int MBT = 4;                       // row tiles per block: M = 128
constexpr int NBT = 8;                       // column tiles per block: N <= 256
constexpr int TC_THREADS = 128;              // 4 warps: one per row tile (tensor-memory lane quarter)
// bytes of one split part of A (MBT row tiles) and of B (NBT row tiles): TF32 4 bytes, BF16 2 bytes an entry;
// TF32 splits in two parts, BF16 in three
template <bool BF> constexpr int a_bytes() { return MBT * TT * (BF ? 2 : 4); }
template <bool BF> constexpr int b_bytes() { return NBT * TT * (BF ? 2 : 4); }
template <bool BF> constexpr int tc_smem() { return (BF ? 3 : 2) * (a_bytes<BF>() + b_bytes<BF>()) + 1024; }
constexpr unsigned TMEM_COLS = 256;
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // about one second at the GB300 clock

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// byte offset of entry (row, k) in the canonical K-major layout of a 32-column (K = 32) operand
__device__ __forceinline__ unsigned canon_off(int row, int k) {
  return (unsigned)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_round(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of entry (row, k) in the canonical K-major layout of a 32-column BF16 operand: core matrices of
// 8 rows x 8 entries, four along K per 8-row group (512 B a group)
__device__ __forceinline__ unsigned canon_off_bf16(int row, int k) {
  return (unsigned)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading-dimension byte offset 128 (next core matrix along
// K), stride-dimension byte offset sbo (next 8-row group: 1024 B for TF32, 512 B for BF16), descriptor
// version 1, no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned sbo = 1024) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N and M
__host__ __device__ constexpr unsigned tf32_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

// instruction descriptor of kind::f16 with BF16 operands: D FP32, A and B BF16 (the same type), both K-major
__host__ __device__ constexpr unsigned bf16_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc, unsigned idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc, unsigned idesc,
                                         int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  return true;
}

// 32 lanes x 32 columns of 32-bit words from tensor memory: thread l gets lane (taddr lane + l)
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ long long tile_index(const EnvDev& E, int s, int I, int J) {
  const int tr = E.sub_trow[s] + I;
  return E.trow_ptr[tr] + (J - E.trow_F[tr]);
}

// stage the split parts of `ntile` tiles (rows 32 t + r, t < ntile, tile t at L + base[t] * TT) into hi/lo,
// zero rows up to ROWS; every load of the loop is independent of the others
template <int ROWS>
__device__ __forceinline__ void stage(const float* __restrict__ L, const long long* base, int ntile, unsigned char* hi,
                                      unsigned char* lo) {
  constexpr int NV = ROWS * (T / 4) / TC_THREADS;   // float4 per thread
  float4 v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i = threadIdx.x + j * TC_THREADS;
    const int row = i >> 3, kc = i & 7, t = row >> 5, r = row & 31;
    v[j] = t < ntile ? __ldg(reinterpret_cast<const float4*>(L + base[t] * TT + r * T + 4 * kc))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i = threadIdx.x + j * TC_THREADS;
    const int row = i >> 3, kc = i & 7;
    float4 h, l;
    h.x = tf32_round(v[j].x); l.x = tf32_round(v[j].x - h.x);
    h.y = tf32_round(v[j].y); l.y = tf32_round(v[j].y - h.y);
    h.z = tf32_round(v[j].z); l.z = tf32_round(v[j].z - h.z);
    h.w = tf32_round(v[j].w); l.w = tf32_round(v[j].w - h.w);
    const unsigned o = canon_off(row, 4 * kc);
    *reinterpret_cast<float4*>(hi + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}

// the BF16 three-way split of `ntile` tiles into p0 (hi), p1 (mid), p2 (lo), zero rows up to ROWS
__device__ __forceinline__ unsigned pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned*>(&v);
}

template <int ROWS>
__device__ __forceinline__ void stage_bf16(const float* __restrict__ L, const long long* base, int ntile,
                                           unsigned char* p0, unsigned char* p1, unsigned char* p2) {
  constexpr int NV = ROWS * (T / 4) / TC_THREADS;   // float4 per thread
  float4 v[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i = threadIdx.x + j * TC_THREADS;
    const int row = i >> 3, kc = i & 7, t = row >> 5, r = row & 31;
    v[j] = t < ntile ? __ldg(reinterpret_cast<const float4*>(L + base[t] * TT + r * T + 4 * kc))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i = threadIdx.x + j * TC_THREADS;
    const int row = i >> 3, kc = i & 7;
    const float x[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
    float h[4], m[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = __bfloat162float(__float2bfloat16_rn(x[q]));
      const float r1 = x[q] - h[q];
      m[q] = __bfloat162float(__float2bfloat16_rn(r1));
      l[q] = r1 - m[q];   // rounded to BF16 by the packing below
    }
    const unsigned o = canon_off_bf16(row, 4 * kc);
    *reinterpret_cast<uint2*>(p0 + o) = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
    *reinterpret_cast<uint2*>(p1 + o) = make_uint2(pack_bf16x2(m[0], m[1]), pack_bf16x2(m[2], m[3]));
    *reinterpret_cast<uint2*>(p2 + o) = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
  }
}

template <bool BF>
__global__ void __launch_bounds__(TC_THREADS) k_chol_update_tc(EnvDev E, float* __restrict__ L, int K,
                                                               const int* __restrict__ panel,
                                                               const int* __restrict__ tasks, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long done_bar;
  __shared__ unsigned tmem_base;
  __shared__ long long a_base[MBT], b_base[NBT], c_base[MBT][NBT];
  constexpr int AB = a_bytes<BF>(), BB = b_bytes<BF>(), NPART = BF ? 3 : 2;
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<size_t>(smem_raw) + 1023) & ~(size_t)1023);
  unsigned char* a_p[3] = {sm, sm + AB, sm + 2 * AB};   // split parts of A (hi, lo / hi, mid, lo)
  unsigned char* b_p[3] = {sm + NPART * AB, sm + NPART * AB + BB, sm + NPART * AB + 2 * BB};
  const int pstart = tasks[4 * blockIdx.x], n = tasks[4 * blockIdx.x + 1];
  const int mb = tasks[4 * blockIdx.x + 2], nb = tasks[4 * blockIdx.x + 3];
  const int s = panel[2 * pstart];
  const int a0 = MBT * mb, na = min(MBT, n - a0);          // row tiles of the block
  const int b0 = NBT * nb, nbt = min(NBT, min(n, a0 + MBT) - b0);   // column tiles
  const int N = T * nbt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tile indices, once per CTA: panel tiles (I, K) of the rows and columns, and the targets (I, J)
  if (threadIdx.x < MBT + NBT) {
    const int t = threadIdx.x;
    const bool row = t < MBT;
    const int e = row ? a0 + t : b0 + (t - MBT);
    if (row ? t < na : t - MBT < nbt) {
      const long long v = tile_index(E, s, panel[2 * (pstart + e) + 1], K);
      if (row) a_base[t] = v; else b_base[t - MBT] = v;
    }
  }
  if (threadIdx.x < MBT * NBT) {
    const int q = threadIdx.x / NBT, u = threadIdx.x % NBT;
    c_base[q][u] = (q < na && u < nbt && b0 + u <= a0 + q)
                       ? tile_index(E, s, panel[2 * (pstart + a0 + q) + 1], panel[2 * (pstart + b0 + u) + 1])
                       : -1;
  }
  __syncthreads();
  if constexpr (BF) {
    stage_bf16<MBT * T>(L, a_base, na, a_p[0], a_p[1], a_p[2]);
    if (nbt > 4) stage_bf16<NBT * T>(L, b_base, nbt, b_p[0], b_p[1], b_p[2]);
    else stage_bf16<4 * T>(L, b_base, nbt, b_p[0], b_p[1], b_p[2]);
  } else {
    stage<MBT * T>(L, a_base, na, a_p[0], a_p[1]);
    if (nbt > 4) stage<NBT * T>(L, b_base, nbt, b_p[0], b_p[1]);
    else stage<4 * T>(L, b_base, nbt, b_p[0], b_p[1]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy stores -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  const unsigned bar = smem_u32(&done_bar);

  if (threadIdx.x == 0) {
    int acc = 0;
    if constexpr (BF) {
      const unsigned idesc = bf16_idesc(MBT * T, N);
      const unsigned a0s = smem_u32(a_p[0]), a1s = smem_u32(a_p[1]), a2s = smem_u32(a_p[2]);
      const unsigned b0s = smem_u32(b_p[0]), b1s = smem_u32(b_p[1]), b2s = smem_u32(b_p[2]);
      // lo*hi, hi*lo, mid*mid, mid*hi, hi*mid, then hi*hi (the small terms first)
      const unsigned as[6] = {a2s, a0s, a1s, a1s, a0s, a0s}, bs[6] = {b0s, b2s, b1s, b0s, b1s, b0s};
#pragma unroll
      for (int pass = 0; pass < 6; ++pass)
#pragma unroll
        for (int ks = 0; ks < T / 16; ++ks) {   // K = 16 per MMA: two core matrices (256 B) along K
          mma_bf16(tmem, smem_desc(as[pass] + 256 * ks, 512), smem_desc(bs[pass] + 256 * ks, 512), idesc, acc);
          acc = 1;
        }
    } else {
      const unsigned idesc = tf32_idesc(MBT * T, N);
      const unsigned ah = smem_u32(a_p[0]), al = smem_u32(a_p[1]), bh = smem_u32(b_p[0]), bl = smem_u32(b_p[1]);
      const unsigned as[3] = {al, ah, ah}, bs[3] = {bh, bl, bh};   // lo*hi, hi*lo, then hi*hi
#pragma unroll
      for (int pass = 0; pass < 3; ++pass)
#pragma unroll
        for (int ks = 0; ks < T / 8; ++ks) {   // K = 8 per MMA: two core matrices (256 B) along K
          mma_tf32(tmem, smem_desc(as[pass] + 256 * ks), smem_desc(bs[pass] + 256 * ks), idesc, acc);
          acc = 1;
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
  }
  const bool ok = mbar_wait_bounded(bar, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int a = a0 + warp;   // this warp's row tile; its rows are tensor-memory lanes 32 warp ..
    if (warp < na) {
      for (int u = 0; u < nbt && b0 + u <= a; ++u) {
        float v[32];
        tmem_ld32(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)(32 * u), v);
        float4* c = reinterpret_cast<float4*>(L + c_base[warp][u] * TT + lane * T);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 x = c[q];
          x.x -= v[4 * q];
          x.y -= v[4 * q + 1];
          x.z -= v[4 * q + 2];
          x.w -= v[4 * q + 3];
          c[q] = x;
        }
      }
    }
  } else {
    if (lane == 0) atomicExch(err + 3, 1);
    mbar_wait_bounded(bar, 0);   // give the MMAs in flight one more bounded chance to land
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

namespace {
template <bool BF>
int launch_tc(const EnvDev& E, float* L, int K, const int* panel_task, const int* tasks, int n, int* err, void* stream) {
  if (n <= 0) return 0;
  {
    static std::mutex mu;
    static std::set<int> done;   // devices whose kernel attribute is set
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      cudaError_t e = cudaFuncSetAttribute(k_chol_update_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<BF>());
      if (e != cudaSuccess) return (int)e;
      done.insert(dev);
    }
  }
  k_chol_update_tc<BF><<<n, TC_THREADS, tc_smem<BF>(), (cudaStream_t)stream>>>(E, L, K, panel_task, tasks, err);
  return (int)cudaGetLastError();
}
}  // namespace

int launch_chol_update_tc(const EnvDev& E, float* L, int K, const int* panel_task, const int* tasks, int n, int* err,
                          void* stream, int bf16) {
  return bf16 ? launch_tc<true>(E, L, K, panel_task, tasks, n, err, stream)
              : launch_tc<false>(E, L, K, panel_task, tasks, n, err, stream);
}

}  // namespace dgasm
