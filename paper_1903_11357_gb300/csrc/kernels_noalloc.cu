// Allocation-free entry point: y = A x together with the energy product x^T A x, for callers that must
// not allocate device memory after start-up: code whose device memory belongs to another runtime's caching
// allocator (which a cudaMalloc would bypass and fragment), and real-time loops whose allocation budget is
// fixed when they start.
//
// The kernel is a variant of the system SpMV: one thread per (element, row) as in dgasm_system_spmv, plus
// a deterministic reduction of x . (A x): every CTA writes its partial sum, and the last CTA (fenced
// atomic counter) adds them in CTA order.  The partial sums and the counter live in a file-scope
// __device__ array of fixed size instead of memory allocated per call.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "common.h"

namespace {

constexpr int NT = 256;
// scratch: the CTA counter (padded to 256 bytes), then one double per CTA
constexpr size_t NOALLOC_MAX_CTAS = 65536;
constexpr size_t NOALLOC_SCRATCH_BYTES = 256 + NOALLOC_MAX_CTAS * sizeof(double);  // 512 KB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(NT) k_spmv_dot_noalloc(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                        const double* __restrict__ vals, int ne, int np, int np2s,
                                                        const double* __restrict__ x, double* __restrict__ y,
                                                        double* __restrict__ xAx, unsigned char* scratch) {
  __shared__ double red[NT / 32];
  __shared__ int last;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch);
  double* part = reinterpret_cast<double*>(scratch + 256);
  const int epi = NT / np;
  const int e_begin = blockIdx.x * epi;
  const int nel = min(epi, ne - e_begin);
  const int t = threadIdx.x;
  double prod = 0.0;
  if (t < nel * np) {
    // the same loop and summation order as the system SpMV, so y matches it bit for bit
    const int e = e_begin + t / np, r = t % np;
    double acc = 0.0;
    for (int kb = rowptr[e]; kb < rowptr[e + 1]; ++kb) {
      const double* blk = vals + (long long)kb * np2s + r;
      const double* xc = x + (long long)col[kb] * np;
      for (int c = 0; c < np; ++c) acc = fma(blk[c * np], xc[c], acc);
    }
    y[(long long)e * np + r] = acc;
    prod = x[(long long)e * np + r] * acc;
  }
  prod = warp_sum(prod);
  if ((t & 31) == 0) red[t >> 5] = prod;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (t < 32) {
    double s = 0.0;
    for (unsigned i = t; i < gridDim.x; i += 32) s += part[i];
    s = warp_sum(s);
    if (t == 0) {
      *xAx = s;
      *counter = 0u;   // leave the counter at zero for the next call
    }
  }
}

// device address of the scratch array, looked up once per device with that device current
std::mutex g_mu;
void* g_addr[64] = {nullptr};

int scratch_address(void** out) {
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return dgasm::set_error(DGASM_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return dgasm::cuda_error((int)e, "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DGASM_OK;
}

}  // namespace

namespace {
// [a, a + na) and [b, b + nb) overlap (byte ranges of two caller arrays)
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + nb && b0 < a0 + na;
}
}  // namespace

extern "C" int dgasm_system_spmv_dot_noalloc(dgasm_system_t s, const double* x, double* y, double* xAx, void* stream) {
  using namespace dgasm;
  clear_error();
  if (!s || !x || !y || !xAx) return set_error(DGASM_EINVAL, "dgasm_system_spmv_dot_noalloc: NULL argument");
  const int ne = s->mesh->m.ne, np = s->np;
  const size_t vbytes = sizeof(double) * (size_t)ne * np;
  // x is read by every thread while y is written: the three arrays must not share memory
  if (overlap(x, vbytes, y, vbytes) || overlap(xAx, sizeof(double), x, vbytes) || overlap(xAx, sizeof(double), y, vbytes))
    return set_error(DGASM_EINVAL, "dgasm_system_spmv_dot_noalloc: x, y and xAx must not overlap");
  const int *rowptr, *col;
  const double* vals;
  int sys_dev;
  {
    // the upload (dgasm_system_spmv, dgasm_setup) publishes these under the same lock; host-only, no allocation
    std::lock_guard<std::mutex> lk(s->dev_mu);
    rowptr = s->d_rowptr.as<int>();
    col = s->d_col.as<int>();
    vals = s->d_vals.as<double>();
    sys_dev = s->dev;
  }
  if (!vals)
    return set_error(DGASM_EINVAL,
                     "dgasm_system_spmv_dot_noalloc: the matrix is not on the device yet; call dgasm_system_spmv "
                     "or dgasm_setup once first (they upload it)");
  int cur = -1;
  DG_CUDA(cudaGetDevice(&cur));
  if (cur != sys_dev)
    return set_error(DGASM_EINVAL, "dgasm_system_spmv_dot_noalloc: the matrix lives on device %d, device %d is current",
                     sys_dev, cur);
  const int epi = NT / np;
  const long long ctas = ((long long)ne + epi - 1) / epi;
  if (ctas > (long long)NOALLOC_MAX_CTAS)
    return set_error(DGASM_ETOOBIG,
                     "dgasm_system_spmv_dot_noalloc: %lld thread blocks needed, the fixed scratch holds %zu "
                     "(at most %zu elements for p = %d)", ctas, NOALLOC_MAX_CTAS, NOALLOC_MAX_CTAS * epi, s->p);
  void* scratch = nullptr;
  DG_TRY(scratch_address(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  // the counter must start at zero (a clear, not an allocation)
  DG_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned int), st));
  k_spmv_dot_noalloc<<<(unsigned)ctas, NT, 0, st>>>(rowptr, col, vals, ne, np, s->np2s, x, y, xAx,
                                                    (unsigned char*)scratch);
  DG_CUDA(cudaGetLastError());
  return DGASM_OK;
}
