// Errors, device allocation hooks, Gauss-Legendre nodes and the Lanczos eigenvalue estimate.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "common.h"

namespace dgasm {

namespace {
thread_local int t_code = DGASM_OK;
thread_local char t_msg[512] = {0};

std::mutex g_alloc_mu;
dgasm_alloc_fn g_alloc = nullptr;
dgasm_free_fn g_free = nullptr;
void* g_alloc_user = nullptr;
}  // namespace

int set_error(int code, const char* fmt, ...) {
  t_code = code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_msg, sizeof(t_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(int cuda_code, const char* what) {
  return set_error(DGASM_ECUDA, "%s failed: %s", what, cudaGetErrorString((cudaError_t)cuda_code));
}

void clear_error() {
  t_code = DGASM_OK;
  t_msg[0] = 0;
}

void* dev_alloc(size_t bytes, void* stream) {
  if (bytes == 0) bytes = 16;
  dgasm_alloc_fn a;
  void* user;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    user = g_alloc_user;
  }
  if (a) return a(bytes, stream, user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, void* stream) {
  if (!p) return;
  dgasm_free_fn f;
  void* user;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_free;
    user = g_alloc_user;
  }
  if (f) {
    f(p, stream, user);
    return;
  }
  cudaFree(p);
}

int DevBuf::alloc(size_t n) {
  reset();
  ptr = dev_alloc(n, nullptr);
  if (!ptr) return set_error(DGASM_ENOMEM, "device allocation of %zu bytes failed", n);
  bytes = n;
  return DGASM_OK;
}

// A cudaMemcpy from pageable host memory returns once the data sit in the driver's staging buffer; the DMA to
// the destination is ordered only on the legacy default stream, and the library's kernels run on non-blocking
// streams.  The upload therefore waits for that stream before it returns, so that a kernel launched afterwards
// on any stream reads the new data, not what the allocation held before.
template <typename T>
int upload(DevBuf& dst, const std::vector<T>& src) {
  DG_TRY(dst.alloc(src.size() * sizeof(T)));
  if (!src.empty()) {
    DG_CUDA(cudaMemcpy(dst.ptr, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    DG_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
  }
  return DGASM_OK;
}
template int upload<int>(DevBuf&, const std::vector<int>&);
template int upload<long long>(DevBuf&, const std::vector<long long>&);
template int upload<double>(DevBuf&, const std::vector<double>&);
template int upload<float>(DevBuf&, const std::vector<float>&);

// Gauss-Legendre rule on [0, 1]: Newton on P_m from the Chebyshev-like guess, P_m by the Bonnet
// recurrence and P_m' = m (t P_m - P_{m-1}) / (t^2 - 1) on [-1, 1], then mapped.
void gauss_legendre01(int m, std::vector<double>& t, std::vector<double>& w) {
  t.assign(m, 0.0);
  w.assign(m, 0.0);
  if (m == 1) {
    t[0] = 0.5;
    w[0] = 1.0;
    return;
  }
  for (int i = 0; i < m; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (m + 0.5));
    double pm = 0, pm1 = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      double a = 1.0, b = x;
      for (int k = 1; k < m; ++k) {
        double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = c;
      }
      pm = b;
      pm1 = a;
      dp = m * (x * pm - pm1) / (x * x - 1.0);
      double dx = pm / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double a = 1.0, b = x;
    for (int k = 1; k < m; ++k) {
      double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
      a = b;
      b = c;
    }
    dp = m * (x * b - a) / (x * x - 1.0);
    // nodes come out in descending order of x: store ascending
    t[m - 1 - i] = 0.5 * (x + 1.0);
    w[m - 1 - i] = 0.5 * 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

}  // namespace dgasm

// ---- Lanczos extremes by Sturm-sequence bisection ------------------------------------------------
namespace {
// number of eigenvalues of the symmetric tridiagonal (d, e) smaller than x
int sturm_count(int k, const double* d, const double* e, double x) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0) ++cnt;
  for (int j = 1; j < k; ++j) {
    double qq = (q == 0.0) ? 1e-300 : q;
    q = d[j] - x - e[j - 1] * e[j - 1] / qq;
    if (q < 0) ++cnt;
  }
  return cnt;
}
}  // namespace

extern "C" int dgasm_lanczos(int k, const double* alpha, const double* beta, double* lmin, double* lmax) {
  using namespace dgasm;
  if (k <= 0 || !alpha || !lmin || !lmax || (k > 1 && !beta))
    return set_error(DGASM_EINVAL, "dgasm_lanczos: bad arguments");
  std::vector<double> d(k), e(k > 1 ? k - 1 : 1, 0.0);
  for (int j = 0; j < k; ++j) {
    d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j < k - 1) e[j] = std::sqrt(beta[j]) / alpha[j];
  }
  // Gershgorin interval
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < k; ++j) {
    double r = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j < k - 1 ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  if (!std::isfinite(lo) || !std::isfinite(hi)) return set_error(DGASM_ENAN, "dgasm_lanczos: non-finite coefficients");
  auto bisect = [&](int idx) {  // idx-th smallest eigenvalue (0-based)
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (a + b);
      if (mid == a || mid == b) break;
      if (sturm_count(k, d.data(), e.data(), mid) > idx) b = mid; else a = mid;
    }
    return 0.5 * (a + b);
  };
  *lmin = bisect(0);
  *lmax = bisect(k - 1);
  return DGASM_OK;
}

extern "C" int dgasm_last_error(char* buf, size_t n) {
  if (buf && n) {
    std::strncpy(buf, dgasm::t_msg, n - 1);
    buf[n - 1] = 0;
  }
  return dgasm::t_code;
}

extern "C" int dgasm_set_allocator(dgasm_alloc_fn alloc, dgasm_free_fn free_, void* user) {
  if ((alloc == nullptr) != (free_ == nullptr))
    return dgasm::set_error(DGASM_EINVAL, "dgasm_set_allocator: give both hooks or neither");
  std::lock_guard<std::mutex> lk(dgasm::g_alloc_mu);
  dgasm::g_alloc = alloc;
  dgasm::g_free = free_;
  dgasm::g_alloc_user = user;
  return DGASM_OK;
}
