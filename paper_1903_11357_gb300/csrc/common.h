// Internal declarations shared by the host (C++) and device (CUDA) parts of libdgasm.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "dgasm.h"

namespace dgasm {

// ---- errors ------------------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(int cuda_code, const char* what);
void clear_error();

#define DG_CUDA(call)                                                  \
  do {                                                                 \
    int _e = (int)(call);                                              \
    if (_e != 0) return ::dgasm::cuda_error(_e, #call);                \
  } while (0)

#define DG_TRY(call)                                                   \
  do {                                                                 \
    int _r = (call);                                                   \
    if (_r < 0) return _r;                                             \
  } while (0)

// ---- device memory -------------------------------------------------------------------------------
void* dev_alloc(size_t bytes, void* stream);
void dev_free(void* p, void* stream);

// Owning device buffer (freed on destruction or reset).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : ptr(o.ptr), bytes(o.bytes) { o.ptr = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { reset(); ptr = o.ptr; bytes = o.bytes; o.ptr = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { reset(); }
  void reset() { if (ptr) dev_free(ptr, nullptr); ptr = nullptr; bytes = 0; }
  int alloc(size_t n);  // returns DGASM_OK or DGASM_ENOMEM; contents undefined
  template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// Upload a host vector into a fresh device buffer (synchronous).
template <typename T>
int upload(DevBuf& dst, const std::vector<T>& src);

// ---- basis and quadrature (library's own implementation) ---------------------------------------
inline int n_basis(int p) { return (p + 1) * (p + 2) / 2; }
void gauss_legendre01(int m, std::vector<double>& t, std::vector<double>& w);

// ---- mesh ---------------------------------------------------------------------------------------
struct MeshData {
  int nv = 0, ne = 0;
  std::vector<double> xy;        // 2 nv
  std::vector<int> ptr, vtx;     // polygon CSR
  std::vector<double> rho, area, cx, cy, diam;
  std::vector<double> bbox;      // 4 ne: x0, x1, y0, y1
  // faces sorted by (e_plus, e_minus, va); e_minus = -1 on the boundary
  std::vector<int> f_ep, f_em, f_va, f_vb;
  int nfi = 0, nfb = 0;
  std::vector<int> ef_ptr, ef_face;  // faces touching each element, ascending face id
};

}  // namespace dgasm

struct dgasm_mesh_s {
  dgasm::MeshData m;
};

struct dgasm_system_s {
  dgasm_mesh_s* mesh = nullptr;
  int p = 1, np = 3, np2s = 10;      // np2s: device block stride (np*np rounded up to even)
  double c_sigma = 10.0;
  // block CSR in the caller's element order; host blocks row-major
  std::vector<int> rowptr, col;
  std::vector<double> vals;
  std::vector<double> b;
  bool has_b = false;
  // device: blocks column-major (entry (a, c) of a block at c*np + a), stride np2s
  dgasm::DevBuf d_rowptr, d_col, d_vals;
  // device geometry for the coarse transfer
  dgasm::DevBuf d_xy, d_pptr, d_pvtx, d_bbox;
  int dev = -1;                      // CUDA device that holds the device arrays (-1: not uploaded yet)
  std::mutex dev_mu;
  int ensure_device();
  int ensure_host();   // host blocks of a device-assembled system
};
