// SIPG assembly on the device (Sec. 2, Eq. Ah with the lifting of Eq. lifting, penalty of Eq. Sigma): the
// same terms, quadrature and summation order as the host assembly, one CTA per element block row.
//
// The element term rho_kappa int grad phi_a . grad phi_b uses the fan of triangles from the vertex average with
// a Duffy-collapsed (p+2)-point Gauss rule per triangle; the faces of the element, in ascending face order,
// use a (p+2)-point Gauss rule and add the weighted-average consistency, symmetry and penalty terms to the
// diagonal block and, for interior faces, to the block of the neighbour.  Per chunk of quadrature points one
// thread per point evaluates every basis function into shared memory (the basis scaling of each box once per
// CTA); then thread t owns entries t, t + 128, ... of the blocks and adds the points' contributions in the
// host's order, so every entry is the same sum as on the host (up to the contraction of products into FMAs and
// the order of the basis scaling products).  The diagonal block is symmetric: only its entries a >= c are
// summed, and both halves stored at the end; the neighbour blocks (zero on entry) receive their face terms.  Blocks are
// written in the device layout: column-major, entry (a, c) at c * nb + a, stride np2s.
#include <cuda_runtime.h>

#include <algorithm>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int AT = 128;        // threads per element
// element quadrature points per shared-memory chunk (one thread per point evaluates every basis function)
template <int NB> constexpr int chunk_points() { return NB <= 21 ? 128 : 64; }

// Legendre polynomials and derivatives up to degree p at t (the host's recurrence)
__device__ __forceinline__ void legendre(int p, double t, double* L, double* dL) {
  L[0] = 1.0;
  dL[0] = 0.0;
  L[1] = t;
  dL[1] = 1.0;
  for (int k = 1; k < p; ++k) {
    L[k + 1] = ((2.0 * k + 1.0) * t * L[k] - k * L[k - 1]) / (k + 1.0);
    dL[k + 1] = dL[k - 1] + (2.0 * k + 1.0) * L[k];
  }
}

// per-box constants of the scaled Legendre basis: c_ij, c_ij 2/w_x, c_ij 2/w_y (function a = (i, j), ordered by
// total degree, then i descending)
struct BoxCoef {
  double cv, cx, cy;
};

template <int NB>
__device__ __forceinline__ void box_coefs(const double* box, const unsigned char* fi, const unsigned char* fj,
                                          BoxCoef* out) {
  const double wx = box[1] - box[0], wy = box[3] - box[2];
  for (int a = threadIdx.x; a < NB; a += blockDim.x) {
    const double i = fi[a], j = fj[a];
    const double c = sqrt((2.0 * i + 1.0) * (2.0 * j + 1.0) / (wx * wy));
    out[a] = BoxCoef{c, c * (2.0 / wx), c * (2.0 / wy)};
  }
}

template <int NB>
__global__ void __launch_bounds__(AT) k_assemble(AsmMesh M, int p, double c_sigma, const double* __restrict__ gt,
                                                 const double* __restrict__ gw, const int* __restrict__ rowptr,
                                                 const int* __restrict__ col, int np2s, double* __restrict__ vals) {
  constexpr int NL = NB * (NB + 1) / 2;     // entries a >= c of the symmetric diagonal block
  constexpr int EL = (NL + AT - 1) / AT;
  constexpr int EO = (NB * NB + AT - 1) / AT;
  extern __shared__ double sh[];
  __shared__ unsigned char fi[NB], fj[NB];
  __shared__ unsigned short la[NL], lc[NL];
  __shared__ BoxCoef own[NB], nbr[NB];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int mq = p + 2;
  const double* box = M.bbox + 4 * (long long)e;
  if (tid == 0) {
    int a = 0;
    for (int d = 0; d <= p; ++d)
      for (int i = d; i >= 0; --i, ++a) { fi[a] = (unsigned char)i; fj[a] = (unsigned char)(d - i); }
    int l = 0;
    for (int r = 0; r < NB; ++r)
      for (int c = 0; c <= r; ++c, ++l) { la[l] = (unsigned short)r; lc[l] = (unsigned short)c; }
  }
  __syncthreads();
  box_coefs<NB>(box, fi, fj, own);
  double D[EL];
#pragma unroll
  for (int u = 0; u < EL; ++u) D[u] = 0.0;
  __syncthreads();
  // ---- element term: points (triangle k, i, j) in the host's order, CHP at a time, one thread per point
  {
    constexpr int CHP = chunk_points<NB>();
    double* sw = sh;                 // [CHP] weight * rho
    double* sgx = sw + CHP;          // [CHP][NB]
    double* sgy = sgx + CHP * NB;
    const int v0 = M.ptr[e], nv = M.ptr[e + 1] - v0;
    double cx = 0.0, cy = 0.0;
    for (int k = 0; k < nv; ++k) {
      cx += M.xy[2 * (long long)M.vtx[v0 + k]];
      cy += M.xy[2 * (long long)M.vtx[v0 + k] + 1];
    }
    cx /= nv;
    cy /= nv;
    const int npts = nv * mq * mq;
    const double rho = M.rho[e];
    const double bx = 0.5 * (box[0] + box[1]), by = 0.5 * (box[2] + box[3]);
    const double wx = box[1] - box[0], wy = box[3] - box[2];
    for (int q0 = 0; q0 < npts; q0 += CHP) {
      const int nq = min(CHP, npts - q0);
      for (int qq = tid; qq < nq; qq += AT) {
        const int qp = q0 + qq;
        const int k = qp / (mq * mq), i = (qp / mq) % mq, j = qp % mq;
        const double* B = M.xy + 2 * (long long)M.vtx[v0 + k];
        const double* Cc = M.xy + 2 * (long long)M.vtx[v0 + (k + 1) % nv];
        const double e1x = B[0] - cx, e1y = B[1] - cy, e2x = Cc[0] - B[0], e2y = Cc[1] - B[1];
        const double u = gt[i], vv = gt[j];
        const double x = cx + u * e1x + u * vv * e2x, y = cy + u * e1y + u * vv * e2y;
        double Lx[10], dLx[10], Ly[10], dLy[10];
        legendre(p, 2.0 * (x - bx) / wx, Lx, dLx);
        legendre(p, 2.0 * (y - by) / wy, Ly, dLy);
#pragma unroll 4
        for (int a = 0; a < NB; ++a) {
          sgx[qq * NB + a] = own[a].cx * dLx[fi[a]] * Ly[fj[a]];
          sgy[qq * NB + a] = own[a].cy * Lx[fi[a]] * dLy[fj[a]];
        }
        sw[qq] = gw[i] * gw[j] * u * fabs(e1x * e2y - e1y * e2x) * rho;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < EL; ++u) {
        const int idx = tid + u * AT;
        if (idx < NL) {
          const int a = la[idx], c = lc[idx];
          double acc = D[u];
          for (int qq = 0; qq < nq; ++qq)
            acc += sw[qq] * (sgx[qq * NB + a] * sgx[qq * NB + c] + sgy[qq * NB + a] * sgy[qq * NB + c]);
          D[u] = acc;
        }
      }
      __syncthreads();
    }
  }
  // ---- faces of e in ascending face order
  double* fw = sh;                  // [mq] weights * length
  double* va = fw + 10;             // [mq][NB] own values
  double* dna = va + 10 * NB;       // [mq][NB] own normal derivatives
  double* vb = dna + 10 * NB;       // [mq][NB] neighbour values
  double* dnb = vb + 10 * NB;       // [mq][NB] neighbour normal derivatives
  const int r0 = rowptr[e], r1 = rowptr[e + 1];
  for (int fi_ = M.ef_ptr[e]; fi_ < M.ef_ptr[e + 1]; ++fi_) {
    const int f = M.ef_face[fi_];
    const int ep = M.f_ep[f], em = M.f_em[f];
    const double* P = M.xy + 2 * (long long)M.f_va[f];
    const double* Q = M.xy + 2 * (long long)M.f_vb[f];
    const double dx = Q[0] - P[0], dy = Q[1] - P[1], len = hypot(dx, dy);
    const double nx = dy / len, ny = -dx / len;   // outward normal of e_plus
    const int other = em < 0 ? -1 : (e == ep ? em : ep);
    if (other >= 0) box_coefs<NB>(M.bbox + 4 * (long long)other, fi, fj, nbr);
    __syncthreads();
    if (tid < 2 * mq && (tid < mq || other >= 0)) {   // one thread per (side, point)
      const int side = tid / mq, qp = tid % mq;
      const double* bb = side == 0 ? box : M.bbox + 4 * (long long)other;
      const BoxCoef* cf = side == 0 ? own : nbr;
      const double x = P[0] + gt[qp] * dx, y = P[1] + gt[qp] * dy;
      double Lx[10], dLx[10], Ly[10], dLy[10];
      legendre(p, 2.0 * (x - 0.5 * (bb[0] + bb[1])) / (bb[1] - bb[0]), Lx, dLx);
      legendre(p, 2.0 * (y - 0.5 * (bb[2] + bb[3])) / (bb[3] - bb[2]), Ly, dLy);
      double* vo = (side == 0 ? va : vb) + qp * NB;
      double* dno = (side == 0 ? dna : dnb) + qp * NB;
      for (int a = 0; a < NB; ++a) {
        vo[a] = cf[a].cv * Lx[fi[a]] * Ly[fj[a]];
        dno[a] = cf[a].cx * dLx[fi[a]] * Ly[fj[a]] * nx + cf[a].cy * Lx[fi[a]] * dLy[fj[a]] * ny;
      }
      if (side == 0) fw[qp] = gw[qp] * len;
    }
    __syncthreads();
    if (other < 0) {
      const double rho = M.rho[e];
      const double sigma = c_sigma * rho * p * p / M.diam[e];
#pragma unroll
      for (int u = 0; u < EL; ++u) {
        const int idx = tid + u * AT;
        if (idx < NL) {
          const int a = la[idx], c = lc[idx];
          double acc = D[u];
          for (int qp = 0; qp < mq; ++qp) {
            const double* vq = va + qp * NB;
            const double* dq = dna + qp * NB;
            acc += fw[qp] * (-rho * vq[a] * dq[c] - rho * vq[c] * dq[a] + sigma * vq[a] * vq[c]);
          }
          D[u] = acc;
        }
      }
    } else {
      const double sa = (e == ep) ? 1.0 : -1.0, sb = -sa;
      const double rh = 2.0 * M.rho[ep] * M.rho[em] / (M.rho[ep] + M.rho[em]);
      const double hh = 2.0 * M.diam[ep] * M.diam[em] / (M.diam[ep] + M.diam[em]);
      const double sigma = c_sigma * rh * p * p / hh;
#pragma unroll
      for (int u = 0; u < EL; ++u) {
        const int idx = tid + u * AT;
        if (idx < NL) {
          const int a = la[idx], c = lc[idx];
          double acc = D[u];
          for (int qp = 0; qp < mq; ++qp) {
            const double* vq = va + qp * NB;
            const double* dq = dna + qp * NB;
            acc += fw[qp] * (-0.5 * rh * sa * vq[a] * dq[c] - 0.5 * rh * sa * vq[c] * dq[a] + sigma * vq[a] * vq[c]);
          }
          D[u] = acc;
        }
      }
      int ko = r0;
      while (ko < r1 && col[ko] != other) ++ko;
      // the sparsity holds every face neighbour; a missing one would be a caller error: skip its block
      if (ko < r1) {
        double* O = vals + (long long)ko * np2s;
#pragma unroll
        for (int u = 0; u < EO; ++u) {
          const int idx = tid + u * AT;
          if (idx < NB * NB) {
            const int a = idx / NB, c = idx % NB;
            double oc = O[c * NB + a];
            for (int qp = 0; qp < mq; ++qp) {
              const double* vq = va + qp * NB;
              const double* dq = dna + qp * NB;
              const double* wq_ = vb + qp * NB;
              const double* eq = dnb + qp * NB;
              oc += fw[qp] * (-0.5 * rh * sa * vq[a] * eq[c] - 0.5 * rh * sb * wq_[c] * dq[a] + sigma * sa * sb * vq[a] * wq_[c]);
            }
            O[c * NB + a] = oc;
          }
        }
      }
    }
    __syncthreads();
  }
  int ks = r0;
  while (ks < r1 && col[ks] != e) ++ks;
  if (ks == r1) return;
  double* Dg = vals + (long long)ks * np2s;
#pragma unroll
  for (int u = 0; u < EL; ++u) {
    const int idx = tid + u * AT;
    if (idx < NL) {
      const int a = la[idx], c = lc[idx];
      Dg[c * NB + a] = D[u];
      Dg[a * NB + c] = D[u];
    }
  }
}

template <int NB>
int launch_nb(const AsmMesh& M, int p, double c_sigma, const double* gt, const double* gw, const int* rowptr,
              const int* col, int np2s, double* vals, cudaStream_t st) {
  constexpr int CHP = chunk_points<NB>();
  const size_t smem = sizeof(double) * (size_t)std::max(CHP + 2 * CHP * NB, 10 + 4 * 10 * NB);
  if (smem > 40 * 1024) {   // with the static tables the total passes the 48 KB default
    cudaError_t e = cudaFuncSetAttribute(k_assemble<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  k_assemble<NB><<<M.ne, AT, smem, st>>>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_assemble(const AsmMesh& M, int p, double c_sigma, const double* gt, const double* gw, const int* rowptr,
                    const int* col, int np2s, double* vals, void* stream) {
  if (M.ne <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  switch (p) {
    case 1: return launch_nb<3>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 2: return launch_nb<6>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 3: return launch_nb<10>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 4: return launch_nb<15>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 5: return launch_nb<21>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 6: return launch_nb<28>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    case 7: return launch_nb<36>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
    default: return launch_nb<45>(M, p, c_sigma, gt, gw, rowptr, col, np2s, vals, st);
  }
}

}  // namespace dgasm
