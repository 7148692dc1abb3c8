// SIPG assembly on the device (Sec. 2, Eq. Ah with the lifting of Eq. lifting, penalty of Eq. Sigma): the
// same terms, quadrature and summation order as the host assembly, one CTA per element block row.
//
// The element term rho_kappa int grad phi_a . grad phi_b uses the fan of triangles from the vertex average with
// a Duffy-collapsed (p+2)-point Gauss rule per triangle; the faces of the element, in ascending face order,
// use a (p+2)-point Gauss rule and add the weighted-average consistency, symmetry and penalty terms to the
// diagonal block and, for interior faces, to the block of the neighbour.  Per quadrature point the CTA first
// evaluates the needed basis functions into shared memory (one thread per (point, function)); then thread t
// owns entries t, t + 128, ... of the blocks and adds the points' contributions in the host's order, so
// every entry is the same sum as on the host (up to the contraction of products into FMAs).  The diagonal
// block is stored once at the end; the neighbour blocks (zero on entry) receive their face terms.  Blocks are
// written in the device layout: column-major, entry (a, c) at c * nb + a, stride np2s.
#include <cuda_runtime.h>

#include <algorithm>

#include "engine.h"

namespace dgasm {

namespace {

constexpr int AT = 128;        // threads per element
// element quadrature points per shared-memory chunk (one thread per point evaluates every basis function)
template <int NB> constexpr int chunk_points() { return NB <= 21 ? 128 : 64; }

// basis function a of P_p on box (x0, x1, y0, y1) at (x, y): value and gradient (scaled Legendre products,
// ordered by total degree, then i descending)
__device__ __forceinline__ void basis_fn(int p, int a, const double* box, double x, double y, double& v, double& gx,
                                         double& gy) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= a) ++d;
  const int i = d - (a - d * (d + 1) / 2), j = d - i;
  const double wx = box[1] - box[0], wy = box[3] - box[2];
  const double xi = 2.0 * (x - 0.5 * (box[0] + box[1])) / wx;
  const double eta = 2.0 * (y - 0.5 * (box[2] + box[3])) / wy;
  double L[2][10], dL[2][10];
  const double tt[2] = {xi, eta};
  for (int s = 0; s < 2; ++s) {
    L[s][0] = 1.0;
    dL[s][0] = 0.0;
    if (p >= 1) { L[s][1] = tt[s]; dL[s][1] = 1.0; }
    for (int k = 1; k < p; ++k) {
      L[s][k + 1] = ((2.0 * k + 1.0) * tt[s] * L[s][k] - k * L[s][k - 1]) / (k + 1.0);
      dL[s][k + 1] = dL[s][k - 1] + (2.0 * k + 1.0) * L[s][k];
    }
  }
  const double c = sqrt((2.0 * i + 1.0) * (2.0 * j + 1.0) / (wx * wy));
  v = c * L[0][i] * L[1][j];
  gx = c * dL[0][i] * (2.0 / wx) * L[1][j];
  gy = c * L[0][i] * dL[1][j] * (2.0 / wy);
}

// gradients of all NB basis functions at (x, y): the Legendre recurrences once per direction
template <int NB>
__device__ __forceinline__ void basis_grads(int p, const double* box, double x, double y, double* gx, double* gy) {
  const double wx = box[1] - box[0], wy = box[3] - box[2];
  const double xi = 2.0 * (x - 0.5 * (box[0] + box[1])) / wx;
  const double eta = 2.0 * (y - 0.5 * (box[2] + box[3])) / wy;
  double L[2][10], dL[2][10];
  const double tt[2] = {xi, eta};
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    L[s][0] = 1.0;
    dL[s][0] = 0.0;
    L[s][1] = tt[s];
    dL[s][1] = 1.0;
    for (int k = 1; k < p; ++k) {
      L[s][k + 1] = ((2.0 * k + 1.0) * tt[s] * L[s][k] - k * L[s][k - 1]) / (k + 1.0);
      dL[s][k + 1] = dL[s][k - 1] + (2.0 * k + 1.0) * L[s][k];
    }
  }
  int a = 0;
  for (int d = 0; d <= p; ++d)
    for (int i = d; i >= 0; --i, ++a) {
      const int j = d - i;
      const double c = sqrt((2.0 * i + 1.0) * (2.0 * j + 1.0) / (wx * wy));
      gx[a] = c * dL[0][i] * (2.0 / wx) * L[1][j];
      gy[a] = c * L[0][i] * dL[1][j] * (2.0 / wy);
    }
}

template <int NB>
__global__ void __launch_bounds__(AT) k_assemble(AsmMesh M, int p, double c_sigma, const double* __restrict__ gt,
                                                 const double* __restrict__ gw, const int* __restrict__ rowptr,
                                                 const int* __restrict__ col, int np2s, double* __restrict__ vals) {
  constexpr int NBB = NB * NB;
  constexpr int ENT = (NBB + AT - 1) / AT;   // block entries per thread
  extern __shared__ double sh[];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int mq = p + 2;
  const double* box = M.bbox + 4 * (long long)e;
  double D[ENT];
#pragma unroll
  for (int u = 0; u < ENT; ++u) D[u] = 0.0;
  // ---- element term: points (triangle k, i, j) in the host's order, CHP at a time
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
        basis_grads<NB>(p, box, x, y, sgx + qq * NB, sgy + qq * NB);
        sw[qq] = gw[i] * gw[j] * u * fabs(e1x * e2y - e1y * e2x) * rho;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < ENT; ++u) {
        const int idx = tid + u * AT;
        if (idx < NBB) {
          const int a = idx / NB, c = idx % NB;
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
  for (int fi = M.ef_ptr[e]; fi < M.ef_ptr[e + 1]; ++fi) {
    const int f = M.ef_face[fi];
    const int ep = M.f_ep[f], em = M.f_em[f];
    const double* P = M.xy + 2 * (long long)M.f_va[f];
    const double* Q = M.xy + 2 * (long long)M.f_vb[f];
    const double dx = Q[0] - P[0], dy = Q[1] - P[1], len = hypot(dx, dy);
    const double nx = dy / len, ny = -dx / len;   // outward normal of e_plus
    const int other = em < 0 ? -1 : (e == ep ? em : ep);
    const double* boxo = other >= 0 ? M.bbox + 4 * (long long)other : box;
    for (int t = tid; t < mq * NB * 2; t += AT) {
      const int side = t / (mq * NB), r = t % (mq * NB), qp = r / NB, a = r % NB;
      if (side == 1 && other < 0) continue;
      const double x = P[0] + gt[qp] * dx, y = P[1] + gt[qp] * dy;
      double v, gx, gy;
      basis_fn(p, a, side == 0 ? box : boxo, x, y, v, gx, gy);
      (side == 0 ? va : vb)[qp * NB + a] = v;
      (side == 0 ? dna : dnb)[qp * NB + a] = gx * nx + gy * ny;
      if (side == 0 && a == 0) fw[qp] = gw[qp] * len;
    }
    __syncthreads();
    if (other < 0) {
      const double rho = M.rho[e];
      const double sigma = c_sigma * rho * p * p / M.diam[e];
#pragma unroll
      for (int u = 0; u < ENT; ++u) {
        const int idx = tid + u * AT;
        if (idx < NBB) {
          const int a = idx / NB, c = idx % NB;
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
      int ko = r0;
      while (ko < r1 && col[ko] != other) ++ko;
      // the sparsity holds every face neighbour; a missing one would be a caller error: skip its block
      double* O = vals + (long long)(ko < r1 ? ko : r0) * np2s;
      const bool have = ko < r1;
#pragma unroll
      for (int u = 0; u < ENT; ++u) {
        const int idx = tid + u * AT;
        if (idx < NBB) {
          const int a = idx / NB, c = idx % NB;
          double acc = D[u];
          double oc = have ? O[c * NB + a] : 0.0;
          for (int qp = 0; qp < mq; ++qp) {
            const double* vq = va + qp * NB;
            const double* dq = dna + qp * NB;
            const double* wq_ = vb + qp * NB;
            const double* eq = dnb + qp * NB;
            acc += fw[qp] * (-0.5 * rh * sa * vq[a] * dq[c] - 0.5 * rh * sa * vq[c] * dq[a] + sigma * vq[a] * vq[c]);
            oc += fw[qp] * (-0.5 * rh * sa * vq[a] * eq[c] - 0.5 * rh * sb * wq_[c] * dq[a] + sigma * sa * sb * vq[a] * wq_[c]);
          }
          D[u] = acc;
          if (have) O[c * NB + a] = oc;
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
  for (int u = 0; u < ENT; ++u) {
    const int idx = tid + u * AT;
    if (idx < NBB) Dg[(idx % NB) * NB + idx / NB] = D[u];
  }
}

template <int NB>
int launch_nb(const AsmMesh& M, int p, double c_sigma, const double* gt, const double* gw, const int* rowptr,
              const int* col, int np2s, double* vals, cudaStream_t st) {
  constexpr int CHP = chunk_points<NB>();
  const size_t smem = sizeof(double) * (size_t)std::max(CHP + 2 * CHP * NB, 10 + 4 * 10 * NB);
  if (smem > 48 * 1024) {
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
