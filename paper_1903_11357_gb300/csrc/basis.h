// Scaled Legendre basis of P_p on an element's axis-aligned bounding box (Sec. 2, basis functions in the
// physical frame): phi_ij(x, y) = c_ij L_i(xi) L_j(eta), i + j <= p, ordered by degree then i descending,
// c_ij = sqrt((2i+1)(2j+1) / (w_x w_y)) so that the functions are orthonormal on the box.
#pragma once

#include <cmath>
#include <vector>

#include "common.h"

namespace dgasm {

struct Basis {
  int p, nb;
  std::vector<int> ii, jj;
  explicit Basis(int p_) : p(p_), nb(n_basis(p_)) {
    for (int d = 0; d <= p; ++d)
      for (int i = d; i >= 0; --i) { ii.push_back(i); jj.push_back(d - i); }
  }
  // values v[nb] and gradients g[2*nb] at (x, y) on box (x0, x1, y0, y1)
  void eval(const double* box, double x, double y, double* v, double* g) const {
    double wx = box[1] - box[0], wy = box[3] - box[2];
    double xi = 2.0 * (x - 0.5 * (box[0] + box[1])) / wx;
    double eta = 2.0 * (y - 0.5 * (box[2] + box[3])) / wy;
    double Lx[16], dLx[16], Ly[16], dLy[16];
    legendre(xi, Lx, dLx);
    legendre(eta, Ly, dLy);
    for (int a = 0; a < nb; ++a) {
      int i = ii[a], j = jj[a];
      double c = std::sqrt((2.0 * i + 1.0) * (2.0 * j + 1.0) / (wx * wy));
      v[a] = c * Lx[i] * Ly[j];
      if (g) {
        g[2 * a] = c * dLx[i] * (2.0 / wx) * Ly[j];
        g[2 * a + 1] = c * Lx[i] * dLy[j] * (2.0 / wy);
      }
    }
  }
  // the scaling c_a of every function on a box (a function of the box alone)
  void coefs(const double* box, double* c) const {
    double wx = box[1] - box[0], wy = box[3] - box[2];
    for (int a = 0; a < nb; ++a) c[a] = std::sqrt((2.0 * ii[a] + 1.0) * (2.0 * jj[a] + 1.0) / (wx * wy));
  }
  // values at n points (x_k, y_k interleaved in xy) with the scaling c from coefs(box), V[k * nb + a]: the
  // same numbers as eval, computed degree by degree over all points.  L holds 2 (p + 1) n doubles.
  void values_at(const double* box, const double* c, const double* xy, int n, double* V, double* L) const {
    const double wx = box[1] - box[0], wy = box[3] - box[2];
    const double mx = 0.5 * (box[0] + box[1]), my = 0.5 * (box[2] + box[3]);
    double* __restrict Lx = L;
    double* __restrict Ly = L + (size_t)(p + 1) * n;
    for (int k = 0; k < n; ++k) {
      Lx[k] = 1.0;
      Ly[k] = 1.0;
    }
    if (p >= 1)
      for (int k = 0; k < n; ++k) {
        Lx[n + k] = 2.0 * (xy[2 * k] - mx) / wx;
        Ly[n + k] = 2.0 * (xy[2 * k + 1] - my) / wy;
      }
    for (int d = 1; d < p; ++d) {
      const double* __restrict tx = Lx + n;
      const double* __restrict ty = Ly + n;
      for (int k = 0; k < n; ++k) {
        Lx[(size_t)(d + 1) * n + k] = ((2.0 * d + 1.0) * tx[k] * Lx[(size_t)d * n + k] - d * Lx[(size_t)(d - 1) * n + k]) / (d + 1.0);
        Ly[(size_t)(d + 1) * n + k] = ((2.0 * d + 1.0) * ty[k] * Ly[(size_t)d * n + k] - d * Ly[(size_t)(d - 1) * n + k]) / (d + 1.0);
      }
    }
    for (int a = 0; a < nb; ++a) {
      const double* __restrict lx = Lx + (size_t)ii[a] * n;
      const double* __restrict ly = Ly + (size_t)jj[a] * n;
      for (int k = 0; k < n; ++k) V[(size_t)k * nb + a] = c[a] * lx[k] * ly[k];
    }
  }
  void legendre(double t, double* L, double* dL) const {
    L[0] = 1.0; dL[0] = 0.0;
    if (p >= 1) { L[1] = t; dL[1] = 1.0; }
    for (int k = 1; k < p; ++k) {
      L[k + 1] = ((2.0 * k + 1.0) * t * L[k] - k * L[k - 1]) / (k + 1.0);
      dL[k + 1] = dL[k - 1] + (2.0 * k + 1.0) * L[k];
    }
  }
};

}  // namespace dgasm
