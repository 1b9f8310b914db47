// Host-side element data for the GB300 SIMP library: the unit Q4 (plane
// stress) and H8 (isotropic) stiffness K0 and the filter stencil.
//
// K0 = integral over the unit element of B^T D B, evaluated with 2-point
// Gauss-Legendre quadrature per axis (exact for the bilinear / trilinear
// element on a rectangle).  D follows the energy density of Section 2.1
// (Eq. "str_energy"): Lame mu = E / (2 (1 + nu)); lambda = E nu / ((1+nu)(1-2nu))
// in 3D and the plane-stress lambda* = E nu / (1 - nu^2) in 2D.
// Local node order: (0,0),(1,0),(1,1),(0,1) [then the same at z = 1];
// DOF order node-major, component-minor.
#include <cmath>
#include <vector>

#include "host.h"

namespace tp {

static inline int corner_off(int c, int axis) {
  const int q = c & 3;
  if (axis == 0) return (q == 1 || q == 2) ? 1 : 0;
  if (axis == 1) return (q >= 2) ? 1 : 0;
  return c >= 4 ? 1 : 0;
}

void element_k0(int dim, double nu, double* K) {
  const int nnode = dim == 2 ? 4 : 8;
  const int nd = dim * nnode;
  const int nv = dim == 2 ? 3 : 6;
  double D[6][6] = {};
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double lam = dim == 2 ? nu / (1.0 - nu * nu) : nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  for (int i = 0; i < dim; i++) {
    for (int j = 0; j < dim; j++) D[i][j] = lam;
    D[i][i] = lam + 2.0 * mu;
  }
  for (int i = dim; i < nv; i++) D[i][i] = mu;
  for (int i = 0; i < nd * nd; i++) K[i] = 0.0;
  const double g = 0.5 / std::sqrt(3.0);
  const double pts[2] = {0.5 - g, 0.5 + g};
  const double w = dim == 2 ? 0.25 : 0.125;
  const int nq = dim == 2 ? 4 : 8;
  std::vector<double> B(nv * nd);
  for (int q = 0; q < nq; q++) {
    double xi[3] = {pts[q & 1], pts[(q >> 1) & 1], pts[(q >> 2) & 1]};
    std::fill(B.begin(), B.end(), 0.0);
    for (int a = 0; a < nnode; a++) {
      double gr[3];
      for (int d = 0; d < dim; d++) {
        double v = 1.0;
        for (int e = 0; e < dim; e++) {
          const int o = corner_off(a, e);
          if (e == d) v *= o ? 1.0 : -1.0;
          else v *= o ? xi[e] : (1.0 - xi[e]);
        }
        gr[d] = v;
      }
      if (dim == 2) {
        B[0 * nd + 2 * a] = gr[0];
        B[1 * nd + 2 * a + 1] = gr[1];
        B[2 * nd + 2 * a] = gr[1];
        B[2 * nd + 2 * a + 1] = gr[0];
      } else {
        B[0 * nd + 3 * a] = gr[0];
        B[1 * nd + 3 * a + 1] = gr[1];
        B[2 * nd + 3 * a + 2] = gr[2];
        B[3 * nd + 3 * a + 1] = gr[2];
        B[3 * nd + 3 * a + 2] = gr[1];
        B[4 * nd + 3 * a] = gr[2];
        B[4 * nd + 3 * a + 2] = gr[0];
        B[5 * nd + 3 * a] = gr[1];
        B[5 * nd + 3 * a + 1] = gr[0];
      }
    }
    for (int i = 0; i < nd; i++)
      for (int j = 0; j < nd; j++) {
        double s = 0.0;
        for (int p = 0; p < nv; p++)
          for (int r = 0; r < nv; r++) s += B[p * nd + i] * D[p][r] * B[r * nd + j];
        K[i * nd + j] += w * s;
      }
  }
}

int filter_taps(int dim, double rmin, int max_taps, int* off, double* wts) {
  const int r = (int)std::ceil(rmin);
  int n = 0;
  for (int dz = (dim == 3 ? -r : 0); dz <= (dim == 3 ? r : 0); dz++)
    for (int dy = -r; dy <= r; dy++)
      for (int dx = -r; dx <= r; dx++) {
        const double d = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
        const double wt = rmin - d;
        if (wt > 0.0) {
          if (n >= max_taps) return -1;
          off[3 * n] = dx;
          off[3 * n + 1] = dy;
          off[3 * n + 2] = dz;
          wts[n] = wt;
          n++;
        }
      }
  return n;
}

}  // namespace tp
