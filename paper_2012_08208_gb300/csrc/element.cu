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

namespace tp {

// Generalised-strain factorisation K0 = G^T C G.
//
// G maps the element displacement vector to generalised strains: Walsh sums
// over the element corners of each displacement component (with weights
// s_x^a s_y^b s_z^c, s = +-1 by corner position), excluding the rigid-body
// combinations.  Its rows are mutually orthogonal, so C follows from the
// projection C = N^-1 G K0 G^T N^-1 with N = G G^T (diagonal).  Rigid modes lie
// in the null space of G exactly, which keeps them exact in FP32 arithmetic.
//
// Row order (2D, 5 rows): a_x(10), a_y(01), a_x(01)+a_y(10), a_x(11), a_y(11)
// Row order (3D, 18 rows), grouped by reflection-symmetry class:
//   0..2  a_x(100), a_y(010), a_z(001)
//   3..4  a_x(010)+a_y(100), a_z(111)
//   5..6  a_x(001)+a_z(100), a_y(111)
//   7..8  a_y(001)+a_z(010), a_x(111)
//   9..10 a_y(110), a_z(101)
//  11..12 a_x(110), a_z(011)
//  13..14 a_x(101), a_y(011)
//  15..17 a_x(011), a_y(101), a_z(110)
// where a_i(abc) = sum over corners of s_x^a s_y^b s_z^c u_i(corner).

static void strain_rows(int dim, std::vector<std::vector<double>>& G) {
  const int nnode = dim == 2 ? 4 : 8, nd = dim * nnode;
  auto walsh = [&](int comp, int a, int b, int c) {
    std::vector<double> r(nd, 0.0);
    for (int k = 0; k < nnode; k++) {
      const double sx = corner_off(k, 0) ? 1.0 : -1.0, sy = corner_off(k, 1) ? 1.0 : -1.0;
      const double sz = corner_off(k, 2) ? 1.0 : -1.0;
      double w = 1.0;
      if (a) w *= sx;
      if (b) w *= sy;
      if (c) w *= sz;
      r[dim * k + comp] = w;
    }
    return r;
  };
  auto add = [](std::vector<double> a, const std::vector<double>& b) {
    for (size_t i = 0; i < a.size(); i++) a[i] += b[i];
    return a;
  };
  G.clear();
  if (dim == 2) {
    G.push_back(walsh(0, 1, 0, 0));
    G.push_back(walsh(1, 0, 1, 0));
    G.push_back(add(walsh(0, 0, 1, 0), walsh(1, 1, 0, 0)));
    G.push_back(walsh(0, 1, 1, 0));
    G.push_back(walsh(1, 1, 1, 0));
    return;
  }
  G.push_back(walsh(0, 1, 0, 0));
  G.push_back(walsh(1, 0, 1, 0));
  G.push_back(walsh(2, 0, 0, 1));
  G.push_back(add(walsh(0, 0, 1, 0), walsh(1, 1, 0, 0)));
  G.push_back(walsh(2, 1, 1, 1));
  G.push_back(add(walsh(0, 0, 0, 1), walsh(2, 1, 0, 0)));
  G.push_back(walsh(1, 1, 1, 1));
  G.push_back(add(walsh(1, 0, 0, 1), walsh(2, 0, 1, 0)));
  G.push_back(walsh(0, 1, 1, 1));
  G.push_back(walsh(1, 1, 1, 0));
  G.push_back(walsh(2, 1, 0, 1));
  G.push_back(walsh(0, 1, 1, 0));
  G.push_back(walsh(2, 0, 1, 1));
  G.push_back(walsh(0, 1, 0, 1));
  G.push_back(walsh(1, 0, 1, 1));
  G.push_back(walsh(0, 0, 1, 1));
  G.push_back(walsh(1, 1, 0, 1));
  G.push_back(walsh(2, 1, 1, 0));
}

int element_strain_C(int dim, const double* K0, double* C, double* recon_err) {
  std::vector<std::vector<double>> G;
  strain_rows(dim, G);
  const int ng = (int)G.size(), nd = (int)G[0].size();
  std::vector<double> N(ng);
  for (int i = 0; i < ng; i++) {
    double s = 0.0;
    for (int k = 0; k < nd; k++) s += G[i][k] * G[i][k];
    N[i] = s;
  }
  for (int i = 0; i < ng; i++)
    for (int j = 0; j < ng; j++) {
      double s = 0.0;
      for (int a = 0; a < nd; a++)
        for (int b = 0; b < nd; b++) s += G[i][a] * K0[a * nd + b] * G[j][b];
      C[i * ng + j] = s / (N[i] * N[j]);
    }
  // reconstruction check: G^T C G == K0
  double err = 0.0;
  for (int a = 0; a < nd; a++)
    for (int b = 0; b < nd; b++) {
      double s = 0.0;
      for (int i = 0; i < ng; i++)
        for (int j = 0; j < ng; j++) s += G[i][a] * C[i * ng + j] * G[j][b];
      err = std::fmax(err, std::fabs(s - K0[a * nd + b]));
    }
  if (recon_err) *recon_err = err;
  return ng;
}

}  // namespace tp
