// The paper's own elements: the boundary-conditioned operator K(rho) u for
// vector P1 on the structured grid cut into triangles (each unit square into
// 2, along the "right" / "left" diagonal or alternating by row) or
// tetrahedra (each unit cube into the 6 Kuhn tetrahedra), with one density
// per cell (Section 4 "Discretization the problem", Section 5 "Working with
// 3D problems"; bilinear form d^p sigma(u) : grad(v), sigma = 2 mu eps +
// lambda tr(eps) I, Section 4.3).
//
// Every cell of the structured grid is a translate of one of a few shapes (4
// triangles, 6 tetrahedra), so the host forms the unit-modulus matrix of each
// shape once, in FP64, from the cell's barycentric gradients, and the kernel
// gathers, for each node, the rows of the cells around it.  FP64 throughout:
// this is the parity form of the operator.
#include <algorithm>
#include <cmath>

#include "../../include/topo.h"
#include "common.cuh"
#include "p1.h"

namespace tp {

// Vertex offsets of each shape.  2D: 0, 1 = the two cells of a square cut
// along (0,0)-(1,1); 2, 3 = cut along (1,0)-(0,1) (cell 0 holds (0,0) and
// (1,0), cell 1 the rest).  3D: the Kuhn path for the axis orderings in
// lexicographic order.
void p1_shape_offsets(int dim, int type, int off[4][3]) {
  for (int v = 0; v < 4; v++)
    for (int a = 0; a < 3; a++) off[v][a] = 0;
  if (dim == 2) {
    static const int tri[4][3][2] = {{{0, 0}, {1, 0}, {1, 1}},
                                     {{0, 0}, {1, 1}, {0, 1}},
                                     {{0, 0}, {1, 0}, {0, 1}},
                                     {{1, 0}, {1, 1}, {0, 1}}};
    for (int v = 0; v < 3; v++) {
      off[v][0] = tri[type][v][0];
      off[v][1] = tri[type][v][1];
    }
    return;
  }
  static const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int p[3] = {0, 0, 0};
  for (int v = 1; v < 4; v++) {
    p[order[type][v - 1]] = 1;
    for (int a = 0; a < 3; a++) off[v][a] = p[a];
  }
}

// Unit-modulus matrix of the simplex with vertices X (nv = dim + 1): the
// barycentric gradients are the rows 1.. of [1 | X]^-1 (Gauss-Jordan with
// partial pivoting), the measure |det [1 | X]| / dim!, and
// K[d i + a][d j + b] = |T| (mu (delta_ab g_i . g_j + g_i[b] g_j[a]) + lambda g_i[a] g_j[b]).
static void simplex_matrix(int dim, const double X[4][3], double lam, double mu, double* K) {
  const int nv = dim + 1;
  double M[4][8];
  for (int r = 0; r < nv; r++) {
    M[r][0] = 1.0;
    for (int a = 0; a < dim; a++) M[r][1 + a] = X[r][a];
    for (int c = 0; c < nv; c++) M[r][nv + c] = r == c ? 1.0 : 0.0;
  }
  double det = 1.0;
  for (int c = 0; c < nv; c++) {
    int piv = c;
    for (int r = c + 1; r < nv; r++)
      if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
    if (piv != c) {
      for (int q = 0; q < 2 * nv; q++) std::swap(M[c][q], M[piv][q]);
      det = -det;
    }
    const double d = M[c][c];
    det *= d;
    for (int q = 0; q < 2 * nv; q++) M[c][q] /= d;
    for (int r = 0; r < nv; r++) {
      if (r == c) continue;
      const double f = M[r][c];
      for (int q = 0; q < 2 * nv; q++) M[r][q] -= f * M[c][q];
    }
  }
  // inverse in M[.][nv ..]; lambda_v = sum_r inv[r][v] * (1, x)_r
  double g[4][3];
  for (int v = 0; v < nv; v++)
    for (int a = 0; a < dim; a++) g[v][a] = M[1 + a][nv + v];
  const double meas = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
  const int nd = dim * nv;
  for (int i = 0; i < nv; i++)
    for (int j = 0; j < nv; j++) {
      double gg = 0.0;
      for (int a = 0; a < dim; a++) gg += g[i][a] * g[j][a];
      for (int a = 0; a < dim; a++)
        for (int b = 0; b < dim; b++)
          K[(dim * i + a) * nd + dim * j + b] =
              meas * (mu * ((a == b ? gg : 0.0) + g[i][b] * g[j][a]) + lam * g[i][a] * g[j][b]);
    }
}

// Unit matrices and vertex offsets of every cell shape of the grid (4 in 2D,
// 6 in 3D), K[t] row-major with dim * (dim + 1) rows.
int p1_shapes(int dim, double lam, double mu, double K[kP1MaxTypes][kP1MaxNd * kP1MaxNd],
              int off[kP1MaxTypes][4][3]) {
  const int ntypes = dim == 2 ? 4 : 6;
  for (int t = 0; t < ntypes; t++) {
    p1_shape_offsets(dim, t, off[t]);
    double X[4][3];
    for (int v = 0; v < 4; v++)
      for (int q = 0; q < 3; q++) X[v][q] = off[t][v][q];
    simplex_matrix(dim, X, lam, mu, K[t]);
  }
  return ntypes;
}

// Filter stencil on cell midpoints (the paper's weights rmin - distance,
// clipped at 0, between cell centroids): for each cell type tau, every cell
// of a square / cube displaced by d (|d_a| <= ceil(rmin) + 1) whose centroid
// lies closer than rmin.  In 2D the neighbour square's cut follows from its
// row: the centre's cut is type / 2, and with the alternating pattern each
// row step flips it.  An entry is (dx, dy, dz, local cell index, weight);
// entries are grouped by centre type.  Returns the number of entries, or -1
// when they exceed `cap`.
int p1_filter_stencil(int dim, int diagonal, double rmin, int cap, int* count, int (*ent)[4], double* w) {
  const int ntypes = dim == 2 ? 4 : 6, ncell = dim == 2 ? 2 : 6;
  double cen[kP1MaxTypes][3] = {};
  for (int t = 0; t < ntypes; t++) {
    int off[4][3];
    p1_shape_offsets(dim, t, off);
    for (int a = 0; a < 3; a++) {
      double sum = 0.0;
      for (int v = 0; v < dim + 1; v++) sum += off[v][a];
      cen[t][a] = sum / (dim + 1);
    }
  }
  const int r = (int)std::ceil(rmin) + 1;
  int n = 0;
  for (int t = 0; t < ntypes; t++) {
    if (dim == 2 && ((diagonal == 0 && t >= 2) || (diagonal == 1 && t < 2))) {
      count[t] = 0;
      continue;
    }
    int c0 = 0;
    for (int dz = (dim == 3 ? -r : 0); dz <= (dim == 3 ? r : 0); dz++)
      for (int dy = -r; dy <= r; dy++)
        for (int dx = -r; dx <= r; dx++) {
          const int cut = dim == 2 ? (diagonal == 2 ? ((t / 2 + dy) % 2 + 2) % 2 : diagonal) : 0;
          for (int l = 0; l < ncell; l++) {
            const int s2 = dim == 2 ? 2 * cut + l : l;
            const double ex = dx + cen[s2][0] - cen[t][0], ey = dy + cen[s2][1] - cen[t][1],
                         ez = dz + cen[s2][2] - cen[t][2];
            const double wt = rmin - std::sqrt(ex * ex + ey * ey + ez * ez);
            if (!(wt > 0.0)) continue;
            if (n >= cap) return -1;
            ent[n][0] = dx;
            ent[n][1] = dy;
            ent[n][2] = dz;
            ent[n][3] = l;
            w[n] = wt;
            n++;
            c0++;
          }
        }
    count[t] = c0;
  }
  return n;
}

namespace {

struct P1Args {
  int nx, ny, nz, diag, nc;
  long long ndof;
  double Emin, penal;
  const double* rho;
  const uint8_t* fixed;
  const double* u;
  double* y;
  P1Shapes sh;
};

// One thread per (node, case): y_i = sum over the cells around the node of
// E_c (K_c u_c) rows of the node, u masked on fixed DOFs; fixed rows y = u.
template <int DIM>
__global__ void p1_matvec_kernel(const __grid_constant__ P1Args a) {
  constexpr int NV = DIM + 1, ND = DIM * NV, NCELL = DIM == 2 ? 2 : 6;
  const long long nxy = (long long)(a.nx + 1) * (a.ny + 1);
  const long long nn = nxy * (DIM == 3 ? a.nz + 1 : 1);
  const int c = blockIdx.y;
  const double* u = a.u + (long long)c * a.ndof;
  double* y = a.y + (long long)c * a.ndof;
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < nn;
       nd += (long long)gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? (int)(nd / nxy) : 0;
    const long long rem = nd - (long long)k * nxy;
    const int j = (int)(rem / (a.nx + 1)), i = (int)(rem - (long long)j * (a.nx + 1));
    double acc[DIM];
#pragma unroll
    for (int q = 0; q < DIM; q++) acc[q] = 0.0;
    for (int ek = (DIM == 3 ? k - 1 : 0); ek <= (DIM == 3 ? k : 0); ek++) {
      if (DIM == 3 && (ek < 0 || ek >= a.nz)) continue;
      for (int ej = j - 1; ej <= j; ej++) {
        if (ej < 0 || ej >= a.ny) continue;
        const int tbase = DIM == 2 ? 2 * (a.diag == 2 ? (ej & 1) : a.diag) : 0;
        for (int ei = i - 1; ei <= i; ei++) {
          if (ei < 0 || ei >= a.nx) continue;
          const long long e = ei + (long long)a.nx * (ej + (long long)a.ny * ek);
          const int li = i - ei, lj = j - ej, lk = k - ek;
          for (int t = 0; t < NCELL; t++) {
            const int type = tbase + t;
            int av = -1;
#pragma unroll
            for (int v = 0; v < NV; v++)
              if (a.sh.off[type][v][0] == li && a.sh.off[type][v][1] == lj && (DIM == 2 || a.sh.off[type][v][2] == lk))
                av = v;
            if (av < 0) continue;
            const double E = a.Emin + pow(a.rho[NCELL * e + t], a.penal) * (1.0 - a.Emin);
#pragma unroll
            for (int m = 0; m < NV; m++) {
              const long long nm = (ei + a.sh.off[type][m][0]) +
                                   (long long)(a.nx + 1) * ((ej + a.sh.off[type][m][1]) +
                                                            (long long)(a.ny + 1) * (DIM == 3 ? ek + a.sh.off[type][m][2] : 0));
#pragma unroll
              for (int s = 0; s < DIM; s++) {
                const long long dof = DIM * nm + s;
                if (a.fixed[dof]) continue;
                const double uv = u[dof];
#pragma unroll
                for (int q = 0; q < DIM; q++) acc[q] += E * a.sh.K[type][(DIM * av + q) * ND + DIM * m + s] * uv;
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < DIM; q++) {
      const long long dof = DIM * nd + q;
      y[dof] = a.fixed[dof] ? u[dof] : acc[q];
    }
  }
}

}  // namespace
}  // namespace tp

extern "C" tp_status tp_p1_matvec(int dim, int nelx, int nely, int nelz, int diagonal, double lam, double mu,
                                  double Emin, double penal, const double* rho, const uint8_t* fixed,
                                  const double* u, double* y, int ncases, void* cuda_stream) {
  if (dim != 2 && dim != 3) return TP_ERR_ARG;
  if (nelx < 1 || nely < 1 || (dim == 3 ? nelz < 1 : nelz != 0)) return TP_ERR_ARG;
  if (dim == 2 ? (diagonal < 0 || diagonal > 2) : diagonal != 0) return TP_ERR_ARG;
  if (!(mu > 0.0) || !(lam + 2.0 * mu / dim > 0.0) || !std::isfinite(lam) || !std::isfinite(mu)) return TP_ERR_ARG;
  if (!(Emin >= 0.0 && Emin < 1.0) || !(penal >= 1.0 && penal <= 10.0)) return TP_ERR_ARG;
  if (ncases < 1 || ncases > 8 || !rho || !fixed || !u || !y) return TP_ERR_ARG;
  const long long nn = (long long)(nelx + 1) * (nely + 1) * (dim == 3 ? nelz + 1 : 1);
  if (nn > (1LL << 31)) return TP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  tp::P1Args a = {};
  tp::p1_shapes(dim, lam, mu, a.sh.K, a.sh.off);
  a.nx = nelx;
  a.ny = nely;
  a.nz = dim == 3 ? nelz : 0;
  a.diag = diagonal;
  a.nc = ncases;
  a.ndof = dim * nn;
  a.Emin = Emin;
  a.penal = penal;
  a.rho = rho;
  a.fixed = fixed;
  a.u = u;
  a.y = y;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TP_ERR_CUDA;
  }
  // grid-stride loop: at most 8 resident CTAs of 256 threads per SM
  const dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 8LL * std::max(nsm, 1)), ncases);
  if (dim == 2) tp::p1_matvec_kernel<2><<<grid, 256, 0, s>>>(a);
  else tp::p1_matvec_kernel<3><<<grid, 256, 0, s>>>(a);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TP_ERR_CUDA;
  }
  return TP_OK;
}

extern "C" tp_status tp_p1_shape_matrices(int dim, double lam, double mu, double* K, int* offsets) {
  if ((dim != 2 && dim != 3) || !K || !offsets) return TP_ERR_ARG;
  if (!(mu > 0.0) || !(lam + 2.0 * mu / dim > 0.0) || !std::isfinite(lam) || !std::isfinite(mu)) return TP_ERR_ARG;
  double Kt[tp::kP1MaxTypes][tp::kP1MaxNd * tp::kP1MaxNd] = {};
  int off[tp::kP1MaxTypes][4][3] = {};
  const int ntypes = tp::p1_shapes(dim, lam, mu, Kt, off);
  const int nd = dim * (dim + 1);
  for (int t = 0; t < ntypes; t++) {
    for (int r = 0; r < nd * nd; r++) K[t * nd * nd + r] = Kt[t][r];
    for (int v = 0; v < dim + 1; v++)
      for (int q = 0; q < dim; q++) offsets[(t * (dim + 1) + v) * dim + q] = off[t][v][q];
  }
  return TP_OK;
}

extern "C" tp_status tp_p1_filter_stencil(int dim, int diagonal, double rmin, int cap, int* count, int* entries,
                                          double* weights, int* n_entries) {
  if ((dim != 2 && dim != 3) || (dim == 2 ? (diagonal < 0 || diagonal > 2) : diagonal != 0)) return TP_ERR_ARG;
  if (!(rmin > 0.0 && rmin <= 16.0) || cap < 1 || !count || !entries || !weights || !n_entries) return TP_ERR_ARG;
  const int n = tp::p1_filter_stencil(dim, diagonal, rmin, cap, count, reinterpret_cast<int(*)[4]>(entries), weights);
  if (n < 0) return TP_ERR_ARG;
  *n_entries = n;
  return TP_OK;
}
