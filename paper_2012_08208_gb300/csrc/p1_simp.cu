// The SIMP loop on the paper's own elements (Section 4: mesh of triangles, P1
// displacement, DG0 density; Section 5 "Working with 3D problems": the same on
// tetrahedra): a problem handle holding one structured grid of unit squares
// (cubes) cut into 2 triangles (6 Kuhn tetrahedra), one density per cell.
//
//   solve        K(rho) u_k = f_k by Jacobi-preconditioned CG in FP64 (the
//                paper factorises K, Section 4.3; the iteration reaches the same
//                true relative residual), all load cases in lock-step
//   sensitivities c = sum_k f_k^T u_k, ce_e = sum_k u_e^T K_e u_e,
//                dc_e = -p rho_e^(p-1) (1 - Emin) ce_e (Section 3.2, 4.4)
//   filter       the mesh-independency filter over cell midpoints
//                (Eq. "filter", "filter_mat"), rows truncated at the boundary
//   oc_update    the OC update with bisection on lambda (Eq. "update"), the
//                same kernel as for Q4 / H8
//
// Every cell is a translate of one of a few shapes, so each kernel receives the
// unit-modulus matrices of the shapes in its parameter block and gathers the
// cells around a node (operator, diagonal) or the vertices of a cell
// (sensitivities).  Dot products are summed per CTA and then over CTAs in a
// fixed order by the last CTA to finish (an arrival ticket), so results do not
// depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/topo.h"
#include "common.cuh"
#include "host.h"
#include "p1.h"

namespace tp {
namespace {

constexpr int kP1T = 256;  // threads per CTA

struct P1Geo {
  int dim, nx, ny, nz, diag, nc;  // squares / cubes per axis (nz = 0 in 2D), cut pattern, cases
  long long nn, ncell, ndof;
};

// Per-case CG scalars kept on the device between the iteration kernels.
struct P1Cg {
  double rz[kMaxCases];      // r^T z of the current residual
  double alpha[kMaxCases];
  double beta[kMaxCases];
  double rr[kMaxCases];      // ||r||^2 (recurrence, or true after a restart)
  double tol2ff[kMaxCases];  // tol^2 ||f_free||^2
  double comp[kMaxCases];    // f_k^T u_k (sensitivities)
  int state[kMaxCases];      // 0 active, 1 converged, 2 breakdown
  int it[kMaxCases];         // CG iterations of the case
  unsigned ticket[kMaxCases];
};

struct P1Args {
  P1Shapes sh;
  P1Geo g;
  const double* E;       // cell moduli
  const uint8_t* fixed;  // per DOF, 1 = Dirichlet
  const double* u;       // [nc][ndof]
  double* y;             // [nc][ndof]
  const double* f;       // loads [nc][ndof] (residual mode)
  double* part;          // per-CTA partial sums
  P1Cg* cg;
  int mode;              // 0 y = K u; 1 CG step q = K p with p^T q -> alpha; 2 y = f - K u (0 on fixed)
};

__device__ __forceinline__ int p1_cut(const P1Geo& g, int j) { return g.diag == 2 ? (j & 1) : g.diag; }

// Rows of node `nd` of sum_cells E_c K_c u_c, u read as 0 on fixed DOFs.
template <int DIM>
__device__ __forceinline__ void p1_node_rows(const P1Shapes& sh, const P1Geo& g, const double* __restrict__ E,
                                             const uint8_t* __restrict__ fixed, const double* __restrict__ u,
                                             long long nd, double (&acc)[DIM]) {
  constexpr int NV = DIM + 1, ND = DIM * NV, NCELL = DIM == 2 ? 2 : 6;
  const long long nxy = (long long)(g.nx + 1) * (g.ny + 1);
  const int k = DIM == 3 ? (int)(nd / nxy) : 0;
  const long long rem = nd - (long long)k * nxy;
  const int j = (int)(rem / (g.nx + 1)), i = (int)(rem - (long long)j * (g.nx + 1));
#pragma unroll
  for (int q = 0; q < DIM; q++) acc[q] = 0.0;
  for (int ek = (DIM == 3 ? k - 1 : 0); ek <= (DIM == 3 ? k : 0); ek++) {
    if (DIM == 3 && (ek < 0 || ek >= g.nz)) continue;
    for (int ej = j - 1; ej <= j; ej++) {
      if (ej < 0 || ej >= g.ny) continue;
      const int tbase = DIM == 2 ? 2 * p1_cut(g, ej) : 0;
      for (int ei = i - 1; ei <= i; ei++) {
        if (ei < 0 || ei >= g.nx) continue;
        const long long e = ei + (long long)g.nx * (ej + (long long)g.ny * ek);
        const int li = i - ei, lj = j - ej, lk = k - ek;
        for (int t = 0; t < NCELL; t++) {
          const int type = tbase + t;
          int av = -1;
#pragma unroll
          for (int v = 0; v < NV; v++)
            if (sh.off[type][v][0] == li && sh.off[type][v][1] == lj && (DIM == 2 || sh.off[type][v][2] == lk))
              av = v;
          if (av < 0) continue;
          const double Ec = E[NCELL * e + t];
#pragma unroll
          for (int m = 0; m < NV; m++) {
            const long long nm = (ei + sh.off[type][m][0]) +
                                 (long long)(g.nx + 1) * ((ej + sh.off[type][m][1]) +
                                                          (long long)(g.ny + 1) * (DIM == 3 ? ek + sh.off[type][m][2] : 0));
#pragma unroll
            for (int s = 0; s < DIM; s++) {
              const long long dof = DIM * nm + s;
              if (fixed[dof]) continue;
              const double uv = u[dof];
#pragma unroll
              for (int q = 0; q < DIM; q++) acc[q] += Ec * sh.K[type][(DIM * av + q) * ND + DIM * m + s] * uv;
            }
          }
        }
      }
    }
  }
}

// Block totals of NV values, stored per case; the last CTA of the case to
// arrive sums all CTAs' totals in a fixed order and returns true with the grand
// totals in v (uniform over the CTA).  `sm` holds 32 * NV doubles.
template <int NV>
__device__ bool case_totals(double (&v)[NV], double* part, unsigned* ticket, double* sm) {
  __shared__ int s_last;
  block_sum<NV>(v, sm);
  const int c = blockIdx.y, nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) part[((size_t)c * NV + i) * nb + blockIdx.x] = v[i];
    __threadfence();
    const unsigned t = atomicAdd(ticket + c, 1u);
    s_last = t == (unsigned)(nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double tot[NV];
#pragma unroll
  for (int i = 0; i < NV; i++) {
    tot[i] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) tot[i] += __ldcg(part + ((size_t)c * NV + i) * nb + b);
  }
  block_sum<NV>(tot, sm);
#pragma unroll
  for (int i = 0; i < NV; i++) v[i] = tot[i];
  if (threadIdx.x == 0) ticket[c] = 0;
  return true;
}

// Operator application over nodes (gridDim.y = cases), in one of three modes.
template <int DIM>
__global__ void __launch_bounds__(kP1T) p1_apply_kernel(const __grid_constant__ P1Args a) {
  __shared__ double sm[32];
  const int c = blockIdx.y;
  if (a.mode == 1 && a.cg->state[c] != 0) return;  // this case is done
  const double* u = a.u + (size_t)c * a.g.ndof;
  double* y = a.y + (size_t)c * a.g.ndof;
  double dot[1] = {0.0};
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < a.g.nn;
       nd += (long long)gridDim.x * blockDim.x) {
    double acc[DIM];
    p1_node_rows<DIM>(a.sh, a.g, a.E, a.fixed, u, nd, acc);
#pragma unroll
    for (int q = 0; q < DIM; q++) {
      const long long dof = DIM * nd + q;
      const bool fx = a.fixed[dof] != 0;
      if (a.mode == 2) {
        y[dof] = fx ? 0.0 : a.f[(size_t)c * a.g.ndof + dof] - acc[q];
      } else {
        y[dof] = fx ? u[dof] : acc[q];
        if (a.mode == 1 && !fx) dot[0] += u[dof] * acc[q];
      }
    }
  }
  if (a.mode != 1) return;
  if (case_totals<1>(dot, a.part, a.cg->ticket, sm) && threadIdx.x == 0) {
    const double pq = dot[0];
    if (!(pq > 0.0) || !isfinite(pq)) {
      a.cg->state[c] = 2;
      a.cg->alpha[c] = 0.0;
    } else {
      a.cg->alpha[c] = a.cg->rz[c] / pq;
    }
  }
}

struct P1Vec {
  long long ndof;
  const uint8_t* fixed;
  const double* invd;
  double* x;
  double* r;
  double* z;
  double* p;
  const double* q;
  double* part;
  P1Cg* cg;
  unsigned mask;  // restart kernel: cases to restart
};

// x += alpha p, r -= alpha q, z = D^-1 r; r^T z and r^T r; the last CTA sets
// beta, the state and the iteration count of the case.
__global__ void __launch_bounds__(kP1T) p1_update_kernel(const __grid_constant__ P1Vec a) {
  __shared__ double sm[64];
  const int c = blockIdx.y;
  if (a.cg->state[c] != 0) return;
  const double alpha = a.cg->alpha[c];
  const size_t o = (size_t)c * a.ndof;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.ndof;
       i += (long long)gridDim.x * blockDim.x) {
    const double pi = a.p[o + i], qi = a.q[o + i];
    a.x[o + i] += alpha * pi;
    const double ri = a.r[o + i] - alpha * qi;
    a.r[o + i] = ri;
    const double zi = a.invd[i] * ri;
    a.z[o + i] = zi;
    v[0] += ri * zi;
    v[1] += ri * ri;
  }
  if (case_totals<2>(v, a.part, a.cg->ticket, sm) && threadIdx.x == 0) {
    P1Cg* cg = a.cg;
    cg->it[c]++;
    cg->rr[c] = v[1];
    if (!isfinite(v[0]) || !isfinite(v[1])) {
      cg->state[c] = 2;
    } else if (v[1] <= cg->tol2ff[c]) {
      cg->state[c] = 1;
    } else {
      cg->beta[c] = cg->rz[c] != 0.0 ? v[0] / cg->rz[c] : 0.0;
    }
    cg->rz[c] = v[0];
  }
}

// p = z + beta p.
__global__ void __launch_bounds__(kP1T) p1_direction_kernel(const __grid_constant__ P1Vec a) {
  const int c = blockIdx.y;
  if (a.cg->state[c] != 0) return;
  const double beta = a.cg->beta[c];
  const size_t o = (size_t)c * a.ndof;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.ndof;
       i += (long long)gridDim.x * blockDim.x)
    a.p[o + i] = a.z[o + i] + beta * a.p[o + i];
}

// Restart from a freshly computed true residual r (cases in `mask`): z = D^-1 r,
// p = z, r^T z and the true ||r||^2 (x is zeroed on fixed DOFs, where the
// residual kernel already read it as 0); the case is converged if the true residual
// meets the tolerance, active otherwise.
__global__ void __launch_bounds__(kP1T) p1_restart_kernel(const __grid_constant__ P1Vec a) {
  __shared__ double sm[64];
  const int c = blockIdx.y;
  if (!((a.mask >> c) & 1u)) return;
  const size_t o = (size_t)c * a.ndof;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.ndof;
       i += (long long)gridDim.x * blockDim.x) {
    if (a.fixed[i]) a.x[o + i] = 0.0;  // u = 0 on Dirichlet DOFs (a user start may hold other values)
    const double ri = a.r[o + i], zi = a.invd[i] * ri;
    a.z[o + i] = zi;
    a.p[o + i] = zi;
    v[0] += ri * zi;
    v[1] += ri * ri;
  }
  if (case_totals<2>(v, a.part, a.cg->ticket, sm) && threadIdx.x == 0) {
    P1Cg* cg = a.cg;
    cg->rz[c] = v[0];
    cg->rr[c] = v[1];
    cg->beta[c] = 0.0;
    cg->state[c] = !isfinite(v[1]) ? 2 : (v[1] <= cg->tol2ff[c] ? 1 : 0);
  }
}

struct P1Cell {
  P1Shapes sh;
  P1Geo g;
  const double* rho;
  double Emin, penal;
  double* E;              // young: E out
  const uint8_t* fixed;   // diag
  double* invd;           // diag out
  const double* x;        // sens: displacements [nc][ndof]
  const double* f;        // sens: loads [nc][ndof]
  double* ce;             // sens out
  double* dc;             // sens out
  double* part;
  P1Cg* cg;
};

__global__ void p1_young_kernel(const double* __restrict__ rho, double* __restrict__ E, long long n, double Emin,
                                double penal) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
    E[c] = Emin + pow(rho[c], penal) * (1.0 - Emin);
}

// Inverse of the diagonal of K(rho) (1 on fixed DOFs), one thread per node.
template <int DIM>
__global__ void __launch_bounds__(kP1T) p1_diag_kernel(const __grid_constant__ P1Cell a) {
  constexpr int NV = DIM + 1, ND = DIM * NV, NCELL = DIM == 2 ? 2 : 6;
  const P1Geo& g = a.g;
  const long long nxy = (long long)(g.nx + 1) * (g.ny + 1);
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < g.nn;
       nd += (long long)gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? (int)(nd / nxy) : 0;
    const long long rem = nd - (long long)k * nxy;
    const int j = (int)(rem / (g.nx + 1)), i = (int)(rem - (long long)j * (g.nx + 1));
    double d[DIM];
#pragma unroll
    for (int q = 0; q < DIM; q++) d[q] = 0.0;
    for (int ek = (DIM == 3 ? k - 1 : 0); ek <= (DIM == 3 ? k : 0); ek++) {
      if (DIM == 3 && (ek < 0 || ek >= g.nz)) continue;
      for (int ej = j - 1; ej <= j; ej++) {
        if (ej < 0 || ej >= g.ny) continue;
        const int tbase = DIM == 2 ? 2 * p1_cut(g, ej) : 0;
        for (int ei = i - 1; ei <= i; ei++) {
          if (ei < 0 || ei >= g.nx) continue;
          const long long e = ei + (long long)g.nx * (ej + (long long)g.ny * ek);
          for (int t = 0; t < NCELL; t++) {
            const int type = tbase + t;
            for (int v = 0; v < NV; v++) {
              if (a.sh.off[type][v][0] != i - ei || a.sh.off[type][v][1] != j - ej ||
                  (DIM == 3 && a.sh.off[type][v][2] != k - ek))
                continue;
              const double Ec = a.E[NCELL * e + t];
#pragma unroll
              for (int q = 0; q < DIM; q++) d[q] += Ec * a.sh.K[type][(DIM * v + q) * ND + DIM * v + q];
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < DIM; q++) {
      const long long dof = DIM * nd + q;
      a.invd[dof] = a.fixed[dof] ? 1.0 : 1.0 / d[q];
    }
  }
}

// Vertex nodes of cell `cell`; returns its shape.
template <int DIM>
__device__ __forceinline__ int p1_cell_nodes(const P1Shapes& sh, const P1Geo& g, long long cell, long long (&nodes)[DIM + 1]) {
  constexpr int NCELL = DIM == 2 ? 2 : 6;
  const long long e = cell / NCELL;
  const int t = (int)(cell - e * NCELL);
  const long long exy = (long long)g.nx * g.ny;
  const int k = DIM == 3 ? (int)(e / exy) : 0;
  const long long rem = e - (long long)k * exy;
  const int j = (int)(rem / g.nx), i = (int)(rem - (long long)j * g.nx);
  const int type = DIM == 2 ? 2 * p1_cut(g, j) + t : t;
#pragma unroll
  for (int v = 0; v < DIM + 1; v++)
    nodes[v] = (i + sh.off[type][v][0]) +
               (long long)(g.nx + 1) * ((j + sh.off[type][v][1]) + (long long)(g.ny + 1) * (DIM == 3 ? k + sh.off[type][v][2] : 0));
  return type;
}

// ce_e = sum_k u_e^T K_e u_e (unit modulus) and dc_e = -p rho^(p-1) (1 - Emin) ce_e,
// one thread per cell.
template <int DIM>
__global__ void __launch_bounds__(kP1T) p1_sens_kernel(const __grid_constant__ P1Cell a) {
  constexpr int NV = DIM + 1, ND = DIM * NV, NT = DIM == 2 ? 4 : 6;
  __shared__ double sK[NT * ND * ND];  // the shapes' matrices, staged once per CTA
  for (int i = threadIdx.x; i < NT * ND * ND; i += blockDim.x) sK[i] = a.sh.K[i / (ND * ND)][i % (ND * ND)];
  __syncthreads();
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < a.g.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    long long nodes[NV];
    const int type = p1_cell_nodes<DIM>(a.sh, a.g, cell, nodes);
    double ce = 0.0;
    for (int c = 0; c < a.g.nc; c++) {
      const double* x = a.x + (size_t)c * a.g.ndof;
      double ue[ND];
#pragma unroll
      for (int v = 0; v < NV; v++)
#pragma unroll
        for (int q = 0; q < DIM; q++) ue[DIM * v + q] = x[DIM * nodes[v] + q];
      const double* K = sK + type * ND * ND;
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < ND; r++) {
        double kr = 0.0;
#pragma unroll
        for (int m = 0; m < ND; m++) kr += K[r * ND + m] * ue[m];
        s += ue[r] * kr;
      }
      ce += s;
    }
    a.ce[cell] = ce;
    a.dc[cell] = -a.penal * pow(a.rho[cell], a.penal - 1.0) * (1.0 - a.Emin) * ce;
  }
}

// f_k^T u_k per case (gridDim.y = cases), summed in a fixed order.
__global__ void __launch_bounds__(kP1T) p1_compliance_kernel(const __grid_constant__ P1Cell a) {
  __shared__ double sm[32];
  const int c = blockIdx.y;
  const double* x = a.x + (size_t)c * a.g.ndof;
  const double* f = a.f + (size_t)c * a.g.ndof;
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.g.ndof;
       i += (long long)gridDim.x * blockDim.x)
    v[0] += f[i] * x[i];
  if (case_totals<1>(v, a.part, a.cg->ticket, sm) && threadIdx.x == 0) a.cg->comp[c] = v[0];
}

struct P1Filt {
  P1Geo g;
  const int4* ent;      // (dx, dy, dz, local cell) per stencil entry
  const double* w;      // weights
  int soff[kP1MaxTypes + 1];  // entries of centre shape t: [soff[t], soff[t + 1])
  const double* rho;
  const double* dc;
  double* out;
};

// dc~_a = sum_b w_ab rho_b dc_b / (rho_a sum_b w_ab) over the cells b of the
// grid (rows truncated at the boundary), one thread per cell.
template <int DIM>
__global__ void __launch_bounds__(kP1T) p1_filter_kernel(const __grid_constant__ P1Filt a) {
  constexpr int NCELL = DIM == 2 ? 2 : 6;
  const P1Geo& g = a.g;
  const long long exy = (long long)g.nx * g.ny;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    const long long e = cell / NCELL;
    const int l = (int)(cell - e * NCELL);
    const int k = DIM == 3 ? (int)(e / exy) : 0;
    const long long rem = e - (long long)k * exy;
    const int j = (int)(rem / g.nx), i = (int)(rem - (long long)j * g.nx);
    const int type = DIM == 2 ? 2 * p1_cut(g, j) + l : l;
    double acc = 0.0, wsum = 0.0;
    for (int s = a.soff[type]; s < a.soff[type + 1]; s++) {
      const int4 en = a.ent[s];
      const int ii = i + en.x, jj = j + en.y, kk = k + en.z;
      if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.ny) continue;
      if (DIM == 3 && (kk < 0 || kk >= g.nz)) continue;
      const long long b = NCELL * (ii + (long long)g.nx * (jj + (long long)g.ny * (DIM == 3 ? kk : 0))) + en.w;
      const double wt = a.w[s];
      acc += wt * (a.rho[b] * a.dc[b]);
      wsum += wt;
    }
    a.out[cell] = acc / (a.rho[cell] * wsum);
  }
}

}  // namespace
}  // namespace tp

// ---------------------------------------------------------------------------
// the handle

struct tp_p1_problem {
  tp_p1_params prm;
  cudaStream_t stream = nullptr;
  int dev = 0, nsm = 0;
  tp::P1Shapes sh;
  tp::P1Geo g;
  double* rho = nullptr;
  double* rho_new = nullptr;
  double* E = nullptr;
  double* invd = nullptr;
  uint8_t* fixed = nullptr;
  int8_t* passive = nullptr;
  double* f = nullptr;
  double* x = nullptr;
  double* r = nullptr;
  double* z = nullptr;
  double* p = nullptr;
  double* q = nullptr;
  double* part = nullptr;
  double* ce = nullptr;
  double* dc = nullptr;
  double* dcf = nullptr;
  double* bscr = nullptr;
  int4* sten_ent = nullptr;
  double* sten_w = nullptr;
  int soff[tp::kP1MaxTypes + 1] = {};
  tp::P1Cg* cg = nullptr;
  tp::GridBar* bar = nullptr;
  tp::OcStatus* ost = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<uint8_t> fixed_h;
  std::vector<double> f_h;
  double ff[tp::kMaxCases] = {};
  bool has_fixed = false, has_loads = false, has_density = false, has_u = false, has_dc = false, has_dcf = false;
  bool has_passive = false, E_dirty = true;
  int oc_passes = 0, oc_root = 0;
  long long launches = 0;
  std::string err;
};

namespace {

tp_status p1_fail(tp_p1_problem* p, tp_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

tp_status p1_cuda_fail(tp_p1_problem* p, cudaError_t e, const char* what) {
  cudaGetLastError();
  return p1_fail(p, e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define P1CK(expr, what)                          \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return p1_cuda_fail(p, e_, what); \
  } while (0)

int grid_for(const tp_p1_problem* p, long long n) {
  const long long b = (n + tp::kP1T - 1) / tp::kP1T;
  return (int)std::max<long long>(1, std::min<long long>(b, 2LL * p->nsm));
}

void p1_free(tp_p1_problem* p) {
  void* bufs[] = {p->rho, p->rho_new, p->E, p->invd, p->fixed, p->passive, p->f, p->x, p->r, p->z, p->p, p->q,
                  p->part, p->ce, p->dc, p->dcf, p->bscr, p->sten_ent, p->sten_w, p->cg, p->bar, p->ost};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
}

template <class T>
cudaError_t dalloc(T** ptr, size_t count) {
  return cudaMalloc((void**)ptr, std::max<size_t>(count, 1) * sizeof(T));
}

cudaMemcpyKind kind(int on_device, bool to_device) {
  if (on_device) return cudaMemcpyDeviceToDevice;
  return to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

tp::P1Args apply_args(tp_p1_problem* p, const double* u, double* y, int mode) {
  tp::P1Args a;
  a.sh = p->sh;
  a.g = p->g;
  a.E = p->E;
  a.fixed = p->fixed;
  a.u = u;
  a.y = y;
  a.f = p->f;
  a.part = p->part;
  a.cg = p->cg;
  a.mode = mode;
  return a;
}

cudaError_t launch_apply(tp_p1_problem* p, const double* u, double* y, int mode) {
  const tp::P1Args a = apply_args(p, u, y, mode);
  const dim3 grid(grid_for(p, p->g.nn), p->g.nc);
  if (p->g.dim == 2) tp::p1_apply_kernel<2><<<grid, tp::kP1T, 0, p->stream>>>(a);
  else tp::p1_apply_kernel<3><<<grid, tp::kP1T, 0, p->stream>>>(a);
  p->launches++;
  return cudaGetLastError();
}

tp::P1Vec vec_args(tp_p1_problem* p, unsigned mask) {
  tp::P1Vec v;
  v.ndof = p->g.ndof;
  v.fixed = p->fixed;
  v.invd = p->invd;
  v.x = p->x;
  v.r = p->r;
  v.z = p->z;
  v.p = p->p;
  v.q = p->q;
  v.part = p->part;
  v.cg = p->cg;
  v.mask = mask;
  return v;
}

tp::P1Cell cell_args(tp_p1_problem* p) {
  tp::P1Cell a;
  a.sh = p->sh;
  a.g = p->g;
  a.rho = p->rho;
  a.Emin = p->prm.Emin;
  a.penal = p->prm.penal;
  a.E = p->E;
  a.fixed = p->fixed;
  a.invd = p->invd;
  a.x = p->x;
  a.f = p->f;
  a.ce = p->ce;
  a.dc = p->dc;
  a.part = p->part;
  a.cg = p->cg;
  return a;
}

// Moduli and the Jacobi diagonal after a density change.
tp_status ensure_E(tp_p1_problem* p) {
  if (!p->E_dirty) return TP_OK;
  const int gc = grid_for(p, p->g.ncell);
  tp::p1_young_kernel<<<gc, tp::kP1T, 0, p->stream>>>(p->rho, p->E, p->g.ncell, p->prm.Emin, p->prm.penal);
  P1CK(cudaGetLastError(), "young kernel");
  const tp::P1Cell a = cell_args(p);
  const int gn = grid_for(p, p->g.nn);
  if (p->g.dim == 2) tp::p1_diag_kernel<2><<<gn, tp::kP1T, 0, p->stream>>>(a);
  else tp::p1_diag_kernel<3><<<gn, tp::kP1T, 0, p->stream>>>(a);
  P1CK(cudaGetLastError(), "diagonal kernel");
  p->launches += 2;
  p->E_dirty = false;
  return TP_OK;
}

// r = f - K x, then restart the cases in `mask` from it; copies the CG state to `hs`.
tp_status restart(tp_p1_problem* p, unsigned mask, tp::P1Cg* hs) {
  P1CK(launch_apply(p, p->x, p->r, 2), "residual kernel");
  const tp::P1Vec v = vec_args(p, mask);
  tp::p1_restart_kernel<<<dim3(grid_for(p, p->g.ndof), p->g.nc), tp::kP1T, 0, p->stream>>>(v);
  P1CK(cudaGetLastError(), "restart kernel");
  p->launches++;
  P1CK(cudaMemcpyAsync(hs, p->cg, sizeof(*hs), cudaMemcpyDeviceToHost, p->stream), "copy state");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

}  // namespace

extern "C" {

tp_status tp_p1_create(const tp_p1_params* prm, void* cuda_stream, tp_p1_problem** out) {
  if (!prm || !out) return TP_ERR_ARG;
  *out = nullptr;
  const tp_p1_params& q = *prm;
  if (q.dim != 2 && q.dim != 3) return TP_ERR_ARG;
  if (q.nelx < 1 || q.nely < 1 || (q.dim == 3 ? q.nelz < 1 : q.nelz != 0)) return TP_ERR_ARG;
  if (q.dim == 2 ? (q.diagonal < 0 || q.diagonal > 2) : q.diagonal != 0) return TP_ERR_ARG;
  if (!(q.mu > 0.0) || !(q.lam + 2.0 * q.mu / q.dim > 0.0) || !std::isfinite(q.lam) || !std::isfinite(q.mu))
    return TP_ERR_ARG;
  if (!(q.Emin > 0.0 && q.Emin < 1.0) || !(q.penal >= 1.0 && q.penal <= 10.0)) return TP_ERR_ARG;
  if (!(q.volfrac > 0.0 && q.volfrac <= 1.0) || !(q.rmin > 0.0 && q.rmin <= 4.0)) return TP_ERR_ARG;
  if (!(q.move > 0.0) || !(q.dmin > 0.0 && q.dmin < 1.0)) return TP_ERR_ARG;
  if (q.n_cases < 1 || q.n_cases > tp::kMaxCases) return TP_ERR_ARG;
  const long long nn = (long long)(q.nelx + 1) * (q.nely + 1) * (q.dim == 3 ? q.nelz + 1 : 1);
  const long long ncell = (q.dim == 2 ? 2LL : 6LL) * q.nelx * q.nely * (q.dim == 3 ? q.nelz : 1);
  if (nn * q.dim * q.n_cases > (1LL << 31) - 1 || ncell > (1LL << 31) - 1) return TP_ERR_ARG;

  // midpoint-filter stencil (host)
  const int ntypes = q.dim == 2 ? 4 : 6;
  const int cap = 1 << 16;
  std::vector<int> ent(4 * (size_t)cap);
  std::vector<double> wts(cap);
  int count[tp::kP1MaxTypes] = {};
  const int nent = tp::p1_filter_stencil(q.dim, q.diagonal, q.rmin, cap, count,
                                         reinterpret_cast<int(*)[4]>(ent.data()), wts.data());
  if (nent < 1) return TP_ERR_ARG;

  tp_p1_problem* p = new tp_p1_problem();
  p->prm = q;
  p->stream = (cudaStream_t)cuda_stream;
  tp::p1_shapes(q.dim, q.lam, q.mu, p->sh.K, p->sh.off);
  p->g.dim = q.dim;
  p->g.nx = q.nelx;
  p->g.ny = q.nely;
  p->g.nz = q.dim == 3 ? q.nelz : 0;
  p->g.diag = q.diagonal;
  p->g.nc = q.n_cases;
  p->g.nn = nn;
  p->g.ncell = ncell;
  p->g.ndof = q.dim * nn;
  p->soff[0] = 0;
  for (int t = 0; t < tp::kP1MaxTypes; t++) p->soff[t + 1] = p->soff[t] + (t < ntypes ? count[t] : 0);
  std::vector<int4> ent4(nent);
  for (int i = 0; i < nent; i++) ent4[i] = make_int4(ent[4 * i], ent[4 * i + 1], ent[4 * i + 2], ent[4 * i + 3]);

  const size_t nv = (size_t)p->g.ndof * q.n_cases;
  cudaError_t e = cudaGetDevice(&p->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
  const int maxgrid = 2 * std::max(p->nsm, 1);
  const size_t npart = std::max<size_t>((size_t)tp::oc_part_doubles(maxgrid), (size_t)2 * tp::kMaxCases * maxgrid);
  if (e == cudaSuccess) e = dalloc(&p->rho, ncell);
  if (e == cudaSuccess) e = dalloc(&p->rho_new, ncell);
  if (e == cudaSuccess) e = dalloc(&p->E, ncell);
  if (e == cudaSuccess) e = dalloc(&p->invd, p->g.ndof);
  if (e == cudaSuccess) e = dalloc(&p->fixed, p->g.ndof);
  if (e == cudaSuccess) e = dalloc(&p->passive, ncell);
  if (e == cudaSuccess) e = dalloc(&p->f, nv);
  if (e == cudaSuccess) e = dalloc(&p->x, nv);
  if (e == cudaSuccess) e = dalloc(&p->r, nv);
  if (e == cudaSuccess) e = dalloc(&p->z, nv);
  if (e == cudaSuccess) e = dalloc(&p->p, nv);
  if (e == cudaSuccess) e = dalloc(&p->q, nv);
  if (e == cudaSuccess) e = dalloc(&p->part, npart);
  if (e == cudaSuccess) e = dalloc(&p->ce, ncell);
  if (e == cudaSuccess) e = dalloc(&p->dc, ncell);
  if (e == cudaSuccess) e = dalloc(&p->dcf, ncell);
  if (e == cudaSuccess) e = dalloc(&p->bscr, ncell);
  if (e == cudaSuccess) e = dalloc(&p->sten_ent, nent);
  if (e == cudaSuccess) e = dalloc(&p->sten_w, nent);
  if (e == cudaSuccess) e = dalloc(&p->cg, 1);
  if (e == cudaSuccess) e = dalloc(&p->bar, 1);
  if (e == cudaSuccess) e = dalloc(&p->ost, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->cg, 0, sizeof(tp::P1Cg), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->x, 0, nv * sizeof(double), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->passive, 0, ncell, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->sten_ent, ent4.data(), nent * sizeof(int4), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->sten_w, wts.data(), nent * sizeof(double), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
  if (e != cudaSuccess) {
    const tp_status s = e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
    cudaGetLastError();
    p1_free(p);
    delete p;
    return s;
  }
  *out = p;
  return TP_OK;
}

void tp_p1_destroy(tp_p1_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  p1_free(p);
  delete p;
}

const char* tp_p1_last_error(const tp_p1_problem* p) { return p ? p->err.c_str() : "null problem"; }

long long tp_p1_launch_count(const tp_p1_problem* p) { return p ? p->launches : 0; }

static void p1_update_ff(tp_p1_problem* p) {
  if (!p->has_fixed || !p->has_loads) return;
  for (int c = 0; c < p->g.nc; c++) {
    double s = 0.0;
    for (long long i = 0; i < p->g.ndof; i++)
      if (!p->fixed_h[i]) s += p->f_h[(size_t)c * p->g.ndof + i] * p->f_h[(size_t)c * p->g.ndof + i];
    p->ff[c] = s;
  }
}

tp_status tp_p1_set_fixed(tp_p1_problem* p, const uint8_t* fixed) {
  if (!p || !fixed) return p1_fail(p, TP_ERR_ARG, "null argument");
  p->fixed_h.assign(p->g.ndof, 0);
  long long nfix = 0;
  for (long long i = 0; i < p->g.ndof; i++) {
    p->fixed_h[i] = fixed[i] ? 1 : 0;
    nfix += p->fixed_h[i];
  }
  if (nfix == 0) return p1_fail(p, TP_ERR_ARG, "no fixed DOF: K would be singular");
  P1CK(cudaMemcpyAsync(p->fixed, p->fixed_h.data(), p->g.ndof, cudaMemcpyHostToDevice, p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  p->has_fixed = true;
  p->E_dirty = true;
  p1_update_ff(p);
  return TP_OK;
}

tp_status tp_p1_set_loads(tp_p1_problem* p, const double* f) {
  if (!p || !f) return p1_fail(p, TP_ERR_ARG, "null argument");
  const size_t nv = (size_t)p->g.ndof * p->g.nc;
  for (size_t i = 0; i < nv; i++)
    if (!std::isfinite(f[i])) return p1_fail(p, TP_ERR_ARG, "non-finite load");
  p->f_h.assign(f, f + nv);
  P1CK(cudaMemcpyAsync(p->f, p->f_h.data(), nv * sizeof(double), cudaMemcpyHostToDevice, p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  p->has_loads = true;
  p1_update_ff(p);
  return TP_OK;
}

tp_status tp_p1_set_passive(tp_p1_problem* p, const int8_t* passive) {
  if (!p || !passive) return p1_fail(p, TP_ERR_ARG, "null argument");
  std::vector<int8_t> m(p->g.ncell);
  bool any = false;
  for (long long i = 0; i < p->g.ncell; i++) {
    m[i] = passive[i] ? 1 : 0;
    any |= m[i] != 0;
  }
  P1CK(cudaMemcpyAsync(p->passive, m.data(), p->g.ncell, cudaMemcpyHostToDevice, p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  p->has_passive = any;
  return TP_OK;
}

tp_status tp_p1_set_density(tp_p1_problem* p, const double* rho, int on_device) {
  if (!p || !rho) return p1_fail(p, TP_ERR_ARG, "null argument");
  std::vector<double> h;
  const double* src = rho;
  if (on_device) {
    h.resize(p->g.ncell);
    P1CK(cudaMemcpyAsync(h.data(), rho, p->g.ncell * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
    P1CK(cudaStreamSynchronize(p->stream), "sync");
    src = h.data();
  }
  for (long long i = 0; i < p->g.ncell; i++)
    if (!(src[i] > 0.0 && src[i] <= 1.0)) return p1_fail(p, TP_ERR_ARG, "densities must lie in (0, 1]");
  P1CK(cudaMemcpyAsync(p->rho, rho, p->g.ncell * sizeof(double), kind(on_device, true), p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  p->has_density = true;
  p->E_dirty = true;
  p->has_dc = p->has_dcf = false;
  return TP_OK;
}

tp_status tp_p1_apply(tp_p1_problem* p, const double* u, double* y, int on_device) {
  if (!p || !u || !y) return p1_fail(p, TP_ERR_ARG, "null argument");
  if (!p->has_fixed || !p->has_density) return p1_fail(p, TP_ERR_STATE, "fixed DOFs and densities must be set");
  const tp_status st = ensure_E(p);
  if (st != TP_OK) return st;
  const size_t nv = (size_t)p->g.ndof * p->g.nc;
  if (on_device) {
    P1CK(launch_apply(p, u, y, 0), "apply kernel");
    return TP_OK;
  }
  P1CK(cudaMemcpyAsync(p->r, u, nv * sizeof(double), cudaMemcpyHostToDevice, p->stream), "copy");
  P1CK(launch_apply(p, p->r, p->q, 0), "apply kernel");
  P1CK(cudaMemcpyAsync(y, p->q, nv * sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_p1_solve(tp_p1_problem* p, const tp_solve_opts* opts, tp_solve_info* info) {
  if (!p || !opts) return p1_fail(p, TP_ERR_ARG, "null argument");
  if (!p->has_fixed || !p->has_loads || !p->has_density)
    return p1_fail(p, TP_ERR_STATE, "fixed DOFs, loads and densities must be set before tp_p1_solve");
  if (!(opts->tol > 0.0) || opts->max_it < 1) return p1_fail(p, TP_ERR_ARG, "tol > 0 and max_it >= 1 required");
  if (opts->precision != TP_PREC_F64 || opts->precond != TP_PRECOND_JACOBI)
    return p1_fail(p, TP_ERR_ARG, "the P1 solve is FP64 Jacobi-PCG (TP_PREC_F64, TP_PRECOND_JACOBI)");
  for (int c = 0; c < p->g.nc; c++)
    if (!(p->ff[c] > 0.0)) return p1_fail(p, TP_ERR_ARG, "a load case has no load on a free DOF");
  tp_status st = ensure_E(p);
  if (st != TP_OK) return st;
  const int nc = p->g.nc;
  const size_t nv = (size_t)p->g.ndof * nc;
  if (opts->warm_start == TP_WARM_ZERO || (opts->warm_start == TP_WARM_PREVIOUS && !p->has_u))
    P1CK(cudaMemsetAsync(p->x, 0, nv * sizeof(double), p->stream), "memset");
  tp::P1Cg hs;
  memset(&hs, 0, sizeof(hs));
  for (int c = 0; c < nc; c++) hs.tol2ff[c] = opts->tol * opts->tol * p->ff[c];
  P1CK(cudaMemcpyAsync(p->cg, &hs, sizeof(hs), cudaMemcpyHostToDevice, p->stream), "copy state");
  P1CK(cudaEventRecord(p->ev0, p->stream), "event");
  const unsigned all = (1u << nc) - 1u;
  st = restart(p, all, &hs);
  if (st != TP_OK) return st;
  double rel0[tp::kMaxCases] = {};
  for (int c = 0; c < nc; c++) rel0[c] = std::sqrt(hs.rr[c] / p->ff[c]);
  double rr_true[tp::kMaxCases];
  for (int c = 0; c < nc; c++) rr_true[c] = hs.rr[c];
  const tp::P1Vec v = vec_args(p, 0);
  const dim3 gv(grid_for(p, p->g.ndof), nc);
  int iters = 0, restarts = 0;
  bool stagnated = false;
  const int chunk = 16;
  for (;;) {
    bool active = false;
    for (int c = 0; c < nc; c++) active |= hs.state[c] == 0;
    if (!active) {
      // every case stopped: confirm the recurrence by the true residual
      unsigned mask = 0;
      for (int c = 0; c < nc; c++)
        if (hs.state[c] == 1) mask |= 1u << c;
      if (!mask) break;
      st = restart(p, mask, &hs);
      if (st != TP_OK) return st;
      bool reopened = false;
      for (int c = 0; c < nc; c++)
        if ((mask >> c) & 1u) {
          rr_true[c] = hs.rr[c];
          reopened |= hs.state[c] == 0;
        }
      if (!reopened) break;
      if (++restarts > 50) {
        stagnated = true;
        break;
      }
      continue;
    }
    if (iters >= opts->max_it) break;
    const int n = std::min(chunk, opts->max_it - iters);
    for (int k = 0; k < n; k++) {
      P1CK(launch_apply(p, p->p, p->q, 1), "CG operator kernel");
      tp::p1_update_kernel<<<gv, tp::kP1T, 0, p->stream>>>(v);
      P1CK(cudaGetLastError(), "CG update kernel");
      tp::p1_direction_kernel<<<gv, tp::kP1T, 0, p->stream>>>(v);
      P1CK(cudaGetLastError(), "CG direction kernel");
      p->launches += 2;
    }
    P1CK(cudaMemcpyAsync(&hs, p->cg, sizeof(hs), cudaMemcpyDeviceToHost, p->stream), "copy state");
    P1CK(cudaStreamSynchronize(p->stream), "sync");
    iters = 0;
    for (int c = 0; c < nc; c++) iters = std::max(iters, hs.it[c]);
  }
  // final true residual of every case that did not break down
  unsigned mask = 0;
  for (int c = 0; c < nc; c++)
    if (hs.state[c] != 2) mask |= 1u << c;
  if (mask) {
    st = restart(p, mask, &hs);
    if (st != TP_OK) return st;
    for (int c = 0; c < nc; c++)
      if ((mask >> c) & 1u) rr_true[c] = hs.rr[c];
  }
  P1CK(cudaEventRecord(p->ev1, p->stream), "event");
  P1CK(cudaEventSynchronize(p->ev1), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  bool conv = true, brk = false;
  for (int c = 0; c < nc; c++) {
    conv &= hs.state[c] == 1;
    brk |= hs.state[c] == 2;
  }
  p->has_u = true;
  p->has_dc = p->has_dcf = false;
  tp_status rs = brk ? TP_ERR_BREAKDOWN : (conv && !stagnated ? TP_OK : TP_ERR_NOT_CONVERGED);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = iters;
    info->updates = restarts;
    info->converged = rs == TP_OK ? 1 : 0;
    info->status = rs;
    for (int c = 0; c < nc; c++) {
      info->rel_res[c] = std::sqrt(rr_true[c] / p->ff[c]);
      info->rel_res_init[c] = rel0[c];
    }
    info->ms = ms;
  }
  if (rs == TP_ERR_BREAKDOWN) return p1_fail(p, rs, "CG breakdown (p^T K p <= 0 or not finite)");
  if (rs == TP_ERR_NOT_CONVERGED) return p1_fail(p, rs, "CG stopped before the tolerance");
  return TP_OK;
}

tp_status tp_p1_sensitivities(tp_p1_problem* p, double* compliance) {
  if (!p) return TP_ERR_ARG;
  if (!p->has_u) return p1_fail(p, TP_ERR_STATE, "tp_p1_solve must precede tp_p1_sensitivities");
  const tp::P1Cell a = cell_args(p);
  const int gc = grid_for(p, p->g.ncell);
  if (p->g.dim == 2) tp::p1_sens_kernel<2><<<gc, tp::kP1T, 0, p->stream>>>(a);
  else tp::p1_sens_kernel<3><<<gc, tp::kP1T, 0, p->stream>>>(a);
  P1CK(cudaGetLastError(), "sensitivity kernel");
  tp::p1_compliance_kernel<<<dim3(grid_for(p, p->g.ndof), p->g.nc), tp::kP1T, 0, p->stream>>>(a);
  P1CK(cudaGetLastError(), "compliance kernel");
  p->launches += 2;
  tp::P1Cg hs;
  P1CK(cudaMemcpyAsync(&hs, p->cg, sizeof(hs), cudaMemcpyDeviceToHost, p->stream), "copy state");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  double c = 0.0;
  for (int k = 0; k < p->g.nc; k++) c += hs.comp[k];
  if (compliance) *compliance = c;
  p->has_dc = true;
  p->has_dcf = false;
  return TP_OK;
}

tp_status tp_p1_filter(tp_p1_problem* p) {
  if (!p) return TP_ERR_ARG;
  if (!p->has_dc) return p1_fail(p, TP_ERR_STATE, "tp_p1_sensitivities (or tp_p1_set(TP_DC)) must precede tp_p1_filter");
  tp::P1Filt a;
  a.g = p->g;
  a.ent = p->sten_ent;
  a.w = p->sten_w;
  for (int t = 0; t <= tp::kP1MaxTypes; t++) a.soff[t] = p->soff[t];
  a.rho = p->rho;
  a.dc = p->dc;
  a.out = p->dcf;
  const int gc = grid_for(p, p->g.ncell);
  if (p->g.dim == 2) tp::p1_filter_kernel<2><<<gc, tp::kP1T, 0, p->stream>>>(a);
  else tp::p1_filter_kernel<3><<<gc, tp::kP1T, 0, p->stream>>>(a);
  P1CK(cudaGetLastError(), "filter kernel");
  p->launches++;
  p->has_dcf = true;
  return TP_OK;
}

tp_status tp_p1_oc_update(tp_p1_problem* p, double* lambda, double* volume, double* change) {
  if (!p) return TP_ERR_ARG;
  if (!p->has_dcf) return p1_fail(p, TP_ERR_STATE, "tp_p1_filter (or tp_p1_set(TP_DCF)) must precede tp_p1_oc_update");
  P1CK(cudaMemsetAsync(p->bar, 0, sizeof(tp::GridBar), p->stream), "memset");
  int grid = 0;
  P1CK(tp::launch_oc(p->stream, p->g.ncell, p->rho, p->dcf, p->has_passive ? p->passive : nullptr, p->prm.volfrac,
                     p->prm.move, p->prm.dmin, p->rho_new, p->bscr, p->part, p->bar, p->ost, p->nsm, &grid,
                     2 * p->nsm),
       "oc kernel");
  p->launches++;
  tp::OcStatus st;
  P1CK(cudaMemcpyAsync(&st, p->ost, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "copy status");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  if (st.flags & tp::ERR_TIMEOUT) return p1_fail(p, TP_ERR_TIMEOUT, "a device-side wait timed out in the OC kernel");
  if (st.flags & tp::ERR_NAN) return p1_fail(p, TP_ERR_ARG, "no multiplier bracket found (non-finite sensitivities?)");
  std::swap(p->rho, p->rho_new);
  p->E_dirty = true;
  p->has_dc = p->has_dcf = false;
  if (lambda) *lambda = st.lambda;
  if (volume) *volume = st.volume;
  if (change) *change = st.change;
  p->oc_passes = st.passes;
  p->oc_root = st.root;
  return TP_OK;
}

tp_status tp_p1_simp_step(tp_p1_problem* p, const tp_solve_opts* opts, tp_step_info* info) {
  if (!p || !opts) return p1_fail(p, TP_ERR_ARG, "null argument");
  tp_step_info loc;
  memset(&loc, 0, sizeof(loc));
  tp_status st = tp_p1_solve(p, opts, &loc.solve);
  if (st == TP_OK) st = tp_p1_sensitivities(p, &loc.compliance);
  if (st == TP_OK) st = tp_p1_filter(p);
  if (st == TP_OK) st = tp_p1_oc_update(p, &loc.lambda, &loc.volume, &loc.change);
  loc.oc_passes = p->oc_passes;
  loc.oc_root = p->oc_root;
  if (info) *info = loc;
  return st;
}

tp_status tp_p1_get(tp_p1_problem* p, int what, void* dst, int on_device) {
  if (!p || !dst) return p1_fail(p, TP_ERR_ARG, "null argument");
  const double* src = nullptr;
  size_t n = (size_t)p->g.ncell;
  switch (what) {
    case TP_RHO:
    case TP_RHO_PHYS: src = p->rho; break;
    case TP_U: src = p->x; n = (size_t)p->g.ndof * p->g.nc; break;
    case TP_DC: src = p->dc; break;
    case TP_DCF: src = p->dcf; break;
    case TP_CE: src = p->ce; break;
    default: return p1_fail(p, TP_ERR_ARG, "unknown quantity");
  }
  P1CK(cudaMemcpyAsync(dst, src, n * sizeof(double), kind(on_device, false), p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_p1_set(tp_p1_problem* p, int what, const void* src, int on_device) {
  if (!p || !src) return p1_fail(p, TP_ERR_ARG, "null argument");
  double* dst = nullptr;
  size_t n = (size_t)p->g.ncell;
  switch (what) {
    case TP_U: dst = p->x; n = (size_t)p->g.ndof * p->g.nc; break;
    case TP_DC: dst = p->dc; break;
    case TP_DCF: dst = p->dcf; break;
    default: return p1_fail(p, TP_ERR_ARG, "TP_U, TP_DC or TP_DCF expected");
  }
  P1CK(cudaMemcpyAsync(dst, src, n * sizeof(double), kind(on_device, true), p->stream), "copy");
  P1CK(cudaStreamSynchronize(p->stream), "sync");
  if (what == TP_U) {
    p->has_u = true;
    p->has_dc = p->has_dcf = false;
  } else if (what == TP_DC) {
    p->has_dc = true;
    p->has_dcf = false;
  } else {
    p->has_dcf = true;
  }
  return TP_OK;
}

}  // extern "C"
