// Internal host-side interface between the C-ABI (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tp {

struct MgCtl;

constexpr int kMaxCases = 8;
constexpr int kMaxTaps = 512;

// Element stiffness (host, FP64) and filter stencil.
void element_k0(int dim, double nu, double* K);
int filter_taps(int dim, double rmin, int max_taps, int* off, double* wts);
// K0 = G^T C G with generalised strains G (5 rows in 2D, 18 in 3D); returns the row count.
int element_strain_C(int dim, const double* K0, double* C, double* recon_err);

// CG state kept in device memory between the persistent CG segments and the
// FP64 true-residual updates.
struct CgState {
  int it;        // CG iterations so far
  int pbuf;      // which of the two direction buffers holds the current p
  int need;      // segment ended because an update is due
  int flags;     // ERR_* bits
  int updates;   // FP64 true-residual evaluations
  int state[kMaxCases];  // 0 = active, 1 = converged, 2 = breakdown, 3 = stagnated
  int stall[kMaxCases];
  double rz[kMaxCases];       // r.z of the current residual
  double rr_ref[kMaxCases];   // true ||r||^2 at the last update
  double beta[kMaxCases];     // next direction update coefficient
  double rr_true[kMaxCases];  // last true ||f - K u||^2
};

struct Solver {
  Grid g;
  int nc;
  int zlen;              // 3D streaming tile depth (planes per tile)
  const void* E;         // operator moduli in the CG precision
  const double* E64;     // FP64 moduli for the true residual
  const uint8_t* mask;   // per-node fixed bits
  const void* invdiag;   // per DOF, CG precision
  const double* f;       // internal layout [node][case][comp]
  double* x64;
  void* xl;
  void* r;
  void* z;
  void* p0;
  void* p1;
  void* q;
  double* part;          // per-CTA / per-tile partial sums
  double* tol2ff_dev;    // device copy of tol^2 ||f_c||^2
  GridBar* bar;
  CgState* cs;
  double tol2ff[kMaxCases];
  double drop2;
  int max_it;
  const double* C;       // generalised-strain matrix (host, FP64), 5x5 or 18x18
  long long* trace;      // optional per-iteration phase timestamps (device), or null
};

// Launchers (return cudaError_t of the launch).
cudaError_t launch_young(cudaStream_t s, const double* rho, float* E32, double* E64, long long ne,
                         double E0, double Emin, double penal);
cudaError_t launch_diag(cudaStream_t s, const Grid& g, const double* K0, const double* E64,
                        const uint8_t* mask, float* inv32, double* inv64);
cudaError_t launch_matvec(cudaStream_t s, const Grid& g, const double* C, bool f64, const void* E,
                          const uint8_t* mask, const void* u, void* y, int ncopies, int zlen,
                          const int* stop = nullptr);
// The same operator in double-word FP32 arithmetic: u, y double; Edw the moduli
// as double-words (launch_dw_moduli converts E64).
cudaError_t launch_dw_moduli(cudaStream_t s, const double* E64, void* Edw, long long ne);
cudaError_t launch_matvec_dw(cudaStream_t s, const Grid& g, const double* C, const void* Edw, const uint8_t* mask,
                             const double* u, double* y, int ncopies, int zlen, const int* stop = nullptr);
// Multigrid finest-level sweep on the FP32 operator (mode 1: smoothing step
// y = ca u + cc w + om D^-1 (b - K u), w optional and y may alias w; mode 2:
// residual y = b - K u; 0 on fixed DOFs), ncopies vectors of stride n_dof;
// returns at once when *stop is set.
cudaError_t launch_mg_sweep(cudaStream_t s, const Grid& g, const double* C, const float* E, const uint8_t* mask,
                            const float* invd, const float* u, const float* w, const float* b, float* y,
                            int ncopies, int zlen, int mode, float ca, float cc, float om, const int* stop,
                            int dots = -1, double* part = nullptr, MgCtl* ctl = nullptr);
// The FP32 3D operator q = K p with p.q formed in its epilogue and completed
// as the PCG scalar step `what` (pcg_dots_complete).
cudaError_t launch_matvec_dots(cudaStream_t s, const Grid& g, const double* C, const float* E32, const uint8_t* mask,
                               const float* u, float* y, int ncopies, int zlen, const int* stop, double* part,
                               MgCtl* ctl, int what);
// FP64 update: x64 += x_l, x_l = 0; r = f - K64 x64; z = D^-1 r; CgState update.
// `init` starts a solve (beta = 0, counters reset).  Returns the number of
// kernels launched through *nlaunch.
cudaError_t launch_true_residual(cudaStream_t s, const Solver& S, bool f64, bool init, int* nlaunch);
// One persistent CG segment (cooperative launch).
cudaError_t launch_cg_segment(cudaStream_t s, const Solver& S, bool f64, int nsm, int* grid_out);
cudaError_t launch_sens(cudaStream_t s, const Grid& g, int nc, const double* C, const double* x64,
                        const double* f, const double* rho, double penal, double dE, double* ce,
                        double* dc, double* part, double* out_c);
cudaError_t launch_to_internal(cudaStream_t s, const double* src, double* dst, long long nn, int dim,
                               int nc, const uint8_t* mask, int zero_fixed);
cudaError_t launch_to_abi(cudaStream_t s, const double* src, double* dst, long long nn, int dim, int nc);

// Filter / OC (opt_kernels.cu).
struct FilterLaunch {
  Grid g;
  int ntaps;
  int off[3 * kMaxTaps];
  double w[kMaxTaps];
};
cudaError_t launch_filter(cudaStream_t s, const FilterLaunch& F, int mode, const double* rho,
                          const double* dc, double* out);
// Helmholtz (PDE) filter (helm.cu): out = T^T (R^2 K_F + M_F)^-1 T in, element
// values in and out.  a[4]: element-matrix entries by corner Hamming distance
// (helm_coefficients); scratch: helm_scratch_doubles(g) doubles, whose last n_nodes
// hold the inverse diagonal written by launch_helm_setup.  The nodal solve is
// Jacobi-PCG in FP64 to relative residual tol (a persistent cooperative kernel;
// zeroes the barrier word); st receives iterations, residual and error bits.
struct HelmStatus {
  int it;
  int flags;
  double rel;
};
void helm_coefficients(int dim, double R, double* a);
size_t helm_scratch_doubles(const Grid& g);
cudaError_t launch_helm_setup(cudaStream_t s, const Grid& g, const double* a, double* scratch);
cudaError_t launch_helm_filter(cudaStream_t s, const Grid& g, const double* a, const double* in, double* out,
                               double* scratch, double* part, GridBar* bar, HelmStatus* st, double tol, int max_it,
                               int nsm);

struct OcStatus {
  double lambda;
  double volume;
  double change;
  int passes;
  int flags;
  int root;  // 1 closed form, 2 piecewise exact root, 0 bisection midpoint
  int pad;
};
cudaError_t launch_oc(cudaStream_t s, long long ne, const double* rho, const double* dcf,
                      const int8_t* passive, double volfrac, double move, double dmin,
                      double* rho_new, double* bscratch, double* part, GridBar* bar, OcStatus* st,
                      int nsm, int* grid_out, int max_grid = 0);
// Partial-sum slots the OC kernel needs for `grid` CTAs (doubles).
// partial sums of the OC kernel (two slots of 15 values and the final 2 per
// CTA), then the list of elements that change clamp state inside the final
// bracket (a counter and 32 entries of 3 doubles)
constexpr long long oc_part_doubles(int grid) { return (long long)(2 * 15 + 2) * grid + 1 + 32 * 3; }

}  // namespace tp
