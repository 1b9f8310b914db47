// Private: the problem handle behind the C-ABI, shared by api.cu and warm.cu.
#pragma once
#include <string>
#include <vector>

#include "../../include/topo.h"
#include "host.h"
#include "mg.h"

struct tp_problem {
  using FilterLaunch = tp::FilterLaunch;
  using Grid = tp::Grid;
  using GridBar = tp::GridBar;
  using CgState = tp::CgState;
  using OcStatus = tp::OcStatus;
  static constexpr int kMaxCases = tp::kMaxCases;
  tp_params prm;
  cudaStream_t stream = nullptr;
  int dev = 0, nsm = 0;
  Grid g;
  long long nn = 0, ne = 0, ndof = 0;
  int nc = 1, dim = 2, nv = 2;
  std::vector<double> K0;
  std::vector<double> C;  // generalised-strain matrix (K0 = G^T C G)
  int zlen = 16;          // 3D streaming tile depth (planes per tile, balanced)
  FilterLaunch* flt = nullptr;

  double* rho = nullptr;
  double* rho_new = nullptr;
  float* E32 = nullptr;
  double* E64 = nullptr;
  uint8_t* mask = nullptr;
  int8_t* passive = nullptr;
  double* f = nullptr;
  double* x64 = nullptr;
  float* inv32 = nullptr;
  double* inv64 = nullptr;
  void* w[6] = {};  // xl, r, z, p0, p1, q (sized for double)
  double* part = nullptr;
  GridBar* bar = nullptr;
  CgState* cgs = nullptr;
  double* tol2 = nullptr;
  OcStatus* ost = nullptr;
  long long* trace = nullptr;  // CG phase timestamps (when enabled)
  double* scal = nullptr;
  double* dc = nullptr;
  double* dcf = nullptr;
  double* ce = nullptr;
  double* bscr = nullptr;
  double* abi = nullptr;

  bool has_fixed = false, has_loads = false, has_density = false, has_u = false;
  bool has_dc = false, has_dcf = false, E_dirty = true, has_passive = false;
  double ff[kMaxCases] = {};
  std::string err;
  long long launches = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int last_grid = 0;
  tp::MgHierarchy* mg = nullptr; // multigrid preconditioner (built on first use)
  long long E_version = 0;       // bumped whenever the moduli are recomputed
  long long diag_version = -1;   // moduli version of inv32 / inv64 (the Jacobi scaling)
  void* Edw = nullptr;           // moduli as double-words (float pairs), formed on first use
  long long dw_version = -1;     // moduli version of Edw
  bool profile = false;          // time the multigrid finest-level launches
  int filter_mode = 0;           // TP_FILTER_SENSITIVITY or TP_FILTER_DENSITY
  int oc_passes = 0, oc_root = 0;  // diagnostics of the last OC update
  unsigned wait_budget = 0;      // grid-barrier wait limit in cycles (0 = default, ~1 s)
  double* rho_phys = nullptr;    // filtered densities (filter modes 1, 2)
  double* helm = nullptr;        // Helmholtz filter scratch (filter mode 2)
  tp::HelmStatus* hst = nullptr;
  double helm_a[4] = {};         // its element-matrix entries
  double* rowsum = nullptr;      // sum_b W_ab per element (filter mode 1)
  double fmax[kMaxCases] = {};   // max |f| per load case (warm-start feature scale)
  // learned warm start scratch (allocated on first use)
  void* nn_feat = nullptr;       // bf16 [n_cases][8][nelz][nely][nelx]
  float* nn_out = nullptr;       // f32 [n_cases][3][nelz][nely][nelx]
  double* nn_scal = nullptr;     // per-case alpha and dot products
};

// Recompute the moduli and the Jacobi diagonal if the densities changed.
tp_status tp_problem_ensure_E(tp_problem* p);
