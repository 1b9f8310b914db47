// Private: geometric multigrid preconditioner (mg.cu) and the FP64 outer-PCG
// vector kernels used with it (api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "strain.cuh"

namespace tp {

struct MgLevel {
  Grid g;
  int f = 1;                // coarsening factor from the finer level
  float* K = nullptr;       // element matrices [ne][ND][ND] (null on level 0: E_e K0)
  float* S = nullptr;       // assembled per-node coupling blocks (null: apply element by element)
  uint8_t* mask = nullptr;  // per-node fixed bits
  bool mask_own = false;
  float* invd = nullptr;    // inverse l1 row sums [n_nodes * dim]
  float* x[2] = {nullptr, nullptr};  // iterates [case][n_nodes * dim]
  float* b = nullptr;       // right-hand side
  float* t = nullptr;       // residual scratch
  float* t2 = nullptr;      // A u on the finest level
};

struct MgHierarchy {
  std::vector<MgLevel> lv;
  int nc = 1, cn = 0;       // cases, DOFs of the coarsest level
  float* cinv = nullptr;    // coarsest dense inverse [cn][cn]
  float* K0d = nullptr;     // level-0 element matrix (unit modulus), device copy
  const float* E0 = nullptr;
  // finest-level operator y = A u for all cases (the library's FP32 operator)
  cudaError_t (*fine_op_fn)(void* ctx, cudaStream_t s, const float* u, float* y) = nullptr;
  void* fine_ctx = nullptr;
  cudaError_t fine_op(cudaStream_t s, const float* u, float* y) const { return fine_op_fn(fine_ctx, s, u, y); }
  float omega = 1.6f;       // l1-Jacobi weight (convergent for any weight below 2)
  int nu = 2;               // sweeps before and after the coarse correction
  bool built = false;
  long long version = -1;   // moduli version the operators were built for
  // optional timing of the finest level's operator launches (event pairs)
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  long long timed_launches = 0;
  double timed_ms = 0.0;
  double fine_bytes() const;  // algorithmic bytes of one finest-level sweep launch
  void collect_timing();      // after the stream has synchronised

  // Level plan for grid g0: 2:1 while possible, then the smallest common odd
  // factor, until the coarsest has <= max_coarse_dofs DOFs.  Allocates all
  // buffers.  cudaErrorInvalidValue when no plan reaches <= 4096 coarse DOFs.
  cudaError_t plan(const Grid& g0, const uint8_t* mask0, int nc, int max_coarse_dofs = 256);
  // Galerkin coarse operators, diagonals and the coarsest inverse for moduli E32.
  cudaError_t build(cudaStream_t s, const double* K0, const float* E32, int* nlaunch);
  // x = V(b) on level li (x starts at zero); input lv[li].b, output lv[li].x[0].
  cudaError_t vcycle(cudaStream_t s, int li, int* nlaunch);
  void release();
  ~MgHierarchy() { release(); }
};

// FP64 vector kernels of the outer PCG (ABI layout, nc cases of n values).
// sc (device): [0,8) alpha, [8,16) beta, [16,24) rz, [24,32) pq / rz_new, [32,40) rr.
cudaError_t pcg_dot2(cudaStream_t s, long long n, int nc, const double* a1, const double* b1, const double* a2,
                     const double* b2, double* part, int* nblocks);
// what 0: pq = <p,q> -> alpha = rz / pq;  what 1: rz_new, rr -> beta = rz_new / rz, rz = rz_new;
// what 2: rz, rr (start)
cudaError_t pcg_scalars(cudaStream_t s, int nblocks, int nc, const double* part, int what, double* sc);
cudaError_t pcg_update_xr(cudaStream_t s, long long n, int nc, const double* sc, double* x, const double* p, double* r,
                          const double* q);
cudaError_t pcg_update_p(cudaStream_t s, long long n, int nc, const double* sc, double* p, const double* z);
cudaError_t pcg_residual(cudaStream_t s, long long n, int nc, const double* f, const double* Ax, const uint8_t* mask,
                         int dim, double* r);
cudaError_t to_f32(cudaStream_t s, long long n, const double* a, float* b);
cudaError_t to_f64(cudaStream_t s, long long n, const float* a, double* b);

}  // namespace tp
