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
  float* r4 = nullptr;      // 3D f = 4: partial restriction sums [case][fine z][coarse y][coarse x][dim]
};

// Device control block of the multigrid PCG.  The scalar kernels keep the
// per-case CG scalars here and, after each iteration, decide on the device
// whether the segment stops; every kernel of an iteration returns at once
// when `stop` is set, so a CUDA graph of several iterations can run past the
// stopping point without changing the iterate.
struct MgCtl {
  double sc[64];       // [0,8) alpha, [8,16) beta, [16,24) rz, [24,32) pq, [32,40) rr
  double rr_start[8];  // rr at the segment start
  double ff[8];        // ||f_c||^2
  double best;         // worst relative rr at its last halving
  double tol2;         // tol^2
  int it;              // iterations of the segment so far
  int best_it;         // iteration of `best`
  int it_limit;        // iterations allowed in the segment
  int stop;            // 0: run, 1: stop (every later kernel of the segment returns)
  int reason;          // MG_STOP_* bits
  int use64;           // FP64 operator (the FP32-accuracy rule does not apply)
  int nc;
  int timeout;         // set by the persistent kernel when a grid barrier timed out
  unsigned ticket;     // last-block counter of the fused dot/scalar kernel (0 between launches)
};
enum : int { MG_STOP_DONE = 1, MG_STOP_INNER = 2, MG_STOP_STALL = 4, MG_STOP_BREAK = 8, MG_STOP_LIMIT = 16 };

// Runs the dense inversion (mg_dense.cu) as one CUDA graph: the launches
// are captured once per (matrix, operands, scratch, size) on the private
// stream `cap`, with the second stream `side` and the two events giving the
// look-ahead its fork and join, and each later call replays the graph on the
// caller's stream (several hundred launches for one host call).
struct DenseInverter {
  cudaStream_t side = nullptr, cap = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key[5] = {};
  int key_n = 0, launches = 0;
  cudaError_t create();
  void destroy();
};

struct MgHierarchy {
  std::vector<MgLevel> lv;
  int nc = 1, cn = 0;       // cases, DOFs of the coarsest level
  float* cinv = nullptr;    // coarsest dense inverse [cn][cn] (FP32)
  float* dscratch = nullptr;  // panels of the dense inversion
  int* dflag = nullptr;       // set when a pivot of the dense inversion is not positive
  DenseInverter dinv;
  bool coarse_ok = true;      // the last build's dense inversion met only positive pivots
  float* K0d = nullptr;     // level-0 element matrix (unit modulus), device copy
  float* A1 = nullptr;      // level-1 child matrices P_ch^T K0 P_ch [f^dim][ND][ND] (unmasked)
  uint8_t* touched1 = nullptr;  // level-1 elements whose footprint holds a fixed fine DOF
  int* touched_list = nullptr;  // those elements (entries after the count: touched_list[0] = count)
  const float* E0 = nullptr;
  // Finest-level sweep for all cases on the library's strain-form FP32
  // operator: mode 1 y = a u + c w + om D^-1 (b - A u) (w may be null when
  // c = 0; y may alias w), mode 2 y = b - A u; 0 on fixed DOFs; returns at
  // once when *stop is set.
  // With dots >= 0 the sweep also forms r.z and r.r (b is the finest r, y = z)
  // and completes them as the PCG scalar step `dots` (pcg_dots_complete).
  cudaError_t (*fine_op_fn)(void* ctx, cudaStream_t s, const float* u, const float* w, const float* b,
                            const float* invd, float* y, int mode, float a, float c, float om,
                            const int* stop, int dots) = nullptr;
  void* fine_ctx = nullptr;
  // the PCG scalar step that the V-cycle's last finest-level step completes
  // (-1: none; the caller then launches the dot kernel)
  int fine_dots = -1;
  MgCtl* ctl = nullptr;     // device control block
  MgCtl* ctl_h = nullptr;   // pinned host mirror
  float* p32 = nullptr;     // FP32 search direction (finest level, all cases)
  float* q32 = nullptr;     // FP32 K p
  float* d32 = nullptr;     // FP32 correction of the current segment
  float* p32b = nullptr;    // second FP32 search-direction buffer (persistent kernel)
  // CUDA graphs of kGraphIters PCG iterations, [FP64 operator][timed]
  static constexpr int kGraphIters = 8;
  cudaGraphExec_t gx[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int gx_launches[2][2] = {{0, 0}, {0, 0}};
  cudaStream_t cap = nullptr;   // capture stream of the graphs
  // second stream of a solve that rebuilds the hierarchy: the first FP64
  // residual runs there while the build runs on the problem's stream
  cudaStream_t side = nullptr;
  std::vector<float> k0abs;  // host copy of the l1 row sums of K0 (the source of an async upload)
  cudaEvent_t fork = nullptr, join = nullptr;
  // Smoother: Chebyshev iteration of degree nu on D_l1^-1 A, whose spectrum
  // lies in (0, 1] (l1 row sums), for the interval [1 / cheb_ratio, 1].
  // Step 1 from x: x + omega D^-1 (b - A x); step k >= 2 (x_k from x_{k-1}, x_{k-2}):
  //   x_k = ca[k] x_{k-1} + cc[k] x_{k-2} + cw[k] D^-1 (b - A x_{k-1}).
  // The same polynomial before and after the coarse correction keeps the
  // V-cycle symmetric.
  int nu = 2;
  // Degree on the finest level: 1 when it holds more than kDegree1Nodes nodes,
  // kDegree1Nodes3D in 3D (then its sweeps dominate an iteration: at
  // 240 x 80 x 80 degree 1 took 29.3 ms per SIMP step against 33.5 ms, the
  // extra iterations outweighed by two fewer finest sweeps per iteration).  In
  // 3D the finest level is scaled by the assembled operator's l1 row sums, which
  // make one step a stronger smoother: at 120 x 40 x 40 degree 1 then took
  // 9.04 ms against 9.18 ms (it was 2 % slower with the element-level sums).
  int nu0 = 2;
  static constexpr long long kDegree1Nodes = 1000000, kDegree1Nodes3D = 100000;
  int degree_at(int li) const { return li == 0 ? nu0 : nu; }
  float cheb_ratio = 60.f;
  float omega = 0.f;
  float ca[8] = {}, cc[8] = {}, cw[8] = {};
  void set_smoother(int degree, float ratio);
  bool built = false;
  long long version = -1;   // moduli version the operators were built for
  // Optional timing (profiling aid): the persistent segment launches (an
  // event pair each), or in the graph path the finest-level sweeps (event
  // nodes captured into the timed graph, read after each replay).
  bool timing = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> sweep_ev;
  int ev_used = 0;
  bool capture_events = false;
  long long timed_launches = 0;
  double timed_ms = 0.0, timed_bytes = 0.0;
  double fine_bytes() const;          // algorithmic bytes of one finest-level sweep launch
  void collect_sweeps(int npairs);    // the first npairs sweep event pairs (stream synchronised)
  // Algorithmic bytes (each value read or written once per phase; operator
  // data once per sweep) of one V-cycle, and of one FP32 PCG iteration
  // (V-cycle plus the operator phase and the vector update).
  double vcycle_bytes() const;
  double iter_bytes() const;

  // Level plan for grid g0: 2:1 while possible (in 3D 4:1 first when every
  // element count divides by 4), then the smallest common odd factor, until
  // the first level with <= max_coarse_dofs DOFs (coarsening at
  // least once); that level is solved with a dense inverse.  Allocates all
  // buffers.  cudaErrorInvalidValue when no plan reaches it.
  cudaError_t plan(const Grid& g0, const uint8_t* mask0, int nc, int max_coarse_dofs = 4096);
  // Galerkin coarse operators, diagonals and the coarsest dense inverse for
  // moduli E32 (FP32 on the device; coarse_ok false if a pivot was not positive).
  cudaError_t build(cudaStream_t s, const double* K0, const float* E32, int* nlaunch);
  // x = V(b) on level li.  On entry lv[li].b holds b and lv[li].x[0] the first
  // sweep from zero, omega D^-1 b (written by whichever kernel produced b);
  // *out receives the buffer holding the result (fixed for a given hierarchy).
  // Every launch returns at once when *stop is set (stop may be null).
  cudaError_t vcycle(cudaStream_t s, int li, int* nlaunch, const int* stop, float** out);
  void drop_graphs();
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
cudaError_t pcg_residual(cudaStream_t s, long long n, int nc, const double* f, const double* Ax, const uint8_t* mask,
                         int dim, double* r);

// Kernels of the graph-captured iteration (ctl in device memory).  Each
// returns at once when ctl->stop is set, except the segment start.
// Segment start: the control block for nc cases (it = 0, stop = 0).
cudaError_t mg_seg_init(cudaStream_t s, MgCtl* ctl, int nc, double tol2, const double* ff, int it_limit, int use64);
// r32 = (float) r and x0 = omega D^-1 r32 (the V-cycle's first sweep).
cudaError_t mg_prep(cudaStream_t s, long long n, int nc, const double* r, float* r32, float* x0, const float* invd,
                    float omega);
// Per-case <a1, b1> (and <a2, b2>) in a fixed order, then the PCG scalars and,
// for what 1, the stopping rule.  a1, a2, b2 are FP32 when a_f32 (then b1
// must be FP32 too), b1 is FP32 when b1_f32; the rest FP64.
//   what 0: pq -> alpha;  what 1: rz_new, rr -> beta, stop rule;  what 2: rz, rr, beta = 0 (segment start)
cudaError_t mg_dotscal(cudaStream_t s, long long n, int nc, const void* a1, bool a_f32, const void* b1, bool b1_f32,
                       const void* a2, const void* b2, double* part, MgCtl* ctl, int what, int* nblocks);
// FP32 inner iteration: d += alpha p, r -= alpha q, x0 = omega D^-1 r.
cudaError_t mg_update32(cudaStream_t s, long long n, int nc, MgCtl* ctl, float* d, const float* p, float* r,
                        const float* q, float* x0, const float* invd, float omega);
// p = z + beta p in FP32 (p = z when beta = 0).
cudaError_t mg_update_p32(cudaStream_t s, long long n, int nc, MgCtl* ctl, float* p, const float* z);
// x += d over n values (end of an FP32 segment).
cudaError_t mg_merge(cudaStream_t s, long long n, double* x, const float* d);
// Dense FP32 inverse of an SPD matrix in place (mg_dense.cu): A (n x n,
// row-major, device) holds the matrix (at least its upper triangle) and
// receives the full inverse.  scratch holds dense_scratch_floats(n) floats;
// *flag (device) is set when a pivot is not positive.  Replays (capturing
// first when needed) the inverter's graph on s; ds must have been created.
size_t dense_scratch_floats(int n);
cudaError_t dense_spd_inverse(cudaStream_t s, DenseInverter& ds, float* A, int n, float* scratch, int* flag,
                              int* nlaunch);
// The coarsest level: assembles its coupling blocks S into A (n = nodes * dim;
// rows and columns of fixed DOFs zero, 1 on their diagonal), then inverts it
// as dense_spd_inverse does; one graph for both.
cudaError_t dense_coarse_inverse(cudaStream_t s, DenseInverter& ds, const Grid& g, const float* S,
                                 const uint8_t* mask, float* A, float* scratch, int* flag, int* nlaunch);
// One FP32 segment as a persistent cooperative kernel (mg_pcg.cu): before the
// launch the control block (mg_seg_init), the finest b = (float) r and x[0] =
// omega D^-1 b (mg_prep) and d = 0 must be in place; zeroes the barrier word.
// The finest operator is the strain-form FP32 operator (constitutive matrix C,
// moduli E32, tile depth zlen).
// trace (optional, 64 int64): globaltimer of CTA 0 after each grid barrier of
// the segment's third iteration.
cudaError_t launch_mg_segment(cudaStream_t s, const MgHierarchy& M, const double* C, const float* E32, int zlen,
                              double* part, GridBar* bar, long long* trace, int nsm, int* grid_out);
// x += alpha p, r -= alpha q (q FP32 when q_f32), r32 = (float) r, x0 = omega D^-1 r32.
cudaError_t mg_update_xr(cudaStream_t s, long long n, int nc, MgCtl* ctl, double* x, const double* p, double* r,
                         const void* q, bool q_f32, float* r32, float* x0, const float* invd, float omega);
// p = z + beta p (p = z when beta = 0), p32 = (float) p.
cudaError_t mg_update_p(cudaStream_t s, long long n, int nc, MgCtl* ctl, double* p, float* p32, const float* z);

}  // namespace tp
