// C-ABI of the GB300 SIMP library (declared in include/topo.h).
// Host-side state machine, argument validation and kernel launches.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/topo.h"
#include "host.h"
#include "problem.h"

using namespace tp;

namespace {

constexpr int kMaxGridPerSm = 16;

tp_status fail(tp_problem* p, tp_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

tp_status cuda_fail(tp_problem* p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(p, e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA, m);
}

#define TPCK(call, what)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, what);  \
  } while (0)

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
  return cudaMalloc((void**)ptr, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
}

void free_all(tp_problem* p) {
  void* ptrs[] = {p->rho, p->rho_new, p->E32, p->E64, p->mask, p->passive, p->f, p->x64,
                  p->inv32, p->inv64, p->w[0], p->w[1], p->w[2], p->w[3], p->w[4], p->w[5],
                  p->part, p->bar, p->cgs, p->tol2, p->ost, p->scal, p->dc, p->dcf, p->ce, p->bscr, p->abi,
                  p->trace, p->nn_feat, p->nn_out, p->nn_scal, p->rho_phys, p->rowsum, p->helm, p->hst, p->Edw};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p->mg;
  p->mg = nullptr;
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p->flt;
}

bool finite_all(const double* a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// Densities that set the stiffness: rho, or its density filter in mode 1.
const double* phys(const tp_problem* p) { return p->filter_mode == TP_FILTER_SENSITIVITY ? p->rho : p->rho_phys; }

// out = H in with the Helmholtz filter (elements in and out); synchronises to
// read the solver status.
tp_status helm_filter(tp_problem* p, const double* in, double* out) {
  TPCK(launch_helm_filter(p->stream, p->g, p->helm_a, in, out, p->helm, p->part, p->bar, p->hst, 1e-14, 2000, p->nsm),
       "Helmholtz filter kernels");
  p->launches += 3;
  tp::HelmStatus st;
  TPCK(cudaMemcpyAsync(&st, p->hst, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "copy status");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  if (st.flags & ERR_TIMEOUT) return fail(p, TP_ERR_TIMEOUT, "a device-side wait timed out in the Helmholtz filter");
  if (st.flags) return fail(p, TP_ERR_NOT_CONVERGED, "the Helmholtz filter solve did not converge");
  return TP_OK;
}

// The moduli as double-words on stream s (the double-word operator's input),
// formed when the moduli changed since the last call.
static tp_status ensure_dw(tp_problem* p, cudaStream_t s) {
  if (!p->Edw) TPCK(cudaMalloc(&p->Edw, (size_t)p->ne * 2 * sizeof(float) + 16), "alloc");
  if (p->dw_version != p->E_version) {
    TPCK(launch_dw_moduli(s, p->E64, p->Edw, p->ne), "moduli kernel");
    p->launches++;
    p->dw_version = p->E_version;
  }
  return TP_OK;
}

tp_status ensure_E(tp_problem* p) {
  if (!p->E_dirty) return TP_OK;
  if (p->filter_mode == TP_FILTER_DENSITY) {
    TPCK(launch_filter(p->stream, *p->flt, 1, p->rho, nullptr, p->rho_phys), "density filter kernel");
    p->launches++;
  } else if (p->filter_mode == TP_FILTER_HELMHOLTZ) {
    const tp_status st = helm_filter(p, p->rho, p->rho_phys);
    if (st != TP_OK) return st;
  }
  TPCK(launch_young(p->stream, phys(p), p->E32, p->E64, p->ne, p->prm.E0, p->prm.Emin, p->prm.penal),
       "young kernel");
  p->launches++;
  p->E_dirty = false;
  p->E_version++;
  return TP_OK;
}

cudaMemcpyKind kind_of(int on_device, bool to_device) {
  if (on_device) return cudaMemcpyDeviceToDevice;
  return to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

}  // namespace

// Depth (node planes) of the 3D streaming tiles.  Each tile of 31 x 7 node
// columns streams zlen + 1 element layers after a two-plane prologue; the
// persistent CG runs `resident` CTAs that take the tiles in rounds.  Pick the
// balanced depth with the least rounds * (zlen + 3).
static int pick_zlen(const Grid& g, int resident) {
  const int tx = (g.nx + 30) / 31, ty = (g.ny + 6) / 7;
  int best = 16;
  long long best_cost = -1;
  for (int zl = 1; zl <= g.nz; zl++) {
    const int chunks = (g.nz + zl - 1) / zl;
    const int zb = (g.nz + chunks - 1) / chunks;
    if (zb != zl) continue;  // only balanced depths
    const long long ntiles = (long long)tx * ty * chunks;
    const long long rounds = (ntiles + resident - 1) / resident;
    const long long cost = rounds * (zl + 3);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zl;
    }
  }
  return best;
}

tp_status tp_problem_ensure_E(tp_problem* p) { return ensure_E(p); }

// Zero the grid-barrier word before a persistent launch, then install the
// problem's wait limit (tp_set_wait_budget) if one is set.
static cudaError_t reset_bar(tp_problem* p) {
  cudaError_t e = cudaMemsetAsync(p->bar, 0, sizeof(GridBar), p->stream);
  if (e == cudaSuccess && p->wait_budget)
    e = cudaMemcpyAsync(&p->bar->budget, &p->wait_budget, sizeof(unsigned), cudaMemcpyHostToDevice, p->stream);
  return e;
}

// Finest multigrid level: the problem's FP32 strain-form operator on all cases.
static cudaError_t mg_fine_op(void* ctx, cudaStream_t s, const float* u, const float* w, const float* b,
                              const float* invd, float* y, int mode, float a, float c, float om, const int* stop,
                              int dots) {
  tp_problem* p = (tp_problem*)ctx;
  return launch_mg_sweep(s, p->g, p->C.data(), p->E32, p->mask, invd, u, w, b, y, p->nc, p->zlen, mode, a, c, om,
                         stop, dots, p->part, p->mg->ctl);
}

// CG preconditioned by one FP32 multigrid V-cycle per iteration
// (TP_PRECOND_MG, TP_PRECOND_MG_FUSED).  Vectors in the ABI layout; the
// solution ends in x64.
//
// The solve is a sequence of segments, each followed by an FP64 true residual
// (restart).  A segment solves K d = r for a correction d with FP32 vectors
// and the FP32 operator and ends with x += d; after a segment that gained less
// than 100x, the segments switch to FP64 vectors and the FP64 operator.  A
// segment stops at the tolerance, when the FP32 operator's error may dominate
// the recurrence, on stagnation, breakdown or the iteration limit; the rule is
// evaluated on the device after every iteration.
//   TP_PRECOND_MG: the iterations run as replays of a CUDA graph of
//     MgHierarchy::kGraphIters iterations; after the stop every later kernel
//     of the replay returns at once, and the host synchronises once per replay.
//   TP_PRECOND_MG_FUSED: an FP32 segment is one persistent cooperative kernel
//     (mg_pcg.cu) with grid barriers between its phases.
static tp_status mg_solve(tp_problem* p, const tp_solve_opts* opts, tp_solve_info* info) {
  const bool fused = opts->precond == TP_PRECOND_MG_FUSED;
  tp_status st = ensure_E(p);
  if (st != TP_OK) return st;
  if (!p->mg) {
    p->mg = new MgHierarchy();
    cudaError_t e = p->mg->plan(p->g, p->mask, p->nc);
    if (e != cudaSuccess) {
      delete p->mg;
      p->mg = nullptr;
      cudaGetLastError();
      if (e == cudaErrorInvalidValue)
        return fail(p, TP_ERR_ARG, "no multigrid hierarchy for this grid (element counts without small common factors)");
      return cuda_fail(p, e, "multigrid allocation");
    }
  }
  MgHierarchy& M = *p->mg;
  const int kIt = MgHierarchy::kGraphIters;
  if (p->profile && !M.ev[0])
    for (auto& ev : M.ev) TPCK(cudaEventCreate(&ev), "event");
  M.timing = p->profile;
  M.fine_op_fn = mg_fine_op;
  M.fine_ctx = p;
  const cudaStream_t s = p->stream;
  const long long n = p->ndof;
  const int nc = p->nc;
  double* x = (double*)p->w[0];
  double* r = (double*)p->w[1];
  double* pp = (double*)p->w[3];
  double* q = (double*)p->w[4];
  double* fA = (double*)p->w[5];
  MgCtl* ctl = M.ctl;
  double* sc = ctl->sc;  // device address of the scalars
  const int* stop = &ctl->stop;
  MgLevel& l0 = M.lv[0];
  int nl = 0;
  TPCK(cudaEventRecord(p->ev0, s), "event");
  // r = f - K x and rr per case into the scalars, on stream cs; read_rr copies
  // rr to the host (synchronises the problem's stream).  K x is the FP64
  // operator, or in 3D at tolerances >= 1e-8 the double-word FP32 operator: its
  // error (about 1e-13 of the element force scale, 1e-11 of |f| on the 3D
  // cantilevers) is far below the tolerance, and it runs on the FP32 pipes
  // instead of GB300's FP64 pipe.
  const bool dw_res = p->dim == 3 && opts->tol >= 1e-8;
  auto issue_rr = [&](cudaStream_t cs) -> tp_status {
    if (dw_res) {
      const tp_status sd = ensure_dw(p, cs);
      if (sd != TP_OK) return sd;
      TPCK(launch_matvec_dw(cs, p->g, p->C.data(), p->Edw, p->mask, x, q, nc, p->zlen), "matvec");
    } else {
      TPCK(launch_matvec(cs, p->g, p->C.data(), true, p->E64, p->mask, x, q, nc, p->zlen), "matvec");
    }
    TPCK(pcg_residual(cs, n, nc, fA, q, p->mask, p->dim, r), "residual kernel");
    int nb = 0;
    TPCK(pcg_dot2(cs, n, nc, r, r, r, r, p->part, &nb), "dot kernel");
    TPCK(pcg_scalars(cs, nb, nc, p->part, 2, sc), "scalar kernel");
    nl += 4;
    return TP_OK;
  };
  auto read_rr = [&](double* rr_out) -> tp_status {
    double h[64];
    TPCK(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s), "copy");
    TPCK(cudaStreamSynchronize(s), "sync");
    for (int c = 0; c < nc; c++) rr_out[c] = h[32 + c];
    return TP_OK;
  };
  auto true_rr = [&](double* rr_out) -> tp_status {
    tp_status t = issue_rr(s);
    return t != TP_OK ? t : read_rr(rr_out);
  };
  // The first residual does not depend on the hierarchy (it reads f, x and the
  // FP64 moduli; the build reads the FP32 moduli and writes only its own
  // buffers).  When a rebuild is due, the residual runs on a second stream,
  // forked from and joined back into the problem's stream by events, while the
  // latency-bound build runs beside the FP64-bound operator.
  const bool rebuild = M.version != p->E_version;
  cudaStream_t sr = s;
  if (rebuild) {
    if (!M.side) TPCK(cudaStreamCreateWithFlags(&M.side, cudaStreamNonBlocking), "stream");
    if (!M.fork) TPCK(cudaEventCreateWithFlags(&M.fork, cudaEventDisableTiming), "event");
    if (!M.join) TPCK(cudaEventCreateWithFlags(&M.join, cudaEventDisableTiming), "event");
    TPCK(cudaEventRecord(M.fork, s), "event");
    TPCK(cudaStreamWaitEvent(M.side, M.fork, 0), "stream wait");
    sr = M.side;
  }
  TPCK(launch_to_abi(sr, p->f, fA, p->nn, p->dim, nc), "layout kernel");
  if (opts->warm_start == TP_WARM_ZERO || (opts->warm_start == TP_WARM_PREVIOUS && !p->has_u))
    TPCK(cudaMemsetAsync(x, 0, (size_t)nc * n * sizeof(double), sr), "memset");
  else
    TPCK(launch_to_abi(sr, p->x64, x, p->nn, p->dim, nc), "layout kernel");
  nl += 2;
  st = issue_rr(sr);
  if (rebuild) {
    // the join is recorded and waited for on every path, so no work of this
    // solve is left in flight on the second stream when it returns
    const cudaError_t ej = cudaEventRecord(M.join, sr);
    const cudaError_t eb = st == TP_OK ? M.build(s, p->K0.data(), p->E32, &nl) : cudaSuccess;
    const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(s, M.join, 0) : cudaStreamSynchronize(sr);
    if (st != TP_OK) return st;
    TPCK(eb, "multigrid setup");
    TPCK(ej, "event");
    TPCK(ew, "stream wait");
    if (!M.coarse_ok) return fail(p, TP_ERR_BREAKDOWN, "multigrid coarsest FP32 inverse met a non-positive pivot");
    M.version = p->E_version;
  }
  if (st != TP_OK) return st;
  // One PCG iteration: q = K p, alpha, the iterate and r, z = V(r), beta and
  // the stopping rule, p.  Default: the segment solves K d = r for a
  // correction d with FP32 vectors and the FP32 operator (FP64 scalars); with
  // u64, x, r, p stay FP64 and the operator is FP64.
  float* z32 = nullptr;
  float* r32 = l0.b;  // the V-cycle's right-hand side doubles as the FP32 residual
  // In 3D the FP32 iteration forms its dot products in the epilogues of the
  // kernels that produce the vectors: p.q in the operator q = K p, r.z and r.r
  // in the V-cycle's last finest-level step (which reads r and writes z); the
  // last CTA of each completes the scalars.  Elsewhere a dot kernel follows.
  const bool fuse_dots = p->dim == 3;
  auto issue_iter = [&](cudaStream_t cs, bool u64, int* nlk) -> cudaError_t {
    cudaError_t e;
    const bool fz = !u64 && fuse_dots;
    if (u64) {
      e = launch_matvec(cs, p->g, p->C.data(), true, p->E64, p->mask, pp, q, nc, p->zlen, stop);
      if (e == cudaSuccess) e = mg_dotscal(cs, n, nc, pp, false, q, false, nullptr, nullptr, p->part, ctl, 0, nullptr);
      if (e == cudaSuccess) e = mg_update_xr(cs, n, nc, ctl, x, pp, r, q, false, r32, l0.x[0], l0.invd, M.omega);
      *nlk += 3;
    } else if (fz) {
      e = launch_matvec_dots(cs, p->g, p->C.data(), p->E32, p->mask, M.p32, M.q32, nc, p->zlen, stop, p->part, ctl,
                             0);
      if (e == cudaSuccess) e = mg_update32(cs, n, nc, ctl, M.d32, M.p32, r32, M.q32, l0.x[0], l0.invd, M.omega);
      *nlk += 2;
    } else {
      e = launch_matvec(cs, p->g, p->C.data(), false, p->E32, p->mask, M.p32, M.q32, nc, p->zlen, stop);
      if (e == cudaSuccess)
        e = mg_dotscal(cs, n, nc, M.p32, true, M.q32, true, nullptr, nullptr, p->part, ctl, 0, nullptr);
      if (e == cudaSuccess) e = mg_update32(cs, n, nc, ctl, M.d32, M.p32, r32, M.q32, l0.x[0], l0.invd, M.omega);
      *nlk += 3;
    }
    M.fine_dots = fz ? 1 : -1;
    if (e == cudaSuccess) e = M.vcycle(cs, 0, nlk, stop, &z32);
    M.fine_dots = -1;
    if (u64) {
      if (e == cudaSuccess) e = mg_dotscal(cs, n, nc, r, false, z32, true, r, r, p->part, ctl, 1, nullptr);
      if (e == cudaSuccess) e = mg_update_p(cs, n, nc, ctl, pp, M.p32, z32);
      *nlk += 2;
    } else {
      if (e == cudaSuccess && !fz)
        e = mg_dotscal(cs, n, nc, r32, true, z32, true, r32, r32, p->part, ctl, 1, nullptr);
      if (e == cudaSuccess) e = mg_update_p32(cs, n, nc, ctl, M.p32, z32);
      *nlk += fz ? 1 : 2;
    }
    return e;
  };
  // The graph of kGraphIters iterations for u64, with the finest sweeps
  // bracketed by event nodes when timing.
  auto graph = [&](bool u64) -> tp_status {
    const int gi = u64 ? 1 : 0, gt = M.timing ? 1 : 0;
    if (M.gx[gi][gt]) return TP_OK;
    if (gt && M.sweep_ev.empty()) {
      M.sweep_ev.resize(2 * 2 * M.nu0 * kIt);  // an event pair per finest-level sweep of the graph
      for (auto& ev : M.sweep_ev) TPCK(cudaEventCreate(&ev), "event");
    }
    // captured on a private stream (the problem's stream may be the legacy
    // default stream, which cannot be captured), replayed on the problem's
    if (!M.cap) TPCK(cudaStreamCreateWithFlags(&M.cap, cudaStreamNonBlocking), "stream");
    TPCK(cudaStreamBeginCapture(M.cap, cudaStreamCaptureModeRelaxed), "graph capture");
    M.capture_events = gt != 0;
    if (gt) M.ev_used = 0;
    int nlk = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kIt && e == cudaSuccess; k++) e = issue_iter(M.cap, u64, &nlk);
    M.capture_events = false;
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(M.cap, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&M.gx[gi][gt], gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      M.gx[gi][gt] = nullptr;
      return cuda_fail(p, e, "multigrid PCG graph");
    }
    M.gx_launches[gi][gt] = nlk;
    return TP_OK;
  };
  double rr[kMaxCases] = {}, rel0[kMaxCases] = {};
  st = read_rr(rr);  // the first residual, issued above
  if (st != TP_OK) return st;
  int fallback = 0;
  for (int c = 0; c < nc; c++) rel0[c] = std::sqrt(rr[c] / p->ff[c]);
  if (opts->warm_start == TP_WARM_USER) {
    const double lim = opts->warm_max_rel > 0.0 ? opts->warm_max_rel : 1.0;
    for (int c = 0; c < nc; c++) fallback |= !(rr[c] <= lim * lim * p->ff[c]);
    if (fallback) {
      TPCK(cudaMemsetAsync(x, 0, (size_t)nc * n * sizeof(double), s), "memset");
      st = true_rr(rr);
      if (st != TP_OK) return st;
    }
  }
  auto done = [&](const double* v) {
    for (int c = 0; c < nc; c++)
      if (!(v[c] <= opts->tol * opts->tol * p->ff[c])) return false;
    return true;
  };
  int it = 0, restarts = 0;
  bool conv = done(rr), brk = false;
  // FP32 inner operator unless FP64 was asked for, or until a restart cycle
  // gains less than 100x (the FP32 operator's error limits the refinement when
  // eps32 * cond(K) is not small)
  bool use64 = opts->precision == TP_PREC_F64;
  while (!conv && it < opts->max_it && !brk) {
    // segment start from the current residual: r32 = r, the first smoothing
    // step, d = 0; then z = V(r), p = z
    TPCK(mg_seg_init(s, ctl, nc, opts->tol * opts->tol, p->ff, opts->max_it - it, use64 ? 1 : 0), "control kernel");
    TPCK(mg_prep(s, n, nc, r, r32, l0.x[0], l0.invd, M.omega), "convert kernel");
    nl += 2;
    int seg_it = 0;
    if (!use64 && fused) {
      // FP32 segment as one persistent cooperative launch
      TPCK(cudaMemsetAsync(M.d32, 0, (size_t)nc * n * sizeof(float), s), "memset");
      if (M.timing) TPCK(cudaEventRecord(M.ev[0], s), "event");
      int grid = 0;
      TPCK(launch_mg_segment(s, M, p->C.data(), p->E32, p->zlen, p->part, p->bar, p->trace, p->nsm, &grid),
           "multigrid kernel");
      if (M.timing) TPCK(cudaEventRecord(M.ev[1], s), "event");
      nl++;
      TPCK(cudaMemcpyAsync(M.ctl_h, ctl, sizeof(MgCtl), cudaMemcpyDeviceToHost, s), "copy");
      TPCK(cudaStreamSynchronize(s), "sync");
      if (M.ctl_h->timeout) return fail(p, TP_ERR_TIMEOUT, "multigrid PCG kernel: grid barrier timed out");
      seg_it = M.ctl_h->it;
      if (M.timing) {
        float ms = 0.f;
        TPCK(cudaEventElapsedTime(&ms, M.ev[0], M.ev[1]), "event");
        M.timed_ms += ms;
        M.timed_launches++;
        M.timed_bytes += M.vcycle_bytes() + seg_it * M.iter_bytes();
      }
    } else {
      // segment start z = V(r), p = z (d = 0), then replays of the graph of
      // kGraphIters iterations with the device-side stop flag
      const bool fz = !use64 && fuse_dots;
      M.fine_dots = fz ? 2 : -1;
      const cudaError_t ev = M.vcycle(s, 0, &nl, nullptr, &z32);
      M.fine_dots = -1;
      TPCK(ev, "v-cycle");
      if (use64) {
        TPCK(mg_dotscal(s, n, nc, r, false, z32, true, r, r, p->part, ctl, 2, nullptr), "dot kernel");
        TPCK(mg_update_p(s, n, nc, ctl, pp, M.p32, z32), "update kernel");
      } else {
        TPCK(cudaMemsetAsync(M.d32, 0, (size_t)nc * n * sizeof(float), s), "memset");
        if (!fz) TPCK(mg_dotscal(s, n, nc, r32, true, z32, true, r32, r32, p->part, ctl, 2, nullptr), "dot kernel");
        TPCK(mg_update_p32(s, n, nc, ctl, M.p32, z32), "update kernel");
      }
      nl += fz ? 1 : 2;
      st = graph(use64);
      if (st != TP_OK) return st;
      const int gi = use64 ? 1 : 0, gt = M.timing ? 1 : 0;
      for (;;) {
        TPCK(cudaGraphLaunch(M.gx[gi][gt], s), "graph launch");
        nl += M.gx_launches[gi][gt];
        TPCK(cudaMemcpyAsync(M.ctl_h, ctl, sizeof(MgCtl), cudaMemcpyDeviceToHost, s), "copy");
        TPCK(cudaStreamSynchronize(s), "sync");
        const int now = M.ctl_h->it;
        if (gt) M.collect_sweeps((now - seg_it) * 2 * M.nu0);  // sweeps of the iterations that ran
        const bool advanced = now > seg_it;
        seg_it = now;
        if (M.ctl_h->stop) break;
        if (!advanced) return fail(p, TP_ERR_CUDA, "multigrid PCG graph made no progress");
      }
    }
    it += seg_it;
    brk = (M.ctl_h->reason & MG_STOP_BREAK) != 0;
    if (!use64) {  // x += d
      TPCK(mg_merge(s, (long long)nc * n, x, M.d32), "merge kernel");
      nl++;
    }
    double before = 0.0, after = 0.0;
    for (int c = 0; c < nc; c++) before = std::max(before, rr[c] / p->ff[c]);
    st = true_rr(rr);
    if (st != TP_OK) return st;
    for (int c = 0; c < nc; c++) after = std::max(after, rr[c] / p->ff[c]);
    conv = done(rr);
    if (!conv && !(after < 1e-2 * before)) use64 = true;
    if (!conv && ++restarts > 12) break;
  }
  TPCK(launch_to_internal(s, x, p->x64, p->nn, p->dim, nc, p->mask, 1), "layout kernel");
  nl++;
  TPCK(cudaEventRecord(p->ev1, s), "event");
  TPCK(cudaEventSynchronize(p->ev1), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  p->launches += nl;
  p->has_u = true;
  p->has_dc = p->has_dcf = false;
  tp_status rs = conv ? TP_OK : (brk ? TP_ERR_BREAKDOWN : TP_ERR_NOT_CONVERGED);
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = it;
    info->updates = restarts + 1;
    info->converged = conv ? 1 : 0;
    info->status = rs;
    for (int c = 0; c < nc; c++) {
      info->rel_res[c] = std::sqrt(rr[c] / p->ff[c]);
      info->rel_res_init[c] = rel0[c];
    }
    info->warm_fallback = fallback;
    info->ms = ms;
  }
  if (rs == TP_ERR_BREAKDOWN) return fail(p, rs, "multigrid PCG breakdown (p^T K p <= 0 or not finite)");
  if (rs == TP_ERR_NOT_CONVERGED) return fail(p, rs, "multigrid PCG stopped before the tolerance");
  return TP_OK;
}

extern "C" {

tp_status tp_create_problem(const tp_params* params, void* cuda_stream, tp_problem** out) {
  if (!params || !out) return TP_ERR_ARG;
  *out = nullptr;
  const tp_params& q = *params;
  if (q.dim != 2 && q.dim != 3) return TP_ERR_ARG;
  if (q.nelx < 1 || q.nely < 1 || (q.dim == 3 && q.nelz < 1)) return TP_ERR_ARG;
  if (!(q.volfrac > 0.0 && q.volfrac <= 1.0) || !(q.rmin > 0.0) || !(q.penal >= 1.0)) return TP_ERR_ARG;
  if (!(q.nu >= 0.0 && q.nu < 0.5) || !(q.Emin > 0.0 && q.Emin < q.E0)) return TP_ERR_ARG;
  if (!(q.dmin > 0.0 && q.dmin < 1.0) || !(q.move > 0.0)) return TP_ERR_ARG;
  if (q.n_cases < 1 || q.n_cases > kMaxCases) return TP_ERR_ARG;
  const long long nx = q.nelx + 1, ny = q.nely + 1, nz = q.dim == 3 ? q.nelz + 1 : 1;
  if (nx * ny * nz * q.dim * q.n_cases > (1LL << 31) - 1) return TP_ERR_ARG;

  tp_problem* p = new tp_problem();
  p->prm = q;
  if (q.dim == 2) p->prm.nelz = 0;
  p->stream = (cudaStream_t)cuda_stream;
  p->dim = q.dim;
  p->nc = q.n_cases;
  p->nv = q.dim * q.n_cases;
  p->g.dim = q.dim;
  p->g.ex = q.nelx;
  p->g.ey = q.nely;
  p->g.ez = q.dim == 3 ? q.nelz : 1;
  p->g.nx = (int)nx;
  p->g.ny = (int)ny;
  p->g.nz = (int)nz;
  p->g.nn = nx * ny * nz;
  p->g.ne = (long long)p->g.ex * p->g.ey * p->g.ez;
  p->nn = p->g.nn;
  p->ne = p->g.ne;
  p->ndof = p->nn * q.dim;
  const int nd = q.dim == 2 ? 8 : 24;
  p->K0.resize(nd * nd);
  element_k0(q.dim, q.nu, p->K0.data());
  p->C.resize(18 * 18);
  double recon = 0.0;
  element_strain_C(q.dim, p->K0.data(), p->C.data(), &recon);
  if (!(recon < 1e-12)) {
    delete p;
    return TP_ERR_ARG;
  }
  p->flt = new FilterLaunch();
  p->flt->g = p->g;
  p->flt->ntaps = filter_taps(q.dim, q.rmin, kMaxTaps, p->flt->off, p->flt->w);
  if (p->flt->ntaps < 1) {
    delete p->flt;
    delete p;
    return TP_ERR_ARG;
  }

  cudaError_t e = cudaGetDevice(&p->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
  if (e == cudaSuccess && q.dim == 3) p->zlen = pick_zlen(p->g, 2 * p->nsm);
  const size_t nvals = (size_t)p->nn * p->nv;
  const size_t maxgrid = (size_t)p->nsm * kMaxGridPerSm;
  if (e == cudaSuccess) e = dalloc(&p->rho, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->rho_new, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->E32, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->E64, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->mask, p->nn);
  if (e == cudaSuccess) e = dalloc(&p->passive, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->f, nvals);
  if (e == cudaSuccess) e = dalloc(&p->x64, nvals);
  if (e == cudaSuccess) e = dalloc(&p->inv32, p->ndof);
  if (e == cudaSuccess) e = dalloc(&p->inv64, p->ndof);
  for (int i = 0; i < 6 && e == cudaSuccess; i++) e = dalloc((double**)&p->w[i], nvals);
  // partial sums: CG segment slots (24 per CTA) or residual tiles (16 per tile)
  // (tile count bound: 32 x 8 node tiles, one plane deep in 3D)
  const size_t tiles_bound = (size_t)((nx + 31) / 32) * (size_t)((ny + 7) / 8) * (size_t)nz;
  const size_t npart = std::max<size_t>((size_t)48 * maxgrid, (size_t)16 * tiles_bound);
  if (e == cudaSuccess) e = dalloc(&p->part, npart);
  if (e == cudaSuccess) e = dalloc(&p->bar, 1);
  if (e == cudaSuccess) e = dalloc(&p->cgs, 1);
  if (e == cudaSuccess) e = dalloc(&p->tol2, kMaxCases);
  if (e == cudaSuccess) e = dalloc(&p->ost, 1);
  if (e == cudaSuccess) e = dalloc(&p->scal, 16);
  if (e == cudaSuccess) e = dalloc(&p->dc, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->dcf, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->ce, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->bscr, p->ne);
  if (e == cudaSuccess) e = dalloc(&p->abi, nvals);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->mask, 0, p->nn, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->passive, 0, p->ne, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->x64, 0, nvals * sizeof(double), p->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
  if (e != cudaSuccess) {
    const tp_status s = e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
    cudaGetLastError();
    free_all(p);
    delete p;
    return s;
  }
  *out = p;
  return TP_OK;
}

void tp_destroy_problem(tp_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  free_all(p);
  delete p;
}

const char* tp_last_error(const tp_problem* p) { return p ? p->err.c_str() : "null problem"; }

long long tp_launch_count(const tp_problem* p) { return p ? p->launches : 0; }

tp_status tp_set_trace(tp_problem* p, int enable) {
  if (!p) return TP_ERR_ARG;
  if (enable && !p->trace) {
    TPCK(cudaMalloc((void**)&p->trace, 32 * 8 * sizeof(long long)), "alloc trace");
    TPCK(cudaMemsetAsync(p->trace, 0, 32 * 8 * sizeof(long long), p->stream), "memset");
  } else if (!enable && p->trace) {
    cudaStreamSynchronize(p->stream);
    cudaFree(p->trace);
    p->trace = nullptr;
  }
  return TP_OK;
}

tp_status tp_set_profile(tp_problem* p, int enable) {
  if (!p) return TP_ERR_ARG;
  p->profile = enable != 0;
  if (p->mg) {
    p->mg->timed_launches = 0;
    p->mg->timed_ms = p->mg->timed_bytes = 0.0;
  }
  return TP_OK;
}

tp_status tp_get_profile(tp_problem* p, double* out) {
  if (!p || !out) return TP_ERR_ARG;
  out[0] = out[1] = out[2] = out[3] = 0.0;
  if (p->mg) {
    out[0] = (double)p->mg->timed_launches;
    out[1] = p->mg->timed_ms;
    out[2] = p->mg->timed_bytes;
    out[3] = (double)p->mg->lv.size();
  }
  return TP_OK;
}

tp_status tp_set_wait_budget(tp_problem* p, long long cycles) {
  if (!p) return TP_ERR_ARG;
  if (cycles < 0 || cycles > 4000000000LL) return fail(p, TP_ERR_ARG, "wait budget outside [0, 4e9] cycles");
  TPCK(cudaStreamSynchronize(p->stream), "sync");  // no launch in flight reads the old value
  p->wait_budget = (unsigned)cycles;
  return TP_OK;
}

tp_status tp_get_trace(tp_problem* p, long long* out) {
  if (!p || !out) return TP_ERR_ARG;
  if (!p->trace) return fail(p, TP_ERR_STATE, "tracing is not enabled");
  TPCK(cudaMemcpyAsync(out, p->trace, 32 * 8 * sizeof(long long), cudaMemcpyDeviceToHost, p->stream), "copy");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_set_fixed(tp_problem* p, const uint8_t* fixed) {
  if (!p || !fixed) return fail(p, TP_ERR_ARG, "null argument");
  std::vector<uint8_t> m(p->nn, 0);
  long long nfix = 0;
  for (long long i = 0; i < p->ndof; i++)
    if (fixed[i]) {
      m[i / p->dim] |= (uint8_t)(1u << (i % p->dim));
      nfix++;
    }
  if (nfix == 0) return fail(p, TP_ERR_ARG, "no fixed DOF: the stiffness would be singular");
  TPCK(cudaMemcpyAsync(p->mask, m.data(), p->nn, cudaMemcpyHostToDevice, p->stream), "copy mask");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  p->has_fixed = true;
  p->has_loads = false;
  p->has_u = false;
  p->E_dirty = true;
  return TP_OK;
}

tp_status tp_set_loads(tp_problem* p, const double* f) {
  if (!p || !f) return fail(p, TP_ERR_ARG, "null argument");
  if (!p->has_fixed) return fail(p, TP_ERR_STATE, "tp_set_fixed must precede tp_set_loads");
  const size_t n = (size_t)p->nc * p->ndof;
  if (!finite_all(f, n)) return fail(p, TP_ERR_ARG, "loads contain NaN or Inf");
  std::vector<uint8_t> m(p->nn);
  TPCK(cudaMemcpyAsync(m.data(), p->mask, p->nn, cudaMemcpyDeviceToHost, p->stream), "copy mask");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  for (int c = 0; c < p->nc; c++) {
    double s = 0.0;
    for (long long i = 0; i < p->ndof; i++) {
      const double v = f[(size_t)c * p->ndof + i];
      if (!((m[i / p->dim] >> (i % p->dim)) & 1)) s += v * v;
    }
    if (!(s > 0.0)) return fail(p, TP_ERR_ARG, "a load case has no load on free DOFs");
    p->ff[c] = s;
    double mx = 0.0;
    for (long long i = 0; i < p->ndof; i++)
      if (!((m[i / p->dim] >> (i % p->dim)) & 1)) mx = std::max(mx, std::fabs(f[(size_t)c * p->ndof + i]));
    p->fmax[c] = mx;
  }
  TPCK(cudaMemcpyAsync(p->abi, f, n * sizeof(double), cudaMemcpyHostToDevice, p->stream), "copy loads");
  TPCK(launch_to_internal(p->stream, p->abi, p->f, p->nn, p->dim, p->nc, p->mask, 1), "layout kernel");
  p->launches++;
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  p->has_loads = true;
  return TP_OK;
}

tp_status tp_set_passive(tp_problem* p, const int8_t* passive) {
  if (!p || !passive) return fail(p, TP_ERR_ARG, "null argument");
  for (long long e = 0; e < p->ne; e++)
    if (passive[e] != 0 && passive[e] != 1) return fail(p, TP_ERR_ARG, "passive entries must be 0 or 1");
  TPCK(cudaMemcpyAsync(p->passive, passive, p->ne, cudaMemcpyHostToDevice, p->stream), "copy passive");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  p->has_passive = true;
  return TP_OK;
}

tp_status tp_set_density(tp_problem* p, const double* rho, int on_device) {
  if (!p || !rho) return fail(p, TP_ERR_ARG, "null argument");
  if (!on_device) {
    for (long long e = 0; e < p->ne; e++)
      if (!(rho[e] > 0.0 && rho[e] <= 1.0)) return fail(p, TP_ERR_ARG, "densities must lie in (0, 1]");
  }
  TPCK(cudaMemcpyAsync(p->rho, rho, p->ne * sizeof(double), kind_of(on_device, true), p->stream),
       "copy density");
  if (!on_device) TPCK(cudaStreamSynchronize(p->stream), "sync");
  p->has_density = true;
  p->E_dirty = true;
  p->has_dc = p->has_dcf = false;
  return TP_OK;
}

tp_status tp_solve(tp_problem* p, const tp_solve_opts* opts, tp_solve_info* info) {
  if (!p || !opts) return fail(p, TP_ERR_ARG, "null argument");
  if (!p->has_fixed || !p->has_loads || !p->has_density)
    return fail(p, TP_ERR_STATE, "fixed DOFs, loads and density must be set before tp_solve");
  if (!(opts->tol > 0.0) || opts->max_it < 1) return fail(p, TP_ERR_ARG, "tol must be > 0, max_it >= 1");
  if (opts->precision != TP_PREC_F64 && opts->precision != TP_PREC_MIXED)
    return fail(p, TP_ERR_ARG, "unknown precision");
  if (opts->warm_start < TP_WARM_ZERO || opts->warm_start > TP_WARM_USER)
    return fail(p, TP_ERR_ARG, "unknown warm_start");
  if (opts->warm_start == TP_WARM_USER && !p->has_u)
    return fail(p, TP_ERR_STATE, "TP_WARM_USER needs tp_set(TP_U, ...) first");
  if (opts->precond != TP_PRECOND_JACOBI && opts->precond != TP_PRECOND_MG && opts->precond != TP_PRECOND_MG_FUSED)
    return fail(p, TP_ERR_ARG, "unknown preconditioner");
  if (opts->precond == TP_PRECOND_MG || opts->precond == TP_PRECOND_MG_FUSED) return mg_solve(p, opts, info);
  double drop = opts->update_drop;
  if (opts->precision == TP_PREC_MIXED) {
    if (drop == 0.0) drop = 1e-2;
    if (!(drop > 0.0 && drop < 1.0)) return fail(p, TP_ERR_ARG, "update_drop must lie in (0, 1)");
  }
  tp_status s = ensure_E(p);
  if (s != TP_OK) return s;
  if (p->diag_version != p->E_version) {  // the Jacobi scaling, formed only for this solver
    TPCK(launch_diag(p->stream, p->g, p->K0.data(), p->E64, p->mask, p->inv32, p->inv64), "diag kernel");
    p->launches++;
    p->diag_version = p->E_version;
  }
  const bool f64 = opts->precision == TP_PREC_F64;
  const size_t nvals = (size_t)p->nn * p->nv;
  if (opts->warm_start == TP_WARM_ZERO || (opts->warm_start == TP_WARM_PREVIOUS && !p->has_u))
    TPCK(cudaMemsetAsync(p->x64, 0, nvals * sizeof(double), p->stream), "memset");
  TPCK(cudaMemsetAsync(p->w[0], 0, nvals * (f64 ? 8 : 4), p->stream), "memset");
  Solver S;
  S.g = p->g;
  S.nc = p->nc;
  S.zlen = p->zlen;
  S.E = f64 ? (const void*)p->E64 : (const void*)p->E32;
  S.E64 = p->E64;
  S.mask = p->mask;
  S.invdiag = f64 ? (const void*)p->inv64 : (const void*)p->inv32;
  S.f = p->f;
  S.x64 = p->x64;
  S.xl = p->w[0];
  S.r = p->w[1];
  S.z = p->w[2];
  S.p0 = p->w[3];
  S.p1 = p->w[4];
  S.q = p->w[5];
  S.part = p->part;
  S.tol2ff_dev = p->tol2;
  S.bar = p->bar;
  S.cs = p->cgs;
  for (int c = 0; c < kMaxCases; c++) S.tol2ff[c] = c < p->nc ? opts->tol * opts->tol * p->ff[c] : 0.0;
  S.drop2 = f64 ? 0.0 : drop * drop;
  S.max_it = opts->max_it;
  S.C = p->C.data();
  S.trace = p->trace;
  TPCK(cudaMemcpyAsync(p->tol2, S.tol2ff, sizeof(S.tol2ff), cudaMemcpyHostToDevice, p->stream), "copy");
  TPCK(cudaEventRecord(p->ev0, p->stream), "event");
  int nl = 0;
  TPCK(launch_true_residual(p->stream, S, f64, true, &nl), "residual kernel");
  p->launches += nl;
  CgState st;
  TPCK(cudaMemcpyAsync(&st, p->cgs, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "copy state");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  double rel0[kMaxCases] = {};
  for (int c = 0; c < p->nc; c++) rel0[c] = std::sqrt(st.rr_true[c] / p->ff[c]);
  int fallback = 0;
  if (opts->warm_start == TP_WARM_USER) {
    // A user (or learned) start whose true residual exceeds warm_max_rel times
    // that of the zero start is dropped: the solve restarts from u = 0.
    const double lim = opts->warm_max_rel > 0.0 ? opts->warm_max_rel : 1.0;
    for (int c = 0; c < p->nc; c++) fallback |= !(st.rr_true[c] <= lim * lim * p->ff[c]);
    if (fallback) {
      TPCK(cudaMemsetAsync(p->x64, 0, nvals * sizeof(double), p->stream), "memset");
      TPCK(launch_true_residual(p->stream, S, f64, true, &nl), "residual kernel");
      p->launches += nl;
    }
  }
  for (int guard = 0; guard < 1000000; guard++) {
    TPCK(cudaMemcpyAsync(&st, p->cgs, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "copy state");
    TPCK(cudaStreamSynchronize(p->stream), "sync");
    bool active = false;
    for (int c = 0; c < p->nc; c++) active |= st.state[c] == 0;
    if (!active || st.it >= opts->max_it || (st.flags & ERR_TIMEOUT)) break;
    TPCK(reset_bar(p), "reset barrier");
    TPCK(launch_cg_segment(p->stream, S, f64, p->nsm, &p->last_grid), "cg kernel");
    p->launches++;
    TPCK(launch_true_residual(p->stream, S, f64, false, &nl), "residual kernel");
    p->launches += nl;
  }
  TPCK(cudaEventRecord(p->ev1, p->stream), "event");
  TPCK(cudaEventSynchronize(p->ev1), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  p->has_u = true;
  p->has_dc = p->has_dcf = false;
  bool conv = true, brk = false;
  for (int c = 0; c < p->nc; c++) {
    conv &= st.state[c] == 1;
    brk |= st.state[c] == 2;
  }
  tp_status rs = TP_OK;
  if (st.flags & ERR_TIMEOUT) rs = TP_ERR_TIMEOUT;
  else if (brk) rs = TP_ERR_BREAKDOWN;
  else if (!conv) rs = TP_ERR_NOT_CONVERGED;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->iters = st.it;
    info->updates = st.updates;
    info->converged = conv ? 1 : 0;
    info->status = rs;
    for (int c = 0; c < p->nc; c++) info->rel_res[c] = std::sqrt(st.rr_true[c] / p->ff[c]);
    info->ms = ms;
    for (int c = 0; c < p->nc; c++) info->rel_res_init[c] = rel0[c];
    info->warm_fallback = fallback;
  }
  if (rs == TP_ERR_TIMEOUT) return fail(p, rs, "a device-side wait timed out in the CG kernel");
  if (rs == TP_ERR_BREAKDOWN) return fail(p, rs, "CG breakdown (p^T K p <= 0 or not finite)");
  if (rs == TP_ERR_NOT_CONVERGED)
    return fail(p, rs, "CG stopped before the tolerance (max_it reached or the true residual stagnated)");
  return TP_OK;
}

tp_status tp_sensitivities(tp_problem* p, double* compliance) {
  if (!p) return TP_ERR_ARG;
  if (!p->has_u) return fail(p, TP_ERR_STATE, "tp_solve must precede tp_sensitivities");
  const double dE = p->prm.E0 - p->prm.Emin;
  TPCK(launch_sens(p->stream, p->g, p->nc, p->C.data(), p->x64, p->f, phys(p), p->prm.penal, dE, p->ce,
                   p->dc, p->part, p->scal),
       "sensitivity kernel");
  p->launches += 2;
  if (compliance) {
    TPCK(cudaMemcpyAsync(compliance, p->scal, sizeof(double), cudaMemcpyDeviceToHost, p->stream), "copy");
    TPCK(cudaStreamSynchronize(p->stream), "sync");
  }
  p->has_dc = true;
  p->has_dcf = false;
  return TP_OK;
}

tp_status tp_set_filter_mode(tp_problem* p, int mode) {
  if (!p) return TP_ERR_ARG;
  if (mode != TP_FILTER_SENSITIVITY && mode != TP_FILTER_DENSITY && mode != TP_FILTER_HELMHOLTZ)
    return fail(p, TP_ERR_ARG, "unknown filter mode");
  if (mode != TP_FILTER_SENSITIVITY && !p->rho_phys) TPCK(dalloc(&p->rho_phys, p->ne), "alloc");
  if (mode == TP_FILTER_DENSITY && !p->rowsum) {
    TPCK(dalloc(&p->rowsum, p->ne), "alloc");
    TPCK(launch_filter(p->stream, *p->flt, 3, nullptr, nullptr, p->rowsum), "row-sum kernel");
    p->launches++;
  }
  if (mode == TP_FILTER_HELMHOLTZ && !p->helm) {
    TPCK(dalloc(&p->helm, helm_scratch_doubles(p->g)), "alloc");
    TPCK(cudaMalloc((void**)&p->hst, sizeof(tp::HelmStatus)), "alloc");
    helm_coefficients(p->dim, p->prm.rmin / (2.0 * std::sqrt(3.0)), p->helm_a);
    TPCK(launch_helm_setup(p->stream, p->g, p->helm_a, p->helm), "Helmholtz setup kernel");
    p->launches++;
  }
  if (mode != p->filter_mode) {
    p->filter_mode = mode;
    p->E_dirty = true;
    p->has_dc = p->has_dcf = false;
  }
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_filter(tp_problem* p, int mode) {
  if (!p) return TP_ERR_ARG;
  if (mode != TP_FILTER_SENSITIVITY && mode != TP_FILTER_DENSITY && mode != TP_FILTER_HELMHOLTZ)
    return fail(p, TP_ERR_ARG, "unknown filter mode");
  if (mode != p->filter_mode)
    return fail(p, TP_ERR_STATE, "tp_filter mode differs from the problem's filter mode (tp_set_filter_mode)");
  if (!p->has_dc || !p->has_density) return fail(p, TP_ERR_STATE, "tp_sensitivities must precede tp_filter");
  if (mode == TP_FILTER_SENSITIVITY) {
    TPCK(launch_filter(p->stream, *p->flt, 0, p->rho, p->dc, p->dcf), "filter kernel");
    p->launches++;
  } else if (mode == TP_FILTER_DENSITY) {
    TPCK(launch_filter(p->stream, *p->flt, 2, p->rowsum, p->dc, p->dcf), "filter chain kernel");
    p->launches++;
  } else {
    const tp_status st = helm_filter(p, p->dc, p->dcf);  // H is symmetric: dc~ = H dc
    if (st != TP_OK) return st;
  }
  p->has_dcf = true;
  return TP_OK;
}

tp_status tp_oc_update(tp_problem* p, double* lambda, double* volume, double* change) {
  if (!p) return TP_ERR_ARG;
  if (!p->has_dcf) return fail(p, TP_ERR_STATE, "tp_filter (or tp_set(TP_DCF)) must precede tp_oc_update");
  TPCK(reset_bar(p), "reset barrier");
  int grid = 0;
  TPCK(launch_oc(p->stream, p->ne, p->rho, p->dcf, p->has_passive ? p->passive : nullptr, p->prm.volfrac,
                 p->prm.move, p->prm.dmin, p->rho_new, p->bscr, p->part, p->bar, p->ost, p->nsm, &grid),
       "oc kernel");
  p->launches++;
  OcStatus st;
  TPCK(cudaMemcpyAsync(&st, p->ost, sizeof(st), cudaMemcpyDeviceToHost, p->stream), "copy status");
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  if (st.flags & ERR_TIMEOUT) return fail(p, TP_ERR_TIMEOUT, "a device-side wait timed out in the OC kernel");
  if (st.flags & ERR_NAN) return fail(p, TP_ERR_ARG, "no multiplier bracket found (non-finite sensitivities?)");
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

tp_status tp_simp_step(tp_problem* p, const tp_solve_opts* opts, tp_step_info* info) {
  if (!p || !opts) return fail(p, TP_ERR_ARG, "null argument");
  tp_step_info loc;
  memset(&loc, 0, sizeof(loc));
  tp_status s = tp_solve(p, opts, &loc.solve);
  if (s != TP_OK && s != TP_ERR_NOT_CONVERGED) {
    if (info) *info = loc;
    return s;
  }
  tp_status s2 = tp_sensitivities(p, &loc.compliance);
  if (s2 == TP_OK) s2 = tp_filter(p, p->filter_mode);
  if (s2 == TP_OK) s2 = tp_oc_update(p, &loc.lambda, &loc.volume, &loc.change);
  if (s2 == TP_OK) {
    loc.oc_passes = p->oc_passes;
    loc.oc_root = p->oc_root;
  }
  if (info) *info = loc;
  if (s2 != TP_OK) return s2;
  return s;
}

tp_status tp_get(tp_problem* p, int what, void* dst, int on_device) {
  if (!p || !dst) return fail(p, TP_ERR_ARG, "null argument");
  const cudaMemcpyKind k = kind_of(on_device, false);
  switch (what) {
    case TP_RHO:
      if (!p->has_density) return fail(p, TP_ERR_STATE, "density not set");
      TPCK(cudaMemcpyAsync(dst, p->rho, p->ne * sizeof(double), k, p->stream), "copy");
      break;
    case TP_RHO_PHYS: {
      if (!p->has_density) return fail(p, TP_ERR_STATE, "density not set");
      tp_status st = ensure_E(p);
      if (st != TP_OK) return st;
      TPCK(cudaMemcpyAsync(dst, phys(p), p->ne * sizeof(double), k, p->stream), "copy");
      break;
    }
    case TP_U:
      if (!p->has_u) return fail(p, TP_ERR_STATE, "no displacement yet");
      TPCK(launch_to_abi(p->stream, p->x64, p->abi, p->nn, p->dim, p->nc), "layout kernel");
      p->launches++;
      TPCK(cudaMemcpyAsync(dst, p->abi, (size_t)p->nc * p->ndof * sizeof(double), k, p->stream), "copy");
      break;
    case TP_DC:
      if (!p->has_dc) return fail(p, TP_ERR_STATE, "no sensitivities yet");
      TPCK(cudaMemcpyAsync(dst, p->dc, p->ne * sizeof(double), k, p->stream), "copy");
      break;
    case TP_CE:
      if (!p->has_dc) return fail(p, TP_ERR_STATE, "no sensitivities yet");
      TPCK(cudaMemcpyAsync(dst, p->ce, p->ne * sizeof(double), k, p->stream), "copy");
      break;
    case TP_DCF:
      if (!p->has_dcf) return fail(p, TP_ERR_STATE, "no filtered sensitivities yet");
      TPCK(cudaMemcpyAsync(dst, p->dcf, p->ne * sizeof(double), k, p->stream), "copy");
      break;
    default:
      return fail(p, TP_ERR_ARG, "unknown quantity");
  }
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_set(tp_problem* p, int what, const void* src, int on_device) {
  if (!p || !src) return fail(p, TP_ERR_ARG, "null argument");
  const cudaMemcpyKind k = kind_of(on_device, true);
  switch (what) {
    case TP_U:
      if (!p->has_fixed) return fail(p, TP_ERR_STATE, "fixed DOFs not set");
      if (!on_device && !finite_all((const double*)src, (size_t)p->nc * p->ndof))
        return fail(p, TP_ERR_ARG, "displacement contains NaN or Inf");
      TPCK(cudaMemcpyAsync(p->abi, src, (size_t)p->nc * p->ndof * sizeof(double), k, p->stream), "copy");
      TPCK(launch_to_internal(p->stream, p->abi, p->x64, p->nn, p->dim, p->nc, p->mask, 1), "layout kernel");
      p->launches++;
      p->has_u = true;
      break;
    case TP_DC:
      TPCK(cudaMemcpyAsync(p->dc, src, p->ne * sizeof(double), k, p->stream), "copy");
      p->has_dc = true;
      break;
    case TP_DCF:
      TPCK(cudaMemcpyAsync(p->dcf, src, p->ne * sizeof(double), k, p->stream), "copy");
      p->has_dcf = true;
      break;
    default:
      return fail(p, TP_ERR_ARG, "unknown quantity");
  }
  TPCK(cudaStreamSynchronize(p->stream), "sync");
  return TP_OK;
}

tp_status tp_matvec(tp_problem* p, const void* u, void* y, int precision, int ncopies, int on_device) {
  if (!p || !u || !y || ncopies < 1) return fail(p, TP_ERR_ARG, "bad argument");
  if (!p->has_fixed || !p->has_density) return fail(p, TP_ERR_STATE, "fixed DOFs and density must be set");
  if (precision != TP_PREC_F64 && precision != TP_PREC_MIXED && precision != TP_PREC_DW)
    return fail(p, TP_ERR_ARG, "unknown precision");
  tp_status s = ensure_E(p);
  if (s != TP_OK) return s;
  const bool dw = precision == TP_PREC_DW;
  if (dw) {
    s = ensure_dw(p, p->stream);
    if (s != TP_OK) return s;
  }
  const bool f64 = precision != TP_PREC_MIXED;
  const size_t bytes = (size_t)ncopies * p->ndof * (f64 ? 8 : 4);
  const void* du = u;
  void* dy = y;
  void* tmp = nullptr;
  if (!on_device) {
    TPCK(cudaMalloc(&tmp, 2 * bytes), "alloc");
    TPCK(cudaMemcpyAsync(tmp, u, bytes, cudaMemcpyHostToDevice, p->stream), "copy");
    du = tmp;
    dy = (char*)tmp + bytes;
  }
  cudaError_t e = dw ? launch_matvec_dw(p->stream, p->g, p->C.data(), p->Edw, p->mask, (const double*)du, (double*)dy,
                                        ncopies, p->zlen)
                     : launch_matvec(p->stream, p->g, p->C.data(), f64,
                                     f64 ? (const void*)p->E64 : (const void*)p->E32, p->mask, du, dy, ncopies, p->zlen);
  p->launches++;
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(p, e, "matvec");
  return TP_OK;
}

}  // extern "C"
