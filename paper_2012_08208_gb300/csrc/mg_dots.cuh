// Completion of the PCG dot products of one kernel launch (gridDim.x CTAs per
// case, blockIdx.y = case): every thread brings its partials of the two
// products; the CTA sums them and stores part[(c nb + b) 2 + k]; the last CTA
// to finish (ticket in the control block) sums every case's partials in a
// fixed order, so the totals do not depend on the order in which CTAs finish,
// forms the PCG scalars (what 0: alpha = rz / pq; 1: beta, rz, rr and the
// segment's stopping rule; 2: the segment start) and resets the ticket.  Every
// thread of the CTA calls it, as the kernel's last step.  Used by the
// standalone dot kernel and by the operator kernels that form the products in
// their epilogues.
#pragma once
#include "common.cuh"
#include "mg.h"

namespace tp {

__device__ __forceinline__ void pcg_dots_complete(double (&acc)[2], double* part, MgCtl* ctl, int what) {
  __shared__ double sred[32 * 2];
  __shared__ double tot[16];
  __shared__ int is_last;
  const int c = blockIdx.y, nb = gridDim.x;
  block_sum<2>(acc, sred);
  if (threadIdx.x == 0) {
    part[((long long)c * nb + blockIdx.x) * 2] = acc[0];
    part[((long long)c * nb + blockIdx.x) * 2 + 1] = acc[1];
    __threadfence();
    const unsigned t = atomicAdd(&ctl->ticket, 1u);
    is_last = t == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int nc = gridDim.y;
  // every thread of the last CTA takes a strided share of the partials (a
  // few loads each, all in flight), then a fixed-order block reduction
  for (int cc = 0; cc < nc; cc++) {
    double v2[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      v2[0] += __ldcg(part + ((long long)cc * nb + b) * 2);
      v2[1] += __ldcg(part + ((long long)cc * nb + b) * 2 + 1);
    }
    block_sum<2>(v2, sred);
    if (threadIdx.x == 0) {
      tot[2 * cc] = v2[0];
      tot[2 * cc + 1] = v2[1];
    }
  }
  __syncthreads();
  double* sc = ctl->sc;
  const int cc = threadIdx.x;
  if (cc < nc) {
    const double s1 = tot[2 * cc], s2 = tot[2 * cc + 1];
    if (what == 0) {  // alpha = rz / pq
      sc[24 + cc] = s1;
      sc[cc] = (s1 > 0.0 && isfinite(s1)) ? sc[16 + cc] / s1 : 0.0;
    } else if (what == 1) {  // beta = rz_new / rz
      sc[8 + cc] = sc[16 + cc] != 0.0 ? s1 / sc[16 + cc] : 0.0;
      sc[16 + cc] = s1;
      sc[32 + cc] = s2;
    } else {  // segment start
      sc[16 + cc] = s1;
      sc[32 + cc] = s2;
      sc[8 + cc] = 0.0;
      ctl->rr_start[cc] = s2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (what == 1) {
      // stop at the tolerance (with margin 1/2 on the recurrence residual),
      // when the FP32 operator's error may dominate the recurrence (1e-5 of
      // the segment's starting residual), on stagnation (no halving of the
      // worst relative residual in 50 iterations), on breakdown, or at the
      // iteration limit
      const int it = ctl->it + 1;
      ctl->it = it;
      bool brk = false, done = true, inner = ctl->use64 == 0;
      double worst = 0.0;
      for (int k = 0; k < nc; k++) {
        const double rec = sc[32 + k];
        brk |= !isfinite(rec) || !(sc[24 + k] > 0.0);
        done &= rec <= 0.25 * ctl->tol2 * ctl->ff[k];
        inner &= rec <= 1e-10 * ctl->rr_start[k];
        worst = fmax(worst, rec / ctl->ff[k]);
      }
      if (ctl->best == 0.0 || worst < 0.25 * ctl->best) {
        ctl->best = worst;
        ctl->best_it = it;
      }
      const bool stall = it - ctl->best_it >= 50, limit = it >= ctl->it_limit;
      const int reason = (done ? MG_STOP_DONE : 0) | (inner ? MG_STOP_INNER : 0) | (stall ? MG_STOP_STALL : 0) |
                         (brk ? MG_STOP_BREAK : 0) | (limit ? MG_STOP_LIMIT : 0);
      ctl->reason = reason;
      ctl->stop = reason != 0;
    }
    ctl->ticket = 0u;
  }
}

}  // namespace tp
