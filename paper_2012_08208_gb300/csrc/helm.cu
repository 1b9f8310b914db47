// Helmholtz (PDE) filter (the filter the paper switches to for its parallel
// runs; Lazarov & Sigmund's form):
//
//   rho~ = T^T (R^2 K_F + M_F)^-1 T x,   R = rmin / (2 sqrt 3),
//
// K_F, M_F the Laplacian stiffness and consistent mass of the bilinear /
// trilinear unit element, T[n, e] = 1 / 2^dim (the integral of N_n over e),
// homogeneous Neumann conditions (the element assembly leaves them natural).
// An entry of the unit element matrix R^2 K_F + M_F depends only on the number
// h of coordinates in which its two corners differ:
//   2D  K_F = {4, -1, -2} / 6,      M_F = {4, 2, 1} / 36
//   3D  K_F = {4, 0, -1, -1} / 12,  M_F = {8, 4, 2, 1} / 216
// so the nodal operator is a constant 3^dim-point stencil whose weights at the
// boundary follow from the elements present.  The nodal system is solved by
// FP64 iterative refinement around Jacobi-PCG in FP32 (one persistent
// cooperative kernel per inner solve, two grid barriers per iteration, FP64
// dot products); the result is the element mean of the nodal field.
#include <cmath>

#include "common.cuh"
#include "host.h"

namespace tp {
namespace {

constexpr int kHelmSlots = 4;  // partial sums per CTA: p.q | r.z, r.r

// Element-matrix entry by Hamming class, and the corners of element (ex, ey, ez).
struct HelmOp {
  Grid g;
  double a[4];
};

// y_n = sum over the elements containing node n, sum over their corners m,
// a[h(n, m)] v_m, with v read through `load(m)`.
template <int DIM, typename T = double, class Load>
__device__ __forceinline__ T helm_row(const HelmOp& op, int i, int j, int k, Load load) {
  const Grid& g = op.g;
  T y = T(0);
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); cz++) {
    const int ez = k - cz;
    if (DIM == 3 && (ez < 0 || ez >= g.ez)) continue;
#pragma unroll
    for (int cy = 0; cy < 2; cy++) {
      const int ey = j - cy;
      if (ey < 0 || ey >= g.ey) continue;
#pragma unroll
      for (int cx = 0; cx < 2; cx++) {
        const int ex = i - cx;
        if (ex < 0 || ex >= g.ex) continue;
        // corners m of element (ex, ey, ez): offsets (mx, my, mz) in {0, 1}
#pragma unroll
        for (int mz = 0; mz < (DIM == 3 ? 2 : 1); mz++)
#pragma unroll
          for (int my = 0; my < 2; my++)
#pragma unroll
            for (int mx = 0; mx < 2; mx++) {
              const int h = (mx != cx) + (my != cy) + (DIM == 3 ? (mz != cz) : 0);
              const long long m = (ex + mx) + (long long)g.nx * ((ey + my) + (long long)g.ny * (DIM == 3 ? ez + mz : 0));
              y = fma((T)op.a[h], load(m), y);
            }
      }
    }
  }
  return y;
}

template <int DIM>
__device__ __forceinline__ void node_ijk(const Grid& g, long long n, int& i, int& j, int& k) {
  const long long nxy = (long long)g.nx * g.ny;
  k = DIM == 3 ? (int)(n / nxy) : 0;
  const long long rem = n - (long long)k * nxy;
  j = (int)(rem / g.nx);
  i = (int)(rem - (long long)j * g.nx);
}

// b_n = (1 / 2^dim) sum over the elements containing n of x_e.
template <int DIM>
__global__ void helm_rhs_kernel(Grid g, const double* __restrict__ x, double* __restrict__ b) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nn; n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_ijk<DIM>(g, n, i, j, k);
    double s = 0.0;
    for (int cz = 0; cz < (DIM == 3 ? 2 : 1); cz++) {
      const int ez = k - cz;
      if (DIM == 3 && (ez < 0 || ez >= g.ez)) continue;
      for (int cy = 0; cy < 2; cy++) {
        const int ey = j - cy;
        if (ey < 0 || ey >= g.ey) continue;
        for (int cx = 0; cx < 2; cx++) {
          const int ex = i - cx;
          if (ex < 0 || ex >= g.ex) continue;
          s += x[ex + (long long)g.ex * (ey + (long long)g.ey * (DIM == 3 ? ez : 0))];
        }
      }
    }
    b[n] = s * (DIM == 2 ? 0.25 : 0.125);
  }
}

// out_e = mean of psi over the corners of e.
template <int DIM>
__global__ void helm_mean_kernel(Grid g, const double* __restrict__ psi, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.ne; e += (long long)gridDim.x * blockDim.x) {
    const long long exy = (long long)g.ex * g.ey;
    const int ez = DIM == 3 ? (int)(e / exy) : 0;
    const long long rem = e - (long long)ez * exy;
    const int ey = (int)(rem / g.ex), ex = (int)(rem - (long long)ey * g.ex);
    double s = 0.0;
    for (int mz = 0; mz < (DIM == 3 ? 2 : 1); mz++)
      for (int my = 0; my < 2; my++)
        for (int mx = 0; mx < 2; mx++)
          s += psi[(ex + mx) + (long long)g.nx * ((ey + my) + (long long)g.ny * (ez + mz))];
    out[e] = s * (DIM == 2 ? 0.25 : 0.125);
  }
}

// Inverse diagonal: a[0] times the number of elements containing the node.
template <int DIM>
__global__ void helm_diag_kernel(HelmOp op, double* __restrict__ invd) {
  const Grid& g = op.g;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nn; n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_ijk<DIM>(g, n, i, j, k);
    const int cx = (i > 0) + (i < g.ex), cy = (j > 0) + (j < g.ey), cz = DIM == 3 ? (k > 0) + (k < g.ez) : 1;
    invd[n] = 1.0 / (op.a[0] * cx * cy * cz);
  }
}

template <typename T>
struct HelmArgs {
  HelmOp op;
  const T* b;
  T* x;
  T* r;
  T* z;
  T* p0;
  T* p1;
  T* q;
  const T* invd;
  double* part;
  GridBar* bar;
  HelmStatus* st;
  double tol2;
  int max_it;
};

// Jacobi-PCG on the nodal system from x = 0, vectors and operator in T (FP64,
// or FP32 for the inner solves of the refinement loop), dot products summed
// in FP64; stops when ||r|| <= sqrt(tol2) ||b||, at max_it, or on breakdown.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) helm_pcg_kernel(const __grid_constant__ HelmArgs<T> a) {
  __shared__ double sred[32 * kHelmSlots];
  __shared__ double stot[kHelmSlots];
  unsigned char* sm = reinterpret_cast<unsigned char*>(sred);
  const Grid& g = a.op.g;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nb = gridDim.x;
  unsigned gen = 0;
  bool ok = true;
  // totals of NV partials of the slot starting at value s0 into stot[s0 ..]
  auto totals = [&](int s0, int nv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < nv) {
      double t = 0.0;
      for (int b = lane; b < nb; b += 32) t += __ldcg(a.part + (size_t)(s0 + warp) * nb + b);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) stot[s0 + warp] = t;
    }
    __syncthreads();
  };
  // start from x = 0: r = b, z = D^-1 r
  {
    double acc[2] = {0.0, 0.0};
    for (long long n = first; n < g.nn; n += stride) {
      const T rv = a.b[n], zv = a.invd[n] * rv;
      a.x[n] = T(0);
      a.r[n] = rv;
      a.z[n] = zv;
      acc[0] = fma((double)rv, (double)zv, acc[0]);
      acc[1] = fma((double)rv, (double)rv, acc[1]);
    }
    block_partial_d<2>(acc, a.part + (size_t)1 * nb, sm);
    ok = grid_sync(a.bar, gen);
    totals(1, 2);
  }
  double rz = stot[1], bb = stot[2], beta = 0.0, rr = bb;
  int it = 0, pbuf = 0;
  while (ok && !(rr <= a.tol2 * bb) && it < a.max_it && bb > 0.0) {
    const T* Pold = pbuf ? a.p1 : a.p0;
    T* Pnew = pbuf ? a.p0 : a.p1;
    const T bt = (T)beta;
    // p = z + beta p_old (formed at every neighbour), q = A p, partial p.q
    double acc[1] = {0.0};
    for (long long n = first; n < g.nn; n += stride) {
      int i, j, k;
      node_ijk<DIM>(g, n, i, j, k);
      const T qv = helm_row<DIM, T>(a.op, i, j, k, [&](long long m) {
        const T zm = __ldcg(a.z + m);
        return bt != T(0) ? fma(bt, __ldcg(Pold + m), zm) : zm;
      });
      const T zn = __ldcg(a.z + n);
      const T pn = bt != T(0) ? fma(bt, __ldcg(Pold + n), zn) : zn;
      Pnew[n] = pn;
      a.q[n] = qv;
      acc[0] = fma((double)pn, (double)qv, acc[0]);
    }
    block_partial_d<1>(acc, a.part, sm);
    if (!(ok = grid_sync(a.bar, gen))) break;
    totals(0, 1);
    const double pq = stot[0];
    if (!(pq > 0.0) || !isfinite(pq)) break;
    const double alpha = rz / pq;
    const T al = (T)alpha;
    // x += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r
    double acc2[2] = {0.0, 0.0};
    for (long long n = first; n < g.nn; n += stride) {
      const T rv = fma(-al, a.q[n], a.r[n]);
      const T zv = a.invd[n] * rv;
      a.x[n] = fma(al, Pnew[n], a.x[n]);
      a.r[n] = rv;
      a.z[n] = zv;
      acc2[0] = fma((double)rv, (double)zv, acc2[0]);
      acc2[1] = fma((double)rv, (double)rv, acc2[1]);
    }
    block_partial_d<2>(acc2, a.part + (size_t)1 * nb, sm);
    if (!(ok = grid_sync(a.bar, gen))) break;
    totals(1, 2);
    const double rzn = stot[1];
    rr = stot[2];
    beta = rzn / rz;
    rz = rzn;
    it++;
    pbuf ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->it = it;
    a.st->rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.st->flags = (ok ? 0 : ERR_TIMEOUT) | ((rr <= a.tol2 * bb || bb == 0.0) ? 0 : ERR_BREAKDOWN);
  }
}

// FP64 residual of the refinement loop: r32 = (float)(b - A x) and per-CTA
// partials of ||b - A x||^2 and ||b||^2 (part[2 cta], part[2 cta + 1]).
template <int DIM>
__global__ void __launch_bounds__(256) helm_residual_kernel(HelmOp op, const double* __restrict__ b,
                                                            const double* __restrict__ x, float* __restrict__ r32,
                                                            double* __restrict__ part) {
  __shared__ double sm[32 * 2];
  const Grid& g = op.g;
  double acc[2] = {0.0, 0.0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nn; n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_ijk<DIM>(g, n, i, j, k);
    const double ax = helm_row<DIM, double>(op, i, j, k, [&](long long m) { return x[m]; });
    const double rv = b[n] - ax;
    r32[n] = (float)rv;
    acc[0] = fma(rv, rv, acc[0]);
    acc[1] = fma(b[n], b[n], acc[1]);
  }
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = acc[0];
    part[2 * blockIdx.x + 1] = acc[1];
  }
}

// The two norms: the CTA partials summed in a fixed order by one thread.
__global__ void helm_norms_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = 0; b < nb; b++) {
    s0 += part[2 * b];
    s1 += part[2 * b + 1];
  }
  out[0] = s0;
  out[1] = s1;
}

// x += (double) d (after an FP32 inner solve).
__global__ void helm_merge_kernel(long long n, double* __restrict__ x, const float* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

__global__ void helm_invd32_kernel(long long n, const double* __restrict__ invd, float* __restrict__ invd32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    invd32[i] = (float)invd[i];
}

int grid_of(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

// Scratch layout (helm_scratch_doubles doubles): FP64 right-hand side b and
// iterate x, then eight FP32 node arrays (inner right-hand side r32, inner
// iterate d, r, z, p0, p1, q, FP32 inverse diagonal), the FP64 inverse
// diagonal in the last n_nodes doubles.
struct HelmBufs {
  double *b, *x, *invd;
  float *r32, *d, *r, *z, *p0, *p1, *q, *invd32;
};
HelmBufs helm_bufs(const Grid& g, double* scratch) {
  const long long nn = g.nn;
  HelmBufs h;
  h.b = scratch;
  h.x = scratch + nn;
  float* f = reinterpret_cast<float*>(scratch + 2 * nn);
  h.r32 = f;
  h.d = f + nn;
  h.r = f + 2 * nn;
  h.z = f + 3 * nn;
  h.p0 = f + 4 * nn;
  h.p1 = f + 5 * nn;
  h.q = f + 6 * nn;
  h.invd32 = f + 7 * nn;
  h.invd = scratch + 7 * nn;
  return h;
}

}  // namespace

void helm_coefficients(int dim, double R, double* a) {
  const double r2 = R * R;
  if (dim == 2) {
    const double K[3] = {4.0 / 6, -1.0 / 6, -2.0 / 6}, M[3] = {4.0 / 36, 2.0 / 36, 1.0 / 36};
    for (int h = 0; h < 3; h++) a[h] = r2 * K[h] + M[h];
    a[3] = 0.0;
  } else {
    const double K[4] = {4.0 / 12, 0.0, -1.0 / 12, -1.0 / 12}, M[4] = {8.0 / 216, 4.0 / 216, 2.0 / 216, 1.0 / 216};
    for (int h = 0; h < 4; h++) a[h] = r2 * K[h] + M[h];
  }
}

size_t helm_scratch_doubles(const Grid& g) { return (size_t)g.nn * 8; }

cudaError_t launch_helm_setup(cudaStream_t s, const Grid& g, const double* a, double* scratch) {
  HelmOp op;
  op.g = g;
  for (int h = 0; h < 4; h++) op.a[h] = a[h];
  const HelmBufs hb = helm_bufs(g, scratch);
  if (g.dim == 2) helm_diag_kernel<2><<<grid_of(g.nn), 256, 0, s>>>(op, hb.invd);
  else helm_diag_kernel<3><<<grid_of(g.nn), 256, 0, s>>>(op, hb.invd);
  helm_invd32_kernel<<<grid_of(g.nn), 256, 0, s>>>(g.nn, hb.invd, hb.invd32);
  return cudaGetLastError();
}

// One FP64 Jacobi-PCG solve of the whole nodal system (the FP64 path: in 2D
// it is shorter than the refinement passes and their synchronisations).
static cudaError_t helm_filter_fp64(cudaStream_t s, const Grid& g, const double* a, const double* in, double* out,
                                    double* scratch, double* part, GridBar* bar, HelmStatus* st, double tol,
                                    int max_it, int nsm) {
  const long long nn = g.nn;
  HelmArgs<double> h;
  h.op.g = g;
  for (int k = 0; k < 4; k++) h.op.a[k] = a[k];
  // FP64 vectors over the scratch: b, x, then r, z, p0, p1, q in doubles
  // 2 .. 6 (the FP32 region of the refinement path), the inverse diagonal last
  h.b = scratch;
  h.x = scratch + nn;
  h.r = scratch + 2 * nn;
  h.z = scratch + 3 * nn;
  h.p0 = scratch + 4 * nn;
  h.p1 = scratch + 5 * nn;
  h.q = scratch + 6 * nn;
  h.invd = scratch + 7 * nn;
  h.part = part;
  h.bar = bar;
  h.st = st;
  h.tol2 = tol * tol;
  h.max_it = max_it;
  if (g.dim == 2) helm_rhs_kernel<2><<<grid_of(nn), 256, 0, s>>>(g, in, scratch);
  else helm_rhs_kernel<3><<<grid_of(nn), 256, 0, s>>>(g, in, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  auto kern = g.dim == 2 ? helm_pcg_kernel<2, double> : helm_pcg_kernel<3, double>;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = (int)std::min<long long>((long long)std::min(per_sm, 2) * nsm, std::max<long long>((nn + 255) / 256, 1));
  void* args[] = {(void*)&h};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, s);
  if (e != cudaSuccess) return e;
  if (g.dim == 2) helm_mean_kernel<2><<<grid_of(g.ne), 256, 0, s>>>(g, h.x, out);
  else helm_mean_kernel<3><<<grid_of(g.ne), 256, 0, s>>>(g, h.x, out);
  return cudaGetLastError();
}

cudaError_t launch_helm_filter(cudaStream_t s, const Grid& g, const double* a, const double* in, double* out,
                               double* scratch, double* part, GridBar* bar, HelmStatus* st, double tol, int max_it,
                               int nsm) {
  // 3D: FP64 iterative refinement around FP32 Jacobi-PCG solves: r = b - A x
  // in FP64; A d = r in FP32 to 1e-5 of ||r|| (the system is well
  // conditioned: R^2 K_F + M_F, a mass term on the diagonal); x += d; until
  // ||b - A x|| <= tol ||b|| in FP64.  Synchronises the stream once per pass.
  // 2D: one FP64 solve.
  if (g.dim == 2) return helm_filter_fp64(s, g, a, in, out, scratch, part, bar, st, tol, max_it, nsm);
  const long long nn = g.nn;
  const HelmBufs hb = helm_bufs(g, scratch);
  HelmOp op;
  op.g = g;
  for (int k = 0; k < 4; k++) op.a[k] = a[k];
  HelmArgs<float> h;
  h.op = op;
  h.b = hb.r32;
  h.x = hb.d;
  h.r = hb.r;
  h.z = hb.z;
  h.p0 = hb.p0;
  h.p1 = hb.p1;
  h.q = hb.q;
  h.invd = hb.invd32;
  h.part = part;
  h.bar = bar;
  h.st = st;
  h.tol2 = 1e-10;  // inner: ||r_inner|| <= 1e-5 ||r||
  h.max_it = max_it;
  if (g.dim == 2) helm_rhs_kernel<2><<<grid_of(nn), 256, 0, s>>>(g, in, hb.b);
  else helm_rhs_kernel<3><<<grid_of(nn), 256, 0, s>>>(g, in, hb.b);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(hb.x, 0, nn * sizeof(double), s);
  if (e != cudaSuccess) return e;
  auto kern = g.dim == 2 ? helm_pcg_kernel<2, float> : helm_pcg_kernel<3, float>;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = (int)std::min<long long>((long long)std::min(per_sm, 2) * nsm, std::max<long long>((nn + 255) / 256, 1));
  const int rgrid = grid_of(nn);
  double* norms = part + 2 * rgrid;  // after the residual partials
  HelmStatus total{0, 0, 1.0};
  for (int pass = 0; pass < 12; pass++) {
    if (g.dim == 2) helm_residual_kernel<2><<<rgrid, 256, 0, s>>>(op, hb.b, hb.x, hb.r32, part);
    else helm_residual_kernel<3><<<rgrid, 256, 0, s>>>(op, hb.b, hb.x, hb.r32, part);
    helm_norms_kernel<<<1, 32, 0, s>>>(part, rgrid, norms);
    double hn[2] = {0.0, 0.0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    total.rel = hn[1] > 0.0 ? std::sqrt(hn[0] / hn[1]) : 0.0;
    if (!(hn[0] > tol * tol * hn[1])) break;  // converged (or a zero right-hand side)
    if (pass == 11) {
      total.flags |= ERR_BREAKDOWN;  // not converged within the passes
      break;
    }
    e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
    void* args[] = {(void*)&h};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, s);
    if (e == cudaSuccess) {
      helm_merge_kernel<<<grid_of(nn), 256, 0, s>>>(nn, hb.x, hb.d);
      e = cudaGetLastError();
    }
    HelmStatus in_st;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&in_st, st, sizeof(in_st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    total.it += in_st.it;
    if (in_st.flags & ERR_TIMEOUT) {
      total.flags |= ERR_TIMEOUT;
      break;
    }
  }
  e = cudaMemcpyAsync(st, &total, sizeof(total), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (g.dim == 2) helm_mean_kernel<2><<<grid_of(g.ne), 256, 0, s>>>(g, hb.x, out);
  else helm_mean_kernel<3><<<grid_of(g.ne), 256, 0, s>>>(g, hb.x, out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // `total` is read by the copy above
  return e;
}

}  // namespace tp
