// OC update for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc / cudaFree at the time
// they want to update densities.  Examples: a host framework whose allocator has
// already reserved the device memory budget, a plugin environment that forbids
// device allocations after start-up, or a tight optimisation loop that must not
// pay for an allocation or for the device-wide synchronisation that cudaFree can
// cause.  tp_oc_update_noalloc serves them: it runs the same OC kernel as
// tp_oc_update, but its scratch memory (the per-element term rho * sqrt(-dc~),
// the per-CTA partial sums, the grid-barrier word and the status record) lives in
// one file-scope device array, sized below, that every GPU which loads this
// library holds until the process exits.  The caller provides only the inputs
// and the output density buffer.
#include <mutex>

#include "../../include/topo.h"
#include "host.h"

namespace {

using tp::GridBar;
using tp::OcStatus;

constexpr long long kMaxElems = TP_NOALLOC_MAX_ELEMENTS;  // per-element scratch capacity
constexpr int kMaxCtas = 512;                             // CTAs whose partial sums fit
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffB = 0;
constexpr size_t kOffPart = round_up(kOffB + (size_t)kMaxElems * sizeof(double));
constexpr size_t kOffBar = round_up(kOffPart + (size_t)tp::oc_part_doubles(kMaxCtas) * sizeof(double));
constexpr size_t kOffStatus = round_up(kOffBar + sizeof(GridBar));
constexpr size_t kScratchBytes = round_up(kOffStatus + sizeof(OcStatus));  // about 8.3 MB

// The scratch array.  In host code its name is only a host-side stand-in; the
// device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_oc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_oc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tp_status tp_oc_update_noalloc(const double* rho, const double* dcf, const int8_t* passive,
                                          long long n_el, double volfrac, double move, double dmin,
                                          double* rho_new, void* cuda_stream, double* lambda,
                                          double* volume, double* change) {
  if (!rho || !dcf || !rho_new) return TP_ERR_ARG;
  if (n_el < 1 || n_el > kMaxElems) return TP_ERR_ARG;  // beyond the scratch capacity
  if (!(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0) || !(dmin > 0.0 && dmin < 1.0)) return TP_ERR_ARG;
  if (rho_new == rho || rho_new == dcf) return TP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return TP_ERR_CUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  double* bscr = reinterpret_cast<double*>(b + kOffB);
  double* part = reinterpret_cast<double*>(b + kOffPart);
  GridBar* bar = reinterpret_cast<GridBar*>(b + kOffBar);
  OcStatus* st = reinterpret_cast<OcStatus*>(b + kOffStatus);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the barrier word starts every launch at zero (the array keeps the last call's contents)
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  int grid = 0;
  if (e == cudaSuccess)
    e = tp::launch_oc(s, n_el, rho, dcf, passive, volfrac, move, dmin, rho_new, bscr, part, bar, st, nsm, &grid,
                      kMaxCtas);
  OcStatus hs;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TP_ERR_CUDA;
  }
  if (hs.flags & tp::ERR_TIMEOUT) return TP_ERR_TIMEOUT;
  if (hs.flags & tp::ERR_NAN) return TP_ERR_ARG;
  if (lambda) *lambda = hs.lambda;
  if (volume) *volume = hs.volume;
  if (change) *change = hs.change;
  return TP_OK;
}
