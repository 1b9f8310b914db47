// 3D instantiations of the persistent CG kernel (separate translation unit
// so the library builds in parallel).
#include "pcg_kernel.cuh"

namespace tp {

cudaError_t launch_pcg3(cudaStream_t s, const PcgLaunch& L, bool f64, int nsm, int* grid_out) {
  return f64 ? pcg_nc<3, double>(s, L, nsm, grid_out) : pcg_nc<3, float>(s, L, nsm, grid_out);
}

}  // namespace tp
