// 2D instantiations of the persistent CG segment kernel (separate translation
// unit so the library builds in parallel).
#include "pcg_kernel.cuh"

namespace tp {

cudaError_t launch_cg_segment2(cudaStream_t s, const Solver& S, bool f64, int nsm, int* grid_out) {
  return f64 ? segment_nc<2, double>(s, S, nsm, grid_out) : segment_nc<2, float>(s, S, nsm, grid_out);
}

}  // namespace tp
