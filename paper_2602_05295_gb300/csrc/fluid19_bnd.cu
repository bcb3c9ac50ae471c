// fluid19_bnd.cu -- the D3Q19 fluid kernel with solids (fluid_kernel.cuh, Q19 and
// BND): solid cells enter the passes at rest and the raw sums of the
// FLUID_BOUNDARY cells go to the side table of the boundary kernel.
#include "fluid_kernel.cuh"

namespace melbm {

cudaError_t launch_fluid19_bnd(int storage, int nx, int ny, int nz, const void* in, void* out,
                               const float* force, float omega, uint32_t t_out, uint32_t seed,
                               const QGrids& grids, const BoundaryTables* bt, cudaStream_t st) {
  return launch_fluid_impl<true, true>(storage, nx, ny, nz, in, out, force, omega, t_out, seed,
                                       grids, bt, st);
}

}  // namespace melbm
