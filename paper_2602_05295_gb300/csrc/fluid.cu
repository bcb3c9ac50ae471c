// fluid.cu -- launchers of the D3Q27 fluid-interior kernel (fluid_kernel.cuh)
// without solids, and of the fluid pass of the mixed-precision scheme.  The
// instantiations with the boundary tables are in fluid_bnd.cu.
#include "fluid_kernel.cuh"

namespace melbm {

cudaError_t launch_fluid(int storage, int nx, int ny, int nz, const void* in, void* out,
                         const float* force, float omega, uint32_t t_out, uint32_t seed,
                         const QGrids& grids, const BoundaryTables* bt, cudaStream_t st,
                         uint32_t* fault, int stall_test) {
  if (bt && bt->solid)
    return launch_fluid_bnd(storage, nx, ny, nz, in, out, force, omega, t_out, seed, grids, bt, st);
  return launch_fluid_impl<false, false>(storage, nx, ny, nz, in, out, force, omega, t_out, seed,
                                         grids, nullptr, st, fault, stall_test);
}

cudaError_t launch_fluid_mixed(int nx, int ny, int nz, const void* q_in, float* p_out,
                               cudaStream_t st) {
  return launch_fluid_mixed_impl<false>(nx, ny, nz, q_in, p_out, st);
}

}  // namespace melbm
