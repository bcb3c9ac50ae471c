// fluid19.cu -- launchers of the fluid kernel on the D3Q19 lattice without solids
// (with or without a body force, FP32 or 16-bit storage, and the fluid pass of
// the mixed-precision scheme): the kernel of fluid_kernel.cuh with Q19 = true.
// The instantiations with the boundary tables are in fluid19_bnd.cu.
#include "fluid_kernel.cuh"

namespace melbm {

cudaError_t launch_fluid19(int storage, int nx, int ny, int nz, const void* in, void* out,
                           const float* force, float omega, uint32_t t_out, uint32_t seed,
                           const QGrids& grids, const BoundaryTables* bt, cudaStream_t st,
                           uint32_t* fault, int stall_test) {
  if (bt && bt->solid)
    return launch_fluid19_bnd(storage, nx, ny, nz, in, out, force, omega, t_out, seed, grids, bt,
                              st);
  return launch_fluid_impl<true, false>(storage, nx, ny, nz, in, out, force, omega, t_out, seed,
                                        grids, nullptr, st, fault, stall_test);
}

cudaError_t launch_fluid_mixed19(int nx, int ny, int nz, const void* q_in, float* p_out,
                                 cudaStream_t st) {
  return launch_fluid_mixed_impl<true>(nx, ny, nz, q_in, p_out, st);
}

}  // namespace melbm
