// fluid19.cu -- launchers of the fluid kernel on the D3Q19 lattice (with or
// without a body force, FP32 or 16-bit storage, and the fluid pass of the
// mixed-precision scheme): the kernel of fluid_kernel.cuh with Q19 = true.
#include "fluid_kernel.cuh"

namespace melbm {

cudaError_t launch_fluid19(int storage, int nx, int ny, int nz, const void* in, void* out,
                           const float* force, float omega, uint32_t t_out, uint32_t seed,
                           const QGrids& grids, cudaStream_t st) {
  FluidParams p;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = in;
  p.out = out;
  p.force = force;
  p.omega = omega;
  p.t_out = t_out;
  p.seed = seed;
  p.chunk16 = nx % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(force) % 16 == 0;
  if (storage == ST_Q16 && !qgrids_16(grids)) {
    KernelParams<ST_Q16, true> q;
    static_cast<FluidParams&>(q) = p;
    q.q = grids;
    return force ? launch_fluid_t<ST_Q16, true, true, true>(q, st)
                 : launch_fluid_t<ST_Q16, false, true, true>(q, st);
  }
  if (storage == ST_Q16) {
    KernelParams<ST_Q16, false> q;
    static_cast<FluidParams&>(q) = p;
    return force ? launch_fluid_t<ST_Q16, true, false, true>(q, st)
                 : launch_fluid_t<ST_Q16, false, false, true>(q, st);
  }
  if (storage != ST_F32) return cudaErrorInvalidValue;
  KernelParams<ST_F32, false> q;
  static_cast<FluidParams&>(q) = p;
  const size_t N = size_t(nx) * ny * nz;
  for (int k = 0; k < 10; ++k) {
    q.in_w[k] = static_cast<const uint32_t*>(in) + k * N;
    q.out_w[k] = static_cast<uint32_t*>(out) + k * N;
  }
  for (int k = 0; k < 3; ++k)
    q.f_w[k] = force ? reinterpret_cast<const uint32_t*>(force) + k * N : nullptr;
  return force ? launch_fluid_t<ST_F32, true, false, true>(q, st)
               : launch_fluid_t<ST_F32, false, false, true>(q, st);
}

// The fluid pass of the mixed-precision scheme on D3Q19 (16-bit post-collision
// moments in, raw FP32 post-streaming sums out; see launch_fluid_mixed).
cudaError_t launch_fluid_mixed19(int nx, int ny, int nz, const void* q_in, float* p_out,
                                 cudaStream_t st) {
  KernelParams<ST_MIXED, false> k;
  FluidParams& p = k;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = q_in;
  p.out = p_out;
  p.force = nullptr;
  p.omega = 0.0f;
  p.t_out = 0;
  p.seed = 0;
  p.chunk16 = 0;
  const size_t N = size_t(nx) * ny * nz;
  for (int w = 0; w < 10; ++w) k.out_w[w] = reinterpret_cast<uint32_t*>(p_out) + w * N;
  return launch_fluid_t<ST_MIXED, false, false, true>(k, st);
}

}  // namespace melbm
