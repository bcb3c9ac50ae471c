// mixed.cu -- the paper's own mixed-precision pipeline with solids (Sec. 5.4,
// "Atomic accumulation with mixed precision", and the solid correction kernel of
// Sec. 4.2), kept as a storage mode to compare against the recompute design.
// Two buffers: Q, the post-collision moments in 16 bits (stored variables
// rho - 1, u+, rho (S+ - u+ u+)), and P, the post-streaming raw moments in FP32
// (rho - 1, sum c f, sum (c c - 1/3) f), 60 B per cell.  One step:
//   1. fluid pass (fluid.cu): Q -> stream -> P, periodic, every cell;
//   2. solid correction: every listed FLUID_BOUNDARY cell adds, for its solid
//      links, Delta f_i = f_wall - f_pulled projected on the moments into P with
//      atomicAdd (f_wall = f+_opp(i)(x), halfway bounce-back; f_pulled the
//      population the fluid pass took from the solid cell); INFLOW cells are set
//      to the inflow equilibrium;
//   3. the outflow copy on P;
//   4. buffer copy: P -> moments -> collision (App. A) -> quantise -> Q.
// The public state is P (post-streaming, as in the other modes).  On D3Q19 the
// fluid pass and the correction use the 19-velocity populations.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

// Hermite moments of a stored post-collision state: its stress is traceless, so
// the collision with omega = 0 only rebuilds the moments.
__device__ __forceinline__ Mom17 post_collision_moments(const void* q, size_t N, size_t n) {
  return collide_moments<false>(load_stored<ST_Q16>(q, N, n), 0.0f, 0.f, 0.f, 0.f);
}

template <bool Q19>
__global__ void mixed_correct_kernel(int nx, int ny, int nz, const void* q, float* p,
                                     const uint32_t* cells, const uint32_t* words, int64_t count,
                                     float in_rho, float in_ux, float in_uy, float in_uz) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const size_t N = size_t(nx) * ny * nz;
  const uint32_t n = cells[k];
  const uint32_t word = words[k];
  if ((word >> 27) == T_INFLOW) {
    const float r[10] = {in_rho - 1.0f,       in_rho * in_ux,      in_rho * in_uy,
                         in_rho * in_uz,      in_rho * in_ux * in_ux, in_rho * in_uy * in_uy,
                         in_rho * in_uz * in_uz, in_rho * in_ux * in_uy, in_rho * in_ux * in_uz,
                         in_rho * in_uy * in_uz};
#pragma unroll
    for (int w = 0; w < 10; ++w) p[w * N + n] = r[w];
    return;
  }
  int x, y, z;
  cell_xyz(n, nx, ny, &x, &y, &z);
  const Mom17 self = post_collision_moments(q, N, n);
  float d[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // each thread over its own solid links (D3Q19: the 19 directions with |c|^2 <= 2)
  uint32_t links = word & (Q19 ? 0x2EBFEBAu : 0x7FFFFFFu);
  while (links) {
    const int i = __ffs(links) - 1;
    links &= links - 1u;
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    const Mom17 src = post_collision_moments(q, N, pull_source(x, y, z, nx, ny, nz, i));
    const float df =
        Q19 ? lattice_weight19(cx, cy, cz) *
                  (hermite_eval19(self, -cx, -cy, -cz) - hermite_eval19(src, cx, cy, cz))
            : lattice_weight(cx, cy, cz) *
                  (hermite_eval(self, -cx, -cy, -cz) - hermite_eval(src, cx, cy, cz));
    d[0] += df;
    d[1] += cx * df;
    d[2] += cy * df;
    d[3] += cz * df;
    d[4] += (cx * cx - 1.0f / 3.0f) * df;
    d[5] += (cy * cy - 1.0f / 3.0f) * df;
    d[6] += (cz * cz - 1.0f / 3.0f) * df;
    d[7] += float(cx * cy) * df;
    d[8] += float(cx * cz) * df;
    d[9] += float(cy * cz) * df;
  }
#pragma unroll
  for (int w = 0; w < 10; ++w) atomicAdd(p + w * N + n, d[w]);
}

// P (raw post-streaming sums) -> stored variables -> collision -> Q.
__global__ void mixed_collide_quantize_kernel(int nx, int ny, int nz, const float* p, void* q,
                                              float omega, uint32_t t, uint32_t seed) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Stored s = finish_moments<false>(p[n], p[N + n], p[2 * N + n], p[3 * N + n], p[4 * N + n],
                                         p[5 * N + n], p[6 * N + n], p[7 * N + n], p[8 * N + n],
                                         p[9 * N + n], 0.f, 0.f, 0.f);
  const Mom17 A = collide_moments<false>(s, omega, 0.f, 0.f, 0.f);
  const float rho = 1.0f + A.m000, inv = __frcp_rn(rho);
  Stored o;
  o.drho = A.m000;
  o.ux = A.m100 * inv;
  o.uy = A.m010 * inv;
  o.uz = A.m001 * inv;
  o.nxx = A.m200 - A.m100 * o.ux;
  o.nyy = A.m020 - A.m010 * o.uy;
  o.nzz = A.m002 - A.m001 * o.uz;
  o.nxy = A.m110 - A.m100 * o.uy;
  o.nxz = A.m101 - A.m100 * o.uz;
  o.nyz = A.m011 - A.m010 * o.uz;
  const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
  store_stored<ST_Q16>(q, N, n, o, x, y, z, t, seed);
}

// Public (rho, u, S) -> raw P (S = u u when NULL).
__global__ void mixed_set_state_kernel(int64_t N_, const float* rho, const float* u, const float* S,
                                       float* p) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float r = rho[n], ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  const float s[6] = {S ? S[n] : ux * ux,         S ? S[N + n] : uy * uy,
                      S ? S[2 * N + n] : uz * uz, S ? S[3 * N + n] : ux * uy,
                      S ? S[4 * N + n] : ux * uz, S ? S[5 * N + n] : uy * uz};
  p[n] = r - 1.0f;
  p[N + n] = r * ux;
  p[2 * N + n] = r * uy;
  p[3 * N + n] = r * uz;
#pragma unroll
  for (int k = 0; k < 6; ++k) p[(4 + k) * N + n] = r * s[k];
}

// Raw P -> public (rho, u, S).
__global__ void mixed_get_moments_kernel(int64_t N_, const float* p, float* rho, float* u,
                                         float* S) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float r = 1.0f + p[n], inv = __frcp_rn(r);
  if (rho) rho[n] = r;
  if (u) {
    u[n] = p[N + n] * inv;
    u[N + n] = p[2 * N + n] * inv;
    u[2 * N + n] = p[3 * N + n] * inv;
  }
  if (S) {
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k * N + n] = p[(4 + k) * N + n] * inv;
  }
}

cudaError_t launch_mixed_correct(int nx, int ny, int nz, const void* q, float* p,
                                 const uint32_t* cells, const uint32_t* words, int64_t count,
                                 const float inflow[4], int lattice, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const unsigned blocks = unsigned((count + 127) / 128);
  if (lattice == 19)
    mixed_correct_kernel<true><<<blocks, 128, 0, st>>>(nx, ny, nz, q, p, cells, words, count,
                                                       inflow[0], inflow[1], inflow[2], inflow[3]);
  else
    mixed_correct_kernel<false><<<blocks, 128, 0, st>>>(nx, ny, nz, q, p, cells, words, count,
                                                        inflow[0], inflow[1], inflow[2], inflow[3]);
  return cudaGetLastError();
}

cudaError_t launch_mixed_collide_quantize(int nx, int ny, int nz, const float* p, void* q,
                                          float omega, uint32_t t, uint32_t seed, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  mixed_collide_quantize_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(nx, ny, nz, p, q, omega,
                                                                           t, seed);
  return cudaGetLastError();
}

cudaError_t launch_mixed_set_state(int64_t N, const float* rho, const float* u, const float* S,
                                   float* p, cudaStream_t st) {
  mixed_set_state_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(N, rho, u, S, p);
  return cudaGetLastError();
}

cudaError_t launch_mixed_get_moments(int64_t N, const float* p, float* rho, float* u, float* S,
                                     cudaStream_t st) {
  mixed_get_moments_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(N, p, rho, u, S);
  return cudaGetLastError();
}

}  // namespace melbm
