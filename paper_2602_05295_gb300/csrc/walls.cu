// walls.cu -- the force and torque the fluid exerts on a solid body (Sec. 3.2,
// solid coupling: the contributions of every node whose links meet the solid are
// summed).  By momentum exchange a solid link i of listed cell x transfers
// -c_i (f_in + f_out) to the solid per step: f_out = f+_{opp(i)}(x), the
// post-collision population leaving x towards the wall, and f_in the population
// the wall returns (f_out again for halfway bounce-back; the reconstruction at the
// moving wall for the moment-based model).  The torque about the body's r0 adds
// (p - r0) x that, p the link's halfway point.  Accumulated in FP64 per thread,
// then per block, then by one block over the block partials in a fixed order.
// On D3Q19 the links, weights and populations are those of the 19-velocity lattice.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr uint32_t D3Q19_LINK_BITS = 0x2EBFEBAu;  // bits i with |c_i|^2 <= 2
constexpr int SF_THREADS = 256;
constexpr int SF_BLOCKS = 608;  // 4 per SM on a 152-SM part

int solid_force_blocks() { return SF_BLOCKS; }

struct SolidForceParams {
  int nx, ny, nz;
  const void* in;
  const float* force;
  float omega;
  const uint32_t* cells;
  const uint32_t* words;
  int64_t count;
  QGrids q;
  int wall_model;
  const uint8_t* mask;
  const float* bodies;
  int body;
  double* partials;
};

template <int STORAGE, bool FORCE, bool Q19>
__global__ void __launch_bounds__(SF_THREADS) solid_force_kernel(SolidForceParams P) {
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t k = int64_t(blockIdx.x) * SF_THREADS + threadIdx.x; k < P.count;
       k += int64_t(gridDim.x) * SF_THREADS) {
    const uint32_t word = P.words[k];
    const uint32_t links = word & 0x7FFFFFFu;
    if ((word >> 27) != T_FLUID_BOUNDARY || !links) continue;
    const uint32_t n = P.cells[k];
    int x, y, z;
    cell_xyz(n, nx, ny, &x, &y, &z);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (FORCE) {
      fx = P.force[n];
      fy = P.force[N + n];
      fz = P.force[2 * N + n];
    }
    const Mom17 A = collide_moments<FORCE>(load_stored<STORAGE>(P.in, N, n, P.q), P.omega, fx, fy, fz);
    // each thread over its own solid links (D3Q19 has no corner links)
    uint32_t lk = Q19 ? (links & D3Q19_LINK_BITS) : links;
    while (lk) {
      const int i = __ffs(lk) - 1;
      lk &= lk - 1u;
      const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
      const int b = P.mask[pull_source(x, y, z, nx, ny, nz, i)];
      if (P.body && b != P.body) continue;
      // the weight of i = that of opp(i)
      const float w = Q19 ? lattice_weight19(cx, cy, cz) : lattice_weight(cx, cy, cz);
      const float px = x - 0.5f * cx, py = y - 0.5f * cy, pz = z - 0.5f * cz;
      const float g_out = Q19 ? hermite_eval19(A, -cx, -cy, -cz) : hermite_eval(A, -cx, -cy, -cz);
      const double f_out = double(w) * (1.0 + double(g_out));
      double f_in = f_out;
      if (P.wall_model == 1) {
        float up[3];
        body_velocity(P.bodies, b, px, py, pz, up);
        const Mom17 Wm = wall_moments(A, up[0], up[1], up[2]);
        const float g_in = Q19 ? hermite_eval19(Wm, cx, cy, cz) : hermite_eval(Wm, cx, cy, cz);
        f_in = double(w) * (1.0 + double(g_in));
      }
      const double s = f_in + f_out;
      const double dF[3] = {-cx * s, -cy * s, -cz * s};
      const float* t = P.bodies + 9 * (P.body ? P.body : b);
      const double r[3] = {double(px) - t[6], double(py) - t[7], double(pz) - t[8]};
      acc[0] += dF[0];
      acc[1] += dF[1];
      acc[2] += dF[2];
      acc[3] += r[1] * dF[2] - r[2] * dF[1];
      acc[4] += r[2] * dF[0] - r[0] * dF[2];
      acc[5] += r[0] * dF[1] - r[1] * dF[0];
    }
  }
  __shared__ double sm[6][SF_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if (lane == 0) sm[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int w = 0; w < SF_THREADS / 32; ++w) t += sm[threadIdx.x][w];
    P.partials[size_t(blockIdx.x) * 6 + threadIdx.x] = t;
  }
}

__global__ void solid_force_final_kernel(const double* partials, int nblocks, double* out) {
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[size_t(b) * 6 + threadIdx.x];
    out[threadIdx.x] = t;
  }
}

cudaError_t launch_solid_force(int storage, int nx, int ny, int nz, const void* in,
                               const float* force, float omega, const uint32_t* cells,
                               const uint32_t* words, int64_t count, const QGrids& q,
                               int wall_model, const uint8_t* mask, const float* bodies, int body,
                               double* partials, double* out, int lattice, cudaStream_t st) {
  SolidForceParams p;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = in;
  p.force = force;
  p.omega = omega;
  p.cells = cells;
  p.words = words;
  p.count = count;
  p.q = q;
  p.wall_model = wall_model;
  p.mask = mask;
  p.bodies = bodies;
  p.body = body;
  p.partials = partials;
  if (lattice == 19) {
    if (storage == ST_Q16) {
      if (force) solid_force_kernel<ST_Q16, true, true><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
      else solid_force_kernel<ST_Q16, false, true><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
    } else {
      if (force) solid_force_kernel<ST_F32, true, true><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
      else solid_force_kernel<ST_F32, false, true><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
    }
  } else if (storage == ST_Q16) {
    if (force) solid_force_kernel<ST_Q16, true, false><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
    else solid_force_kernel<ST_Q16, false, false><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
  } else {
    if (force) solid_force_kernel<ST_F32, true, false><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
    else solid_force_kernel<ST_F32, false, false><<<SF_BLOCKS, SF_THREADS, 0, st>>>(p);
  }
  solid_force_final_kernel<<<1, 32, 0, st>>>(partials, SF_BLOCKS, out);
  return cudaGetLastError();
}

}  // namespace melbm
