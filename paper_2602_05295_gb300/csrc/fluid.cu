// fluid.cu -- the fluid-interior kernel of the split design (Sec. 4.2, Alg. 2):
// one uniform, branch-free update of every cell:
//   load stored moments -> collide (App. A) -> Hermite coefficients of f+
//   (Eq. three_order_f) -> pull stream (Eq. streaming) -> moments (Eq. rho_u_stress)
//   -> store (FP32, or 16-bit with dither, Sec. 5.4).
// Boundary cells are overwritten afterwards by the boundary kernel; the stream
// here is periodic in all three directions.
//
// Streaming and moment recovery are done separably: the populations of D3Q27 are
// the tensor product of three D1Q3 sets, so "pull f_i from x - c_i, then take
// moments" factors into three 1D passes (x, then y, then z) on the Hermite
// moments of f+, each a 3-point stencil.  Only the moments that can reach the
// ten output moments are carried: 17 -> 24 after x, -> 18 after y, -> 10 after z.
//
// Work decomposition (one thread per (x, y) column, marching along z):
//   * a block is 32 lanes (x) by FY warps (y); lanes cover x0-1 .. x0+30 and warps
//     y0-1 .. y0+FY-2, so lanes 0/31 and warps 0/FY-1 are a recomputed halo ring;
//   * the x pass exchanges directional populations with warp shuffles;
//   * the y pass exchanges them through double-buffered shared memory (one
//     barrier per plane);
//   * the z pass keeps the previous planes' populations in registers.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr int FX = 32;
constexpr int FY = 16;
constexpr int FXI = FX - 2;
constexpr int FYI = FY - 2;
constexpr int NSY = 9;  // y-pass slices exchanged through shared memory
constexpr int SM_PLANE = 2 * NSY * FY * FX;  // floats per buffer (phi+ and phi-)

struct FluidParams {
  int nx, ny, nz, zc;
  const void* in;
  void* out;
  const float* force;
  float omega;
  uint32_t t_out, seed;
};

// The y-pass slices are indexed s = 3 p + r' (p: x-order, r': input z-order).
template <int STORAGE, bool FORCE>
__global__ void __launch_bounds__(FX* FY, 1) fluid_kernel(FluidParams P) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x, row = threadIdx.y;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz;
  const int x = int(blockIdx.x) * FXI - 1 + lane;
  const int y = int(blockIdx.y) * FYI - 1 + row;
  const int xw = wrapi(x, nx), yw = wrapi(y, ny);
  const bool mid_row = (row >= 1 && row <= FY - 2);  // warp-uniform
  const bool do_store = mid_row && lane >= 1 && lane <= FX - 2 && x < nx && y < ny;
  const int z0 = int(blockIdx.z) * P.zc;
  const int z1 = min(z0 + P.zc, nz);
  const size_t col = size_t(xw) + size_t(nx) * yw;
  const size_t plane = size_t(nx) * ny;
  const float omega = P.omega;

  // z-march state for the six (p, q) slices: phi+ of plane z-1, phi0 and phi+ of z
  float zpm[6], zp0[6], zpp[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) zpm[k] = zp0[k] = zpp[k] = 0.f;
  float fprev[3] = {0.f, 0.f, 0.f};

  int parity = 0;
  for (int zz = z0 - 1; zz <= z1; ++zz, parity ^= 1) {
    const int zw = wrapi(zz, nz);
    const size_t n = col + plane * zw;
    const Stored s = load_stored<STORAGE>(P.in, N, n);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (FORCE) {
      fx = __ldg(P.force + n);
      fy = __ldg(P.force + N + n);
      fz = __ldg(P.force + 2 * N + n);
    }
    const Mom17 A = collide_moments<FORCE>(s, omega, fx, fy, fz);

    // ---------------- x pass: slices (q', r'), inputs p' = 0, 1, 2 -> outputs p = 0, 1, 2
    float X[3][3][3];  // X[p][q'][r'] (only the 24 reachable entries are set/used)
#define MELBM_XPASS(Q, R, A0, A1, A2)                                   \
  {                                                                     \
    const Phi ph = phi3(A0, A1, A2);                                    \
    const float pl = __shfl_up_sync(FULL, ph.p, 1);                     \
    const float mr = __shfl_down_sync(FULL, ph.m, 1);                   \
    X[0][Q][R] = proj0(pl, ph.z, mr);                                   \
    X[1][Q][R] = proj1(pl, mr);                                         \
    X[2][Q][R] = proj2(pl, mr, X[0][Q][R]);                               \
  }
    MELBM_XPASS(0, 0, A.m000, A.m100, A.m200)
    MELBM_XPASS(1, 0, A.m010, A.m110, A.m210)
    MELBM_XPASS(0, 1, A.m001, A.m101, A.m201)
    MELBM_XPASS(2, 0, A.m020, A.m120, 0.f)
    MELBM_XPASS(0, 2, A.m002, A.m102, 0.f)
    MELBM_XPASS(1, 1, A.m011, A.m111, 0.f)
    MELBM_XPASS(2, 1, A.m021, 0.f, 0.f)
    MELBM_XPASS(1, 2, A.m012, 0.f, 0.f)
#undef MELBM_XPASS
    X[2][2][2] = 0.f;  // (q', r') = (2, 2) has no input coefficient
    X[0][2][2] = X[1][2][2] = 0.f;

    // ---------------- y pass, part 1: directional populations along y
    float* sp = smem + parity * SM_PLANE;
    float yz0[NSY];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const Phi ph = phi3(X[p][0][r], X[p][1][r], X[p][2][r]);
        const int s_ = 3 * p + r;
        sp[(s_ * FY + row) * FX + lane] = ph.p;
        sp[((NSY + s_) * FY + row) * FX + lane] = ph.m;
        yz0[s_] = ph.z;
      }
    __syncthreads();
    if (!mid_row) continue;  // halo rows only feed their neighbours

    // ---------------- y pass, part 2: pull and project -> Y[p][q][r'], q <= 2 - p
    float Y[3][3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int s_ = 3 * p + r;
        const float pl = sp[(s_ * FY + row - 1) * FX + lane];
        const float mr = sp[((NSY + s_) * FY + row + 1) * FX + lane];
        Y[p][0][r] = proj0(pl, yz0[s_], mr);
        if (p <= 1) Y[p][1][r] = proj1(pl, mr);
        if (p == 0) Y[p][2][r] = proj2(pl, mr, Y[p][0][r]);
      }

    // ---------------- z pass: directional populations along z for slices (p, q)
    const int PQ[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    float zm[6], z0n[6], zpn[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int p = PQ[k][0], q = PQ[k][1];
      const Phi ph = phi3(Y[p][q][0], Y[p][q][1], Y[p][q][2]);
      zm[k] = ph.m;
      z0n[k] = ph.z;
      zpn[k] = ph.p;
    }
    if (zz >= z0 + 1) {
      // finish plane zz-1 from phi+(zz-2), phi0(zz-1), phi-(zz)
      float M[6][3];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        M[k][0] = proj0(zpm[k], zp0[k], zm[k]);
        M[k][1] = proj1(zpm[k], zm[k]);
        M[k][2] = proj2(zpm[k], zm[k], M[k][0]);
      }
      // slices: 0:(0,0) 1:(1,0) 2:(0,1) 3:(2,0) 4:(1,1) 5:(0,2)
      const Stored o = finish_moments<FORCE>(M[0][0], M[1][0], M[2][0], M[0][1], M[3][0], M[5][0],
                                             M[0][2], M[4][0], M[1][1], M[2][1], fprev[0],
                                             fprev[1], fprev[2]);
      if (do_store) {
        const int zo = zz - 1;
        store_stored<STORAGE>(P.out, N, col + plane * zo, o, uint32_t(xw), uint32_t(yw),
                              uint32_t(zo), P.t_out, P.seed);
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      zpm[k] = zpp[k];
      zp0[k] = z0n[k];
      zpp[k] = zpn[k];
    }
    if (FORCE) {
      fprev[0] = fx;
      fprev[1] = fy;
      fprev[2] = fz;
    }
  }
}

template <int STORAGE, bool FORCE>
static cudaError_t launch_fluid_t(const FluidParams& p, dim3 grid, cudaStream_t st) {
  const size_t smem = size_t(2) * SM_PLANE * sizeof(float);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fluid_kernel<STORAGE, FORCE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  fluid_kernel<STORAGE, FORCE><<<grid, dim3(FX, FY), smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fluid(int storage, int nx, int ny, int nz, const void* in, void* out,
                         const float* force, float omega, uint32_t t_out, uint32_t seed,
                         cudaStream_t st) {
  FluidParams p;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.zc = nz < 32 ? nz : 32;
  p.in = in;
  p.out = out;
  p.force = force;
  p.omega = omega;
  p.t_out = t_out;
  p.seed = seed;
  dim3 grid((nx + FXI - 1) / FXI, (ny + FYI - 1) / FYI, (nz + p.zc - 1) / p.zc);
  if (storage == ST_Q16)
    return force ? launch_fluid_t<ST_Q16, true>(p, grid, st) : launch_fluid_t<ST_Q16, false>(p, grid, st);
  return force ? launch_fluid_t<ST_F32, true>(p, grid, st) : launch_fluid_t<ST_F32, false>(p, grid, st);
}

}  // namespace melbm
