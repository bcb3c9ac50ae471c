// boundary.cu -- the boundary side of the split design (Sec. 4.2): after the
// uniform fluid kernel has written every cell, the listed cells are rewritten.
//   * FLUID_BOUNDARY: with solids the fluid kernel lets solid cells enter the
//     stream at rest (zero post-collision moments about the rest state), so the
//     raw post-streaming sums it leaves for such a cell in the side table hold
//     every population pulled through a non-solid link and nothing through a
//     solid one.  Halfway bounce-back, f_i(x) = f+_{opp(i)}(x) when x - c_i is
//     solid, needs only the cell's own post-collision state: this kernel
//     collides the cell's input state (App. A), adds the bounced population of
//     every solid link to the sums and finishes and stores the moments.  This
//     replaces the paper's additive per-triangle correction (Alg. 3), which needs
//     a mesh; the sums are completed before the single rounding of the 16-bit
//     store, with no atomics.
//     With the moment-based wall model (Sec. 3.2, solid coupling) a solid link
//     instead receives the Hermite population of (rho, u^p, S^p) at the link's
//     halfway point p, u^p the rigid velocity of the body the solid cell
//     belongs to (its mask value) and S^p = u^p u^p + (S - u u) from the cell's
//     own post-collision moments.
//   * INFLOW: reset to the equilibrium (rho_in, u_in, S = u_in u_in).
// The outflow pass then copies the stored state of x = nx-2 onto x = nx-1.
// On the D3Q19 lattice the same update runs over its 19 directions and weights.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

struct BoundaryParams {
  int nx, ny, nz;
  const void* in;
  void* out;
  const float* force;
  float omega;
  const uint32_t* cells;
  const uint32_t* words;
  int64_t count;
  const float* side;       // [count][12]: raw post-streaming sums (FLUID_BOUNDARY entries),
                           // times -1, 2, 2, 2, 1, 1, 1, -4, -4, -4, and two pad floats
  int wall_model;          // 0 halfway bounce-back, 1 moment-based reconstruction
  const uint8_t* mask;     // body id of every cell (wall model 1)
  const float* bodies;     // 256 x 9: V, Om, r0 of each body (wall model 1)
  float in_rho, in_ux, in_uy, in_uz;
  uint32_t t_out, seed;
  QGrids q;
};

// Bits i of the 19 directions with |c|^2 <= 2.
constexpr uint32_t d3q19_links() {
  uint32_t m = 0;
  for (int i = 0; i < 27; ++i) {
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    if (cx * cx + cy * cy + cz * cz <= 2) m |= 1u << i;
  }
  return m;
}
constexpr uint32_t D3Q19_LINKS = d3q19_links();
static_assert(D3Q19_LINKS == 0x2EBFEBAu, "19 directions");

// The halfway bounce-back sums of one D3Q27 cell, all links at once.  With F(c)
// = f+(c) - w(c) the cell's own post-collision populations (rest removed), a
// solid link i returns F(-c_i), so the sums are  sum_{i in S} F(-c_i) e(c_i),
// e = (1, c, c c - 1/3).  Substituting j = opp(i) = 26 - i they are the moments
// of F masked by the reversed link set S'(j) = S(26 - j), with the odd (first)
// moments negated.  F on the 27 directions is the tensor product of the D1Q3
// population maps (phi3) applied along x, y and z to the 17 Hermite moments
// (Eq. three_order_f), and the masked moments are three separable sums, so the
// cost does not depend on the number of solid links.
__device__ __forceinline__ void bounce_sums27(const Mom17& A, uint32_t links, float dm[10]) {
  // x: the eight (q, r) slices (the (2, 2) slice carries no D3Q27 moment)
  Phi X[3][3];  // X[q][r] over cx
  X[0][0] = phi3(A.m000, A.m100, A.m200);
  X[1][0] = phi3(A.m010, A.m110, A.m210);
  X[2][0] = phi3(A.m020, A.m120, 0.f);
  X[0][1] = phi3(A.m001, A.m101, A.m201);
  X[1][1] = phi3(A.m011, A.m111, 0.f);
  X[2][1] = phi3(A.m021, 0.f, 0.f);
  X[0][2] = phi3(A.m002, A.m102, 0.f);
  X[1][2] = phi3(A.m012, 0.f, 0.f);
  X[2][2] = Phi{0.f, 0.f, 0.f};
  const uint32_t rs = __brev(links) >> 5;  // bit j: the link opp(j) is solid
  // y then z per x direction; F(cx, cy, cz) is bit (cx+1) + 3 (cy+1) + 9 (cz+1)
  // of the reversed mask.  The masked populations are summed back to moments
  // along z, y and x.
  float Sx[3][6];  // per cx: the (q, r) moments (00) (10) (01) (20) (11) (02) of the masked F
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // a = cx + 1
    auto comp = [&](const Phi& p) { return a == 2 ? p.p : (a == 1 ? p.z : p.m); };
    Phi Y[3];  // Y[r] over cy
#pragma unroll
    for (int r = 0; r < 3; ++r) Y[r] = phi3(comp(X[0][r]), comp(X[1][r]), comp(X[2][r]));
    float T[3][3];  // T[cy+1][r'] : z-moments (r' = 0, 1, 2) of the masked column
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // b = cy + 1
      auto compy = [&](const Phi& p) { return b == 2 ? p.p : (b == 1 ? p.z : p.m); };
      const Phi Z = phi3(compy(Y[0]), compy(Y[1]), compy(Y[2]));
      const int j0 = a + 3 * b;  // cz = -1; cz = 0 at j0 + 9, cz = +1 at j0 + 18
      const float fm = (rs >> j0) & 1u ? Z.m : 0.f;
      const float fz = (rs >> (j0 + 9)) & 1u ? Z.z : 0.f;
      const float fp = (rs >> (j0 + 18)) & 1u ? Z.p : 0.f;
      const float lr = fp + fm;
      T[b][0] = lr + fz;
      T[b][1] = fp - fm;
      T[b][2] = __fmaf_rn(T[b][0], -1.0f / 3.0f, lr);
    }
    // y moments q of each z moment r'
    auto ysum = [&](int r, int q) {
      const float lr = T[2][r] + T[0][r];
      if (q == 0) return lr + T[1][r];
      if (q == 1) return T[2][r] - T[0][r];
      return __fmaf_rn(lr + T[1][r], -1.0f / 3.0f, lr);
    };
    Sx[a][0] = ysum(0, 0);
    Sx[a][1] = ysum(0, 1);
    Sx[a][2] = ysum(1, 0);
    Sx[a][3] = ysum(0, 2);
    Sx[a][4] = ysum(1, 1);
    Sx[a][5] = ysum(2, 0);
  }
  // x moments: (p, q, r) for the ten outputs; S[2] is cx = +1, S[0] cx = -1
  auto xs = [&](int k, int p) {
    const float lr = Sx[2][k] + Sx[0][k];
    if (p == 0) return lr + Sx[1][k];
    if (p == 1) return Sx[2][k] - Sx[0][k];
    return __fmaf_rn(lr + Sx[1][k], -1.0f / 3.0f, lr);
  };
  // the reflection j = opp(i) flips the sign of the first moments
  dm[0] = xs(0, 0);
  dm[1] = -xs(0, 1);
  dm[2] = -xs(1, 0);
  dm[3] = -xs(2, 0);
  dm[4] = xs(0, 2);
  dm[5] = xs(3, 0);
  dm[6] = xs(5, 0);
  dm[7] = xs(1, 1);
  dm[8] = xs(2, 1);
  dm[9] = xs(4, 0);
}

template <int STORAGE, bool FORCE, bool MOVING, bool Q19 = false>
__global__ void __launch_bounds__(128) boundary_kernel(BoundaryParams P) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= P.count) return;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz;
  const uint32_t n = P.cells[k];
  const uint32_t word = P.words[k];
  const uint32_t type = word >> 27;
  const int x = int(n % uint32_t(nx));
  const int y = int((n / uint32_t(nx)) % uint32_t(ny));
  const int z = int(n / (uint32_t(nx) * uint32_t(ny)));
  if (type == T_INFLOW) {
    Stored s;
    s.drho = P.in_rho - 1.0f;
    s.ux = P.in_ux;
    s.uy = P.in_uy;
    s.uz = P.in_uz;
    s.nxx = s.nyy = s.nzz = s.nxy = s.nxz = s.nyz = 0.f;
    store_stored<STORAGE>(P.out, N, n, s, x, y, z, P.t_out, P.seed, false, P.q);
    return;
  }
  // the raw sums of the fluid kernel, stored times the scale factors of its passes
  const float4* rec = reinterpret_cast<const float4*>(P.side) + size_t(3) * size_t(k);
  const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
  float m000 = -r0.x, m100 = 0.5f * r0.y, m010 = 0.5f * r0.z, m001 = 0.5f * r0.w,
        m200 = r1.x, m020 = r1.y, m002 = r1.z, m110 = -0.25f * r1.w,
        m101 = -0.25f * r2.x, m011 = -0.25f * r2.y;
  float fx0 = 0.f, fy0 = 0.f, fz0 = 0.f;
  if (FORCE) {
    fx0 = __ldg(P.force + n);
    fy0 = __ldg(P.force + N + n);
    fz0 = __ldg(P.force + 2 * N + n);
  }
  const Mom17 A =
      collide_moments<FORCE>(load_stored<STORAGE>(P.in, N, n, P.q), P.omega, fx0, fy0, fz0);
  uint32_t links = word & 0x7FFFFFFu;
  if constexpr (!MOVING && !Q19) {
    float dm[10];
    bounce_sums27(A, links, dm);
    m000 += dm[0];
    m100 += dm[1];
    m010 += dm[2];
    m001 += dm[3];
    m200 += dm[4];
    m020 += dm[5];
    m002 += dm[6];
    m110 += dm[7];
    m101 += dm[8];
    m011 += dm[9];
    links = 0;
  }
  // otherwise each thread loops over its own solid links (bit scan of its link
  // mask), so a warp runs as many iterations as its busiest cell
  if (Q19) links &= D3Q19_LINKS;
  while (links) {
    const int i = __ffs(links) - 1;
    links &= links - 1u;
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    float g;  // f_i / w_i - 1 of the population the solid link returns along c_i
    if constexpr (MOVING) {
      float up[3];
      body_velocity(P.bodies, P.mask[pull_source(x, y, z, nx, ny, nz, i)], x - 0.5f * cx,
                    y - 0.5f * cy, z - 0.5f * cz, up);
      const Mom17 Wm = wall_moments(A, up[0], up[1], up[2]);
      g = Q19 ? hermite_eval19(Wm, cx, cy, cz) : hermite_eval(Wm, cx, cy, cz);
    } else {
      // halfway bounce-back: population opp(i) of x itself
      g = Q19 ? hermite_eval19(A, -cx, -cy, -cz) : hermite_eval(A, -cx, -cy, -cz);
    }
    const float w = Q19 ? lattice_weight19(cx, cy, cz) : lattice_weight(cx, cy, cz);
    const float f = w * g;
    m000 += f;
    m100 += cx * f;
    m010 += cy * f;
    m001 += cz * f;
    m200 += (cx * cx - (1.0f / 3.0f)) * f;
    m020 += (cy * cy - (1.0f / 3.0f)) * f;
    m002 += (cz * cz - (1.0f / 3.0f)) * f;
    m110 += float(cx * cy) * f;
    m101 += float(cx * cz) * f;
    m011 += float(cy * cz) * f;
  }
  const Stored o = finish_moments<FORCE>(m000, m100, m010, m001, m200, m020, m002, m110, m101,
                                         m011, fx0, fy0, fz0);
  store_stored<STORAGE>(P.out, N, n, o, x, y, z, P.t_out, P.seed, false, P.q);
}

cudaError_t launch_boundary(int storage, int nx, int ny, int nz, const void* in, void* out,
                            const float* force, float omega, const uint32_t* cells,
                            const uint32_t* words, int64_t count, const BoundaryTables& bt,
                            const float inflow[4], uint32_t t_out, uint32_t seed, const QGrids& q,
                            int wall_model, const uint8_t* mask, const float* bodies, int lattice,
                            cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  BoundaryParams p;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = in;
  p.out = out;
  p.force = force;
  p.omega = omega;
  p.cells = cells;
  p.words = words;
  p.count = count;
  p.side = bt.side;
  p.in_rho = inflow[0];
  p.in_ux = inflow[1];
  p.in_uy = inflow[2];
  p.in_uz = inflow[3];
  p.t_out = t_out;
  p.seed = seed;
  p.q = q;
  p.wall_model = wall_model;
  p.mask = mask;
  p.bodies = bodies;
  const unsigned blocks = unsigned((count + 127) / 128);
  const bool mv = wall_model == 1;
  if (lattice == 19) {
    if (storage == ST_Q16) {
      if (force) {
        if (mv) boundary_kernel<ST_Q16, true, true, true><<<blocks, 128, 0, st>>>(p);
        else boundary_kernel<ST_Q16, true, false, true><<<blocks, 128, 0, st>>>(p);
      } else {
        if (mv) boundary_kernel<ST_Q16, false, true, true><<<blocks, 128, 0, st>>>(p);
        else boundary_kernel<ST_Q16, false, false, true><<<blocks, 128, 0, st>>>(p);
      }
    } else {
      if (force) {
        if (mv) boundary_kernel<ST_F32, true, true, true><<<blocks, 128, 0, st>>>(p);
        else boundary_kernel<ST_F32, true, false, true><<<blocks, 128, 0, st>>>(p);
      } else {
        if (mv) boundary_kernel<ST_F32, false, true, true><<<blocks, 128, 0, st>>>(p);
        else boundary_kernel<ST_F32, false, false, true><<<blocks, 128, 0, st>>>(p);
      }
    }
    return cudaGetLastError();
  }
  if (storage == ST_Q16) {
    if (force) {
      if (mv) boundary_kernel<ST_Q16, true, true><<<blocks, 128, 0, st>>>(p);
      else boundary_kernel<ST_Q16, true, false><<<blocks, 128, 0, st>>>(p);
    } else {
      if (mv) boundary_kernel<ST_Q16, false, true><<<blocks, 128, 0, st>>>(p);
      else boundary_kernel<ST_Q16, false, false><<<blocks, 128, 0, st>>>(p);
    }
  } else {
    if (force) {
      if (mv) boundary_kernel<ST_F32, true, true><<<blocks, 128, 0, st>>>(p);
      else boundary_kernel<ST_F32, true, false><<<blocks, 128, 0, st>>>(p);
    } else {
      if (mv) boundary_kernel<ST_F32, false, true><<<blocks, 128, 0, st>>>(p);
      else boundary_kernel<ST_F32, false, false><<<blocks, 128, 0, st>>>(p);
    }
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------- outflow
template <int WORDS>
__global__ void outflow_kernel(int nx, int ny, int nz, uint32_t* buf, const uint8_t* type) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // (y, z) index
  const int64_t M = int64_t(ny) * nz;
  if (k >= M) return;
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(nx - 1) + size_t(nx) * size_t(k);
  if (type[n] != T_OUTFLOW) return;
#pragma unroll
  for (int w = 0; w < WORDS; ++w) buf[w * N + n] = buf[w * N + n - 1];
}

cudaError_t launch_outflow(int storage, int nx, int ny, int nz, void* buf, const uint8_t* type,
                           cudaStream_t st) {
  if (nx < 2) return cudaSuccess;
  const int64_t M = int64_t(ny) * nz;
  const unsigned blocks = unsigned((M + 255) / 256);
  if (storage == ST_Q16)
    outflow_kernel<5><<<blocks, 256, 0, st>>>(nx, ny, nz, static_cast<uint32_t*>(buf), type);
  else
    outflow_kernel<10><<<blocks, 256, 0, st>>>(nx, ny, nz, static_cast<uint32_t*>(buf), type);
  return cudaGetLastError();
}

}  // namespace melbm
