// boundary.cu -- the boundary side of the split design (Sec. 4.2).
//   * FLUID_BOUNDARY: halfway bounce-back, f_i(x) = f+_{opp(i)}(x) when x - c_i is
//     solid, changes only the populations of the cell's solid links, and what
//     they return depends on the cell's own post-collision state alone.  Moments
//     are linear in f, so the new moments are the sums over the non-solid links
//     (what the fluid kernel pulls when solid cells enter its passes at rest)
//     plus the sums of the returned populations.  The bounce kernel computes the
//     latter first, per listed cell, from its input state (App. A collision) into
//     a side record; the fluid kernel adds the record to its pulled sums and
//     rounds and stores the finished moments once, in its own coalesced stores.
//     This replaces the paper's additive per-triangle correction (Alg. 3), which
//     needs a mesh: the sums are completed before the single rounding of the
//     16-bit store, with no atomics and no second pass over the output.
//     With the moment-based wall model (Sec. 3.2, solid coupling) a solid link
//     instead returns the Hermite population of (rho, u^p, S^p) at the link's
//     halfway point p, u^p the rigid velocity of the body the solid cell
//     belongs to (its mask value) and S^p = u^p u^p + (S - u u) from the cell's
//     own post-collision moments.
//   * INFLOW: reset to the equilibrium (rho_in, u_in, S = u_in u_in) after the
//     fluid kernel, by a pass over face 0.
// The outflow pass then copies the stored state of x = nx-2 onto x = nx-1.
// On the D3Q19 lattice the same update runs over its 19 directions and weights.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

struct BoundaryParams {
  int nx, ny, nz;
  const void* in;
  const float* force;
  float omega;
  const uint32_t* cells;
  const uint32_t* words;
  int64_t count;
  float* side;             // [count][12]: the bounce-back sums of the FLUID_BOUNDARY entries,
                           // times -1, 2, 2, 2, 1, 1, 1, -4, -4, -4, and two pad floats
  int wall_model;          // 0 halfway bounce-back, 1 moment-based reconstruction
  const uint8_t* mask;     // body id of every cell (wall model 1)
  const float* bodies;     // 256 x 9: V, Om, r0 of each body (wall model 1)
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
// cost does not depend on the number of solid links.  On D3Q19 (Q19) the same
// maps take the cell's 27 tensor moments: the 16 with mu_111 = 0 and the ten of
// closure19, for which the tensor product gives the D3Q19 populations (zero on
// the corners) exactly; the link set holds D3Q19 directions only.
template <bool Q19>
__device__ __forceinline__ void bounce_sums(const Mom17& A, uint32_t links, float dm[10]) {
  Phi X[3][3];  // X[q][r] over cx
  if constexpr (Q19) {
    const Closure19T<float> E = closure19(A);
    X[0][0] = phi3(A.m000, A.m100, A.m200);
    X[1][0] = phi3(A.m010, A.m110, A.m210);
    X[2][0] = phi3(A.m020, A.m120, E.m220);
    X[0][1] = phi3(A.m001, A.m101, A.m201);
    X[1][1] = phi3(A.m011, 0.f, E.m211);
    X[2][1] = phi3(A.m021, E.m121, E.m221);
    X[0][2] = phi3(A.m002, A.m102, E.m202);
    X[1][2] = phi3(A.m012, E.m112, E.m212);
    X[2][2] = phi3(E.m022, E.m122, E.m222);
  } else {
    // x: the eight (q, r) slices (the (2, 2) slice carries no D3Q27 moment)
    X[0][0] = phi3(A.m000, A.m100, A.m200);
    X[1][0] = phi3(A.m010, A.m110, A.m210);
    X[2][0] = phi3(A.m020, A.m120, 0.f);
    X[0][1] = phi3(A.m001, A.m101, A.m201);
    X[1][1] = phi3(A.m011, A.m111, 0.f);
    X[2][1] = phi3(A.m021, 0.f, 0.f);
    X[0][2] = phi3(A.m002, A.m102, 0.f);
    X[1][2] = phi3(A.m012, 0.f, 0.f);
    X[2][2] = Phi{0.f, 0.f, 0.f};
  }
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

// Bounce kernel, before the fluid kernel (in -> side): for every FLUID_BOUNDARY
// cell of the list, the sums of the populations its solid links return -- from
// the cell's own post-collision state alone -- written into its side record in
// the scaling of the fluid kernel's passes (-1, 2, 2, 2, 1, 1, 1, -4, -4, -4),
// which adds them to the pulled sums before its one rounding and store.
template <int STORAGE, bool FORCE, bool MOVING, bool Q19 = false>
__global__ void __launch_bounds__(128) bounce_kernel(BoundaryParams P) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= P.count) return;
  const uint32_t word = P.words[k];
  if ((word >> 27) != T_FLUID_BOUNDARY) return;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz;
  const uint32_t n = P.cells[k];
  float fx0 = 0.f, fy0 = 0.f, fz0 = 0.f;
  if (FORCE) {
    fx0 = __ldg(P.force + n);
    fy0 = __ldg(P.force + N + n);
    fz0 = __ldg(P.force + 2 * N + n);
  }
  const Mom17 A =
      collide_moments<FORCE>(load_stored<STORAGE>(P.in, N, n, P.q), P.omega, fx0, fy0, fz0);
  uint32_t links = word & 0x7FFFFFFu;
  float dm[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (!MOVING) {
    bounce_sums<Q19>(A, Q19 ? (links & D3Q19_LINKS) : links, dm);
  } else {
    // each thread loops over its own solid links (bit scan of its link mask), so
    // a warp runs as many iterations as its busiest cell
    const int x = int(n % uint32_t(nx));
    const int y = int((n / uint32_t(nx)) % uint32_t(ny));
    const int z = int(n / (uint32_t(nx) * uint32_t(ny)));
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
      dm[0] += f;
      dm[1] += cx * f;
      dm[2] += cy * f;
      dm[3] += cz * f;
      dm[4] += (cx * cx - (1.0f / 3.0f)) * f;
      dm[5] += (cy * cy - (1.0f / 3.0f)) * f;
      dm[6] += (cz * cz - (1.0f / 3.0f)) * f;
      dm[7] += float(cx * cy) * f;
      dm[8] += float(cx * cz) * f;
      dm[9] += float(cy * cz) * f;
    }
  }
  // the scale factors are powers of two: the fluid kernel's sum is the same
  float4* rec = reinterpret_cast<float4*>(P.side) + size_t(3) * size_t(k);
  rec[0] = make_float4(-dm[0], 2.0f * dm[1], 2.0f * dm[2], 2.0f * dm[3]);
  rec[1] = make_float4(dm[4], dm[5], dm[6], -4.0f * dm[7]);
  rec[2] = make_float4(-4.0f * dm[8], -4.0f * dm[9], 0.f, 0.f);
}

template <bool FORCE, bool MOVING, bool Q19>
cudaError_t launch_bounce_l(int storage, BoundaryParams& p, unsigned blocks, cudaStream_t st) {
  if (storage == ST_Q16)
    bounce_kernel<ST_Q16, FORCE, MOVING, Q19><<<blocks, 128, 0, st>>>(p);
  else
    bounce_kernel<ST_F32, FORCE, MOVING, Q19><<<blocks, 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bounce(int storage, int nx, int ny, int nz, const void* in, const float* force,
                          float omega, const uint32_t* cells, const uint32_t* words, int64_t count,
                          const BoundaryTables& bt, const QGrids& q, int wall_model,
                          const uint8_t* mask, const float* bodies, int lattice, cudaStream_t st) {
  if (count <= 0 || !bt.side) return cudaSuccess;
  BoundaryParams p = {};
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = in;
  p.force = force;
  p.omega = omega;
  p.cells = cells;
  p.words = words;
  p.count = count;
  p.side = bt.side;
  p.q = q;
  p.wall_model = wall_model;
  p.mask = mask;
  p.bodies = bodies;
  const unsigned blocks = unsigned((count + 127) / 128);
  const bool mv = wall_model == 1;
  if (lattice == 19) {
    if (force) return mv ? launch_bounce_l<true, true, true>(storage, p, blocks, st)
                         : launch_bounce_l<true, false, true>(storage, p, blocks, st);
    return mv ? launch_bounce_l<false, true, true>(storage, p, blocks, st)
              : launch_bounce_l<false, false, true>(storage, p, blocks, st);
  }
  if (force) return mv ? launch_bounce_l<true, true, false>(storage, p, blocks, st)
                       : launch_bounce_l<true, false, false>(storage, p, blocks, st);
  return mv ? launch_bounce_l<false, true, false>(storage, p, blocks, st)
            : launch_bounce_l<false, false, false>(storage, p, blocks, st);
}

// ----------------------------------------------------------------- inflow
// After the fluid kernel: the INFLOW cells of face 0 (x = 0) are reset to the
// equilibrium (rho_in, u_in, u_in u_in); one thread per (y, z).
template <int STORAGE>
__global__ void inflow_kernel(int nx, int ny, int nz, void* out, const uint8_t* type, float in_rho,
                              float in_ux, float in_uy, float in_uz, uint32_t t_out, uint32_t seed,
                              QGrids q) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // (y, z) index
  if (k >= int64_t(ny) * nz) return;
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(nx) * size_t(k);
  if (type[n] != T_INFLOW) return;
  Stored s;
  s.drho = in_rho - 1.0f;
  s.ux = in_ux;
  s.uy = in_uy;
  s.uz = in_uz;
  s.nxx = s.nyy = s.nzz = s.nxy = s.nxz = s.nyz = 0.f;
  store_stored<STORAGE>(out, N, n, s, 0, int(k % ny), int(k / ny), t_out, seed, false, q);
}

cudaError_t launch_inflow(int storage, int nx, int ny, int nz, void* out, const uint8_t* type,
                          const float inflow[4], uint32_t t_out, uint32_t seed, const QGrids& q,
                          cudaStream_t st) {
  const int64_t M = int64_t(ny) * nz;
  const unsigned blocks = unsigned((M + 255) / 256);
  if (storage == ST_Q16)
    inflow_kernel<ST_Q16><<<blocks, 256, 0, st>>>(nx, ny, nz, out, type, inflow[0], inflow[1],
                                                  inflow[2], inflow[3], t_out, seed, q);
  else
    inflow_kernel<ST_F32><<<blocks, 256, 0, st>>>(nx, ny, nz, out, type, inflow[0], inflow[1],
                                                  inflow[2], inflow[3], t_out, seed, q);
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
