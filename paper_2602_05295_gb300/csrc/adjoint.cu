// adjoint.cu -- hand-written discrete adjoint of the FP32-storage step, with
// 16-bit checkpointing (the paper has no adjoint; inverse design motivates it,
// Sec. 1).  One forward step is  m' = Fin(Stream(Coll(m, F)), F)  per cell, with
// bounce-back, inflow and outflow applied by the boundary kernels.  Its
// vector-Jacobian product is taken by one fused kernel and one list kernel:
//   1. adj_stream_kernel, over every cell: lambda_M = (dFin/dM)^T lambda' (and
//      dL/dF from the F/2 of Eq. rho_u_stress), zero for solid, inflow and
//      outflow cells; then the transpose of the separable pull stream of the
//      fluid kernel (Eq. streaming), back onto the 17 Hermite moments of each
//      source cell, with three transposed 1D passes (x by shuffles, y through
//      shared memory, z in registers); then (dColl/dm)^T (App. A transposed by
//      hand);
//   2. adj_boundary_kernel, over the listed FLUID_BOUNDARY cells: the bounce-back
//      terms f_i(x) = f+_opp(i)(x) of their own solid links, through the same
//      (dColl/dm)^T, added (the map is linear in the moment adjoints).
// The forward states of each segment are recomputed in FP32 from a 16-bit
// checkpoint (deterministic rounding) taken every K steps; the initial state is
// rebuilt exactly from u0.
#include <algorithm>
#include <cstdint>
#include <new>

#include "../../include/melbm.h"
#include "melbm_adjoint.h"
#include "melbm_device.cuh"
#include "melbm_handle.h"
#include "melbm_launch.h"

namespace melbm {

struct AdjointState {
  int nsteps = 0, K = 0, nck = 0;
  int64_t N = 0;
  bool ready = false;
  bool seg_filled = false;    // nsteps <= K: the forward pass kept every state in seg
  float* u0 = nullptr;        // 3N
  uint32_t* ckpt = nullptr;   // nck x 5N (16-bit states at t = K, 2K, ...)
  float* seg = nullptr;       // (K + 1) x 10N FP32 states of one segment
  // With more than one segment the backward pass recomputes segment s - 1 into the
  // second buffer on its own stream while the adjoint runs over segment s.
  float* seg2 = nullptr;      // (K + 1) x 10N, only with checkpoints
  cudaStream_t rs = nullptr;  // the recompute stream
  cudaEvent_t ev_start = nullptr;    // work issued on the handle's stream so far
  cudaEvent_t ev_rec[2] = {};        // the recompute into buffer b is done
  cudaEvent_t ev_used[2] = {};       // the adjoint has finished reading buffer b
  float* lam = nullptr;       // 10N adjoint of the stored variables
  float* lam2 = nullptr;      // 10N
  float* gF = nullptr;        // 3N accumulated dL/dF
  int64_t bytes = 0;          // device bytes held (melbm_memory_bytes)
};

void adjoint_free(AdjointState* a) {
  if (!a) return;
  cudaFree(a->u0);
  cudaFree(a->ckpt);
  cudaFree(a->seg);
  cudaFree(a->seg2);
  cudaFree(a->lam);
  cudaFree(a->lam2);
  cudaFree(a->gF);
  if (a->rs) cudaStreamDestroy(a->rs);
  if (a->ev_start) cudaEventDestroy(a->ev_start);
  for (int b = 0; b < 2; ++b) {
    if (a->ev_rec[b]) cudaEventDestroy(a->ev_rec[b]);
    if (a->ev_used[b]) cudaEventDestroy(a->ev_used[b]);
  }
  delete a;
}

namespace {

constexpr int AT = 256;

__device__ __forceinline__ Stored load_f32(const float* b, size_t N, size_t n) {
  return load_stored<ST_F32>(b, N, n);
}

// ------------------------------------------------------------------ state kernels
__global__ void init_from_u0_kernel(const float* u0, float* buf, int64_t N_) {
  const size_t N = size_t(N_), n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  for (int k = 0; k < 10; ++k) buf[k * N + n] = 0.f;  // rho = 1, S = u u: n = 0
  buf[N + n] = u0[n];
  buf[2 * N + n] = u0[N + n];
  buf[3 * N + n] = u0[2 * N + n];
}

__global__ void f32_to_q16_kernel(const float* s, uint32_t* w, int nx, int ny, int nz) {
  const size_t N = size_t(nx) * ny * nz, n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  store_stored<ST_Q16>(w, N, n, load_f32(s, N, n), 0, 0, 0, 0, 0, true);
}

__global__ void q16_to_f32_kernel(const uint32_t* w, float* s, int64_t N_) {
  const size_t N = size_t(N_), n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  store_stored<ST_F32>(s, N, n, load_stored<ST_Q16>(w, N, n), 0, 0, 0, 0, 0);
}

// dL/d(stored) from dL/d(public): rho = 1 + drho, u = u, S_ab = n_ab / rho + u_a u_b.
__global__ void pub_vjp_kernel(const float* m, const float* g, float* lam, int64_t N_) {
  const size_t N = size_t(N_), n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  const Stored s = load_f32(m, N, n);
  const float rho = 1.0f + s.drho, inv = 1.0f / rho;
  const float u[3] = {s.ux, s.uy, s.uz};
  const float nn[6] = {s.nxx, s.nyy, s.nzz, s.nxy, s.nxz, s.nyz};
  const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  float ldr = g[n], lu[3] = {g[N + n], g[2 * N + n], g[3 * N + n]};
  for (int k = 0; k < 6; ++k) {
    const float gs = g[(4 + k) * N + n];
    ldr -= gs * nn[k] * inv * inv;
    lu[A[k]] += gs * u[B[k]];
    lu[B[k]] += gs * u[A[k]];
    lam[(4 + k) * N + n] = gs * inv;
  }
  lam[n] = ldr;
  lam[N + n] = lu[0];
  lam[2 * N + n] = lu[1];
  lam[3 * N + n] = lu[2];
}

// Outflow copy transposed: the outflow cell's output came from (nx-2, y, z).
__global__ void outflow_vjp_kernel(float* lam, const uint8_t* type, int nx, int ny, int nz) {
  const int64_t k = int64_t(blockIdx.x) * AT + threadIdx.x;
  if (k >= int64_t(ny) * nz || nx < 2) return;
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(nx - 1) + size_t(nx) * size_t(k);
  if (type[n] != T_OUTFLOW) return;
  for (int c = 0; c < 10; ++c) {
    lam[c * N + n - 1] += lam[c * N + n];
    lam[c * N + n] = 0.f;
  }
}

// ------------------------------------------------------------------ Fin^T
// Forward: drho' = M000, J = M1 + F/2, inv = 1/(1 + M000), u' = J inv,
// n'_ab = M_ab - J_a J_b inv.  The streamed moments are recovered from the output
// o.  lam: the adjoint of the stored output variables; lamM: that of the ten
// streamed moments (M000, M100, M010, M001, M200, M020, M002, M110, M101, M011);
// lJ: the adjoint of J, of which F/2 takes half.
__device__ __forceinline__ void fin_vjp_cell(const Stored& o, const float lam[10], float lamM[10],
                                             float lJ[3]) {
  const float rho = 1.0f + o.drho, inv = __fdividef(1.0f, rho);  // rho ~ 1: 2-ulp reciprocal
  const float J[3] = {o.ux * rho, o.uy * rho, o.uz * rho};
  const float* lu = lam + 1;
  const float* ln = lam + 4;
  const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  lJ[0] = lu[0];
  lJ[1] = lu[1];
  lJ[2] = lu[2];
  float linv = 0.f;
  for (int a = 0; a < 3; ++a) linv += lu[a] * J[a];
  for (int k = 0; k < 6; ++k) {
    lJ[A[k]] -= ln[k] * J[B[k]];
    lJ[B[k]] -= ln[k] * J[A[k]];
    linv -= ln[k] * J[A[k]] * J[B[k]];
  }
  for (int a = 0; a < 3; ++a) lJ[a] *= inv;
  lamM[0] = lam[0] - linv * inv * inv;
  lamM[1] = lJ[0];
  lamM[2] = lJ[1];
  lamM[3] = lJ[2];
  for (int k = 0; k < 6; ++k) lamM[4 + k] = ln[k];
}

__device__ __forceinline__ bool special_type(uint8_t t) {
  return t == T_SOLID || t == T_INFLOW || t == T_OUTFLOW;  // output not from the stream
}

// ------------------------------------------------------------------ Coll^T
// Reverse of collide_moments (App. A in stored variables), accumulated by hand.
template <bool FORCE>
__device__ void collide_vjp(const Stored& s, float omega, const float f[3], const float lmu[17],
                            float lin[10], float lf[3]) {
  // ---- forward recomputation (as collide_moments)
  const float rho = 1.0f + s.drho, om1 = 1.0f - omega;
  const float u[3] = {s.ux, s.uy, s.uz};
  float m[6] = {s.nxx, s.nyy, s.nzz, s.nxy, s.nxz, s.nyz};
  const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  float inv = 0.f;
  if (FORCE) {
    inv = __fdividef(1.0f, rho);
    for (int k = 0; k < 3; ++k) m[k] += f[k] * u[k];
    for (int k = 3; k < 6; ++k) m[k] += 0.5f * (f[A[k]] * u[B[k]] + f[B[k]] * u[A[k]]);
  }
  const float tr = (m[0] + m[1] + m[2]) * (1.0f / 3.0f);
  float e[6];
  for (int k = 0; k < 3; ++k) e[k] = om1 * (m[k] - tr);
  for (int k = 3; k < 6; ++k) e[k] = om1 * m[k];
  const float q = -0.25f * inv, h = 0.5f * inv;
  if (FORCE)
    for (int k = 0; k < 6; ++k) e[k] += q * f[A[k]] * f[B[k]];
  float U[3];
  for (int a = 0; a < 3; ++a) U[a] = FORCE ? u[a] + h * f[a] : u[a];
  float rU[3];
  for (int a = 0; a < 3; ++a) rU[a] = rho * U[a];
  float mu2[6];  // mu_aa, mu_ab (rho S+)
  for (int k = 0; k < 6; ++k) mu2[k] = rU[A[k]] * U[B[k]] + e[k];
  // Mom17 order: 000, 100, 010, 001, 200, 020, 002, 110, 101, 011,
  //              210 (xxy), 120 (xyy), 201 (xxz), 102 (xzz), 021 (yyz), 012 (yzz), 111
  // third-order: mu_aab = U_b mu_aa + 2 U_a e_ab, listed as (a, b, k_ab)
  const int TA[6] = {0, 1, 0, 2, 1, 2}, TB[6] = {1, 0, 2, 0, 2, 1}, TK[6] = {3, 3, 4, 4, 5, 5};

  // ---- reverse
  float lrU[3] = {0.f, 0.f, 0.f}, lU[3] = {0.f, 0.f, 0.f}, le[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float lmu2[6];
  for (int k = 0; k < 6; ++k) lmu2[k] = lmu[4 + k];
  float lrho = 0.f;
  lin[0] = lmu[0];  // mu000 = drho
  for (int a = 0; a < 3; ++a) lrU[a] += lmu[1 + a];
  for (int t = 0; t < 6; ++t) {
    const int a = TA[t], b = TB[t], kab = TK[t];
    const float l = lmu[10 + t];
    lU[b] += l * mu2[a];
    lmu2[a] += l * U[b];
    lU[a] += 2.0f * l * e[kab];
    le[kab] += 2.0f * l * U[a];
  }
  {  // mu111 = rU_x U_y U_z + e_xy U_z + e_xz U_y + e_yz U_x
#ifdef MELBM_HERMITE_XYZ_LITERAL
    const float l = 0.5f * lmu[16];  // mu111 is halved under the literal xyz factor
#else
    const float l = lmu[16];
#endif
    lrU[0] += l * U[1] * U[2];
    lU[1] += l * (rU[0] * U[2] + e[4]);
    lU[2] += l * (rU[0] * U[1] + e[3]);
    lU[0] += l * e[5];
    le[3] += l * U[2];
    le[4] += l * U[1];
    le[5] += l * U[0];
  }
  for (int k = 0; k < 6; ++k) {  // mu2_k = rU_A U_B + e_k
    lrU[A[k]] += lmu2[k] * U[B[k]];
    lU[B[k]] += lmu2[k] * rU[A[k]];
    le[k] += lmu2[k];
  }
  for (int a = 0; a < 3; ++a) {  // rU = rho U
    lrho += lrU[a] * U[a];
    lU[a] += lrU[a] * rho;
  }
  float lu[3] = {lU[0], lU[1], lU[2]};
  float linv = 0.f;
  if (FORCE) {
    float lq = 0.f, lh = 0.f;
    for (int a = 0; a < 3; ++a) {  // U = u + h f
      lh += lU[a] * f[a];
      lf[a] += lU[a] * h;
    }
    for (int k = 0; k < 6; ++k) {  // e_k += q f_A f_B
      lq += le[k] * f[A[k]] * f[B[k]];
      lf[A[k]] += le[k] * q * f[B[k]];
      lf[B[k]] += le[k] * q * f[A[k]];
    }
    linv = -0.25f * lq + 0.5f * lh;
  }
  // e = om1 dev(m)
  float lm[6];
  const float ltr = le[0] + le[1] + le[2];
  for (int k = 0; k < 3; ++k) lm[k] = om1 * (le[k] - ltr * (1.0f / 3.0f));
  for (int k = 3; k < 6; ++k) lm[k] = om1 * le[k];
  if (FORCE) {
    for (int k = 0; k < 3; ++k) {  // m_aa = n_aa + f_a u_a
      lf[k] += lm[k] * u[k];
      lu[k] += lm[k] * f[k];
    }
    for (int k = 3; k < 6; ++k) {  // m_ab = n_ab + (f_a u_b + f_b u_a)/2
      lf[A[k]] += 0.5f * lm[k] * u[B[k]];
      lf[B[k]] += 0.5f * lm[k] * u[A[k]];
      lu[B[k]] += 0.5f * lm[k] * f[A[k]];
      lu[A[k]] += 0.5f * lm[k] * f[B[k]];
    }
    lrho -= linv * inv * inv;
  }
  lin[0] += lrho;
  lin[1] = lu[0];
  lin[2] = lu[1];
  lin[3] = lu[2];
  for (int k = 0; k < 6; ++k) lin[4 + k] = lm[k];
}

// d f_i / d mu_pqr = w_i N_pqr P_p(cx) P_q(cy) P_r(cz): the Hermite population of
// direction c as a function of the 17 moments (N = inverse D1Q3 norms).
__device__ __forceinline__ void add_population_adjoint(int cx, int cy, int cz, float lf,
                                                       float lmu[17]) {
  const float w = (cx ? (1.0f / 6.0f) : (2.0f / 3.0f)) * (cy ? (1.0f / 6.0f) : (2.0f / 3.0f)) *
                  (cz ? (1.0f / 6.0f) : (2.0f / 3.0f));
  const float g = w * lf;
  const float px = float(cx), py = float(cy), pz = float(cz);
  const float qx = px * px - (1.0f / 3.0f), qy = py * py - (1.0f / 3.0f), qz = pz * pz - (1.0f / 3.0f);
  lmu[0] += g;
  lmu[1] += 3.0f * g * px;
  lmu[2] += 3.0f * g * py;
  lmu[3] += 3.0f * g * pz;
  lmu[4] += 4.5f * g * qx;
  lmu[5] += 4.5f * g * qy;
  lmu[6] += 4.5f * g * qz;
  lmu[7] += 9.0f * g * px * py;
  lmu[8] += 9.0f * g * px * pz;
  lmu[9] += 9.0f * g * py * pz;
  lmu[10] += 13.5f * g * qx * py;  // xxy
  lmu[11] += 13.5f * g * px * qy;  // xyy
  lmu[12] += 13.5f * g * qx * pz;  // xxz
  lmu[13] += 13.5f * g * px * qz;  // xzz
  lmu[14] += 13.5f * g * qy * pz;  // yyz
  lmu[15] += 13.5f * g * py * qz;  // yzz
  lmu[16] += 27.0f * g * px * py * pz;
}

// The same for a D3Q19 population, f_i = w19_i (1 + hermite_eval19): the third
// order through the projected pairs, no xyz term.
__device__ __forceinline__ void add_population_adjoint19(int cx, int cy, int cz, float lf,
                                                         float lmu[17]) {
  const float g = lattice_weight19(cx, cy, cz) * lf;
  const float px = float(cx), py = float(cy), pz = float(cz);
  const float qx = px * px - (1.0f / 3.0f), qy = py * py - (1.0f / 3.0f), qz = pz * pz - (1.0f / 3.0f);
  lmu[0] += g;
  lmu[1] += 3.0f * g * px;
  lmu[2] += 3.0f * g * py;
  lmu[3] += 3.0f * g * pz;
  lmu[4] += 4.5f * g * qx;
  lmu[5] += 4.5f * g * qy;
  lmu[6] += 4.5f * g * qz;
  lmu[7] += 9.0f * g * px * py;
  lmu[8] += 9.0f * g * px * pz;
  lmu[9] += 9.0f * g * py * pz;
  const float hy1 = qx * py, hy2 = py * qz, hx1 = px * qy, hx2 = px * qz, hz1 = qx * pz, hz2 = qy * pz;
  lmu[10] += g * (18.0f * hy1 + 9.0f * hy2);  // xxy
  lmu[15] += g * (9.0f * hy1 + 18.0f * hy2);  // yzz
  lmu[11] += g * (18.0f * hx1 + 9.0f * hx2);  // xyy
  lmu[13] += g * (9.0f * hx1 + 18.0f * hx2);  // xzz
  lmu[12] += g * (18.0f * hz1 + 9.0f * hz2);  // xxz
  lmu[14] += g * (9.0f * hz1 + 18.0f * hz2);  // yyz
}

// ------------------------------------------------------------------ stream^T
// The pull stream followed by the moment sums is the separable map of the fluid
// kernel: per axis, (mu0, mu1, mu2) -> phi = (phi+, phi0, phi-) with
// s = mu0/6 + mu2/2, phi0 = mu0 - 2 s, phi+- = s +- mu1/2; pull phi+ from the
// minus side and phi- from the plus side; project m0 = pl + z + mr, m1 = pl - mr,
// m2 = (2/3)(pl + mr) - z/3.  Its transpose, per axis, is the same three-point
// stencil read the other way (the three axis maps act on different indices of the
// tensor moments, so their transposes may be applied in any order; the kernel
// takes x, then y, then z, so that the x halo of a tile needs Fin^T alone):
//   proj^T: lpl = l0 + l1 + (2/3) l2,  lmr = l0 - l1 + (2/3) l2,  lz = l0 - l2/3;
//   push:   lphi+(x) = lpl(x + 1), lphi-(x) = lmr(x - 1), lphi0 = lz;
//   phi^T:  ls = lphi+ + lphi- - 2 lphi0, lmu0 = lphi0 + ls/6, lmu1 = (lphi+ - lphi-)/2,
//           lmu2 = ls/2.
// Carried adjoints: 10 -> 18 (x, six (q, r) slices) -> 27 (y, nine (p, r) slices)
// -> 17 (z, eight (p, q) slices); on D3Q19 the z pass yields all 27 tensor moments
// (nine slices), folded back onto the 17 through the transposed closure.
struct LamT {
  float p, z, m;  // lpl, lz, lmr of one cell, before the push
};
__device__ __forceinline__ LamT proj_t(float l0, float l1, float l2) {
  const float a = fmaf(l2, 2.0f / 3.0f, l0);
  LamT r;
  r.p = a + l1;
  r.m = a - l1;
  r.z = fmaf(l2, -1.0f / 3.0f, l0);
  return r;
}
// lp = lphi+ (the plus neighbour's lpl), lz = own lz, lm = lphi- (the minus
// neighbour's lmr) -> (lmu0, lmu1, lmu2)
__device__ __forceinline__ void phi_t(float lp, float lz, float lm, float& l0, float& l1, float& l2) {
  const float ls = fmaf(lz, -2.0f, lp + lm);
  l1 = 0.5f * (lp - lm);
  l0 = fmaf(ls, 1.0f / 6.0f, lz);
  l2 = 0.5f * ls;
}

// Tile: 32 lanes (the columns x0 .. x0+31, fewer in a ragged last tile) by AFY
// warps (the rows y0-1 .. y0+AFY-2, wrapped); warps 0 and AFY-1 are halo rows,
// which take Fin^T, x^T and the y projection of their row and, instead of the
// y^T, z^T and Coll^T of the owned rows, compute the x-halo cells of the tile
// two planes ahead.
#ifndef MELBM_ADJ_FY
#define MELBM_ADJ_FY 16
#endif
constexpr int AFX = 32;
constexpr int AFY = MELBM_ADJ_FY;
constexpr int AIY = AFY - 2;  // rows a tile owns
static_assert(AFY >= 3 && AFY <= AFX, "the halo warps give one lane to each row");
// shared memory: the y-pass buffers, [parity][lpl, lmr][row][2][lane] float4 (the
// y slices 0 .. 7) and [parity][lpl, lmr][row][lane] float (slice 8), then the
// x-halo buffers [parity][left, right][row][8] float (six slices, padded)
constexpr int AY4 = 2 * 2 * AFY * 2 * AFX;
constexpr int AY1 = 2 * 2 * AFY * AFX;
constexpr int AHB = 2 * 2 * AFY * 8;
constexpr size_t ADJ_SMEM = size_t(AY4) * sizeof(float4) + size_t(AY1 + AHB) * sizeof(float);

// Each field is a [k][N] array of planes addressed from one base pointer with a
// 32-bit index n + k N (the launcher requires 10 N < 2^32); per-plane pointers
// in the parameters were reloaded from the constant bank at every access.
struct AdjStreamParams {
  int nx, ny, nz, zc;
  const float* lam_next;  // [10][N] adjoint of the output state (stored variables)
  const float* m_next;    // [4][N]: output state, rho - 1 and u (planes of a [10][N] state)
  const float* m_t;       // [10][N] input state
  const float* force;     // [3][N], null without force
  const uint8_t* type;    // N or null
  float* lam_out;         // [10][N] adjoint of the input state
  float* gF;              // [3][N] accumulated dL/dF
  float omega;
};

// Fin^T of one cell (rho - 1 and u of its output in M): lM, lJ; zero when the
// output does not come from the stream.
__device__ __forceinline__ void fin_t_or_zero(bool skip, const float L[10], const float M[4],
                                              float lM[10], float lJ[3]) {
  if (skip) {
#pragma unroll
    for (int k = 0; k < 10; ++k) lM[k] = 0.f;
    lJ[0] = lJ[1] = lJ[2] = 0.f;
    return;
  }
  Stored o;  // fin_vjp_cell reads rho - 1 and u of the output only
  o.drho = M[0];
  o.ux = M[1];
  o.uy = M[2];
  o.uz = M[3];
  o.nxx = o.nyy = o.nzz = o.nxy = o.nxz = o.nyz = 0.f;
  fin_vjp_cell(o, L, lM, lJ);
}

// The x projections of the six (q, r) slices (00) (10) (01) (20) (11) (02), inputs
// over p, from the ten moment adjoints (M000 M100 M010 M001 M200 M020 M002 M110 M101 M011).
__device__ __forceinline__ void x_proj(const float lM[10], LamT t[6]) {
  t[0] = proj_t(lM[0], lM[1], lM[4]);
  t[1] = proj_t(lM[2], lM[7], 0.f);
  t[2] = proj_t(lM[3], lM[8], 0.f);
  t[3] = proj_t(lM[5], 0.f, 0.f);
  t[4] = proj_t(lM[9], 0.f, 0.f);
  t[5] = proj_t(lM[6], 0.f, 0.f);
}

// A plane index in [-nz, 2 nz) wrapped into [0, nz).
__device__ __forceinline__ uint32_t wrap_plane(int z, int nz) {
  return uint32_t(z < 0 ? z + nz : (z >= nz ? z - nz : z));
}

// Block (bx, by, bz) owns the columns x0 .. x0+w-1 (x0 = 32 bx) of the rows
// y0 .. y0+AIY-1 (y0 = AIY by) over the planes zs .. ze-1 of z-chunk bz; the grid
// is one wave, so neighbouring tiles march through the same planes together and
// their halo reads hit L2.  Iteration i handles plane zz = zs - 1 + i:
//   A (every warp): Fin^T at zz, x^T (shuffles; lane 0 and the tile's last lane
//     take the halo columns' values from shared memory), the y projection into
//     shared-memory buffer i & 1; the next plane's loads are issued here;
//   barrier;
//   B (owned rows): y^T from the rows above and below, the z projection, and,
//     for i >= 2, z^T and Coll^T of plane zz - 1, stored;
//   B (halo warps): Fin^T and the x projection of the halo cells (x0 - 1, y) and
//     (x0 + w, y) of every row at plane zz + 2, into halo buffer i & 1.
// Periodic in all directions; cells whose output does not come from the stream
// contribute no adjoint (special_type), and solid cells get none; the bounce-back
// terms of listed cells are added by adj_boundary_kernel.
template <bool FORCE, bool TYPED, bool Q19>
__global__ void __launch_bounds__(AFX* AFY, 1) adj_stream_kernel(const __grid_constant__ AdjStreamParams P) {
  extern __shared__ float4 adj_smem[];
  constexpr int NZS = Q19 ? 9 : 8;  // z^T slices (p, q)
  const int lane = threadIdx.x, row = threadIdx.y;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const uint32_t plane = uint32_t(nx) * uint32_t(ny);
  const uint32_t NN = plane * uint32_t(nz);  // cells: the plane stride of every field
  const int x0 = int(blockIdx.x) * AFX, y0 = int(blockIdx.y) * AIY;
  const int zs = int(blockIdx.z) * P.zc, ze = min(zs + P.zc, nz);
  const int w = min(AFX, nx - x0);  // columns of this tile; lane w - 1 takes the right halo
  const bool owned_row = row >= 1 && row <= AFY - 2;  // warp-uniform
  const bool own = owned_row && y0 - 1 + row < ny && lane < w;
  const bool left_end = lane == 0, right_end = lane == w - 1;
  const int yr = wrapi(y0 - 1 + row, ny);
  const uint32_t col = uint32_t(min(x0 + lane, nx - 1)) + uint32_t(nx) * uint32_t(yr);
  // halo warps: warp 0 the column left of the tile, warp AFY-1 the one right of it
  const int hside = row == 0 ? 0 : 1;
  const bool hlane = !owned_row && lane < AFY;
  const uint32_t hcol = uint32_t(hside == 0 ? wrapi(x0 - 1, nx) : wrapi(x0 + w, nx)) +
                        uint32_t(nx) * uint32_t(wrapi(y0 - 1 + lane, ny));
  // shared memory
  // (this thread's entries in parity 0; parity 1 is AY4 / 2 float4 or AY1 / 2 floats on)
  float4* const yp4 = adj_smem + (0 * AFY + row) * 2 * AFX + lane;
  float4* const ym4 = adj_smem + (1 * AFY + row) * 2 * AFX + lane;
  float* const y1 = reinterpret_cast<float*>(adj_smem + AY4);
  float* const yp1 = y1 + (0 * AFY + row) * AFX + lane;
  float* const ym1 = y1 + (1 * AFY + row) * AFX + lane;
  float* const hb = y1 + AY1;
  const int n_it = ze - zs + 2;

  // ---- halo cells: loads one step ahead of their use
  float HL[10], HM[4];
  bool hskip = false;
  auto halo_loads = [&](int zp) {
    if (!hlane) return;
    const uint32_t n = hcol + plane * wrap_plane(zp, nz);
    hskip = TYPED && special_type(P.type[n]);
#pragma unroll
    for (int k = 0; k < 10; ++k) HL[k] = __ldg(P.lam_next + (n + uint32_t(k) * NN));
#pragma unroll
    for (int k = 0; k < 4; ++k) HM[k] = __ldg(P.m_next + (n + uint32_t(k) * NN));
  };
  auto halo_finish = [&](int buf) {
    if (!hlane) return;
    float lM[10], lJ[3];
    fin_t_or_zero(hskip, HL, HM, lM, lJ);
    LamT t[6];
    x_proj(lM, t);
    float* h = hb + ((buf * 2 + hside) * AFY + lane) * 8;
    // the left column pushes its lmr to x0, the right column its lpl to x0 + w - 1
    *reinterpret_cast<float4*>(h) = hside == 0 ? make_float4(t[0].m, t[1].m, t[2].m, t[3].m)
                                               : make_float4(t[0].p, t[1].p, t[2].p, t[3].p);
    *reinterpret_cast<float2*>(h + 4) =
        hside == 0 ? make_float2(t[4].m, t[5].m) : make_float2(t[4].p, t[5].p);
  };

  // ---- the tile's own cells: plane zz's lambda' and output state one step ahead
  float Lnext[10], Mnext[4];
  bool skip_next = false;
  auto load_plane = [&](int zp) {
    const uint32_t n = col + plane * wrap_plane(zp, nz);
    skip_next = TYPED && special_type(P.type[n]);
#pragma unroll
    for (int k = 0; k < 10; ++k) Lnext[k] = __ldg(P.lam_next + (n + uint32_t(k) * NN));
#pragma unroll
    for (int k = 0; k < 4; ++k) Mnext[k] = __ldg(P.m_next + (n + uint32_t(k) * NN));
  };
  load_plane(zs - 1);
  halo_loads(zs - 1);
  halo_finish(0);
  halo_loads(zs);
  halo_finish(1);
  halo_loads(zs + 1);
  __syncthreads();

  float zl[NZS], m1[NZS], m2[NZS];  // z-march state per (p, q) slice
#pragma unroll
  for (int k = 0; k < NZS; ++k) zl[k] = m1[k] = m2[k] = 0.f;
  float gprev[3] = {0.f, 0.f, 0.f};  // F/2 share of Fin^T at plane zz - 1
  uint32_t no = col + plane * uint32_t(zs);  // the cell of plane zz - 1 once i >= 2
#pragma unroll 2  // two trips per pass, so the carried registers alternate instead of moving
  for (int i = 0; i < n_it; ++i) {
    const int zz = zs - 1 + i;
    const bool out_plane = i >= 2;  // plane zz - 1 is finished in this iteration
    const int buf = i & 1;
    // the input state (and force, gradient) of plane zz - 1, used in phase B
    float mt[10], fo[3] = {0.f, 0.f, 0.f}, go[3] = {0.f, 0.f, 0.f};
    bool solid_out = false;
    if (out_plane && own) {
      solid_out = TYPED && P.type[no] == T_SOLID;
#pragma unroll
      for (int k = 0; k < 10; ++k) mt[k] = __ldg(P.m_t + (no + uint32_t(k) * NN));
      if (FORCE)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          fo[a] = __ldg(P.force + (no + uint32_t(a) * NN));
          go[a] = P.gF[no + uint32_t(a) * NN];
        }
    }
    // ---- phase A: Fin^T at plane zz
    float lam[10], mn[4];
    const bool skip = skip_next;
#pragma unroll
    for (int k = 0; k < 10; ++k) lam[k] = Lnext[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) mn[k] = Mnext[k];
    if (i + 1 < n_it) load_plane(zz + 1);
    float lM[10], lJ[3];
    fin_t_or_zero(skip, lam, mn, lM, lJ);
    // x^T: lpl from x + 1, lmr from x - 1; the tile's ends from the halo buffer
    LamT tx[6];
    x_proj(lM, tx);
    const float* hl = hb + (buf * 2 * AFY + row) * 8;
    const float* hr = hl + AFY * 8;
    const float4 hl4 = *reinterpret_cast<const float4*>(hl);
    const float2 hl2 = *reinterpret_cast<const float2*>(hl + 4);
    const float4 hr4 = *reinterpret_cast<const float4*>(hr);
    const float2 hr2 = *reinterpret_cast<const float2*>(hr + 4);
    const float hlv[6] = {hl4.x, hl4.y, hl4.z, hl4.w, hl2.x, hl2.y};
    const float hrv[6] = {hr4.x, hr4.y, hr4.z, hr4.w, hr2.x, hr2.y};
    float X[6][3];  // [x slice (q, r)][p]
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      float lp = __shfl_down_sync(FULL, tx[s].p, 1);
      float lm = __shfl_up_sync(FULL, tx[s].m, 1);
      lm = left_end ? hlv[s] : lm;
      lp = right_end ? hrv[s] : lp;
      phi_t(lp, tx[s].z, lm, X[s][0], X[s][1], X[s][2]);
    }
    // y projection of the nine (p, r) slices (slot 3 p + r), inputs over q
    float yp[9], ym[9], yz[9];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const LamT a = proj_t(X[0][p], X[1][p], X[3][p]);
      const LamT b = proj_t(X[2][p], X[4][p], 0.f);
      const LamT c = proj_t(X[5][p], 0.f, 0.f);
      yp[3 * p] = a.p, ym[3 * p] = a.m, yz[3 * p] = a.z;
      yp[3 * p + 1] = b.p, ym[3 * p + 1] = b.m, yz[3 * p + 1] = b.z;
      yp[3 * p + 2] = c.p, ym[3 * p + 2] = c.m, yz[3 * p + 2] = c.z;
    }
    const int o4 = buf * (AY4 / 2), o1 = buf * (AY1 / 2);
    yp4[o4] = make_float4(yp[0], yp[1], yp[2], yp[3]);
    yp4[o4 + AFX] = make_float4(yp[4], yp[5], yp[6], yp[7]);
    ym4[o4] = make_float4(ym[0], ym[1], ym[2], ym[3]);
    ym4[o4 + AFX] = make_float4(ym[4], ym[5], ym[6], ym[7]);
    yp1[o1] = yp[8];
    ym1[o1] = ym[8];
    const float gcur[3] = {gprev[0], gprev[1], gprev[2]};
    gprev[0] = 0.5f * lJ[0];
    gprev[1] = 0.5f * lJ[1];
    gprev[2] = 0.5f * lJ[2];
    __syncthreads();
    if (!owned_row) {
      // ---- phase B of the halo warps: plane zz + 2's halo cells into buffer i & 1
      if (i + 2 < n_it) {
        halo_finish(buf);
        if (i + 3 < n_it) halo_loads(zz + 3);
      }
      continue;
    }
    // ---- phase B: y^T (lpl of y + 1, lmr of y - 1)
    float Y[3][3][3];  // [p][r][q]
    {
      const float4 pa = yp4[o4 + 2 * AFX], pb = yp4[o4 + 3 * AFX];  // row + 1
      const float4 ma = ym4[o4 - 2 * AFX], mb = ym4[o4 - AFX];      // row - 1
      const float lp[9] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w, yp1[o1 + AFX]};
      const float lm[9] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w, ym1[o1 - AFX]};
#pragma unroll
      for (int s = 0; s < 9; ++s)
        phi_t(lp[s], yz[s], lm[s], Y[s / 3][s % 3][0], Y[s / 3][s % 3][1], Y[s / 3][s % 3][2]);
    }
    // z projection of the (p, q) slices (00) (10) (01) (20) (02) (11) (21) (12) [(22)],
    // inputs over r; z^T of plane zz - 1 with its carried lz and plane zz - 2's lmr
    constexpr int ZP[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2}, ZQ[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
    float Z[NZS][3];
#pragma unroll
    for (int k = 0; k < NZS; ++k) {
      const LamT t = proj_t(Y[ZP[k]][0][ZQ[k]], Y[ZP[k]][1][ZQ[k]], Y[ZP[k]][2][ZQ[k]]);
      phi_t(t.p, zl[k], m2[k], Z[k][0], Z[k][1], Z[k][2]);
      m2[k] = m1[k];
      m1[k] = t.m;
      zl[k] = t.z;
    }
    if (!out_plane) continue;
    const uint32_t n_out = no;
    no += plane;
    if (!own) continue;
    // ---- Coll^T at plane zz - 1
    if (solid_out) {
#pragma unroll
      for (int k = 0; k < 10; ++k) P.lam_out[n_out + uint32_t(k) * NN] = 0.f;
      continue;
    }
    // Mom17 order: 000 100 010 001 200 020 002 110 101 011 210 120 201 102 021 012 111
    float lmu[17] = {Z[0][0], Z[1][0], Z[2][0], Z[0][1], Z[3][0], Z[4][0],
                     Z[0][2], Z[5][0], Z[1][1], Z[2][1], Z[6][0], Z[7][0],
                     Z[3][1], Z[1][2], Z[4][1], Z[2][2], Z[5][1]};
    if constexpr (Q19) {
      // D3Q19: mu_111 = 0, and the ten further tensor moments are the linear
      // closure of the others (closure19), whose transpose adds their adjoints
      lmu[16] = 0.f;
      const float l202 = Z[3][2], l022 = Z[4][2], l112 = Z[5][2];
      const float l211 = Z[6][1], l212 = Z[6][2], l121 = Z[7][1], l122 = Z[7][2];
      const float l220 = Z[NZS - 1][0], l221 = Z[NZS - 1][1], l222 = Z[NZS - 1][2];
      lmu[6] -= l220 * (1.0f / 6.0f) + l222 * (1.0f / 18.0f);
      lmu[5] -= l202 * (1.0f / 6.0f) + l222 * (1.0f / 18.0f);
      lmu[4] -= l022 * (1.0f / 6.0f) + l222 * (1.0f / 18.0f);
      lmu[9] -= l211 * (1.0f / 3.0f);
      lmu[8] -= l121 * (1.0f / 3.0f);
      lmu[7] -= l112 * (1.0f / 3.0f);
      lmu[12] -= l221 * (1.0f / 3.0f);
      lmu[14] -= l221 * (1.0f / 3.0f);
      lmu[3] -= l221 * (1.0f / 9.0f);
      lmu[10] -= l212 * (1.0f / 3.0f);
      lmu[15] -= l212 * (1.0f / 3.0f);
      lmu[2] -= l212 * (1.0f / 9.0f);
      lmu[11] -= l122 * (1.0f / 3.0f);
      lmu[13] -= l122 * (1.0f / 3.0f);
      lmu[1] -= l122 * (1.0f / 9.0f);
      lmu[0] -= l222 * (1.0f / 27.0f);
    }
    float lf[3] = {0.f, 0.f, 0.f};
    Stored st;
    st.drho = mt[0];
    st.ux = mt[1];
    st.uy = mt[2];
    st.uz = mt[3];
    st.nxx = mt[4];
    st.nyy = mt[5];
    st.nzz = mt[6];
    st.nxy = mt[7];
    st.nxz = mt[8];
    st.nyz = mt[9];
    float lin[10];
    collide_vjp<FORCE>(st, P.omega, fo, lmu, lin, lf);
#pragma unroll
    for (int k = 0; k < 10; ++k) P.lam_out[n_out + uint32_t(k) * NN] = lin[k];
    if (FORCE)
#pragma unroll
      for (int a = 0; a < 3; ++a) P.gF[n_out + uint32_t(a) * NN] = go[a] + (lf[a] + gcur[a]);
  }
}

// Bounce-back terms of the listed FLUID_BOUNDARY cells: a solid link i of cell x
// took f_i(x) = f+_opp(i)(x), so lambda_f_i(x) flows back onto x's own Hermite
// moments; Coll^T is linear in them, so its image is added to lam_out.
template <bool FORCE, bool Q19>
__global__ void adj_boundary_kernel(const float* lam_next, const float* m_next, const float* m_t,
                                    const float* F, const uint32_t* cells, const uint32_t* words,
                                    int64_t count, float* lam_out, float* gF, float omega, int64_t N_) {
  const int64_t k = int64_t(blockIdx.x) * AT + threadIdx.x;
  if (k >= count) return;
  const uint32_t word = words[k];
  const uint32_t links = word & 0x7FFFFFFu;
  if ((word >> 27) != T_FLUID_BOUNDARY || !links) return;
  const size_t N = size_t(N_), n = cells[k];
  float lam[10], lM[10], lJ[3];
  for (int c = 0; c < 10; ++c) lam[c] = lam_next[c * N + n];
  fin_vjp_cell(load_stored<ST_F32>(m_next, N, n), lam, lM, lJ);
  float lmu[17];
  for (int c = 0; c < 17; ++c) lmu[c] = 0.f;
  for (int i = 0; i < 27; ++i) {
    if (!((links >> i) & 1u)) continue;
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    if (Q19 && !in_d3q19(cx, cy, cz)) continue;
    const float fx = float(cx), fy = float(cy), fz = float(cz);
    const float lf = lM[0] + fx * lM[1] + fy * lM[2] + fz * lM[3] +
                     (fx * fx - (1.0f / 3.0f)) * lM[4] + (fy * fy - (1.0f / 3.0f)) * lM[5] +
                     (fz * fz - (1.0f / 3.0f)) * lM[6] + fx * fy * lM[7] + fx * fz * lM[8] +
                     fy * fz * lM[9];
    if (Q19)
      add_population_adjoint19(-cx, -cy, -cz, lf, lmu);
    else
      add_population_adjoint(-cx, -cy, -cz, lf, lmu);
  }
  float f[3] = {0.f, 0.f, 0.f}, lff[3] = {0.f, 0.f, 0.f};
  if (FORCE)
    for (int a = 0; a < 3; ++a) f[a] = F[a * N + n];
  float lin[10];
  collide_vjp<FORCE>(load_stored<ST_F32>(m_t, N, n), omega, f, lmu, lin, lff);
  for (int c = 0; c < 10; ++c) lam_out[c * N + n] += lin[c];
  if (FORCE)
    for (int a = 0; a < 3; ++a) gF[a * N + n] += lff[a];
}

unsigned blocks_for(int64_t N) { return unsigned((N + AT - 1) / AT); }

template <bool FORCE, bool TYPED, bool Q19>
cudaError_t launch_adj_stream_t(AdjStreamParams& p, cudaStream_t st) {
  constexpr int MAX_DEV = 64;
  static int sms[MAX_DEV] = {};  // per device, once: SM count and the shared-memory opt-in
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  if (!sms[dev]) {
    int n = 0;
    e = cudaFuncSetAttribute(adj_stream_kernel<FORCE, TYPED, Q19>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(ADJ_SMEM));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms[dev] = n > 0 ? n : 1;
  }
  // z-chunk: minimise waves (one block per SM) times the planes a block marches
  const int64_t tiles = int64_t((p.nx + AFX - 1) / AFX) * ((p.ny + AIY - 1) / AIY);
  int best = 1;
  int64_t best_cost = INT64_MAX;
  for (int zc = std::min(p.nz, 256); zc >= 1; --zc) {
    const int64_t blocks = tiles * ((p.nz + zc - 1) / zc);
    const int64_t cost = (blocks + sms[dev] - 1) / sms[dev] * (zc + 2);
    if (cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  p.zc = best;
  const dim3 grid((p.nx + AFX - 1) / AFX, (p.ny + AIY - 1) / AIY, (p.nz + best - 1) / best);
  adj_stream_kernel<FORCE, TYPED, Q19><<<grid, dim3(AFX, AFY), ADJ_SMEM, st>>>(p);
  return cudaGetLastError();
}

template <bool Q19>
cudaError_t launch_adj_stream_l(AdjStreamParams& p, bool force, cudaStream_t st) {
  if (force)
    return p.type ? launch_adj_stream_t<true, true, Q19>(p, st)
                  : launch_adj_stream_t<true, false, Q19>(p, st);
  return p.type ? launch_adj_stream_t<false, true, Q19>(p, st)
                : launch_adj_stream_t<false, false, Q19>(p, st);
}

cudaError_t launch_adj_stream(AdjStreamParams& p, bool force, int lattice, cudaStream_t st) {
  return lattice == 19 ? launch_adj_stream_l<true>(p, force, st) : launch_adj_stream_l<false>(p, force, st);
}

}  // namespace
}  // namespace melbm

using namespace melbm;

namespace {
bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int adj_fail(melbm_t h, int code, const char* msg) {
  h->err = msg;
  return code;
}

#define ADJ_CUDA(h, call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      h->err = std::string(#call ": ") + cudaGetErrorString(e_);             \
      return MELBM_ECUDA;                                                    \
    }                                                                        \
  } while (0)
}  // namespace

extern "C" int melbm_forward_checkpointed(melbm_t h, const float* u0, int nsteps, int K) {
  if (!h) return MELBM_EINVAL;
  if (!u0 || !is_dev(u0)) return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: u0 must be a device pointer");
  if (nsteps < 1 || K < 1) return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: nsteps and K must be >= 1");
  if (h->storage != MELBM_F32)
    return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: requires MELBM_F32 storage");
  if (h->wall_model != 0)
    return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: the adjoint covers halfway bounce-back walls only");
  if (10 * uint64_t(h->N) >= (uint64_t(1) << 32))
    return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: the adjoint takes grids of fewer than 429496730 cells");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error)
    return adj_fail(h, MELBM_ESTATE, "melbm_forward_checkpointed: the last boundary setup failed");
  ADJ_CUDA(h, join_transfers(h));
  const size_t N = size_t(h->N);
  AdjointState* a = h->adj;
  const int nck = (nsteps - 1) / K;  // checkpoints at t = K, 2K, ... < nsteps
  if (!a || a->N != h->N || a->K != K || a->nck < nck) {
    if (a) {
      h->mem_bytes -= a->bytes;
      adjoint_free(a);
    }
    a = new (std::nothrow) AdjointState;
    if (!a) return adj_fail(h, MELBM_ENOMEM, "melbm_forward_checkpointed: host allocation failed");
    h->adj = a;
    a->N = h->N;
    a->K = K;
    a->nck = nck;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&a->u0, N * 12);
    if (e == cudaSuccess && nck) e = cudaMalloc(&a->ckpt, N * 20 * size_t(nck));
    if (e == cudaSuccess) e = cudaMalloc(&a->seg, N * 40 * size_t(K + 1));
    if (e == cudaSuccess) e = cudaMalloc(&a->lam, N * 40);
    if (e == cudaSuccess) e = cudaMalloc(&a->lam2, N * 40);
    if (e == cudaSuccess) e = cudaMalloc(&a->gF, N * 12);
    if (e == cudaSuccess && nck) e = cudaMalloc(&a->seg2, N * 40 * size_t(K + 1));
    if (e == cudaSuccess && nck) e = cudaStreamCreateWithFlags(&a->rs, cudaStreamNonBlocking);
    if (e == cudaSuccess && nck) e = cudaEventCreateWithFlags(&a->ev_start, cudaEventDisableTiming);
    for (int b = 0; b < 2 && nck; ++b) {
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->ev_rec[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->ev_used[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      adjoint_free(a);
      h->adj = nullptr;
      return adj_fail(h, MELBM_ENOMEM, "melbm_forward_checkpointed: device allocation failed");
    }
    a->bytes = a->N * 4 * (3 + 10 * (K + 1) * (nck ? 2 : 1) + 23) + a->N * 20 * int64_t(nck);
    h->mem_bytes += a->bytes;
  }
  a->ready = false;
  a->seg_filled = false;
  a->nsteps = nsteps;
  ADJ_CUDA(h, cudaMemcpyAsync(a->u0, u0, N * 12, cudaMemcpyDeviceToDevice, h->stream));
  if (nsteps <= K) {
    // one segment: its states stay in seg, so the backward pass needs no recompute
    // (the same kernels on the same inputs: the states it would recompute)
    init_from_u0_kernel<<<blocks_for(h->N), AT, 0, h->stream>>>(a->u0, a->seg, h->N);
    ADJ_CUDA(h, cudaGetLastError());
    for (int t = 0; t < nsteps; ++t)
      ADJ_CUDA(h, forward_step(h, a->seg + size_t(t) * 10 * N, a->seg + size_t(t + 1) * 10 * N,
                               uint32_t(t + 1)));
    ADJ_CUDA(h, cudaMemcpyAsync(h->buf[h->cur], a->seg + size_t(nsteps) * 10 * N, N * 40,
                                cudaMemcpyDeviceToDevice, h->stream));
    h->t = nsteps;
    a->seg_filled = true;
    a->ready = true;
    return MELBM_OK;
  }
  init_from_u0_kernel<<<blocks_for(h->N), AT, 0, h->stream>>>(a->u0, static_cast<float*>(h->buf[h->cur]), h->N);
  ADJ_CUDA(h, cudaGetLastError());
  h->t = 0;
  for (int t = 0; t < nsteps; ++t) {
    if (t > 0 && t % K == 0) {
      f32_to_q16_kernel<<<blocks_for(h->N), AT, 0, h->stream>>>(
          static_cast<const float*>(h->buf[h->cur]), a->ckpt + size_t(t / K - 1) * 5 * N, h->nx,
          h->ny, h->nz);
      ADJ_CUDA(h, cudaGetLastError());
    }
    ADJ_CUDA(h, forward_step(h, h->buf[h->cur], h->buf[1 - h->cur], uint32_t(t + 1)));
    h->cur = 1 - h->cur;
    h->t += 1;
  }
  a->ready = true;
  return MELBM_OK;
}

extern "C" int melbm_backward(melbm_t h, const float* dL_dm, float* dL_du0, float* dL_dF) {
  if (!h) return MELBM_EINVAL;
  AdjointState* a = h->adj;
  if (!a || !a->ready)
    return adj_fail(h, MELBM_ESTATE, "melbm_backward: call melbm_forward_checkpointed first");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error)
    return adj_fail(h, MELBM_ESTATE, "melbm_backward: the last boundary setup failed");
  if (!dL_dm || !dL_du0 || !is_dev(dL_dm) || !is_dev(dL_du0) || (dL_dF && !is_dev(dL_dF)))
    return adj_fail(h, MELBM_EINVAL, "melbm_backward: gradients must be device pointers");
  ADJ_CUDA(h, join_transfers(h));
  const size_t N = size_t(h->N);
  const unsigned nb = blocks_for(h->N);
  const float omega = 1.0f / h->tau;
  cudaStream_t st = h->stream;
  pub_vjp_kernel<<<nb, AT, 0, st>>>(static_cast<const float*>(h->buf[h->cur]), dL_dm, a->lam, h->N);
  ADJ_CUDA(h, cudaGetLastError());
  ADJ_CUDA(h, cudaMemsetAsync(a->gF, 0, N * 12, st));
  const int K = a->K, nsteps = a->nsteps;
  const int nseg = (nsteps + K - 1) / K;
  float* lam = a->lam;
  float* lam2 = a->lam2;
  // Segment sg's FP32 states live in buffer sg & 1 (seg or seg2).  The recompute
  // of segment sg - 1 runs on the stream rs while the adjoint walks segment sg on
  // the handle's stream; ev_rec orders each adjoint segment after its recompute,
  // ev_used each recompute after the adjoint that last read its buffer.
  auto segbuf = [&](int sg) { return (sg & 1) ? a->seg2 : a->seg; };
  auto recompute = [&](int sg) -> cudaError_t {
    const int s0 = sg * K, e0 = (s0 + K < nsteps) ? s0 + K : nsteps;
    float* b = segbuf(sg);
    if (sg == 0)
      init_from_u0_kernel<<<nb, AT, 0, a->rs>>>(a->u0, b, h->N);
    else
      q16_to_f32_kernel<<<nb, AT, 0, a->rs>>>(a->ckpt + size_t(sg - 1) * 5 * N, b, h->N);
    cudaError_t e = cudaGetLastError();
    for (int j = 1; j <= e0 - s0 && e == cudaSuccess; ++j)
      e = forward_step_on(h, b + size_t(j - 1) * 10 * N, b + size_t(j) * 10 * N, uint32_t(s0 + j),
                          a->rs);
    if (e == cudaSuccess) e = cudaEventRecord(a->ev_rec[sg & 1], a->rs);
    return e;
  };
  if (!a->seg_filled) {
    // the recompute stream follows everything issued on the handle's stream so far
    ADJ_CUDA(h, cudaEventRecord(a->ev_start, st));
    ADJ_CUDA(h, cudaStreamWaitEvent(a->rs, a->ev_start, 0));
    ADJ_CUDA(h, recompute(nseg - 1));
  }
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s = sg * K, e = (s + K < nsteps) ? s + K : nsteps;
    const float* sb = a->seg_filled ? a->seg : segbuf(sg);
    if (!a->seg_filled) {
      if (sg >= 1) {
        // buffer (sg - 1) & 1 was last read by the adjoint of segment sg + 1
        if (sg + 1 < nseg) ADJ_CUDA(h, cudaStreamWaitEvent(a->rs, a->ev_used[(sg + 1) & 1], 0));
        ADJ_CUDA(h, recompute(sg - 1));
      }
      ADJ_CUDA(h, cudaStreamWaitEvent(st, a->ev_rec[sg & 1], 0));
    }
    for (int t = e - 1; t >= s; --t) {
      const int j = t - s;
      const float* m_t = sb + size_t(j) * 10 * N;
      const float* m_next = sb + size_t(j + 1) * 10 * N;
      if (h->outflow_on && h->type) {
        outflow_vjp_kernel<<<blocks_for(int64_t(h->ny) * h->nz), AT, 0, st>>>(lam, h->type, h->nx,
                                                                             h->ny, h->nz);
        ADJ_CUDA(h, cudaGetLastError());
      }
      AdjStreamParams ap;
      ap.nx = h->nx;
      ap.ny = h->ny;
      ap.nz = h->nz;
      ap.zc = 0;
      ap.lam_next = lam;
      ap.m_t = m_t;
      ap.lam_out = lam2;
      ap.m_next = m_next;
      ap.force = h->force;
      ap.gF = a->gF;
      ap.type = h->type;
      ap.omega = omega;
      ADJ_CUDA(h, launch_adj_stream(ap, h->force != nullptr, h->lattice, st));
      if (h->L) {
        const unsigned lb = blocks_for(h->L);
        const bool q19 = h->lattice == MELBM_D3Q19;
        if (h->force && q19)
          adj_boundary_kernel<true, true><<<lb, AT, 0, st>>>(lam, m_next, m_t, h->force, h->list_cell,
                                                             h->list_word, h->L, lam2, a->gF, omega, h->N);
        else if (h->force)
          adj_boundary_kernel<true, false><<<lb, AT, 0, st>>>(lam, m_next, m_t, h->force, h->list_cell,
                                                              h->list_word, h->L, lam2, a->gF, omega, h->N);
        else if (q19)
          adj_boundary_kernel<false, true><<<lb, AT, 0, st>>>(lam, m_next, m_t, nullptr, h->list_cell,
                                                              h->list_word, h->L, lam2, a->gF, omega, h->N);
        else
          adj_boundary_kernel<false, false><<<lb, AT, 0, st>>>(lam, m_next, m_t, nullptr, h->list_cell,
                                                               h->list_word, h->L, lam2, a->gF, omega, h->N);
        ADJ_CUDA(h, cudaGetLastError());
      }
      float* tmp = lam;
      lam = lam2;
      lam2 = tmp;
    }
    if (!a->seg_filled) ADJ_CUDA(h, cudaEventRecord(a->ev_used[sg & 1], st));
  }
  a->lam = lam;
  a->lam2 = lam2;
  // initial state (rho, u, n) = (1, u0, 0): only the velocity depends on u0
  ADJ_CUDA(h, cudaMemcpyAsync(dL_du0, lam + N, N * 12, cudaMemcpyDeviceToDevice, st));
  if (dL_dF) ADJ_CUDA(h, cudaMemcpyAsync(dL_dF, a->gF, N * 12, cudaMemcpyDeviceToDevice, st));
  return MELBM_OK;
}
