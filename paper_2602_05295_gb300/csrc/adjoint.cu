// adjoint.cu -- hand-written discrete adjoint of the FP32-storage step, with
// 16-bit checkpointing (the paper has no adjoint; inverse design motivates it,
// Sec. 1).  One forward step is  m' = Fin(Stream(Coll(m, F)), F)  per cell, with
// bounce-back, inflow and outflow applied by the boundary kernels.  Its
// vector-Jacobian product is taken by one fused kernel and one list kernel:
//   1. adj_stream_kernel, over every cell: lambda_M = (dFin/dM)^T lambda' (and
//      dL/dF from the F/2 of Eq. rho_u_stress), zero for solid, inflow and
//      outflow cells; then the transpose of the separable pull stream of the
//      fluid kernel (Eq. streaming), back onto the 17 Hermite moments of each
//      source cell, with three transposed 1D passes (z in registers, y through
//      shared memory, x by shuffles); then (dColl/dm)^T (App. A transposed by
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
  float* lam = nullptr;       // 10N adjoint of the stored variables
  float* lam2 = nullptr;      // 10N
  float* gF = nullptr;        // 3N accumulated dL/dF
};

void adjoint_free(AdjointState* a) {
  if (!a) return;
  cudaFree(a->u0);
  cudaFree(a->ckpt);
  cudaFree(a->seg);
  cudaFree(a->lam);
  cudaFree(a->lam2);
  cudaFree(a->gF);
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
  const float rho = 1.0f + o.drho, inv = 1.0f / rho;
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
    inv = 1.0f / rho;
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
// m2 = (2/3)(pl + mr) - z/3.  Its transpose, per axis and in reverse order
// (z, then y, then x), is the same three-point stencil read the other way:
//   proj^T: lpl = l0 + l1 + (2/3) l2,  lmr = l0 - l1 + (2/3) l2,  lz = l0 - l2/3;
//   push:   lphi+(x) = lpl(x + 1), lphi-(x) = lmr(x - 1), lphi0 = lz;
//   phi^T:  ls = lphi+ + lphi- - 2 lphi0, lmu0 = lphi0 + ls/6, lmu1 = (lphi+ - lphi-)/2,
//           lmu2 = ls/2.
// Carried adjoints mirror the forward's moment counts: 10 -> 18 (z) -> 24 (y) -> 17 (x);
// on D3Q19 the x pass yields all 27 tensor moments, folded back onto the 17 through
// the transposed closure.
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

constexpr int AFX = 32;             // lanes: columns x0 .. x0+31, lanes 0 and 31 halo
constexpr int AFY = 16;             // warps: rows y0 .. y0+15, warps 0 and 15 halo
constexpr int AIX = AFX - 2, AIY = AFY - 2;
constexpr int ANS = 9;              // y-pass slices (d, r)
constexpr int ASM = 2 * ANS * AFY * AFX;  // floats per buffer (lpl and lmr)
constexpr size_t ADJ_SMEM = size_t(2) * ASM * sizeof(float);

struct AdjStreamParams {
  int nx, ny, nz, zc;
  const float* lam_next;  // adjoint of the output state (10N, stored variables)
  const float* m_next;    // output state (10N)
  const float* m_t;       // input state (10N)
  const float* force;     // 3N or null
  const uint8_t* type;    // N or null
  float* lam_out;         // adjoint of the input state (10N)
  float* gF;              // 3N, accumulated
  float omega;
};

// One thread per (x, y) column marching in z: fin^T and the z^T projection at
// plane zz, the rest of z^T, y^T (shared memory), x^T (shuffles) and Coll^T
// for the plane zz - 1.  Periodic in all directions; cells whose output does
// not come from the stream contribute no adjoint (special_type), and solid cells
// get none; the bounce-back terms of listed cells are added by adj_boundary_kernel.
template <bool FORCE, bool TYPED, bool Q19>
__global__ void __launch_bounds__(AFX* AFY, 1) adj_stream_kernel(AdjStreamParams P) {
  extern __shared__ float asm_[];
  const int lane = threadIdx.x, row = threadIdx.y;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz, plane = size_t(nx) * ny;
  const int x = int(blockIdx.x) * AIX - 1 + lane, y = int(blockIdx.y) * AIY - 1 + row;
  const size_t col = size_t(wrapi(x, nx)) + size_t(nx) * wrapi(y, ny);
  const bool mid_row = row >= 1 && row <= AFY - 2;
  const bool own = mid_row && lane >= 1 && lane <= AFX - 2 && x < nx && y < ny;
  const int z0 = int(blockIdx.z) * P.zc, z1 = min(z0 + P.zc, nz);
  // z-march state per (d, e) slice: lz of plane zz-1, lmr of planes zz-1 and zz-2
  float zl[6], m1[6], m2[6];
  for (int k = 0; k < 6; ++k) zl[k] = m1[k] = m2[k] = 0.f;
  float gprev[3] = {0.f, 0.f, 0.f};  // F/2 share of fin^T at plane zz-1
  // plane zz's lambda' and output state are loaded one iteration ahead (of the
  // output state Fin^T needs only rho - 1 and u)
  float Lnext[10], Mnext[4];
  bool skip_next = false;
  auto load_plane = [&](int zp) {
    const size_t n = col + plane * size_t(wrapi(zp, nz));
    skip_next = TYPED && special_type(P.type[n]);
#pragma unroll
    for (int k = 0; k < 10; ++k) Lnext[k] = __ldg(P.lam_next + k * N + n);
#pragma unroll
    for (int k = 0; k < 4; ++k) Mnext[k] = __ldg(P.m_next + k * N + n);
  };
  load_plane(z0 - 1);
  int parity = 0;
  for (int zz = z0 - 1; zz <= z1; ++zz, parity ^= 1) {
    const int zo = zz - 1;  // the plane finished in this iteration
    const bool out_plane = zo >= z0;
    // the input state (and force, gradient) of plane zo, used after the passes
    const bool do_out = out_plane && own;
    float mt[10], fo[3] = {0.f, 0.f, 0.f}, go[3] = {0.f, 0.f, 0.f};
    bool solid_out = false;
    const size_t no = col + plane * size_t(zo < 0 ? 0 : zo);
    if (do_out) {
      solid_out = TYPED && P.type[no] == T_SOLID;
#pragma unroll
      for (int k = 0; k < 10; ++k) mt[k] = __ldg(P.m_t + k * N + no);
      if (FORCE)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          fo[a] = __ldg(P.force + a * N + no);
          go[a] = P.gF[a * N + no];
        }
    }
    // ---- fin^T at plane zz, then proj^T along z of the six (d, e) slices
    float lam[10], mn[4];
    const bool skip = skip_next;
#pragma unroll
    for (int k = 0; k < 10; ++k) lam[k] = Lnext[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) mn[k] = Mnext[k];
    if (zz + 1 <= z1) load_plane(zz + 1);
    float lM[10];
    float lJ[3] = {0.f, 0.f, 0.f};
    if (skip) {
      for (int k = 0; k < 10; ++k) lM[k] = 0.f;
    } else {
      Stored o;  // fin_vjp_cell reads rho - 1 and u of the output only
      o.drho = mn[0];
      o.ux = mn[1];
      o.uy = mn[2];
      o.uz = mn[3];
      o.nxx = o.nyy = o.nzz = o.nxy = o.nxz = o.nyz = 0.f;
      fin_vjp_cell(o, lam, lM, lJ);
    }
    // slices (d, e) = (0,0) (1,0) (0,1) (2,0) (1,1) (0,2), inputs over f
    const LamT t[6] = {proj_t(lM[0], lM[3], lM[6]), proj_t(lM[1], lM[8], 0.f),
                       proj_t(lM[2], lM[9], 0.f),   proj_t(lM[4], 0.f, 0.f),
                       proj_t(lM[7], 0.f, 0.f),     proj_t(lM[5], 0.f, 0.f)};
    float Z[6][3];  // lZ[(d, e)][r] of plane zo
    for (int k = 0; k < 6; ++k) {
      phi_t(t[k].p, zl[k], m2[k], Z[k][0], Z[k][1], Z[k][2]);
      m2[k] = m1[k];
      m1[k] = t[k].m;
      zl[k] = t[k].z;
    }
    const float gcur[3] = {gprev[0], gprev[1], gprev[2]};
    gprev[0] = 0.5f * lJ[0];
    gprev[1] = 0.5f * lJ[1];
    gprev[2] = 0.5f * lJ[2];
    if (!out_plane) continue;  // block-uniform
    // ---- y^T on slices (d, r): inputs over e
    float* sp = asm_ + parity * ASM;
    // lZ by (d, e): index of (d, e) in the six slices, -1 = absent
    const int DE[3][3] = {{0, 2, 5}, {1, 4, -1}, {3, -1, -1}};
    float yz[ANS];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float e0 = Z[DE[d][0]][r];
        const float e1 = DE[d][1] >= 0 ? Z[DE[d][1]][r] : 0.f;
        const float e2 = DE[d][2] >= 0 ? Z[DE[d][2]][r] : 0.f;
        const LamT u = proj_t(e0, e1, e2);
        const int s_ = 3 * d + r;
        sp[(s_ * AFY + row) * AFX + lane] = u.p;
        sp[((ANS + s_) * AFY + row) * AFX + lane] = u.m;
        yz[s_] = u.z;
      }
    __syncthreads();
    if (!mid_row) continue;
    float Y[3][3][3];  // lY[d][q][r]
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int s_ = 3 * d + r;
        const float lp = sp[(s_ * AFY + row + 1) * AFX + lane];         // lpl of y + 1
        const float lm = sp[((ANS + s_) * AFY + row - 1) * AFX + lane];  // lmr of y - 1
        phi_t(lp, yz[s_], lm, Y[d][0][r], Y[d][1][r], Y[d][2][r]);
      }
    // ---- x^T on slices (q, r): inputs over d, exchanged by shuffles
    float X[3][3][3];  // lmu[p][q][r]
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (!Q19 && q == 2 && r == 2) continue;  // no D3Q27 Hermite moment has q = r = 2
        const LamT u = proj_t(Y[0][q][r], Y[1][q][r], Y[2][q][r]);
        const float lp = __shfl_down_sync(FULL, u.p, 1);  // lpl of x + 1
        const float lm = __shfl_up_sync(FULL, u.m, 1);    // lmr of x - 1
        phi_t(lp, u.z, lm, X[0][q][r], X[1][q][r], X[2][q][r]);
      }
    if (!own) continue;
    // ---- Coll^T at plane zo
    if (solid_out) {
      for (int k = 0; k < 10; ++k) P.lam_out[k * N + no] = 0.f;
      continue;
    }
    // Mom17 order: 000 100 010 001 200 020 002 110 101 011 210 120 201 102 021 012 111
    float lmu[17] = {X[0][0][0], X[1][0][0], X[0][1][0], X[0][0][1], X[2][0][0],
                     X[0][2][0], X[0][0][2], X[1][1][0], X[1][0][1], X[0][1][1],
                     X[2][1][0], X[1][2][0], X[2][0][1], X[1][0][2], X[0][2][1],
                     X[0][1][2], X[1][1][1]};
    if constexpr (Q19) {
      // D3Q19: mu_111 = 0, and the ten further tensor moments are the linear
      // closure of the others (closure19), whose transpose adds their adjoints
      lmu[16] = 0.f;
      const float l220 = X[2][2][0], l202 = X[2][0][2], l022 = X[0][2][2];
      const float l211 = X[2][1][1], l121 = X[1][2][1], l112 = X[1][1][2];
      const float l221 = X[2][2][1], l212 = X[2][1][2], l122 = X[1][2][2], l222 = X[2][2][2];
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
    for (int k = 0; k < 10; ++k) P.lam_out[k * N + no] = lin[k];
    if (FORCE)
      for (int a = 0; a < 3; ++a) P.gF[a * N + no] = go[a] + (lf[a] + gcur[a]);
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
  const int64_t tiles = int64_t((p.nx + AIX - 1) / AIX) * ((p.ny + AIY - 1) / AIY);
  int best = 1;
  int64_t best_cost = INT64_MAX;
  for (int zc = std::min(p.nz, 128); zc >= 1; --zc) {
    const int64_t blocks = tiles * ((p.nz + zc - 1) / zc);
    const int64_t cost = (blocks + sms[dev] - 1) / sms[dev] * (zc + 2);
    if (cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  p.zc = best;
  const dim3 grid((p.nx + AIX - 1) / AIX, (p.ny + AIY - 1) / AIY, (p.nz + best - 1) / best);
  adj_stream_kernel<FORCE, TYPED, Q19><<<grid, dim3(AFX, AFY), ADJ_SMEM, st>>>(p);
  return cudaGetLastError();
}

template <bool Q19>
cudaError_t launch_adj_stream_l(AdjStreamParams& p, cudaStream_t st) {
  if (p.force)
    return p.type ? launch_adj_stream_t<true, true, Q19>(p, st)
                  : launch_adj_stream_t<true, false, Q19>(p, st);
  return p.type ? launch_adj_stream_t<false, true, Q19>(p, st)
                : launch_adj_stream_t<false, false, Q19>(p, st);
}

cudaError_t launch_adj_stream(AdjStreamParams& p, int lattice, cudaStream_t st) {
  return lattice == 19 ? launch_adj_stream_l<true>(p, st) : launch_adj_stream_l<false>(p, st);
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
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error)
    return adj_fail(h, MELBM_ESTATE, "melbm_forward_checkpointed: the last boundary setup failed");
  ADJ_CUDA(h, join_transfers(h));
  const size_t N = size_t(h->N);
  AdjointState* a = h->adj;
  const int nck = (nsteps - 1) / K;  // checkpoints at t = K, 2K, ... < nsteps
  if (!a || a->N != h->N || a->K != K || a->nck < nck) {
    if (a) {
      h->mem_bytes -= a->N * 4 * (3 + 10 * (a->K + 1) + 23) + a->N * 20 * int64_t(a->nck);
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
    if (e != cudaSuccess) {
      cudaGetLastError();
      adjoint_free(a);
      h->adj = nullptr;
      return adj_fail(h, MELBM_ENOMEM, "melbm_forward_checkpointed: device allocation failed");
    }
    h->mem_bytes += a->N * 4 * (3 + 10 * (K + 1) + 23) + a->N * 20 * int64_t(nck);
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
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s = sg * K, e = (s + K < nsteps) ? s + K : nsteps;
    float* seg0 = a->seg;
    if (!a->seg_filled) {
      if (sg == 0)
        init_from_u0_kernel<<<nb, AT, 0, st>>>(a->u0, seg0, h->N);
      else
        q16_to_f32_kernel<<<nb, AT, 0, st>>>(a->ckpt + size_t(sg - 1) * 5 * N, seg0, h->N);
      ADJ_CUDA(h, cudaGetLastError());
      for (int j = 1; j <= e - s; ++j)
        ADJ_CUDA(h, forward_step(h, a->seg + size_t(j - 1) * 10 * N, a->seg + size_t(j) * 10 * N,
                                 uint32_t(s + j)));
    }
    for (int t = e - 1; t >= s; --t) {
      const int j = t - s;
      const float* m_t = a->seg + size_t(j) * 10 * N;
      const float* m_next = a->seg + size_t(j + 1) * 10 * N;
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
      ap.m_next = m_next;
      ap.m_t = m_t;
      ap.force = h->force;
      ap.type = h->type;
      ap.lam_out = lam2;
      ap.gF = a->gF;
      ap.omega = omega;
      ADJ_CUDA(h, launch_adj_stream(ap, h->lattice, st));
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
  }
  a->lam = lam;
  a->lam2 = lam2;
  // initial state (rho, u, n) = (1, u0, 0): only the velocity depends on u0
  ADJ_CUDA(h, cudaMemcpyAsync(dL_du0, lam + N, N * 12, cudaMemcpyDeviceToDevice, st));
  if (dL_dF) ADJ_CUDA(h, cudaMemcpyAsync(dL_dF, a->gF, N * 12, cudaMemcpyDeviceToDevice, st));
  return MELBM_OK;
}
