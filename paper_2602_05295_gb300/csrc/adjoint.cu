// adjoint.cu -- hand-written discrete adjoint of the FP32-storage step, with
// 16-bit checkpointing (the paper has no adjoint; inverse design motivates it,
// Sec. 1).  One forward step is  m' = Fin(Stream(Coll(m, F)), F)  per cell, with
// bounce-back, inflow and outflow applied by the boundary kernels.  Its
// vector-Jacobian product is taken in two per-cell kernels:
//   1. fin_vjp:  lambda_M = (dFin/dM)^T lambda'   (and dL/dF from the F/2 of
//      Eq. rho_u_stress), zero for solid, inflow and outflow cells;
//   2. stream_collide_vjp, in gather form: the source cell y collects, from each
//      destination y + c_i that pulled population i from it, the adjoint of that
//      population, lambda_f_i = (dM/df_i)^T lambda_M(y + c_i), maps it back onto
//      its 17 Hermite moments with df_i/dmu (the transpose of the pull of
//      Eq. streaming), adds the bounce-back terms f_i(y) = f+_opp(i)(y) of its own
//      solid links, and applies (dColl/dm)^T (App. A transposed by hand).
// The forward states of each segment are recomputed in FP32 from a 16-bit
// checkpoint (deterministic rounding) taken every K steps; the initial state is
// rebuilt exactly from u0.
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
  float* u0 = nullptr;        // 3N
  uint32_t* ckpt = nullptr;   // nck x 5N (16-bit states at t = K, 2K, ...)
  float* seg = nullptr;       // (K + 1) x 10N FP32 states of one segment
  float* lam = nullptr;       // 10N adjoint of the stored variables
  float* lam2 = nullptr;      // 10N
  float* lamM = nullptr;      // 10N adjoint of the streamed moments
  float* gF = nullptr;        // 3N accumulated dL/dF
};

void adjoint_free(AdjointState* a) {
  if (!a) return;
  cudaFree(a->u0);
  cudaFree(a->ckpt);
  cudaFree(a->seg);
  cudaFree(a->lam);
  cudaFree(a->lam2);
  cudaFree(a->lamM);
  cudaFree(a->gF);
  delete a;
}

namespace {

constexpr int AT = 256;

__device__ __forceinline__ void cell_xyz(size_t n, int nx, int ny, int& x, int& y, int& z) {
  x = int(n % size_t(nx));
  y = int((n / size_t(nx)) % size_t(ny));
  z = int(n / (size_t(nx) * size_t(ny)));
}

__device__ __forceinline__ size_t cell_index(int x, int y, int z, int nx, int ny, int nz) {
  return size_t(wrapi(x, nx)) + size_t(nx) * (size_t(wrapi(y, ny)) + size_t(ny) * wrapi(z, nz));
}

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
// n'_ab = M_ab - J_a J_b inv.  The streamed moments are recovered from the output.
template <bool FORCE>
__global__ void fin_vjp_kernel(const float* mnext, const float* F, const uint8_t* type,
                               const float* lam, float* lamM, float* gF, int64_t N_) {
  const size_t N = size_t(N_), n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  const uint8_t t = type ? type[n] : T_FLUID;
  if (t == T_SOLID || t == T_INFLOW || t == T_OUTFLOW) {
    for (int k = 0; k < 10; ++k) lamM[k * N + n] = 0.f;
    return;
  }
  const Stored o = load_f32(mnext, N, n);
  const float rho = 1.0f + o.drho, inv = 1.0f / rho;
  const float J[3] = {o.ux * rho, o.uy * rho, o.uz * rho};
  const float lu[3] = {lam[N + n], lam[2 * N + n], lam[3 * N + n]};
  const float ln[6] = {lam[4 * N + n], lam[5 * N + n], lam[6 * N + n],
                       lam[7 * N + n], lam[8 * N + n], lam[9 * N + n]};
  const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
  float lJ[3] = {lu[0], lu[1], lu[2]};
  float linv = 0.f;
  for (int a = 0; a < 3; ++a) linv += lu[a] * J[a];
  for (int k = 0; k < 6; ++k) {
    lJ[A[k]] -= ln[k] * J[B[k]];
    lJ[B[k]] -= ln[k] * J[A[k]];
    linv -= ln[k] * J[A[k]] * J[B[k]];
  }
  for (int a = 0; a < 3; ++a) lJ[a] *= inv;
  lamM[n] = lam[n] - linv * inv * inv;  // M000
  lamM[N + n] = lJ[0];
  lamM[2 * N + n] = lJ[1];
  lamM[3 * N + n] = lJ[2];
  for (int k = 0; k < 6; ++k) lamM[(4 + k) * N + n] = ln[k];
  if (FORCE)
    for (int a = 0; a < 3; ++a) gF[a * N + n] += 0.5f * lJ[a];
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
    const float l = lmu[16];
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

// lambda_f_i at a destination cell: (dM/df_i)^T lambda_M with
// M = (sum f, sum c f, sum (c c - delta/3) f).
__device__ __forceinline__ float population_lambda(const float* lamM, size_t N, size_t d, int cx,
                                                   int cy, int cz) {
  const float fx = float(cx), fy = float(cy), fz = float(cz);
  return lamM[d] + fx * lamM[N + d] + fy * lamM[2 * N + d] + fz * lamM[3 * N + d] +
         (fx * fx - (1.0f / 3.0f)) * lamM[4 * N + d] + (fy * fy - (1.0f / 3.0f)) * lamM[5 * N + d] +
         (fz * fz - (1.0f / 3.0f)) * lamM[6 * N + d] + fx * fy * lamM[7 * N + d] +
         fx * fz * lamM[8 * N + d] + fy * fz * lamM[9 * N + d];
}

template <bool FORCE>
__global__ void stream_collide_vjp_kernel(const float* m, const float* F, const uint8_t* type,
                                          const float* lamM, float* lam_out, float* gF, float omega,
                                          int nx, int ny, int nz) {
  const size_t N = size_t(nx) * ny * nz, n = size_t(blockIdx.x) * AT + threadIdx.x;
  if (n >= N) return;
  const uint8_t t = type ? type[n] : T_FLUID;
  if (t == T_SOLID) {
    for (int k = 0; k < 10; ++k) lam_out[k * N + n] = 0.f;
    return;
  }
  int x, y, z;
  cell_xyz(n, nx, ny, x, y, z);
  float lmu[17];
  for (int k = 0; k < 17; ++k) lmu[k] = 0.f;
  for (int i = 0; i < 27; ++i) {
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    // destination y + c_i pulled population i from this (non-solid) cell
    const size_t d = cell_index(x + cx, y + cy, z + cz, nx, ny, nz);
    add_population_adjoint(cx, cy, cz, population_lambda(lamM, N, d, cx, cy, cz), lmu);
    // own solid link i (source x - c_i solid): f_i(x) = f+_opp(i)(x)
    if (t == T_FLUID_BOUNDARY && type[cell_index(x - cx, y - cy, z - cz, nx, ny, nz)] == T_SOLID)
      add_population_adjoint(-cx, -cy, -cz, population_lambda(lamM, N, n, cx, cy, cz), lmu);
  }
  float f[3] = {0.f, 0.f, 0.f}, lf[3] = {0.f, 0.f, 0.f};
  if (FORCE)
    for (int a = 0; a < 3; ++a) f[a] = F[a * N + n];
  float lin[10];
  collide_vjp<FORCE>(load_f32(m, N, n), omega, f, lmu, lin, lf);
  for (int k = 0; k < 10; ++k) lam_out[k * N + n] = lin[k];
  if (FORCE)
    for (int a = 0; a < 3; ++a) gF[a * N + n] += lf[a];
}

unsigned blocks_for(int64_t N) { return unsigned((N + AT - 1) / AT); }

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
  if (h->lattice != MELBM_D3Q27)
    return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: requires the D3Q27 lattice");
  if (h->wall_model != 0)
    return adj_fail(h, MELBM_EINVAL, "melbm_forward_checkpointed: the adjoint covers halfway bounce-back walls only");
  const size_t N = size_t(h->N);
  AdjointState* a = h->adj;
  const int nck = (nsteps - 1) / K;  // checkpoints at t = K, 2K, ... < nsteps
  if (!a || a->N != h->N || a->K != K || a->nck < nck) {
    if (a) {
      h->mem_bytes -= a->N * 4 * (3 + 10 * (a->K + 1) + 33) + a->N * 20 * int64_t(a->nck);
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
    if (e == cudaSuccess) e = cudaMalloc(&a->lamM, N * 40);
    if (e == cudaSuccess) e = cudaMalloc(&a->gF, N * 12);
    if (e != cudaSuccess) {
      cudaGetLastError();
      adjoint_free(a);
      h->adj = nullptr;
      return adj_fail(h, MELBM_ENOMEM, "melbm_forward_checkpointed: device allocation failed");
    }
    h->mem_bytes += a->N * 4 * (3 + 10 * (K + 1) + 33) + a->N * 20 * int64_t(nck);
  }
  a->ready = false;
  a->nsteps = nsteps;
  ADJ_CUDA(h, cudaMemcpyAsync(a->u0, u0, N * 12, cudaMemcpyDeviceToDevice, h->stream));
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
  if (!dL_dm || !dL_du0 || !is_dev(dL_dm) || !is_dev(dL_du0) || (dL_dF && !is_dev(dL_dF)))
    return adj_fail(h, MELBM_EINVAL, "melbm_backward: gradients must be device pointers");
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
    if (sg == 0)
      init_from_u0_kernel<<<nb, AT, 0, st>>>(a->u0, seg0, h->N);
    else
      q16_to_f32_kernel<<<nb, AT, 0, st>>>(a->ckpt + size_t(sg - 1) * 5 * N, seg0, h->N);
    ADJ_CUDA(h, cudaGetLastError());
    for (int j = 1; j <= e - s; ++j)
      ADJ_CUDA(h, forward_step(h, a->seg + size_t(j - 1) * 10 * N, a->seg + size_t(j) * 10 * N,
                               uint32_t(s + j)));
    for (int t = e - 1; t >= s; --t) {
      const int j = t - s;
      const float* m_t = a->seg + size_t(j) * 10 * N;
      const float* m_next = a->seg + size_t(j + 1) * 10 * N;
      if (h->outflow_on && h->type) {
        outflow_vjp_kernel<<<blocks_for(int64_t(h->ny) * h->nz), AT, 0, st>>>(lam, h->type, h->nx,
                                                                             h->ny, h->nz);
        ADJ_CUDA(h, cudaGetLastError());
      }
      if (h->force) {
        fin_vjp_kernel<true><<<nb, AT, 0, st>>>(m_next, h->force, h->type, lam, a->lamM, a->gF, h->N);
        stream_collide_vjp_kernel<true><<<nb, AT, 0, st>>>(m_t, h->force, h->type, a->lamM, lam2,
                                                           a->gF, omega, h->nx, h->ny, h->nz);
      } else {
        fin_vjp_kernel<false><<<nb, AT, 0, st>>>(m_next, nullptr, h->type, lam, a->lamM, a->gF, h->N);
        stream_collide_vjp_kernel<false><<<nb, AT, 0, st>>>(m_t, nullptr, h->type, a->lamM, lam2,
                                                            a->gF, omega, h->nx, h->ny, h->nz);
      }
      ADJ_CUDA(h, cudaGetLastError());
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
