// state.cu -- conversions between the public state (rho, u, S) and the stored
// variables (rho - 1, u, rho S^neq = rho (S - u u)) of Sec. 5.4 (range reduction),
// and the codec on caller buffers.  The quantised form uses the grids of the
// handle's bit widths (QGrids).
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

template <int STORAGE>
__global__ void set_state_kernel(int nx, int ny, int nz, const float* rho, const float* u,
                                 const float* S, void* buf, uint32_t t, uint32_t seed, int det,
                                 QGrids q) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float r = rho[n];
  const float ux = u[n], uy = u[N + n], uz = u[2 * N + n];
  float sxx = ux * ux, syy = uy * uy, szz = uz * uz, sxy = ux * uy, sxz = ux * uz, syz = uy * uz;
  if (S) {
    sxx = S[n];
    syy = S[N + n];
    szz = S[2 * N + n];
    sxy = S[3 * N + n];
    sxz = S[4 * N + n];
    syz = S[5 * N + n];
  }
  Stored s;
  s.drho = r - 1.0f;
  s.ux = ux;
  s.uy = uy;
  s.uz = uz;
  s.nxx = r * (sxx - ux * ux);
  s.nyy = r * (syy - uy * uy);
  s.nzz = r * (szz - uz * uz);
  s.nxy = r * (sxy - ux * uy);
  s.nxz = r * (sxz - ux * uz);
  s.nyz = r * (syz - uy * uz);
  const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
  store_stored<STORAGE>(buf, N, n, s, x, y, z, t, seed, det != 0, q);
}

cudaError_t launch_set_state(int storage, int nx, int ny, int nz, const float* rho, const float* u,
                             const float* S, void* buf, uint32_t t, uint32_t seed, int det,
                             const QGrids& q, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16)
    set_state_kernel<ST_Q16><<<blocks, 256, 0, st>>>(nx, ny, nz, rho, u, S, buf, t, seed, det, q);
  else
    set_state_kernel<ST_F32><<<blocks, 256, 0, st>>>(nx, ny, nz, rho, u, S, buf, t, seed, det, q);
  return cudaGetLastError();
}

template <int STORAGE>
__global__ void rest_state_kernel(int nx, int ny, int nz, void* buf, uint32_t seed, QGrids q) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Stored s;
  s.drho = s.ux = s.uy = s.uz = 0.f;
  s.nxx = s.nyy = s.nzz = s.nxy = s.nxz = s.nyz = 0.f;
  const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
  store_stored<STORAGE>(buf, N, n, s, x, y, z, 0u, seed, false, q);
}

cudaError_t launch_rest_state(int storage, int nx, int ny, int nz, void* buf, uint32_t seed,
                              const QGrids& q, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16) rest_state_kernel<ST_Q16><<<blocks, 256, 0, st>>>(nx, ny, nz, buf, seed, q);
  else rest_state_kernel<ST_F32><<<blocks, 256, 0, st>>>(nx, ny, nz, buf, seed, q);
  return cudaGetLastError();
}

template <int STORAGE>
__global__ void get_moments_kernel(int64_t N_, const void* buf, float* rho, float* u, float* S,
                                   QGrids q) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Stored s = load_stored<STORAGE>(buf, N, n, q);
  const float r = 1.0f + s.drho;
  if (rho) rho[n] = r;
  if (u) {
    u[n] = s.ux;
    u[N + n] = s.uy;
    u[2 * N + n] = s.uz;
  }
  if (S) {
    const float inv = __frcp_rn(r);
    S[n] = s.nxx * inv + s.ux * s.ux;
    S[N + n] = s.nyy * inv + s.uy * s.uy;
    S[2 * N + n] = s.nzz * inv + s.uz * s.uz;
    S[3 * N + n] = s.nxy * inv + s.ux * s.uy;
    S[4 * N + n] = s.nxz * inv + s.ux * s.uz;
    S[5 * N + n] = s.nyz * inv + s.uy * s.uz;
  }
}

cudaError_t launch_get_moments(int storage, int64_t N, const void* buf, float* rho, float* u,
                               float* S, const QGrids& q, cudaStream_t st) {
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16)
    get_moments_kernel<ST_Q16><<<blocks, 256, 0, st>>>(N, buf, rho, u, S, q);
  else
    get_moments_kernel<ST_F32><<<blocks, 256, 0, st>>>(N, buf, rho, u, S, q);
  return cudaGetLastError();
}

// Codec on caller buffers: stored[10][N] with component 0 = rho itself.
__global__ void q16_encode_kernel(const float* v, int nx, int ny, int nz, uint32_t t,
                                  uint32_t seed, int det, uint32_t* words, QGrids q) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Dither d;
  if (det) {
#pragma unroll
    for (int k = 0; k < 10; ++k) d.d[k] = 0.5f;
  } else {
    d = dither10(uint32_t(n % nx), uint32_t((n / nx) % ny), uint32_t(n / (size_t(nx) * ny)), t,
                 seed);
  }
  // component 0 is rho; the codec works on rho - 1 (exact in FP32 for rho in [0.5, 2])
  Stored s;
  s.drho = v[n] - 1.0f;
  s.ux = v[N + n];
  s.uy = v[2 * N + n];
  s.uz = v[3 * N + n];
  s.nxx = v[4 * N + n];
  s.nyy = v[5 * N + n];
  s.nzz = v[6 * N + n];
  s.nxy = v[7 * N + n];
  s.nxz = v[8 * N + n];
  s.nyz = v[9 * N + n];
  uint32_t w[5];
  encode_words(s, d, w, q);
#pragma unroll
  for (int k = 0; k < 5; ++k) words[k * N + n] = w[k];
}

__global__ void q16_decode_kernel(const uint32_t* words, int64_t N_, float* v, QGrids q) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t w0 = words[n], w1 = words[N + n], w2 = words[2 * N + n], w3 = words[3 * N + n],
                 w4 = words[4 * N + n];
  const uint32_t w[5] = {w0, w1, w2, w3, w4};
  const Stored s = decode_words(w, q);
  v[n] = 1.0f + s.drho;
  v[N + n] = s.ux;
  v[2 * N + n] = s.uy;
  v[3 * N + n] = s.uz;
  v[4 * N + n] = s.nxx;
  v[5 * N + n] = s.nyy;
  v[6 * N + n] = s.nzz;
  v[7 * N + n] = s.nxy;
  v[8 * N + n] = s.nxz;
  v[9 * N + n] = s.nyz;
}

cudaError_t launch_q16_encode(const float* stored, int nx, int ny, int nz, uint32_t t,
                              uint32_t seed, int det, uint32_t* words, const QGrids& q,
                              cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  q16_encode_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(stored, nx, ny, nz, t, seed, det,
                                                              words, q);
  return cudaGetLastError();
}

cudaError_t launch_q16_decode(const uint32_t* words, int64_t N, float* stored, const QGrids& q,
                              cudaStream_t st) {
  q16_decode_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(words, N, stored, q);
  return cudaGetLastError();
}

}  // namespace melbm
