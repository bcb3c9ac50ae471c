// state.cu -- conversions between the public state (rho, u, S) and the stored
// variables (rho - 1, u, rho S^neq = rho (S - u u)) of Sec. 5.4 (range reduction),
// and the 16-bit codec on caller buffers.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

template <int STORAGE>
__global__ void set_state_kernel(int nx, int ny, int nz, const float* rho, const float* u,
                                 const float* S, void* buf, uint32_t t, uint32_t seed, int det) {
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
  store_stored<STORAGE>(buf, N, n, s, x, y, z, t, seed, det != 0);
}

cudaError_t launch_set_state(int storage, int nx, int ny, int nz, const float* rho, const float* u,
                             const float* S, void* buf, uint32_t t, uint32_t seed, int det,
                             cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16)
    set_state_kernel<ST_Q16><<<blocks, 256, 0, st>>>(nx, ny, nz, rho, u, S, buf, t, seed, det);
  else
    set_state_kernel<ST_F32><<<blocks, 256, 0, st>>>(nx, ny, nz, rho, u, S, buf, t, seed, det);
  return cudaGetLastError();
}

template <int STORAGE>
__global__ void rest_state_kernel(int nx, int ny, int nz, void* buf, uint32_t seed) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Stored s;
  s.drho = s.ux = s.uy = s.uz = 0.f;
  s.nxx = s.nyy = s.nzz = s.nxy = s.nxz = s.nyz = 0.f;
  const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
  store_stored<STORAGE>(buf, N, n, s, x, y, z, 0u, seed);
}

cudaError_t launch_rest_state(int storage, int nx, int ny, int nz, void* buf, uint32_t seed,
                              cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16) rest_state_kernel<ST_Q16><<<blocks, 256, 0, st>>>(nx, ny, nz, buf, seed);
  else rest_state_kernel<ST_F32><<<blocks, 256, 0, st>>>(nx, ny, nz, buf, seed);
  return cudaGetLastError();
}

template <int STORAGE>
__global__ void get_moments_kernel(int64_t N_, const void* buf, float* rho, float* u, float* S) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Stored s = load_stored<STORAGE>(buf, N, n);
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
                               float* S, cudaStream_t st) {
  const unsigned blocks = unsigned((N + 255) / 256);
  if (storage == ST_Q16)
    get_moments_kernel<ST_Q16><<<blocks, 256, 0, st>>>(N, buf, rho, u, S);
  else
    get_moments_kernel<ST_F32><<<blocks, 256, 0, st>>>(N, buf, rho, u, S);
  return cudaGetLastError();
}

// Codec on caller buffers: stored[10][N] with component 0 = rho itself.
__global__ void q16_encode_kernel(const float* v, int nx, int ny, int nz, uint32_t t,
                                  uint32_t seed, int det, uint32_t* words) {
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
  words[n] = q_pack(q_encode_bits<0>(v[n] - 1.0f, d.d[0]), q_encode_bits<1>(v[N + n], d.d[1]));
  words[N + n] = q_pack(q_encode_bits<1>(v[2 * N + n], d.d[2]), q_encode_bits<1>(v[3 * N + n], d.d[3]));
  words[2 * N + n] = q_pack(q_encode_bits<2>(v[4 * N + n], d.d[4]), q_encode_bits<2>(v[5 * N + n], d.d[5]));
  words[3 * N + n] = q_pack(q_encode_bits<2>(v[6 * N + n], d.d[6]), q_encode_bits<2>(v[7 * N + n], d.d[7]));
  words[4 * N + n] = q_pack(q_encode_bits<2>(v[8 * N + n], d.d[8]), q_encode_bits<2>(v[9 * N + n], d.d[9]));
}

__global__ void q16_decode_kernel(const uint32_t* words, int64_t N_, float* v) {
  const size_t N = size_t(N_);
  const size_t n = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const uint32_t w0 = words[n], w1 = words[N + n], w2 = words[2 * N + n], w3 = words[3 * N + n],
                 w4 = words[4 * N + n];
  const uint32_t w[5] = {w0, w1, w2, w3, w4};
  const Stored s = decode_words(w);
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
                              uint32_t seed, int det, uint32_t* words, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  q16_encode_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(stored, nx, ny, nz, t, seed, det,
                                                              words);
  return cudaGetLastError();
}

cudaError_t launch_q16_decode(const uint32_t* words, int64_t N, float* stored, cudaStream_t st) {
  q16_decode_kernel<<<unsigned((N + 255) / 256), 256, 0, st>>>(words, N, stored);
  return cudaGetLastError();
}

}  // namespace melbm
