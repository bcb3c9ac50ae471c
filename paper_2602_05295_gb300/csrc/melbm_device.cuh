// melbm_device.cuh -- device helpers shared by the CUDA kernels of the library:
// stored-variable layout, the 16-bit codec of Sec. 5.4 with its dither, the
// moment-space collision of App. A written in stored variables, and the
// tensor-product form of the third-order Hermite reconstruction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace melbm {

constexpr unsigned FULL = 0xffffffffu;

enum : uint8_t { T_FLUID = 0, T_FLUID_BOUNDARY = 1, T_INFLOW = 2, T_OUTFLOW = 3, T_SOLID = 4 };
enum { ST_F32 = 0, ST_Q16 = 1 };

// ---------------------------------------------------------------------------
// Stored variables of one cell.  Both storages keep the same ten quantities:
//   drho = rho - 1, u_a, and n_ab = rho S^neq_ab = rho (S_ab - u_a u_b)
// ordered (xx, yy, zz, xy, xz, yz).  Keeping rho - 1 instead of rho removes the
// O(1) rest state from every FP32 sum (its populations w_i stream to themselves).
// FP32 storage: ten planes [10][N] with plane 0 = drho.
// Q16 storage:  five u32 planes [5][N]; word k holds components (2k, 2k+1) in its
//               (low, high) halves; component 0 is rho itself in [0.8, 1.5].
// ---------------------------------------------------------------------------
struct Stored {
  float drho;
  float ux, uy, uz;
  float nxx, nyy, nzz, nxy, nxz, nyz;
};

// ----------------------------------------------------------------- 16-bit codec
// Ranges (Sec. 5.4): rho [0.8, 1.5]; u [-0.4, 0.4]; rho S^neq [-0.1, 0.1].
// Group 0 = rho, 1 = velocity, 2 = rho S^neq.  Constants are the FP32 roundings
// of the exact FP64 values.
template <int G> struct QRange;
template <> struct QRange<0> {
  static constexpr float lo = 0.8f;
  static constexpr float s = float(1.0 / (1.5 - 0.8));
  static constexpr float o = float(-0.8 / (1.5 - 0.8));
  static constexpr float step = float((1.5 - 0.8) / 65535.0);
};
template <> struct QRange<1> {
  static constexpr float lo = -0.4f;
  static constexpr float s = float(1.0 / 0.8);
  static constexpr float o = float(0.4 / 0.8);
  static constexpr float step = float(0.8 / 65535.0);
};
template <> struct QRange<2> {
  static constexpr float lo = -0.1f;
  static constexpr float s = float(1.0 / 0.2);
  static constexpr float o = float(0.1 / 0.2);
  static constexpr float step = float(0.2 / 65535.0);
};

// Encode one value with dither d in [0, 1): q = floor(sat(m s + o) * 65535 + d).
// Returns the bits of the float 2^23 + q, whose low 16 bits are q.
template <int G>
__device__ __forceinline__ uint32_t q_encode_bits(float m, float d) {
  const float t = __saturatef(__fmaf_rn(m, QRange<G>::s, QRange<G>::o));
  const float v = __fmaf_rn(t, 65535.0f, d);
  return __float_as_uint(__fadd_rd(v, 8388608.0f));  // 2^23 + floor(v), exact for v < 2^23
}
__device__ __forceinline__ uint32_t q_pack(uint32_t lo_bits, uint32_t hi_bits) {
  return __byte_perm(lo_bits, hi_bits, 0x5410);
}
// Decode: the code as an exact float, then m = lo + q * step.
__device__ __forceinline__ float q_lo(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7610)) - 8388608.0f;
}
__device__ __forceinline__ float q_hi(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7632)) - 8388608.0f;
}
template <int G>
__device__ __forceinline__ float q_decode(float q) {
  return __fmaf_rn(q, QRange<G>::step, QRange<G>::lo);
}

// Counter-based dither: pcg4d of Jarzynski & Olano, "Hash Functions for GPU
// Rendering", JCGT 9(3) 2020, on (x, y, z, t ^ seed).  Components 0..7 take the
// 12-bit fields [0,12) (even) and [12,24) (odd) of word k/2; components 8 and 9
// take 16 bits made of the top bytes of words (0,1) and (2,3).
struct Dither {
  float d[10];
};
__device__ __forceinline__ Dither dither10(uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                           uint32_t seed) {
  uint32_t v0 = x * 1664525u + 1013904223u;
  uint32_t v1 = y * 1664525u + 1013904223u;
  uint32_t v2 = z * 1664525u + 1013904223u;
  uint32_t v3 = (t ^ seed) * 1664525u + 1013904223u;
  v0 += v1 * v3;
  v1 += v2 * v0;
  v2 += v0 * v1;
  v3 += v1 * v2;
  v0 ^= v0 >> 16;
  v1 ^= v1 >> 16;
  v2 ^= v2 >> 16;
  v3 ^= v3 >> 16;
  v0 += v1 * v3;
  v1 += v2 * v0;
  v2 += v0 * v1;
  v3 += v1 * v2;
  Dither r;
  const uint32_t w[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // the float with bits 0x4B000000 | f (f < 2^23) is 2^23 + f, so
    // (2^23 + f) / 4096 - 2048 = f / 4096 exactly
    r.d[2 * k] = __fmaf_rn(__uint_as_float(0x4B000000u | (w[k] & 0xFFFu)), 1.0f / 4096.0f, -2048.0f);
    r.d[2 * k + 1] =
        __fmaf_rn(__uint_as_float(0x4B000000u | ((w[k] >> 12) & 0xFFFu)), 1.0f / 4096.0f, -2048.0f);
  }
  const uint32_t f8 = (v0 >> 24) | ((v1 >> 24) << 8);
  const uint32_t f9 = (v2 >> 24) | ((v3 >> 24) << 8);
  r.d[8] = __fmaf_rn(__uint_as_float(0x4B000000u | f8), 1.0f / 65536.0f, -128.0f);
  r.d[9] = __fmaf_rn(__uint_as_float(0x4B000000u | f9), 1.0f / 65536.0f, -128.0f);
  return r;
}

// ----------------------------------------------------------------- load / store
template <int STORAGE>
__device__ __forceinline__ Stored load_stored(const void* buf, size_t N, size_t n);

template <>
__device__ __forceinline__ Stored load_stored<ST_F32>(const void* buf, size_t N, size_t n) {
  const float* b = static_cast<const float*>(buf);
  Stored s;
  s.drho = __ldg(b + n);
  s.ux = __ldg(b + N + n);
  s.uy = __ldg(b + 2 * N + n);
  s.uz = __ldg(b + 3 * N + n);
  s.nxx = __ldg(b + 4 * N + n);
  s.nyy = __ldg(b + 5 * N + n);
  s.nzz = __ldg(b + 6 * N + n);
  s.nxy = __ldg(b + 7 * N + n);
  s.nxz = __ldg(b + 8 * N + n);
  s.nyz = __ldg(b + 9 * N + n);
  return s;
}

template <>
__device__ __forceinline__ Stored load_stored<ST_Q16>(const void* buf, size_t N, size_t n) {
  const uint32_t* b = static_cast<const uint32_t*>(buf);
  const uint32_t w0 = __ldg(b + n), w1 = __ldg(b + N + n), w2 = __ldg(b + 2 * N + n),
                 w3 = __ldg(b + 3 * N + n), w4 = __ldg(b + 4 * N + n);
  Stored s;
  s.drho = q_decode<0>(q_lo(w0)) - 1.0f;
  s.ux = q_decode<1>(q_hi(w0));
  s.uy = q_decode<1>(q_lo(w1));
  s.uz = q_decode<1>(q_hi(w1));
  s.nxx = q_decode<2>(q_lo(w2));
  s.nyy = q_decode<2>(q_hi(w2));
  s.nzz = q_decode<2>(q_lo(w3));
  s.nxy = q_decode<2>(q_hi(w3));
  s.nxz = q_decode<2>(q_lo(w4));
  s.nyz = q_decode<2>(q_hi(w4));
  return s;
}

// Store with the dither of (x, y, z, t ^ seed) (Q16) or as FP32.  deterministic
// rounding (dither 1/2) when det is true.
template <int STORAGE>
__device__ __forceinline__ void store_stored(void* buf, size_t N, size_t n, const Stored& s,
                                             uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                             uint32_t seed, bool det = false);

template <>
__device__ __forceinline__ void store_stored<ST_F32>(void* buf, size_t N, size_t n, const Stored& s,
                                                     uint32_t, uint32_t, uint32_t, uint32_t,
                                                     uint32_t, bool) {
  float* b = static_cast<float*>(buf);
  b[n] = s.drho;
  b[N + n] = s.ux;
  b[2 * N + n] = s.uy;
  b[3 * N + n] = s.uz;
  b[4 * N + n] = s.nxx;
  b[5 * N + n] = s.nyy;
  b[6 * N + n] = s.nzz;
  b[7 * N + n] = s.nxy;
  b[8 * N + n] = s.nxz;
  b[9 * N + n] = s.nyz;
}

__device__ __forceinline__ void encode_words(const Stored& s, const Dither& d, uint32_t w[5]) {
  w[0] = q_pack(q_encode_bits<0>(1.0f + s.drho, d.d[0]), q_encode_bits<1>(s.ux, d.d[1]));
  w[1] = q_pack(q_encode_bits<1>(s.uy, d.d[2]), q_encode_bits<1>(s.uz, d.d[3]));
  w[2] = q_pack(q_encode_bits<2>(s.nxx, d.d[4]), q_encode_bits<2>(s.nyy, d.d[5]));
  w[3] = q_pack(q_encode_bits<2>(s.nzz, d.d[6]), q_encode_bits<2>(s.nxy, d.d[7]));
  w[4] = q_pack(q_encode_bits<2>(s.nxz, d.d[8]), q_encode_bits<2>(s.nyz, d.d[9]));
}

template <>
__device__ __forceinline__ void store_stored<ST_Q16>(void* buf, size_t N, size_t n, const Stored& s,
                                                     uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                                     uint32_t seed, bool det) {
  Dither d;
  if (det) {
#pragma unroll
    for (int k = 0; k < 10; ++k) d.d[k] = 0.5f;
  } else {
    d = dither10(x, y, z, t, seed);
  }
  uint32_t w[5];
  encode_words(s, d, w);
  uint32_t* b = static_cast<uint32_t*>(buf);
#pragma unroll
  for (int k = 0; k < 5; ++k) b[k * N + n] = w[k];
}

// ----------------------------------------------------------------- collision
// The 17 nonzero Hermite moments mu_pqr = sum_i P_p(cx) P_q(cy) P_r(cz) f+_i of
// the post-collision populations, with P_0 = 1, P_1 = c, P_2 = c^2 - 1/3 and the
// rest populations w_i removed (mu_000 = rho - 1):
//   mu_a = rho u_a, mu_aa = rho S_aa, mu_ab = rho S_ab, mu_aab = rho T_aab,
//   mu_xyz = rho T_xyz   (Eq. three_order_f: f+ is the third-order Hermite
// expansion with exactly these moments, T_abg = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g).
struct Mom17 {
  float m000, m100, m010, m001;
  float m200, m020, m002, m110, m101, m011;
  float m210, m120, m201, m102, m021, m012, m111;
};

// Moment-space collision of App. A applied to the stored variables.  With
// S = n/rho + u u the collision reads
//   u+ = u + F/(2 rho)
//   rho (S+ - u+ u+) = (1 - 1/tau) dev(n + sym(F u)) - F F / (4 rho)
// where dev() removes the trace and sym(F u)_ab = (F_a u_b + F_b u_a)/2: the
// trace of the non-equilibrium stress is reset, its deviator relaxes by (1 - 1/tau).
template <bool FORCE>
__device__ __forceinline__ Mom17 collide_moments(const Stored& s, float omega, float fx, float fy,
                                                 float fz) {
  const float rho = 1.0f + s.drho;
  const float om1 = 1.0f - omega;
  float ux = s.ux, uy = s.uy, uz = s.uz;
  float mxx = s.nxx, myy = s.nyy, mzz = s.nzz, mxy = s.nxy, mxz = s.nxz, myz = s.nyz;
  float inv = 0.f;
  if (FORCE) {
    inv = __frcp_rn(rho);
    mxx += fx * ux;
    myy += fy * uy;
    mzz += fz * uz;
    mxy += 0.5f * (fx * uy + fy * ux);
    mxz += 0.5f * (fx * uz + fz * ux);
    myz += 0.5f * (fy * uz + fz * uy);
  }
  const float tr = (mxx + myy + mzz) * (1.0f / 3.0f);
  float exx = om1 * (mxx - tr), eyy = om1 * (myy - tr), ezz = om1 * (mzz - tr);
  float exy = om1 * mxy, exz = om1 * mxz, eyz = om1 * myz;
  if (FORCE) {
    const float q = 0.25f * inv;
    exx -= q * fx * fx;
    eyy -= q * fy * fy;
    ezz -= q * fz * fz;
    exy -= q * fx * fy;
    exz -= q * fx * fz;
    eyz -= q * fy * fz;
    const float h = 0.5f * inv;
    ux += h * fx;
    uy += h * fy;
    uz += h * fz;
  }
  // rho u+, rho S+ = rho u+ u+ + rho E
  const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
  Mom17 A;
  A.m000 = s.drho;
  A.m100 = rux;
  A.m010 = ruy;
  A.m001 = ruz;
  A.m200 = rux * ux + exx;
  A.m020 = ruy * uy + eyy;
  A.m002 = ruz * uz + ezz;
  A.m110 = rux * uy + exy;
  A.m101 = rux * uz + exz;
  A.m011 = ruy * uz + eyz;
  // rho T_aab = u_b rho S_aa + 2 u_a rho E_ab
  A.m210 = uy * A.m200 + 2.0f * ux * exy;  // xxy
  A.m120 = ux * A.m020 + 2.0f * uy * exy;  // xyy
  A.m201 = uz * A.m200 + 2.0f * ux * exz;  // xxz
  A.m102 = ux * A.m002 + 2.0f * uz * exz;  // xzz
  A.m021 = uz * A.m020 + 2.0f * uy * eyz;  // yyz
  A.m012 = uy * A.m002 + 2.0f * uz * eyz;  // yzz
  // rho T_xyz = rho ux uy uz + rho (E_xy uz + E_xz uy + E_yz ux)
  A.m111 = rux * uy * uz + exy * uz + exz * uy + eyz * ux;
  return A;
}

// ----------------------------------------------------------------- 1D lattice pass
// One axis of the separable stream: D3Q27 is the tensor product of three D1Q3
// lattices (c in {-1, 0, 1}, weights 1/6, 2/3, 1/6).  Along one axis the local
// moments (mu0, mu1, mu2) on (P_0, P_1, P_2) define the three directional
// populations  phi_c = w(c) (mu0 + 3 c mu1 + 9/2 P_2(c) mu2):
//   phi_s = mu0/6 + mu2/2,  phi_0 = mu0 - 2 phi_s,  phi_(+-1) = phi_s +- mu1/2.
// Streaming pulls phi_+ from x-1 and phi_- from x+1; the new moments are
//   m0 = phi_+ + phi_0 + phi_-,  m1 = phi_+ - phi_-,  m2 = phi_+ + phi_- - m0/3.
// Written this way the sums of m0 and m1 over the grid equal those of mu0 and
// mu1 whatever the FP32 rounding of 1/6: mass and momentum are conserved up to
// unbiased rounding instead of drifting with the rounded lattice weights.
struct Phi {
  float p, z, m;  // phi_{+1}, phi_0, phi_{-1}
};
__device__ __forceinline__ Phi phi3(float mu0, float mu1, float mu2) {
  Phi r;
  const float s = __fmaf_rn(mu0, 1.0f / 6.0f, 0.5f * mu2);
  r.z = __fmaf_rn(-2.0f, s, mu0);
  r.p = __fmaf_rn(0.5f, mu1, s);
  r.m = __fmaf_rn(-0.5f, mu1, s);
  return r;
}
// Projection after streaming: pl = phi_+ pulled from the minus side, z = own
// phi_0, mr = phi_- pulled from the plus side.
__device__ __forceinline__ float proj0(float pl, float z, float mr) { return pl + z + mr; }
__device__ __forceinline__ float proj1(float pl, float mr) { return pl - mr; }
__device__ __forceinline__ float proj2(float pl, float mr, float o0) {
  return __fmaf_rn(-1.0f / 3.0f, o0, pl + mr);
}

// Stored variables from the ten streamed moments (rest removed):
//   rho' = 1 + m000, rho' u' = m_a + F_a/2, rho' S'_ab = m_ab, n'_ab = m_ab - (rho' u'_a) u'_b.
template <bool FORCE>
__device__ __forceinline__ Stored finish_moments(float m000, float m100, float m010, float m001,
                                                 float m200, float m020, float m002, float m110,
                                                 float m101, float m011, float fx, float fy,
                                                 float fz) {
  Stored o;
  o.drho = m000;
  const float rho = 1.0f + m000;
  const float inv = __frcp_rn(rho);
  float jx = m100, jy = m010, jz = m001;
  if (FORCE) {
    jx += 0.5f * fx;
    jy += 0.5f * fy;
    jz += 0.5f * fz;
  }
  o.ux = jx * inv;
  o.uy = jy * inv;
  o.uz = jz * inv;
  o.nxx = m200 - jx * o.ux;
  o.nyy = m020 - jy * o.uy;
  o.nzz = m002 - jz * o.uz;
  o.nxy = m110 - jx * o.uy;
  o.nxz = m101 - jx * o.uz;
  o.nyz = m011 - jy * o.uz;
  return o;
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

}  // namespace melbm
