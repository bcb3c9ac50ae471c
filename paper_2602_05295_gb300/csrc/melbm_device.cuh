// melbm_device.cuh -- device helpers shared by the CUDA kernels of the library:
// stored-variable layout, the 16-bit codec of Sec. 5.4 with its dither, the
// moment-space collision of App. A written in stored variables, and the
// tensor-product (D1Q3 x D1Q3 x D1Q3) form of the streaming of the third-order
// Hermite populations.  The per-cell arithmetic is written once for T = float
// and T = float2; the float2 form runs on the packed FP32x2 instructions
// (FFMA2/FADD2/FMUL2) of sm_100-class GPUs and processes two cells at once.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "melbm_launch.h"

namespace melbm {

constexpr unsigned FULL = 0xffffffffu;

enum : uint8_t { T_FLUID = 0, T_FLUID_BOUNDARY = 1, T_INFLOW = 2, T_OUTFLOW = 3, T_SOLID = 4 };
enum { ST_F32 = 0, ST_Q16 = 1, ST_MIXED = 2 };  // MIXED: 16-bit post-collision + FP32 post-streaming

// ----------------------------------------------------------------- scalar / pair math
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }
template <class T> __device__ __forceinline__ T vset(float a);
template <> __device__ __forceinline__ float vset<float>(float a) { return a; }

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);  // exact negation, one rounding
}
// Reciprocal of a pair: the hardware approximation (PTX rcp.approx) refined by one
// Newton-Raphson step r' = r + r (1 - a r) on packed FP32x2; for the densities
// here (a ~ 1) the refined value is the correctly rounded one up to rare last-bit
// differences, so it carries no systematic bias into u = J / rho.
__device__ __forceinline__ float2 vrcp(float2 a) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(a.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(a.y));
  const float2 e = __ffma2_rn(make_float2(-a.x, -a.y), r, make_float2(1.0f, 1.0f));
  return __ffma2_rn(r, e, r);
}
template <> __device__ __forceinline__ float2 vset<float2>(float a) { return make_float2(a, a); }
// a * b + c with scalar constant b
__device__ __forceinline__ float vfmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfmac(float2 a, float b, float2 c) {
  return __ffma2_rn(a, make_float2(b, b), c);
}
__device__ __forceinline__ float vmulc(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmulc(float2 a, float b) { return __fmul2_rn(a, make_float2(b, b)); }

// ---------------------------------------------------------------------------
// Stored variables of one cell.  Both storages keep the same ten quantities:
//   drho = rho - 1, u_a, and n_ab = rho S^neq_ab = rho (S_ab - u_a u_b)
// ordered (xx, yy, zz, xy, xz, yz).  Keeping rho - 1 instead of rho removes the
// O(1) rest state from every FP32 sum (its populations w_i stream to themselves).
// FP32 storage: ten planes [10][N] with plane 0 = drho.
// Q16 storage:  five u32 planes [5][N]; word k holds components (2k, 2k+1) in its
//               (low, high) halves.
// ---------------------------------------------------------------------------
template <class T>
struct StoredT {
  T drho;
  T ux, uy, uz;
  T nxx, nyy, nzz, nxy, nxz, nyz;
};
using Stored = StoredT<float>;

// ----------------------------------------------------------------- 16-bit codec
// Sec. 5.4: ranges rho [0.8, 1.5], u [-0.4, 0.4], rho S^neq [-0.1, 0.1];
// q = floor((m - m_min)/step + d), step = (m_max - m_min)/(2^16 - 1), d in [0, 1)
// the dither.  The map is evaluated relative to the code qc nearest to the centre
// of the values (rho = 1 in the variable rho - 1; u = 0; rho S^neq = 0), so that
// the FP32 rounding of the constants only scales the zero-mean deviation from
// the centre, and the floor of w + d is taken exactly with round-down adds:
//   w = m' K + b,  q = qc + floor(clamp(w, -qc, 65535 - qc) + d),
//   m' = c + (q - qc) step,  c = value of code qc.
// Group 0 = rho (m' = rho - 1), 1 = velocity, 2 = rho S^neq.  Constants are the
// FP32 roundings of the FP64 expressions.
template <int G> struct QRange;
template <> struct QRange<0> {
  static constexpr double lo = 0.8 - 1.0, hi = 1.5 - 1.0;
  static constexpr float qc = 18724.0f;
};
template <> struct QRange<1> {
  static constexpr double lo = -0.4, hi = 0.4;
  static constexpr float qc = 32768.0f;
};
template <> struct QRange<2> {
  static constexpr double lo = -0.1, hi = 0.1;
  static constexpr float qc = 32768.0f;
};
template <int G> struct QConst {
  static constexpr double lo = QRange<G>::lo, hi = QRange<G>::hi;
  static constexpr double qcd = double(QRange<G>::qc);
  static constexpr float step = float((hi - lo) / 65535.0);
  static constexpr float K = float(65535.0 / (hi - lo));
  static constexpr float b = float((0.0 - lo) * 65535.0 / (hi - lo) - qcd);
  static constexpr float c = float(lo + qcd * (hi - lo) / 65535.0);
  static constexpr float wlo = float(-qcd), whi = float(65535.0 - qcd);
  static constexpr float magic = float(8388608.0 + qcd);  // 2^23 + qc
  static constexpr float qc = QRange<G>::qc;
};

// Encoded bits of one value: the float 2^23 + q, whose low 16 bits are q.
template <int G>
__device__ __forceinline__ uint32_t q_encode_bits(float m, float d) {
  float w = __fmaf_rn(m, QConst<G>::K, QConst<G>::b);
  w = fminf(fmaxf(w, QConst<G>::wlo), QConst<G>::whi);  // NaN -> wlo (code 0)
  const float z = __fadd_rd(__fadd_rd(w, d), QConst<G>::magic);
  return __float_as_uint(z);
}
// Pair form: q = qc + floor(w + d) as floor(fl_rd(fl_rd(w + d) + qc)) -- both
// round-down adds keep the floor exact -- converted by cvt.rmi.u16, which
// saturates to [0, 65535] (and maps NaN to 0), the same codes as clamping w first.
// Returns the two codes (zero-extended).
template <int G>
__device__ __forceinline__ uint2 q_encode_codes(float2 m, float2 d) {
  const float2 w = __ffma2_rn(m, make_float2(QConst<G>::K, QConst<G>::K),
                              make_float2(QConst<G>::b, QConst<G>::b));
  const float2 z = __fadd2_rd(__fadd2_rd(w, d), make_float2(QConst<G>::qc, QConst<G>::qc));
  unsigned short qa, qb;
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qa) : "f"(z.x));
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qb) : "f"(z.y));
  return make_uint2(qa, qb);
}
// The pair form with the dither given as 1 + d (dither_one_plus): the same codes,
// q = qc + floor(w + d) = (qc - 1) + floor(w + (1 + d)), one packed FMA fewer.
// SC: the value comes multiplied by SC (1, -1 or -4), which the grid factor K
// divides out exactly (K / SC is K times a power of two).
template <int G, int SC = 1>
__device__ __forceinline__ uint2 q_encode_codes1(float2 m, float2 D) {
  constexpr float K = QConst<G>::K / float(SC);
  const float2 w = __ffma2_rn(m, make_float2(K, K), make_float2(QConst<G>::b, QConst<G>::b));
  const float qm = QConst<G>::qc - 1.0f;
  const float2 z = __fadd2_rd(__fadd2_rd(w, D), make_float2(qm, qm));
  unsigned short qa, qb;
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qa) : "f"(z.x));
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qb) : "f"(z.y));
  return make_uint2(qa, qb);
}
__device__ __forceinline__ uint32_t q_pack(uint32_t lo_bits, uint32_t hi_bits) {
  return __byte_perm(lo_bits, hi_bits, 0x5410);
}
// The float 2^23 + q of the low / high code of a word.
__device__ __forceinline__ float q_lo_magic(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7610));
}
__device__ __forceinline__ float q_hi_magic(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7632));
}
// m' = c + (q - qc) step from the float 2^23 + q.
template <int G>
__device__ __forceinline__ float q_decode(float magic_q) {
  return __fmaf_rn(magic_q - QConst<G>::magic, QConst<G>::step, QConst<G>::c);
}
template <int G>
__device__ __forceinline__ float2 q_decode(float2 magic_q) {
  const float2 f = __fadd2_rn(magic_q, make_float2(-QConst<G>::magic, -QConst<G>::magic));
  return __ffma2_rn(f, make_float2(QConst<G>::step, QConst<G>::step),
                    make_float2(QConst<G>::c, QConst<G>::c));
}

// The same maps with runtime grid constants (b-bit codes): the clamp to
// [-qc, 2^b - 1 - qc] is explicit, since cvt's saturation is at 65535.
__device__ __forceinline__ uint32_t qg_encode_bits(const QGrid& g, float m, float d) {
  float w = __fmaf_rn(m, g.K, g.b);
  w = fminf(fmaxf(w, g.wlo), g.whi);  // NaN -> wlo (code 0)
  return __float_as_uint(__fadd_rd(__fadd_rd(w, d), g.magic));
}
// Pair form without the upper clamp: cvt.rmi.u16 saturates below at 0 (NaN -> 0),
// which is the lower clamp; the codes above 2^b - 1 are cut by qg_clamp_word on
// the packed word.  Both give the codes of the clamped form for every input: w
// below -qc or above 2^b - 1 - qc floors to a code at or beyond the same end.
__device__ __forceinline__ uint2 qg_encode_codes(const QGrid& g, float2 m, float2 d) {
  const float2 w = __ffma2_rn(m, make_float2(g.K, g.K), make_float2(g.b, g.b));
  const float2 z = __fadd2_rd(__fadd2_rd(w, d), make_float2(g.qc, g.qc));
  unsigned short qa, qb;
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qa) : "f"(z.x));
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qb) : "f"(z.y));
  return make_uint2(qa, qb);
}
// With the dither given as 1 + d (see q_encode_codes1).
__device__ __forceinline__ uint2 qg_encode_codes1(const QGrid& g, float2 m, float2 D,
                                                 float kscale = 1.0f) {
  const float K = g.K * kscale;  // kscale: 1, -1 or -1/4 (exact)
  const float2 w = __ffma2_rn(m, make_float2(K, K), make_float2(g.b, g.b));
  const float qm = g.qc - 1.0f;
  const float2 z = __fadd2_rd(__fadd2_rd(w, D), make_float2(qm, qm));
  unsigned short qa, qb;
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qa) : "f"(z.x));
  asm("cvt.rmi.u16.f32 %0, %1;" : "=h"(qb) : "f"(z.y));
  return make_uint2(qa, qb);
}
// Both codes of a word share one group's 2^b - 1 (rho and u use b_rho_u).
__device__ __forceinline__ uint32_t qg_clamp_word(uint32_t w, uint32_t qmax) {
  return __vminu2(w, qmax * 0x10001u);
}
__device__ __forceinline__ float qg_decode(const QGrid& g, float magic_q) {
  return __fmaf_rn(magic_q - g.magic, g.step, g.c);
}
__device__ __forceinline__ float2 qg_decode(const QGrid& g, float2 magic_q) {
  const float2 f = __fadd2_rn(magic_q, make_float2(-g.magic, -g.magic));
  return __ffma2_rn(f, make_float2(g.step, g.step), make_float2(g.c, g.c));
}

// Counter-based dither: pcg4d of Jarzynski & Olano, "Hash Functions for GPU
// Rendering", JCGT 9(3) 2020, on (x, y, z, t ^ seed): 128 bits per cell and time
// index, from which the ten components take 16-bit fields (below).
struct DitherBits {
  uint32_t w[4];
};
__device__ __forceinline__ DitherBits pcg4d(uint32_t x, uint32_t y, uint32_t z, uint32_t t,
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
  DitherBits r;
  r.w[0] = v0;
  r.w[1] = v1;
  r.w[2] = v2;
  r.w[3] = v3;
  return r;
}
// The dither of component k: a 16-bit field f -- components 0..7 the low (even k)
// and high (odd k) half of word k/2, component 8 the low half of w0 ^ w2,
// component 9 the high half of w1 ^ w3 -- mapped to the midpoint
// d = (f + 1/2) / 2^16, whose mean over f is exactly 1/2.  One byte permute places
// f in the float 2^23 + f; from it d and 1 + d follow by one FMA each, exactly
// (their values have at most 18 significant bits).
__device__ __forceinline__ uint32_t dither_word(const DitherBits& h, int k) {
  return k < 8 ? h.w[k >> 1] : (k == 8 ? (h.w[0] ^ h.w[2]) : (h.w[1] ^ h.w[3]));
}
__device__ __forceinline__ float dither_magic(const DitherBits& h, int k) {  // 2^23 + f
  return __uint_as_float(__byte_perm(dither_word(h, k), 0x4B000000u, (k & 1) ? 0x7632 : 0x7610));
}
constexpr float DITHER_SCALE = 1.0f / 65536.0f;
constexpr float DITHER_OFF = -(128.0f - 1.0f / 131072.0f);      // d = magic 2^-16 + DITHER_OFF
constexpr float DITHER_OFF1 = -(127.0f - 1.0f / 131072.0f);     // 1 + d
__device__ __forceinline__ float dither_value(float magic) {
  return __fmaf_rn(magic, DITHER_SCALE, DITHER_OFF);
}
// 1 + d, for the encode below, which adds it in place of d: the code is unchanged,
// since floor(w + 1 + d) - 1 = floor(w + d) and both round-down adds keep the floor.
__device__ __forceinline__ float dither_one_plus(const DitherBits& h, int k) {
  return __fmaf_rn(dither_magic(h, k), DITHER_SCALE, DITHER_OFF1);
}
// The same for the two cells of a pair (packed).
__device__ __forceinline__ float2 dither_one_plus2(const DitherBits& a, const DitherBits& b, int k) {
  return __ffma2_rn(make_float2(dither_magic(a, k), dither_magic(b, k)),
                    make_float2(DITHER_SCALE, DITHER_SCALE), make_float2(DITHER_OFF1, DITHER_OFF1));
}
struct Dither {
  float d[10];
};
__device__ __forceinline__ Dither dither10(uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                           uint32_t seed) {
  const DitherBits h = pcg4d(x, y, z, t, seed);
  Dither r;
#pragma unroll
  for (int k = 0; k < 10; ++k) r.d[k] = dither_value(dither_magic(h, k));
  return r;
}

// ----------------------------------------------------------------- scalar load / store
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

__device__ __forceinline__ Stored decode_words(const uint32_t w[5]) {
  Stored s;
  s.drho = q_decode<0>(q_lo_magic(w[0]));
  s.ux = q_decode<1>(q_hi_magic(w[0]));
  s.uy = q_decode<1>(q_lo_magic(w[1]));
  s.uz = q_decode<1>(q_hi_magic(w[1]));
  s.nxx = q_decode<2>(q_lo_magic(w[2]));
  s.nyy = q_decode<2>(q_hi_magic(w[2]));
  s.nzz = q_decode<2>(q_lo_magic(w[3]));
  s.nxy = q_decode<2>(q_hi_magic(w[3]));
  s.nxz = q_decode<2>(q_lo_magic(w[4]));
  s.nyz = q_decode<2>(q_hi_magic(w[4]));
  return s;
}

template <>
__device__ __forceinline__ Stored load_stored<ST_Q16>(const void* buf, size_t N, size_t n) {
  const uint32_t* b = static_cast<const uint32_t*>(buf);
  uint32_t w[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) w[k] = __ldg(b + k * N + n);
  return decode_words(w);
}

__device__ __forceinline__ Stored decode_words(const uint32_t w[5], const QGrids& q) {
  Stored s;
  s.drho = qg_decode(q.g[0], q_lo_magic(w[0]));
  s.ux = qg_decode(q.g[1], q_hi_magic(w[0]));
  s.uy = qg_decode(q.g[1], q_lo_magic(w[1]));
  s.uz = qg_decode(q.g[1], q_hi_magic(w[1]));
  s.nxx = qg_decode(q.g[2], q_lo_magic(w[2]));
  s.nyy = qg_decode(q.g[2], q_hi_magic(w[2]));
  s.nzz = qg_decode(q.g[2], q_lo_magic(w[3]));
  s.nxy = qg_decode(q.g[2], q_hi_magic(w[3]));
  s.nxz = qg_decode(q.g[2], q_lo_magic(w[4]));
  s.nyz = qg_decode(q.g[2], q_hi_magic(w[4]));
  return s;
}

// Load with the handle's grids (b-bit codes); FP32 storage ignores them.
template <int STORAGE>
__device__ __forceinline__ Stored load_stored(const void* buf, size_t N, size_t n, const QGrids& q) {
  if constexpr (STORAGE == ST_F32) {
    return load_stored<ST_F32>(buf, N, n);
  } else {
    const uint32_t* b = static_cast<const uint32_t*>(buf);
    uint32_t w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = __ldg(b + k * N + n);
    return decode_words(w, q);
  }
}

__device__ __forceinline__ void encode_words(const Stored& s, const Dither& d, uint32_t w[5],
                                             const QGrids& q) {
  w[0] = q_pack(qg_encode_bits(q.g[0], s.drho, d.d[0]), qg_encode_bits(q.g[1], s.ux, d.d[1]));
  w[1] = q_pack(qg_encode_bits(q.g[1], s.uy, d.d[2]), qg_encode_bits(q.g[1], s.uz, d.d[3]));
  w[2] = q_pack(qg_encode_bits(q.g[2], s.nxx, d.d[4]), qg_encode_bits(q.g[2], s.nyy, d.d[5]));
  w[3] = q_pack(qg_encode_bits(q.g[2], s.nzz, d.d[6]), qg_encode_bits(q.g[2], s.nxy, d.d[7]));
  w[4] = q_pack(qg_encode_bits(q.g[2], s.nxz, d.d[8]), qg_encode_bits(q.g[2], s.nyz, d.d[9]));
}

__device__ __forceinline__ void encode_words(const Stored& s, const Dither& d, uint32_t w[5]) {
  w[0] = q_pack(q_encode_bits<0>(s.drho, d.d[0]), q_encode_bits<1>(s.ux, d.d[1]));
  w[1] = q_pack(q_encode_bits<1>(s.uy, d.d[2]), q_encode_bits<1>(s.uz, d.d[3]));
  w[2] = q_pack(q_encode_bits<2>(s.nxx, d.d[4]), q_encode_bits<2>(s.nyy, d.d[5]));
  w[3] = q_pack(q_encode_bits<2>(s.nzz, d.d[6]), q_encode_bits<2>(s.nxy, d.d[7]));
  w[4] = q_pack(q_encode_bits<2>(s.nxz, d.d[8]), q_encode_bits<2>(s.nyz, d.d[9]));
}

// Store with the dither of (x, y, z, t ^ seed) (Q16) or as FP32; deterministic
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

// Store with the handle's grids (b-bit codes); FP32 storage ignores them.
template <int STORAGE>
__device__ __forceinline__ void store_stored(void* buf, size_t N, size_t n, const Stored& s,
                                             uint32_t x, uint32_t y, uint32_t z, uint32_t t,
                                             uint32_t seed, bool det, const QGrids& q) {
  if constexpr (STORAGE == ST_F32) {
    store_stored<ST_F32>(buf, N, n, s, x, y, z, t, seed, det);
  } else {
    Dither d;
    if (det) {
#pragma unroll
      for (int k = 0; k < 10; ++k) d.d[k] = 0.5f;
    } else {
      d = dither10(x, y, z, t, seed);
    }
    uint32_t w[5];
    encode_words(s, d, w, q);
    uint32_t* b = static_cast<uint32_t*>(buf);
#pragma unroll
    for (int k = 0; k < 5; ++k) b[k * N + n] = w[k];
  }
}

// ----------------------------------------------------------------- collision
// The 17 nonzero Hermite moments mu_pqr = sum_i P_p(cx) P_q(cy) P_r(cz) f+_i of
// the post-collision populations, with P_0 = 1, P_1 = c, P_2 = c^2 - 1/3 and the
// rest populations w_i removed (mu_000 = rho - 1):
//   mu_a = rho u_a, mu_aa = rho S_aa, mu_ab = rho S_ab, mu_aab = rho T_aab,
//   mu_xyz = rho T_xyz (half of it when built with MELBM_HERMITE_XYZ_LITERAL,
//   the printed 1/(2 c_s^6) on the xyz term, kept as an ablation of that reading)
//   (Eq. three_order_f: f+ is the third-order Hermite
// expansion with exactly these moments, T_abg = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g).
template <class T>
struct Mom17T {
  T m000, m100, m010, m001;
  T m200, m020, m002, m110, m101, m011;
  T m210, m120, m201, m102, m021, m012, m111;
};
using Mom17 = Mom17T<float>;

// Moment-space collision of App. A applied to the stored variables.  With
// S = n/rho + u u the collision reads
//   u+ = u + F/(2 rho)
//   rho (S+ - u+ u+) = (1 - 1/tau) dev(n + sym(F u)) - F F / (4 rho)
// where dev() removes the trace and sym(F u)_ab = (F_a u_b + F_b u_a)/2: the
// trace of the non-equilibrium stress is reset, its deviator relaxes by (1 - 1/tau).
template <bool FORCE, class T>
__device__ __forceinline__ Mom17T<T> collide_moments(const StoredT<T>& s, float omega, T fx, T fy,
                                                     T fz) {
  const T rho = vadd(s.drho, vset<T>(1.0f));
  const float om1 = 1.0f - omega;
  T ux = s.ux, uy = s.uy, uz = s.uz;
  T mxx = s.nxx, myy = s.nyy, mzz = s.nzz, mxy = s.nxy, mxz = s.nxz, myz = s.nyz;
  T inv = vset<T>(0.f);
  if (FORCE) {
    inv = vrcp(rho);
    mxx = vfma(fx, ux, mxx);
    myy = vfma(fy, uy, myy);
    mzz = vfma(fz, uz, mzz);
    mxy = vfmac(vfma(fx, uy, vmul(fy, ux)), 0.5f, mxy);
    mxz = vfmac(vfma(fx, uz, vmul(fz, ux)), 0.5f, mxz);
    myz = vfmac(vfma(fy, uz, vmul(fz, uy)), 0.5f, myz);
  }
  const T tr = vmulc(vadd(vadd(mxx, myy), mzz), 1.0f / 3.0f);
  T exx = vmulc(vsub(mxx, tr), om1), eyy = vmulc(vsub(myy, tr), om1), ezz = vmulc(vsub(mzz, tr), om1);
  T exy = vmulc(mxy, om1), exz = vmulc(mxz, om1), eyz = vmulc(myz, om1);
  if (FORCE) {
    const T q = vmulc(inv, -0.25f);
    exx = vfma(vmul(q, fx), fx, exx);
    eyy = vfma(vmul(q, fy), fy, eyy);
    ezz = vfma(vmul(q, fz), fz, ezz);
    exy = vfma(vmul(q, fx), fy, exy);
    exz = vfma(vmul(q, fx), fz, exz);
    eyz = vfma(vmul(q, fy), fz, eyz);
    const T h = vmulc(inv, 0.5f);
    ux = vfma(h, fx, ux);
    uy = vfma(h, fy, uy);
    uz = vfma(h, fz, uz);
  }
  // rho u+, rho S+ = rho u+ u+ + rho E
  const T rux = vmul(rho, ux), ruy = vmul(rho, uy), ruz = vmul(rho, uz);
  Mom17T<T> A;
  A.m000 = s.drho;
  A.m100 = rux;
  A.m010 = ruy;
  A.m001 = ruz;
  A.m200 = vfma(rux, ux, exx);
  A.m020 = vfma(ruy, uy, eyy);
  A.m002 = vfma(ruz, uz, ezz);
  A.m110 = vfma(rux, uy, exy);
  A.m101 = vfma(rux, uz, exz);
  A.m011 = vfma(ruy, uz, eyz);
  // rho T_aab = u_b rho S_aa + 2 u_a rho E_ab
  const T ux2 = vadd(ux, ux), uy2 = vadd(uy, uy), uz2 = vadd(uz, uz);
  A.m210 = vfma(uy, A.m200, vmul(ux2, exy));  // xxy
  A.m120 = vfma(ux, A.m020, vmul(uy2, exy));  // xyy
  A.m201 = vfma(uz, A.m200, vmul(ux2, exz));  // xxz
  A.m102 = vfma(ux, A.m002, vmul(uz2, exz));  // xzz
  A.m021 = vfma(uz, A.m020, vmul(uy2, eyz));  // yyz
  A.m012 = vfma(uy, A.m002, vmul(uz2, eyz));  // yzz
  // rho T_xyz = rho ux uy uz + rho (E_xy uz + E_xz uy + E_yz ux)
  A.m111 = vfma(vmul(rux, uy), uz, vfma(exy, uz, vfma(exz, uy, vmul(eyz, ux))));
#ifdef MELBM_HERMITE_XYZ_LITERAL
  A.m111 = vmulc(A.m111, 0.5f);  // the printed 1/(2 c_s^6) on xyz halves its moment
#endif
  return A;
}

// D3Q19 (the 19-velocity set of Table 1's D3Q19 scene, |c|^2 <= 2): the
// post-collision populations are the third-order Hermite expansion projected on
// what that lattice carries (the xyz term vanishes there, and each pair
// H_aab, H_bgg enters through its orthogonal sum and difference), which
// reproduces rho, rho u, rho S and the six rho T_aab.  Extended by zero to the
// eight corners they are a function on the D3Q27 cube, whose tensor moments
// mu_pqr (rest state removed: mu_000 = rho - 1, mu_222 + 1/27) are those of
// Mom17T with mu_111 = 0 plus the ten below; each follows from the populations'
// vanishing at the corners, so c_a^2 c_b c_g and c_x^2 c_y^2 c_z^2 have zero sum,
// and from the even part of the edge populations for sum c_a^2 c_b^2 f:
//   mu_aabb = -mu_gg / 6,  mu_aabg = -mu_bg / 3,
//   mu_aabbg = -(mu_aag + mu_bbg) / 3 - mu_g / 9,
//   mu_xxyyzz = -mu_000 / 27 - (mu_xx + mu_yy + mu_zz) / 18.
template <class T>
struct Closure19T {
  T m220, m202, m022, m211, m121, m112, m221, m212, m122, m222;
};
template <class T>
__device__ __forceinline__ Closure19T<T> closure19(const Mom17T<T>& A) {
  Closure19T<T> E;
  E.m220 = vmulc(A.m002, -1.0f / 6.0f);
  E.m202 = vmulc(A.m020, -1.0f / 6.0f);
  E.m022 = vmulc(A.m200, -1.0f / 6.0f);
  E.m211 = vmulc(A.m011, -1.0f / 3.0f);
  E.m121 = vmulc(A.m101, -1.0f / 3.0f);
  E.m112 = vmulc(A.m110, -1.0f / 3.0f);
  E.m221 = vfmac(A.m001, -1.0f / 9.0f, vmulc(vadd(A.m201, A.m021), -1.0f / 3.0f));
  E.m212 = vfmac(A.m010, -1.0f / 9.0f, vmulc(vadd(A.m210, A.m012), -1.0f / 3.0f));
  E.m122 = vfmac(A.m100, -1.0f / 9.0f, vmulc(vadd(A.m120, A.m102), -1.0f / 3.0f));
  E.m222 = vfmac(A.m000, -1.0f / 27.0f,
                 vmulc(vadd(vadd(A.m200, A.m020), A.m002), -1.0f / 18.0f));
  return E;
}

// f+_i / w_i - 1 from the Hermite moments: the coefficient of P_p P_q P_r is
// mu_pqr divided by the D1Q3 norms (1, 1/3, 2/9) of each factor (P_2(c) = c^2 - 1/3).
__device__ __forceinline__ float hermite_eval(const Mom17& A, int cx, int cy, int cz) {
  const float fx = float(cx), fy = float(cy), fz = float(cz);
  const float qx = fx * fx - (1.0f / 3.0f), qy = fy * fy - (1.0f / 3.0f),
              qz = fz * fz - (1.0f / 3.0f);
  return A.m000 + 3.0f * (A.m100 * fx + A.m010 * fy + A.m001 * fz) +
         4.5f * (A.m200 * qx + A.m020 * qy + A.m002 * qz) +
         9.0f * (A.m110 * fx * fy + A.m101 * fx * fz + A.m011 * fy * fz) +
         13.5f * (A.m210 * qx * fy + A.m120 * fx * qy + A.m201 * qx * fz + A.m102 * fx * qz +
                  A.m021 * qy * fz + A.m012 * fy * qz) +
         27.0f * A.m111 * fx * fy * fz;
}

// f+_i / w19_i - 1 on the D3Q19 lattice (|c|^2 <= 2, weights 1/3, 1/18, 1/36):
// the same zeroth to second order terms, and the third order projected on what
// the lattice carries -- for each pair of triples (a a b, b g g) with moments
// (A, B) and Hermite polynomials (h1, h2) = (P2(c_a) c_b, c_b P2(c_g)),
//   (A + B)(h1 + h2)/(2 c_s^6) + (A - B)(h1 - h2)/(6 c_s^6) = A (18 h1 + 9 h2) + B (9 h1 + 18 h2),
// and no xyz term.
__device__ __forceinline__ float hermite_eval19(const Mom17& A, int cx, int cy, int cz) {
  const float fx = float(cx), fy = float(cy), fz = float(cz);
  const float qx = fx * fx - (1.0f / 3.0f), qy = fy * fy - (1.0f / 3.0f),
              qz = fz * fz - (1.0f / 3.0f);
  const float hy1 = qx * fy, hy2 = fy * qz;  // xxy, yzz
  const float hx1 = fx * qy, hx2 = fx * qz;  // xyy, xzz
  const float hz1 = qx * fz, hz2 = qy * fz;  // xxz, yyz
  return A.m000 + 3.0f * (A.m100 * fx + A.m010 * fy + A.m001 * fz) +
         4.5f * (A.m200 * qx + A.m020 * qy + A.m002 * qz) +
         9.0f * (A.m110 * fx * fy + A.m101 * fx * fz + A.m011 * fy * fz) +
         A.m210 * (18.0f * hy1 + 9.0f * hy2) + A.m012 * (9.0f * hy1 + 18.0f * hy2) +
         A.m120 * (18.0f * hx1 + 9.0f * hx2) + A.m102 * (9.0f * hx1 + 18.0f * hx2) +
         A.m201 * (18.0f * hz1 + 9.0f * hz2) + A.m021 * (9.0f * hz1 + 18.0f * hz2);
}
__device__ __forceinline__ constexpr bool in_d3q19(int cx, int cy, int cz) {
  return cx * cx + cy * cy + cz * cz <= 2;
}
__device__ __forceinline__ float lattice_weight19(int cx, int cy, int cz) {
  const int n2 = cx * cx + cy * cy + cz * cz;
  return n2 == 0 ? (1.0f / 3.0f) : (n2 == 1 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}

// Hermite moments of the wall state of the moment-based reconstruction (Sec.
// 3.2): rho^p = rho of the cell, u^p the wall velocity, and the non-equilibrium
// stress rho (S - u u) of the cell's post-collision moments A kept, i.e.
// S^p = u^p u^p + (S - u u); third moments from the same closure as the collision.
__device__ __forceinline__ Mom17 wall_moments(const Mom17& A, float upx, float upy, float upz) {
  const float rho = 1.0f + A.m000;
  const float inv = __frcp_rn(rho);
  const float exx = A.m200 - A.m100 * A.m100 * inv, eyy = A.m020 - A.m010 * A.m010 * inv,
              ezz = A.m002 - A.m001 * A.m001 * inv;
  const float exy = A.m110 - A.m100 * A.m010 * inv, exz = A.m101 - A.m100 * A.m001 * inv,
              eyz = A.m011 - A.m010 * A.m001 * inv;
  const float rux = rho * upx, ruy = rho * upy, ruz = rho * upz;
  Mom17 W;
  W.m000 = A.m000;
  W.m100 = rux;
  W.m010 = ruy;
  W.m001 = ruz;
  W.m200 = __fmaf_rn(rux, upx, exx);
  W.m020 = __fmaf_rn(ruy, upy, eyy);
  W.m002 = __fmaf_rn(ruz, upz, ezz);
  W.m110 = __fmaf_rn(rux, upy, exy);
  W.m101 = __fmaf_rn(rux, upz, exz);
  W.m011 = __fmaf_rn(ruy, upz, eyz);
  W.m210 = __fmaf_rn(upy, W.m200, 2.0f * upx * exy);
  W.m120 = __fmaf_rn(upx, W.m020, 2.0f * upy * exy);
  W.m201 = __fmaf_rn(upz, W.m200, 2.0f * upx * exz);
  W.m102 = __fmaf_rn(upx, W.m002, 2.0f * upz * exz);
  W.m021 = __fmaf_rn(upz, W.m020, 2.0f * upy * eyz);
  W.m012 = __fmaf_rn(upy, W.m002, 2.0f * upz * eyz);
  W.m111 = __fmaf_rn(rux * upy, upz, exy * upz + exz * upy + eyz * upx);
#ifdef MELBM_HERMITE_XYZ_LITERAL
  W.m111 *= 0.5f;
#endif
  return W;
}

// Velocity of body b at point p: V + Om x (p - r0), table[9 b ..] = (V, Om, r0).
__device__ __forceinline__ void body_velocity(const float* table, int b, float px, float py,
                                              float pz, float* up) {
  const float* t = table + 9 * b;
  const float rx = px - t[6], ry = py - t[7], rz = pz - t[8];
  up[0] = t[0] + t[4] * rz - t[5] * ry;
  up[1] = t[1] + t[5] * rx - t[3] * rz;
  up[2] = t[2] + t[3] * ry - t[4] * rx;
}

// Linear index of the neighbour x - c_i (periodic, one-step wrap).
__device__ __forceinline__ uint32_t pull_source(int x, int y, int z, int nx, int ny, int nz, int i) {
  const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
  int sx = x - cx, sy = y - cy, sz = z - cz;
  sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
  sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
  sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
  return uint32_t(sx) + uint32_t(nx) * (uint32_t(sy) + uint32_t(ny) * uint32_t(sz));
}

__device__ __forceinline__ void cell_xyz(uint32_t n, int nx, int ny, int* x, int* y, int* z) {
  *x = int(n % uint32_t(nx));
  *y = int((n / uint32_t(nx)) % uint32_t(ny));
  *z = int(n / (uint32_t(nx) * uint32_t(ny)));
}

// Lattice weight of direction i = (cx+1) + 3 (cy+1) + 9 (cz+1).
__device__ __forceinline__ float lattice_weight(int cx, int cy, int cz) {
  return (cx ? (1.0f / 6.0f) : (2.0f / 3.0f)) * (cy ? (1.0f / 6.0f) : (2.0f / 3.0f)) *
         (cz ? (1.0f / 6.0f) : (2.0f / 3.0f));
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
template <class T>
struct PhiT {
  T p, z, m;  // phi_{+1}, phi_0, phi_{-1}
};
using Phi = PhiT<float>;
template <class T>
__device__ __forceinline__ PhiT<T> phi3(T mu0, T mu1, T mu2) {
  PhiT<T> r;
  const T s = vfmac(mu0, 1.0f / 6.0f, vmulc(mu2, 0.5f));
  r.z = vfmac(s, -2.0f, mu0);
  r.p = vfmac(mu1, 0.5f, s);
  r.m = vfmac(mu1, -0.5f, s);
  return r;
}
// Projection after streaming: pl = phi_+ pulled from the minus side, z = own
// phi_0, mr = phi_- pulled from the plus side.  m0 is summed as (pl + mr) + z so
// that m2 reuses pl + mr.
template <class T>
__device__ __forceinline__ T proj0(T pl, T z, T mr) { return vadd(vadd(pl, mr), z); }
template <class T>
__device__ __forceinline__ T proj1(T pl, T mr) { return vsub(pl, mr); }
template <class T>
__device__ __forceinline__ T proj2(T pl, T mr, T o0) { return vfmac(o0, -1.0f / 3.0f, vadd(pl, mr)); }

// Stored variables from the ten streamed moments (rest removed):
//   rho' = 1 + m000, rho' u' = m_a + F_a/2, rho' S'_ab = m_ab, n'_ab = m_ab - (rho' u'_a) u'_b.
template <bool FORCE, class T>
__device__ __forceinline__ StoredT<T> finish_moments(T m000, T m100, T m010, T m001, T m200,
                                                     T m020, T m002, T m110, T m101, T m011, T fx,
                                                     T fy, T fz) {
  StoredT<T> o;
  o.drho = m000;
  const T inv = vrcp(vadd(m000, vset<T>(1.0f)));
  T jx = m100, jy = m010, jz = m001;
  if (FORCE) {
    jx = vfmac(fx, 0.5f, jx);
    jy = vfmac(fy, 0.5f, jy);
    jz = vfmac(fz, 0.5f, jz);
  }
  o.ux = vmul(jx, inv);
  o.uy = vmul(jy, inv);
  o.uz = vmul(jz, inv);
  const T njx = vmulc(jx, -1.0f), njy = vmulc(jy, -1.0f), njz = vmulc(jz, -1.0f);  // exact
  o.nxx = vfma(njx, o.ux, m200);
  o.nyy = vfma(njy, o.uy, m020);
  o.nzz = vfma(njz, o.uz, m002);
  o.nxy = vfma(njx, o.uy, m110);
  o.nxz = vfma(njx, o.uz, m101);
  o.nyz = vfma(njy, o.uz, m011);
  return o;
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

}  // namespace melbm
