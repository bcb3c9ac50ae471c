#pragma once
// fluid_kernel.cuh -- the fluid-interior kernel of the split design (Sec. 4.2, Alg. 2):
// one uniform, branch-free update of every cell:
//   load stored moments -> collide (App. A) -> Hermite moments of f+
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
//   * a block is 32 lanes (x) by FY warps (y); the lanes are the 32 columns
//     x0 .. x0+31 and the warps cover rows y0-1 .. y0+FY-2, so warps 0 and FY-1
//     are recomputed halo rows;
//   * warp 0 also computes, one plane pair ahead, the x-pass populations of the
//     columns x0-1 (phi+) and x0+32 (phi-) for every row and passes them through
//     shared memory; after the x shuffles they replace the values that lane 0
//     and lane 31 received from the far end of the warp.  The stored words of
//     those two columns reach a double-buffered staging area by cp.async,
//     issued two pairs ahead, so they occupy no registers while the warp does
//     its own row.  In 16-bit storage each word is copied alone (4 bytes); in
//     FP32 storage the 16-byte aligned chunk holding it is copied past L1, so
//     the gather of 32 rows does not crowd the L1 lines that the other warps'
//     loads are landing in;
//   * each iteration advances two z-planes held as the two halves of float2
//     values, so every arithmetic step is one packed FP32x2 instruction;
//   * the x pass exchanges directional populations with warp shuffles;
//   * the y pass exchanges them through double-buffered shared memory (64-bit
//     accesses, one barrier per plane pair);
//   * the z pass keeps the previous pair's populations in registers;
//   * the next pair's loads are issued before the current pair is processed.
//
// D3Q19 (Q19 = true) runs the same three passes.  Its post-collision populations,
// zero on the eight corners of the 27-velocity cube, have tensor Hermite moments
// mu_pqr for all 27 (p, q, r); the sixteen that the reconstruction is built from
// are those of D3Q27 with mu_111 = 0, and the other ten follow from them in
// closed form (closure19).  The x pass then has nine full slices instead of
// eight partial ones; the y and z passes and the stored form are unchanged.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

// Tile shape: FY warps per block (rows), at most ZCHUNK planes per block (even;
// the launcher picks the length per grid), and the
// minimum number of resident blocks per SM requested from the compiler.
#ifndef MELBM_FLUID_FY
#define MELBM_FLUID_FY 16
#endif
#ifndef MELBM_FLUID_ZCHUNK
#define MELBM_FLUID_ZCHUNK 128
#endif
#ifndef MELBM_FLUID_MINB
#define MELBM_FLUID_MINB 1
#endif
// 32-bit words per staged halo entry of the 16-bit kernel (1: the word alone
// through L1; 4: its 16-byte aligned chunk, L2 only)
#ifndef MELBM_Q16_HALO_CHUNK
#define MELBM_Q16_HALO_CHUNK 1
#endif
// z-loop unroll factor, an expression of the kernel's STORAGE and FORCE parameters
#ifndef MELBM_FLUID_ZUNROLL
#define MELBM_FLUID_ZUNROLL (STORAGE == ST_F32 && !FORCE ? 2 : 1)
#endif
constexpr int FX = 32;
constexpr int FY = MELBM_FLUID_FY;
constexpr int FYI = FY - 2;
constexpr int NSX = 8;                      // x-pass slices (D3Q27; nine for D3Q19)
constexpr int NSY = 9;                      // y-pass slices exchanged through shared memory
constexpr int SM_BUF = 2 * NSY * FY * FX;  // float2 per buffer (phi+ and phi-)
template <bool Q19>
constexpr int nsx() { return Q19 ? NSX + 1 : NSX; }
template <bool Q19>
constexpr int halo_buf() { return 2 * FY * nsx<Q19>(); }  // float2 per halo buffer (two columns)
static_assert(2 * FY <= 32, "warp 0 covers both halo columns of every row");
constexpr int ZCHUNK = MELBM_FLUID_ZCHUNK;
static_assert(ZCHUNK % 2 == 0, "planes are processed in pairs");

// Warp 0's halo staging, two buffers: per halo lane, 2 W entries (word w of
// plane h at entry 2 w + h) plus 6 for the forces; an entry is CHUNK 32-bit
// words, laid out [buffer][entry][lane][CHUNK].
template <int STORAGE, bool FORCE, bool Q19 = false>
struct HaloStage {
  static constexpr int W = STORAGE == ST_Q16 ? 5 : 10;     // stored 32-bit words per cell
  static constexpr int CHUNK = STORAGE == ST_Q16 ? MELBM_Q16_HALO_CHUNK : 4;  // 4: 16-byte chunk
  static constexpr int ENTRIES = 2 * W + (FORCE ? 6 : 0);
  static constexpr int BUF_WORDS = ENTRIES * 32 * CHUNK;
  static constexpr size_t SMEM =
      size_t(2) * (SM_BUF + halo_buf<Q19>()) * sizeof(float2) + size_t(2) * BUF_WORDS * 4;
};

struct FluidParams {
  int nx, ny, nz, zc;
  const void* in;
  void* out;
  const float* force;
  float omega;
  uint32_t t_out, seed;
  int chunk16;  // FP32 storage: 16-byte aligned rows, so the halo gather copies chunks
};

template <int STORAGE, bool RT> struct KernelParams;
// the grid constants of the RT kernel (nullptr for the others)
template <class KP>
__device__ __forceinline__ const QGrids* grids_of(const KP& p) {
  if constexpr (std::is_same_v<KP, KernelParams<ST_Q16, true>>)
    return &p.q;
  else
    return nullptr;
}

// Kernel parameters per storage: the FP32 kernel also gets per-word plane
// pointers of in / out and of the force components; the quantised kernel with
// bit widths other than 16/16 (RT) gets the grid constants.
template <int STORAGE, bool RT>
struct KernelParams : FluidParams {};
template <>
struct KernelParams<ST_Q16, true> : FluidParams {
  QGrids q;
};
template <>
struct KernelParams<ST_MIXED, false> : FluidParams {
  uint32_t* out_w[10];  // the raw FP32 post-streaming moment planes
};
template <>
struct KernelParams<ST_F32, false> : FluidParams {
  const uint32_t* in_w[10];
  uint32_t* out_w[10];
  const uint32_t* f_w[3];
};

// ----------------------------------------------------------------- plane-pair I/O
template <int STORAGE> struct RawPair;
template <> struct RawPair<ST_Q16> { uint32_t a[5], b[5]; };
template <> struct RawPair<ST_F32> { float a[10], b[10]; };

// FP32 word planes are addressed through per-word base pointers held in the
// kernel parameters (uniform), so each access adds one per-thread offset; the
// five 16-bit planes are addressed as base + k N (each form measured the faster
// one for its storage).
using WordPlanes = const uint32_t* const*;

__device__ __forceinline__ void load_pair(RawPair<ST_Q16>& r, const void* buf, size_t N, size_t na,
                                          size_t nb) {
  const uint32_t* p = static_cast<const uint32_t*>(buf);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    r.a[k] = __ldg(p + k * N + na);
    r.b[k] = __ldg(p + k * N + nb);
  }
}
__device__ __forceinline__ void load_pair(RawPair<ST_F32>& r, WordPlanes w, size_t na, size_t nb) {
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    r.a[k] = __uint_as_float(__ldg(w[k] + na));
    r.b[k] = __uint_as_float(__ldg(w[k] + nb));
  }
}

__device__ __forceinline__ StoredT<float2> decode_pair(const RawPair<ST_Q16>& r) {
  StoredT<float2> s;
  s.drho = q_decode<0>(make_float2(q_lo_magic(r.a[0]), q_lo_magic(r.b[0])));
  s.ux = q_decode<1>(make_float2(q_hi_magic(r.a[0]), q_hi_magic(r.b[0])));
  s.uy = q_decode<1>(make_float2(q_lo_magic(r.a[1]), q_lo_magic(r.b[1])));
  s.uz = q_decode<1>(make_float2(q_hi_magic(r.a[1]), q_hi_magic(r.b[1])));
  s.nxx = q_decode<2>(make_float2(q_lo_magic(r.a[2]), q_lo_magic(r.b[2])));
  s.nyy = q_decode<2>(make_float2(q_hi_magic(r.a[2]), q_hi_magic(r.b[2])));
  s.nzz = q_decode<2>(make_float2(q_lo_magic(r.a[3]), q_lo_magic(r.b[3])));
  s.nxy = q_decode<2>(make_float2(q_hi_magic(r.a[3]), q_hi_magic(r.b[3])));
  s.nxz = q_decode<2>(make_float2(q_lo_magic(r.a[4]), q_lo_magic(r.b[4])));
  s.nyz = q_decode<2>(make_float2(q_hi_magic(r.a[4]), q_hi_magic(r.b[4])));
  return s;
}
__device__ __forceinline__ StoredT<float2> decode_pair(const RawPair<ST_Q16>& r, const QGrids& q) {
  StoredT<float2> s;
  s.drho = qg_decode(q.g[0], make_float2(q_lo_magic(r.a[0]), q_lo_magic(r.b[0])));
  s.ux = qg_decode(q.g[1], make_float2(q_hi_magic(r.a[0]), q_hi_magic(r.b[0])));
  s.uy = qg_decode(q.g[1], make_float2(q_lo_magic(r.a[1]), q_lo_magic(r.b[1])));
  s.uz = qg_decode(q.g[1], make_float2(q_hi_magic(r.a[1]), q_hi_magic(r.b[1])));
  s.nxx = qg_decode(q.g[2], make_float2(q_lo_magic(r.a[2]), q_lo_magic(r.b[2])));
  s.nyy = qg_decode(q.g[2], make_float2(q_hi_magic(r.a[2]), q_hi_magic(r.b[2])));
  s.nzz = qg_decode(q.g[2], make_float2(q_lo_magic(r.a[3]), q_lo_magic(r.b[3])));
  s.nxy = qg_decode(q.g[2], make_float2(q_hi_magic(r.a[3]), q_hi_magic(r.b[3])));
  s.nxz = qg_decode(q.g[2], make_float2(q_lo_magic(r.a[4]), q_lo_magic(r.b[4])));
  s.nyz = qg_decode(q.g[2], make_float2(q_hi_magic(r.a[4]), q_hi_magic(r.b[4])));
  return s;
}
__device__ __forceinline__ StoredT<float2> decode_pair(const RawPair<ST_F32>& r) {
  StoredT<float2> s;
  s.drho = make_float2(r.a[0], r.b[0]);
  s.ux = make_float2(r.a[1], r.b[1]);
  s.uy = make_float2(r.a[2], r.b[2]);
  s.uz = make_float2(r.a[3], r.b[3]);
  s.nxx = make_float2(r.a[4], r.b[4]);
  s.nyy = make_float2(r.a[5], r.b[5]);
  s.nzz = make_float2(r.a[6], r.b[6]);
  s.nxy = make_float2(r.a[7], r.b[7]);
  s.nxz = make_float2(r.a[8], r.b[8]);
  s.nyz = make_float2(r.a[9], r.b[9]);
  return s;
}

// Store the pair (planes za, zb = za + 1) -- each half only if its flag is set.
using OutPlanes = uint32_t* const*;

__device__ __forceinline__ void store_pair_f32(OutPlanes w, size_t na, size_t nb,
                                               const StoredT<float2>& o, bool sa, bool sb) {
  const float2 v[10] = {o.drho, o.ux, o.uy, o.uz, o.nxx, o.nyy, o.nzz, o.nxy, o.nxz, o.nyz};
  if (sa) {
#pragma unroll
    for (int k = 0; k < 10; ++k) w[k][na] = __float_as_uint(v[k].x);
  }
  if (sb) {
#pragma unroll
    for (int k = 0; k < 10; ++k) w[k][nb] = __float_as_uint(v[k].y);
  }
}

template <bool RT>
__device__ __forceinline__ void store_pair_q16(void* buf, size_t N, size_t na, size_t nb,
                                               const StoredT<float2>& o, bool sa, bool sb, uint32_t x,
                                               uint32_t y, uint32_t za, uint32_t zb, uint32_t t,
                                               uint32_t seed, const QGrids* q) {
  const DitherBits ha = pcg4d(x, y, za, t, seed);
  const DitherBits hb = pcg4d(x, y, zb, t, seed);
  float2 d[10];
#pragma unroll
  for (int k = 0; k < 10; ++k)
    d[k] = dither_value(make_float2(dither_magic(ha, k), dither_magic(hb, k)), k);
  uint2 e0, e1, e2, e3, e4, e5, e6, e7, e8, e9;
  if constexpr (RT) {
    e0 = qg_encode_codes(q->g[0], o.drho, d[0]), e1 = qg_encode_codes(q->g[1], o.ux, d[1]);
    e2 = qg_encode_codes(q->g[1], o.uy, d[2]), e3 = qg_encode_codes(q->g[1], o.uz, d[3]);
    e4 = qg_encode_codes(q->g[2], o.nxx, d[4]), e5 = qg_encode_codes(q->g[2], o.nyy, d[5]);
    e6 = qg_encode_codes(q->g[2], o.nzz, d[6]), e7 = qg_encode_codes(q->g[2], o.nxy, d[7]);
    e8 = qg_encode_codes(q->g[2], o.nxz, d[8]), e9 = qg_encode_codes(q->g[2], o.nyz, d[9]);
  } else {
    e0 = q_encode_codes<0>(o.drho, d[0]), e1 = q_encode_codes<1>(o.ux, d[1]);
    e2 = q_encode_codes<1>(o.uy, d[2]), e3 = q_encode_codes<1>(o.uz, d[3]);
    e4 = q_encode_codes<2>(o.nxx, d[4]), e5 = q_encode_codes<2>(o.nyy, d[5]);
    e6 = q_encode_codes<2>(o.nzz, d[6]), e7 = q_encode_codes<2>(o.nxy, d[7]);
    e8 = q_encode_codes<2>(o.nxz, d[8]), e9 = q_encode_codes<2>(o.nyz, d[9]);
  }
  uint32_t* p = static_cast<uint32_t*>(buf);
  if constexpr (RT) {
    const uint32_t qr = q->g[1].qmax, qs = q->g[2].qmax;
    if (sa) {
      p[na] = qg_clamp_word(q_pack(e0.x, e1.x), qr);
      p[N + na] = qg_clamp_word(q_pack(e2.x, e3.x), qr);
      p[2 * N + na] = qg_clamp_word(q_pack(e4.x, e5.x), qs);
      p[3 * N + na] = qg_clamp_word(q_pack(e6.x, e7.x), qs);
      p[4 * N + na] = qg_clamp_word(q_pack(e8.x, e9.x), qs);
    }
    if (sb) {
      p[nb] = qg_clamp_word(q_pack(e0.y, e1.y), qr);
      p[N + nb] = qg_clamp_word(q_pack(e2.y, e3.y), qr);
      p[2 * N + nb] = qg_clamp_word(q_pack(e4.y, e5.y), qs);
      p[3 * N + nb] = qg_clamp_word(q_pack(e6.y, e7.y), qs);
      p[4 * N + nb] = qg_clamp_word(q_pack(e8.y, e9.y), qs);
    }
  } else {
    if (sa) {
      p[na] = q_pack(e0.x, e1.x);
      p[N + na] = q_pack(e2.x, e3.x);
      p[2 * N + na] = q_pack(e4.x, e5.x);
      p[3 * N + na] = q_pack(e6.x, e7.x);
      p[4 * N + na] = q_pack(e8.x, e9.x);
    }
    if (sb) {
      p[nb] = q_pack(e0.y, e1.y);
      p[N + nb] = q_pack(e2.y, e3.y);
      p[2 * N + nb] = q_pack(e4.y, e5.y);
      p[3 * N + nb] = q_pack(e6.y, e7.y);
      p[4 * N + nb] = q_pack(e8.y, e9.y);
    }
  }
}

// Asynchronous global -> shared copies (cp.async, completed per thread): 4 bytes
// through L1, or 16 bytes (aligned) cached in L2 only.
__device__ __forceinline__ void cp_async4(uint32_t* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_l2(uint32_t* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

template <int STORAGE>
__device__ __forceinline__ void set_word(RawPair<STORAGE>& r, int h, int w, uint32_t v);
template <>
__device__ __forceinline__ void set_word<ST_Q16>(RawPair<ST_Q16>& r, int h, int w, uint32_t v) {
  (h ? r.b : r.a)[w] = v;
}
template <>
__device__ __forceinline__ void set_word<ST_F32>(RawPair<ST_F32>& r, int h, int w, uint32_t v) {
  (h ? r.b : r.a)[w] = __uint_as_float(v);
}

__device__ __forceinline__ float2 shfl_idx2(float2 v, int src) {
  return make_float2(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src));
}

// ----------------------------------------------------------------- kernel
// The y-pass slices are indexed s = 3 p + r' (p: x-order, r': input z-order).
template <int STORAGE, bool FORCE, bool RT, bool Q19 = false>
__global__ void __launch_bounds__(FX* FY, MELBM_FLUID_MINB) fluid_kernel(KernelParams<STORAGE, RT> P) {
  // the input side reads 16-bit codes in the mixed scheme (post-collision moments)
  constexpr int IN = STORAGE == ST_MIXED ? ST_Q16 : STORAGE;
  using HS = HaloStage<IN, FORCE, Q19>;
  constexpr int NSXL = nsx<Q19>();
  constexpr int HALO_BUF = halo_buf<Q19>();
  auto decode = [&](const RawPair<IN>& r) {
    if constexpr (IN == ST_Q16 && RT) return decode_pair(r, P.q);
    else return decode_pair(r);
  };
  extern __shared__ float2 sm2[];
  float2* const hb = sm2 + 2 * SM_BUF;  // halo populations [buffer][row][slice][side]
  uint32_t* const stg = reinterpret_cast<uint32_t*>(hb + 2 * HALO_BUF);  // warp 0 staging
  const int lane = threadIdx.x, row = threadIdx.y;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const size_t N = size_t(nx) * ny * nz;
  const int x0 = int(blockIdx.x) * FX, y0 = int(blockIdx.y) * FYI - 1;
  const int x = x0 + lane, y = y0 + row;
  const int xw = wrapi(x, nx), yw = wrapi(y, ny);
  const bool mid_row = (row >= 1 && row <= FY - 2);  // warp-uniform
  const bool col_ok = mid_row && x < nx && y < ny;
  const int z0 = int(blockIdx.z) * P.zc;
  const int z1 = min(z0 + P.zc, nz);
  const size_t col = size_t(xw) + size_t(nx) * yw;
  const size_t plane = size_t(nx) * ny;
  const float omega = P.omega;
  const int src_up = (lane + 31) & 31, src_dn = (lane + 1) & 31;
  // plane index of z in [z0 - 1, z1 + 3]: one conditional wrap when nz > 3
  const bool small_nz = nz <= 3;
  auto wz = [&](int zv) {
    return small_nz ? wrapi(zv, nz) : (zv < 0 ? zv + nz : (zv >= nz ? zv - nz : zv));
  };

  // warp 0's halo cell of this lane: row (lane % FY) of column x0-1 (side 0) or
  // x0+32 (side 1); lanes past 2 FY (FY < 16) compute a copy and store nothing
  const bool halo_warp = (row == 0);  // warp-uniform
  const int hrow = lane % FY, side = (lane / FY) & 1;
  const bool halo_lane = lane < 2 * FY;
  const size_t hcol =
      size_t(wrapi(side ? x0 + FX : x0 - 1, nx)) + size_t(nx) * wrapi(y0 + hrow, ny);

  // z-march state of the six (p, q) slices: phi+ of the previous pair's two
  // planes and phi0 of its second plane
  float2 zP[6];
  float zZ[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    zP[k] = make_float2(0.f, 0.f);
    zZ[k] = 0.f;
  }
  float fprev[3] = {0.f, 0.f, 0.f};

  // Issue the staging of the halo pair (za, za + 1) into staging buffer b.  The
  // pair with index j = (za - z0 + 1) / 2 uses halo buffer j & 1, written one
  // pair ahead (before the barrier of pair j - 1) and read by the x pass of pair j.
  const bool chunk16 = HS::CHUNK == 4 && P.chunk16;
  auto halo_issue = [&](int za, int b) {
    const size_t na = hcol + plane * wz(za), nb = hcol + plane * wz(za + 1);
    uint32_t* d = stg + b * HS::BUF_WORDS + lane * HS::CHUNK;
    const uint32_t* src = static_cast<const uint32_t*>(P.in);
    const float* fsrc = P.force;
    auto copy = [&](int e, const void* g, size_t n) {  // entry e <- element n of g
      if (chunk16)
        cp_async16_l2(d + e * 32 * HS::CHUNK, static_cast<const uint32_t*>(g) + (n & ~size_t(3)));
      else
        cp_async4(d + e * 32 * HS::CHUNK, static_cast<const uint32_t*>(g) + n);
    };
#pragma unroll
    for (int w = 0; w < HS::W; ++w) {
      if constexpr (IN == ST_Q16) {
        copy(2 * w, src + w * N, na);
        copy(2 * w + 1, src + w * N, nb);
      } else {
        copy(2 * w, P.in_w[w], na);
        copy(2 * w + 1, P.in_w[w], nb);
      }
    }
    if (FORCE) {
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        if constexpr (IN == ST_Q16) {
          copy(2 * HS::W + 2 * w, fsrc + w * N, na);
          copy(2 * HS::W + 2 * w + 1, fsrc + w * N, nb);
        } else {
          copy(2 * HS::W + 2 * w, P.f_w[w], na);
          copy(2 * HS::W + 2 * w + 1, P.f_w[w], nb);
        }
      }
    }
    cp_async_commit();
  };
  // Write the x-pass populations of the pair staged in buffer b (its copies have
  // completed) into halo buffer hbuf, laid out [row][slice] as
  // {phi+ of column x0-1, phi- of column x0+32}.
  auto halo_finish = [&](int b, int hbuf) {
    const uint32_t* d = stg + b * HS::BUF_WORDS + lane * HS::CHUNK + (chunk16 ? int(hcol & 3) : 0);
    RawPair<IN> hr;
#pragma unroll
    for (int w = 0; w < HS::W; ++w) {
      set_word<IN>(hr, 0, w, d[(2 * w) * 32 * HS::CHUNK]);
      set_word<IN>(hr, 1, w, d[(2 * w + 1) * 32 * HS::CHUNK]);
    }
    const StoredT<float2> hs = decode(hr);
    float2 hfx = make_float2(0.f, 0.f), hfy = hfx, hfz = hfx;
    if (FORCE) {
      const float* sf = reinterpret_cast<const float*>(d) + 2 * HS::W * 32 * HS::CHUNK;
      hfx = make_float2(sf[0 * 32 * HS::CHUNK], sf[1 * 32 * HS::CHUNK]);
      hfy = make_float2(sf[2 * 32 * HS::CHUNK], sf[3 * 32 * HS::CHUNK]);
      hfz = make_float2(sf[4 * 32 * HS::CHUNK], sf[5 * 32 * HS::CHUNK]);
    }
    const Mom17T<float2> H = collide_moments<FORCE>(hs, omega, hfx, hfy, hfz);
    const float2 zero = make_float2(0.f, 0.f);
    float2 mu[NSXL][3];
    if constexpr (Q19) {
      const Closure19T<float2> E = closure19(H);
      const float2 m[NSXL][3] = {{H.m000, H.m100, H.m200}, {H.m010, H.m110, H.m210},
                                 {H.m020, H.m120, E.m220}, {H.m001, H.m101, H.m201},
                                 {H.m011, zero, E.m211},   {H.m021, E.m121, E.m221},
                                 {H.m002, H.m102, E.m202}, {H.m012, E.m112, E.m212},
                                 {E.m022, E.m122, E.m222}};
#pragma unroll
      for (int k = 0; k < NSXL; ++k)
        for (int j = 0; j < 3; ++j) mu[k][j] = m[k][j];
    } else {
      const float2 m[NSX][3] = {{H.m000, H.m100, H.m200}, {H.m010, H.m110, H.m210},
                                {H.m020, H.m120, zero},   {H.m001, H.m101, H.m201},
                                {H.m011, H.m111, zero},   {H.m021, zero, zero},
                                {H.m002, H.m102, zero},   {H.m012, zero, zero}};
#pragma unroll
      for (int k = 0; k < NSX; ++k)
        for (int j = 0; j < 3; ++j) mu[k][j] = m[k][j];
    }
    float2* dst = hb + hbuf * HALO_BUF + hrow * NSXL * 2 + side;
#pragma unroll
    for (int k = 0; k < NSXL; ++k) {
      const PhiT<float2> ph = phi3(mu[k][0], mu[k][1], mu[k][2]);
      if (halo_lane) dst[2 * k] = side ? ph.m : ph.p;
    }
  };

  RawPair<IN> raw;
  if constexpr (IN == ST_Q16)
    load_pair(raw, P.in, N, col + plane * wz(z0 - 1), col + plane * wz(z0));
  else
    load_pair(raw, P.in_w, col + plane * wz(z0 - 1), col + plane * wz(z0));
  // Staging schedule (pair j = (zz - z0 + 1) / 2, window j = the work between the
  // barriers of pairs j - 1 and j): pair j + 2 is issued at the start of window j
  // into staging buffer j & 1, and pair j + 1 is consumed at its end.
  if (halo_warp) {
    halo_issue(z0 - 1, 0);
    if (z0 + 1 <= z1) {
      halo_issue(z0 + 1, 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    halo_finish(0, 0);
  }
  __syncthreads();
  int parity = 0;
  // FP32 storage without force: two plane pairs per loop trip (the loop-carried
  // z-pass state then alternates registers instead of being copied; measured
  // +2.5%); the other kernels stay rolled (unrolled they spill, and the 16-bit
  // one runs 2% slower).
#define MELBM_PRAGMA_STR(x) #x
#define MELBM_PRAGMA_UNROLL(n) _Pragma(MELBM_PRAGMA_STR(unroll n))
  MELBM_PRAGMA_UNROLL(MELBM_FLUID_ZUNROLL)
  for (int zz = z0 - 1; zz <= z1; zz += 2, parity ^= 1) {
    const bool halo_next = halo_warp && zz + 2 <= z1;
    const bool halo_ahead = halo_warp && zz + 4 <= z1;
    if (halo_ahead) halo_issue(zz + 4, parity);
    const StoredT<float2> s = decode(raw);
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx;
    if (FORCE) {
      const size_t na = col + plane * wz(zz), nb = col + plane * wz(zz + 1);
      if constexpr (IN == ST_Q16) {
        fx = make_float2(__ldg(P.force + na), __ldg(P.force + nb));
        fy = make_float2(__ldg(P.force + N + na), __ldg(P.force + N + nb));
        fz = make_float2(__ldg(P.force + 2 * N + na), __ldg(P.force + 2 * N + nb));
      } else {
        fx = make_float2(__uint_as_float(__ldg(P.f_w[0] + na)), __uint_as_float(__ldg(P.f_w[0] + nb)));
        fy = make_float2(__uint_as_float(__ldg(P.f_w[1] + na)), __uint_as_float(__ldg(P.f_w[1] + nb)));
        fz = make_float2(__uint_as_float(__ldg(P.f_w[2] + na)), __uint_as_float(__ldg(P.f_w[2] + nb)));
      }
    }
    if (zz + 2 <= z1)  // prefetch the next pair
    {
      if constexpr (IN == ST_Q16)
        load_pair(raw, P.in, N, col + plane * wz(zz + 2), col + plane * wz(zz + 3));
      else
        load_pair(raw, P.in_w, col + plane * wz(zz + 2), col + plane * wz(zz + 3));
    }
    const Mom17T<float2> A = collide_moments<FORCE>(s, omega, fx, fy, fz);

    // ---------------- x pass on slices (q', r'), then the y-pass populations of
    // the slices (p, r') as soon as their three inputs X[p][0..2][r'] exist
    // (grouped by r' so that only nine X values are live at a time)
    const float2 zero = make_float2(0.f, 0.f);
    float2* sp = sm2 + parity * SM_BUF;
    float2 yz0[NSY];
    float2 X[3][3];  // X[p][q'] of the current r'
    const float4* hbp = reinterpret_cast<const float4*>(hb + parity * HALO_BUF) + row * NSXL;
    int xs = 0;  // x-pass slice index (halo buffer order)
#define MELBM_XPASS(Q, A0, A1, A2)                                      \
  {                                                                     \
    const PhiT<float2> ph = phi3(A0, A1, A2);                           \
    const float4 h = hbp[xs];                                           \
    float2 pl = shfl_idx2(ph.p, src_up);                                \
    float2 mr = shfl_idx2(ph.m, src_dn);                                \
    if (lane == 0) pl = make_float2(h.x, h.y);                          \
    if (lane == FX - 1) mr = make_float2(h.z, h.w);                     \
    X[0][Q] = proj0(pl, ph.z, mr);                                      \
    X[1][Q] = proj1(pl, mr);                                            \
    X[2][Q] = proj2(pl, mr, X[0][Q]);                                   \
    ++xs;                                                               \
  }
#define MELBM_YPHI(R)                                                   \
  _Pragma("unroll") for (int p = 0; p < 3; ++p) {                       \
    const PhiT<float2> ph = phi3(X[p][0], X[p][1], X[p][2]);            \
    const int s_ = 3 * p + (R);                                         \
    sp[(s_ * FY + row) * FX + lane] = ph.p;                             \
    sp[((NSY + s_) * FY + row) * FX + lane] = ph.m;                     \
    yz0[s_] = ph.z;                                                     \
  }
    if constexpr (Q19) {
      const Closure19T<float2> E = closure19(A);
      MELBM_XPASS(0, A.m000, A.m100, A.m200)  // r' = 0
      MELBM_XPASS(1, A.m010, A.m110, A.m210)
      MELBM_XPASS(2, A.m020, A.m120, E.m220)
      MELBM_YPHI(0)
      MELBM_XPASS(0, A.m001, A.m101, A.m201)  // r' = 1; mu_111 = 0
      MELBM_XPASS(1, A.m011, zero, E.m211)
      MELBM_XPASS(2, A.m021, E.m121, E.m221)
      MELBM_YPHI(1)
      MELBM_XPASS(0, A.m002, A.m102, E.m202)  // r' = 2
      MELBM_XPASS(1, A.m012, E.m112, E.m212)
      MELBM_XPASS(2, E.m022, E.m122, E.m222)
      MELBM_YPHI(2)
    } else {
      MELBM_XPASS(0, A.m000, A.m100, A.m200)  // r' = 0
      MELBM_XPASS(1, A.m010, A.m110, A.m210)
      MELBM_XPASS(2, A.m020, A.m120, zero)
      MELBM_YPHI(0)
      MELBM_XPASS(0, A.m001, A.m101, A.m201)  // r' = 1
      MELBM_XPASS(1, A.m011, A.m111, zero)
      MELBM_XPASS(2, A.m021, zero, zero)
      MELBM_YPHI(1)
      MELBM_XPASS(0, A.m002, A.m102, zero)    // r' = 2; (q', r') = (2, 2) has no input
      MELBM_XPASS(1, A.m012, zero, zero)
      X[0][2] = X[1][2] = X[2][2] = zero;
      MELBM_YPHI(2)
    }
#undef MELBM_XPASS
#undef MELBM_YPHI
    if (halo_next) {
      if (halo_ahead) cp_async_wait<1>();
      else cp_async_wait<0>();
      halo_finish(parity ^ 1, parity ^ 1);
    }
    __syncthreads();
    if (!mid_row) continue;

    // ---------------- y pass, part 2: pull and project -> Y[p][q][r'], q <= 2 - p
    float2 Y[3][3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int s_ = 3 * p + r;
        const float2 pl = sp[(s_ * FY + row - 1) * FX + lane];
        const float2 mr = sp[((NSY + s_) * FY + row + 1) * FX + lane];
        Y[p][0][r] = proj0(pl, yz0[s_], mr);
        if (p <= 1) Y[p][1][r] = proj1(pl, mr);
        if (p == 0) Y[p][2][r] = proj2(pl, mr, Y[p][0][r]);
      }

    // ---------------- z pass for slices (p, q): planes (zz, zz+1) in, (zz-1, zz) out
    const int PQ[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    float2 M[6][3];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int p = PQ[k][0], q = PQ[k][1];
      const PhiT<float2> ph = phi3(Y[p][q][0], Y[p][q][1], Y[p][q][2]);
      // out(zz-1) = proj(phi+(zz-2), phi0(zz-1), phi-(zz)); out(zz) = proj(phi+(zz-1), phi0(zz), phi-(zz+1))
      // (phi_0 of the output pair straddles two input pairs: its sum with pl + mr
      // is taken per half, so no register pair has to be assembled for it)
      const float2 pl = zP[k];
      const float2 mr = ph.m;
      const float2 lr = vadd(pl, mr);
      M[k][0] = make_float2(__fadd_rn(lr.x, zZ[k]), __fadd_rn(lr.y, ph.z.x));
      M[k][1] = proj1(pl, mr);
      M[k][2] = vfmac(M[k][0], -1.0f / 3.0f, lr);
      zP[k] = ph.p;
      zZ[k] = ph.z.y;
    }
    if (zz - 1 >= z0) {
      float2 ox = zero, oy = zero, oz = zero;
      if (FORCE) {
        ox = make_float2(fprev[0], fx.x);
        oy = make_float2(fprev[1], fy.x);
        oz = make_float2(fprev[2], fz.x);
      }
      // slices: 0:(0,0) 1:(1,0) 2:(0,1) 3:(2,0) 4:(1,1) 5:(0,2)
      const int za = zz - 1, zb = zz;
      if constexpr (STORAGE == ST_MIXED) {
        // the raw post-streaming sums rho - 1, sum c f, sum (c c - 1/3) f
        StoredT<float2> r;
        r.drho = M[0][0], r.ux = M[1][0], r.uy = M[2][0], r.uz = M[0][1];
        r.nxx = M[3][0], r.nyy = M[5][0], r.nzz = M[0][2];
        r.nxy = M[4][0], r.nxz = M[1][1], r.nyz = M[2][1];
        store_pair_f32(P.out_w, col + plane * za, col + plane * (zb < nz ? zb : 0), r, col_ok,
                       col_ok && zb < z1);
        continue;
      }
      const StoredT<float2> o =
          finish_moments<FORCE>(M[0][0], M[1][0], M[2][0], M[0][1], M[3][0], M[5][0], M[0][2],
                                M[4][0], M[1][1], M[2][1], ox, oy, oz);
      if constexpr (STORAGE == ST_Q16)
        store_pair_q16<RT>(P.out, N, col + plane * za, col + plane * (zb < nz ? zb : 0), o, col_ok,
                       col_ok && zb < z1, uint32_t(xw), uint32_t(yw), uint32_t(za), uint32_t(zb),
                       P.t_out, P.seed, grids_of(P));
      else
        store_pair_f32(P.out_w, col + plane * za, col + plane * (zb < nz ? zb : 0), o, col_ok,
                       col_ok && zb < z1);
    }
    if (FORCE) {
      fprev[0] = fx.y;
      fprev[1] = fy.y;
      fprev[2] = fz.y;
    }
  }
}

// z-chunk length: the even length (ZCHUNK = 128 down to 4) minimising the number of
// waves times the plane pairs a block iterates over (chunk / 2 + 1, the first
// pair feeding the z pass only), so that small grids still fill the GPU.
inline int choose_zchunk(int64_t tiles_xy, int nz, int64_t resident_blocks) {
  int best = ZCHUNK;
  int64_t best_cost = INT64_MAX;
  for (int zc = ZCHUNK; zc >= 4; zc -= 2) {
    const int64_t blocks = tiles_xy * ((nz + zc - 1) / zc);
    const int64_t cost = (blocks + resident_blocks - 1) / resident_blocks * (zc / 2 + 1);
    if (cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

template <int STORAGE, bool FORCE, bool RT, bool Q19 = false>
cudaError_t launch_fluid_t(KernelParams<STORAGE, RT>& p, cudaStream_t st) {
  const size_t smem = HaloStage<STORAGE == ST_MIXED ? ST_Q16 : STORAGE, FORCE, Q19>::SMEM;
  // per device: the shared-memory opt-in of this instantiation and the number of
  // its blocks resident on the whole GPU (set once; a racing first call writes
  // the same values)
  constexpr int MAX_DEV = 64;
  static int resident[MAX_DEV] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  if (!resident[dev]) {
    int sms = 0, per_sm = 0;
    e = cudaFuncSetAttribute(fluid_kernel<STORAGE, FORCE, RT, Q19>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_kernel<STORAGE, FORCE, RT, Q19>,
                                                        FX * FY, smem);
    if (e != cudaSuccess) return e;
    resident[dev] = std::max(1, sms * per_sm);
  }
  const int64_t tiles_xy = int64_t((p.nx + FX - 1) / FX) * ((p.ny + FYI - 1) / FYI);
  p.zc = choose_zchunk(tiles_xy, p.nz, resident[dev]);
  dim3 grid((p.nx + FX - 1) / FX, (p.ny + FYI - 1) / FYI, (p.nz + p.zc - 1) / p.zc);
  fluid_kernel<STORAGE, FORCE, RT, Q19><<<grid, dim3(FX, FY), smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace melbm
