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
// Per pair j the work splits into pre(j) (decode, collide, x pass, y-pass
// populations into shared-memory buffer j & 1) and post(j) (y pass from that
// buffer, z pass, moments, encode, store), with one barrier between them.  The
// 16-bit kernel runs post(j - 1) and pre(j) in one straight block between two
// barriers (they use different buffers), so that the integer work of one pair
// (dither hash, decode, packing) and the arithmetic of the other can be
// interleaved; the FP32 kernel, which has twice the bytes in flight, keeps
// pre(j), barrier, post(j) with two pairs per loop trip.  The 16-bit word planes
// are addressed by 32-bit cell offsets from per-plane base pointers.
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
#define MELBM_FLUID_ZCHUNK 256
#endif
#ifndef MELBM_FLUID_MINB
#define MELBM_FLUID_MINB 1
#endif
// 32-bit words per staged halo entry of the 16-bit kernel (1: the word alone
// through L1; 4: its 16-byte aligned chunk, L2 only)
#ifndef MELBM_Q16_HALO_CHUNK
#define MELBM_Q16_HALO_CHUNK 1
#endif
// z-loop unroll factor of the FP32 kernel, an expression of its FORCE parameter
#ifndef MELBM_FLUID_ZUNROLL
#define MELBM_FLUID_ZUNROLL (!FORCE ? 2 : 1)
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
template <int STORAGE, bool FORCE, bool Q19 = false, bool BND = false>
struct HaloStage {
  static constexpr int W = STORAGE == ST_Q16 ? 5 : 10;     // stored 32-bit words per cell
  static constexpr int CHUNK = STORAGE == ST_Q16 ? MELBM_Q16_HALO_CHUNK : 4;  // 4: 16-byte chunk
  // the state words of both planes, the force, and with solids the solid-bit
  // words of both planes (copied alone, into the first word of their entries)
  static constexpr int ENTRIES = 2 * W + (FORCE ? 6 : 0) + (BND ? 2 : 0);
  static constexpr int BUF_WORDS = ENTRIES * 32 * CHUNK;
  // with solids, the bounce-back records of the pair a thread stores next: five
  // 16-byte slots per thread (two per plane, and one for both planes' last 8 bytes)
  static constexpr size_t REC_BYTES = BND ? size_t(5) * FY * FX * 16 : 0;
  static constexpr size_t SMEM = size_t(2) * (SM_BUF + halo_buf<Q19>()) * sizeof(float2) +
                                 size_t(2) * BUF_WORDS * 4 + REC_BYTES;
};

struct FluidParams {
  int nx, ny, nz, zc;
  const void* in;
  void* out;
  const float* force;
  float omega;
  uint32_t t_out, seed;
  int chunk16;  // FP32 storage: 16-byte aligned rows, so the halo gather copies chunks
  const uint32_t* qin[5];  // 16-bit words: the five word planes of the input
  uint32_t* qout[5];       // and of the output (16-bit storage)
  // With solids (BND kernels): per 32-cell word (tx, y, z) of a row, the bits of
  // its SOLID and FLUID_BOUNDARY cells and the list index of its first listed
  // cell after an INFLOW cell at its lane 0; side[L][12] holds, for every
  // FLUID_BOUNDARY cell (list order), the sums of the populations its solid links
  // return, times the scale factors of the passes (-1, 2, 2, 2, 1, 1, 1, -4, -4,
  // -4), written by the bounce kernel before this one.
  const uint32_t* cls_solid;
  const uint32_t* cls_fb;
  const uint32_t* cls_pref;
  float* side;
  int64_t L;
  int ntx;  // words per row, ceil(nx / 32)
  // 16-bit kernels without the tables synchronise their rows by per-row barriers
  // whose waits are bounded: a wait that runs out sets *fault (mapped host memory,
  // may be null) and returns.  stall_test != 0 initialises warp 0's barriers for
  // twice the arrivals they receive, so that the waits on them run out (a test
  // of that path; nothing else sets it).
  uint32_t* fault;
  int stall_test;
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

// ----------------------------------------------------------------- scaled passes
// The passes carry every tensor moment mu_pqr multiplied by s(p) s(q) s(r), with
// s = (-1, 2, 1) for the orders 0, 1, 2 along each axis.  In that scaling one
// axis of the stream needs no multiply beyond the fused ones: from the inputs
// (a0, a1, a2) = (-mu0, 2 mu1, mu2) of a slice
//   sigma = a0 (-1/3) + a2  (= mu0/3 + mu2),   P+- = sigma +- a1/2  (= 2 phi+-),
//   Zn = sigma + a0  (= -phi0),
// and after the pull (pl = P+ of the minus neighbour, mr = P- of the plus one)
//   b0 = (pl + mr)(-1/2) + Zn  (= -m0),  b1 = pl - mr  (= 2 m1),
//   b2 = b0 (-2/3) + Zn  (= m2),
// which are the next axis' inputs in the same scaling (the D1Q3 map of
// melbm_device.cuh's phi3 / proj written for scaled moments; the sums of b0 and
// b1 over the grid still equal those of a0 and a1 up to unbiased rounding).  A
// full slice costs eight packed operations, one with a2 = 0 the same with a
// multiply for sigma, one with only a0 six.
template <class T>
struct PhiS {
  T p, zn, m;  // P+, Zn, P-
};
template <class T>
__device__ __forceinline__ PhiS<T> phis(T a0, T a1, T a2) {
  PhiS<T> r;
  const T sg = vfmac(a0, -1.0f / 3.0f, a2);
  r.p = vfmac(a1, 0.5f, sg);
  r.m = vfmac(a1, -0.5f, sg);
  r.zn = vadd(sg, a0);
  return r;
}
template <class T>
__device__ __forceinline__ PhiS<T> phis_a2zero(T a0, T a1) {  // a2 = 0
  PhiS<T> r;
  const T sg = vmulc(a0, -1.0f / 3.0f);
  r.p = vfmac(a1, 0.5f, sg);
  r.m = vfmac(a1, -0.5f, sg);
  r.zn = vadd(sg, a0);
  return r;
}
template <class T>
__device__ __forceinline__ PhiS<T> phis_a1zero(T a0, T a2) {  // a1 = 0
  PhiS<T> r;
  r.p = r.m = vfmac(a0, -1.0f / 3.0f, a2);
  r.zn = vadd(r.p, a0);
  return r;
}
template <class T>
__device__ __forceinline__ PhiS<T> phis_a0only(T a0) {  // a1 = a2 = 0
  PhiS<T> r;
  r.p = r.m = vmulc(a0, -1.0f / 3.0f);
  r.zn = vadd(r.p, a0);
  return r;
}
// The first x slice takes drho = mu000 unscaled (a0 = -drho, folded in).
template <class T>
__device__ __forceinline__ PhiS<T> phis_drho(T drho, T a1, T a2) {
  PhiS<T> r;
  const T sg = vfmac(drho, 1.0f / 3.0f, a2);
  r.p = vfmac(a1, 0.5f, sg);
  r.m = vfmac(a1, -0.5f, sg);
  r.zn = vsub(sg, drho);
  return r;
}
template <class T>
__device__ __forceinline__ T projs0(T pl, T zn, T mr) { return vfmac(vadd(pl, mr), -0.5f, zn); }
template <class T>
__device__ __forceinline__ T projs1(T pl, T mr) { return vsub(pl, mr); }
template <class T>
__device__ __forceinline__ T projs2(T b0, T zn) { return vfmac(b0, -2.0f / 3.0f, zn); }

// App. A collision (as collide_moments) returning the scaled Hermite moments of
// the passes, A_pqr = s(p) s(q) s(r) mu_pqr, except A.m000, which holds
// drho = mu000 itself (phis_drho takes it).  With E = (1 - 1/tau) times the
// non-equilibrium stress after the trace reset, and the factors -2 u, 2 rho u
// and -4 E that the scaling asks for made once:
//   A_aa = rho u_a u_a + E_aa,  A_a = 2 rho u_a,  A_ab = (2 rho u_a)(-2 u_b) + (-4 E_ab),
//   A_aab = (-2 u_b) A_aa + u_a (-4 E_ab),  A_xyz = 8 (rho u u u + E u terms).
template <bool FORCE, class T>
__device__ __forceinline__ Mom17T<T> collide_scaled(const StoredT<T>& s, float omega, T fx, T fy,
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
  const T s3n = vmulc(vadd(vadd(mxx, myy), mzz), -om1 * (1.0f / 3.0f));
  T exx = vfmac(mxx, om1, s3n), eyy = vfmac(myy, om1, s3n), ezz = vfmac(mzz, om1, s3n);
  T exy = vmulc(mxy, -4.0f * om1), exz = vmulc(mxz, -4.0f * om1), eyz = vmulc(myz, -4.0f * om1);
  if (FORCE) {
    // E += -F F / (4 rho) (times -4 off the diagonal), u += F / (2 rho)
    const T q = vmulc(inv, -0.25f);
    exx = vfma(vmul(q, fx), fx, exx);
    eyy = vfma(vmul(q, fy), fy, eyy);
    ezz = vfma(vmul(q, fz), fz, ezz);
    exy = vfma(vmul(inv, fx), fy, exy);
    exz = vfma(vmul(inv, fx), fz, exz);
    eyz = vfma(vmul(inv, fy), fz, eyz);
    const T h = vmulc(inv, 0.5f);
    ux = vfma(h, fx, ux);
    uy = vfma(h, fy, uy);
    uz = vfma(h, fz, uz);
  }
  const T rux = vmul(rho, ux), ruy = vmul(rho, uy), ruz = vmul(rho, uz);
  Mom17T<T> A;
  A.m000 = s.drho;
  A.m200 = vfma(rux, ux, exx);
  A.m020 = vfma(ruy, uy, eyy);
  A.m002 = vfma(ruz, uz, ezz);
  A.m100 = vadd(rux, rux);
  A.m010 = vadd(ruy, ruy);
  A.m001 = vadd(ruz, ruz);
  const T uxn = vmulc(ux, -2.0f), uyn = vmulc(uy, -2.0f), uzn = vmulc(uz, -2.0f);
  A.m110 = vfma(A.m100, uyn, exy);
  A.m101 = vfma(A.m100, uzn, exz);
  A.m011 = vfma(A.m010, uzn, eyz);
  A.m210 = vfma(uyn, A.m200, vmul(ux, exy));  // xxy
  A.m120 = vfma(uxn, A.m020, vmul(uy, exy));  // xyy
  A.m201 = vfma(uzn, A.m200, vmul(ux, exz));  // xxz
  A.m102 = vfma(uxn, A.m002, vmul(uz, exz));  // xzz
  A.m021 = vfma(uzn, A.m020, vmul(uy, eyz));  // yyz
  A.m012 = vfma(uyn, A.m002, vmul(uz, eyz));  // yzz
  A.m111 = vfma(vmul(A.m100, uyn), uzn, vfma(exy, uzn, vfma(exz, uyn, vmul(eyz, uxn))));
#ifdef MELBM_HERMITE_XYZ_LITERAL
  A.m111 = vmulc(A.m111, 0.5f);  // the printed 1/(2 c_s^6) on xyz halves its moment
#endif
  return A;
}

// closure19 in the scaling of the passes (A.m000 = drho unscaled).
template <class T>
__device__ __forceinline__ Closure19T<T> closure19_scaled(const Mom17T<T>& A) {
  Closure19T<T> E;
  E.m220 = vmulc(A.m002, 1.0f / 6.0f);
  E.m202 = vmulc(A.m020, 1.0f / 6.0f);
  E.m022 = vmulc(A.m200, 1.0f / 6.0f);
  E.m211 = vmulc(A.m011, 1.0f / 3.0f);
  E.m121 = vmulc(A.m101, 1.0f / 3.0f);
  E.m112 = vmulc(A.m110, 1.0f / 3.0f);
  E.m221 = vfmac(A.m001, -1.0f / 9.0f, vmulc(vadd(A.m201, A.m021), 1.0f / 3.0f));
  E.m212 = vfmac(A.m010, -1.0f / 9.0f, vmulc(vadd(A.m210, A.m012), 1.0f / 3.0f));
  E.m122 = vfmac(A.m100, -1.0f / 9.0f, vmulc(vadd(A.m120, A.m102), 1.0f / 3.0f));
  E.m222 = vfmac(A.m000, -1.0f / 27.0f,
                 vmulc(vadd(vadd(A.m200, A.m020), A.m002), -1.0f / 18.0f));
  return E;
}

// x-pass populations of slice K (halo-buffer order: (q', r') = (0,0) (1,0) (2,0)
// (0,1) (1,1) (2,1) (0,2) (1,2), and (2,2) on D3Q19) from the scaled moments.
template <bool Q19, int K>
__device__ __forceinline__ PhiS<float2> xslice(const Mom17T<float2>& A, const Closure19T<float2>& E) {
  if constexpr (K == 0) return phis_drho(A.m000, A.m100, A.m200);
  else if constexpr (K == 1) return phis(A.m010, A.m110, A.m210);
  else if constexpr (K == 2) {
    if constexpr (Q19) return phis(A.m020, A.m120, E.m220);
    else return phis_a2zero(A.m020, A.m120);
  } else if constexpr (K == 3) return phis(A.m001, A.m101, A.m201);
  else if constexpr (K == 4) {
    if constexpr (Q19) return phis_a1zero(A.m011, E.m211);  // mu_111 = 0
    else return phis_a2zero(A.m011, A.m111);
  } else if constexpr (K == 5) {
    if constexpr (Q19) return phis(A.m021, E.m121, E.m221);
    else return phis_a0only(A.m021);
  } else if constexpr (K == 6) {
    if constexpr (Q19) return phis(A.m002, A.m102, E.m202);
    else return phis_a2zero(A.m002, A.m102);
  } else if constexpr (K == 7) {
    if constexpr (Q19) return phis(A.m012, E.m112, E.m212);
    else return phis_a0only(A.m012);
  } else {
    return phis(E.m022, E.m122, E.m222);
  }
}

// Stored variables from the scaled streamed moments M_pqr = s(p) s(q) s(r) m_pqr
// (finish_moments in that scaling).  The result holds -drho in .drho and
// -4 n_ab in .nxy, .nxz, .nyz; the encoders take the scale in their constants.
template <bool FORCE, class T>
__device__ __forceinline__ StoredT<T> finish_scaled(T M000, T M100, T M010, T M001, T M200, T M020,
                                                    T M002, T M110, T M101, T M011, T fx, T fy,
                                                    T fz) {
  StoredT<T> o;
  o.drho = M000;
  const T inv2 = vrcp(vfmac(M000, -2.0f, vset<T>(2.0f)));  // 1 / (2 rho')
  T jx = M100, jy = M010, jz = M001;                       // 2 rho' u'
  if (FORCE) {
    jx = vadd(jx, fx);
    jy = vadd(jy, fy);
    jz = vadd(jz, fz);
  }
  o.ux = vmul(jx, inv2);
  o.uy = vmul(jy, inv2);
  o.uz = vmul(jz, inv2);
  const T njx = vmulc(jx, -0.5f), njy = vmulc(jy, -0.5f), njz = vmulc(jz, -0.5f);  // exact
  o.nxx = vfma(njx, o.ux, M200);
  o.nyy = vfma(njy, o.uy, M020);
  o.nzz = vfma(njz, o.uz, M002);
  const T pjx = vadd(jx, jx), pjy = vadd(jy, jy);  // 4 rho' u'
  o.nxy = vfma(pjx, o.uy, M110);
  o.nxz = vfma(pjx, o.uz, M101);
  o.nyz = vfma(pjy, o.uz, M011);
  return o;
}

// ----------------------------------------------------------------- plane-pair I/O
template <int STORAGE> struct RawPair;
template <> struct RawPair<ST_Q16> { uint32_t a[5], b[5]; };
template <> struct RawPair<ST_F32> { float a[10], b[10]; };

// Word planes are addressed through per-plane base pointers held in the kernel
// parameters (uniform), so each access adds one per-thread offset (64-bit offsets
// for the FP32 planes, 32-bit cell offsets for the 16-bit ones).
using WordPlanes = const uint32_t* const*;

__device__ __forceinline__ void load_pair_w(RawPair<ST_Q16>& r, WordPlanes w, uint32_t na, uint32_t nb) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    r.a[k] = __ldg(w[k] + na);
    r.b[k] = __ldg(w[k] + nb);
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
__device__ __forceinline__ void store_pair_q16_w(uint32_t* const* w, uint32_t na, uint32_t nb,
                                                 const StoredT<float2>& o, bool sa, bool sb,
                                                 const DitherBits& ha, const DitherBits& hb,
                                                 const QGrids* q) {
  float2 d[10];  // 1 + the dither of each component
#pragma unroll
  for (int k = 0; k < 10; ++k) d[k] = dither_one_plus2(ha, hb, k);
  // o holds -drho and -4 n_ab (finish_scaled): their grid factors K carry
  // -1 and -1/4, power-of-two factors that leave every code unchanged
  uint2 e0, e1, e2, e3, e4, e5, e6, e7, e8, e9;
  if constexpr (RT) {
    e0 = qg_encode_codes1(q->g[0], o.drho, d[0], -1.0f), e1 = qg_encode_codes1(q->g[1], o.ux, d[1]);
    e2 = qg_encode_codes1(q->g[1], o.uy, d[2]), e3 = qg_encode_codes1(q->g[1], o.uz, d[3]);
    e4 = qg_encode_codes1(q->g[2], o.nxx, d[4]), e5 = qg_encode_codes1(q->g[2], o.nyy, d[5]);
    e6 = qg_encode_codes1(q->g[2], o.nzz, d[6]);
    e7 = qg_encode_codes1(q->g[2], o.nxy, d[7], -0.25f);
    e8 = qg_encode_codes1(q->g[2], o.nxz, d[8], -0.25f);
    e9 = qg_encode_codes1(q->g[2], o.nyz, d[9], -0.25f);
  } else {
    e0 = q_encode_codes1<0, -1>(o.drho, d[0]), e1 = q_encode_codes1<1>(o.ux, d[1]);
    e2 = q_encode_codes1<1>(o.uy, d[2]), e3 = q_encode_codes1<1>(o.uz, d[3]);
    e4 = q_encode_codes1<2>(o.nxx, d[4]), e5 = q_encode_codes1<2>(o.nyy, d[5]);
    e6 = q_encode_codes1<2>(o.nzz, d[6]), e7 = q_encode_codes1<2, -4>(o.nxy, d[7]);
    e8 = q_encode_codes1<2, -4>(o.nxz, d[8]), e9 = q_encode_codes1<2, -4>(o.nyz, d[9]);
  }
  if constexpr (RT) {
    const uint32_t qr = q->g[1].qmax, qs = q->g[2].qmax;
    if (sa) {
      w[0][na] = qg_clamp_word(q_pack(e0.x, e1.x), qr);
      w[1][na] = qg_clamp_word(q_pack(e2.x, e3.x), qr);
      w[2][na] = qg_clamp_word(q_pack(e4.x, e5.x), qs);
      w[3][na] = qg_clamp_word(q_pack(e6.x, e7.x), qs);
      w[4][na] = qg_clamp_word(q_pack(e8.x, e9.x), qs);
    }
    if (sb) {
      w[0][nb] = qg_clamp_word(q_pack(e0.y, e1.y), qr);
      w[1][nb] = qg_clamp_word(q_pack(e2.y, e3.y), qr);
      w[2][nb] = qg_clamp_word(q_pack(e4.y, e5.y), qs);
      w[3][nb] = qg_clamp_word(q_pack(e6.y, e7.y), qs);
      w[4][nb] = qg_clamp_word(q_pack(e8.y, e9.y), qs);
    }
  } else {
    if (sa) {
      w[0][na] = q_pack(e0.x, e1.x);
      w[1][na] = q_pack(e2.x, e3.x);
      w[2][na] = q_pack(e4.x, e5.x);
      w[3][na] = q_pack(e6.x, e7.x);
      w[4][na] = q_pack(e8.x, e9.x);
    }
    if (sb) {
      w[0][nb] = q_pack(e0.y, e1.y);
      w[1][nb] = q_pack(e2.y, e3.y);
      w[2][nb] = q_pack(e4.y, e5.y);
      w[3][nb] = q_pack(e6.y, e7.y);
      w[4][nb] = q_pack(e8.y, e9.y);
    }
  }
}

// Asynchronous global -> shared copies (cp.async, completed per thread): 4 bytes
// through L1, or 16 bytes (aligned) cached in L2 only.
__device__ __forceinline__ void cp_async4(uint32_t* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
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
#define MELBM_PRAGMA_STR(x) #x
#define MELBM_PRAGMA_UNROLL(n) _Pragma(MELBM_PRAGMA_STR(unroll n))

// mbarriers in shared memory (arrival counts of whole warps)
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(uint32_t(__cvta_generic_to_shared(b))),
               "r"(count)
               : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
// Wait for the phase of parity `par` to complete, polling at most 2^18 times
// (milliseconds; a wait of the kernel below lasts about one plane pair, a few
// microseconds).  When it runs out, *fault is set and the wait returns.
constexpr int MB_MAX_POLLS = 1 << 18;
__device__ __forceinline__ void mb_wait(uint32_t a, uint32_t par, uint32_t* fault) {
  for (int it = 0; it < MB_MAX_POLLS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(par)
        : "memory");
    if (done) return;
  }
  if (fault) *reinterpret_cast<volatile uint32_t*>(fault) = 1u;
}

template <int STORAGE, bool FORCE, bool RT, bool Q19 = false, bool BND = false>
__global__ void __launch_bounds__(FX* FY, MELBM_FLUID_MINB) fluid_kernel(KernelParams<STORAGE, RT> P) {
  // 16-bit storage on the 16/16 grids without the tables: the rows synchronise
  // through per-row barriers (measured faster there; the FP32 kernel, the kernel
  // with the tables and the runtime-grid kernel each ran slower with them)
  constexpr bool LOCAL_SYNC = STORAGE == ST_Q16 && !BND && !RT;
  // The y exchange of the FP32 kernel without the tables and without a force
  // moves slices r and r + 3 of a row as one 128-bit value (slice r + 6 as a
  // 64-bit one): 12 instead of 18 shared-memory accesses per thread and plane
  // pair, measured faster there (the 16-bit kernel with its row barriers and the
  // FP32 kernel with a force measured slower with it)
  constexpr bool YPAIR = STORAGE == ST_F32 && !BND && !FORCE;
  // one barrier per row and one of the whole block, in a set for the even and a
  // set for the odd barriers of the pair loop: a row can be one barrier ahead of
  // a row that waits on it, never two, so the phase parity of a set is unambiguous
  __shared__ uint64_t rowbar[LOCAL_SYNC ? 2 : 1][FY + 1];
  // the input side reads 16-bit codes in the mixed scheme (post-collision moments)
  constexpr int IN = STORAGE == ST_MIXED ? ST_Q16 : STORAGE;
  using HS = HaloStage<IN, FORCE, Q19, BND>;
  constexpr int NSXL = nsx<Q19>();
  constexpr int HALO_BUF = halo_buf<Q19>();
  auto decode = [&](const RawPair<IN>& r) {
    if constexpr (IN == ST_Q16 && RT) return decode_pair(r, P.q);
    else return decode_pair(r);
  };
  extern __shared__ __align__(16) float2 sm2[];
  float2* const hb = sm2 + 2 * SM_BUF;  // halo populations [buffer][row][slice][side]
  uint32_t* const stg = reinterpret_cast<uint32_t*>(hb + 2 * HALO_BUF);  // warp 0 staging
  // bounce-back record slots (BND): slot c of thread (row, lane) at [c][row][lane]
  float4* const recs = reinterpret_cast<float4*>(stg + 2 * HS::BUF_WORDS);
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
  const int hx = wrapi(side ? x0 + FX : x0 - 1, nx), hy = wrapi(y0 + hrow, ny);
  const size_t hcol = size_t(hx) + size_t(nx) * hy;

  // Solid cells (BND kernels) enter the passes with zero post-collision moments
  // about the rest state, so a FLUID_BOUNDARY cell receives nothing through its
  // solid links and the boundary kernel adds the bounced populations from the
  // cell's own state: apply_keep multiplies a pair's state and force by (1, 1)
  // for two fluid cells, with 0 in place of a solid one (0 * value is exactly 0).
  auto apply_keep = [&](StoredT<float2>& v, float2& fx, float2& fy, float2& fz, float2 k) {
    v.drho = vmul(v.drho, k);
    v.ux = vmul(v.ux, k);
    v.uy = vmul(v.uy, k);
    v.uz = vmul(v.uz, k);
    v.nxx = vmul(v.nxx, k);
    v.nyy = vmul(v.nyy, k);
    v.nzz = vmul(v.nzz, k);
    v.nxy = vmul(v.nxy, k);
    v.nxz = vmul(v.nxz, k);
    v.nyz = vmul(v.nyz, k);
    if (FORCE) {
      fx = vmul(fx, k);
      fy = vmul(fy, k);
      fz = vmul(fz, k);
    }
  };

  // z-march state of the six (p, q) slices: phi+ of the previous pair's two
  // planes and phi0 of its second plane
  float2 zP[6];
  float zZ[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    zP[k] = make_float2(0.f, 0.f);
    zZ[k] = 0.f;
  }

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
    if constexpr (BND) {
      const int e = 2 * HS::W + (FORCE ? 6 : 0);
      const uint32_t wh = uint32_t(hx >> 5) + uint32_t(P.ntx) * uint32_t(hy);
      const uint32_t rw = uint32_t(P.ntx) * uint32_t(ny);
      cp_async4(d + e * 32 * HS::CHUNK, P.cls_solid + wh + rw * uint32_t(wz(za)));
      cp_async4(d + (e + 1) * 32 * HS::CHUNK, P.cls_solid + wh + rw * uint32_t(wz(za + 1)));
    }
    cp_async_commit();
  };
  // Write the x-pass populations of the pair staged in buffer b (its copies have
  // completed) into halo buffer hbuf, laid out [row][slice] as
  // {phi+ of column x0-1, phi- of column x0+32}.
  auto halo_finish = [&](int b, int hbuf, int hz) {
    const uint32_t* d = stg + b * HS::BUF_WORDS + lane * HS::CHUNK + (chunk16 ? int(hcol & 3) : 0);
    RawPair<IN> hr;
#pragma unroll
    for (int w = 0; w < HS::W; ++w) {
      set_word<IN>(hr, 0, w, d[(2 * w) * 32 * HS::CHUNK]);
      set_word<IN>(hr, 1, w, d[(2 * w + 1) * 32 * HS::CHUNK]);
    }
    StoredT<float2> hs = decode(hr);
    (void)hz;
    float2 hfx = make_float2(0.f, 0.f), hfy = hfx, hfz = hfx;
    if (FORCE) {
      const float* sf = reinterpret_cast<const float*>(d) + 2 * HS::W * 32 * HS::CHUNK;
      hfx = make_float2(sf[0 * 32 * HS::CHUNK], sf[1 * 32 * HS::CHUNK]);
      hfy = make_float2(sf[2 * 32 * HS::CHUNK], sf[3 * 32 * HS::CHUNK]);
      hfz = make_float2(sf[4 * 32 * HS::CHUNK], sf[5 * 32 * HS::CHUNK]);
    }
    if constexpr (BND) {  // the staged solid words of the two planes
      const uint32_t* dw = stg + b * HS::BUF_WORDS + lane * HS::CHUNK +
                           (2 * HS::W + (FORCE ? 6 : 0)) * 32 * HS::CHUNK;
      const uint32_t sa = dw[0], sb = dw[32 * HS::CHUNK];
      apply_keep(hs, hfx, hfy, hfz,
                 make_float2(((sa >> (hx & 31)) & 1u) ? 0.f : 1.f, ((sb >> (hx & 31)) & 1u) ? 0.f : 1.f));
    }
    const Mom17T<float2> H = collide_scaled<FORCE>(hs, omega, hfx, hfy, hfz);
    Closure19T<float2> E;
    if constexpr (Q19) E = closure19_scaled(H);
    float2* dst = hb + hbuf * HALO_BUF + hrow * NSXL * 2 + side;
    auto put = [&](int k, const PhiS<float2>& ph) {
      if (halo_lane) dst[2 * k] = side ? ph.m : ph.p;
    };
    put(0, xslice<Q19, 0>(H, E));
    put(1, xslice<Q19, 1>(H, E));
    put(2, xslice<Q19, 2>(H, E));
    put(3, xslice<Q19, 3>(H, E));
    put(4, xslice<Q19, 4>(H, E));
    put(5, xslice<Q19, 5>(H, E));
    put(6, xslice<Q19, 6>(H, E));
    put(7, xslice<Q19, 7>(H, E));
    if constexpr (Q19) put(8, xslice<Q19, 8>(H, E));
  };

  RawPair<IN> raw;
  if constexpr (IN == ST_Q16)
    load_pair_w(raw, P.qin, uint32_t(col) + uint32_t(plane) * uint32_t(wz(z0 - 1)),
                uint32_t(col) + uint32_t(plane) * uint32_t(wz(z0)));
  else
    load_pair(raw, P.in_w, col + plane * wz(z0 - 1), col + plane * wz(z0));
  if (halo_warp) {
    halo_issue(z0 - 1, 0);
    if (z0 + 1 <= z1) {
      halo_issue(z0 + 1, 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    halo_finish(0, 0, z0 - 1);
  }
  if constexpr (LOCAL_SYNC) {
    if (row == 0 && lane < 2) {
      for (int r = 0; r < FY; ++r) mb_init(&rowbar[lane][r], (r == 0 && P.stall_test) ? 2 * FX : FX);
      mb_init(&rowbar[lane][FY], FX * FY);
    }
  }
  __syncthreads();
  // The i-th barrier of the pair loop after the first two (which stay block-wide):
  // a row waits for its two neighbour rows, whose y-exchange slots it reads and
  // overwrites next, and for warp 0, whose x-halo buffer it reads next; warp 0
  // waits for the whole block before it overwrites a halo buffer.
  const uint32_t rb0 = uint32_t(__cvta_generic_to_shared(&rowbar[0][0]));
  auto sync_rows = [&](int i) {
    if constexpr (LOCAL_SYNC) {
      const uint32_t b = rb0 + ((i & 1) ? uint32_t(8 * (FY + 1)) : 0u);
      const uint32_t par = uint32_t(i >> 1) & 1u;
      mb_arrive(b + 8u * row);
      mb_arrive(b + 8u * FY);
      if (row == 0) {
        mb_wait(b + 8u * FY, par, P.fault);
      } else {
        mb_wait(b + 8u * (row - 1), par, P.fault);
        if (row + 1 < FY) mb_wait(b + 8u * (row + 1), par, P.fault);
        if (row != 1) mb_wait(b, par, P.fault);
      }
    } else {
      (void)i;
      __syncthreads();
    }
  };

  const float2 zero = make_float2(0.f, 0.f);
  float2 yz0[NSY];  // phi_0 of the y pass of this thread's row, pair in flight

  // ---------------- pre(pair at zz): decode, prefetch the next pair (or re-read
  // this one when there is none), collide, x pass, y-pass populations -> buffer parity
  // BND: the solid words of the pair that pre() takes next (this lane's cells) and
  // the FLUID_BOUNDARY words of the output planes of the next two post() calls
  // (the tile's words), loaded one pair ahead like the state
  const uint32_t cls_rw = uint32_t(P.ntx) * uint32_t(ny);
  const uint32_t cls_own = uint32_t(xw >> 5) + uint32_t(P.ntx) * uint32_t(yw);
  const uint32_t cls_tile = uint32_t(blockIdx.x) + uint32_t(P.ntx) * uint32_t(yw);
  uint32_t sw0 = 0, sw1 = 0, fbA0 = 0, fbA1 = 0, fbB0 = 0, fbB1 = 0;
  // and the list index of the first listed cell of those FLUID_BOUNDARY words, also
  // a pair ahead: read where it is used, it stalled every warp holding such a cell
  // for a memory latency, and the block with it at the next barrier
  uint32_t pfA0 = 0, pfA1 = 0, pfB0 = 0, pfB1 = 0;
  if constexpr (BND) {
    sw0 = __ldg(P.cls_solid + cls_own + cls_rw * uint32_t(wz(z0 - 1)));
    sw1 = __ldg(P.cls_solid + cls_own + cls_rw * uint32_t(wz(z0)));
  }
  auto pre = [&](int zz, int parity, float2& fx, float2& fy, float2& fz, bool next) {
    StoredT<float2> s = decode(raw);
    fx = fy = fz = zero;
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
    {
      const int zn = next ? zz + 2 : zz;
      if constexpr (IN == ST_Q16)
        load_pair_w(raw, P.qin, uint32_t(col) + uint32_t(plane) * uint32_t(wz(zn)),
                    uint32_t(col) + uint32_t(plane) * uint32_t(wz(zn + 1)));
      else
        load_pair(raw, P.in_w, col + plane * wz(zn), col + plane * wz(zn + 1));
    }
    if constexpr (BND) {
      const float2 k = make_float2(((sw0 >> (xw & 31)) & 1u) ? 0.f : 1.f,
                                   ((sw1 >> (xw & 31)) & 1u) ? 0.f : 1.f);
      apply_keep(s, fx, fy, fz, k);
      fbA0 = fbB0;
      fbA1 = fbB1;
      sw0 = __ldg(P.cls_solid + cls_own + cls_rw * uint32_t(wz(zz + 2)));
      sw1 = __ldg(P.cls_solid + cls_own + cls_rw * uint32_t(wz(zz + 3)));
      fbB0 = __ldg(P.cls_fb + cls_tile + cls_rw * uint32_t(wz(zz + 1)));
      fbB1 = __ldg(P.cls_fb + cls_tile + cls_rw * uint32_t(wz(zz + 2)));
      pfA0 = pfB0;
      pfA1 = pfB1;
      pfB0 = __ldg(P.cls_pref + cls_tile + cls_rw * uint32_t(wz(zz + 1)));
      pfB1 = __ldg(P.cls_pref + cls_tile + cls_rw * uint32_t(wz(zz + 2)));
      // the bounce-back records of the pair the next post() stores (words fbA):
      // staged into this thread's slots now, added to the pulled sums there
      if (mid_row) {  // warp-uniform: only the stored rows (the halo warps' groups stay apart)
        const uint32_t lt = (1u << lane) - 1u;
        const float4* rec = reinterpret_cast<const float4*>(P.side);
        float4* slot = recs + row * FX + lane;
        constexpr int CS = FY * FX;  // slot stride
        if (col_ok && ((fbA0 >> lane) & 1u)) {
          const float4* r = rec + size_t(3) * (pfA0 + __popc(fbA0 & lt));
          cp_async16(slot, r);
          cp_async16(slot + CS, r + 1);
          cp_async8(slot + 4 * CS, r + 2);
        }
        if (col_ok && ((fbA1 >> lane) & 1u)) {
          const float4* r = rec + size_t(3) * (pfA1 + __popc(fbA1 & lt));
          cp_async16(slot + 2 * CS, r);
          cp_async16(slot + 3 * CS, r + 1);
          cp_async8(reinterpret_cast<float2*>(slot + 4 * CS) + 1, r + 2);
        }
        cp_async_commit();
      }
    }
    const Mom17T<float2> A = collide_scaled<FORCE>(s, omega, fx, fy, fz);
    Closure19T<float2> E;
    if constexpr (Q19) E = closure19_scaled(A);
    float2* sp = sm2 + parity * SM_BUF;
    // YPAIR layout: six float4 groups (phi+ of slices (r', r' + 3) at group r',
    // phi- at group 3 + r'), then six float2 groups (slice r' + 6)
    float4* const sp4 = reinterpret_cast<float4*>(sp);
    float2* const sp2 = sp + 12 * FY * FX;
    float2 X[3][3];  // X[p][q'] of the current r'
    const float4* hbp = reinterpret_cast<const float4*>(hb + parity * HALO_BUF) + row * NSXL;
#define MELBM_XPASS(K, Q)                                               \
  {                                                                     \
    const PhiS<float2> ph = xslice<Q19, K>(A, E);                       \
    const float4 h = hbp[K];                                            \
    float2 pl = shfl_idx2(ph.p, src_up);                                \
    float2 mr = shfl_idx2(ph.m, src_dn);                                \
    if (lane == 0) pl = make_float2(h.x, h.y);                          \
    if (lane == FX - 1) mr = make_float2(h.z, h.w);                     \
    X[0][Q] = projs0(pl, ph.zn, mr);                                    \
    X[1][Q] = projs1(pl, mr);                                           \
    X[2][Q] = projs2(X[0][Q], ph.zn);                                   \
  }
#define MELBM_YPHI(R, PH)                                                              \
  if constexpr (YPAIR) {                                                               \
    PhiS<float2> a_, b_, c_;                                                           \
    {                                                                                  \
      constexpr int p = 0;                                                             \
      a_ = PH;                                                                         \
    }                                                                                  \
    {                                                                                  \
      constexpr int p = 1;                                                             \
      b_ = PH;                                                                         \
    }                                                                                  \
    yz0[(R)] = a_.zn;                                                                  \
    yz0[3 + (R)] = b_.zn;                                                              \
    sp4[((R) * FY + row) * FX + lane] = make_float4(a_.p.x, a_.p.y, b_.p.x, b_.p.y);   \
    sp4[((3 + (R)) * FY + row) * FX + lane] = make_float4(a_.m.x, a_.m.y, b_.m.x, b_.m.y); \
    {                                                                                  \
      constexpr int p = 2;                                                             \
      c_ = PH;                                                                         \
    }                                                                                  \
    yz0[6 + (R)] = c_.zn;                                                              \
    sp2[((R) * FY + row) * FX + lane] = c_.p;                                          \
    sp2[((3 + (R)) * FY + row) * FX + lane] = c_.m;                                    \
  } else {                                                                             \
    _Pragma("unroll") for (int p = 0; p < 3; ++p) {                                    \
      const PhiS<float2> ph = PH;                                                      \
      const int s_ = 3 * p + (R);                                                      \
      sp[(s_ * FY + row) * FX + lane] = ph.p;                                          \
      sp[((NSY + s_) * FY + row) * FX + lane] = ph.m;                                  \
      yz0[s_] = ph.zn;                                                                 \
    }                                                                                  \
  }
    MELBM_XPASS(0, 0)  // r' = 0
    MELBM_XPASS(1, 1)
    MELBM_XPASS(2, 2)
    MELBM_YPHI(0, phis(X[p][0], X[p][1], X[p][2]))
    MELBM_XPASS(3, 0)  // r' = 1
    MELBM_XPASS(4, 1)
    MELBM_XPASS(5, 2)
    MELBM_YPHI(1, phis(X[p][0], X[p][1], X[p][2]))
    MELBM_XPASS(6, 0)  // r' = 2
    MELBM_XPASS(7, 1)
    if constexpr (Q19) {
      MELBM_XPASS(8, 2)
      MELBM_YPHI(2, phis(X[p][0], X[p][1], X[p][2]))
    } else {
      // (q', r') = (2, 2) carries no D3Q27 moment
      MELBM_YPHI(2, phis_a2zero(X[p][0], X[p][1]))
    }
#undef MELBM_XPASS
#undef MELBM_YPHI
  };

  // ---------------- post(pair at zz): y pass from buffer parity, z pass, and the
  // store of planes (zz - 1, zz) (skipped for the first pair of the chunk)
  auto post = [&](int zz, int parity, float2 ox, float2 oy, float2 oz, bool store) {
    const int za = zz - 1, zb = zz;
    // the dither of the two output planes first: integer work that does not
    // depend on the arithmetic below, so the scheduler can interleave the two
    DitherBits ha, hb2;
    if constexpr (STORAGE == ST_Q16) {
      if (store) {
        ha = pcg4d(uint32_t(xw), uint32_t(yw), uint32_t(za), P.t_out, P.seed);
        hb2 = pcg4d(uint32_t(xw), uint32_t(yw), uint32_t(zb), P.t_out, P.seed);
      }
    }
    const float2* sp = sm2 + parity * SM_BUF;
    float2 Y[3][3][3];
    if constexpr (YPAIR) {
      const float4* const sp4 = reinterpret_cast<const float4*>(sp);
      const float2* const sp2 = sp + 12 * FY * FX;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        // phi+ of the row above and phi- of the row below, slices r, r + 3, r + 6
        const float4 a = sp4[(r * FY + row - 1) * FX + lane];
        const float4 b = sp4[((3 + r) * FY + row + 1) * FX + lane];
        const float2 pls[3] = {make_float2(a.x, a.y), make_float2(a.z, a.w),
                               sp2[(r * FY + row - 1) * FX + lane]};
        const float2 mrs[3] = {make_float2(b.x, b.y), make_float2(b.z, b.w),
                               sp2[((3 + r) * FY + row + 1) * FX + lane]};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const int s_ = 3 * p + r;
          Y[p][0][r] = projs0(pls[p], yz0[s_], mrs[p]);
          if (p <= 1) Y[p][1][r] = projs1(pls[p], mrs[p]);
          if (p == 0) Y[p][2][r] = projs2(Y[p][0][r], yz0[s_]);
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int s_ = 3 * p + r;
          const float2 pl = sp[(s_ * FY + row - 1) * FX + lane];
          const float2 mr = sp[((NSY + s_) * FY + row + 1) * FX + lane];
          Y[p][0][r] = projs0(pl, yz0[s_], mr);
          if (p <= 1) Y[p][1][r] = projs1(pl, mr);
          if (p == 0) Y[p][2][r] = projs2(Y[p][0][r], yz0[s_]);
        }
    }
    // z pass: planes (zz, zz + 1) in, (zz - 1, zz) out; the Zn of the output
    // pair straddles two input pairs, so the terms that use it are taken per half
    const int PQ[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    float2 M[6][3];  // scaled streamed moments M_pqr of the output pair
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int p = PQ[k][0], q = PQ[k][1];
      const PhiS<float2> ph = phis(Y[p][q][0], Y[p][q][1], Y[p][q][2]);
      const float2 pl = zP[k];
      const float2 mr = ph.m;
      const float2 lr = vadd(pl, mr);
      M[k][0] = make_float2(__fmaf_rn(lr.x, -0.5f, zZ[k]), __fmaf_rn(lr.y, -0.5f, ph.zn.x));
      M[k][1] = projs1(pl, mr);
      M[k][2] = make_float2(__fmaf_rn(M[k][0].x, -2.0f / 3.0f, zZ[k]),
                            __fmaf_rn(M[k][0].y, -2.0f / 3.0f, ph.zn.x));
      zP[k] = ph.p;
      zZ[k] = ph.zn.y;
    }
    if (!store) return;
    if constexpr (BND) {
      // this pair's FLUID_BOUNDARY cells pulled nothing through their solid links:
      // add what those links return (the bounce kernel's records, staged by pre())
      const uint32_t fa = fbA0, fb = zb < z1 ? fbA1 : 0u;
      // warp-uniform (every lane read the same two words); wait for every copy
      // pre() issued, also those of a plane past the chunk that is not stored
      if ((fbA0 | fbA1) != 0u) cp_async_wait<0>();
      if ((fa | fb) != 0u) {
        const float4* slot = recs + row * FX + lane;
        constexpr int CS = FY * FX;
        if (col_ok && ((fa >> lane) & 1u)) {
          const float4 r0 = slot[0], r1 = slot[CS], r2 = slot[4 * CS];
          M[0][0].x += r0.x, M[1][0].x += r0.y, M[2][0].x += r0.z, M[0][1].x += r0.w;
          M[3][0].x += r1.x, M[5][0].x += r1.y, M[0][2].x += r1.z, M[4][0].x += r1.w;
          M[1][1].x += r2.x, M[2][1].x += r2.y;
        }
        if (col_ok && ((fb >> lane) & 1u)) {
          const float4 r0 = slot[2 * CS], r1 = slot[3 * CS], r2 = slot[4 * CS];
          M[0][0].y += r0.x, M[1][0].y += r0.y, M[2][0].y += r0.z, M[0][1].y += r0.w;
          M[3][0].y += r1.x, M[5][0].y += r1.y, M[0][2].y += r1.z, M[4][0].y += r1.w;
          M[1][1].y += r2.z, M[2][1].y += r2.w;
        }
      }
    }
    if constexpr (STORAGE == ST_MIXED) {
      StoredT<float2> r;  // the unscaled raw sums
      r.drho = vmulc(M[0][0], -1.0f), r.ux = vmulc(M[1][0], 0.5f), r.uy = vmulc(M[2][0], 0.5f);
      r.uz = vmulc(M[0][1], 0.5f);
      r.nxx = M[3][0], r.nyy = M[5][0], r.nzz = M[0][2];
      r.nxy = vmulc(M[4][0], -0.25f), r.nxz = vmulc(M[1][1], -0.25f), r.nyz = vmulc(M[2][1], -0.25f);
      store_pair_f32(P.out_w, col + plane * za, col + plane * (zb < nz ? zb : 0), r, col_ok,
                     col_ok && zb < z1);
      return;
    }
    StoredT<float2> o =  // -drho and -4 n_ab in place of drho and n_ab (finish_scaled)
        finish_scaled<FORCE>(M[0][0], M[1][0], M[2][0], M[0][1], M[3][0], M[5][0], M[0][2],
                             M[4][0], M[1][1], M[2][1], ox, oy, oz);
    if constexpr (STORAGE == ST_Q16)
      store_pair_q16_w<RT>(P.qout, uint32_t(col) + uint32_t(plane) * uint32_t(za),
                           uint32_t(col) + uint32_t(plane) * uint32_t(zb < nz ? zb : 0), o, col_ok,
                           col_ok && zb < z1, ha, hb2, grids_of(P));
    else {
      o.drho = vmulc(o.drho, -1.0f);
      o.nxy = vmulc(o.nxy, -0.25f);
      o.nxz = vmulc(o.nxz, -0.25f);
      o.nyz = vmulc(o.nyz, -0.25f);
      store_pair_f32(P.out_w, col + plane * za, col + plane * (zb < nz ? zb : 0), o, col_ok,
                     col_ok && zb < z1);
    }
  };

  // Pairs j = 0 .. npairs-1 at zz = z0 - 1 + 2 j.  The window of pair j runs
  // between the barriers of pairs j - 1 and j.
  const int npairs = (z1 - z0 + 1) / 2 + 1;
  if constexpr (IN == ST_F32) {
    // FP32 storage: pre(j), barrier, post(j) per pair, two pairs per loop trip
    // (twice the bytes of the 16-bit form are in flight; measured faster)
    float fprev[3] = {0.f, 0.f, 0.f};
    MELBM_PRAGMA_UNROLL(MELBM_FLUID_ZUNROLL)
    for (int j = 0; j < npairs; ++j) {
      const int zz = z0 - 1 + 2 * j;
      const int parity = j & 1;
      const bool halo_next = halo_warp && j + 1 < npairs;
      const bool halo_ahead = halo_warp && j + 2 < npairs;
      if (halo_ahead) halo_issue(zz + 4, parity);
      float2 f[3];
      pre(zz, parity, f[0], f[1], f[2], j + 1 < npairs);
      if (halo_next) {
        if (halo_ahead) cp_async_wait<1>();
        else cp_async_wait<0>();
        halo_finish(parity ^ 1, parity ^ 1, zz + 2);
      }
      __syncthreads();
      if (mid_row)
        post(zz, parity, make_float2(fprev[0], f[0].x), make_float2(fprev[1], f[1].x),
             make_float2(fprev[2], f[2].x), j > 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) fprev[k] = f[k].y;
    }
  } else if (mid_row) {
    // 16-bit input: window j holds post(j - 1) and pre(j) in one straight block,
    // so the codec's integer work and the passes' arithmetic of two pairs can be
    // interleaved by the scheduler (the y-halo rows run the loop below)
    float2 fc[3], fn[3];
    float fprev[3];
    pre(z0 - 1, 0, fc[0], fc[1], fc[2], npairs > 1);
    __syncthreads();
    post(z0 - 1, 0, zero, zero, zero, false);
#pragma unroll
    for (int k = 0; k < 3; ++k) fprev[k] = fc[k].y;
    pre(z0 + 1, 1, fc[0], fc[1], fc[2], npairs > 2);
    __syncthreads();
    int parity = 0;
    for (int j = 2; j < npairs; ++j, parity ^= 1) {
      const int zz = z0 - 1 + 2 * j;
      post(zz - 2, parity ^ 1, make_float2(fprev[0], fc[0].x), make_float2(fprev[1], fc[1].x),
           make_float2(fprev[2], fc[2].x), true);
#pragma unroll
      for (int k = 0; k < 3; ++k) fprev[k] = fc[k].y;
      pre(zz, parity, fn[0], fn[1], fn[2], j + 1 < npairs);
#pragma unroll
      for (int k = 0; k < 3; ++k) fc[k] = fn[k];
      sync_rows(j - 2);
    }
    post(z0 - 1 + 2 * (npairs - 1), (npairs - 1) & 1, make_float2(fprev[0], fc[0].x),
         make_float2(fprev[1], fc[1].x), make_float2(fprev[2], fc[2].x), true);
  } else {
    // y-halo rows: their x-pass populations only; warp 0 also stages and
    // computes the x halo of the next pair
    for (int j = 0; j < npairs; ++j) {
      const int zz = z0 - 1 + 2 * j;
      const int parity = j & 1;
      const bool halo_next = halo_warp && j + 1 < npairs;
      const bool halo_ahead = halo_warp && j + 2 < npairs;
      if (halo_ahead) halo_issue(zz + 4, parity);
      float2 f0, f1, f2;
      pre(zz, parity, f0, f1, f2, j + 1 < npairs);
      if (halo_next) {
        if (halo_ahead) cp_async_wait<1>();
        else cp_async_wait<0>();
        halo_finish(parity ^ 1, parity ^ 1, zz + 2);
      }
      if (j < 2) __syncthreads();
      else sync_rows(j - 2);
    }
  }
}

// z-chunk length: the even length (ZCHUNK = 256 down to 4) minimising the number of
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

template <int STORAGE, bool FORCE, bool RT, bool Q19 = false, bool BND = false>
cudaError_t launch_fluid_t(KernelParams<STORAGE, RT>& p, cudaStream_t st) {
  const size_t smem = HaloStage<STORAGE == ST_MIXED ? ST_Q16 : STORAGE, FORCE, Q19, BND>::SMEM;
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
    e = cudaFuncSetAttribute(fluid_kernel<STORAGE, FORCE, RT, Q19, BND>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_kernel<STORAGE, FORCE, RT, Q19, BND>,
                                                        FX * FY, smem);
    if (e != cudaSuccess) return e;
    resident[dev] = std::max(1, sms * per_sm);
  }
  const int64_t tiles_xy = int64_t((p.nx + FX - 1) / FX) * ((p.ny + FYI - 1) / FYI);
  p.zc = choose_zchunk(tiles_xy, p.nz, resident[dev]);
  dim3 grid((p.nx + FX - 1) / FX, (p.ny + FYI - 1) / FYI, (p.nz + p.zc - 1) / p.zc);
  fluid_kernel<STORAGE, FORCE, RT, Q19, BND><<<grid, dim3(FX, FY), smem, st>>>(p);
  return cudaGetLastError();
}

// Fill the parameters of one step and launch the instantiation for the storage,
// bit widths and force (Q19: the D3Q19 lattice; BND: with the boundary tables).
template <bool Q19, bool BND>
cudaError_t launch_fluid_impl(int storage, int nx, int ny, int nz, const void* in, void* out,
                              const float* force, float omega, uint32_t t_out, uint32_t seed,
                              const QGrids& grids, const BoundaryTables* bt, cudaStream_t st,
                              uint32_t* fault = nullptr, int stall_test = 0) {
  FluidParams p = {};
  p.fault = fault;
  p.stall_test = stall_test;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = in;
  p.out = out;
  p.force = force;
  p.omega = omega;
  p.t_out = t_out;
  p.seed = seed;
  // 16-byte chunks need 16-byte aligned rows: nx % 4 == 0 and aligned bases
  p.chunk16 = nx % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(force) % 16 == 0;
  const size_t N = size_t(nx) * ny * nz;
  for (int k = 0; k < 5; ++k) {
    p.qin[k] = static_cast<const uint32_t*>(in) + k * N;
    p.qout[k] = static_cast<uint32_t*>(out) + k * N;
  }
  if constexpr (BND) {
    p.cls_solid = bt->solid;
    p.cls_fb = bt->fb;
    p.cls_pref = bt->pref;
    p.side = bt->side;
    p.L = bt->L;
    p.ntx = (nx + 31) / 32;
  }
  if (storage == ST_Q16 && !qgrids_16(grids)) {
    KernelParams<ST_Q16, true> q;
    static_cast<FluidParams&>(q) = p;
    q.q = grids;
    return force ? launch_fluid_t<ST_Q16, true, true, Q19, BND>(q, st)
                 : launch_fluid_t<ST_Q16, false, true, Q19, BND>(q, st);
  }
  if (storage == ST_Q16) {
    KernelParams<ST_Q16, false> q;
    static_cast<FluidParams&>(q) = p;
    return force ? launch_fluid_t<ST_Q16, true, false, Q19, BND>(q, st)
                 : launch_fluid_t<ST_Q16, false, false, Q19, BND>(q, st);
  }
  if (storage != ST_F32) return cudaErrorInvalidValue;
  KernelParams<ST_F32, false> q;
  static_cast<FluidParams&>(q) = p;
  for (int k = 0; k < 10; ++k) {
    q.in_w[k] = static_cast<const uint32_t*>(in) + k * N;
    q.out_w[k] = static_cast<uint32_t*>(out) + k * N;
  }
  for (int k = 0; k < 3; ++k)
    q.f_w[k] = force ? reinterpret_cast<const uint32_t*>(force) + k * N : nullptr;
  return force ? launch_fluid_t<ST_F32, true, false, Q19, BND>(q, st)
               : launch_fluid_t<ST_F32, false, false, Q19, BND>(q, st);
}

// The fluid pass of the mixed-precision scheme: 16-bit post-collision moments
// (stored variables rho - 1, u+, rho (S+ - u+ u+)) in, raw FP32 post-streaming
// sums out.  The stored stress is already traceless, so the collision with
// omega = 0 only rebuilds the Hermite moments.
template <bool Q19>
cudaError_t launch_fluid_mixed_impl(int nx, int ny, int nz, const void* q_in, float* p_out,
                                    cudaStream_t st) {
  KernelParams<ST_MIXED, false> k;
  FluidParams& p = k;
  p = FluidParams{};
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.in = q_in;
  p.out = p_out;
  p.omega = 0.0f;
  const size_t N = size_t(nx) * ny * nz;
  for (int w = 0; w < 5; ++w) p.qin[w] = static_cast<const uint32_t*>(q_in) + w * N;
  for (int w = 0; w < 10; ++w) k.out_w[w] = reinterpret_cast<uint32_t*>(p_out) + w * N;
  return launch_fluid_t<ST_MIXED, false, false, Q19>(k, st);
}

}  // namespace melbm
