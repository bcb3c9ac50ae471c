// melbm_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace melbm {

// Grid constants of one codec group for b-bit codes (Sec. 5.4 with the adaptive
// bit allocation of the quantization results: rho and u on b_rho_u bits, rho
// S^neq on b_S bits).  The same FP32 roundings of FP64 expressions as the
// compile-time 16-bit constants; qmax = 2^b - 1.
struct QGrid {
  float step, K, b, c, wlo, whi, magic, qc;
  uint32_t qmax;
};
struct QGrids {
  QGrid g[3];  // group 0 = rho - 1, 1 = velocity, 2 = rho S^neq
  int bits_ru, bits_s;
};
inline QGrids make_qgrids(int bits_ru, int bits_s) {
  const double lo[3] = {0.8 - 1.0, -0.4, -0.1}, hi[3] = {1.5 - 1.0, 0.4, 0.1};
  QGrids r;
  r.bits_ru = bits_ru;
  r.bits_s = bits_s;
  for (int G = 0; G < 3; ++G) {
    const double Q = double((1u << (G < 2 ? bits_ru : bits_s)) - 1u);
    const double t = (0.0 - lo[G]) * Q / (hi[G] - lo[G]);
    const double qcd = double(int64_t(t + 0.5));  // floor(t + 1/2), t > 0
    QGrid& g = r.g[G];
    g.step = float((hi[G] - lo[G]) / Q);
    g.K = float(Q / (hi[G] - lo[G]));
    g.b = float(t - qcd);
    g.c = float(lo[G] + qcd * (hi[G] - lo[G]) / Q);
    g.wlo = float(-qcd);
    g.whi = float(Q - qcd);
    g.magic = float(8388608.0 + qcd);  // 2^23 + qc
    g.qc = float(qcd);
    g.qmax = uint32_t(Q);
  }
  return r;
}
inline bool qgrids_16(const QGrids& g) { return g.bits_ru == 16 && g.bits_s == 16; }

// The classification of a handle with solids as the fluid kernel reads it: per
// 32-cell word (tx, y, z) of a row (word index tx + ntx (y + ny z), ntx =
// ceil(nx / 32), bit = x - 32 tx) the bits of its SOLID cells and of its
// FLUID_BOUNDARY cells, and pref = the list index of the word's first listed cell
// (the number of listed cells before the word, plus one if its lane-0 cell is an
// INFLOW cell, so that a FLUID_BOUNDARY lane's index is pref + the number of
// FLUID_BOUNDARY lanes below it); side[L][SIDE_FLOATS] is the table of the sums
// (m000, m100, m010, m001, m200, m020, m002, m110, m101, m011, then two pad floats)
// of the populations the solid links of each FLUID_BOUNDARY cell return (list
// order), each times the scale of the fluid kernel's passes (-1, 2, 2, 2, 1, 1, 1,
// -4, -4, -4): the bounce kernel writes them, the fluid kernel adds them to the
// sums it pulls.  One 48-byte record per cell, moved as three 16-byte pieces.
constexpr int SIDE_FLOATS = 12;
struct BoundaryTables {
  const uint32_t* solid;
  const uint32_t* fb;
  const uint32_t* pref;
  float* side;
  int64_t L;
};

// Fluid kernel over every cell: in -> out (storage layout of melbm_device.cuh).
// q: the grids of the handle's bit widths (16/16 runs the kernel instantiation
// with compile-time grid constants).  bt: the boundary tables (NULL or solid ==
// NULL without solids).  fault: a word of mapped host memory (device address, or
// NULL) that the 16-bit kernel without tables sets to 1 when one of its bounded
// barrier waits runs out; stall_test != 0 makes those waits run out (tests).
cudaError_t launch_fluid(int storage, int nx, int ny, int nz, const void* in, void* out,
                         const float* force, float omega, uint32_t t_out, uint32_t seed,
                         const QGrids& q, const BoundaryTables* bt, cudaStream_t st,
                         uint32_t* fault = nullptr, int stall_test = 0);
cudaError_t launch_fluid_bnd(int storage, int nx, int ny, int nz, const void* in, void* out,
                             const float* force, float omega, uint32_t t_out, uint32_t seed,
                             const QGrids& q, const BoundaryTables* bt, cudaStream_t st);
// The same on the D3Q19 lattice (fluid19.cu, fluid19_bnd.cu; F32 or Q16 storage).
cudaError_t launch_fluid19(int storage, int nx, int ny, int nz, const void* in, void* out,
                           const float* force, float omega, uint32_t t_out, uint32_t seed,
                           const QGrids& q, const BoundaryTables* bt, cudaStream_t st,
                           uint32_t* fault = nullptr, int stall_test = 0);
cudaError_t launch_fluid19_bnd(int storage, int nx, int ny, int nz, const void* in, void* out,
                               const float* force, float omega, uint32_t t_out, uint32_t seed,
                               const QGrids& q, const BoundaryTables* bt, cudaStream_t st);

// The mixed-precision scheme (mixed.cu): fluid pass Q -> P (fluid.cu), solid
// correction with atomicAdd into P, collision + quantisation P -> Q, and the
// public-state conversions of P.
cudaError_t launch_fluid_mixed(int nx, int ny, int nz, const void* q_in, float* p_out,
                               cudaStream_t st);
cudaError_t launch_fluid_mixed19(int nx, int ny, int nz, const void* q_in, float* p_out,
                                 cudaStream_t st);
cudaError_t launch_mixed_correct(int nx, int ny, int nz, const void* q, float* p,
                                 const uint32_t* cells, const uint32_t* words, int64_t count,
                                 const float inflow[4], int lattice, cudaStream_t st);
cudaError_t launch_mixed_collide_quantize(int nx, int ny, int nz, const float* p, void* q,
                                          float omega, uint32_t t, uint32_t seed, cudaStream_t st);
cudaError_t launch_mixed_set_state(int64_t N, const float* rho, const float* u, const float* S,
                                   float* p, cudaStream_t st);
cudaError_t launch_mixed_get_moments(int64_t N, const float* p, float* rho, float* u, float* S,
                                     cudaStream_t st);

// Bounce kernel over the list, before the fluid kernel with the boundary tables
// (reads in): every FLUID_BOUNDARY cell writes into its bt.side record the sums of
// the populations its solid links return (halfway bounce-back, or the moving wall
// with wall_model 1), computed from its own post-collision state, in the scaling
// of the fluid kernel's passes; the fluid kernel adds them before its store.  No-op
// without a side table (no solids).
cudaError_t launch_bounce(int storage, int nx, int ny, int nz, const void* in, const float* force,
                          float omega, const uint32_t* cells, const uint32_t* words, int64_t count,
                          const BoundaryTables& bt, const QGrids& q, int wall_model,
                          const uint8_t* mask, const float* bodies, int lattice, cudaStream_t st);
// After the fluid kernel: the INFLOW cells of face 0 (type[] from the
// classification) are reset to the inflow equilibrium (rho, ux, uy, uz).
cudaError_t launch_inflow(int storage, int nx, int ny, int nz, void* out, const uint8_t* type,
                          const float inflow[4], uint32_t t_out, uint32_t seed, const QGrids& q,
                          cudaStream_t st);

// Force and torque (about r0 of the body) the next step transfers to the solid
// cells of body `body` (0: every solid) by momentum exchange over the solid
// links of the listed cells; 6 doubles into out (device), fixed-order sums.
int solid_force_blocks();
cudaError_t launch_solid_force(int storage, int nx, int ny, int nz, const void* in,
                               const float* force, float omega, const uint32_t* cells,
                               const uint32_t* words, int64_t count, const QGrids& q,
                               int wall_model, const uint8_t* mask, const float* bodies, int body,
                               double* partials, double* out, int lattice, cudaStream_t st);

// Outflow copy on the plane x = nx-1 (cells typed OUTFLOW), in place on buf.
cudaError_t launch_outflow(int storage, int nx, int ny, int nz, void* buf, const uint8_t* type,
                           cudaStream_t st);

// Classification (classify.cu), by 32-cell row words (tx, y, z), ntx =
// ceil(nx / 32) words per row, word index tx + ntx (y + ny z), W of them:
// pack_mask packs the mask to one bit per cell (W words); pass 1 writes the types
// (N), the mask of listed cells of every word (lbits, W words), the number of
// listed cells of each block of words (classify_blocks of them) and, when solid_w
// is given, the SOLID and FLUID_BOUNDARY bits of every word; after an exclusive
// scan of the block counts, pass 2 writes the list in ascending n and, when pref_w
// is given, the list index of every word's first listed cell (see BoundaryTables).
// mbits NULL: no solids.
int64_t classify_words(int nx, int ny, int nz);
int64_t classify_blocks(int nx, int ny, int nz);
cudaError_t launch_pack_mask(const uint8_t* mask, int nx, int ny, int nz, uint32_t* bits,
                             cudaStream_t st);
cudaError_t launch_classify_count(int nx, int ny, int nz, const uint32_t* mbits, int inflow,
                                  int outflow, uint8_t* type, uint32_t* solid_w, uint32_t* fb_w,
                                  uint32_t* lbits, uint32_t* block_cnt, cudaStream_t st);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                  cudaStream_t st);
cudaError_t launch_classify_scatter(int nx, int ny, int nz, const uint32_t* mbits, int inflow,
                                    int outflow, const uint32_t* lbits, const uint32_t* block_off,
                                    uint32_t* cells, uint32_t* words, uint32_t* pref_w,
                                    cudaStream_t st);

// FP64 reductions: partial sums per block, then one block sums the partials in
// a fixed order.  out[0] = mass, out[1] = kinetic energy, out[2] = saturated codes.
int reduce_blocks();
cudaError_t launch_reduce(int storage, int64_t N, const void* buf, const uint8_t* type,
                          double* partials, double* out, const QGrids& q, cudaStream_t st);

// State conversions (public FP32 <-> stored) and the codec on caller buffers.
cudaError_t launch_set_state(int storage, int nx, int ny, int nz, const float* rho, const float* u,
                             const float* S, void* buf, uint32_t t, uint32_t seed, int det,
                             const QGrids& q, cudaStream_t st);
cudaError_t launch_rest_state(int storage, int nx, int ny, int nz, void* buf, uint32_t seed,
                              const QGrids& q, cudaStream_t st);
cudaError_t launch_get_moments(int storage, int64_t N, const void* buf, float* rho, float* u,
                               float* S, const QGrids& q, cudaStream_t st);
cudaError_t launch_q16_encode(const float* stored, int nx, int ny, int nz, uint32_t t,
                              uint32_t seed, int det, uint32_t* words, const QGrids& q,
                              cudaStream_t st);
cudaError_t launch_q16_decode(const uint32_t* words, int64_t N, float* stored, const QGrids& q,
                              cudaStream_t st);

}  // namespace melbm
