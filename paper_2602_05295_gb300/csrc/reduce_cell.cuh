// reduce_cell.cuh -- the per-cell terms of the FP64 conservation diagnostics,
// shared by melbm_reduce and the allocation-free reduction so that both sum the
// same values.  Per non-solid cell: rho - 1 as stored (FP32, exact in FP64), the
// kinetic energy rho |u|^2 / 2 evaluated in FP32 (about 1e-7 relative per term,
// rounding to nearest), and the number of 16-bit codes on a range limit.  The
// accumulation is FP64 (the counts integer), so only four of the ten stored
// values are decoded and two FP64 additions are spent per cell.
#pragma once

#include "melbm_device.cuh"

namespace melbm {

struct CellTerms {
  float drho, ke;
  uint32_t rails;
};

__device__ __forceinline__ uint32_t rail_count(uint32_t w, uint32_t qmax_lo, uint32_t qmax_hi) {
  const uint32_t lo = w & 0xFFFFu, hi = w >> 16;
  return (lo == 0u || lo == qmax_lo) + (hi == 0u || hi == qmax_hi);
}

// q: the grids of the bit widths (NULL: the compile-time 16-bit grids).
template <int STORAGE>
__device__ __forceinline__ CellTerms reduce_cell(const void* buf, size_t N, size_t n,
                                                 const QGrids* q) {
  CellTerms t;
  float ux, uy, uz;
  t.rails = 0;
  if constexpr (STORAGE == ST_MIXED) {  // raw post-streaming sums rho - 1, rho u
    const float* p = static_cast<const float*>(buf);
    t.drho = p[n];
    const float inv = 1.0f / (1.0f + t.drho);
    ux = p[N + n] * inv;
    uy = p[2 * N + n] * inv;
    uz = p[3 * N + n] * inv;
  } else if constexpr (STORAGE == ST_F32) {
    const float* p = static_cast<const float*>(buf);
    t.drho = p[n];
    ux = p[N + n];
    uy = p[2 * N + n];
    uz = p[3 * N + n];
  } else {
    const uint32_t* b = static_cast<const uint32_t*>(buf);
    uint32_t w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = b[size_t(k) * N + n];
    if (q) {
      t.drho = qg_decode(q->g[0], q_lo_magic(w[0]));
      ux = qg_decode(q->g[1], q_hi_magic(w[0]));
      uy = qg_decode(q->g[1], q_lo_magic(w[1]));
      uz = qg_decode(q->g[1], q_hi_magic(w[1]));
      const uint32_t qr = q->g[1].qmax, qs = q->g[2].qmax;  // rho and u share b_rho_u
      t.rails = rail_count(w[0], qr, qr) + rail_count(w[1], qr, qr) + rail_count(w[2], qs, qs) +
                rail_count(w[3], qs, qs) + rail_count(w[4], qs, qs);
    } else {
      t.drho = q_decode<0>(q_lo_magic(w[0]));
      ux = q_decode<1>(q_hi_magic(w[0]));
      uy = q_decode<1>(q_lo_magic(w[1]));
      uz = q_decode<1>(q_hi_magic(w[1]));
#pragma unroll
      for (int k = 0; k < 5; ++k) t.rails += rail_count(w[k], 0xFFFFu, 0xFFFFu);
    }
  }
  t.ke = 0.5f * (1.0f + t.drho) * (ux * ux + uy * uy + uz * uz);
  return t;
}

}  // namespace melbm
