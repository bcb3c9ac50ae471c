// classify.cu -- cell classification and boundary-list compaction, the analogue of
// the paper's surface-marking preprocessing (Sec. 4.2, "Accelerating solid
// intersection test"): instead of marking voxels that hold triangles, every cell
// gets a type and the cells that need the boundary kernel are compacted into a
// list in ascending linear index.
//   type: SOLID if mask; else INFLOW if inflow and x == 0; else OUTFLOW if outflow,
//         x == nx-1 and (nx-2, y, z) is not solid; else FLUID_BOUNDARY if some
//         x - c_i is solid (periodic wrap); else FLUID.
//   list: INFLOW and FLUID_BOUNDARY cells; word = (type << 27) | link mask, bit i
//         of the link mask set iff x - c_i is solid.
// The grid is walked by 32-cell row words (tx, y, z) -- cells x = 32 tx + lane of
// one row, the order of ascending n -- one warp per word: for each of the nine
// neighbour rows (y - c_y, z - c_z) a ballot of the lanes' mask bytes, with the
// two wrapped cells beside the word, gives every lane its three bits x + 1, x,
// x - 1 by one shift of a 34-bit window, so the 27-bit link mask takes nine row
// loads per cell and no division.  Two passes with a scan of per-block counts in
// between (no atomics), so the list order is deterministic and bit-exact; the
// same passes write the per-word tables of the fluid kernel with solids (the
// SOLID and FLUID_BOUNDARY bits, and the list index of the word's first listed
// cell).
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr int CL_WARPS = 8;                        // warps per block
constexpr int CL_WPW = 16;                         // consecutive words per warp
constexpr int CL_WORDS = CL_WARPS * CL_WPW;        // words per block

int64_t classify_words(int nx, int ny, int nz) { return int64_t((nx + 31) / 32) * ny * nz; }
int64_t classify_blocks(int nx, int ny, int nz) {
  return (classify_words(nx, ny, nz) + CL_WORDS - 1) / CL_WORDS;
}

__device__ __forceinline__ bool listed(uint8_t t) { return t == T_INFLOW || t == T_FLUID_BOUNDARY; }

// v wrapped into [0, n) for v in [-1, n + 32] (a loop only when n < 33).
__device__ __forceinline__ int wrap_near(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

// Type and link mask of lane `lane`'s cell x = 32 tx + lane in row (y, z) (the
// whole warp calls it; lanes with x >= nx get a copy of the wrapped cell and
// valid = false).
struct WordCell {
  bool valid;
  uint32_t n;
  uint8_t type;
  uint32_t links;
};
__device__ __forceinline__ WordCell word_cell(const uint8_t* __restrict__ mask, int nx, int ny,
                                              int nz, int tx, int y, int z, int lane, int inflow,
                                              int outflow) {
  WordCell c;
  const int x = 32 * tx + lane;
  c.valid = x < nx;
  const int xs = c.valid ? x : wrap_near(x, nx);
  const size_t rowc = size_t(nx) * (size_t(y) + size_t(ny) * z);
  c.n = uint32_t(rowc + xs);
  bool own = false, left = false;
  uint32_t links = 0;
  if (mask) {
    const int xl = wrap_near(32 * tx - 1, nx), xr = wrap_near(32 * tx + 32, nx);
    const int ys[3] = {y == ny - 1 ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};  // y - c_y
    const int zs[3] = {z == nz - 1 ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const uint8_t* row = mask + size_t(nx) * (size_t(ys[ky]) + size_t(ny) * zs[kz]);
        const uint32_t b = __ballot_sync(FULL, __ldg(row + xs) != 0);
        // window bit j = cell x0 + 32 - j (j = 0 .. 33): lane l reads x + 1, x, x - 1
        // at bits 31 - l .. 33 - l, i.e. c_x = -1, 0, 1
        const uint64_t win = (uint64_t(__ldg(row + xl) != 0) << 33) |
                             (uint64_t(__brev(b)) << 1) | uint64_t(__ldg(row + xr) != 0);
        const uint32_t f = uint32_t(win >> (31 - lane)) & 7u;
        links |= f << (3 * ky + 9 * kz);
        if (ky == 1 && kz == 1) {
          own = (f >> 1) & 1u;
          left = (f >> 2) & 1u;
        }
      }
  }
  if (own) {
    c.type = T_SOLID;
    links = 0;
  } else if (inflow && x == 0) {
    c.type = T_INFLOW;
  } else if (outflow && x == nx - 1 && nx >= 2 && !left) {
    c.type = T_OUTFLOW;
  } else {
    c.type = links ? T_FLUID_BOUNDARY : T_FLUID;
  }
  c.links = links;
  return c;
}

// (tx, y, z) of word w (32-bit divisions; W < 2^32), and the step to word w + 1.
__device__ __forceinline__ void word_coords(uint32_t w, int ntx, int ny, int* tx, int* y, int* z) {
  const uint32_t row = w / uint32_t(ntx);
  *tx = int(w - row * uint32_t(ntx));
  *z = int(row / uint32_t(ny));
  *y = int(row - uint32_t(*z) * uint32_t(ny));
}
__device__ __forceinline__ void next_word(int ntx, int ny, int* tx, int* y, int* z) {
  if (++*tx == ntx) {
    *tx = 0;
    if (++*y == ny) {
      *y = 0;
      ++*z;
    }
  }
}

// Pass 1: types, the SOLID / FLUID_BOUNDARY bits of each word (when solid_w is
// given) and the number of listed cells of each block of CL_WORDS words.
__global__ void __launch_bounds__(CL_WARPS * 32) classify_count_kernel(
    int nx, int ny, int nz, const uint8_t* mask, int inflow, int outflow, uint8_t* type,
    uint32_t* solid_w, uint32_t* fb_w, uint32_t* block_counts) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntx = (nx + 31) / 32;
  const int64_t W = int64_t(ntx) * ny * nz;
  const int64_t w0 = (int64_t(blockIdx.x) * CL_WARPS + warp) * CL_WPW;
  uint32_t cnt = 0;
  int tx = 0, y = 0, z = 0;
  if (w0 < W) word_coords(uint32_t(w0), ntx, ny, &tx, &y, &z);
  for (int k = 0; k < CL_WPW; ++k, next_word(ntx, ny, &tx, &y, &z)) {
    const int64_t w = w0 + k;
    if (w >= W) break;  // warp-uniform
    const WordCell c = word_cell(mask, nx, ny, nz, tx, y, z, lane, inflow, outflow);
    if (c.valid) type[c.n] = c.type;
    const uint32_t sb = __ballot_sync(FULL, c.valid && c.type == T_SOLID);
    const uint32_t fb = __ballot_sync(FULL, c.valid && c.type == T_FLUID_BOUNDARY);
    const uint32_t lb = __ballot_sync(FULL, c.valid && listed(c.type));
    if (solid_w && lane == 0) {
      solid_w[w] = sb;
      fb_w[w] = fb;
    }
    cnt += __popc(lb);
  }
  __shared__ uint32_t wc[CL_WARPS];
  if (lane == 0) wc[warp] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int v = 0; v < CL_WARPS; ++v) s += wc[v];
    block_counts[blockIdx.x] = s;
  }
}

cudaError_t launch_classify_count(int nx, int ny, int nz, const uint8_t* mask, int inflow,
                                  int outflow, uint8_t* type, uint32_t* solid_w, uint32_t* fb_w,
                                  uint32_t* block_counts, cudaStream_t st) {
  classify_count_kernel<<<unsigned(classify_blocks(nx, ny, nz)), CL_WARPS * 32, 0, st>>>(
      nx, ny, nz, mask, inflow, outflow, type, solid_w, fb_w, block_counts);
  return cudaGetLastError();
}

// Exclusive scan of n counts by one block of 1024 threads, tile by tile with a carry.
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const uint32_t* in, uint32_t* out,
                                                             int64_t n, uint32_t* total) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < n ? in[i] : 0u;
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint32_t wt = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, wt, o);
        if (lane >= o) wt += t;
      }
      warp_tot[lane] = wt;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t carry = carry_s;
    const uint32_t before = (wid ? warp_tot[wid - 1] : 0u) + inc - v;
    if (i < n) out[i] = carry + before;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry_s;
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                  cudaStream_t st) {
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(in, out, n, total);
  return cudaGetLastError();
}

// Pass 2: the list in ascending n (block offsets from the scan of pass 1's
// counts) and, when pref_w is given, the list index of each word's first listed
// cell after an INFLOW cell at its lane 0 (the FLUID_BOUNDARY lanes of the word
// then sit at pref + the number of FLUID_BOUNDARY lanes below them).
__global__ void __launch_bounds__(CL_WARPS * 32) classify_scatter_kernel(
    int nx, int ny, int nz, const uint8_t* mask, int inflow, int outflow, const uint8_t* type,
    const uint32_t* block_offsets, uint32_t* cells, uint32_t* words, uint32_t* pref_w) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntx = (nx + 31) / 32;
  const int64_t W = int64_t(ntx) * ny * nz;
  const int64_t w0 = (int64_t(blockIdx.x) * CL_WARPS + warp) * CL_WPW;
  const uint32_t lt = (1u << lane) - 1u;
  // listed cells of this warp's words, from the types of pass 1
  uint32_t cnt = 0;
  int tx0 = 0, y0 = 0, z0 = 0;
  if (w0 < W) word_coords(uint32_t(w0), ntx, ny, &tx0, &y0, &z0);
  int tx = tx0, y = y0, z = z0;
  for (int k = 0; k < CL_WPW; ++k, next_word(ntx, ny, &tx, &y, &z)) {
    const int64_t w = w0 + k;
    if (w >= W) break;
    const int x = 32 * tx + lane;
    const uint8_t t = x < nx ? type[size_t(nx) * (size_t(y) + size_t(ny) * z) + x] : uint8_t(T_SOLID);
    cnt += __popc(__ballot_sync(FULL, listed(t)));
  }
  __shared__ uint32_t wc[CL_WARPS];
  if (lane == 0) wc[warp] = cnt;
  __syncthreads();
  uint32_t running = block_offsets[blockIdx.x];
  for (int v = 0; v < warp; ++v) running += wc[v];
  tx = tx0, y = y0, z = z0;
  for (int k = 0; k < CL_WPW; ++k, next_word(ntx, ny, &tx, &y, &z)) {
    const int64_t w = w0 + k;
    if (w >= W) break;
    const int x = 32 * tx + lane;
    const size_t n = size_t(nx) * (size_t(y) + size_t(ny) * z) + (x < nx ? x : 0);
    const uint8_t t = x < nx ? type[n] : uint8_t(T_SOLID);
    const uint32_t lb = __ballot_sync(FULL, listed(t));
    if (pref_w && lane == 0) {
      const bool in0 = lb & 1u && t == T_INFLOW;  // lane 0's own type
      pref_w[w] = running + (in0 ? 1u : 0u);
    }
    if (lb) {  // warp-uniform
      const WordCell c = word_cell(mask, nx, ny, nz, tx, y, z, lane, inflow, outflow);
      if ((lb >> lane) & 1u) {
        const uint32_t pos = running + __popc(lb & lt);
        cells[pos] = c.n;
        words[pos] = (uint32_t(c.type) << 27) | c.links;
      }
    }
    running += __popc(lb);
  }
}

cudaError_t launch_classify_scatter(int nx, int ny, int nz, const uint8_t* mask, int inflow,
                                    int outflow, const uint8_t* type, const uint32_t* block_offsets,
                                    uint32_t* cells, uint32_t* words, uint32_t* pref_w,
                                    cudaStream_t st) {
  classify_scatter_kernel<<<unsigned(classify_blocks(nx, ny, nz)), CL_WARPS * 32, 0, st>>>(
      nx, ny, nz, mask, inflow, outflow, type, block_offsets, cells, words, pref_w);
  return cudaGetLastError();
}

}  // namespace melbm
