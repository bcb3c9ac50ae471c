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
// The work is done on 32-cell row words (tx, y, z) -- cells x = 32 tx + j, j =
// 0 .. 31, of one row -- with the mask packed to one bit per cell first.  For a
// word and each of its nine neighbour rows (y - c_y, z - c_z), the row's words
// tx - 1, tx, tx + 1 (wrapped within the row) give by one shift each the three
// bit-planes "x - c_i is solid" of the 32 cells (c_x = -1, 0, 1), so a thread
// holds the 27 link planes of its word and types all 32 cells with bit
// operations.  Pass 1 writes the types, the per-word tables of the fluid kernel
// with solids (the SOLID and FLUID_BOUNDARY bits), the mask of listed cells of
// every word and the number of listed cells of every block of words; after an
// exclusive scan of the block counts, pass 2 ranks the words of a block by a block
// scan, writes the list index of every word's first listed cell, and has each
// word with listed cells rebuild its planes and write its cells in ascending n.
// No atomics: the list is bit-exact.
#include <algorithm>

#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr int CL_T = 256;  // threads (words) per block of the two passes

int64_t classify_words(int nx, int ny, int nz) { return int64_t((nx + 31) / 32) * ny * nz; }
int64_t classify_blocks(int nx, int ny, int nz) {
  return (classify_words(nx, ny, nz) + CL_T - 1) / CL_T;
}

__device__ __forceinline__ uint32_t valid_bits(int nv) { return nv >= 32 ? ~0u : (1u << nv) - 1u; }

// Pack: bit j of word (tx, row) = mask of cell 32 tx + j of the row (zero past nx).
// One warp per row and group of eight words, one ballot per word.
__global__ void __launch_bounds__(256) pack_mask_kernel(const uint8_t* __restrict__ mask, int nx,
                                                        int64_t rows, uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x & 31;
  const int64_t row = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
  if (row >= rows) return;
  const int ntx = (nx + 31) / 32;
  const int tx0 = int(blockIdx.y) * 8;
  const uint8_t* r = mask + row * nx;
  uint32_t mine = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int x = 32 * (tx0 + k) + lane;
    const uint32_t b = __ballot_sync(FULL, x < nx && __ldg(r + x) != 0);
    if (lane == k) mine = b;
  }
  if (lane < 8 && tx0 + lane < ntx) bits[row * ntx + tx0 + lane] = mine;
}

// The 27 link planes of word (tx, y, z): bit j of B[i] is set iff the neighbour
// x - c_i of cell x = 32 tx + j is solid (periodic), i = (c_x + 1) + 3 (c_y + 1)
// + 9 (c_z + 1).  The cell after the row's last cell is its cell 0 and the cell
// before cell 0 its last one, also when the last word is partial.
__device__ __forceinline__ void link_planes(const uint32_t* __restrict__ mb, int nx, int ny, int nz,
                                            int ntx, int tx, int y, int z, uint32_t B[27]) {
  const int txl = tx == 0 ? ntx - 1 : tx - 1, txr = tx == ntx - 1 ? 0 : tx + 1;
  const int nv = min(32, nx - 32 * tx), nvl = min(32, nx - 32 * txl);
  const uint32_t vm = valid_bits(nv);
#pragma unroll
  for (int kz = 0; kz < 3; ++kz) {
    const int zz = kz == 0 ? (z == nz - 1 ? 0 : z + 1) : kz == 1 ? z : (z == 0 ? nz - 1 : z - 1);
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int yy = ky == 0 ? (y == ny - 1 ? 0 : y + 1) : ky == 1 ? y : (y == 0 ? ny - 1 : y - 1);
      const uint32_t* r = mb + (size_t(yy) + size_t(ny) * zz) * ntx;
      const uint32_t wc = __ldg(r + tx), wl = __ldg(r + txl), wr = __ldg(r + txr);
      B[3 * ky + 9 * kz] = ((wc >> 1) | ((wr & 1u) << (nv - 1))) & vm;      // c_x = -1: x + 1
      B[3 * ky + 9 * kz + 1] = wc;                                          // c_x = 0
      B[3 * ky + 9 * kz + 2] = ((wc << 1) | ((wl >> (nvl - 1)) & 1u)) & vm;  // c_x = +1: x - 1
    }
  }
}

// Per-cell type bits of a word from its planes (disjoint masks within the valid bits).
struct WordTypes {
  uint32_t solid, inflow, outflow, fb, valid;
};
__device__ __forceinline__ WordTypes word_types(const uint32_t B[27], int nx, int ntx, int tx,
                                                int inflow, int outflow) {
  WordTypes t;
  const int nv = min(32, nx - 32 * tx);
  t.valid = valid_bits(nv);
  t.solid = B[13];                    // the cell itself
  const uint32_t left = B[14];        // x - 1 (same row)
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < 27; ++i) any |= B[i];
  t.inflow = (inflow && tx == 0) ? (1u & ~t.solid) : 0u;
  t.outflow = (outflow && nx >= 2 && tx == ntx - 1) ? ((1u << (nv - 1)) & ~t.solid & ~left) : 0u;
  t.fb = any & ~t.solid & ~t.inflow & ~t.outflow & t.valid;
  return t;
}

// Bytes of four cells 4 g .. 4 g + 3 of a word from its type masks.
__device__ __forceinline__ uint32_t spread4(uint32_t m, int g) {
  return (((m >> (4 * g)) & 15u) * 0x00204081u) & 0x01010101u;
}
__device__ __forceinline__ uint32_t type_bytes(const WordTypes& t, int g) {
  return 4u * spread4(t.solid, g) + 2u * spread4(t.inflow, g) + 3u * spread4(t.outflow, g) +
         spread4(t.fb, g);
}

struct ClassifyArgs {
  int nx, ny, nz;
  const uint32_t* mbits;  // packed mask, null: no solids
  int inflow, outflow;
  uint8_t* type;
  uint32_t* solid_w;  // null: no word tables
  uint32_t* fb_w;
  uint32_t* pref_w;
  uint32_t* lbits;        // listed cells of every word
  uint32_t* block_cnt;    // pass 1 out: listed cells per block of CL_T words
  const uint32_t* block_off;  // pass 2 in: their exclusive scan
  uint32_t* cells;
  uint32_t* words;
};

__device__ __forceinline__ void word_coords(int64_t w, int ntx, int ny, int* tx, int* y, int* z) {
  const int64_t row = w / ntx;
  *tx = int(w - row * ntx);
  *z = int(row / ny);
  *y = int(row - int64_t(*z) * ny);
}

// Pass 1: one thread per word.
__global__ void __launch_bounds__(CL_T) classify_types_kernel(const __grid_constant__ ClassifyArgs A) {
  const int nx = A.nx, ny = A.ny, nz = A.nz, ntx = (nx + 31) / 32;
  const int64_t W = int64_t(ntx) * ny * nz;
  const int64_t w = int64_t(blockIdx.x) * CL_T + threadIdx.x;
  uint32_t cnt = 0;
  if (w < W) {
    int tx, y, z;
    word_coords(w, ntx, ny, &tx, &y, &z);
    uint32_t B[27];
    if (A.mbits) {
      link_planes(A.mbits, nx, ny, nz, ntx, tx, y, z, B);
    } else {
#pragma unroll
      for (int i = 0; i < 27; ++i) B[i] = 0u;
    }
    const WordTypes t = word_types(B, nx, ntx, tx, A.inflow, A.outflow);
    const uint32_t lb = t.fb | t.inflow;
    A.lbits[w] = lb;
    if (A.solid_w) {
      A.solid_w[w] = t.solid;
      A.fb_w[w] = t.fb;
    }
    cnt = __popc(lb);
    uint8_t* out = A.type + (size_t(y) + size_t(ny) * z) * nx + 32 * tx;
    if ((nx & 15) == 0) {  // 16-byte aligned words of 16 or 32 cells
      uint4* o = reinterpret_cast<uint4*>(out);
      o[0] = make_uint4(type_bytes(t, 0), type_bytes(t, 1), type_bytes(t, 2), type_bytes(t, 3));
      if (nx - 32 * tx >= 32)
        o[1] = make_uint4(type_bytes(t, 4), type_bytes(t, 5), type_bytes(t, 6), type_bytes(t, 7));
    } else {
      const int nv = min(32, nx - 32 * tx);
      for (int j = 0; j < nv; ++j) out[j] = uint8_t(type_bytes(t, j >> 2) >> (8 * (j & 3)));
    }
  }
  // block sum
  __shared__ uint32_t ws[CL_T / 32];
  cnt = __reduce_add_sync(FULL, cnt);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < CL_T / 32; ++k) s += ws[k];
    A.block_cnt[blockIdx.x] = s;
  }
}

// Pass 2: one thread per word; the block's words are ranked by a block scan.
__global__ void __launch_bounds__(CL_T) classify_list_kernel(const __grid_constant__ ClassifyArgs A) {
  const int nx = A.nx, ny = A.ny, nz = A.nz, ntx = (nx + 31) / 32;
  const int64_t W = int64_t(ntx) * ny * nz;
  const int64_t w = int64_t(blockIdx.x) * CL_T + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lb = w < W ? A.lbits[w] : 0u;
  const uint32_t c = __popc(lb);
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += v;
  }
  __shared__ uint32_t ws[CL_T / 32];
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  uint32_t before = A.block_off[blockIdx.x];
  for (int k = 0; k < wid; ++k) before += ws[k];
  const uint32_t pos0 = before + inc - c;  // list index of the word's first listed cell
  if (w >= W) return;
  int tx, y, z;
  word_coords(w, ntx, ny, &tx, &y, &z);
  if (A.pref_w) A.pref_w[w] = pos0 + ((A.inflow && tx == 0 && (lb & 1u)) ? 1u : 0u);
  if (!lb) return;
  uint32_t B[27];
  if (A.mbits) {
    link_planes(A.mbits, nx, ny, nz, ntx, tx, y, z, B);
  } else {
#pragma unroll
    for (int i = 0; i < 27; ++i) B[i] = 0u;
  }
  const uint32_t n0 = uint32_t((size_t(y) + size_t(ny) * z) * nx + 32 * tx);  // N < 2^31
  uint32_t pos = pos0;
  for (uint32_t m = lb; m; m &= m - 1u, ++pos) {
    const int j = __ffs(m) - 1;
    uint32_t links = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) links |= ((B[i] >> j) & 1u) << i;
    const uint32_t type = (A.inflow && tx == 0 && j == 0) ? T_INFLOW : T_FLUID_BOUNDARY;
    A.cells[pos] = n0 + uint32_t(j);
    A.words[pos] = (type << 27) | links;
  }
}

cudaError_t launch_pack_mask(const uint8_t* mask, int nx, int ny, int nz, uint32_t* bits,
                             cudaStream_t st) {
  const int64_t rows = int64_t(ny) * nz;
  const dim3 grid(unsigned((rows + 7) / 8), unsigned(((nx + 31) / 32 + 7) / 8));
  pack_mask_kernel<<<grid, 256, 0, st>>>(mask, nx, rows, bits);
  return cudaGetLastError();
}

cudaError_t launch_classify_count(int nx, int ny, int nz, const uint32_t* mbits, int inflow,
                                  int outflow, uint8_t* type, uint32_t* solid_w, uint32_t* fb_w,
                                  uint32_t* lbits, uint32_t* block_cnt, cudaStream_t st) {
  ClassifyArgs a = {};
  a.nx = nx, a.ny = ny, a.nz = nz;
  a.mbits = mbits, a.inflow = inflow, a.outflow = outflow;
  a.type = type, a.solid_w = solid_w, a.fb_w = fb_w, a.lbits = lbits, a.block_cnt = block_cnt;
  classify_types_kernel<<<unsigned(classify_blocks(nx, ny, nz)), CL_T, 0, st>>>(a);
  return cudaGetLastError();
}

// Exclusive scan of n counts by one block of 1024 threads: each thread sums a
// contiguous run of ceil(n / 1024) entries, the run sums are scanned across the
// block, and each thread writes its run's prefixes.
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(const uint32_t* in, uint32_t* out,
                                                             int64_t n, uint32_t* total) {
  __shared__ uint32_t warp_tot[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int64_t per = (n + 1023) / 1024;
  const int64_t b0 = int64_t(t) * per, b = b0 < n ? b0 : n, e = b + per < n ? b + per : n;
  uint32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += in[i];
  uint32_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t wt = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULL, wt, o);
      if (lane >= o) wt += v;
    }
    warp_tot[lane] = wt;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (wid ? warp_tot[wid - 1] : 0u) + inc - s;
  for (int64_t i = b; i < e; ++i) {
    const uint32_t v = in[i];
    out[i] = run;
    run += v;
  }
  if (t == 1023) *total = warp_tot[31];
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                  cudaStream_t st) {
  exclusive_scan_kernel<<<1, 1024, 0, st>>>(in, out, n, total);
  return cudaGetLastError();
}

cudaError_t launch_classify_scatter(int nx, int ny, int nz, const uint32_t* mbits, int inflow,
                                    int outflow, const uint32_t* lbits, const uint32_t* block_off,
                                    uint32_t* cells, uint32_t* words, uint32_t* pref_w,
                                    cudaStream_t st) {
  ClassifyArgs a = {};
  a.nx = nx, a.ny = ny, a.nz = nz;
  a.mbits = mbits, a.inflow = inflow, a.outflow = outflow;
  a.lbits = const_cast<uint32_t*>(lbits), a.block_off = block_off;
  a.cells = cells, a.words = words, a.pref_w = pref_w;
  classify_list_kernel<<<unsigned(classify_blocks(nx, ny, nz)), CL_T, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace melbm
