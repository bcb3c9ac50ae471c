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
// Two passes with a scan of per-block counts in between (no atomics), so the list
// order is deterministic and bit-exact.
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr int CL_THREADS = 256;
constexpr int CL_ROUNDS = 8;
constexpr int CL_CHUNK = CL_THREADS * CL_ROUNDS;  // cells per block, consecutive

int64_t classify_blocks(int64_t N) { return (N + CL_CHUNK - 1) / CL_CHUNK; }

__device__ __forceinline__ uint32_t solid_links(const uint8_t* mask, int nx, int ny, int nz, int x,
                                                int y, int z) {
  uint32_t bits = 0;
#pragma unroll 1
  for (int i = 0; i < 27; ++i) {
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    const size_t s = size_t(wrapi(x - cx, nx)) +
                     size_t(nx) * (size_t(wrapi(y - cy, ny)) + size_t(ny) * wrapi(z - cz, nz));
    if (mask[s]) bits |= 1u << i;
  }
  return bits;
}

__device__ __forceinline__ uint8_t cell_type(const uint8_t* mask, int inflow, int outflow, int nx,
                                             int ny, int nz, size_t n, int x, int y, int z,
                                             uint32_t* links) {
  *links = 0;
  if (mask && mask[n]) return T_SOLID;
  const uint32_t bits = mask ? solid_links(mask, nx, ny, nz, x, y, z) : 0u;
  *links = bits;
  if (inflow && x == 0) return T_INFLOW;
  if (outflow && x == nx - 1 && nx >= 2 && !(mask && mask[n - 1])) return T_OUTFLOW;
  return bits ? T_FLUID_BOUNDARY : T_FLUID;
}

__device__ __forceinline__ bool listed(uint8_t t) { return t == T_INFLOW || t == T_FLUID_BOUNDARY; }

__global__ void __launch_bounds__(CL_THREADS) classify_count_kernel(int nx, int ny, int nz,
                                                                   const uint8_t* mask, int inflow,
                                                                   int outflow, uint8_t* type,
                                                                   uint32_t* block_counts) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t base = size_t(blockIdx.x) * CL_CHUNK;
  uint32_t cnt = 0;
  for (int r = 0; r < CL_ROUNDS; ++r) {
    const size_t n = base + size_t(r) * CL_THREADS + threadIdx.x;
    if (n >= N) break;
    const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
    uint32_t links;
    const uint8_t t = cell_type(mask, inflow, outflow, nx, ny, nz, n, x, y, z, &links);
    type[n] = t;
    cnt += listed(t) ? 1u : 0u;
  }
  __shared__ uint32_t warp_sum[CL_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(FULL, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < CL_THREADS / 32; ++w) s += warp_sum[w];
    block_counts[blockIdx.x] = s;
  }
}

cudaError_t launch_classify_count(int nx, int ny, int nz, const uint8_t* mask, int inflow,
                                  int outflow, uint8_t* type, uint32_t* block_counts,
                                  cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  classify_count_kernel<<<unsigned(classify_blocks(N)), CL_THREADS, 0, st>>>(
      nx, ny, nz, mask, inflow, outflow, type, block_counts);
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

__global__ void __launch_bounds__(CL_THREADS) classify_scatter_kernel(
    int nx, int ny, int nz, const uint8_t* mask, const uint8_t* type, const uint32_t* block_offsets,
    uint32_t* cells, uint32_t* words) {
  const size_t N = size_t(nx) * ny * nz;
  const size_t base = size_t(blockIdx.x) * CL_CHUNK;
  __shared__ uint32_t warp_cnt[CL_THREADS / 32];
  uint32_t running = block_offsets[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = 0; r < CL_ROUNDS; ++r) {
    const size_t n = base + size_t(r) * CL_THREADS + threadIdx.x;
    const bool in_range = n < N;
    const uint8_t t = in_range ? type[n] : T_SOLID;
    const bool f = in_range && listed(t);
    const uint32_t ballot = __ballot_sync(FULL, f);
    if (lane == 0) warp_cnt[wid] = __popc(ballot);
    __syncthreads();
    uint32_t before = 0, round_total = 0;
    for (int w = 0; w < CL_THREADS / 32; ++w) {
      if (w < wid) before += warp_cnt[w];
      round_total += warp_cnt[w];
    }
    if (f) {
      const uint32_t pos = running + before + __popc(ballot & ((1u << lane) - 1u));
      const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (size_t(nx) * ny));
      const uint32_t links = mask ? solid_links(mask, nx, ny, nz, x, y, z) : 0u;
      cells[pos] = uint32_t(n);
      words[pos] = (uint32_t(t) << 27) | links;
    }
    running += round_total;
    __syncthreads();
  }
}

cudaError_t launch_classify_scatter(int nx, int ny, int nz, const uint8_t* mask,
                                    const uint8_t* type, const uint32_t* block_offsets,
                                    uint32_t* cells, uint32_t* words, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  classify_scatter_kernel<<<unsigned(classify_blocks(N)), CL_THREADS, 0, st>>>(
      nx, ny, nz, mask, type, block_offsets, cells, words);
  return cudaGetLastError();
}

}  // namespace melbm
