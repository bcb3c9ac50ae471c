// sources.cu -- the source set of the boundary update (split design, Sec. 4.2).
// A listed FLUID_BOUNDARY cell x needs the post-collision state (App. A) of its
// pull sources x - c_i over non-solid links and of itself (halfway bounce-back,
// f_i(x) = f+_{opp(i)}(x), for solid links).  Neighbouring listed cells share
// most of these sources, so the source cells are compacted once per
// classification (ascending linear index) and collided once per step:
//   setup  : mark the sources, compact them (count / scan / scatter, no
//            atomics), and give every listed cell the 27 slots of its sources;
//   phase A: collide every source once and evaluate its 27 post-collision
//            populations (the boundary kernel, phase B, then only gathers).
#include "melbm_device.cuh"
#include "melbm_launch.h"

namespace melbm {

constexpr int SRC_THREADS = 256;
constexpr int SRC_ROUNDS = 8;
constexpr int SRC_CHUNK = SRC_THREADS * SRC_ROUNDS;  // flags per block, consecutive

int64_t source_flag_blocks(int64_t N) { return (N + SRC_CHUNK - 1) / SRC_CHUNK; }

__global__ void mark_sources_kernel(int nx, int ny, int nz, const uint32_t* cells,
                                    const uint32_t* words, int64_t L, uint8_t* mark) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const uint32_t word = words[k];
  if ((word >> 27) != T_FLUID_BOUNDARY) return;
  const uint32_t n = cells[k];
  int x, y, z;
  cell_xyz(n, nx, ny, &x, &y, &z);
  mark[n] = 1;  // bounced links read the cell itself
#pragma unroll 1
  for (int i = 0; i < 27; ++i)
    if (!((word >> i) & 1u)) mark[pull_source(x, y, z, nx, ny, nz, i)] = 1;
}

__global__ void __launch_bounds__(SRC_THREADS) flag_count_kernel(const uint8_t* flag, int64_t N,
                                                                 uint32_t* block_counts) {
  const int64_t base = int64_t(blockIdx.x) * SRC_CHUNK;
  uint32_t cnt = 0;
  for (int r = 0; r < SRC_ROUNDS; ++r) {
    const int64_t n = base + int64_t(r) * SRC_THREADS + threadIdx.x;
    if (n < N && flag[n]) ++cnt;
  }
  __shared__ uint32_t warp_sum[SRC_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(FULL, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < SRC_THREADS / 32; ++w) s += warp_sum[w];
    block_counts[blockIdx.x] = s;
  }
}

// Flagged cells in ascending order: cells_out[pos] = n and slot_of[n] = pos.
__global__ void __launch_bounds__(SRC_THREADS) flag_scatter_kernel(const uint8_t* flag, int64_t N,
                                                                   const uint32_t* block_offsets,
                                                                   uint32_t* cells_out,
                                                                   uint32_t* slot_of) {
  const int64_t base = int64_t(blockIdx.x) * SRC_CHUNK;
  __shared__ uint32_t warp_cnt[SRC_THREADS / 32];
  uint32_t running = block_offsets[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = 0; r < SRC_ROUNDS; ++r) {
    const int64_t n = base + int64_t(r) * SRC_THREADS + threadIdx.x;
    const bool f = n < N && flag[n];
    const uint32_t ballot = __ballot_sync(FULL, f);
    if (lane == 0) warp_cnt[wid] = __popc(ballot);
    __syncthreads();
    uint32_t before = 0, round_total = 0;
    for (int w = 0; w < SRC_THREADS / 32; ++w) {
      if (w < wid) before += warp_cnt[w];
      round_total += warp_cnt[w];
    }
    if (f) {
      const uint32_t pos = running + before + __popc(ballot & ((1u << lane) - 1u));
      cells_out[pos] = uint32_t(n);
      slot_of[n] = pos;
    }
    running += round_total;
    __syncthreads();
  }
}

// table[i L + k]: slot of the source of direction i of listed cell k (the cell
// itself for a solid link); INFLOW entries are not read.
__global__ void source_table_kernel(int nx, int ny, int nz, const uint32_t* cells,
                                    const uint32_t* words, int64_t L, const uint32_t* slot_of,
                                    uint32_t* table) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const uint32_t word = words[k];
  if ((word >> 27) != T_FLUID_BOUNDARY) return;
  const uint32_t n = cells[k];
  int x, y, z;
  cell_xyz(n, nx, ny, &x, &y, &z);
  const uint32_t self = slot_of[n];
#pragma unroll 1
  for (int i = 0; i < 27; ++i)
    table[int64_t(i) * L + k] =
        ((word >> i) & 1u) ? self : slot_of[pull_source(x, y, z, nx, ny, nz, i)];
}

cudaError_t launch_source_setup_mark(int nx, int ny, int nz, const uint32_t* cells,
                                     const uint32_t* words, int64_t L, uint8_t* mark,
                                     uint32_t* block_counts, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  cudaError_t e = cudaMemsetAsync(mark, 0, size_t(N), st);
  if (e != cudaSuccess) return e;
  mark_sources_kernel<<<unsigned((L + 255) / 256), 256, 0, st>>>(nx, ny, nz, cells, words, L, mark);
  flag_count_kernel<<<unsigned(source_flag_blocks(N)), SRC_THREADS, 0, st>>>(mark, N, block_counts);
  return cudaGetLastError();
}

cudaError_t launch_source_setup_fill(int nx, int ny, int nz, const uint32_t* cells,
                                     const uint32_t* words, int64_t L, const uint8_t* mark,
                                     const uint32_t* block_offsets, uint32_t* src_cells,
                                     uint32_t* slot_of, uint32_t* table, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  flag_scatter_kernel<<<unsigned(source_flag_blocks(N)), SRC_THREADS, 0, st>>>(
      mark, N, block_offsets, src_cells, slot_of);
  source_table_kernel<<<unsigned((L + 255) / 256), 256, 0, st>>>(nx, ny, nz, cells, words, L,
                                                                 slot_of, table);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- phase A
// pop[i S + s] = f+_i / w_i - 1 at source cell src_cells[s] (App. A with its
// force, then the Hermite population of direction i).  D3Q19 (Q19): the 19
// directions with |c|^2 <= 2 and their own weights; the corner rows stay unused.
template <int STORAGE, bool FORCE, bool Q19>
__global__ void __launch_bounds__(256) source_collide_kernel(const void* in, size_t N,
                                                             const float* force, float omega,
                                                             const uint32_t* src_cells, int64_t S,
                                                             float* pop, QGrids q) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const uint32_t n = src_cells[s];
  float fx = 0.f, fy = 0.f, fz = 0.f;
  if (FORCE) {
    fx = __ldg(force + n);
    fy = __ldg(force + N + n);
    fz = __ldg(force + 2 * N + n);
  }
  const Mom17 A = collide_moments<FORCE>(load_stored<STORAGE>(in, N, n, q), omega, fx, fy, fz);
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    if (Q19 && !in_d3q19(cx, cy, cz)) continue;
    pop[int64_t(i) * S + s] = Q19 ? hermite_eval19(A, cx, cy, cz) : hermite_eval(A, cx, cy, cz);
  }
}

template <bool Q19>
static void launch_source_collide_t(int storage, size_t N, const void* in, const float* force,
                                    float omega, const uint32_t* src_cells, int64_t S, float* pop,
                                    const QGrids& q, cudaStream_t st) {
  const unsigned blocks = unsigned((S + 255) / 256);
  if (storage == ST_Q16) {
    if (force) source_collide_kernel<ST_Q16, true, Q19><<<blocks, 256, 0, st>>>(in, N, force, omega, src_cells, S, pop, q);
    else source_collide_kernel<ST_Q16, false, Q19><<<blocks, 256, 0, st>>>(in, N, force, omega, src_cells, S, pop, q);
  } else {
    if (force) source_collide_kernel<ST_F32, true, Q19><<<blocks, 256, 0, st>>>(in, N, force, omega, src_cells, S, pop, q);
    else source_collide_kernel<ST_F32, false, Q19><<<blocks, 256, 0, st>>>(in, N, force, omega, src_cells, S, pop, q);
  }
}

cudaError_t launch_source_collide(int storage, size_t N, const void* in, const float* force,
                                  float omega, const uint32_t* src_cells, int64_t S, float* pop,
                                  const QGrids& q, int lattice, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  if (lattice == 19)
    launch_source_collide_t<true>(storage, N, in, force, omega, src_cells, S, pop, q, st);
  else
    launch_source_collide_t<false>(storage, N, in, force, omega, src_cells, S, pop, q, st);
  return cudaGetLastError();
}

}  // namespace melbm
