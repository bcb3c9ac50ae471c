// sources.cu -- the source set of the boundary update (split design, Sec. 4.2).
// A listed FLUID_BOUNDARY cell x needs the post-collision state (App. A) of its
// pull sources x - c_i over non-solid links and of itself (halfway bounce-back,
// f_i(x) = f+_{opp(i)}(x), for solid links).  Neighbouring listed cells share
// most of these sources, so the source cells are compacted once per
// classification (ascending linear index) and collided once per step:
//   setup  : mark the sources, compact them (count / scan / scatter, no
//            atomics), and map every FLUID_BOUNDARY cell to its list index;
//   phase A: collide every source s once and push each population that a listed
//            cell reads into that cell's row: f+_i(s) to direction i of the
//            listed cell s + c_i, and, when s is itself listed, f+_{opp(i)}(s) to
//            each of its solid links i.  Every (direction, listed cell) entry of
//            a FLUID_BOUNDARY cell has exactly one writer (sources are never
//            solid, so s + c_i pulls from s through a non-solid link), and the
//            boundary kernel, phase B, reads its 27 entries contiguously.
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

// Flagged cells in ascending order: cells_out[pos] = n.
__global__ void __launch_bounds__(SRC_THREADS) flag_scatter_kernel(const uint8_t* flag, int64_t N,
                                                                   const uint32_t* block_offsets,
                                                                   uint32_t* cells_out) {
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
    }
    running += round_total;
    __syncthreads();
  }
}

// lidx[n] = k for the listed FLUID_BOUNDARY cell n = cells[k] (0xFFFFFFFF
// everywhere else, set by the caller).
__global__ void list_index_kernel(const uint32_t* cells, const uint32_t* words, int64_t L,
                                  uint32_t* lidx) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L) return;
  if ((words[k] >> 27) != T_FLUID_BOUNDARY) return;
  lidx[cells[k]] = uint32_t(k);
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
                                     uint32_t* lidx, cudaStream_t st) {
  const int64_t N = int64_t(nx) * ny * nz;
  flag_scatter_kernel<<<unsigned(source_flag_blocks(N)), SRC_THREADS, 0, st>>>(
      mark, N, block_offsets, src_cells);
  cudaError_t e = cudaMemsetAsync(lidx, 0xFF, size_t(N) * 4, st);
  if (e != cudaSuccess) return e;
  list_index_kernel<<<unsigned((L + 255) / 256), 256, 0, st>>>(cells, words, L, lidx);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- phase A
// pop[i L + k] = f+_i / w_i - 1 of the cell that direction i of listed cell k
// reads (App. A with its force, then the Hermite population), pushed by that
// source.  D3Q19 (Q19): the 19 directions with |c|^2 <= 2 and their own
// weights; the corner rows stay unused.  Entries of INFLOW cells are not written
// (nor read).
struct SourceParams {
  const void* in;
  size_t N;
  int nx, ny, nz;
  const float* force;
  float omega;
  const uint32_t* src_cells;
  int64_t S;
  const uint32_t* lidx;   // list index of each FLUID_BOUNDARY cell, else 0xFFFFFFFF
  const uint32_t* words;  // type and link mask of each listed cell
  int64_t L;
  float* pop;             // [27][L]
  QGrids q;
};

template <int STORAGE, bool FORCE, bool Q19>
__global__ void __launch_bounds__(256) source_collide_kernel(SourceParams P) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= P.S) return;
  const uint32_t n = P.src_cells[s];
  const size_t N = P.N;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  if (FORCE) {
    fx = __ldg(P.force + n);
    fy = __ldg(P.force + N + n);
    fz = __ldg(P.force + 2 * N + n);
  }
  const Mom17 A = collide_moments<FORCE>(load_stored<STORAGE>(P.in, N, n, P.q), P.omega, fx, fy, fz);
  int x, y, z;
  cell_xyz(n, P.nx, P.ny, &x, &y, &z);
  const uint32_t L = uint32_t(P.L);
  const uint32_t self = __ldg(P.lidx + n);
  const uint32_t self_word = self < L ? __ldg(P.words + self) : 0u;
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    if (Q19 && !in_d3q19(cx, cy, cz)) continue;
    // the listed cell that pulls population i from here (x + c_i, periodic)
    const uint32_t t = __ldg(P.lidx + pull_source(x, y, z, P.nx, P.ny, P.nz, 26 - i));
    const bool push = t < L;
    const bool bounce = (self_word >> (26 - i)) & 1u;  // solid link opp(i) of this cell
    if (push || bounce) {
      const float f = Q19 ? hermite_eval19(A, cx, cy, cz) : hermite_eval(A, cx, cy, cz);
      if (push) P.pop[int64_t(i) * P.L + t] = f;
      if (bounce) P.pop[int64_t(26 - i) * P.L + self] = f;
    }
  }
}

template <bool Q19>
static void launch_source_collide_t(int storage, const SourceParams& p, cudaStream_t st) {
  const unsigned blocks = unsigned((p.S + 255) / 256);
  if (storage == ST_Q16) {
    if (p.force) source_collide_kernel<ST_Q16, true, Q19><<<blocks, 256, 0, st>>>(p);
    else source_collide_kernel<ST_Q16, false, Q19><<<blocks, 256, 0, st>>>(p);
  } else {
    if (p.force) source_collide_kernel<ST_F32, true, Q19><<<blocks, 256, 0, st>>>(p);
    else source_collide_kernel<ST_F32, false, Q19><<<blocks, 256, 0, st>>>(p);
  }
}

cudaError_t launch_source_collide(int storage, int nx, int ny, int nz, const void* in,
                                  const float* force, float omega, const uint32_t* src_cells,
                                  int64_t S, const uint32_t* lidx, const uint32_t* words,
                                  int64_t L, float* pop, const QGrids& q, int lattice,
                                  cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  SourceParams p;
  p.in = in;
  p.N = size_t(nx) * ny * nz;
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.force = force;
  p.omega = omega;
  p.src_cells = src_cells;
  p.S = S;
  p.lidx = lidx;
  p.words = words;
  p.L = L;
  p.pop = pop;
  p.q = q;
  if (lattice == 19) launch_source_collide_t<true>(storage, p, st);
  else launch_source_collide_t<false>(storage, p, st);
  return cudaGetLastError();
}

}  // namespace melbm
