// melbm_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace melbm {

// Fluid kernel over every cell: in -> out (storage layout of melbm_device.cuh).
cudaError_t launch_fluid(int storage, int nx, int ny, int nz, const void* in, void* out,
                         const float* force, float omega, uint32_t t_out, uint32_t seed,
                         cudaStream_t st);

// Boundary update over the list: phase A collides the S source cells and keeps
// their 27 populations in pop[27][S] (sources.cu), then the boundary kernel
// recomputes every listed cell (bounce-back through its 27 source slots in
// table[27][count], inflow reset), in -> out.
cudaError_t launch_boundary(int storage, int nx, int ny, int nz, const void* in, void* out,
                            const float* force, float omega, const uint32_t* cells,
                            const uint32_t* words, int64_t count, const uint32_t* src_cells,
                            int64_t S, const uint32_t* table, float* pop, const float inflow[4],
                            uint32_t t_out, uint32_t seed, cudaStream_t st);

// Source set of the boundary update (sources.cu).  Setup, after the list is
// built: mark the sources (mark[N] bytes) and count them per block of
// source_flag_blocks(N); after an exclusive scan of the counts, fill src_cells
// (ascending), slot_of[N] and table[27][L].  Per step: phase A.
int64_t source_flag_blocks(int64_t N);
cudaError_t launch_source_setup_mark(int nx, int ny, int nz, const uint32_t* cells,
                                     const uint32_t* words, int64_t L, uint8_t* mark,
                                     uint32_t* block_counts, cudaStream_t st);
cudaError_t launch_source_setup_fill(int nx, int ny, int nz, const uint32_t* cells,
                                     const uint32_t* words, int64_t L, const uint8_t* mark,
                                     const uint32_t* block_offsets, uint32_t* src_cells,
                                     uint32_t* slot_of, uint32_t* table, cudaStream_t st);
cudaError_t launch_source_collide(int storage, size_t N, const void* in, const float* force,
                                  float omega, const uint32_t* src_cells, int64_t S, float* pop,
                                  cudaStream_t st);

// Outflow copy on the plane x = nx-1 (cells typed OUTFLOW), in place on buf.
cudaError_t launch_outflow(int storage, int nx, int ny, int nz, void* buf, const uint8_t* type,
                           cudaStream_t st);

// Classification: types (N) and per-block counts of listed cells; then the
// ordered scatter into the list.  nblocks_out receives the block count.
int64_t classify_blocks(int64_t N);
cudaError_t launch_classify_count(int nx, int ny, int nz, const uint8_t* mask, int inflow,
                                  int outflow, uint8_t* type, uint32_t* block_counts,
                                  cudaStream_t st);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                                  cudaStream_t st);
cudaError_t launch_classify_scatter(int nx, int ny, int nz, const uint8_t* mask,
                                    const uint8_t* type, const uint32_t* block_offsets,
                                    uint32_t* cells, uint32_t* words, cudaStream_t st);

// FP64 reductions: partial sums per block, then one block sums the partials in
// a fixed order.  out[0] = mass, out[1] = kinetic energy, out[2] = saturated codes.
int reduce_blocks();
cudaError_t launch_reduce(int storage, int64_t N, const void* buf, const uint8_t* type,
                          double* partials, double* out, cudaStream_t st);

// State conversions (public FP32 <-> stored) and the codec on caller buffers.
cudaError_t launch_set_state(int storage, int nx, int ny, int nz, const float* rho, const float* u,
                             const float* S, void* buf, uint32_t t, uint32_t seed, int det,
                             cudaStream_t st);
cudaError_t launch_rest_state(int storage, int nx, int ny, int nz, void* buf, uint32_t seed,
                              cudaStream_t st);
cudaError_t launch_get_moments(int storage, int64_t N, const void* buf, float* rho, float* u,
                               float* S, cudaStream_t st);
cudaError_t launch_q16_encode(const float* stored, int nx, int ny, int nz, uint32_t t,
                              uint32_t seed, int det, uint32_t* words, cudaStream_t st);
cudaError_t launch_q16_decode(const uint32_t* words, int64_t N, float* stored, cudaStream_t st);

}  // namespace melbm
