// reduce.cu -- FP64 conservation diagnostics: total mass sum(rho) and kinetic
// energy sum(rho |u|^2 / 2) over non-solid cells, plus (quantised storage) the
// number of non-solid codes sitting on a range limit (0 or 2^b - 1), which flags saturation
// without any atomic in the hot kernels.  Per-block partial sums, then one block
// adds the partials in a fixed order, so the result is deterministic.
#include "melbm_device.cuh"
#include "melbm_launch.h"
#include "reduce_cell.cuh"

namespace melbm {

constexpr int RD_THREADS = 256;
constexpr int RD_BLOCKS = 608;  // 4 per SM on a 152-SM part

int reduce_blocks() { return RD_BLOCKS; }

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

template <int STORAGE>
__global__ void __launch_bounds__(RD_THREADS) reduce_partial_kernel(int64_t N, const void* buf,
                                                                   const uint8_t* type,
                                                                   double* partials, QGrids q) {
  double dmass = 0.0, ke = 0.0;  // sums of rho - 1 and of rho |u|^2 / 2
  uint32_t fluid = 0, rails = 0;
  for (int64_t n = int64_t(blockIdx.x) * RD_THREADS + threadIdx.x; n < N;
       n += int64_t(gridDim.x) * RD_THREADS) {
    if (type && type[n] == T_SOLID) continue;
    const CellTerms t = reduce_cell<STORAGE>(buf, size_t(N), size_t(n), &q);
    dmass += double(t.drho);
    ke += double(t.ke);
    fluid += 1u;
    rails += t.rails;
  }
  // per thread: mass = cells + sum (rho - 1); at most 2^31 cells in all
  double mass = double(fluid) + dmass, kes = ke, sat = double(rails);
  __shared__ double sm[3][RD_THREADS / 32];
  mass = warp_sum_d(mass);
  kes = warp_sum_d(kes);
  sat = warp_sum_d(sat);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][wid] = mass;
    sm[1][wid] = kes;
    sm[2][wid] = sat;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < RD_THREADS / 32; ++w) t += sm[threadIdx.x][w];
    partials[size_t(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

__global__ void reduce_final_kernel(const double* partials, int nblocks, double* out) {
  // one thread per quantity, fixed order
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partials[size_t(b) * 3 + threadIdx.x];
    out[threadIdx.x] = t;
  }
}

cudaError_t launch_reduce(int storage, int64_t N, const void* buf, const uint8_t* type,
                          double* partials, double* out, const QGrids& q, cudaStream_t st) {
  if (storage == ST_Q16)
    reduce_partial_kernel<ST_Q16><<<RD_BLOCKS, RD_THREADS, 0, st>>>(N, buf, type, partials, q);
  else if (storage == ST_MIXED)
    reduce_partial_kernel<ST_MIXED><<<RD_BLOCKS, RD_THREADS, 0, st>>>(N, buf, type, partials, q);
  else
    reduce_partial_kernel<ST_F32><<<RD_BLOCKS, RD_THREADS, 0, st>>>(N, buf, type, partials, q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_final_kernel<<<1, 32, 0, st>>>(partials, RD_BLOCKS, out);
  return cudaGetLastError();
}

}  // namespace melbm
