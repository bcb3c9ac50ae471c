// reduce_noalloc.cu -- an allocation-free variant of the FP64 conservation
// reduction (total mass, kinetic energy and saturated 16-bit codes).
//
// Why it exists: some callers cannot allocate device memory at the point where
// they want these diagnostics.  Examples are a frame or control loop with a fixed
// memory budget that forbids allocation after start-up, a host where another
// allocator (for instance a framework's caching allocator) has reserved the whole
// device pool, and code that must not risk the implicit device synchronisation
// that cudaMalloc/cudaFree may perform.  melbm_reduce needs a handle, whose
// creation allocates; this entry point works on a state buffer the caller already
// owns and keeps its scratch -- the per-chunk partial sums -- in a fixed array
// compiled into the library.
//
// The scratch is a file-scope __device__ array, so every GPU that loads the
// library holds it (NOALLOC_MAX_CHUNKS x 3 doubles = 96 KiB) until the process
// exits.  Host code cannot use the array's name as a device address (on the host
// it names a stand-in object), so the first call on each device looks the address
// up with cudaGetSymbolAddress while that device is current, and caches it for the
// life of the process.  A cudaDeviceReset (or anything else that destroys and
// re-creates the device's primary context) reloads the module, which may move the
// array; the cached address is then stale, so this entry point must not be used on
// a device after such a reset.
// Every call reuses the same array: calls that overlap on the GPU (from several
// streams or host threads) race on it and must be serialised by the caller.  Each
// call writes every partial it later reads, so nothing has to be cleared first.
#include <mutex>

#include "../../include/melbm.h"
#include "melbm_device.cuh"
#include "melbm_handle.h"
#include "reduce_cell.cuh"

namespace melbm {
namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_CHUNK = 65536;         // cells summed by one block
constexpr int64_t NOALLOC_MAX_CHUNKS = 4096;  // => at most 2^28 cells per call
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_CHUNKS * 3];

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// One block per contiguous chunk of NA_CHUNK cells, fixed order inside the block.
template <int STORAGE>
__global__ void __launch_bounds__(NA_THREADS) noalloc_partial_kernel(int64_t N, const void* buf,
                                                                    const uint8_t* type,
                                                                    double* partials) {
  const int64_t begin = int64_t(blockIdx.x) * NA_CHUNK;
  const int64_t end = begin + NA_CHUNK < N ? begin + NA_CHUNK : N;
  double dmass = 0.0, ke = 0.0;
  uint32_t fluid = 0, rails = 0;
  for (int64_t n = begin + threadIdx.x; n < end; n += NA_THREADS) {
    if (type && type[n] == T_SOLID) continue;
    const CellTerms t = reduce_cell<STORAGE>(buf, size_t(N), size_t(n), nullptr);
    dmass += double(t.drho);
    ke += double(t.ke);
    fluid += 1u;
    rails += t.rails;
  }
  double mass = double(fluid) + dmass, kes = ke, sat = double(rails);
  __shared__ double sm[3][NA_THREADS / 32];
  mass = warp_sum(mass);
  kes = warp_sum(kes);
  sat = warp_sum(sat);
  if ((threadIdx.x & 31) == 0) {
    sm[0][threadIdx.x >> 5] = mass;
    sm[1][threadIdx.x >> 5] = kes;
    sm[2][threadIdx.x >> 5] = sat;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) t += sm[threadIdx.x][w];
    partials[size_t(blockIdx.x) * 3 + threadIdx.x] = t;
  }
}

__global__ void noalloc_final_kernel(const double* partials, int64_t nchunks, double* out) {
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int64_t b = 0; b < nchunks; ++b) t += partials[size_t(b) * 3 + threadIdx.x];
    out[threadIdx.x] = t;
  }
}

std::mutex g_setup_mutex;
double* g_partials_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace melbm

extern "C" int melbm_reduce_state_noalloc(const void* state, int storage, int64_t N,
                                          const uint8_t* type, double* out, void* cuda_stream) {
  using namespace melbm;
  static const char* const fn = "melbm_reduce_state_noalloc";
  if (!state || !out) return handleless_fail(MELBM_EINVAL, "%s: NULL state or out", fn);
  if (storage != MELBM_F32 && storage != MELBM_Q16)
    return handleless_fail(MELBM_EINVAL, "%s: storage %d is neither MELBM_F32 nor MELBM_Q16", fn,
                           storage);
  if (N <= 0) return handleless_fail(MELBM_EINVAL, "%s: N = %lld", fn, (long long)N);
  // The scratch array holds NOALLOC_MAX_CHUNKS partial sums of NA_CHUNK cells:
  // larger grids are refused rather than overrunning it.
  const int64_t nchunks = (N + NA_CHUNK - 1) / NA_CHUNK;
  if (nchunks > NOALLOC_MAX_CHUNKS)
    return handleless_fail(MELBM_EINVAL, "%s: N = %lld exceeds the %lld cells of its fixed scratch",
                           fn, (long long)N, (long long)(NOALLOC_MAX_CHUNKS * NA_CHUNK));
  double* partials = nullptr;
  cudaError_t e = scratch_address(&partials);
  if (e != cudaSuccess)
    return handleless_fail(MELBM_ECUDA, "%s: scratch address lookup: %s", fn, cudaGetErrorString(e));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (storage == MELBM_Q16)
    noalloc_partial_kernel<ST_Q16><<<unsigned(nchunks), NA_THREADS, 0, st>>>(N, state, type, partials);
  else
    noalloc_partial_kernel<ST_F32><<<unsigned(nchunks), NA_THREADS, 0, st>>>(N, state, type, partials);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    noalloc_final_kernel<<<1, 32, 0, st>>>(partials, nchunks, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return handleless_fail(MELBM_ECUDA, "%s: launch: %s", fn, cudaGetErrorString(e));
  return MELBM_OK;
}
