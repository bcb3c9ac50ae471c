// api.cu -- the extern "C" entry points declared in include/melbm.h: handle
// life cycle, argument checks, host/device pointer handling and the step loop
// (fluid kernel -> boundary kernel -> outflow copy, Sec. 4.2).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/melbm.h"
#include "melbm_device.cuh"
#include "melbm_launch.h"
#include "melbm_adjoint.h"
#include "melbm_handle.h"

using namespace melbm;


namespace {

thread_local std::string g_err;

int fail(melbm_t h, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (h) h->err = msg;
  else g_err = msg;
  return code;
}

int cuda_fail(melbm_t h, cudaError_t e, const char* where) {
  if (h) h->poisoned = true;
  return fail(h, MELBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// A bounded barrier wait of an earlier fluid-kernel launch ran out: the state it
// wrote is undefined.  Reported once (the word is cleared); the handle then
// refuses to step until a new state is set.
int kernel_fault(melbm_t h, const char* where) {
  volatile uint32_t* f = h->fault_host;
  if (!f || *f == 0u) return MELBM_OK;
  *f = 0u;
  h->poisoned = true;
  return fail(h, MELBM_ECUDA,
              "%s: a barrier wait of the fluid kernel ran out; the state is undefined, "
              "call melbm_set_state",
              where);
}

// A new state replaces one that a fault may have left: the fault of the work
// issued before it is no longer this state's (cleared once that work has run).
int clear_fault(melbm_t h, const char* where) {
  volatile uint32_t* f = h->fault_host;
  if (!f || *f == 0u) return MELBM_OK;
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  *f = 0u;
  return MELBM_OK;
}

#define MELBM_CUDA(h, call)                                       \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);        \
  } while (0)

// Failure injection on the host: with MELBM_FAIL_ALLOC_AFTER = k in the
// environment, the device allocations of this process after the first k fail
// as if the device were out of memory (read once, at the first allocation).
bool injected_alloc_failure() {
  static const long limit = [] {
    const char* v = std::getenv("MELBM_FAIL_ALLOC_AFTER");
    return v && *v ? std::strtol(v, nullptr, 10) : -1L;
  }();
  static std::atomic<long> count{0};
  return limit >= 0 && count.fetch_add(1) >= limit;
}

// An NVTX range over the scope (seen by profilers that are attached; a no-op
// otherwise).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int dev_alloc(melbm_t h, void** p, size_t bytes) {
  if (bytes == 0) {
    *p = nullptr;
    return MELBM_OK;
  }
  if (injected_alloc_failure()) {
    *p = nullptr;
    return fail(h, MELBM_ENOMEM, "device allocation of %zu bytes failed (MELBM_FAIL_ALLOC_AFTER)",
                bytes);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, MELBM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  if (h) h->mem_bytes += int64_t(bytes);
  return MELBM_OK;
}

void dev_free(melbm_t h, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  if (h) h->mem_bytes -= int64_t(bytes);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bytes of the state a raw-state call moves (0: the mixed scheme has none).
size_t state_bytes(const melbm_sim* h) {
  if (h->storage == MELBM_MIXED) return 0;
  return size_t(h->N) * (h->storage == MELBM_Q16 ? 20 : 40);
}

// Bytes of buffer k: the ping-pong pair, or Q (16-bit post-collision) and P
// (FP32 post-streaming) of the mixed scheme.
size_t buf_bytes(const melbm_sim* h, int k) {
  if (h->storage == MELBM_MIXED) return size_t(h->N) * (k == 0 ? 20 : 40);
  return state_bytes(h);
}

float* mixed_p(const melbm_sim* h) { return static_cast<float*>(h->buf[1]); }

int mixed_unsupported(melbm_t h, const char* what) {
  return fail(h, MELBM_EINVAL, "%s: not available with MELBM_MIXED storage", what);
}

int ensure_staging(melbm_t h, size_t bytes) {
  if (h->staging_bytes >= bytes) return MELBM_OK;
  dev_free(h, h->staging, h->staging_bytes);
  h->staging = nullptr;
  h->staging_bytes = 0;
  int rc = dev_alloc(h, &h->staging, bytes);
  if (rc) return rc;
  h->staging_bytes = bytes;
  return MELBM_OK;
}

void free_list(melbm_t h) {
  dev_free(h, h->cls_solid, size_t(h->W) * 4);
  dev_free(h, h->cls_fb, size_t(h->W) * 4);
  dev_free(h, h->cls_pref, size_t(h->W) * 4);
  dev_free(h, h->side, size_t(h->L_cap) * SIDE_FLOATS * 4);
  h->cls_solid = h->cls_fb = h->cls_pref = nullptr;
  h->side = nullptr;
  h->W = 0;
  dev_free(h, h->list_cell, size_t(h->L_cap) * 4);
  dev_free(h, h->list_word, size_t(h->L_cap) * 4);
  h->list_cell = h->list_word = nullptr;
  h->L = h->L_cap = 0;
}

BoundaryTables boundary_tables(const melbm_sim* h) {
  BoundaryTables t;
  t.solid = h->cls_solid;
  t.fb = h->cls_fb;
  t.pref = h->cls_pref;
  t.side = h->side;
  t.L = h->L;
  return t;
}

// Classification (classify.cu): types, the list, and with solids the tables the
// fluid kernel reads (per 32-cell word of a row the SOLID and FLUID_BOUNDARY bits
// and the list index of its first listed cell) and the [L][12] side table it
// fills every step (the mixed scheme corrects its own fluid pass and needs no
// tables).
int reclassify_lists(melbm_t h) {
  if (!h->mask && !h->inflow_on && !h->outflow_on) {
    free_list(h);
    dev_free(h, h->type, size_t(h->N));
    h->type = nullptr;
    return MELBM_OK;
  }
  // a classification of the same grid reuses the arrays of the last one (the
  // list arrays and the side table while they are large enough)
  int rc;
  if (!h->type && (rc = dev_alloc(h, (void**)&h->type, size_t(h->N)))) return rc;
  const bool tables = h->mask && h->storage != MELBM_MIXED;
  if (!tables && h->cls_solid) free_list(h);  // the tables go; the list is rebuilt below
  if (tables && !h->cls_solid) {
    h->W = classify_words(h->nx, h->ny, h->nz);  // before the allocations (free_list)
    if ((rc = dev_alloc(h, (void**)&h->cls_solid, size_t(h->W) * 4)) ||
        (rc = dev_alloc(h, (void**)&h->cls_fb, size_t(h->W) * 4)))
      return rc;
  }
  const int64_t nb = classify_blocks(h->nx, h->ny, h->nz);
  const size_t Wb = size_t(classify_words(h->nx, h->ny, h->nz)) * 4;
  if (!h->cl_counts) {
    if ((rc = dev_alloc(h, (void**)&h->cl_counts, size_t(nb) * 4))) return rc;
    if ((rc = dev_alloc(h, (void**)&h->cl_offsets, size_t(nb) * 4))) return rc;
    if ((rc = dev_alloc(h, (void**)&h->cl_total, 4))) return rc;
    if ((rc = dev_alloc(h, (void**)&h->cl_mbits, Wb))) return rc;
    if ((rc = dev_alloc(h, (void**)&h->cl_lbits, Wb))) return rc;
  }
  if (h->mask)
    MELBM_CUDA(h, launch_pack_mask(h->mask, h->nx, h->ny, h->nz, h->cl_mbits, h->stream));
  const uint32_t* mbits = h->mask ? h->cl_mbits : nullptr;
  MELBM_CUDA(h, launch_classify_count(h->nx, h->ny, h->nz, mbits, h->inflow_on, h->outflow_on,
                                     h->type, tables ? h->cls_solid : nullptr,
                                     tables ? h->cls_fb : nullptr, h->cl_lbits, h->cl_counts,
                                     h->stream));
  MELBM_CUDA(h, launch_exclusive_scan(h->cl_counts, h->cl_offsets, nb, h->cl_total, h->stream));
  uint32_t total = 0;
  MELBM_CUDA(h, cudaMemcpyAsync(&total, h->cl_total, 4, cudaMemcpyDeviceToHost, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (int64_t(total) > h->L_cap) {
    dev_free(h, h->list_cell, size_t(h->L_cap) * 4);
    dev_free(h, h->list_word, size_t(h->L_cap) * 4);
    dev_free(h, h->side, size_t(h->L_cap) * SIDE_FLOATS * 4);
    h->list_cell = h->list_word = nullptr;
    h->side = nullptr;
    h->L = h->L_cap = 0;
  }
  if (total) {
    if (!h->list_cell) {
      h->L_cap = total;  // before the allocations (free_list)
      if ((rc = dev_alloc(h, (void**)&h->list_cell, size_t(total) * 4))) return rc;
      if ((rc = dev_alloc(h, (void**)&h->list_word, size_t(total) * 4))) return rc;
    }
    if (tables && !h->cls_pref && (rc = dev_alloc(h, (void**)&h->cls_pref, size_t(h->W) * 4)))
      return rc;
    if (tables && !h->side && (rc = dev_alloc(h, (void**)&h->side, size_t(h->L_cap) * SIDE_FLOATS * 4)))
      return rc;
    h->L = total;
    MELBM_CUDA(h, launch_classify_scatter(h->nx, h->ny, h->nz, mbits, h->inflow_on,
                                          h->outflow_on, h->cl_lbits, h->cl_offsets, h->list_cell,
                                          h->list_word, tables ? h->cls_pref : nullptr, h->stream));
  } else {
    h->L = 0;
    // the fluid kernel with solids reads every word's list index a pair ahead,
    // listed cells or not: with an empty list the table is all zeros
    if (tables && !h->cls_pref && (rc = dev_alloc(h, (void**)&h->cls_pref, size_t(h->W) * 4)))
      return rc;
    if (tables) MELBM_CUDA(h, cudaMemsetAsync(h->cls_pref, 0, size_t(h->W) * 4, h->stream));
  }
  return MELBM_OK;
}

// A failed setup leaves no partial lists behind, and the handle refuses to step
// (its boundaries are undefined) until a later setup succeeds.
int reclassify(melbm_t h) {
  const int rc = reclassify_lists(h);
  if (rc != MELBM_OK) free_list(h);
  h->boundary_error = rc != MELBM_OK;
  h->boundary_pending = false;
  return rc;
}

// melbm_set_solid / melbm_set_inflow / melbm_set_outflow only record the change;
// the classification runs once, at the first call that needs the types or the
// list.  Its failure is that call's status (and later calls refuse, as after a
// failed setup).
int mark_boundaries_changed(melbm_t h) {
  h->boundary_pending = true;
  h->boundary_error = false;
  return MELBM_OK;
}

int boundary_refusal(melbm_t h, const char* what) {
  return fail(h, MELBM_ESTATE, "%s: the last boundary setup failed; set the solids, inflow or "
              "outflow again", what);
}

void release_transfers(melbm_t h) {
  if (!h->transfers) return;
  if (h->up_stream) cudaStreamSynchronize(h->up_stream);
  if (h->down_stream) cudaStreamSynchronize(h->down_stream);
  cudaEvent_t* evs[8] = {&h->ev_issue,      &h->ev_uploaded,   &h->ev_read[0],
                         &h->ev_read[1],    &h->ev_read[2],    &h->ev_retired[0],
                         &h->ev_retired[1], &h->ev_retired[2]};
  for (cudaEvent_t* ev : evs) {
    if (*ev) cudaEventDestroy(*ev);
    *ev = nullptr;
  }
  if (h->up_stream) cudaStreamDestroy(h->up_stream);
  if (h->down_stream) cudaStreamDestroy(h->down_stream);
  h->up_stream = h->down_stream = nullptr;
  dev_free(h, h->spare, state_bytes(h));
  h->spare = nullptr;
  h->transfers = false;
}

// Streams, events and the spare buffer of the asynchronous raw-state transfers,
// created once (the spare holds one state: 20 or 40 B per cell).
int ensure_transfers(melbm_t h) {
  if (h->transfers) return MELBM_OK;
  h->transfers = true;
  if (int rc = dev_alloc(h, &h->spare, state_bytes(h))) {
    release_transfers(h);
    return rc;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->down_stream, cudaStreamNonBlocking);
  cudaEvent_t* evs[8] = {&h->ev_issue,      &h->ev_uploaded,   &h->ev_read[0],
                         &h->ev_read[1],    &h->ev_read[2],    &h->ev_retired[0],
                         &h->ev_retired[1], &h->ev_retired[2]};
  for (int k = 0; k < 8 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(evs[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_transfers(h);
    return fail(h, MELBM_ECUDA, "creating the transfer streams: %s", cudaGetErrorString(e));
  }
  return MELBM_OK;
}

int check_raw_bytes(melbm_t h, const char* what, int64_t bytes) {
  if (h->storage == MELBM_MIXED) return mixed_unsupported(h, what);
  if (bytes != int64_t(state_bytes(h)))
    return fail(h, MELBM_EINVAL, "%s: bytes %lld != %lld", what, (long long)bytes,
                (long long)state_bytes(h));
  return MELBM_OK;
}

}  // namespace

namespace melbm {
cudaError_t forward_step_on(melbm_sim* h, const void* in, void* out, uint32_t t_out,
                            cudaStream_t st) {
  const float omega = 1.0f / h->tau;
  const BoundaryTables bt = boundary_tables(h);
  cudaError_t e = cudaSuccess;
  if (h->L)  // the bounce-back sums of the listed cells, from their input state
    e = launch_bounce(h->storage, h->nx, h->ny, h->nz, in, h->force, omega, h->list_cell,
                      h->list_word, h->L, bt, h->grids, h->wall_model, h->mask, h->bodies,
                      h->lattice, st);
  if (e == cudaSuccess)
    e = h->lattice == MELBM_D3Q19
          ? launch_fluid19(h->storage, h->nx, h->ny, h->nz, in, out, h->force, omega, t_out,
                           h->seed, h->grids, &bt, st, h->fault_dev, h->stall_test)
          : launch_fluid(h->storage, h->nx, h->ny, h->nz, in, out, h->force, omega, t_out,
                         h->seed, h->grids, &bt, st, h->fault_dev, h->stall_test);
  if (e == cudaSuccess && h->inflow_on && h->type)
    e = launch_inflow(h->storage, h->nx, h->ny, h->nz, out, h->type, h->inflow, t_out, h->seed,
                      h->grids, st);
  if (e == cudaSuccess && h->outflow_on && h->type)
    e = launch_outflow(h->storage, h->nx, h->ny, h->nz, out, h->type, st);
  return e;
}

cudaError_t forward_step(melbm_sim* h, const void* in, void* out, uint32_t t_out) {
  return forward_step_on(h, in, out, t_out, h->stream);
}

int ensure_boundaries(melbm_sim* h) {
  if (!h->boundary_pending) return MELBM_OK;
  return reclassify(h);
}

int handleless_fail(int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  g_err = msg;
  return code;
}

cudaError_t join_transfers(melbm_sim* h) {
  if (!h->transfers) return cudaSuccess;
  cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_uploaded, 0);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(h->stream, h->ev_read[k], 0);
  return e;
}
}  // namespace melbm

extern "C" {

int melbm_create(int nx, int ny, int nz, int lattice, float tau, int storage, melbm_t* out) {
  if (!out) return fail(nullptr, MELBM_EINVAL, "melbm_create: out is NULL");
  *out = nullptr;
  if (lattice != MELBM_D3Q27 && lattice != MELBM_D3Q19)
    return fail(nullptr, MELBM_EINVAL, "melbm_create: lattice %d unsupported (27 or 19)", lattice);
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(nullptr, MELBM_EINVAL, "melbm_create: bad grid %d x %d x %d", nx, ny, nz);
  const int64_t N = int64_t(nx) * ny * nz;
  if (N >= (int64_t(1) << 31))
    return fail(nullptr, MELBM_EINVAL, "melbm_create: %lld cells exceed 2^31 - 1", (long long)N);
  if (!(tau > 0.5f) || !(tau < 1e6f))
    return fail(nullptr, MELBM_EINVAL, "melbm_create: tau = %g must exceed 1/2", double(tau));
  if (storage != MELBM_F32 && storage != MELBM_Q16 && storage != MELBM_MIXED)
    return fail(nullptr, MELBM_EINVAL, "melbm_create: storage %d unknown", storage);
  melbm_sim* h = new (std::nothrow) melbm_sim;
  if (!h) return fail(nullptr, MELBM_ENOMEM, "melbm_create: host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->N = N;
  h->tau = tau;
  h->storage = storage;
  h->lattice = lattice;
  int rc;
  if ((rc = dev_alloc(h, &h->buf[0], buf_bytes(h, 0))) ||
      (rc = dev_alloc(h, &h->buf[1], buf_bytes(h, 1))) ||
      (rc = dev_alloc(h, (void**)&h->red_partials, size_t(reduce_blocks()) * 3 * 8)) ||
      (rc = dev_alloc(h, (void**)&h->red_out, 3 * 8))) {
    g_err = h->err;
    melbm_destroy(h);
    return rc;
  }
  {
    cudaError_t e = cudaHostAlloc((void**)&h->fault_host, sizeof(uint32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) {
      *h->fault_host = 0u;
      e = cudaHostGetDevicePointer((void**)&h->fault_dev, h->fault_host, 0);
    }
    if (e != cudaSuccess) {
      cuda_fail(h, e, "melbm_create: the kernel fault word");
      g_err = h->err;
      melbm_destroy(h);
      return MELBM_ECUDA;
    }
    const char* v = std::getenv("MELBM_TEST_STALL_BARRIER");
    h->stall_test = (v && std::atoi(v) != 0) ? 1 : 0;
  }
  // rest state (rho = 1, u = 0, S = 0) at time index 0
  cudaError_t e;
  if (storage == MELBM_MIXED) {
    e = cudaMemsetAsync(h->buf[1], 0, buf_bytes(h, 1), h->stream);
    if (e == cudaSuccess)
      e = launch_mixed_collide_quantize(nx, ny, nz, mixed_p(h), h->buf[0], 1.0f / tau, 0, 0,
                                        h->stream);
  } else {
    e = launch_rest_state(storage, nx, ny, nz, h->buf[0], 0, h->grids, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cuda_fail(h, e, "melbm_create: initialising the rest state");
    g_err = h->err;
    melbm_destroy(h);
    return MELBM_ECUDA;
  }
  *out = h;
  return MELBM_OK;
}

int melbm_destroy(melbm_t h) {
  if (!h) return MELBM_OK;
  release_transfers(h);
  if (h->adj) adjoint_free(h->adj);
  dev_free(h, h->buf[0], buf_bytes(h, 0));
  dev_free(h, h->buf[1], buf_bytes(h, 1));
  dev_free(h, h->mask, size_t(h->N));
  dev_free(h, h->type, size_t(h->N));
  free_list(h);
  dev_free(h, h->cl_counts, 0);
  dev_free(h, h->cl_offsets, 0);
  dev_free(h, h->cl_total, 0);
  dev_free(h, h->cl_mbits, 0);
  dev_free(h, h->cl_lbits, 0);
  dev_free(h, h->force, 0);
  dev_free(h, h->staging, 0);
  dev_free(h, h->red_partials, 0);
  dev_free(h, h->red_out, 0);
  dev_free(h, h->bodies, 256 * 9 * 4);
  dev_free(h, h->sf_partials, size_t(solid_force_blocks()) * 6 * 8);
  dev_free(h, h->sf_out, 6 * 8);
  if (h->fault_host) cudaFreeHost(h->fault_host);
  delete h;
  return MELBM_OK;
}

int melbm_set_stream(melbm_t h, void* s) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_stream: NULL handle");
  cudaStream_t next = static_cast<cudaStream_t>(s);
  if (next != h->stream) {
    // the new stream waits for the work already enqueued on the old one
    cudaEvent_t ev;
    MELBM_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(next, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(h, e, "melbm_set_stream");
  }
  h->stream = next;
  return MELBM_OK;
}

int melbm_set_seed(melbm_t h, uint32_t seed) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_seed: NULL handle");
  h->seed = seed;
  return MELBM_OK;
}

int melbm_set_state(melbm_t h, const float* rho, const float* u, const float* S) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_state: NULL handle");
  if (!rho || !u) return fail(h, MELBM_EINVAL, "melbm_set_state: rho and u are required");
  MELBM_CUDA(h, join_transfers(h));
  if (int rc = clear_fault(h, "melbm_set_state")) return rc;
  const size_t N = size_t(h->N);
  const bool dev = is_device_ptr(rho) && is_device_ptr(u) && (!S || is_device_ptr(S));
  const float *r = rho, *uu = u, *ss = S;
  if (!dev) {
    int rc = ensure_staging(h, N * 4 * (S ? 10 : 4));
    if (rc) return rc;
    float* st = static_cast<float*>(h->staging);
    const cudaMemcpyKind k = cudaMemcpyDefault;
    MELBM_CUDA(h, cudaMemcpyAsync(st, rho, N * 4, k, h->stream));
    MELBM_CUDA(h, cudaMemcpyAsync(st + N, u, N * 12, k, h->stream));
    if (S) MELBM_CUDA(h, cudaMemcpyAsync(st + 4 * N, S, N * 24, k, h->stream));
    r = st;
    uu = st + N;
    ss = S ? st + 4 * N : nullptr;
  }
  if (h->storage == MELBM_MIXED) {
    MELBM_CUDA(h, launch_mixed_set_state(h->N, r, uu, ss, mixed_p(h), h->stream));
    MELBM_CUDA(h, launch_mixed_collide_quantize(h->nx, h->ny, h->nz, mixed_p(h), h->buf[0],
                                                1.0f / h->tau, 0, h->seed, h->stream));
  } else {
    MELBM_CUDA(h, launch_set_state(h->storage, h->nx, h->ny, h->nz, r, uu, ss, h->buf[h->cur], 0,
                                   h->seed, 0, h->grids, h->stream));
  }
  if (!dev) MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->t = 0;
  h->poisoned = false;
  return MELBM_OK;
}

int melbm_get_moments(melbm_t h, float* rho, float* u, float* S) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_get_moments: NULL handle");
  if (!rho && !u && !S) return fail(h, MELBM_EINVAL, "melbm_get_moments: no output");
  MELBM_CUDA(h, join_transfers(h));
  const size_t N = size_t(h->N);
  const bool dev = (!rho || is_device_ptr(rho)) && (!u || is_device_ptr(u)) && (!S || is_device_ptr(S));
  if (dev && h->storage == MELBM_MIXED) {
    MELBM_CUDA(h, launch_mixed_get_moments(h->N, mixed_p(h), rho, u, S, h->stream));
    return MELBM_OK;
  }
  if (dev) {
    MELBM_CUDA(h, launch_get_moments(h->storage, h->N, h->buf[h->cur], rho, u, S, h->grids,
                                     h->stream));
    return MELBM_OK;
  }
  int rc = ensure_staging(h, N * 40);
  if (rc) return rc;
  float* st = static_cast<float*>(h->staging);
  if (h->storage == MELBM_MIXED)
    MELBM_CUDA(h, launch_mixed_get_moments(h->N, mixed_p(h), st, st + N, st + 4 * N, h->stream));
  else
    MELBM_CUDA(h, launch_get_moments(h->storage, h->N, h->buf[h->cur], st, st + N, st + 4 * N,
                                     h->grids, h->stream));
  const cudaMemcpyKind k = cudaMemcpyDefault;
  if (rho) MELBM_CUDA(h, cudaMemcpyAsync(rho, st, N * 4, k, h->stream));
  if (u) MELBM_CUDA(h, cudaMemcpyAsync(u, st + N, N * 12, k, h->stream));
  if (S) MELBM_CUDA(h, cudaMemcpyAsync(S, st + 4 * N, N * 24, k, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_set_solid(melbm_t h, const uint8_t* mask) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_solid: NULL handle");
  const Range range("melbm_set_solid");
  if (mask && !is_device_ptr(mask)) return fail(h, MELBM_EINVAL, "melbm_set_solid: mask must be a device pointer");
  if (!mask) {
    dev_free(h, h->mask, size_t(h->N));
    h->mask = nullptr;
  } else {
    int rc;
    if (!h->mask && (rc = dev_alloc(h, (void**)&h->mask, size_t(h->N)))) return rc;
    MELBM_CUDA(h, cudaMemcpyAsync(h->mask, mask, size_t(h->N), cudaMemcpyDeviceToDevice, h->stream));
  }
  return mark_boundaries_changed(h);
}

int melbm_set_inflow(melbm_t h, int face, float rho, float ux, float uy, float uz) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_inflow: NULL handle");
  if (face != 0) return fail(h, MELBM_EINVAL, "melbm_set_inflow: only face 0 (x = 0) is supported");
  if (!(rho > 0.f)) return fail(h, MELBM_EINVAL, "melbm_set_inflow: rho must be positive");
  h->inflow_on = 1;
  h->inflow[0] = rho;
  h->inflow[1] = ux;
  h->inflow[2] = uy;
  h->inflow[3] = uz;
  return mark_boundaries_changed(h);
}

int melbm_set_outflow(melbm_t h, int face) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_outflow: NULL handle");
  if (face != 1) return fail(h, MELBM_EINVAL, "melbm_set_outflow: only face 1 (x = nx-1) is supported");
  h->outflow_on = 1;
  return mark_boundaries_changed(h);
}

int melbm_get_boundary_list(melbm_t h, uint32_t* cells, uint32_t* words, int64_t capacity,
                            int64_t* count) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_get_boundary_list: NULL handle");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error) return boundary_refusal(h, "melbm_get_boundary_list");
  if (count) *count = h->L;
  if ((cells || words) && capacity < h->L)
    return fail(h, MELBM_EINVAL, "melbm_get_boundary_list: capacity %lld < %lld",
                (long long)capacity, (long long)h->L);
  if (h->L) {
    if (cells) MELBM_CUDA(h, cudaMemcpyAsync(cells, h->list_cell, size_t(h->L) * 4, cudaMemcpyDefault, h->stream));
    if (words) MELBM_CUDA(h, cudaMemcpyAsync(words, h->list_word, size_t(h->L) * 4, cudaMemcpyDefault, h->stream));
    MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return MELBM_OK;
}

int melbm_get_types(melbm_t h, uint8_t* types) {
  if (!h || !types) return fail(h, MELBM_EINVAL, "melbm_get_types: NULL argument");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error) return boundary_refusal(h, "melbm_get_types");
  if (h->type) {
    MELBM_CUDA(h, cudaMemcpyAsync(types, h->type, size_t(h->N), cudaMemcpyDefault, h->stream));
  } else {
    MELBM_CUDA(h, cudaMemsetAsync(types, 0, size_t(h->N), h->stream));
  }
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_set_force(melbm_t h, const float* F) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_force: NULL handle");
  if (h->storage == MELBM_MIXED) return mixed_unsupported(h, "melbm_set_force");
  if (!F) {
    dev_free(h, h->force, size_t(h->N) * 12);
    h->force = nullptr;
    return MELBM_OK;
  }
  int rc;
  if (!h->force && (rc = dev_alloc(h, (void**)&h->force, size_t(h->N) * 12))) return rc;
  MELBM_CUDA(h, cudaMemcpyAsync(h->force, F, size_t(h->N) * 12, cudaMemcpyDefault, h->stream));
  return MELBM_OK;
}

int melbm_step(melbm_t h, int n) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_step: NULL handle");
  const Range range("melbm_step");
  if (n < 0) return fail(h, MELBM_EINVAL, "melbm_step: n = %d < 0", n);
  if (int rc = kernel_fault(h, "melbm_step")) return rc;
  if (h->poisoned) return fail(h, MELBM_ESTATE, "melbm_step: an earlier CUDA failure left the state undefined; call melbm_set_state");
  if (h->boundary_error) return boundary_refusal(h, "melbm_step");
  if (n > 0)
    if (int rc = ensure_boundaries(h)) return rc;
  if (h->transfers && n > 0) {
    // the uploaded state must have landed; a download may still read the input
    // buffer, but not one that this call overwrites
    MELBM_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_uploaded, 0));
    if (n > 1) {
      MELBM_CUDA(h, join_transfers(h));
    } else {
      MELBM_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_read[h->buf_id[1 - h->cur]], 0));
    }
  }
  for (int s = 0; s < n; ++s) {
    const uint32_t t_out = uint32_t(h->t + 1);
    if (h->storage == MELBM_MIXED) {
      if (h->lattice == MELBM_D3Q19)
        MELBM_CUDA(h, launch_fluid_mixed19(h->nx, h->ny, h->nz, h->buf[0], mixed_p(h), h->stream));
      else
        MELBM_CUDA(h, launch_fluid_mixed(h->nx, h->ny, h->nz, h->buf[0], mixed_p(h), h->stream));
      if (h->L)
        MELBM_CUDA(h, launch_mixed_correct(h->nx, h->ny, h->nz, h->buf[0], mixed_p(h), h->list_cell,
                                           h->list_word, h->L, h->inflow, h->lattice, h->stream));
      if (h->outflow_on && h->type)
        MELBM_CUDA(h, launch_outflow(MELBM_F32, h->nx, h->ny, h->nz, mixed_p(h), h->type, h->stream));
      MELBM_CUDA(h, launch_mixed_collide_quantize(h->nx, h->ny, h->nz, mixed_p(h), h->buf[0],
                                                  1.0f / h->tau, t_out, h->seed, h->stream));
    } else {
      MELBM_CUDA(h, forward_step(h, h->buf[h->cur], h->buf[1 - h->cur], t_out));
      h->cur = 1 - h->cur;
    }
    h->t += 1;
  }
  return MELBM_OK;
}

int melbm_reduce(melbm_t h, double* mass, double* ke) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_reduce: NULL handle");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error) return boundary_refusal(h, "melbm_reduce");
  MELBM_CUDA(h, join_transfers(h));
  const void* state = h->storage == MELBM_MIXED ? h->buf[1] : h->buf[h->cur];
  MELBM_CUDA(h, launch_reduce(h->storage, h->N, state, h->type, h->red_partials, h->red_out,
                              h->grids, h->stream));
  double out[3];
  MELBM_CUDA(h, cudaMemcpyAsync(out, h->red_out, sizeof out, cudaMemcpyDeviceToHost, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (int rc = kernel_fault(h, "melbm_reduce")) return rc;
  if (mass) *mass = out[0];
  if (ke) *ke = out[1];
  if (h->storage == MELBM_Q16 && out[2] > 0.0)
    return fail(h, MELBM_WSATURATED, "melbm_reduce: %.0f non-solid 16-bit codes on a range limit", out[2]);
  return MELBM_OK;
}

int melbm_time_index(melbm_t h, int64_t* t) {
  if (!h || !t) return fail(h, MELBM_EINVAL, "melbm_time_index: NULL argument");
  *t = h->t;
  return MELBM_OK;
}

int melbm_memory_bytes(melbm_t h, int64_t* bytes) {
  if (!h || !bytes) return fail(h, MELBM_EINVAL, "melbm_memory_bytes: NULL argument");
  *bytes = h->mem_bytes;
  return MELBM_OK;
}

int melbm_state_bytes(melbm_t h, int64_t* bytes) {
  if (!h || !bytes) return fail(h, MELBM_EINVAL, "melbm_state_bytes: NULL argument");
  *bytes = int64_t(state_bytes(h));
  return MELBM_OK;
}

int melbm_get_raw_state(melbm_t h, void* dst, int64_t bytes) {
  if (!h || !dst) return fail(h, MELBM_EINVAL, "melbm_get_raw_state: NULL argument");
  if (int rc = check_raw_bytes(h, "melbm_get_raw_state", bytes)) return rc;
  MELBM_CUDA(h, join_transfers(h));
  MELBM_CUDA(h, cudaMemcpyAsync(dst, h->buf[h->cur], size_t(bytes), cudaMemcpyDefault, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_set_raw_state(melbm_t h, const void* src, int64_t bytes, int64_t time_index) {
  if (!h || !src) return fail(h, MELBM_EINVAL, "melbm_set_raw_state: NULL argument");
  if (int rc = check_raw_bytes(h, "melbm_set_raw_state", bytes)) return rc;
  if (time_index < 0) return fail(h, MELBM_EINVAL, "melbm_set_raw_state: negative time index");
  MELBM_CUDA(h, join_transfers(h));
  if (int rc = clear_fault(h, "melbm_set_raw_state")) return rc;
  MELBM_CUDA(h, cudaMemcpyAsync(h->buf[h->cur], src, size_t(bytes), cudaMemcpyDefault, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->t = time_index;
  h->poisoned = false;
  return MELBM_OK;
}

// The upload lands in the spare buffer, after the work that was issued while the
// spare was last in a slot and after any download still reading it; the spare then
// takes the current state's slot and the buffer it replaces retires to the spare
// (once the work issued so far has run: a step in flight may still write it, a
// download read it).  So an upload runs beside the step in flight and beside the
// download of its result.  The download reads the current state after the work
// already issued and after the upload that produced it.  Neither blocks the host.
int melbm_upload_raw_state_async(melbm_t h, const void* src, int64_t bytes, int64_t time_index) {
  if (!h || !src) return fail(h, MELBM_EINVAL, "melbm_upload_raw_state_async: NULL argument");
  if (int rc = check_raw_bytes(h, "melbm_upload_raw_state_async", bytes)) return rc;
  if (time_index < 0)
    return fail(h, MELBM_EINVAL, "melbm_upload_raw_state_async: negative time index");
  if (int rc = ensure_transfers(h)) return rc;
  if (int rc = clear_fault(h, "melbm_upload_raw_state_async")) return rc;
  const int s = h->spare_id, c = h->buf_id[h->cur];
  MELBM_CUDA(h, cudaStreamWaitEvent(h->up_stream, h->ev_retired[s], 0));
  MELBM_CUDA(h, cudaStreamWaitEvent(h->up_stream, h->ev_read[s], 0));
  MELBM_CUDA(h, cudaMemcpyAsync(h->spare, src, size_t(bytes), cudaMemcpyDefault, h->up_stream));
  MELBM_CUDA(h, cudaEventRecord(h->ev_uploaded, h->up_stream));
  MELBM_CUDA(h, cudaEventRecord(h->ev_retired[c], h->stream));
  void* p = h->buf[h->cur];
  h->buf[h->cur] = h->spare;
  h->buf_id[h->cur] = s;
  h->spare = p;
  h->spare_id = c;
  h->t = time_index;
  h->poisoned = false;
  return MELBM_OK;
}

int melbm_download_raw_state_async(melbm_t h, void* dst, int64_t bytes) {
  if (!h || !dst) return fail(h, MELBM_EINVAL, "melbm_download_raw_state_async: NULL argument");
  if (int rc = check_raw_bytes(h, "melbm_download_raw_state_async", bytes)) return rc;
  if (int rc = ensure_transfers(h)) return rc;
  MELBM_CUDA(h, cudaEventRecord(h->ev_issue, h->stream));
  MELBM_CUDA(h, cudaStreamWaitEvent(h->down_stream, h->ev_issue, 0));
  MELBM_CUDA(h, cudaStreamWaitEvent(h->down_stream, h->ev_uploaded, 0));
  MELBM_CUDA(h, cudaMemcpyAsync(dst, h->buf[h->cur], size_t(bytes), cudaMemcpyDefault,
                                h->down_stream));
  MELBM_CUDA(h, cudaEventRecord(h->ev_read[h->buf_id[h->cur]], h->down_stream));
  return MELBM_OK;
}

int melbm_sync_transfers(melbm_t h) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_sync_transfers: NULL handle");
  if (!h->transfers) return MELBM_OK;
  MELBM_CUDA(h, cudaStreamSynchronize(h->up_stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->down_stream));
  return MELBM_OK;
}

int melbm_q16_encode(const float* stored, int nx, int ny, int nz, uint32_t t, uint32_t seed,
                     int deterministic, uint32_t* words, void* stream) {
  if (!stored || !words) return fail(nullptr, MELBM_EINVAL, "melbm_q16_encode: NULL pointer");
  if (nx < 1 || ny < 1 || nz < 1 || int64_t(nx) * ny * nz >= (int64_t(1) << 31))
    return fail(nullptr, MELBM_EINVAL, "melbm_q16_encode: bad grid");
  cudaError_t e = launch_q16_encode(stored, nx, ny, nz, t, seed, deterministic, words,
                                    make_qgrids(16, 16), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "melbm_q16_encode");
  return MELBM_OK;
}

int melbm_codec_encode(const float* stored, int nx, int ny, int nz, uint32_t t, uint32_t seed,
                       int deterministic, int bits_rho_u, int bits_S, uint32_t* words,
                       void* stream) {
  if (!stored || !words) return fail(nullptr, MELBM_EINVAL, "melbm_codec_encode: NULL pointer");
  if (nx < 1 || ny < 1 || nz < 1 || int64_t(nx) * ny * nz >= (int64_t(1) << 31))
    return fail(nullptr, MELBM_EINVAL, "melbm_codec_encode: bad grid");
  if (bits_rho_u < 8 || bits_rho_u > 16 || bits_S < 8 || bits_S > 16)
    return fail(nullptr, MELBM_EINVAL, "melbm_codec_encode: bit widths %d/%d outside 8..16",
                bits_rho_u, bits_S);
  cudaError_t e = launch_q16_encode(stored, nx, ny, nz, t, seed, deterministic, words,
                                    make_qgrids(bits_rho_u, bits_S),
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "melbm_codec_encode");
  return MELBM_OK;
}

int melbm_codec_decode(const uint32_t* words, int64_t N, int bits_rho_u, int bits_S, float* stored,
                       void* stream) {
  if (!stored || !words || N < 0 || N >= (int64_t(1) << 31))
    return fail(nullptr, MELBM_EINVAL, "melbm_codec_decode: bad argument");
  if (bits_rho_u < 8 || bits_rho_u > 16 || bits_S < 8 || bits_S > 16)
    return fail(nullptr, MELBM_EINVAL, "melbm_codec_decode: bit widths %d/%d outside 8..16",
                bits_rho_u, bits_S);
  if (N == 0) return MELBM_OK;
  cudaError_t e = launch_q16_decode(words, N, stored, make_qgrids(bits_rho_u, bits_S),
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "melbm_codec_decode");
  return MELBM_OK;
}

int melbm_set_wall_model(melbm_t h, int model) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_wall_model: NULL handle");
  if (h->storage == MELBM_MIXED && model != 0) return mixed_unsupported(h, "melbm_set_wall_model");
  if (model != 0 && model != 1) return fail(h, MELBM_EINVAL, "melbm_set_wall_model: model %d unknown", model);
  if (!h->bodies) {
    int rc = dev_alloc(h, (void**)&h->bodies, 256 * 9 * 4);
    if (rc) return rc;
    MELBM_CUDA(h, cudaMemcpyAsync(h->bodies, h->bodies_host, 256 * 9 * 4, cudaMemcpyHostToDevice,
                                  h->stream));
    MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  h->wall_model = model;
  return MELBM_OK;
}

int melbm_set_body_motion(melbm_t h, int body, const float* V, const float* Omega, const float* r0) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_body_motion: NULL handle");
  if (body < 1 || body > 255) return fail(h, MELBM_EINVAL, "melbm_set_body_motion: body %d outside 1..255", body);
  float* t = h->bodies_host + 9 * body;
  for (int a = 0; a < 3; ++a) {
    t[a] = V ? V[a] : 0.f;
    t[3 + a] = Omega ? Omega[a] : 0.f;
    t[6 + a] = r0 ? r0[a] : 0.f;
  }
  if (!h->bodies) {
    int rc = dev_alloc(h, (void**)&h->bodies, 256 * 9 * 4);
    if (rc) return rc;
  }
  MELBM_CUDA(h, cudaMemcpyAsync(h->bodies, h->bodies_host, 256 * 9 * 4, cudaMemcpyHostToDevice,
                                h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_solid_force(melbm_t h, int body, double* out) {
  if (!h || !out) return fail(h, MELBM_EINVAL, "melbm_solid_force: NULL argument");
  if (body < 0 || body > 255) return fail(h, MELBM_EINVAL, "melbm_solid_force: body %d outside 0..255", body);
  if (h->storage == MELBM_MIXED) return mixed_unsupported(h, "melbm_solid_force");
  if (int rc = ensure_boundaries(h)) return rc;
  if (h->boundary_error) return boundary_refusal(h, "melbm_solid_force");
  for (int k = 0; k < 6; ++k) out[k] = 0.0;
  if (!h->L || !h->mask) return MELBM_OK;
  int rc;
  if (!h->bodies && (rc = melbm_set_wall_model(h, h->wall_model))) return rc;
  if (!h->sf_partials) {
    if ((rc = dev_alloc(h, (void**)&h->sf_partials, size_t(solid_force_blocks()) * 6 * 8)) ||
        (rc = dev_alloc(h, (void**)&h->sf_out, 6 * 8)))
      return rc;
  }
  MELBM_CUDA(h, join_transfers(h));
  MELBM_CUDA(h, launch_solid_force(h->storage, h->nx, h->ny, h->nz, h->buf[h->cur], h->force,
                                   1.0f / h->tau, h->list_cell, h->list_word, h->L, h->grids,
                                   h->wall_model, h->mask, h->bodies, body, h->sf_partials,
                                   h->sf_out, h->lattice, h->stream));
  MELBM_CUDA(h, cudaMemcpyAsync(out, h->sf_out, 6 * 8, cudaMemcpyDeviceToHost, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_set_bits(melbm_t h, int bits_rho_u, int bits_S) {
  if (!h) return fail(nullptr, MELBM_EINVAL, "melbm_set_bits: NULL handle");
  if (h->storage != MELBM_Q16)
    return fail(h, MELBM_EINVAL, "melbm_set_bits: only the quantised storage has bit widths");
  if (bits_rho_u < 8 || bits_rho_u > 16 || bits_S < 8 || bits_S > 16)
    return fail(h, MELBM_EINVAL, "melbm_set_bits: bit widths %d/%d outside 8..16", bits_rho_u,
                bits_S);
  if (h->grids.bits_ru == bits_rho_u && h->grids.bits_s == bits_S) return MELBM_OK;
  // re-encode the current state: decode on the old grids, encode on the new ones
  // (dither of the current time index)
  const size_t N = size_t(h->N);
  int rc = ensure_staging(h, N * 40);
  if (rc) return rc;
  float* st = static_cast<float*>(h->staging);
  MELBM_CUDA(h, join_transfers(h));
  MELBM_CUDA(h, launch_get_moments(h->storage, h->N, h->buf[h->cur], st, st + N, st + 4 * N,
                                   h->grids, h->stream));
  h->grids = make_qgrids(bits_rho_u, bits_S);
  MELBM_CUDA(h, launch_set_state(h->storage, h->nx, h->ny, h->nz, st, st + N, st + 4 * N,
                                 h->buf[h->cur], uint32_t(h->t), h->seed, 0, h->grids, h->stream));
  MELBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return MELBM_OK;
}

int melbm_q16_decode(const uint32_t* words, int64_t N, float* stored, void* stream) {
  if (!stored || !words || N < 0 || N >= (int64_t(1) << 31))
    return fail(nullptr, MELBM_EINVAL, "melbm_q16_decode: bad argument");
  if (N == 0) return MELBM_OK;
  cudaError_t e = launch_q16_decode(words, N, stored, make_qgrids(16, 16),
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "melbm_q16_decode");
  return MELBM_OK;
}

const char* melbm_last_error(melbm_t h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"
