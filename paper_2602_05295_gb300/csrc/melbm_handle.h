// melbm_handle.h -- the simulation handle behind the opaque melbm_t (internal).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "melbm_launch.h"

namespace melbm {
struct AdjointState;
}

struct melbm_sim {
  int nx = 0, ny = 0, nz = 0;
  int64_t N = 0;
  int storage = 0;
  int lattice = 27;  // 27 or 19 (periodic only)
  melbm::QGrids grids = melbm::make_qgrids(16, 16);  // bit widths of the quantised form
  float tau = 0.f;
  uint32_t seed = 0;
  int64_t t = 0;
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  // boundaries
  uint8_t* mask = nullptr;
  uint8_t* type = nullptr;
  uint32_t* list_cell = nullptr;
  uint32_t* list_word = nullptr;
  int64_t L = 0;
  int64_t L_cap = 0;  // entries the list arrays and the side table hold
  // tables of the fluid kernel with solids (melbm::BoundaryTables): per 32-cell
  // word of a row (W words) the SOLID and FLUID_BOUNDARY bits and the list index
  // of its first listed cell, and the [L][12] side table of raw post-streaming
  // sums of the FLUID_BOUNDARY cells
  uint32_t* cls_solid = nullptr;
  uint32_t* cls_fb = nullptr;
  uint32_t* cls_pref = nullptr;
  float* side = nullptr;
  int64_t W = 0;
  // solids, inflow or outflow changed since the last classification: the next
  // call that needs the types or the list classifies first
  bool boundary_pending = false;
  // classification scratch: listed cells per block of words and the blocks'
  // first list indices, their total, the packed mask and the listed cells of
  // every word (W words each)
  uint32_t* cl_counts = nullptr;
  uint32_t* cl_offsets = nullptr;
  uint32_t* cl_total = nullptr;
  uint32_t* cl_mbits = nullptr;
  uint32_t* cl_lbits = nullptr;
  int inflow_on = 0;
  float inflow[4] = {1.f, 0.f, 0.f, 0.f};
  int outflow_on = 0;
  // solid walls: model (0 halfway bounce-back, 1 moment-based reconstruction) and
  // the rigid motion (V, Om, r0) of each body id, host copy and device copy
  int wall_model = 0;
  float bodies_host[256 * 9] = {};
  float* bodies = nullptr;
  double* sf_partials = nullptr;
  double* sf_out = nullptr;
  // force, staging, reductions
  float* force = nullptr;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  double* red_partials = nullptr;
  double* red_out = nullptr;
  int64_t mem_bytes = 0;
  bool poisoned = false;
  // A word of mapped host memory that the fluid kernel sets when one of its
  // bounded barrier waits runs out (host and device addresses); stall_test makes
  // those waits run out (MELBM_TEST_STALL_BARRIER=1 at melbm_create, for tests).
  uint32_t* fault_host = nullptr;
  uint32_t* fault_dev = nullptr;
  int stall_test = 0;
  bool boundary_error = false;  // the last boundary setup failed: lists are empty
  // Asynchronous raw-state transfers (created at their first use): an upload and a
  // download stream, a third state buffer (the spare) that uploads land in, and the
  // events that order the transfers against the handle's stream.  The three state
  // buffers are numbered 0, 1 (the initial pair) and 2 (the spare); buf_id[k] is
  // the number of the buffer in slot buf[k], spare_id that of the spare.
  bool transfers = false;
  cudaStream_t up_stream = nullptr, down_stream = nullptr;
  void* spare = nullptr;
  int buf_id[2] = {0, 1};
  int spare_id = 2;
  cudaEvent_t ev_issue = nullptr;        // the handle's stream when a download is issued
  cudaEvent_t ev_uploaded = nullptr;     // the last upload has landed
  cudaEvent_t ev_read[3] = {};           // the last download of buffer k has read it
  cudaEvent_t ev_retired[3] = {};        // the work issued while buffer k was in a slot
  std::string err;
  melbm::AdjointState* adj = nullptr;  // checkpoints of melbm_forward_checkpointed
};

namespace melbm {
// Launch one forward step in -> out with the handle's boundaries (used by the
// adjoint's recomputation); t_out is the time index of the output state.
cudaError_t forward_step(melbm_sim* h, const void* in, void* out, uint32_t t_out);
// the same step issued on another stream (the boundary side table is shared: one
// step at a time per handle)
cudaError_t forward_step_on(melbm_sim* h, const void* in, void* out, uint32_t t_out,
                            cudaStream_t st);
// Run the classification a melbm_set_solid / set_inflow / set_outflow left
// pending (no-op otherwise); returns its status.
int ensure_boundaries(melbm_sim* h);
// Record the message of a failed call that has no handle (read by
// melbm_last_error(NULL)) and return code.
int handleless_fail(int code, const char* fmt, ...);
// Make the handle's stream wait for every asynchronous raw-state transfer issued
// so far (a no-op when none was).
cudaError_t join_transfers(melbm_sim* h);
}  // namespace melbm
