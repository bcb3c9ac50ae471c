/* melbm.h -- C ABI of the GB300 moment-encoded lattice Boltzmann library.
 *
 * The library advances a D3Q27 (or D3Q19) moment-encoded (HOME-LBM) fluid in
 * which every cell stores only its ten low-order moments (rho, u, S) instead of
 * the 27 (19) populations (arXiv 2602.05295, Sec. 3.2).  One step (Sec. 4.2, Alg. 2 and the
 * split-kernel design) is:
 *   1. with solids, a kernel over a compacted list of boundary cells: what the
 *      solid links of each cell return (halfway bounce-back or moving walls),
 *      from the cell's own post-collision state;
 *   2. a branch-free fluid kernel over all cells: load the moments, collide in
 *      moment space (App. A), rebuild the post-collision populations by the
 *      third-order Hermite expansion (Eq. three_order_f), pull them from the
 *      neighbours (Eq. streaming), add the returned populations of step 1 and
 *      re-form the moments (Eq. rho_u_stress);
 *   3. the inflow reset and a zero-gradient copy onto the outflow plane.
 * Moments are stored either as FP32 or in the paper's 16-bit stability-bounded
 * fixed-point form (Sec. 5.4): rho in [0.8, 1.5], u in [-0.4, 0.4] and
 * rho S^neq = rho (S - u u) in [-0.1, 0.1], dithered rounding, two codes per
 * 32-bit word, five words per cell.
 *
 * Conventions shared by every entry point
 *   Grid nx x ny x nz, linear cell index n = x + nx (y + ny z) (x fastest),
 *   N = nx ny nz.  Field arrays are structure-of-arrays, component-major:
 *   rho[N]; u[3][N] = (ux, uy, uz); S[6][N] = (Sxx, Syy, Szz, Sxy, Sxz, Syz).
 *   S is the per-mass Hermite second moment, S = sum (c c - c_s^2 I) f / rho,
 *   whose equilibrium value is u u.  rho and u are the post-streaming values at
 *   integer time (the physical velocity, which includes F/2).
 *   Lattice directions i = (cx+1) + 3 (cy+1) + 9 (cz+1), opposite = 26 - i (the
 *   same numbering on D3Q19, whose directions are those with |c|^2 <= 2).
 *   Every call returns an int status (melbm_status); on failure the handle keeps
 *   a message for melbm_last_error().  No C++ exception crosses the ABI.
 *   Unless stated otherwise pointers are CUDA device pointers on the current
 *   device, owned by the caller, contiguous, not aliased with library memory.
 *   Work is enqueued on the handle's stream (melbm_set_stream); calls that
 *   return host values synchronise that stream.
 *   Testing hook: with MELBM_FAIL_ALLOC_AFTER=k in the environment, every device
 *   allocation of the process after the first k fails with MELBM_ENOMEM (the
 *   handle stays usable).  melbm_step and melbm_set_solid open NVTX ranges.
 */
#ifndef MELBM_H
#define MELBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MELBM_API __attribute__((visibility("default")))
#else
#define MELBM_API
#endif

typedef struct melbm_sim* melbm_t;

typedef enum melbm_status {
  MELBM_OK = 0,
  MELBM_EINVAL = 1,      /* bad argument: NULL handle/pointer, size, tau <= 1/2, ... */
  MELBM_ENOMEM = 2,      /* a device or host allocation failed */
  MELBM_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  MELBM_ESTATE = 4,      /* call out of order (e.g. step after a failed call) */
  MELBM_WSATURATED = 5   /* warning: some 16-bit codes sit on the range limits */
} melbm_status;

enum { MELBM_D3Q27 = 27, MELBM_D3Q19 = 19 };
enum { MELBM_F32 = 0, MELBM_Q16 = 1, MELBM_MIXED = 2 };
/* cell types, priority SOLID > INFLOW > OUTFLOW > FLUID_BOUNDARY > FLUID */
enum { MELBM_FLUID = 0, MELBM_FLUID_BOUNDARY = 1, MELBM_INFLOW = 2, MELBM_OUTFLOW = 3,
       MELBM_SOLID = 4 };

/* Create a simulation (Sec. 4.2).  lattice is MELBM_D3Q27 or MELBM_D3Q19; tau > 1/2 is the
 * relaxation time (nu = (tau - 1/2)/3); storage is MELBM_F32 (40 B/cell per
 * buffer) or MELBM_Q16 (20 B/cell per buffer, Sec. 5.4).  Allocates two state
 * buffers on the current device, initialised to rest (rho = 1, u = 0, S = 0).
 * MELBM_MIXED is the paper's own mixed-precision scheme with solids (Sec. 5.4,
 * "Atomic accumulation with mixed precision"; kept for comparison): the
 * post-collision moments in 16 bits (20 B/cell) and the post-streaming raw moments
 * in FP32 (40 B/cell); a step is the fluid pass, the solid correction with
 * atomicAdd (halfway bounce-back), the outflow copy and the collision with
 * re-quantisation.  It supports solids, inflow and outflow, but not forces, bit
 * widths, the moving-wall model, solid forces, raw state or the adjoint
 * (MELBM_EINVAL).  N must be below 2^31.  *out receives the handle (NULL on
 * failure).
 * MELBM_D3Q19 (the 19-velocity lattice of Table 1's D3Q19 scene) keeps the same
 * ten stored moments, collision and storage forms; its post-collision populations
 * are the third-order Hermite expansion projected on the polynomials that lattice
 * carries (the xyz term vanishes on it; each pair of triples T_aab, T_bgg enters
 * through its sum and difference), which reproduces rho, rho u, rho S and the six
 * rho T_aab.  A D3Q19 handle takes the same boundaries over its 19 directions
 * (halfway bounce-back or the moving-wall model at solid cells, with their
 * momentum-exchange force and torque; inflow; outflow), with or without a body
 * force, in MELBM_F32 or MELBM_Q16 storage (any bit widths), the mixed scheme
 * (MELBM_MIXED) with its 19-velocity correction, and the adjoint. */
MELBM_API int melbm_create(int nx, int ny, int nz, int lattice, float tau, int storage, melbm_t* out);

/* Free every device and host resource of the handle.  NULL is accepted. */
MELBM_API int melbm_destroy(melbm_t h);

/* Stream on which all later work of the handle is enqueued (a cudaStream_t;
 * NULL = the legacy default stream).  Work already enqueued on the previous
 * stream is ordered before it (the new stream waits for it on the device). */
MELBM_API int melbm_set_stream(melbm_t h, void* cuda_stream);

/* Seed of the dither generator (Sec. 5.4 dithering), default 0.  The dither of
 * the state at time t is pcg4d(x, y, z, t ^ seed) (Jarzynski & Olano 2020). */
MELBM_API int melbm_set_seed(melbm_t h, uint32_t seed);

/* Set the state at time t = 0 from rho[N], u[3N] and S[6N] (S may be NULL, which
 * means S = u u, the equilibrium).  The pointers may be device or host memory
 * (pinned or pageable); host data is copied in on the handle's stream.  In
 * 16-bit storage the values are encoded with the dither of time index 0;
 * values outside the ranges saturate.  Resets the time index to 0. */
MELBM_API int melbm_set_state(melbm_t h, const float* rho, const float* u, const float* S);

/* Read the current state as FP32 (rho[N], u[3N], S[6N]; S may be NULL).
 * Device or host pointers; 16-bit storage is dequantised
 * m = m_min + q (m_max - m_min)/(2^16 - 1) (Sec. 5.4).  Values of SOLID cells are
 * unspecified (the fluid kernel updates them uniformly; nothing reads them). */
MELBM_API int melbm_get_moments(melbm_t h, float* rho, float* u, float* S);

/* Solid mask[N] (uint8, nonzero = solid; device pointer, NULL = no solid),
 * copied.  The classification and compaction kernels (analogue of the surface
 * marking of Sec. 4.2) then give every cell a type and a 27-bit mask whose bit i
 * is set iff x - c_i is SOLID (periodic wrap), and list the INFLOW and
 * FLUID_BOUNDARY cells in ascending n.  melbm_set_solid, melbm_set_inflow and
 * melbm_set_outflow only record their change: the classification runs once, at
 * the next call that needs the types or the list (melbm_step with n > 0,
 * melbm_get_boundary_list, melbm_get_types, melbm_reduce, melbm_solid_force,
 * melbm_forward_checkpointed, melbm_backward), which synchronises to read the list
 * length and returns the classification's MELBM_ENOMEM or MELBM_ECUDA if it
 * fails.  The lists are then freed, and those calls return MELBM_ESTATE until a
 * later melbm_set_solid / melbm_set_inflow / melbm_set_outflow. */
MELBM_API int melbm_set_solid(melbm_t h, const uint8_t* mask);

/* Equilibrium inflow on face 0 (x = 0): INFLOW cells are reset every step to
 * (rho, u, u u), i.e. the Hermite equilibrium of Sec. 3.2 (S = u u) with the given
 * density and velocity.  The paper's flow-past-solid scenes (Sec. 6.4 and Table 1)
 * drive the flow by an inlet without stating its form; this Dirichlet-equilibrium reading
 * is the one the oracle pins.  Typed and listed by the classification kernel
 * (INFLOW outranks OUTFLOW and FLUID_BOUNDARY); a pass over face 0 applies the
 * reset after the fluid kernel (split design of Sec. 4.2).  The classification
 * runs at the next call that needs it, as for melbm_set_solid.  Only face 0 is
 * supported: another face returns MELBM_EINVAL. */
MELBM_API int melbm_set_inflow(melbm_t h, int face, float rho, float ux, float uy, float uz);

/* Zero-gradient outflow on face 1 (x = nx-1): after each step OUTFLOW cells copy
 * the NEW stored state of (nx-2, y, z) (a cell of x = nx-1 is OUTFLOW only where
 * (nx-2, y, z) is not solid).  Like the inflow, the paper's flow-past-solid
 * scenes (Sec. 6.4) leave the outlet's form open; the zero-gradient copy is the reading
 * the oracle pins.  It runs as its own small pass after the fluid kernel and the
 * inflow reset, one thread per (y, z).  The classification runs at the next call that needs it,
 * as for melbm_set_solid.  Only face 1: another face returns MELBM_EINVAL. */
MELBM_API int melbm_set_outflow(melbm_t h, int face);

/* The compacted boundary-cell list built by the classification kernel -- the
 * voxel analogue of the surface marking that the paper's solid correction uses
 * to skip empty nodes (Sec. 4.2, "Accelerating solid intersection test"; Alg. 3
 * visits only marked nodes).  cells[k] = n in ascending order, words[k] =
 * (type << 27) | link mask, bit i of the mask set iff x - c_i is SOLID (periodic
 * wrap); the list holds the INFLOW and FLUID_BOUNDARY cells.  cells and words
 * are device pointers with room for `capacity` entries each (either may be
 * NULL); *count (host pointer) receives the list length even when it exceeds
 * capacity, in which case nothing is copied and MELBM_EINVAL is returned.
 * Synchronises the handle's stream when it copies. */
MELBM_API int melbm_get_boundary_list(melbm_t h, uint32_t* cells, uint32_t* words, int64_t capacity,
                            int64_t* count);

/* Cell types[N] (uint8, device pointer). */
MELBM_API int melbm_get_types(melbm_t h, uint8_t* types);

/* Body force F[3N] (device pointer, copied; NULL removes the force).  Applied
 * in the collision and in the moment recovery exactly as App. A and
 * Eq. rho_u_stress state (momentum gain F per step). */
MELBM_API int melbm_set_force(melbm_t h, const float* F);

/* Advance n >= 0 steps (Alg. 2 with the split design of Sec. 4.2), asynchronously
 * on the handle's stream.  One step is
 *   1. with solids, the bounce kernel over the compacted list (the solid
 *      correction of Sec. 4.2, done first): for each FLUID_BOUNDARY cell the sums
 *      of what its solid links return -- halfway bounce-back from the cell's own
 *      post-collision state, or the moment-based wall of Sec. 3.2 -- into a
 *      record per listed cell;
 *   2. the fluid update kernel (Alg. 2) over every cell: load (and in 16-bit
 *      storage dequantise, Sec. 5.4) the stored moments, collide in moment space
 *      (App. A), rebuild the post-collision populations (Eq. three_order_f),
 *      pull them from x - c_i (Eq. streaming; solid cells enter at rest, so a
 *      solid link brings nothing), add the record of each FLUID_BOUNDARY cell,
 *      re-form the moments (Eq. rho_u_stress) and store them once (16-bit:
 *      range-reduced, dithered and packed, Sec. 5.4), periodic in every
 *      direction.  MELBM_MIXED runs the paper's own additive atomicAdd
 *      correction and re-quantisation instead;
 *   3. with an inflow face, the reset of its INFLOW cells; with an outflow face,
 *      the zero-gradient copy onto x = nx-1.
 * In 16-bit storage at 16/16 bits without solids the rows of a fluid-kernel
 * block synchronise through per-row barriers whose waits are bounded
 * (milliseconds); a wait that runs out sets a word of the handle in mapped host
 * memory instead of hanging.
 * The state and time index advance by n.  Returns MELBM_EINVAL for n < 0 or a
 * NULL handle, MELBM_ESTATE after a failed boundary setup, the classification's
 * status when a pending one fails (melbm_set_solid), MELBM_ECUDA if a launch
 * fails or if a barrier wait of an earlier step ran out (the handle then refuses
 * further steps with MELBM_ESTATE until melbm_set_state, melbm_set_raw_state or
 * melbm_upload_raw_state_async gives it a new state).  Kernel faults surface at
 * the next synchronising call. */
MELBM_API int melbm_step(melbm_t h, int n);

/* FP64 total mass sum(rho) and kinetic energy sum(rho |u|^2 / 2) over non-solid
 * cells (host pointers; synchronises).  Diagnostics of the update rather than a
 * step of it: the fluid update conserves mass and momentum exactly in a periodic
 * box (its moments are sums of streamed populations, Eq. rho_u_stress), and
 * Sec. 5.4 motivates the dithered rounding by the drift that plain rounding
 * would add, so these two sums are what the conservation and kinetic-energy
 * checks of the 16-bit storage read.  Per cell the stored rho - 1 and
 * rho |u|^2 / 2 are summed in FP64 in a fixed order (deterministic).  In 16-bit
 * storage returns MELBM_WSATURATED (values still written) when any non-solid
 * code is 0 or 2^b - 1 (saturation, Sec. 5.4 ranges).  MELBM_EINVAL for NULL
 * pointers; MELBM_ECUDA (sums undefined) when a barrier wait of a step before
 * it ran out (see melbm_step). */
MELBM_API int melbm_reduce(melbm_t h, double* mass, double* kinetic_energy);

/* Steps taken since the last melbm_set_state (host pointer). */
MELBM_API int melbm_time_index(melbm_t h, int64_t* t);

/* Device bytes held by the handle (host pointer). */
MELBM_API int melbm_memory_bytes(melbm_t h, int64_t* bytes);

/* Raw packed state for bit-exact checkpoint/resume: bytes = 40 N (F32) or 20 N
 * (Q16); dst/src device or host.  set_raw_state also sets the time index. */
MELBM_API int melbm_state_bytes(melbm_t h, int64_t* bytes);
MELBM_API int melbm_get_raw_state(melbm_t h, void* dst, int64_t bytes);
MELBM_API int melbm_set_raw_state(melbm_t h, const void* src, int64_t bytes, int64_t time_index);

/* Asynchronous raw-state transfers, for moving a state to or from pinned host
 * memory while the GPU computes (with pageable host memory they still work but
 * do not overlap).  They run on two streams of the handle's own, in issue order
 * with the work already enqueued on the handle's stream, and return at once; the
 * caller must neither change src nor read dst before melbm_sync_transfers.  The
 * first upload allocates a third state buffer (melbm_state_bytes more device
 * memory, held until melbm_destroy).
 *   melbm_upload_raw_state_async: the state src (bytes as for set_raw_state)
 *     becomes the current state with time index time_index.  It lands in the
 *     third buffer, which then replaces the buffer of the current state, so it
 *     runs beside a step still in flight and beside a download of that step's
 *     result.
 *   melbm_download_raw_state_async: copies the current state into dst; a
 *     following melbm_step(h, 1) runs while it does (it reads that buffer and
 *     writes another one).
 *   melbm_sync_transfers: blocks until every transfer issued has completed.
 * melbm_step waits for the upload it steps from and for the downloads still
 * reading a buffer it overwrites; every other call that touches the state
 * waits for all transfers.  MELBM_MIXED storage returns MELBM_EINVAL. */
MELBM_API int melbm_upload_raw_state_async(melbm_t h, const void* src, int64_t bytes,
                                           int64_t time_index);
MELBM_API int melbm_download_raw_state_async(melbm_t h, void* dst, int64_t bytes);
MELBM_API int melbm_sync_transfers(melbm_t h);

/* Differentiation (not in the paper; inverse problems motivate it, Sec. 1).
 * melbm_forward_checkpointed: from the initial velocity u0[3N] (device) with
 * rho = 1 and S = u0 u0, runs nsteps FP32-storage steps with the current force,
 * storing a 16-bit checkpoint (deterministic rounding) every K steps; when
 * nsteps <= K it keeps every FP32 state instead (K + 1 states of 40 N bytes) and
 * the backward pass runs no recompute.
 * melbm_backward: given dL/d(rho, u, S) of the final state (10N device floats,
 * component-major as melbm_get_moments), writes dL/du0[3N] and dL/dF[3N]
 * (device; dL_dF may be NULL) by the hand-written discrete adjoint, recomputing
 * each segment in FP32 from its checkpoint.  With checkpoints the handle holds two
 * segment buffers (2 (K + 1) states of 40 N bytes) and recomputes segment s - 1 on
 * a stream of its own while the adjoint runs over segment s; the call returns
 * with all of its work ordered on the handle's stream.  Requires MELBM_F32 storage,
 * halfway bounce-back walls (wall model 0) and fewer than 429,496,730 cells
 * (10 N < 2^32; else MELBM_EINVAL); either lattice. */
MELBM_API int melbm_forward_checkpointed(melbm_t h, const float* u0, int nsteps, int K);
MELBM_API int melbm_backward(melbm_t h, const float* dL_dm_final, float* dL_du0, float* dL_dF);

/* 16-bit codec of Sec. 5.4 on caller buffers (device pointers), for tests and
 * tools.  stored[10][N] are the stored variables (rho, u, rho S^neq) in FP32;
 * words[5][N] holds codes (2k, 2k+1) in the low and high half of word k.
 * deterministic != 0 rounds to nearest (dither 1/2); otherwise the dither of
 * (x, y, z, t ^ seed).  cuda_stream may be NULL. */
MELBM_API int melbm_q16_encode(const float* stored, int nx, int ny, int nz, uint32_t t, uint32_t seed,
                     int deterministic, uint32_t* words, void* cuda_stream);
MELBM_API int melbm_q16_decode(const uint32_t* words, int64_t N, float* stored, void* cuda_stream);

/* Allocation-free diagnostics (this entry point has no counterpart in the paper;
 * it is a service for callers that cannot allocate device memory where they
 * need the numbers: a frame or control loop with a fixed memory budget, a host
 * whose device pool is owned by another allocator, or code that must avoid the
 * implicit synchronisation cudaMalloc/cudaFree can cause).  It computes what
 * melbm_reduce computes -- out[0] = sum(rho), out[1] = sum(rho |u|^2 / 2) over
 * non-solid cells, out[2] = number of non-solid 16-bit codes equal to 0 or 65535
 * (always 0 for MELBM_F32) -- from a raw state buffer the caller owns (the layout
 * of melbm_get_raw_state, storage MELBM_F32 or MELBM_Q16, N cells; type[N] as from
 * melbm_get_types, or NULL when no cell is solid).  out is a device pointer to 3
 * doubles, written asynchronously on cuda_stream (NULL = legacy stream).
 * It allocates nothing: its scratch is a fixed 96 KiB array inside the library,
 * held on every GPU that loads the library until the process exits, so N is
 * limited to 2^28 cells (larger N returns MELBM_EINVAL without any GPU work).
 * The first call on each device looks up the scratch address (cudaGetSymbolAddress)
 * with that device current and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset (or any destruction of
 * the device's primary context) may move the scratch and leaves that address
 * stale: do not use this call on a device after a reset.  All calls share the
 * scratch: calls that overlap on the GPU race and must be serialised by the
 * caller.  Q16 states are read on the default 16/16-bit grids only: a state
 * written after melbm_set_bits with other widths gives wrong numbers (the
 * call cannot tell).  Returns MELBM_EINVAL for bad arguments and MELBM_ECUDA if
 * the address lookup or a launch fails, with a message for
 * melbm_last_error(NULL). */
MELBM_API int melbm_reduce_state_noalloc(const void* state, int storage, int64_t N,
                                         const uint8_t* type, double* out, void* cuda_stream);

/* Solid walls (Sec. 3.2, solid coupling).  model 0 (default): halfway bounce-back,
 * f_i(x) = f+_opp(i)(x) for a solid link.  model 1: moment-based reconstruction --
 * the link receives the third-order Hermite population of (rho^p, u^p, S^p) with
 * rho^p = rho of x, u^p the velocity of the solid at the link's halfway point p
 * and S^p = u^p u^p + (S - u u) from the post-collision moments of x.  Solid cells
 * belong to bodies: the value of melbm_set_solid's mask (1..255) is the body id.
 * Body b moves rigidly: u^p = V + Omega x (p - r0), p in cell units with cell
 * (x, y, z) at (x, y, z); melbm_set_body_motion sets (V, Omega, r0) (host
 * pointers, NULL = zeros; bodies never set are at rest).  The geometry itself
 * does not move.  melbm_forward_checkpointed requires model 0 (MELBM_EINVAL). */
MELBM_API int melbm_set_wall_model(melbm_t h, int model);
MELBM_API int melbm_set_body_motion(melbm_t h, int body, const float* V, const float* Omega,
                                    const float* r0);

/* Force and torque (out[0..2], out[3..5], host, FP64) that the next step
 * transfers to the solid cells of body `body` (0: every solid; torques then each
 * about their own body's r0), by momentum exchange: every solid link i of a
 * FLUID_BOUNDARY cell adds -c_i (f_in + f_out), f_out = f+_opp(i)(x) and f_in
 * the population the wall returns; the torque adds (p - r0) x that.  Sums in a
 * fixed order (deterministic); synchronises.  Zero without solids. */
MELBM_API int melbm_solid_force(melbm_t h, int body, double* out);

/* Adaptive bit allocation (Sec. 6.2.2, "b_rho_u / b_S"): rho and u are stored
 * with bits_rho_u bits and rho S^neq with bits_S bits, each on the Sec. 5.4 grid
 * m_min + q (m_max - m_min)/(2^b - 1) (the same centre-anchored FP32 evaluation
 * and dither as the 16-bit codec), still two codes per 32-bit word.  Only for
 * MELBM_Q16 handles; 8 <= bits <= 16 each (else MELBM_EINVAL); 16/16 is the
 * default.  The current state is re-encoded (decoded on the old grids, encoded
 * on the new ones with the dither of the current time index); synchronises.
 * Every later step, set_state, get_moments and reduce use the new grids
 * (reduce counts codes on 0 or 2^b - 1).  Checkpoints of
 * melbm_forward_checkpointed and melbm_reduce_state_noalloc keep 16/16. */
MELBM_API int melbm_set_bits(melbm_t h, int bits_rho_u, int bits_S);

/* The codec of melbm_q16_encode / melbm_q16_decode with bit widths
 * bits_rho_u / bits_S (8..16 each, else MELBM_EINVAL): codes 0 .. 2^b - 1 in the
 * same word layout.  Device pointers; cuda_stream may be NULL. */
MELBM_API int melbm_codec_encode(const float* stored, int nx, int ny, int nz, uint32_t t,
                                 uint32_t seed, int deterministic, int bits_rho_u, int bits_S,
                                 uint32_t* words, void* cuda_stream);
MELBM_API int melbm_codec_decode(const uint32_t* words, int64_t N, int bits_rho_u, int bits_S,
                                 float* stored, void* cuda_stream);

/* Message of the last failure of h (or of the last handle-less call if h is
 * NULL).  Valid until the next call on the same handle. */
MELBM_API const char* melbm_last_error(melbm_t h);

#ifdef __cplusplus
}
#endif
#endif /* MELBM_H */
