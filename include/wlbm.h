/*
 * wlbm.h - C ABI of libwlbm, a GB300 (sm_103a) implementation of the worm lattice
 * Boltzmann method for the gray phonon Boltzmann transport equation (Hammer, Fritz,
 * Bedoya-Martinez, arXiv 1911.00180).
 *
 * Conventions for every entry point
 *  - Plain C types only.  "device" pointers are CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary CPU memory.
 *  - Calls that touch the GPU are asynchronous on the handle's stream unless stated;
 *    they return a wlbm_status and never abort or throw.  A failed call leaves a
 *    message readable with wlbm_last_error(handle) (or wlbm_last_error(NULL) for
 *    failures before a handle exists).
 *  - Lattice units: one grid spacing, one time step, group velocity v_g = 1.  The grid
 *    has nx x ny interior cells, row-major (x fastest).  Temperatures are absolute in
 *    kelvin except where a "dT" (deviation T - t_ref, kelvin) is named: deviations keep
 *    full float32 precision near 300 K.
 *  - The library owns the lattice state (two copies of Q direction planes, the local
 *    energy planes, the relaxation-weight plane); the caller owns every buffer it passes.
 */
#ifndef WLBM_H
#define WLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum wlbm_status {
  WLBM_OK = 0,
  WLBM_ERR_INVALID_ARG = 1, /* bad size, kind, pointer or Q (Q must be 8M, 8 <= Q <= 1024) */
  WLBM_ERR_UNSTABLE = 2,    /* max W_corr > 1: the paused step is unstable (Appendix A) */
  WLBM_ERR_OOM = 3,         /* the allocator returned NULL */
  WLBM_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
  WLBM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  WLBM_ERR_STATE = 6        /* call out of order (e.g. step before init) */
} wlbm_status;

/* Boundary kinds of Sec. 2.6 of the paper. */
enum {
  WLBM_BC_PERIODIC = 0,          /* periodic link to the opposite wall (must be paired) */
  WLBM_BC_ISOTHERMAL = 1,        /* isotropic blackbody wall, Eq. isotropic            */
  WLBM_BC_ADIABATIC_DIFFUSE = 2, /* adiabatic diffuse wall, Eq. adiabatic-diffuse;     *
                                  * partly specular with wlbm_boundary.specularity     */
  WLBM_BC_ADIABATIC_SPECULAR = 3 /* adiabatic specular wall, Eq. adiabatic-specular     */
};

/* Storage of the direction planes.  Both store the deviation of e_i from the reference
 * equilibrium w_i e_eq(t_ref); arithmetic is float32 in both. */
enum {
  WLBM_STORE_FP32_DEV = 0,  /* float32 deviation                                   */
  WLBM_STORE_BF16_DEV = 1   /* bfloat16 deviation divided by a per-run scale (RNE)  */
};

typedef struct wlbm_grid {
  int32_t nx, ny;      /* interior cells, >= 1 each; (nx+2)(ny+2) <= 2^31 - 1 and     */
                       /* ny <= 917488 (WLBM_ERR_INVALID_ARG otherwise)               */
  int32_t q;           /* directions Q = 8M of the worm-D2Q[8M] scheme (Sec. 2.5)       */
  int32_t storage;     /* WLBM_STORE_*                                                 */
  int32_t emulate_3d;  /* 1: apply the 3/2 factor of Eq. W-correction (2D emulating 3D) */
  int32_t relax_mode;  /* 0: W_corr as in Eq. W-correction (the paper).  1: opt-in
                          1 - exp(-W_corr), stable for MFP < 1 cell (not in the paper)  */
  double t_ref;        /* reference temperature, K (e.g. 300)                          */
  double theta;        /* hbar omega0 / k_B, K (624.8 for the paper's 81.8e12 rad/s)   */
  double speed;        /* propagation speed v in (0, 1] cells per step (0 means 1): the
                          TAS extended beyond the unit speed (Sec. 1) for one band of a
                          multigray run (Sec. 2.1).  The hop test of Eq. algorithm uses
                          v n in place of n, the relaxation per step is W = v / MFP
                          before Eq. W-correction, and the heat flux carries v_g = v.     */
} wlbm_grid;

/* Adiabatic walls (Sec. 2.6).  A ghost cell of a wall with specularity p in [0, 1] (1 for
 * WLBM_BC_ADIABATIC_SPECULAR, specularity[k] for WLBM_BC_ADIABATIC_DIFFUSE; the paper's
 * specular-diffusive wall is their linear combination) moves p of each outward component
 * to its mirror direction (normal component flipped, Eq. adiabatic-specular) and 1 - p to
 * the diffuse collection, which it re-emits into the inward directions with fractions
 * w_i (s_i . n) / sum_k w_k (s_k . n) (Eq. adiabatic-diffuse, normalised to conserve
 * energy); components parallel to the wall keep p of their value.  A corner between two
 * adiabatic walls uses the diffuse rule about the quadrant diagonal. */
typedef struct wlbm_boundary {
  int32_t kind[4];     /* WLBM_BC_* for the walls x-, x+, y-, y+                        */
  double t_wall[4];    /* wall temperature (K) of isothermal walls; ignored otherwise   */
  double specularity[4]; /* specular fraction of WLBM_BC_ADIABATIC_DIFFUSE walls, [0, 1]
                            (0: fully diffuse); ignored for other kinds                */
} wlbm_boundary;

/* Device-memory provider.  alloc returns a device pointer of at least `bytes` bytes
 * aligned to 256 bytes, or NULL (the library then fails with WLBM_ERR_OOM).  NULL for the
 * whole struct means cudaMalloc / cudaFree. */
typedef struct wlbm_allocator {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} wlbm_allocator;

typedef struct wlbm_handle wlbm_handle;

/* ---------------------------------------------------------------- lifecycle -------
 * wlbm_create: build the lattice for one grid (Sec. 2.2-2.5): the Q ring directions,
 * the angular weights (Eq. weight), the worm paths (Eq. worm-paths), Lambda_corr
 * (Eq. W-correction-factor-generalized) and the per-cell corrected relaxation weight
 * W_corr = f W (1 - W + W Lambda_corr), W = v / MFP (Eq. W-Kn and Eq. W-correction; v the
 * grid's propagation speed, 1 unless set).
 *   mfp_cells    device, nx*ny float32 mean free path in cells (row-major), or NULL to
 *                use mfp_uniform for every cell.  +inf gives W = 0 (ballistic).
 *   stream       cudaStream_t used for every later call (NULL = legacy default stream).
 * Fails with WLBM_ERR_UNSTABLE if any W_corr > 1 (relax_mode 0), WLBM_ERR_INVALID_ARG
 * for an unpaired periodic wall, Q not a multiple of 8, non-positive MFP or sizes, a
 * speed outside (0, 1] or a specularity outside [0, 1].
 * Synchronous (copies the MFP field to the host once).  The state starts at zero
 * deviation (uniform t_ref) and must be set by wlbm_init_temperature or wlbm_set_state.
 */
wlbm_status wlbm_create(const wlbm_grid* grid, const float* mfp_cells, double mfp_uniform,
                        const wlbm_boundary* bc, const wlbm_allocator* alloc,
                        void* stream, wlbm_handle** out);
void wlbm_destroy(wlbm_handle* h);
const char* wlbm_last_error(const wlbm_handle* h);
wlbm_status wlbm_set_stream(wlbm_handle* h, void* stream);

/* wlbm_init_temperature: local-equilibrium start e_i = w_i e_eq(t_ref + dT) in every
 * interior cell (Sec. 2.4: the weights set initial conditions); ghost cells copy their
 * nearest interior cell.  dT: device, nx*ny float32 (K).  Resets the step counter and
 * the TAS schedule.  With BF16 storage the per-run scale is set here from max |dT| and
 * the wall temperatures (synchronous in that case). */
wlbm_status wlbm_init_temperature(wlbm_handle* h, const float* dT);

/* wlbm_step: advance n >= 0 time steps.  Each step applies the wall conditions to the
 * ghost frame (Sec. 2.6), the internal sources (wlbm_set_sources) and the periodic links,
 * then the fused update of every cell and direction (Eq.
 * lbm-energy with e_i^eq = w_i E, Eq. lbm-energy-density, and the TAS rule of Eq.
 * algorithm along the worm paths of Eq. worm-paths). */
wlbm_status wlbm_step(wlbm_handle* h, int64_t n);
int64_t wlbm_step_count(const wlbm_handle* h);

/* wlbm_moments: temperature deviation T - t_ref by Eq. pseudo-T (computed in a
 * cancellation-free form) and heat flux q = v_g sum_i e_i s_i (Eq. q_corr, v_g the grid's
 * propagation speed) of the current state.  Each output is device nx*ny float32, or NULL
 * to skip it. */
wlbm_status wlbm_moments(wlbm_handle* h, float* dT, float* qx, float* qy);

/* wlbm_moments_mean: advance n >= 1 steps and write the means of the moments of
 * wlbm_moments over the n states reached (the running average over 10 steps of Sec. 4.3,
 * which smooths the step-to-step fluctuations of the TAS pauses).  Same outputs as
 * wlbm_moments (device nx*ny float32 each, or NULL); each term is weighted by 1/n and
 * added in float32 in step order. */
wlbm_status wlbm_moments_mean(wlbm_handle* h, int32_t n, float* dT, float* qx, float* qy);

/* wlbm_reduce: float64 reductions over the current state, written to host
 * out[WLBM_REDUCE_N].  On the GPU each cell's sums over its directions and its temperature
 * are float32 (as in wlbm_moments: the stored values are float32 or coarser); the sums and
 * the maximum over cells are float64, combined in a fixed order (the same bits on every
 * call for the same state).  Lattice units: cell =
 * step = v_g = 1, energy as E - e_ref with the paper's unit prefactor set to 1.
 *   out[0] sum over interior cells of E - e_ref   (energy conservation, Eq.
 *          lbm-energy-density)
 *   out[1] the same plus the ghost cells of adiabatic (diffuse or specular) walls
 *          (energy they hold; a corner counts when both its walls are adiabatic).
 *          Periodic ghosts are copies and isothermal ghosts the imposed reservoir, so
 *          neither counts.
 *   out[2] mean of q_x over interior cells, out[3] mean of q_y  (Eq. q_corr)
 *   out[4] mean of q_x over the central band of columns x0 <= x < x0 + m, x0 = nx / 4,
 *          m = nx / 2 (integer division; NaN if m < 1)
 *   out[5] least-squares slope dE/dx of the y-averaged E over that band (NaN if m < 2)
 *   out[6] apparent effective conductivity over the bulk one (Sec. 4.5; the paper calls
 *          it apparent, Sec. 1): out[2] * nx / (D (e(T_x-) - e(T_x+))), where D = MFP/3
 *          (grid.emulate_3d) or MFP/2 is the bulk diffusivity and e(T) = 1/(exp(theta/T)
 *          - 1); NaN unless both x walls are isothermal at different temperatures, and
 *          NaN for a per-cell MFP field
 *   out[7] band effective conductivity over the bulk one: out[4] / (-D out[5]), free of
 *          the temperature jumps at the x walls; NaN where out[5] is 0 or NaN, or for a
 *          per-cell MFP field
 *   out[8] steady-state residual: max over interior cells of |T^n - T^m| / (n - m) in
 *          K per step, n the current step and m the step of the previous wlbm_reduce on
 *          this handle (temperatures by Eq. pseudo-T); NaN on the first call
 *          after wlbm_init_temperature / wlbm_set_state / wlbm_adjoint_backward and when
 *          no step ran since the previous call.  Each call takes the next snapshot
 *          (library memory: nx*ny float64).
 * Synchronous. */
#define WLBM_REDUCE_N 9
wlbm_status wlbm_reduce(wlbm_handle* h, double* out);

/* wlbm_run_steady: run to steady state.  The TAS pauses (Eq. algorithm) make the field,
 * and above all the heat flux, fluctuate from step to step (Sec. 4.3: up to ~10 % of the
 * flux on coarse grids, less on finer ones), so the test compares window means: each
 * check runs check_every steps, the last avg_steps of them each followed by a reduction
 * (10 steps in Sec. 4.3) that adds T - T_ref of every interior cell to a float64 window
 * sum.  The residual of a check is max over interior cells of |mean of this window -
 * mean of the previous window| / check_every (K per step; NaN for the first window).
 * Checks repeat until the residual is <= tol or the next check would pass max_steps.
 *   steps_run  host int64 (may be NULL): steps taken (a multiple of check_every)
 *   converged  host int32 (may be NULL): 1 if the last residual was <= tol
 *   out        host double[WLBM_REDUCE_N] (may be NULL): out[2..5] are the means of the
 *              last window's avg_steps reductions, out[6..7] follow from those means,
 *              out[0..1] are those of the last step, out[8] is the last window residual.
 * Library memory: two nx*ny float64 planes, allocated on the first call.  Synchronous;
 * WLBM_ERR_INVALID_ARG unless max_steps >= check_every >= avg_steps >= 1 and tol >= 0. */
wlbm_status wlbm_run_steady(wlbm_handle* h, int64_t max_steps, int64_t check_every, double tol,
                            int32_t avg_steps, int64_t* steps_run, int32_t* converged,
                            double* out);

/* wlbm_get_state / wlbm_set_state: the deviations e_i - w_i e_ref of the current state,
 * unscaled float32, layout [Q][ny+2][nx+2] including the one-cell ghost frame (index
 * (y+1, x+1) is interior cell (x, y)).  device pointers.  set_state also recomputes the
 * local energy and keeps the step counter and schedule. */
wlbm_status wlbm_get_state(wlbm_handle* h, float* framed);
wlbm_status wlbm_set_state(wlbm_handle* h, const float* framed);

/* wlbm_set_sources: internal temperature and radiation sources (Sec. 2.6: the isotropic
 * blackbody and anisotropic radiation conditions are "equivalently" internal sources).
 * n cells (host int32 xy[2n]: x in [-1, nx], y in [-1, ny], not on the ghost frame of a
 * periodic side) whose DDEDs are overwritten at every step, after the wall pass and
 * before the periodic links, either with w_i e_eq(t[k]) (host double t[n], K; Eq.
 * isotropic) or, when e_imposed is given, with the imposed absolute DDEDs e_imposed[k][i]
 * (host double [n][Q]; Eq. anisotropic).  Sources on a wall's ghost cells make an
 * anisotropic radiation wall.  n = 0 removes all sources.  Each call replaces the previous
 * set (library memory).  Not for batch-owned handles (WLBM_ERR_STATE); the adjoint refuses
 * handles with sources (WLBM_ERR_STATE).  Synchronous. */
wlbm_status wlbm_set_sources(wlbm_handle* h, int32_t n, const int32_t* xy, const double* t,
                             const double* e_imposed);

/* wlbm_save / wlbm_load: checkpoint and resume.  A checkpoint holds the current state
 * planes as stored (framed, float32 or bfloat16), the local-energy plane (and, with
 * bfloat16 storage, the reference-energy plane), the storage scale and the schedule
 * cursor of Eq. algorithm (step n, per-direction displacement p_i and worm-hop counter,
 * plane buffer parity), so that stepping a loaded handle gives bit-for-bit the states of
 * the uninterrupted run.
 *   wlbm_save  dst: host buffer of capacity bytes, or NULL to only query the size;
 *              *written (host, may be NULL) receives the checkpoint size.  Synchronous.
 *              WLBM_ERR_INVALID_ARG if capacity is too small.
 *   wlbm_load  src: host buffer of size bytes written by wlbm_save for a handle of the same
 *              nx, ny, Q, storage and wall kinds (WLBM_ERR_INVALID_ARG otherwise, or for a
 *              truncated or corrupt header).  The handle's MFP field, wall temperatures and
 *              options are its own: load into a handle created with the same arguments.
 *              Only the frame of each plane is read from src (rows 1 .. ny+2 of the
 *              framed rows, the nx+2 framed columns): the pads of the library's planes
 *              stay zero whatever src holds there.  Clears the residual snapshot of
 *              wlbm_reduce and any adjoint forward run.  Synchronous.  Handles owned by a
 *              batch are not supported. */
wlbm_status wlbm_save(wlbm_handle* h, void* dst, size_t capacity, size_t* written);
wlbm_status wlbm_load(wlbm_handle* h, const void* src, size_t size);

/* ------------------------------------------------------------------------ adjoint --
 * Reverse-mode gradients of a run (the paper has no adjoint; the reverse step is the
 * exact transpose of Eq. lbm-energy / Eq. algorithm and of the wall passes of Sec. 2.6).
 * float32 storage only.
 *
 * wlbm_adjoint_forward: wlbm_init_temperature(dT0) followed by n_steps steps, saving the
 * state every ckpt_every steps (checkpoints, library memory: ceil(n/K) states plus K
 * states of recompute tape).  The handle's state afterwards is the final state.
 *   dT0  device nx*ny float32 start field (K), copied.
 *
 * wlbm_adjoint_backward: for an objective J of the final temperature field and heat flux
 * (Eq. pseudo-T, Eq. q_corr), given as its derivatives
 *   dJ_dT, dJ_dqx, dJ_dqy  device nx*ny float32 each: dJ/dT, dJ/dq_x, dJ/dq_y per interior
 *             cell (NULL: zero; at least one is needed).  The apparent conductivity of a
 *             film, mean q_x * nx / (D (e(T_x-) - e(T_x+))), has dJ_dqx = nx / (D de cells)
 *             everywhere; its explicit dependence on the wall temperatures through de
 *             is the caller's to add.
 * returns
 *   dJ_dmfp   device nx*ny float32: dJ / dMFP per cell (through W_corr, Eq. W-correction)
 *   dJ_dTwall host double[4]: dJ / dT_wall for isothermal walls (0 for other walls)
 *   dJ_ddT0   device nx*ny float32: dJ / d(start field)
 * (any output may be NULL).  Each segment between checkpoints is recomputed from its
 * checkpoint, then swept backwards.  Requires that the handle was not stepped after the
 * checkpointed forward run (WLBM_ERR_STATE otherwise).  Synchronous. */
wlbm_status wlbm_adjoint_forward(wlbm_handle* h, const float* dT0, int64_t n_steps,
                                 int32_t ckpt_every);
wlbm_status wlbm_adjoint_backward(wlbm_handle* h, const float* dJ_dT, const float* dJ_dqx,
                                  const float* dJ_dqy, float* dJ_dmfp, double* dJ_dTwall,
                                  float* dJ_ddT0);

/* wlbm_set_option: tuning knobs that do not change results.
 *   WLBM_OPT_STEP_VARIANT  0: step kernel with register-pipelined loads; 1: step kernel
 *                          with a per-warp ring of bulk async copies; 2: warp-specialised
 *                          step kernel (a producer warp issues the bulk copies of all
 *                          rows, consumer warps compute); 3 (default where the driver can
 *                          describe the planes as a TMA tensor, else 1): one tiled tensor
 *                          copy per direction and 128 x 14 tile, register-resident cell
 *                          data, directions processed grouped by hop kind.  Variants 0-2
 *                          give bit-identical results; variant 3 sums E' in another order
 *                          (equal up to float rounding).  Variant 3 computes ghost cells
 *                          only where an adiabatic-diffuse wall reads them: after a step
 *                          the ghost cells of periodic and isothermal sides hold what the
 *                          last boundary pass wrote (copies or wall values, not state).
 *                          Variant 3 never fuses the periodic mirrors: with
 *                          WLBM_OPT_FUSE_PERIODIC set it still runs the periodic pass.
 *   WLBM_OPT_GRAPH_STEPS   0 (default): launch every step's kernels directly; G > 0, a
 *                          multiple of 6: run chunks of G steps as one captured CUDA
 *                          graph (fewer launch gaps).  Replay needs a stream of its own:
 *                          on the legacy default stream (NULL) the steps are launched
 *                          directly, which WLBM_OPT_GRAPH_REPLAYS shows.
 *   WLBM_OPT_FUSE_PERIODIC 0 (default): a separate periodic pass before every step; 1:
 *                          when both axes are periodic the step kernel also writes the
 *                          ghost cells mirroring each edge cell (no separate pass).
 *   WLBM_OPT_GRAPH_REPLAYS read only (wlbm_get_option): how many chunks of steps this
 *                          handle has run as replays of a captured graph.
 *   WLBM_OPT_RING_STAGES   variant 3 ring depth of the tensor copies: 0 (default: by Q,
 *                          6 float32 / 6 bfloat16 for Q <= 64, else 4 / 8), or 6 or 4
 *                          (float32), 8 or 16 (bfloat16), or 6 (bfloat16: the form that
 *                          keeps the cell terms in shared memory, four blocks per SM; the
 *                          others keep them in registers, two blocks per SM).  bfloat16
 *                          single grids take these 128-column forms with
 *                          WLBM_OPT_BF16_WIDE = 0 or the tile loop; batches with
 *                          WLBM_OPT_BF16_WIDE = 0 take the cell-tile form with 8 stages.
 *   WLBM_OPT_TILE_LOOP     variant 3: 0 (default) one block per 128 x 14 tile; 1 a grid of
 *                          resident blocks that take the tiles in turn (no partial last
 *                          wave; bfloat16 runs three such blocks per SM where the ring
 *                          fits).  Same results bit for bit.
 *   WLBM_OPT_BF16_WIDE     variant 3, bfloat16 storage: 1 (default) tiles of 256 columns
 *                          read as one box of 32-bit words (pairs of columns) per direction,
 *                          two consumer warps per row pair, two blocks of 15 warps per SM
 *                          (one block per tile; the tile-loop option and the adjoint's
 *                          recompute keep the 128-column kernels); 0 tiles of 128 columns
 *                          (the forms WLBM_OPT_RING_STAGES selects).  Same results bit for
 *                          bit either way.  Setting 1 returns WLBM_ERR_INVALID_ARG for
 *                          float32 storage or where the planes have no tensor map.
 * wlbm_check: synchronises the stream and returns WLBM_ERR_TIMEOUT if a bounded wait
 * inside a kernel gave up since the last check (the status is then cleared). */
enum { WLBM_OPT_STEP_VARIANT = 1, WLBM_OPT_GRAPH_STEPS = 2, WLBM_OPT_FUSE_PERIODIC = 3,
       WLBM_OPT_GRAPH_REPLAYS = 4, WLBM_OPT_PERSISTENT = 5, WLBM_OPT_RING_STAGES = 6,
       WLBM_OPT_WAIT_LIMIT = 7, WLBM_OPT_STALL_TEST = 8, WLBM_OPT_TILE_LOOP = 9,
       WLBM_OPT_BF16_WIDE = 10 };
wlbm_status wlbm_set_option(wlbm_handle* h, int32_t key, int64_t value);
/* wlbm_get_option: the current value of a wlbm_set_option key in *value (host). */
wlbm_status wlbm_get_option(const wlbm_handle* h, int32_t key, int64_t* value);
wlbm_status wlbm_check(wlbm_handle* h);

/* wlbm_profile: CUDA-event timing of the fused step kernel on the handle's stream: an
 * event pair around every `every`-th step-kernel launch from this call on (1: every
 * launch; 0: off).  A stride above 1 keeps the event records off most steps, so the
 * steps between timed launches run as they do without profiling.  Under graph replay
 * (WLBM_OPT_GRAPH_STEPS = G) the timed launches are the steps t of each replayed chunk
 * with t % every == 0, recorded by event nodes of the graph; a graph's pairs are read
 * before it replays again (two chunks later: the host may wait for that replay to end).
 * Changing the stride drops the captured graphs.  WLBM_ERR_INVALID_ARG for every < 0.
 * wlbm_profile_read: synchronises the stream, returns the summed duration (ms) and count
 * of the timed step-kernel launches since the last read (then resets them), and the
 * number of kernels this handle has launched since it was created.  Any output may be
 * NULL. */
wlbm_status wlbm_profile(wlbm_handle* h, int32_t every);
wlbm_status wlbm_profile_read(wlbm_handle* h, double* step_ms, int64_t* step_launches,
                              int64_t* all_launches);

/* wlbm_reduce_state_noalloc: the first four float64 values of wlbm_reduce (same meaning
 * and order), computed from a caller-owned state instead of a handle, without allocating any
 * device memory.  The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory where they call it: code running inside a host
 * application that has reserved the device memory for its own pool, or a monitoring
 * hook in a latency-critical loop where an allocation (and the device synchronisation it
 * may imply) is not acceptable.
 *   framed   device float32 [q][ny+2][nx+2]: deviations e_i - w_i e_ref including the
 *            ghost frame, as written by wlbm_get_state
 *   speed    the band's propagation speed v_g in cells per step, (0, 1] (wlbm_grid.speed;
 *            1 for a single gray band): the mean fluxes out[2], out[3] carry it as
 *            wlbm_reduce's do (Eq. q_corr)
 *   bc_kind  host int32[4] wall kinds x-, x+, y-, y+ (decides which ghost cells count
 *            towards out[1])
 *   out      device double[4], written on the stream
 *   stream   cudaStream_t (NULL = legacy default stream)
 * Scratch: a file-scope device array of 1 MiB that every device loading the library keeps
 * until the process exits; it covers frames of up to 8,388,608 cells ((nx+2)*(ny+2)), and
 * larger frames (and a speed outside (0, 1]) are rejected with WLBM_ERR_INVALID_ARG and a
 * message.  The first call on a
 * device looks up the array's device address (once per device, with that device current);
 * make that first call before any stream capture.  Every call reuses the same array and
 * overwrites each entry it reads before reading it, so nothing needs clearing; calls whose
 * executions overlap on the GPU (other streams, other threads) race on it.  Asynchronous. */
wlbm_status wlbm_reduce_state_noalloc(const float* framed, int32_t nx, int32_t ny, int32_t q,
                                      double speed, const int32_t* bc_kind, double* out,
                                      void* stream);

/* wlbm_autotune: native search over WLBM_OPT_STEP_VARIANT (0 - 3) x WLBM_OPT_GRAPH_STEPS
 * (0 and the largest multiple of 6 <= trial_steps) for this grid: each candidate runs trial_steps (>= 6) steps after a warm-up; the fastest is kept
 * and returned (any output may be NULL).  The trial steps advance the state: call it
 * before wlbm_init_temperature. */
wlbm_status wlbm_autotune(wlbm_handle* h, int32_t trial_steps, int32_t* variant,
                          int32_t* graph_steps, double* ms_per_step);

/* -------------------------------------------------------------------------- batches --
 * Many independent grids (instances: films of different sizes, Knudsen numbers and Q)
 * advanced together; the multigray extension of Sec. 2.1 maps onto the same path.  Each
 * step is one wall launch and one step launch for the whole batch (the batched kernels
 * find their instance from the block index), optionally replayed as a CUDA graph.
 *   grids, bcs          host arrays of n entries (one storage type for all)
 *   mfp_cells           host array of n device pointers (NULL entries: uniform), or NULL
 *   mfp_uniform         host array of n uniform MFPs (used where mfp_cells[k] is NULL)
 * wlbm_batch_instance returns the handle of instance k (owned by the batch) for
 * moments, reductions and state access.  Options (wlbm_batch_set_option) are those of
 * wlbm_set_option, for every instance: WLBM_OPT_STEP_VARIANT 0, 1 or 3 (default 3 when
 * every instance has a tensor map), WLBM_OPT_GRAPH_STEPS, WLBM_OPT_FUSE_PERIODIC, and
 * WLBM_OPT_BF16_WIDE (bfloat16 per-step launches of variant 3 in 256-column tiles; default
 * 1 when every instance has a word tensor map; the persistent kernel keeps 128 columns).
 * Instances with a periodic axis whose edges the step kernel does not mirror get their own
 * periodic pass each step; graph replay then keeps one captured graph per starting
 * energy-plane phase of those instances (at most three).  Options of batches only:
 *   WLBM_OPT_PERSISTENT    0 (default): one wall launch and one step launch per step; 1:
 *                          one persistent launch per chunk of steps (64, or the
 *                          WLBM_OPT_GRAPH_STEPS of a replayed graph) on a fixed grid of
 *                          resident blocks that take, step by step, the wall chunks of
 *                          every instance and then the step tiles of every instance from a
 *                          queue, each item waiting only for the items of its own instance
 *                          it reads (results equal the
 *                          per-step launches of variant 3 bit for bit).  Needs variant 3
 *                          and no instance with a periodic axis (WLBM_ERR_INVALID_ARG).
 *                          Profiling then times whole launches: wlbm_batch_profile_read
 *                          reports their steps as step_launches.
 *   WLBM_OPT_RING_STAGES   ring depth of the persistent kernel's tensor copies: 0
 *                          (default: 6 float32, 8 bfloat16) or 4 (float32) / 16 (bfloat16).
 *   WLBM_OPT_WAIT_LIMIT    clock cycles a dependency wait of the persistent kernel may take
 *                          before it gives up (0, default: about two seconds); a wait that
 *                          gives up sets the status word of its instance, and every block
 *                          of the launch leaves (wlbm_batch_check reports it).
 *   WLBM_OPT_STALL_TEST    failure-detection hook for tests (0 default): 1 makes the step
 *                          tiles of instance 0 wait for one wall chunk more than exists,
 *                          so that their wait runs out after WLBM_OPT_WAIT_LIMIT cycles.
 *                          The states are then those of a partial step: initialise them
 *                          again before use. */
typedef struct wlbm_batch wlbm_batch;
wlbm_status wlbm_batch_create(int32_t n, const wlbm_grid* grids, const float* const* mfp_cells,
                              const double* mfp_uniform, const wlbm_boundary* bcs,
                              const wlbm_allocator* alloc, void* stream, wlbm_batch** out);
void wlbm_batch_destroy(wlbm_batch* b);
const char* wlbm_batch_last_error(const wlbm_batch* b);
int32_t wlbm_batch_size(const wlbm_batch* b);
wlbm_handle* wlbm_batch_instance(wlbm_batch* b, int32_t k);
/* dT: host array of n device pointers (nx*ny float32 each). */
wlbm_status wlbm_batch_init_temperature(wlbm_batch* b, const float* const* dT);
wlbm_status wlbm_batch_set_option(wlbm_batch* b, int32_t key, int64_t value);
wlbm_status wlbm_batch_get_option(const wlbm_batch* b, int32_t key, int64_t* value);
wlbm_status wlbm_batch_step(wlbm_batch* b, int64_t n);
wlbm_status wlbm_batch_profile(wlbm_batch* b, int32_t every);   /* as wlbm_profile */
/* wlbm_batch_check: synchronises the batch's stream and returns WLBM_ERR_TIMEOUT if a bounded
 * wait in a kernel of any instance gave up since the last check (the status words are
 * then cleared), as wlbm_check does for one handle. */
wlbm_status wlbm_batch_check(wlbm_batch* b);
wlbm_status wlbm_batch_profile_read(wlbm_batch* b, double* step_ms, int64_t* step_launches,
                                    int64_t* all_launches);
/* wlbm_batch_autotune: as wlbm_autotune over variants 0, 1 and 3 with per-step launches,
 * and, where the batch allows it, the persistent kernel at both of its ring depths, each
 * with and without graph replay (steps per launch: the graph's or 64), for the whole
 * batch (call before init).  The winner's options are set; WLBM_OPT_PERSISTENT and
 * WLBM_OPT_RING_STAGES report the persistent choice. */
wlbm_status wlbm_batch_autotune(wlbm_batch* b, int32_t trial_steps, int32_t* variant,
                                int32_t* graph_steps, double* ms_per_step);

/* ------------------------------------------------------------ host-only queries ----
 * No GPU needed.  wlbm_lattice: the lattice of Sec. 2.4-2.5 for Q directions.
 *   dirs      host int32[2Q] lattice vectors (x, y) of the ring directions, counter-
 *             clockwise from +x; weights host double[Q] (Eq. weight); worm host
 *             int8[Q*M] basic-hop indices K_{s,n} (Eq. worm-paths; hops numbered
 *             (1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)); lam_corr host
 *             double[1].  Any output may be NULL. */
wlbm_status wlbm_lattice(int32_t q, int32_t* dirs, double* weights, int8_t* worm,
                         double* lam_corr);

/* wlbm_schedule: the TAS schedule (Eq. algorithm) of steps 1..n_steps at propagation
 * speed v (wlbm_grid.speed; 0 means 1): host uint8[n_steps*Q]; entry [t][i] = hop index
 * (bits 0-2) | paused << 3. */
wlbm_status wlbm_schedule(int32_t q, int64_t n_steps, double speed, uint8_t* codes);

#ifdef __cplusplus
}
#endif
#endif /* WLBM_H */
