// Internal declarations shared by the C-ABI layer and the kernels of libwlbm.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wlbm.h"
#include "lattice.hpp"

namespace wlbm {

// Framed geometry of every plane (in cells, any element type).
//   rows: 0 = zero pad, 1 = ghost, 2..ny+1 = interior y = 0..ny-1, ny+2 = ghost,
//         ny+3 = zero pad.
//   cols: kGhostCol = ghost x = -1, kX0 = kGhostCol+1.. = interior, kX0+nx = ghost, the
//         column after it is a zero pad; columns before kGhostCol are zero pads.
// The interior starts on a 32-element boundary, so tiles of interior cells start 128-byte
// aligned (and tensor-copy boxes 16-byte aligned).  Pads are never written, so shifted
// reads past the frame read zero.
constexpr int kX0 = 32;
constexpr int kGhostCol = kX0 - 1;
constexpr int kMaxQ = 1024;
constexpr int kStepRows = 8;   // rows (warps) per block of the step kernels

struct Geom {
  int nx = 0, ny = 0, q = 0;
  int pitch = 0;        // elements per row, multiple of 32
  int rows = 0;         // ny + 4
  int64_t plane = 0;    // pitch * rows
  int64_t cell(int x, int y) const { return int64_t(y + 2) * pitch + (x + kX0); }
};

struct ParityMask {
  uint32_t bits[kMaxQ / 32];
};

// Stored plane values.  float32 storage keeps d_i = e_i - w_i e_ref directly.  bfloat16
// storage keeps v_i = (d_i - w_i R) / scale, where R is a per-cell reference energy: the
// local energy of the state that was read when the value was written (the previous
// step's E).  Near local equilibrium v is small, so the bfloat16 rounding error is small
// relative to the signal; R is kept in a third energy plane ("e_ref", nullptr for
// float32).  Every kernel that reads or writes plane values applies the same R.

// Step kernel arguments.
struct StepArgs {
  void* planes;          // [2][q][plane] elements of the storage type
  int64_t plane;         // elements per plane
  int pitch, rows, nx, ny, q;
  const uint8_t* codes;  // this step's codes [q]: hop | paused<<3 | parity<<4
  const float* w;        // weights [q]
  const float* e_in;     // local energy of the current state (framed, float32)
  const float* e_ref;    // reference of the stored current values (bfloat16 only)
  float* e_out;          // local energy of the new state
  const float* wfield;   // framed W_corr or nullptr (uniform)
  float w0;              // uniform W_corr of interior cells
  float scale, inv_scale;         // bfloat16 value scale and its inverse
  int xper, yper;        // periodic axes (uniform W: their ghost cells carry w0)
  int variant;           // 0: register-pipelined loads, 1: per-warp bulk-copy ring
  int* status;           // device status word: bit 0 set when a bounded wait gave up
  // tape mode (adjoint recompute): every plane i is read from planes + i*plane and
  // written to tape_dst + i*plane, whatever its parity or pause flag
  int tape;
  void* tape_dst;
  // both axes periodic: ghost rows/columns are not computed; instead every edge cell
  // also writes its new value (and E') into the ghost cells that mirror it, so the next
  // step needs no separate periodic pass
  int wrap;
  // host pointer to the planes' CUtensorMap (128 bytes, variant 3), or nullptr; read by
  // the launcher on the host, never by a kernel
  const void* tmap;
  // variant 3: this step's directions sorted by kind (hop | paused << 3, stable), q
  // entries, followed by the 17 starts of the 16 kinds; nullptr selects variant 1
  const uint16_t* order;
  // variant 3: the frame cells the step computes, columns cmin..cmax and rows rmin..rmax
  // (ghost cells only on adiabatic-diffuse sides: the other boundary passes overwrite
  // theirs before the next step), and the first column of the first tile
  int cmin, cmax, rmin, rmax, cbase;
  // variant 3 in tape mode: tensor-map plane index of plane 0 of the source slot
  int tape_z0;
  // variant 3, single grids: ring depth (0: by Q) and, when loop_blocks > 0, a grid of
  // that many blocks that each take every loop_blocks-th tile in turn (no last partial
  // wave of blocks); 0: one block per tile
  int ring_stages;
  int loop_blocks;
  // bfloat16 single grids: 1 = the wide-tile kernel (256-column tiles) through tmap_w, the
  // host pointer to the planes' 32-bit-word tensor map
  int wide;
  const void* tmap_w;
};

// Stable sort of one step's directions by kind = hop | paused << 3 (16 kinds): writes the
// sorted direction indices to out[0..q) and the start of every kind to out[q..q+17).
inline void sort_by_kind(const uint8_t* codes, int q, uint16_t* out) {
  uint16_t* start = out + q;
  for (int k = 0; k <= 16; ++k) start[k] = 0;
  for (int i = 0; i < q; ++i) ++start[(codes[i] & 15) + 1];
  for (int k = 0; k < 16; ++k) start[k + 1] = uint16_t(start[k + 1] + start[k]);
  uint16_t next[16];
  for (int k = 0; k < 16; ++k) next[k] = start[k];
  for (int i = 0; i < q; ++i) out[next[codes[i] & 15]++] = uint16_t(i);
}

#ifdef __CUDACC__
// Uniform W_corr of a frame cell: w0 inside the frame, 0 on pads and on the ghost cells of
// walls (wall cells do not scatter); periodic ghost cells carry w0.
__device__ __forceinline__ float uniform_w(const StepArgs& a, int r, int c) {
  if (r < 1 || r > a.ny + 2 || c < kGhostCol || c > kX0 + a.nx) return 0.f;  // pads
  const bool gx = (c == kGhostCol) || (c == kX0 + a.nx);
  const bool gy = (r == 1) || (r == a.ny + 2);
  if (gx && !a.xper) return 0.f;
  if (gy && !a.yper) return 0.f;
  return a.w0;
}
#endif

// Wall segment for the boundary kernel (one warp per ghost cell).
struct WallSeg {
  int count;             // ghost cells in this segment
  int r0, c0, dr, dc;    // first cell (row, col) and step between cells
  int action;            // 1 isothermal, 2 diffuse
  int table;             // diffuse re-emission table index into rho[]
  float iso;             // isothermal e_eq(T_w) - e_ref (times w_i per direction)
  int wall;              // wall (0..3) whose temperature an isothermal cell takes
  float spec;            // specularity p of an adiabatic edge (0: diffuse)
  int mirror;            // mirror table: 0 flips c_x (x walls), 1 flips c_y (y walls)
};
constexpr int kMaxSeg = 8;
struct WallArgs {
  void* planes;
  int64_t plane;
  int pitch, q, nseg;
  float* e_ref;          // reference energy of the stored values (bfloat16 only)
  float scale, inv_scale;
  const uint8_t* codes;  // current parity from the next step's codes
  const float* w;
  const float* rho;      // [8][q] re-emission fractions (0 = collected direction)
  const int16_t* mirror; // [2][q] direction index with c_x (row 0) or c_y (row 1) flipped
  int tape;              // 1: all planes at `planes` (parity ignored)
  int any_spec;          // a segment has specularity > 0 (selects the kernel with that path)
  WallSeg seg[kMaxSeg];
};

// Wall passes: a segment along a row (horizontal wall) is cut into chunks of
// kWallChunk consecutive cells, one block each, four consecutive cells per lane (one
// vector access per direction); other segments (vertical walls, corners) give every cell
// one warp, lanes over the directions, kWallCellsPerBlock cells a block.
constexpr int kWallChunk = 128;
constexpr int kWallCellsPerBlock = 8;
#ifdef __CUDACC__
__host__ __device__ inline bool wall_seg_rowwise(const WallSeg& g) {
  return g.dr == 0 && g.dc != 0 && g.count > 1;
}
__host__ __device__ inline int wall_seg_blocks(const WallSeg& g) {
  const int per = wall_seg_rowwise(g) ? kWallChunk : kWallCellsPerBlock;
  return (g.count + per - 1) / per;
}
__host__ __device__ inline int wall_chunk_count(int nseg, const WallSeg* seg) {
  int n = 0;
  for (int s = 0; s < nseg; ++s) n += wall_seg_blocks(seg[s]);
  return n;
}
// Segment of block `chunk` (nseg when out of range) and the block's index within it.
__host__ __device__ inline int wall_chunk_segment(int nseg, const WallSeg* seg, int chunk,
                                                  int* local) {
  int s = 0;
  while (s < nseg) {
    const int nb = wall_seg_blocks(seg[s]);
    if (chunk < nb) break;
    chunk -= nb;
    ++s;
  }
  *local = chunk;
  return s;
}
#endif


struct PeriodicArgs {
  void* planes;
  int64_t plane;
  int pitch, nx, ny, q;
  const uint8_t* codes;
  float* e_cur;          // local energy plane copied along with the direction planes
  float* e_ref;          // reference energy plane (bfloat16 only), copied likewise
  int xper, yper;
  int tape;              // 1: all planes at `planes` (parity ignored)
  const ParityMask* par; // if non-null, plane parities come from this mask, not codes
};

struct InitArgs {
  void* planes;
  int64_t plane;
  int pitch, nx, ny, q;
  const float* dT;       // interior nx*ny
  const float* w;
  float* e_cur;
  float* e_refp;         // reference energy plane (bfloat16 only): set to e_cur
  double t_ref, theta, e_ref;
  float scale, inv_scale;
};

struct MomentArgs {
  const void* planes;
  int64_t plane;
  int pitch, nx, ny, q;
  ParityMask par;
  const float* e_cur;
  const float* e_refp;
  const float* w;
  const float* sx;
  const float* sy;
  float* dT;
  float* qx;
  float* qy;
  float scale;
  float vg;              // propagation speed: q = v_g sum_i e_i s_i (Eq. q_corr)
  float weight;          // outputs take weight * moment (1 for plain moments)
  int accumulate;        // 1: add to the outputs instead of overwriting them
  float e_ref, e_ref1, l_ref, theta;   // e_ref, e_ref + 1, ln(1 + 1/e_ref), theta
};

struct ReduceArgs {
  const void* planes;
  int64_t plane;
  int pitch, nx, ny, q;
  ParityMask par;
  const float* e_cur;
  const float* e_refp;
  const float* w;
  const float* sx;
  const float* sy;
  double* out;           // [kReduceOut], written by the second stage
  double* part;          // [kReduceBlocks][kReduceOut] per-block partials (scratch)
  double scale;
  int diff_mask;         // bit k: side k (x-, x+, y-, y+) is an adiabatic-diffuse wall
  // central band of columns band_x0 <= x < band_x0 + band_w (conductivity fit)
  int band_x0, band_w;
  double band_xbar;      // mean column of the band
  // temperature residual: snap[y * nx + x] holds T - T_ref of the previous reduction (a
  // float32 per-cell value kept in float64); read where has_snap, always overwritten
  double* snap;
  int has_snap;
  double e_ref, e_ref1, l_ref, theta;   // e_ref, e_ref + 1, ln(1 + 1/e_ref), theta
  // window means of T - T_ref (steady-state test): win accumulates T over the reductions
  // of a window (set on its first, added on the others); on its last the mean win * win_inv
  // is compared with win_prev (where win_has_prev) and replaces it.  win == nullptr: off.
  double* win;
  double* win_prev;
  int win_first, win_last, win_has_prev;
  double win_inv;
};
// k_reduce outputs: [0] sum E interior, [1] + adiabatic-wall ghost cells, [2] sum q_x, [3] sum q_y,
// [4] sum q_x over the band, [5] sum (x - xbar) E over the band, [6] max |dT - dT_snap|,
// [7] max |window mean - previous window mean| (6, 7: bits of non-negative doubles,
// combined with an unsigned max).
constexpr int kReduceSums = 6;
constexpr int kReduceOut = 8;
constexpr int kReduceBlocks = 152 * 8;   // grid-stride blocks of the first stage

struct StateArgs {
  void* planes;
  int64_t plane;
  int pitch, nx, ny, q;
  ParityMask par;
  float* framed;         // [q][ny+2][nx+2]
  float* e_cur;
  const float* e_refp;
  const float* w;
  float scale, inv_scale;
};

// One instance of a batch: its constant step arguments plus what changes per step.  The
// batched kernels fill codes / e_in / e_out / e_ref for step t of the chunk from these.
struct BatchInst {
  StepArgs a;             // per-instance constants (codes, e_* are set per step)
  float* e[3];            // local-energy planes; roles rotate with the step
  const uint8_t* codes;   // this instance's codes of the chunk, [t][q]
  int n_e;                // 2 (float32) or 3 (bfloat16: with the reference plane)
  int phase;              // index of the current energy plane at the start of the chunk
  int tiles_x;            // step-kernel tiles per row
  int first_tile;         // first block of this instance in the batched grid
  const uint16_t* order;  // variant 3: kind-sorted directions of the chunk, [t][q + 17]
  const void* tmap;       // variant 3: device address of the instance's CUtensorMap
  int n_tiles;            // step-kernel tiles of this instance
  // bfloat16 256-column tiles (per-step launches with WLBM_OPT_BF16_WIDE): tiles per row,
  // first block in that batched grid, first column of the first tile, and the device
  // address of the instance's 32-bit-word tensor map
  int tiles_x_w, first_tile_w, cbase_w;
  const void* tmap_w;
};

struct BatchWalls {
  WallArgs w;             // per-instance wall segments (codes / e_ref set per step)
  float* e[3];
  const uint8_t* codes;
  int n_e, phase;
  int first_block;        // first block of this instance in the batched wall grid
  int n_blocks;           // wall blocks (chunks of ghost cells) of this instance
};

// Persistent batched kernel (variant 3 tiles and the wall pass in one launch for a chunk
// of steps): its work items are, for every step t of the chunk, the wall chunks of every
// instance (in instance order), then the step tiles of every instance, taken in that order
// from a queue.
// A wall chunk of instance k at step t waits until every tile of k's step t - 1 is done; a
// tile waits until every wall chunk of k's step t is done (and every tile of step t - 1).
struct PersistArgs {
  const BatchInst* insts;
  const BatchWalls* walls;
  const int* wall_inst;   // [wall_items] instance of every wall chunk of a step
  const int* tile_inst;   // [tile_items] instance of every step tile of a step
  int n;                  // instances
  int wall_items, tile_items;   // per step
  int steps;              // steps of this launch (codes of steps 0 .. steps-1 of the chunk)
  unsigned* ctr;          // [1 + 2n] zeroed before the launch: item queue, walls done per
                          // instance, tiles done per instance
  int* abort_flag;        // zeroed before the launch; set when a wait gave up
  long long wait_limit;   // clock cycles a dependency wait may take
  int stall_test;         // failure-detection test: instance 0's tiles wait for one wall
                          // chunk more than exists, so their wait runs out
};

// Reverse-step arguments (float32 storage only).
// The adjoint of a state is kept factored as l_k(x) = lh_k(x) + s(x): per-direction planes
// lh plus one plane s shared by all directions (the reverse relaxation adds the same
// W sigma to every direction of a cell, so it lands in s instead of in q planes).
struct AdjArgs {
  const float* lam_in;   // lh of the step's output, [q][plane]
  float* lam_out;        // lh of the step's input (before the boundary transposes)
  const float* s_in;     // s of the step's output (framed plane)
  float* s_out;          // s of the step's input
  const float* dtil;     // recorded step input (after the boundary pass), [q][plane]
  const uint8_t* codes;  // the step's codes
  const float* w;
  const float* wfield;   // framed W_corr or nullptr (uniform w0 with the frame rule)
  float w0;
  int xper, yper;
  float* gw;             // framed dJ/dW_corr accumulator
  int nx, ny, q, pitch;
  int64_t plane;
  // isothermal wall cells, transposed inside the reverse step: wall index (0..3) of the
  // edge cells of side k (x-, x+, y-, y+; corners excluded) and of corner k ((1, x-),
  // (1, x+), (ny+2, x-), (ny+2, x+)), or -1; their sum_i w_i l_i goes to gtw[wall]
  int iso_side[4], iso_corner[4];
  double* gtw;
};

#ifdef __CUDACC__
// W_corr of frame cell (r, c) for the reverse step: the framed field, or w0 by the frame
// rule (pads and wall ghosts 0).
__device__ __forceinline__ float w_at(const AdjArgs& a, int r, int c) {
  if (a.wfield) return a.wfield[int64_t(r) * a.pitch + c];
  if (r < 1 || r > a.ny + 2 || c < kGhostCol || c > kX0 + a.nx) return 0.f;
  const bool gx = (c == kGhostCol) || (c == kX0 + a.nx);
  const bool gy = (r == 1) || (r == a.ny + 2);
  if ((gx && !a.xper) || (gy && !a.yper)) return 0.f;
  return a.w0;
}

// Wall index of an isothermal wall cell (r, c), or -1.
__device__ __forceinline__ int iso_wall_of(const AdjArgs& a, int r, int c) {
  const bool xl = c == kGhostCol, xr = c == kX0 + a.nx, yb = r == 1, yt = r == a.ny + 2;
  if ((xl || xr) && (yb || yt)) return a.iso_corner[(yt ? 2 : 0) + (xr ? 1 : 0)];
  if (xl) return a.iso_side[0];
  if (xr) return a.iso_side[1];
  if (yb) return a.iso_side[2];
  if (yt) return a.iso_side[3];
  return -1;
}
#endif

// Sets the message returned by wlbm_last_error(NULL).
void set_global_error_msg(const std::string& m);

// Kernel launchers (k_step.cu, k_aux.cu).  Return cudaGetLastError().
cudaError_t launch_step(int storage, const StepArgs& a, cudaStream_t s);
cudaError_t prepare_step_kernels();   // per-device kernel attributes; call before capture
cudaError_t configure_walls();        // the same for the single-grid wall pass
// Variant 3 (TMA tiles): kernel attributes, launch, and the planes' tensor map (written to
// `out`, 128 bytes, 64-byte aligned; false with a reason when it cannot be made).
cudaError_t configure_step_tma();
cudaError_t launch_step_tma(int storage, const StepArgs& a, cudaStream_t s);
// Ring depths compiled for single grids (0 picks by Q) and the blocks of the tile-looping
// grid for this storage, depth, W kind and Q (resident blocks per SM x SMs; 0 on error).
bool step_tma_stages_ok(int storage, int stages);
int step_tma_loop_blocks(int storage, int stages, bool field_w, int q);
// Batched variant 3 (one block per 128 x 14 tile of every instance) and its tile shape.
cudaError_t launch_step_tma_batch(int storage, const BatchInst* insts,
                                  const int* tile_inst, int n, int max_q,
                                  int total_tiles, int t, cudaStream_t s);
int tma_tile_width();
int tma_tile_rows();
// Cells and tiles of a variant-3 step for sides of the given kinds (x-, x+, y-, y+):
// sets a->cmin..cbase, returns the tile counts along x and y.
void tma_cover(const int bc_kind[4], int nx, int ny, StepArgs* a, int* tiles_x, int* tiles_y);
bool make_plane_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                           std::string* why);
// The same with a box of box_rows rows (the 128 + 2V columns of a tile).
bool make_box_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                         int box_rows, std::string* why, int box_cols = 0);
// bfloat16 planes as 32-bit words with the wide-tile kernel's box (136 words x 14 rows).
bool make_word_tensor_map(void* out, void* planes, const Geom& g, int nplanes,
                          std::string* why);
// 256-column tiles of a variant-3 step whose covered cells tma_cover set in `cover`: the
// first column of the first tile and the tiles per row.
void tma_cover_wide(const StepArgs& cover, int* cbase, int* tiles_x);
// One step of every instance of a batch in 256-column bfloat16 tiles (total_tiles of them).
cudaError_t launch_step_tma_batch_wide(const BatchInst* insts, const int* tile_inst, int n,
                                       int max_q, int total_tiles, int t, cudaStream_t s);
// Reverse step with TMA tiles (float32): lam_map describes the q planes of a.lam_in with
// boxes of kAdjTmaBoxRows rows (paused directions with a vertical hop component read both x
// and x + c_k), lam_map14 the same planes with boxes of kAdjTmaRows rows (propagating
// directions read x + c_k only; paused horizontal hops x and x + c_k of the same rows),
// tape_map the adjoint tape with boxes of kAdjTmaRows rows of the tile's kAdjTmaCols columns
// (no column halo); tape_z0 is the plane index of the step's slot in the tape, order the
// step's kind-sorted directions.
constexpr int kAdjTmaBoxRows = 15;
constexpr int kAdjTmaRows = 14;
constexpr int kAdjTmaCols = 128;
cudaError_t configure_adj_tma();
cudaError_t launch_adj_tma(const AdjArgs& a, const void* lam_map, const void* lam_map14,
                           const void* tape_map, int tape_z0, const uint16_t* order,
                           int* status, cudaStream_t s);
// Batched launches (one launch per step for all instances of a batch).
int step_tile_width(int storage, int variant);
cudaError_t launch_step_batch(int storage, int variant, const BatchInst* insts, int n,
                              int total_tiles, int t, cudaStream_t s);
int wall_blocks(const WallArgs& a);   // blocks of the wall pass of one grid (32 cells each)
cudaError_t launch_walls_batch(int storage, const BatchWalls* b, const int* block_inst,
                               int total_blocks, int t, bool any_spec, cudaStream_t s);
// Persistent batched kernel (k_batch_persistent.cu): attributes, resident blocks per SM and
// one launch of p.steps steps on `grid` blocks (ring depth `stages`: 0 takes the default).
cudaError_t configure_batch_persistent();
int batch_persistent_blocks_per_sm(int storage, int stages, int max_q);
bool batch_persistent_stages_ok(int storage, int stages);
cudaError_t launch_batch_persistent(int storage, int stages, const PersistArgs& p, int max_q,
                                    int grid, bool any_spec, cudaStream_t s);
cudaError_t launch_walls(int storage, const WallArgs& a, cudaStream_t s);
cudaError_t launch_periodic(int storage, const PeriodicArgs& a, cudaStream_t s);
cudaError_t launch_init(int storage, const InitArgs& a, cudaStream_t s);
cudaError_t launch_moments(int storage, const MomentArgs& a, cudaStream_t s);
cudaError_t launch_reduce(int storage, const ReduceArgs& a, cudaStream_t s);
cudaError_t launch_get_state(int storage, const StateArgs& a, cudaStream_t s);
cudaError_t launch_set_state(int storage, const StateArgs& a, cudaStream_t s);
// Adjoint launchers (k_adjoint.cu).
cudaError_t launch_adj_step(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_periodic_T(float* planes, int64_t plane, int pitch, int nx, int ny,
                              int nplanes, int xper, int yper, cudaStream_t s);
// Transposed wall pass after the periodic transpose.  Isothermal cells were transposed by
// the reverse step: only the two end cells of each isothermal segment (where the periodic
// transpose of the other axis may have added corner images) are transposed again.
cudaError_t launch_walls_T(const WallArgs& wa, float* lam, double* gtw, cudaStream_t s);
// Internal sources and radiation cells: framed cells whose deviations are overwritten
// every step (after the wall pass, before the periodic pass) with fixed values.
struct SourceArgs {
  void* planes;
  int64_t plane;
  int q, n;
  const int64_t* off;    // [n] framed offsets within a plane
  const float* val;      // [n][q] deviations d_i to impose
  const float* esum;     // [n] their sum (the cell's local energy deviation)
  float* e_cur;          // local-energy plane of the current state
  float* e_ref;          // reference-energy plane (bfloat16 only)
  const float* w;
  const uint8_t* codes;  // current parity from the next step's codes
  float inv_scale;
};
cudaError_t launch_sources(int storage, const SourceArgs& a, cudaStream_t s);

cudaError_t launch_adj_seed(const AdjArgs& a, const float* dJ_dT, const float* dJ_dqx,
                            const float* dJ_dqy, const float* sx, const float* sy, float vg,
                            const float* e_final, double e_ref, double theta, cudaStream_t s);
cudaError_t launch_adj_final(const AdjArgs& a, const float* dwc, float* dJ_dmfp,
                             const float* lam0, const float* s0, const float* dT0,
                             float* dJ_ddT0, double t_ref, double theta, cudaStream_t s);

}  // namespace wlbm
