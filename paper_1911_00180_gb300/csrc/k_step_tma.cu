// Step kernel variant 3: tensor-memory-access (TMA) tiles, register-resident cell data.
//
// Same update as the other step kernels (Eq. lbm-energy with the due worm hop c of each
// direction, Eq. worm-paths; E' = sum_i d_i', Eq. lbm-energy-density), organised so that
// the per-element work is a handful of instructions:
//   * one producer thread per block issues, for direction i, ONE tiled 3-D tensor copy of
//     the shifted source box (14 rows x 128 + 2V columns of plane par*q + i) into a stage
//     of a shared-memory ring; full/empty mbarriers pair it with 7 consumer warps.  Tall
//     boxes matter: the copy engine's throughput grows with the rows per box (7-row boxes
//     streamed less than half of what 14-16-row boxes do);
//   * a consumer warp owns 2 adjacent rows; a lane owns 4 consecutive cells of each and
//     keeps 1 - W and the source term of the 4 x 6 cells around them in registers, loaded
//     once per step (bfloat16 also keeps W E of those cells in a lane-private stretch of
//     shared memory, read only by paused directions);
//   * the directions of the step are processed sorted by kind (8 hops x paused or not;
//     the host sorts them, stably), as 16 loops with specialised bodies: every neighbour
//     index is a compile-time register, no per-direction indirect branch is taken, source
//     values arrive with one or two vector shared-memory loads, and results leave with
//     one 8- or 16-byte streaming store per lane and row.  E' sums the directions in that
//     order, so the result equals the other variants' up to float rounding.
// A block is 8 warps, so two blocks of up to 128 registers a thread fit on an SM.  Edge
// groups (columns past the right ghost) store element by element, so pad columns stay
// zero.  This kernel never mirrors periodic edges into the ghost frame (a separate
// periodic pass does).  It also serves the adjoint's tape mode: the recompute of a segment
// reads slot j of the tape through the tape's own tensor map and writes slot j + 1.
#include <cuda.h>

#include <algorithm>

#include "elem.cuh"
#include "mbar.cuh"
#include "step_tile.cuh"
#include "step_tile_wide.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

template <typename T, int S, bool FIELD_W, bool REF>
__global__ void __maxnreg__(128)
    k_step_tma(const StepArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t g0 = 0;
  // single grids: the register-tile form (two blocks per SM)
  step_tma_tile<T, S, FIELD_W, REF, false, false>(a, &tmap, int(blockIdx.x), int(blockIdx.y),
                                                  smem, g0);
}

// bfloat16 cell-tile form for single grids: the cell terms in the block-shared tile, so a
// block needs 64 registers a thread and, with a 6-stage ring, 51 KB of shared memory:
// four blocks per SM (28 consumer warps).
template <int S, bool FIELD_W>
__global__ void __launch_bounds__(32 * (kWarps3 + 1), 4)
    k_step_tma_cells(const StepArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t g0 = 0;
  step_tma_tile<__nv_bfloat16, S, FIELD_W, true, false, true>(a, &tmap, int(blockIdx.x),
                                                              int(blockIdx.y), smem, g0);
}

// bfloat16 wide-tile form for single grids: 256 x 14 tiles of the planes seen as 32-bit
// words (one 136-word box per direction), two consumer warps per row pair, the cell terms in
// the block-shared tile.  Two blocks of 15 warps per SM (a 6-stage ring of 7.6 KB boxes
// and a 50 KB cell tile each).
template <int S, bool FIELD_W>
__global__ void __launch_bounds__(kWThreads, 2)
    k_step_tma_wide(const StepArgs a, const __grid_constant__ CUtensorMap tmap, int cbase) {
  extern __shared__ __align__(128) unsigned char smem[];
  step_tma_tile_wide<S, FIELD_W>(a, &tmap, cbase, int(blockIdx.x), int(blockIdx.y), smem);
}

// Batched wide-tile form: block b belongs to instance tile_inst[b]; the instance's word
// tensor map sits in global memory.
template <int S>
__global__ void __launch_bounds__(kWThreads, 2)
    k_step_tma_batch_wide(const BatchInst* insts, const int* tile_inst, int t) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ const void* tm;
  __shared__ int tile[3];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int b = int(blockIdx.x);
    const BatchInst& I = insts[tile_inst[b]];
    sa = I.a;
    sa.codes = I.codes + size_t(t) * I.a.q;
    sa.order = I.order + size_t(t) * (I.a.q + 17);
    const int cur = (I.phase + t) % I.n_e;
    sa.e_in = I.e[cur];
    sa.e_out = I.e[(cur + 1) % I.n_e];
    sa.e_ref = I.e[(cur + 2) % 3];
    tm = I.tmap_w;
    const int local = b - I.first_tile_w;
    tile[0] = local % I.tiles_x_w;
    tile[1] = local / I.tiles_x_w;
    tile[2] = I.cbase_w;
  }
  __syncthreads();
  if (sa.wfield) step_tma_tile_wide<S, true>(sa, tm, tile[2], tile[0], tile[1], smem);
  else step_tma_tile_wide<S, false>(sa, tm, tile[2], tile[0], tile[1], smem);
}

// Tile-looping form: a grid of resident blocks (three per SM for bfloat16, whose cell
// terms sit in shared memory; two for float32) in which block b takes tiles b, b + grid,
// ... in turn, so no partial last wave of blocks idles the GPU, and whose producer streams
// the boxes of all its tiles without a pause at tile edges.
template <typename T>
constexpr int loop_min_blocks() { return sizeof(T) == 2 ? 3 : 2; }

template <typename T, int S, bool FIELD_W, bool REF>
__global__ void __launch_bounds__(32 * (kWarps3 + 1), loop_min_blocks<T>())
    k_step_tma_loop(const StepArgs a, const __grid_constant__ CUtensorMap tmap, int tiles_x,
                    int ntiles) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int fail;
  step_tma_loop<T, S, FIELD_W, REF>(a, &tmap, tiles_x, ntiles, smem, &fail);
}

// Batched form: block b belongs to instance tile_inst[b] (a host-built table: one load
// where a search over the instances' first tiles would take a chain of them); the
// instance's tensor map sits in global memory.
template <typename T, int S, bool REF>
__global__ void __maxnreg__(128) k_step_tma_batch(const BatchInst* insts, const int* tile_inst,
                                                  int t) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ const void* tm;
  __shared__ int tile[2];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int b = int(blockIdx.x);
    const BatchInst& I = insts[tile_inst[b]];
    sa = I.a;
    sa.codes = I.codes + size_t(t) * I.a.q;
    sa.order = I.order + size_t(t) * (I.a.q + 17);
    const int cur = (I.phase + t) % I.n_e;
    sa.e_in = I.e[cur];
    sa.e_out = I.e[(cur + 1) % I.n_e];
    sa.e_ref = I.n_e == 3 ? I.e[(cur + 2) % 3] : nullptr;
    tm = I.tmap;
    const int local = b - I.first_tile;
    tile[0] = local % I.tiles_x;
    tile[1] = local / I.tiles_x;
  }
  __syncthreads();
  uint32_t g0 = 0;
  if (sa.wfield) step_tma_tile<T, S, true, REF>(sa, tm, tile[0], tile[1], smem, g0);
  else step_tma_tile<T, S, false, REF>(sa, tm, tile[0], tile[1], smem, g0);
}

// BATCH: also the batched form of the same storage and ring depth.
template <typename T, int S, bool BATCH>
cudaError_t configure_tma_t() {
  const int bytes = int(TmaLayout<T, S>::bytes(kMaxQ));
  const void* fns[5] = {(const void*)k_step_tma<T, S, false, sizeof(T) == 2>,
                        (const void*)k_step_tma<T, S, true, sizeof(T) == 2>,
                        (const void*)k_step_tma_loop<T, S, false, sizeof(T) == 2>,
                        (const void*)k_step_tma_loop<T, S, true, sizeof(T) == 2>,
                        BATCH ? (const void*)k_step_tma_batch<T, S, sizeof(T) == 2> : nullptr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 5 && fns[k] && e == cudaSuccess; ++k) {
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // several blocks per SM: ask for the largest shared-memory carveout
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[k], cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
  }
  return e;
}

template <typename T, int S>
cudaError_t launch_tma_t(const StepArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  using LY = TmaLayout<T, S>;
  const dim3 block(32, kWarps3 + 1);
  const dim3 grid((a.cmax - a.cbase) / kTW3 + 1, (a.rmax - a.rmin + kRows3) / kRows3);
  const size_t bytes = LY::bytes(a.q);
  constexpr bool REF = sizeof(T) == 2;
  if (a.loop_blocks > 0 && !a.tape) {
    const int ntiles = int(grid.x * grid.y);
    const int nb = std::min(a.loop_blocks, ntiles);
    if (a.wfield)
      k_step_tma_loop<T, S, true, REF><<<nb, 32 * (kWarps3 + 1), bytes, s>>>(a, tm, int(grid.x),
                                                                             ntiles);
    else
      k_step_tma_loop<T, S, false, REF><<<nb, 32 * (kWarps3 + 1), bytes, s>>>(a, tm, int(grid.x),
                                                                              ntiles);
    return cudaGetLastError();
  }
  if (a.wfield) k_step_tma<T, S, true, REF><<<grid, block, bytes, s>>>(a, tm);
  else k_step_tma<T, S, false, REF><<<grid, block, bytes, s>>>(a, tm);
  return cudaGetLastError();
}

template <typename T, int S>
int loop_blocks_t(bool field_w, int q) {
  int per_sm = 0, dev = 0, sms = 0;
  const void* fn = field_w ? (const void*)k_step_tma_loop<T, S, true, sizeof(T) == 2>
                           : (const void*)k_step_tma_loop<T, S, false, sizeof(T) == 2>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * (kWarps3 + 1),
                                                    TmaLayout<T, S>::bytes(q)) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

constexpr int kStagesF32 = 6;    // 6 x 7.4 KB of boxes in flight per block
constexpr int kStagesBF16 = 8;   // 8 x 4 KB
// Ring depth by Q for single grids, from sweeps on 2048^2 x Q64 and 4096 x 256 x Q128:
// bfloat16 Q <= kDeepMaxQ takes 16 stages (Q64 0.223 -> 0.217 ms a launch against 8, while
// the Q128 film slowed from 0.108 to 0.114 ms); float32 Q > kDeepMaxQ takes 4 (Q128 film
// 0.181 -> 0.175 ms against 6, while Q64 slowed from 0.337 to 0.343 ms).  Batches keep
// kStagesF32 / kStagesBF16.
constexpr int kStagesBF16Deep = 16;
constexpr int kStagesF32Shallow = 4;
constexpr int kDeepMaxQ = 64;
// bfloat16 single grids with this ring depth run the cell-tile form (four blocks per SM)
constexpr int kStagesBF16Cells = 6;

template <int S>
cudaError_t configure_cells_t() {
  const int bytes = int(TmaLayout<__nv_bfloat16, S>::bytes(kMaxQ));
  const void* fns[2] = {(const void*)k_step_tma_cells<S, false>,
                        (const void*)k_step_tma_cells<S, true>};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[k], cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
  }
  return e;
}

template <int S>
cudaError_t launch_cells_t(const StepArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  const dim3 block(32, kWarps3 + 1);
  const dim3 grid((a.cmax - a.cbase) / kTW3 + 1, (a.rmax - a.rmin + kRows3) / kRows3);
  const size_t bytes = TmaLayout<__nv_bfloat16, S>::bytes(a.q);
  if (a.wfield) k_step_tma_cells<S, true><<<grid, block, bytes, s>>>(a, tm);
  else k_step_tma_cells<S, false><<<grid, block, bytes, s>>>(a, tm);
  return cudaGetLastError();
}

// Wide-tile ring depth by Q, from a sweep of 5, 6 and 7 stages: 2048^2 x Q64 0.1918 / 0.1901
// / 0.1890 ms a launch, the 4096 x 256 x Q128 film 0.0990 / 0.1012 / 0.1020 ms.
constexpr int kStagesBF16Wide = 7;        // Q <= kDeepMaxQ
constexpr int kStagesBF16WideHighQ = 5;

template <int S>
cudaError_t configure_wide_t() {
  const int bytes = int(WideLayout<S>::bytes(kMaxQ));
  const void* fns[3] = {(const void*)k_step_tma_wide<S, false>,
                        (const void*)k_step_tma_wide<S, true>,
                        (const void*)k_step_tma_batch_wide<S>};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[k], cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
  }
  return e;
}

// First column of the first wide tile: kX0, or with a computed left ghost column kX0 - 8
// (a multiple of 8 columns, so that every box starts on a 16-byte boundary).
int wide_cbase(const StepArgs& a) { return a.cmin < kX0 ? kX0 - 8 : kX0; }

template <int S>
cudaError_t launch_batch_wide_t(const BatchInst* insts, const int* tile_inst, int max_q,
                                int total_tiles, int t, cudaStream_t s) {
  k_step_tma_batch_wide<S><<<total_tiles, dim3(32, kWWarps + 1), WideLayout<S>::bytes(max_q),
                             s>>>(insts, tile_inst, t);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_wide_t(const StepArgs& a, const CUtensorMap& tm, cudaStream_t s) {
  const dim3 block(32, kWWarps + 1);
  const int cbase = wide_cbase(a);
  const dim3 grid((a.cmax - cbase) / kWTW + 1, (a.rmax - a.rmin + kRows3) / kRows3);
  const size_t bytes = WideLayout<S>::bytes(a.q);
  if (a.wfield) k_step_tma_wide<S, true><<<grid, block, bytes, s>>>(a, tm, cbase);
  else k_step_tma_wide<S, false><<<grid, block, bytes, s>>>(a, tm, cbase);
  return cudaGetLastError();
}

}  // namespace

cudaError_t configure_step_tma() {
  cudaError_t e = configure_tma_t<float, kStagesF32, true>();
  if (e == cudaSuccess) e = configure_tma_t<__nv_bfloat16, kStagesBF16, true>();
  if (e == cudaSuccess) e = configure_tma_t<__nv_bfloat16, kStagesBF16Deep, false>();
  if (e == cudaSuccess) e = configure_tma_t<float, kStagesF32Shallow, false>();
  if (e == cudaSuccess) e = configure_cells_t<kStagesBF16Cells>();
  if (e == cudaSuccess) e = configure_wide_t<kStagesBF16Wide>();
  if (e == cudaSuccess) e = configure_wide_t<kStagesBF16WideHighQ>();
  return e;
}

cudaError_t launch_step_tma_batch(int storage, const BatchInst* insts,
                                  const int* tile_inst, int n, int max_q,
                                  int total_tiles, int t, cudaStream_t s) {
  (void)n;
  if (total_tiles <= 0) return cudaSuccess;
  const dim3 block(32, kWarps3 + 1);
  if (storage == WLBM_STORE_BF16_DEV) {
    using LY = TmaLayout<__nv_bfloat16, kStagesBF16>;
    k_step_tma_batch<__nv_bfloat16, kStagesBF16, true>
        <<<total_tiles, block, LY::bytes(max_q), s>>>(insts, tile_inst, t);
  } else {
    using LY = TmaLayout<float, kStagesF32>;
    k_step_tma_batch<float, kStagesF32, false>
        <<<total_tiles, block, LY::bytes(max_q), s>>>(insts, tile_inst, t);
  }
  return cudaGetLastError();
}

void tma_cover_wide(const StepArgs& cover, int* cbase, int* tiles_x) {
  *cbase = wide_cbase(cover);
  *tiles_x = (cover.cmax - *cbase) / kWTW + 1;
}

cudaError_t launch_step_tma_batch_wide(const BatchInst* insts, const int* tile_inst, int n,
                                       int max_q, int total_tiles, int t, cudaStream_t s) {
  (void)n;
  if (total_tiles <= 0) return cudaSuccess;
  return max_q <= kDeepMaxQ
             ? launch_batch_wide_t<kStagesBF16Wide>(insts, tile_inst, max_q, total_tiles, t, s)
             : launch_batch_wide_t<kStagesBF16WideHighQ>(insts, tile_inst, max_q, total_tiles,
                                                          t, s);
}

int tma_tile_width() { return kTW3; }
int tma_tile_rows() { return kRows3; }

void tma_cover(const int bc_kind[4], int nx, int ny, StepArgs* a, int* tiles_x, int* tiles_y) {
  // ghost outputs are read only by the adiabatic-diffuse wall pass; periodic and isothermal
  // passes overwrite their ghost cells before the next step reads them
  const bool gl = bc_kind[0] == WLBM_BC_ADIABATIC_DIFFUSE;
  const bool gr = bc_kind[1] == WLBM_BC_ADIABATIC_DIFFUSE;
  const bool gb = bc_kind[2] == WLBM_BC_ADIABATIC_DIFFUSE;
  const bool gt = bc_kind[3] == WLBM_BC_ADIABATIC_DIFFUSE;
  a->cmin = gl ? kGhostCol : kX0;
  a->cmax = gr ? kX0 + nx : kX0 + nx - 1;
  a->rmin = gb ? 1 : 2;
  a->rmax = gt ? ny + 2 : ny + 1;
  a->cbase = gl ? kX0 - kTW3 : kX0;   // a left ghost column gets a tile of its own
  *tiles_x = (a->cmax - a->cbase) / kTW3 + 1;
  *tiles_y = (a->rmax - a->rmin + kRows3) / kRows3;
}

// Ring depth of a single-grid step: the explicit choice, else by Q (see above; bfloat16
// with Q <= kDeepMaxQ runs the cell-tile form, measured on 2048^2 x Q64 at 0.200 ms a
// launch against 0.202 for the 16-stage register form, and 0.058 against 0.062 ms on
// 1024^2 x Q64; the Q128 film keeps the 8-stage register form, 0.104 against 0.105 ms).
static int single_stages(int storage, int stages, int q) {
  if (storage == WLBM_STORE_BF16_DEV)
    return stages ? stages : (q <= kDeepMaxQ ? kStagesBF16Cells : kStagesBF16);
  return stages ? stages : (q <= kDeepMaxQ ? kStagesF32 : kStagesF32Shallow);
}

bool step_tma_stages_ok(int storage, int stages) {
  if (stages == 0) return true;
  if (storage == WLBM_STORE_BF16_DEV)
    return stages == kStagesBF16 || stages == kStagesBF16Deep || stages == kStagesBF16Cells;
  return stages == kStagesF32 || stages == kStagesF32Shallow;
}

int step_tma_loop_blocks(int storage, int stages, bool field_w, int q) {
  const int st = single_stages(storage, stages, q);
  if (storage == WLBM_STORE_BF16_DEV)
    return st == kStagesBF16Deep ? loop_blocks_t<__nv_bfloat16, kStagesBF16Deep>(field_w, q)
                                 : loop_blocks_t<__nv_bfloat16, kStagesBF16>(field_w, q);
  return st == kStagesF32 ? loop_blocks_t<float, kStagesF32>(field_w, q)
                          : loop_blocks_t<float, kStagesF32Shallow>(field_w, q);
}

cudaError_t launch_step_tma(int storage, const StepArgs& a, cudaStream_t s) {
  const CUtensorMap& tm = *static_cast<const CUtensorMap*>(a.tmap);
  const int st = single_stages(storage, a.ring_stages, a.q);
  if (storage == WLBM_STORE_BF16_DEV) {
    if (a.wide && a.tmap_w && !a.tape && a.loop_blocks == 0) {
      const CUtensorMap& tw = *static_cast<const CUtensorMap*>(a.tmap_w);
      return a.q <= kDeepMaxQ ? launch_wide_t<kStagesBF16Wide>(a, tw, s)
                              : launch_wide_t<kStagesBF16WideHighQ>(a, tw, s);
    }
    if (st == kStagesBF16Cells && !a.tape && a.loop_blocks == 0)
      return launch_cells_t<kStagesBF16Cells>(a, tm, s);
    return st == kStagesBF16Deep ? launch_tma_t<__nv_bfloat16, kStagesBF16Deep>(a, tm, s)
                                 : launch_tma_t<__nv_bfloat16, kStagesBF16>(a, tm, s);
  }
  return st == kStagesF32 ? launch_tma_t<float, kStagesF32>(a, tm, s)
                          : launch_tma_t<float, kStagesF32Shallow>(a, tm, s);
}

// Tensor map of the 2q direction planes as a 3-D tensor (columns, rows, planes) with the
// box of one TMA stage.  The encoder comes from the driver through the runtime's entry
// point query, so the library does not link the driver library directly.
bool make_plane_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                           std::string* why) {
  return make_box_tensor_map(out, planes, storage, g, nplanes, kRows3, why);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled tensor_map_encoder(std::string* why) {
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      *why = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  return encode;
}

// The bfloat16 planes as 32-bit words (pairs of columns): boxes of kWBoxWords words x kRows3
// rows for the wide-tile kernel.  The tensor ends at the word holding the right ghost
// column; when that word also holds the first pad column, the copy reads the pad from
// memory, where it is zero (pads are never written).
bool make_word_tensor_map(void* out, void* planes, const Geom& g, int nplanes,
                          std::string* why) {
  const EncodeTiled encode = tensor_map_encoder(why);
  if (!encode) return false;
  const cuuint64_t dims[3] = {cuuint64_t(kX0 + g.nx + 2) / 2, cuuint64_t(g.rows),
                              cuuint64_t(nplanes)};
  const cuuint64_t strides[2] = {cuuint64_t(g.pitch) * 2, cuuint64_t(g.plane) * 2};
  const cuuint32_t box[3] = {cuuint32_t(kWBoxWords), cuuint32_t(kRows3), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                            planes, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled failed with code " + std::to_string(int(r));
    return false;
  }
  return true;
}

bool make_box_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                         int box_rows, std::string* why, int box_cols) {
  const EncodeTiled encode = tensor_map_encoder(why);
  if (!encode) return false;
  const bool bf = storage == WLBM_STORE_BF16_DEV;
  const cuuint64_t es = bf ? 2 : 4;
  const cuuint32_t V = cuuint32_t(16 / es);
  // columns past the right ghost column are zero pads: as out-of-bounds columns of the
  // tensor the copy engine fills them with zeros without reading them
  const cuuint64_t dims[3] = {cuuint64_t(kX0 + g.nx + 1), cuuint64_t(g.rows),
                              cuuint64_t(nplanes)};
  const cuuint64_t strides[2] = {cuuint64_t(g.pitch) * es, cuuint64_t(g.plane) * es};
  const cuuint32_t box[3] = {box_cols > 0 ? cuuint32_t(box_cols) : cuuint32_t(kTW3) + 2 * V,
                             cuuint32_t(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(out),
                            bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                            3, planes, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled failed with code " + std::to_string(int(r));
    return false;
  }
  return true;
}

}  // namespace wlbm
