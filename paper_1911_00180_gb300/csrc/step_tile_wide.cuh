// bfloat16 step tiles 256 columns wide (single grids, WLBM_OPT_BF16_WIDE).
//
// The same update as the other variant-3 tiles (Eq. lbm-energy with the due worm hop of
// each direction, Eq. worm-paths, Eq. algorithm; E' = sum_i d_i', Eq. lbm-energy-density)
// in the cell-tile form, with the bfloat16 planes seen by the copy engine as 32-bit words:
// a tile of 256 columns plus 8 halo columns on each side is one box of 136 words x 14 rows
// (7.6 KB, the float32 kernel's box), where a 128-column bfloat16 box is 4 KB, so the copy
// engine moves half as many boxes for the same bytes.  Two consumer warps share a row
// pair, one per 128-column half, and a lane owns 4 cells of 2 rows as in the 128-column
// cell-tile form: a block is 14 consumer warps and a producer warp, two blocks per SM.
#pragma once
#include "step_tile.cuh"

namespace wlbm {

namespace {

constexpr int kWTW = 256;                    // tile columns
constexpr int kWBoxWords = kWTW / 2 + 8;     // box width in 32-bit words (8 halo bf16 a side)
constexpr int kWBW = 2 * kWBoxWords;         // ring row length in bfloat16 elements
constexpr int kWWarps = 2 * kWarps3;         // consumer warps: row pair w % 7, half w / 7
constexpr int kWThreads = 32 * (kWWarps + 1);
constexpr int kWCellG = kWTW / 4 + 2;        // groups of 4 cells: -1 .. 64
constexpr int kWCellArr = 4 * kCellRows * kWCellG;

template <int S>
struct WideLayout {
  static constexpr uint32_t kBoxBytes = uint32_t(kWBoxWords) * 4 * kRows3;
  static constexpr size_t kStage = (size_t(kBoxBytes) + 127) / 128 * 128;
  static constexpr size_t off_f = size_t(S) * kStage;
  static constexpr size_t f_bytes = size_t(3) * kWCellArr * 4;
  static constexpr size_t off_bar = (off_f + f_bytes + 127) / 128 * 128;
  static constexpr size_t off_kind = off_bar + 2 * S * 8;
  static constexpr size_t off_table = (off_kind + 17 * 4 + 127) / 128 * 128;
  static size_t bytes(int q) { return off_table + size_t(q) * sizeof(Dir3); }
};

struct WideIndex {
  __device__ int operator()(int rr, int cc) const { return cell_index<kWCellG>(rr, cc); }
};

// One 256 x 14 tile (bx, by) of one grid; `tmap` is the planes' tensor map over 32-bit
// words (box 136 x 14); cbase the first column of the first tile (a multiple of 8).
template <int S, bool FIELD_W>
__device__ __forceinline__ void step_tma_tile_wide(const StepArgs& a, const void* tmap, int cbase,
                                                   int bx, int by, unsigned char* smem) {
  using LY = WideLayout<S>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);
  uint64_t* empty = full + S;
  int* kind_start = reinterpret_cast<int*>(smem + LY::off_kind);
  Dir3* table = reinterpret_cast<Dir3*>(smem + LY::off_table);
  float* cells = reinterpret_cast<float*>(smem + LY::off_f);
  const int tid = int(threadIdx.y * blockDim.x + threadIdx.x);
  const int lane = tid & 31, ty = tid >> 5;
  const int col0 = cbase + bx * kWTW;
  const int row0 = a.rmin + by * kRows3;
  const int nrows = min(kRows3, a.rmax - row0 + 1);
  const int npairs = (nrows + kRPW - 1) / kRPW;      // row pairs with rows (two warps each)

  for (int k = tid; k <= 16; k += kWThreads) kind_start[k] = a.order[a.q + k];
  for (int j = tid; j < a.q; j += kWThreads) {
    const int i = a.order[j];
    const int code = a.codes[i];
    const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
    Dir3 d;
    d.dst = int64_t((paused ? par : 1 - par) * a.q + i) * a.plane;
    d.wi = a.w[i];
    d.zdy = (par * a.q + i) * 4 + (paused ? 0 : -c_hop_y[hop]) + 1;
    table[j] = d;
  }
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], npairs > 0 ? 2 * npairs : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows <= 0) return;

  if (ty == kWWarps) {
    if (lane != 0) return;
    for (int i = 0; i < a.q; ++i) {
      const int st = i % S, k = i / S;
      if (k > 0 && !mbar_wait(&empty[st], uint32_t(k - 1) & 1u, kWaitCycles)) {
        atomicOr(a.status, 1);
        for (int j = (i > S ? i - S : 0); j < i; ++j)   // copies still in flight
          mbar_wait(&full[j % S], uint32_t(j / S) & 1u, kWaitCycles);
        return;
      }
      const Dir3 d = table[i];
      mbar_expect(&full[st], LY::kBoxBytes);
      // word column (col0 - 8) / 2: col0 - 8 is a multiple of 8 bfloat16 (16 bytes)
      tma_load_3d(smem + st * LY::kStage, tmap, (col0 - 8) / 2, row0 + (d.zdy & 3) - 1,
                  d.zdy >> 2, &full[st]);
    }
    return;
  }

  // consumers: the cell tile (rows row0 - 1 .. row0 + 14, columns col0 - 1 .. col0 + 256)
  fill_cell_terms<kWTW, 5, WideIndex, 32 * kWWarps>(a, FIELD_W, col0, row0, tid, cells,
                                                    kWCellArr, WideIndex{});
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kWWarps) : "memory");
  const int rp = ty % kWarps3, half = ty / kWarps3;
  if (rp >= npairs) return;
  const int r = row0 + kRPW * rp;
  const int nrw = min(kRPW, a.rmax - r + 1);
  const int grp = 32 * half + lane;                  // the lane's group of 4 cells
  const int c0 = col0 + 4 * grp;
  const unsigned vm = lane_mask(a, c0);
  RegsB t;
#pragma unroll
  for (int k = 0; k < kRPW; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = r + k, c = c0 + j;
      const bool on = ((vm >> j) & 1u) && row < a.rows;
      t.eins[k][j] = on ? __fmul_rn(a.e_in[int64_t(row) * a.pitch + c], a.inv_scale) : 0.f;
      t.acc[k][j] = 0.f;
    }
  float accw = 0.f;
  DirCtx<__nv_bfloat16> ctx;
  ctx.cells = cells + 2 * rp * kWCellG + grp + 1;
  ctx.pitch = a.pitch;
  ctx.plane = a.plane;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = 0;
  __nv_bfloat16* obase = static_cast<__nv_bfloat16*>(a.planes) + int64_t(r) * a.pitch + c0;
  const int ring_off = kRPW * rp * kWBW + 4 * 32 * half;
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P, F)                                                           \
  ok = ok && run_kind_bf16<S, CX, CY, P, F, kWCellG, kWBW, LY::kStage>(                      \
                j, kind_start[K + 1], t, ctx, accw, table, smem, full, empty, obase, ring_off, \
                a.status)
  if (nrw == kRPW && __all_sync(0xffffffffu, vm == 0xFu)) {
    WLBM_KINDS16(WLBM_KIND, true);
  } else {
    WLBM_KINDS16(WLBM_KIND, false);
  }
#undef WLBM_KIND
  if (!ok) return;
  store_e_bf16(a, t, accw, r, nrw, c0, vm);
}

}  // namespace

}  // namespace wlbm
