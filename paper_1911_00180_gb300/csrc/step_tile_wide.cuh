// bfloat16 step tiles 256 columns wide (single grids, WLBM_OPT_BF16_WIDE).
//
// The same update as the other variant-3 tiles (Eq. lbm-energy with the due worm hop of
// each direction, Eq. worm-paths, Eq. algorithm; E' = sum_i d_i', Eq. lbm-energy-density)
// in the cell-tile form, with the bfloat16 planes seen by the copy engine as 32-bit words:
// a tile of 256 columns plus 8 halo columns on each side is one box of 136 words x 14 rows
// (7.6 KB, the float32 kernel's box), where a 128-column bfloat16 box is 4 KB.  A lane owns
// 8 consecutive cells of 2 rows: one 16-byte ring read and one 16-byte store per row and
// direction.
#pragma once
#include "step_tile.cuh"

namespace wlbm {

namespace {

constexpr int kWTW = 256;                    // tile columns
constexpr int kWBoxWords = kWTW / 2 + 8;     // box width in 32-bit words (8 halo bf16 a side)
constexpr int kWCellG = kWTW / 8 + 2;        // groups of 8 cells: -1 .. 32
constexpr int kWCellArr = 8 * kCellRows * kWCellG;

// Cell tile: column col0 + 8 g + p (local column cc = 8 g + p + 1) at [p][rr][g + 1].
__device__ __forceinline__ int wcell_index(int rr, int cc) {
  const int x = cc - 1;
  return ((x & 7) * kCellRows + rr) * kWCellG + (x >> 3) + 1;
}
// Offset from a lane's base (cells + 2 ty * kWCellG + lane + 1) of position (lr, lc): row
// r - 1 + lr, column c0 - 1 + lc (c0 = col0 + 8 lane).
__host__ __device__ constexpr int wcell_off(int lr, int lc) {
  return (((lc + 7) & 7) * kCellRows + lr) * kWCellG + (lc == 0 ? -1 : (lc - 1) / 8);
}

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

struct RegsW {
  float eins[kRPW][8];
  float acc[kRPW][8];
};

// Source values of the lane's 8 cells for a DDED shift DX as four pairs, from a box row
// of 32-bit words (the lane's cells start at word 4 + 4 lane).
template <int DX>
__device__ __forceinline__ void ring_pairs8(const uint32_t* row, int lane, float2 (&v)[4]) {
  const uint32_t* p = row + 4 + 4 * lane;      // 16-byte aligned
  const uint4 q = *reinterpret_cast<const uint4*>(p);
  if constexpr (DX == 0) {
    v[0] = make_float2(bf_lo(q.x), bf_hi(q.x));
    v[1] = make_float2(bf_lo(q.y), bf_hi(q.y));
    v[2] = make_float2(bf_lo(q.z), bf_hi(q.z));
    v[3] = make_float2(bf_lo(q.w), bf_hi(q.w));
  } else if constexpr (DX < 0) {
    v[0] = make_float2(bf_hi(p[-1]), bf_lo(q.x));
    v[1] = make_float2(bf_hi(q.x), bf_lo(q.y));
    v[2] = make_float2(bf_hi(q.y), bf_lo(q.z));
    v[3] = make_float2(bf_hi(q.z), bf_lo(q.w));
  } else {
    v[0] = make_float2(bf_hi(q.x), bf_lo(q.y));
    v[1] = make_float2(bf_hi(q.y), bf_lo(q.z));
    v[2] = make_float2(bf_hi(q.z), bf_lo(q.w));
    v[3] = make_float2(bf_hi(q.w), bf_lo(p[4]));
  }
}

// bfloat16 store of the lane's 8 new values of one row (mask vm: bit j = cell j computed);
// returns the packed words.
__device__ __forceinline__ uint4 store8_bf16(__nv_bfloat16* dst, const float2 (&o)[4],
                                             unsigned vm) {
  uint32_t w[4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const __nv_bfloat162 p = __float22bfloat162_rn(o[h]);
    w[h] = *reinterpret_cast<const uint32_t*>(&p);
  }
  if (vm == 0xFFu) {
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(w[0], w[1], w[2], w[3]));
  } else {
    unsigned short* d = reinterpret_cast<unsigned short*>(dst);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((vm >> j) & 1u)
        __stcs(d + j, static_cast<unsigned short>(j & 1 ? w[j >> 1] >> 16 : w[j >> 1] & 0xffffu));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

struct CtxW {
  const uint32_t* ring_row;   // the warp's first row in the stage (32-bit words)
  __nv_bfloat16* dst;         // the lane's first cell in the warp's first row, plane i
  const float* cells;         // the lane's base in the cell tile
  int64_t pitch;
  float wi;
  int lane, nrw;
  unsigned vm;
  uint32_t g0;
};

template <int CX, bool PAUSED, bool FULL>
__device__ __forceinline__ void dir_body_w(RegsW& t, const CtxW& c, const float2 (&Gk)[kRPW][4],
                                           const float2 (&Dk)[kRPW][4]) {
  constexpr int DX = PAUSED ? 0 : -CX;
  const float2 wi2 = make_float2(c.wi, c.wi);
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (!FULL && k >= c.nrw) break;
    float2 v[4];
    ring_pairs8<DX>(c.ring_row + k * kWBoxWords, c.lane, v);
    float2 o[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) o[h] = __ffma2_rn(Gk[k][h], v[h], __fmul2_rn(wi2, Dk[k][h]));
    const uint4 w = store8_bf16(c.dst + k * c.pitch, o, FULL ? 0xFFu : c.vm);
    add_bf16x2(w.x, t.acc[k][0], t.acc[k][1]);
    add_bf16x2(w.y, t.acc[k][2], t.acc[k][3]);
    add_bf16x2(w.z, t.acc[k][4], t.acc[k][5]);
    add_bf16x2(w.w, t.acc[k][6], t.acc[k][7]);
  }
}

// All directions of one kind; the per-kind terms from the cell tile as in run_kind_bf16.
template <int S, int CX, int CY, bool PAUSED, bool FULL>
__device__ __forceinline__ bool run_kind_w(int& j, int end, RegsW& t, CtxW& c, float& accw,
                                           const Dir3* table, const unsigned char* smem,
                                           uint64_t* full, uint64_t* empty,
                                           __nv_bfloat16* obase, int ty, int* status) {
  using LY = WideLayout<S>;
  if (j >= end) return true;
  float2 Gk[kRPW][4], Dk[kRPW][4];
  {
    const float* G = c.cells;
    const float* X = c.cells + kWCellArr;
    const float* F = c.cells + 2 * kWCellArr;
    constexpr int SC = PAUSED ? 1 : 1 - CX;
    constexpr int FC = 1 - CX;
#pragma unroll
    for (int k = 0; k < kRPW; ++k) {
      const int SR = PAUSED ? 1 + k : 1 + k - CY;
      const int FR = 1 + k - CY;
      float g[8], d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        g[q] = G[wcell_off(SR, SC + q)];
        const float tt =
            PAUSED ? __fadd_rn(__fsub_rn(X[wcell_off(1 + k, 1 + q)], F[wcell_off(1 + k, 1 + q)]),
                               F[wcell_off(FR, FC + q)])
                   : X[wcell_off(SR, SC + q)];
        d[q] = __fsub_rn(tt, t.eins[k][q]);
      }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        Gk[k][h] = make_float2(g[2 * h], g[2 * h + 1]);
        Dk[k][h] = make_float2(d[2 * h], d[2 * h + 1]);
      }
    }
  }
  for (; j < end; ++j) {
    const uint32_t gj = c.g0 + uint32_t(j);
    const int st = int(gj % S);
    if (!mbar_wait(&full[st], (gj / S) & 1u, kWaitCycles)) {
      if (c.lane == 0) atomicOr(status, 1);
      return false;
    }
    const Dir3 d = table[j];
    c.ring_row = reinterpret_cast<const uint32_t*>(smem + st * LY::kStage) + kRPW * ty * kWBoxWords;
    c.dst = obase + d.dst;
    c.wi = d.wi;
    accw += d.wi;
    if (FULL || c.vm) dir_body_w<CX, PAUSED, FULL>(t, c, Gk, Dk);
    __syncwarp();
    mbar_arrive_if(&empty[st], c.lane == 0);
  }
  return true;
}

// One 256 x 14 tile (bx, by) of one grid; `tmap` is the planes' tensor map over 32-bit
// words (box 136 x 14); cbase the first column of the first tile.
template <int S, bool FIELD_W>
__device__ __forceinline__ void step_tma_tile_wide(const StepArgs& a, const void* tmap, int cbase,
                                                   int bx, int by, unsigned char* smem) {
  using LY = WideLayout<S>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);
  uint64_t* empty = full + S;
  int* kind_start = reinterpret_cast<int*>(smem + LY::off_kind);
  Dir3* table = reinterpret_cast<Dir3*>(smem + LY::off_table);
  float* cells = reinterpret_cast<float*>(smem + LY::off_f);
  const int tid = int(threadIdx.y * blockDim.x + threadIdx.x), nthr = 32 * (kWarps3 + 1);
  const int lane = tid & 31, ty = tid >> 5;
  const int col0 = cbase + bx * kWTW;
  const int row0 = a.rmin + by * kRows3;
  const int nrows = min(kRows3, a.rmax - row0 + 1);
  const int nwarps = (nrows + kRPW - 1) / kRPW;

  for (int k = tid; k <= 16; k += nthr) kind_start[k] = a.order[a.q + k];
  for (int j = tid; j < a.q; j += nthr) {
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
      mbar_init(&empty[st], nwarps > 0 ? nwarps : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows <= 0) return;

  if (ty == kWarps3) {
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
      // word column (col0 - 8) / 2: col0 - 8 is a multiple of 8 bf16, so 16-byte aligned
      tma_load_3d(smem + st * LY::kStage, tmap, (col0 - 8) / 2, row0 + (d.zdy & 3) - 1,
                  d.zdy >> 2, &full[st]);
    }
    return;
  }

  // consumers: the cell tile (rows row0 - 1 .. row0 + 14, columns col0 - 1 .. col0 + 256)
  fill_cell_terms<kWTW, 5>(a, FIELD_W, col0, row0, tid, cells, kWCellArr,
                        [](int rr, int cc) { return wcell_index(rr, cc); });
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kWarps3) : "memory");
  if (ty >= nwarps) return;
  const int r = row0 + kRPW * ty;
  const int nrw = min(kRPW, a.rmax - r + 1);
  const int c0 = col0 + 8 * lane;
  unsigned vm = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) vm |= (c0 + j >= a.cmin && c0 + j <= a.cmax) ? 1u << j : 0u;
  RegsW t;
#pragma unroll
  for (int k = 0; k < kRPW; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int row = r + k, c = c0 + j;
      const bool on = ((vm >> j) & 1u) && row < a.rows;
      t.eins[k][j] = on ? __fmul_rn(a.e_in[int64_t(row) * a.pitch + c], a.inv_scale) : 0.f;
      t.acc[k][j] = 0.f;
    }
  float accw = 0.f;
  CtxW ctx;
  ctx.cells = cells + 2 * ty * kWCellG + lane + 1;
  ctx.pitch = a.pitch;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = 0;
  __nv_bfloat16* obase = static_cast<__nv_bfloat16*>(a.planes) + int64_t(r) * a.pitch + c0;
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P, F)                                                            \
  ok = ok && run_kind_w<S, CX, CY, P, F>(j, kind_start[K + 1], t, ctx, accw, table, smem, full, \
                                         empty, obase, ty, a.status)
  if (nrw == kRPW && __all_sync(0xffffffffu, vm == 0xFFu)) {
    WLBM_KINDS16(WLBM_KIND, true);
  } else {
    WLBM_KINDS16(WLBM_KIND, false);
  }
#undef WLBM_KIND
  if (!ok) return;
  // E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density), d' = scale v' + w_i E_in(y)
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (k >= nrw) break;
    const int64_t own = int64_t(r + k) * a.pitch + c0;
    float eo[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const float ein = ((vm >> jj) & 1u) ? a.e_in[own + jj] : 0.f;
      eo[jj] = fmaf(t.acc[k][jj], a.scale, __fmul_rn(ein, accw));
    }
    float* e_out = a.e_out + own;
    if (vm == 0xFFu) {
      reinterpret_cast<float4*>(e_out)[0] = make_float4(eo[0], eo[1], eo[2], eo[3]);
      reinterpret_cast<float4*>(e_out)[1] = make_float4(eo[4], eo[5], eo[6], eo[7]);
    } else {
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if ((vm >> jj) & 1u) e_out[jj] = eo[jj];
    }
  }
}

}  // namespace

}  // namespace wlbm
