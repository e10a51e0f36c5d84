// Device code of one 128 x 14 tile of the TMA step kernel (variant 3), shared by the
// single-grid and batched kernels (k_step_tma.cu) and the persistent batched kernel
// (k_batch_persistent.cu).  The update is Eq. lbm-energy with the due worm hop of each
// direction (Eq. worm-paths, Eq. algorithm), E' = sum_i d_i' (Eq. lbm-energy-density).
#pragma once
#include <cuda.h>

#include "elem.cuh"
#include "mbar.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kWarps3 = 7;              // consumer warps per block; + 1 producer warp
constexpr int kRPW = 2;                 // rows per consumer warp
constexpr int kRows3 = kWarps3 * kRPW;  // rows per block (box height)
constexpr int kCPT3 = 4;                // consecutive cells per lane
constexpr int kTW3 = 32 * kCPT3;        // tile width
constexpr int kTR = kRPW + 2;           // register-tile rows (one halo row each side)

// Per-direction record built once per block (16 bytes, one shared-memory vector load).
struct alignas(16) Dir3 {
  int64_t dst;       // element offset of the destination plane from the output base
  float wi;          // angular weight w_i
  int32_t zdy;       // source plane (tensor-map z coordinate) << 2 | (row shift + 1)
};
static_assert(sizeof(Dir3) == 16, "one 16-byte shared-memory load per direction");

// bfloat16 cell tile in shared memory: 1 - W, X = ((1 - W) R + W E) / scale and
// F = W E / scale of the block's cells, rows row0 - 1 .. row0 + kRows3 (local row rr) and
// columns col0 - 1 .. col0 + kTW3 (local column cc).  Column col0 + 4 g + p is stored at
// [p][rr][g + 1]: the lanes of a warp own the groups g = lane of 4 cells, so a read of
// one tile position by a warp touches consecutive words (no bank conflicts).
constexpr int kCellRows = kRows3 + 2;
constexpr int kCellG = kTW3 / 4 + 2;                 // groups -1 .. kTW3 / 4
constexpr int kCellArr = 4 * kCellRows * kCellG;     // floats per array
// (CG: groups per row of the tile, kCellG for 128-column tiles.)
template <int CG = kCellG>
__device__ __forceinline__ int cell_index(int rr, int cc) {
  const int x = cc - 1;                              // column - col0, -1 .. tile width
  return ((x & 3) * kCellRows + rr) * CG + (x >> 2) + 1;
}
// Offset from a lane's base (cells + 2 ty * CG + g + 1, g = the lane's group) of its
// register-tile position (lr, lc): row r - 1 + lr, column c0 - 1 + lc of the warp's first
// row r and the lane's first cell c0 = col0 + 4 g.
template <int CG = kCellG>
__host__ __device__ constexpr int cell_off(int lr, int lc) {
  return (((lc + 3) & 3) * kCellRows + lr) * CG + (lc == 0 ? -1 : (lc - 1) / 4);
}

template <typename T, int S>
struct TmaLayout {
  static constexpr bool REF = sizeof(T) == 2;
  static constexpr int V = 16 / int(sizeof(T));          // elements per 16 bytes
  static constexpr int BW = kTW3 + 2 * V;                // box width: columns col0-V ..
  static constexpr int kBoxElems = BW * kRows3;
  static constexpr uint32_t kBoxBytes = uint32_t(kBoxElems) * sizeof(T);
  static constexpr size_t kStage = (size_t(kBoxBytes) + 127) / 128 * 128;   // aligned stride
  // bfloat16: the cell tile (three arrays: 1 - W, X, F), or in the register-tile form the
  // lanes' W E / scale stretches (smaller; the same region)
  static constexpr size_t off_f = size_t(S) * kStage;
  static constexpr size_t f_bytes = REF ? size_t(3) * kCellArr * 4 : 0;
  static_assert(size_t(kWarps3) * kTR * 6 * 32 * 4 <= size_t(3) * kCellArr * 4,
                "the register-tile stretches fit the cell tile's region");
  static constexpr size_t off_bar = (off_f + f_bytes + 127) / 128 * 128;
  static constexpr size_t off_kind = off_bar + 2 * S * 8;           // 17 ints
  static constexpr size_t off_table = (off_kind + 17 * 4 + 127) / 128 * 128;
  static size_t bytes(int q) { return off_table + size_t(q) * sizeof(Dir3); }
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// float32 register tile of one lane: rows r-1 .. r+kRPW (index 0..kTR-1) and columns
// c0-1 .. c0+4 (index 0..5) around its cells (rows r, r+1; columns c0 .. c0+3).
struct Regs3 {
  float G[kTR][6];      // 1 - W
  float X[kTR][6];      // W E
  float acc[kRPW][4];   // sum over directions of the new values
};

// bfloat16 registers of one lane: the own cells' E_in / scale and the sums of the stored
// new values (the cell terms live in the shared cell tile).
struct RegsB {
  float eins[kRPW][4];
  float acc[kRPW][4];
};

// bfloat16 register tile of one lane (the form of the single-grid kernels, two blocks per
// SM): as Regs3 with X = ((1 - W) R + W E) / scale, plus the own cells' E_in / scale; W E /
// scale of the same cells sits in a lane-private stretch of shared memory (read only at
// the start of a paused kind).
struct RegsR {
  float G[kTR][6];
  float X[kTR][6];
  float eins[kRPW][4];
  float acc[kRPW][4];
};

// Source values of the 4 cells for a DDED shift DX (-1, 0, +1) from a ring row.
template <typename T, int DX>
__device__ __forceinline__ void ring_values(const T* row, int lane, float (&v)[4]) {
  constexpr int V = 16 / int(sizeof(T));
  if constexpr (sizeof(T) == 4) {
    const float* p = reinterpret_cast<const float*>(row) + V + 4 * lane;   // 16-byte aligned
    const float4 q = *reinterpret_cast<const float4*>(p);
    if constexpr (DX == 0) {
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (DX < 0) {
      v[0] = p[-1]; v[1] = q.x; v[2] = q.y; v[3] = q.z;
    } else {
      v[0] = q.y; v[1] = q.z; v[2] = q.w; v[3] = p[4];
    }
  } else {
    const uint32_t* p = reinterpret_cast<const uint32_t*>(row) + (V + 4 * lane) / 2;  // 8 B
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    if constexpr (DX == 0) {
      v[0] = bf_lo(q.x); v[1] = bf_hi(q.x); v[2] = bf_lo(q.y); v[3] = bf_hi(q.y);
    } else if constexpr (DX < 0) {
      v[0] = bf_hi(p[-1]); v[1] = bf_lo(q.x); v[2] = bf_hi(q.x); v[3] = bf_lo(q.y);
    } else {
      v[0] = bf_hi(q.x); v[1] = bf_lo(q.y); v[2] = bf_hi(q.y); v[3] = bf_lo(p[2]);
    }
  }
}

// Store the new values of the cells in mask vm (bit j: cell j is computed; a group at the
// edge of the covered cells stores element by element) and return what was stored
// (bfloat16: the rounded values).
template <typename T>
__device__ __forceinline__ void store4(T* dst, const float (&o)[4], unsigned vm, float (&s)[4]) {
  if constexpr (sizeof(T) == 4) {
    if (vm == 0xFu) {
      __stcs(reinterpret_cast<float4*>(dst), make_float4(o[0], o[1], o[2], o[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((vm >> j) & 1u) __stcs(reinterpret_cast<float*>(dst) + j, o[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = o[j];
  } else {
    const __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]);
    const __nv_bfloat162 p1 = __floats2bfloat162_rn(o[2], o[3]);
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&p0);
    const uint32_t w1 = *reinterpret_cast<const uint32_t*>(&p1);
    if (vm == 0xFu) {
      __stcs(reinterpret_cast<uint2*>(dst), make_uint2(w0, w1));
    } else {
      unsigned short* d = reinterpret_cast<unsigned short*>(dst);
      const unsigned short h[4] = {static_cast<unsigned short>(w0 & 0xffffu),
                                   static_cast<unsigned short>(w0 >> 16),
                                   static_cast<unsigned short>(w1 & 0xffffu),
                                   static_cast<unsigned short>(w1 >> 16)};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((vm >> j) & 1u) __stcs(d + j, h[j]);
    }
    s[0] = bf_lo(w0); s[1] = bf_hi(w0); s[2] = bf_lo(w1); s[3] = bf_hi(w1);
  }
}

// acc0 += lower bfloat16 of w, acc1 += upper one, each widened exactly and added with one
// float32 rounding (the mixed-precision add of sm_100 and later: one instruction per value
// instead of a widening and an add).
__device__ __forceinline__ void add_bf16x2(uint32_t w, float& acc0, float& acc1) {
  asm("{\n .reg .b16 l, h;\n mov.b32 {l, h}, %2;\n"
      " add.rn.f32.bf16 %0, l, %0;\n add.rn.f32.bf16 %1, h, %1;\n}"
      : "+f"(acc0), "+f"(acc1)
      : "r"(w));
}

// bfloat16 store of the 4 new values of the cells in mask vm; returns the packed words.
__device__ __forceinline__ uint2 store4_bf16(__nv_bfloat16* dst, const float2 (&o)[2],
                                             unsigned vm) {
  const __nv_bfloat162 p0 = __float22bfloat162_rn(o[0]);
  const __nv_bfloat162 p1 = __float22bfloat162_rn(o[1]);
  const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&p0);
  const uint32_t w1 = *reinterpret_cast<const uint32_t*>(&p1);
  if (vm == 0xFu) {
    __stcs(reinterpret_cast<uint2*>(dst), make_uint2(w0, w1));
  } else {
    unsigned short* d = reinterpret_cast<unsigned short*>(dst);
    const unsigned short h[4] = {static_cast<unsigned short>(w0 & 0xffffu),
                                 static_cast<unsigned short>(w0 >> 16),
                                 static_cast<unsigned short>(w1 & 0xffffu),
                                 static_cast<unsigned short>(w1 >> 16)};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((vm >> j) & 1u) __stcs(d + j, h[j]);
  }
  return make_uint2(w0, w1);
}

// Arguments of one direction for one lane.
template <typename T>
struct DirCtx {
  const T* ring_row;   // first of the warp's rows in the stage
  T* dst;              // destination of the lane's first cell in the warp's first row
  const float* cells;  // bfloat16: this lane's base in the cell tile (see cell_off), or
                       // of its W E / scale stretch (register-tile form, stride 32 floats)
  int64_t pitch, plane;
  float wi;
  int lane, nrw;   // nrw: computed rows of this warp (1 or 2)
  unsigned vm;     // bit j: the lane's cell j is computed
  uint32_t g0;     // ring uses before this tile (persistent blocks carry it across tiles)
};

// float32: one direction for the lane's cells; hop (CX, CY), paused or propagating.
template <typename T, int CX, int CY, bool PAUSED>
__device__ __forceinline__ void dir_body(Regs3& t, const DirCtx<T>& c) {
  constexpr int BW = kTW3 + 2 * (16 / int(sizeof(T)));
  constexpr int DX = PAUSED ? 0 : -CX;
  constexpr int SC = PAUSED ? 1 : 1 - CX;   // tile column of the DDED source of cell 0
  constexpr int FC = 1 - CX;                // tile column of the EED source (y - c)
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (k >= c.nrw) break;
    const int SR = PAUSED ? 1 + k : 1 + k - CY;   // tile row of the DDED source
    const int FR = 1 + k - CY;                    // tile row of the EED source
    float v[4], o[4], s[4];
    ring_values<T, DX>(c.ring_row + k * BW, c.lane, v);
    if constexpr (!PAUSED && SC % 2 == 0) {
      // source columns start on an even register: the per-element arithmetic runs on
      // pairs (same rounded operations)
      const float2 wi2 = make_float2(c.wi, c.wi);
#pragma unroll
      for (int jp = 0; jp < 4; jp += 2) {
        const float2 g2 = make_float2(t.G[SR][SC + jp], t.G[SR][SC + jp + 1]);
        const float2 v2 = make_float2(v[jp], v[jp + 1]);
        const float2 m2 = __fmul2_rn(wi2, make_float2(t.X[FR][FC + jp], t.X[FR][FC + jp + 1]));
        const float2 o2 = __ffma2_rn(g2, v2, m2);
        o[jp] = o2.x;
        o[jp + 1] = o2.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        o[j] = fmaf(t.G[SR][SC + j], v[j], __fmul_rn(c.wi, t.X[FR][FC + j]));
    }
    store4<T>(c.dst + k * c.pitch, o, c.vm, s);
#pragma unroll
    for (int jp = 0; jp < 4; jp += 2) {
      const float2 a2 = __fadd2_rn(make_float2(t.acc[k][jp], t.acc[k][jp + 1]),
                                   make_float2(s[jp], s[jp + 1]));
      t.acc[k][jp] = a2.x;
      t.acc[k][jp + 1] = a2.y;
    }
  }
}

// bfloat16: one direction for the lane's cells with the kind's source terms hoisted: the
// new stored value is v' = (1 - W) v + w_i D, where (1 - W) (Gk) and D (Dk) depend on the
// hop kind only (see run_kind), so each value costs a widening, a paired multiply-add and
// its share of a paired conversion, store and mixed-precision sum.
// FULL: every lane of the warp has all 4 cells of both rows to compute (an interior warp),
// so the row count and the edge stores need no checks.
// bfloat16 source values of the lane's 4 cells as two pairs for a DDED shift DX.
template <int DX>
__device__ __forceinline__ void ring_pairs(const __nv_bfloat16* row, int lane, float2 (&v)[2]) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(row) + (8 + 4 * lane) / 2;  // 8 B
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  if constexpr (DX == 0) {
    v[0] = make_float2(bf_lo(q.x), bf_hi(q.x));
    v[1] = make_float2(bf_lo(q.y), bf_hi(q.y));
  } else if constexpr (DX < 0) {
    v[0] = make_float2(bf_hi(p[-1]), bf_lo(q.x));
    v[1] = make_float2(bf_hi(q.x), bf_lo(q.y));
  } else {
    v[0] = make_float2(bf_hi(q.x), bf_lo(q.y));
    v[1] = make_float2(bf_hi(q.y), bf_lo(p[2]));
  }
}

// BW: ring row length (elements).
template <int CX, bool PAUSED, bool FULL, typename R, int BW = kTW3 + 16>
__device__ __forceinline__ void dir_body_ref(R& t, const DirCtx<__nv_bfloat16>& c,
                                             const float2 (&Gk)[kRPW][2],
                                             const float2 (&Dk)[kRPW][2]) {
  constexpr int DX = PAUSED ? 0 : -CX;
  const float2 wi2 = make_float2(c.wi, c.wi);
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (!FULL && k >= c.nrw) break;
    float2 v[2];
    ring_pairs<DX>(c.ring_row + k * BW, c.lane, v);
    float2 o[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) o[h] = __ffma2_rn(Gk[k][h], v[h], __fmul2_rn(wi2, Dk[k][h]));
    const uint2 w = store4_bf16(c.dst + k * c.pitch, o, FULL ? 0xFu : c.vm);
    add_bf16x2(w.x, t.acc[k][0], t.acc[k][1]);
    add_bf16x2(w.y, t.acc[k][2], t.acc[k][3]);
  }
}

// All directions of one kind (hop (CX, CY), paused or not): entries j .. end-1 of the
// kind-sorted table.  Returns false when a bounded wait gave up.  float32 storage.
template <typename T, int S, int CX, int CY, bool PAUSED>
__device__ __forceinline__ bool run_kind(int& j, int end, Regs3& t, DirCtx<T>& c,
                                         const Dir3* table, const unsigned char* smem,
                                         uint64_t* full, uint64_t* empty, T* obase, int ty,
                                         int* status) {
  using LY = TmaLayout<T, S>;
  for (; j < end; ++j) {
    const uint32_t gj = c.g0 + uint32_t(j);
    const int st = int(gj % S);
    if (!mbar_wait(&full[st], (gj / S) & 1u, kWaitCycles)) {
      if (c.lane == 0) atomicOr(status, 1);
      return false;
    }
    const Dir3 d = table[j];
    c.ring_row = reinterpret_cast<const T*>(smem + st * LY::kStage) + kRPW * ty * LY::BW;
    c.dst = obase + d.dst;
    c.wi = d.wi;
    if (c.vm) dir_body<T, CX, CY, PAUSED>(t, c);
    __syncwarp();
    mbar_arrive_if(&empty[st], c.lane == 0);
  }
  return true;
}

// The same for bfloat16 storage.  The per-kind parts of the update of the lane's cells are
// computed once per kind from the cell tile (the same float32 operations, in the same
// order, as computing them per direction):
//   propagating  Gk = 1 - W(s),  D = X(s) - E_in(y) / scale
//   paused       Gk = 1 - W(y),  D = (X(y) - W(y) E(y) / scale) + W(s) E(s) / scale
//                                    - E_in(y) / scale
// with s = y - c and X = ((1 - W) R + W E) / scale (R: the reference energy of the stored
// values the step reads, E their local energy).  FULL: see dir_body_ref.
// The register-tile form: the same per-kind terms from the lane's registers and its W E /
// scale stretch.
template <int S, int CX, int CY, bool PAUSED, bool FULL>
__device__ __forceinline__ bool run_kind_bf16r(int& j, int end, RegsR& t,
                                               DirCtx<__nv_bfloat16>& c, float& accw,
                                               const Dir3* table, const unsigned char* smem,
                                               uint64_t* full, uint64_t* empty,
                                               __nv_bfloat16* obase, int ty, int* status) {
  using LY = TmaLayout<__nv_bfloat16, S>;
  if (j >= end) return true;
  float2 Gk[kRPW][2], Dk[kRPW][2];
  {
    const float* fsc = c.cells;
    constexpr int SC = PAUSED ? 1 : 1 - CX;
    constexpr int FC = 1 - CX;
#pragma unroll
    for (int k = 0; k < kRPW; ++k) {
      const int SR = PAUSED ? 1 + k : 1 + k - CY;
      const int FR = 1 + k - CY;
      float g[4], d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        g[q] = t.G[SR][SC + q];
        const float tt =
            PAUSED ? __fadd_rn(__fsub_rn(t.X[1 + k][1 + q], fsc[((1 + k) * 6 + 1 + q) * 32]),
                               fsc[(FR * 6 + FC + q) * 32])
                   : t.X[SR][SC + q];
        d[q] = __fsub_rn(tt, t.eins[k][q]);
      }
      Gk[k][0] = make_float2(g[0], g[1]);
      Gk[k][1] = make_float2(g[2], g[3]);
      Dk[k][0] = make_float2(d[0], d[1]);
      Dk[k][1] = make_float2(d[2], d[3]);
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
    c.ring_row =
        reinterpret_cast<const __nv_bfloat16*>(smem + st * LY::kStage) + kRPW * ty * LY::BW;
    c.dst = obase + d.dst;
    c.wi = d.wi;
    accw += d.wi;
    if (FULL || c.vm) dir_body_ref<CX, PAUSED, FULL>(t, c, Gk, Dk);
    __syncwarp();
    mbar_arrive_if(&empty[st], c.lane == 0);
  }
  return true;
}

// The cell-tile form (CG groups per tile row, ring rows of BW elements, stages STAGE bytes
// apart; ring_off: the warp's first ring element in a stage).
template <int S, int CX, int CY, bool PAUSED, bool FULL, int CG = kCellG, int BW = kTW3 + 16,
          size_t STAGE = TmaLayout<__nv_bfloat16, S>::kStage>
__device__ __forceinline__ bool run_kind_bf16(int& j, int end, RegsB& t,
                                              DirCtx<__nv_bfloat16>& c, float& accw,
                                              const Dir3* table, const unsigned char* smem,
                                              uint64_t* full, uint64_t* empty,
                                              __nv_bfloat16* obase, int ring_off, int* status) {
  if (j >= end) return true;
  float2 Gk[kRPW][2], Dk[kRPW][2];
  {
    const float* G = c.cells;
    constexpr int kArr = 4 * kCellRows * CG;            // floats per array of the tile
    const float* X = c.cells + kArr;
    const float* F = c.cells + 2 * kArr;
    constexpr int SC = PAUSED ? 1 : 1 - CX;
    constexpr int FC = 1 - CX;
#pragma unroll
    for (int k = 0; k < kRPW; ++k) {
      const int SR = PAUSED ? 1 + k : 1 + k - CY;
      const int FR = 1 + k - CY;
      float g[4], d[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        g[q] = G[cell_off<CG>(SR, SC + q)];
        const float tt =
            PAUSED ? __fadd_rn(__fsub_rn(X[cell_off<CG>(1 + k, 1 + q)], F[cell_off<CG>(1 + k, 1 + q)]),
                               F[cell_off<CG>(FR, FC + q)])
                   : X[cell_off<CG>(SR, SC + q)];
        d[q] = __fsub_rn(tt, t.eins[k][q]);
      }
      Gk[k][0] = make_float2(g[0], g[1]);
      Gk[k][1] = make_float2(g[2], g[3]);
      Dk[k][0] = make_float2(d[0], d[1]);
      Dk[k][1] = make_float2(d[2], d[3]);
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
    c.ring_row = reinterpret_cast<const __nv_bfloat16*>(smem + st * STAGE) + ring_off;
    c.dst = obase + d.dst;
    c.wi = d.wi;
    accw += d.wi;
    if (FULL || c.vm) dir_body_ref<CX, PAUSED, FULL, RegsB, BW>(t, c, Gk, Dk);
    __syncwarp();
    mbar_arrive_if(&empty[st], c.lane == 0);
  }
  return true;
}

// ------------------------------------------------------------------------ tile pieces
// Shared-memory views of a block: ring stages, cell tile, barriers, kind starts, table.
template <typename T, int S>
struct TileSmem {
  unsigned char* base;
  uint64_t* full;
  uint64_t* empty;
  int* kind_start;
  Dir3* table;
  __device__ explicit TileSmem(unsigned char* smem)
      : base(smem),
        full(reinterpret_cast<uint64_t*>(smem + TmaLayout<T, S>::off_bar)),
        empty(reinterpret_cast<uint64_t*>(smem + TmaLayout<T, S>::off_bar) + S),
        kind_start(reinterpret_cast<int*>(smem + TmaLayout<T, S>::off_kind)),
        table(reinterpret_cast<Dir3*>(smem + TmaLayout<T, S>::off_table)) {}
};

// The step's kind-sorted direction table and kind starts (all threads of the block).
template <typename T, int S>
__device__ __forceinline__ void build_table(const StepArgs& a, const TileSmem<T, S>& m, int tid,
                                            int nthr) {
  for (int k = tid; k <= 16; k += nthr) m.kind_start[k] = a.order[a.q + k];
  for (int j = tid; j < a.q; j += nthr) {
    const int i = a.order[j];
    const int code = a.codes[i];
    const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
    Dir3 d;
    // tape mode (adjoint recompute): plane i of the source slot to plane i of the next slot
    d.dst = int64_t(a.tape ? i : (paused ? par : 1 - par) * a.q + i) * a.plane;
    d.wi = a.w[i];
    const int z = a.tape ? a.tape_z0 + i : par * a.q + i;
    d.zdy = z * 4 + (paused ? 0 : -c_hop_y[hop]) + 1;
    m.table[j] = d;
  }
}

// Producer thread: the q boxes of the tile at (col0, row0) as ring uses g, g+1, ...; g is
// advanced.  On a wait that gives up: sets the status, waits for the copies in flight and
// returns false.
template <typename T, int S>
__device__ __forceinline__ bool produce_tile(const StepArgs& a, const void* tmap, int col0,
                                             int row0, uint32_t& g, const TileSmem<T, S>& m) {
  using LY = TmaLayout<T, S>;
  for (int i = 0; i < a.q; ++i, ++g) {
    const int st = int(g % S);
    const uint32_t k = g / S;
    if (k > 0 && !mbar_wait(&m.empty[st], (k - 1) & 1u, kWaitCycles)) {
      atomicOr(a.status, 1);
      // uses g - S .. g - 1 may still be in flight (earlier ones were released); a use
      // before this block's first (a fresh ring) has nothing to wait for
      for (uint32_t gj = g >= S ? g - S : 0u; gj < g; ++gj)
        mbar_wait(&m.full[gj % S], (gj / S) & 1u, kWaitCycles);
      return false;
    }
    const Dir3 d = m.table[i];
    mbar_expect(&m.full[st], LY::kBoxBytes);
    tma_load_3d(m.base + st * LY::kStage, tmap, col0 - LY::V, row0 + (d.zdy & 3) - 1,
                d.zdy >> 2, &m.full[st]);
  }
  return true;
}

// A consumer warp without rows in this tile: wait for each box and release it, so the
// barriers keep one phase per ring use (blocks whose empty barriers count every warp).
template <typename T, int S>
__device__ __forceinline__ bool drain_tile(const StepArgs& a, uint32_t& g, int lane,
                                           const TileSmem<T, S>& m) {
  for (int i = 0; i < a.q; ++i, ++g) {
    if (!mbar_wait(&m.full[g % S], (g / S) & 1u, kWaitCycles)) {
      if (lane == 0) atomicOr(a.status, 1);
      return false;
    }
    __syncwarp();
    mbar_arrive_if(&m.empty[g % S], lane == 0);
  }
  return true;
}

// The 16 kind loops of a consumer warp (kind = hop | paused << 3; hop numbering of the
// host lattice: (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)).
#define WLBM_KINDS16(KIND, F)        \
  KIND(0, 1, 0, false, F);           \
  KIND(1, 0, 1, false, F);           \
  KIND(2, -1, 0, false, F);          \
  KIND(3, 0, -1, false, F);          \
  KIND(4, 1, 1, false, F);           \
  KIND(5, -1, 1, false, F);          \
  KIND(6, -1, -1, false, F);         \
  KIND(7, 1, -1, false, F);          \
  KIND(8, 1, 0, true, F);            \
  KIND(9, 0, 1, true, F);            \
  KIND(10, -1, 0, true, F);          \
  KIND(11, 0, -1, true, F);          \
  KIND(12, 1, 1, true, F);           \
  KIND(13, -1, 1, true, F);          \
  KIND(14, -1, -1, true, F);         \
  KIND(15, 1, -1, true, F)

// Computed cells of lane `lane` in a warp's row block: bit j for cell c0 + j.
__device__ __forceinline__ unsigned lane_mask(const StepArgs& a, int c0) {
  unsigned vm = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) vm |= (c0 + j >= a.cmin && c0 + j <= a.cmax) ? 1u << j : 0u;
  return vm;
}

// bfloat16 E' (Eq. lbm-energy-density) of the warp's rows: d' = scale v' + w_i E_in(y).
template <typename R>
__device__ __forceinline__ void store_e_bf16(const StepArgs& a, const R& t, float accw, int r,
                                             int nrw, int c0, unsigned vm) {
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (k >= nrw) break;
    const int64_t own = int64_t(r + k) * a.pitch + c0;
    float eo[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const float ein = ((vm >> jj) & 1u) ? a.e_in[own + jj] : 0.f;
      eo[jj] = fmaf(t.acc[k][jj], a.scale, __fmul_rn(ein, accw));
    }
    float* e_out = a.e_out + own;
    if (vm == 0xFu) {
      *reinterpret_cast<float4*>(e_out) = make_float4(eo[0], eo[1], eo[2], eo[3]);
    } else {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if ((vm >> jj) & 1u) e_out[jj] = eo[jj];
    }
  }
}

// float32 consumer warp with rows: register tile, 16 kind loops, E'.
template <typename T, int S, bool FIELD_W>
__device__ __forceinline__ bool consume_f32(const StepArgs& a, int col0, int row0, int ty,
                                            int lane, uint32_t g, const TileSmem<T, S>& m) {
  const int r = row0 + kRPW * ty;                      // first row of this warp
  const int nrw = min(kRPW, a.rmax - r + 1);           // 1 or 2 computed rows
  const int c0 = col0 + 4 * lane;
  const unsigned vm = lane_mask(a, c0);
  Regs3 t;
#pragma unroll
  for (int rr = 0; rr < kTR; ++rr) {
    const int row = r - 1 + rr;
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int c = c0 - 1 + cc;
      float wv = 0.f, ev = 0.f;
      if (row < a.rows && c >= 0 && c < a.pitch) {
        const int64_t o = int64_t(row) * a.pitch + c;
        ev = a.e_in[o];
        wv = FIELD_W ? a.wfield[o] : uniform_w(a, row, c);
      }
      t.G[rr][cc] = __fsub_rn(1.f, wv);
      t.X[rr][cc] = __fmul_rn(wv, ev);
    }
  }
#pragma unroll
  for (int k = 0; k < kRPW; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) t.acc[k][j] = 0.f;
  DirCtx<T> ctx;
  ctx.cells = nullptr;
  ctx.pitch = a.pitch;
  ctx.plane = a.plane;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = g;
  T* obase = static_cast<T*>(a.tape ? a.tape_dst : a.planes) + int64_t(r) * a.pitch + c0;
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P, F)                                                           \
  ok = ok && run_kind<T, S, CX, CY, P>(j, m.kind_start[K + 1], t, ctx, m.table, m.base,      \
                                       m.full, m.empty, obase, ty, a.status)
  WLBM_KINDS16(WLBM_KIND, 0);
#undef WLBM_KIND
  if (!ok) return false;
  // E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density)
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (k >= nrw) break;
    float* e_out = a.e_out + int64_t(r + k) * a.pitch + c0;
    if (vm == 0xFu) {
      *reinterpret_cast<float4*>(e_out) =
          make_float4(t.acc[k][0], t.acc[k][1], t.acc[k][2], t.acc[k][3]);
    } else {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
        if ((vm >> jj) & 1u) e_out[jj] = t.acc[k][jj];
    }
  }
  return true;
}

// bfloat16 consumer warp with rows, register-tile form.
template <int S, bool FIELD_W>
__device__ __forceinline__ bool consume_bf16r(const StepArgs& a, int col0, int row0, int ty,
                                              int lane, uint32_t g,
                                              const TileSmem<__nv_bfloat16, S>& m) {
  using LY = TmaLayout<__nv_bfloat16, S>;
  const int r = row0 + kRPW * ty;
  const int nrw = min(kRPW, a.rmax - r + 1);
  const int c0 = col0 + 4 * lane;
  const unsigned vm = lane_mask(a, c0);
  float* fsc = reinterpret_cast<float*>(m.base + LY::off_f) + size_t(ty) * kTR * 6 * 32 + lane;
  RegsR t;
#pragma unroll
  for (int rr = 0; rr < kTR; ++rr) {
    const int row = r - 1 + rr;
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int c = c0 - 1 + cc;
      float wv = 0.f, ev = 0.f, rv = 0.f;
      if (row < a.rows && c >= 0 && c < a.pitch) {
        const int64_t o = int64_t(row) * a.pitch + c;
        ev = a.e_in[o];
        wv = FIELD_W ? a.wfield[o] : uniform_w(a, row, c);
        rv = a.e_ref[o];
      }
      const float fv = __fmul_rn(wv, ev), gv = __fsub_rn(1.f, wv);
      t.G[rr][cc] = gv;
      t.X[rr][cc] = __fmul_rn(fmaf(gv, rv, fv), a.inv_scale);
      fsc[(rr * 6 + cc) * 32] = __fmul_rn(fv, a.inv_scale);
      if (rr >= 1 && rr <= kRPW && cc >= 1 && cc <= 4)
        t.eins[rr - 1][cc - 1] = ((vm >> (cc - 1)) & 1u) ? __fmul_rn(ev, a.inv_scale) : 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < kRPW; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) t.acc[k][j] = 0.f;
  float accw = 0.f;
  DirCtx<__nv_bfloat16> ctx;
  ctx.cells = fsc;
  ctx.pitch = a.pitch;
  ctx.plane = a.plane;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = g;
  __nv_bfloat16* obase =
      static_cast<__nv_bfloat16*>(a.tape ? a.tape_dst : a.planes) + int64_t(r) * a.pitch + c0;
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P, F)                                                           \
  ok = ok && run_kind_bf16r<S, CX, CY, P, F>(j, m.kind_start[K + 1], t, ctx, accw, m.table, \
                                             m.base, m.full, m.empty, obase, ty, a.status)
  // warps whose lanes all compute 4 cells of 2 rows take loops without row and edge checks
  if (nrw == kRPW && __all_sync(0xffffffffu, vm == 0xFu)) {
    WLBM_KINDS16(WLBM_KIND, true);
  } else {
    WLBM_KINDS16(WLBM_KIND, false);
  }
#undef WLBM_KIND
  if (!ok) return false;
  store_e_bf16(a, t, accw, r, nrw, c0, vm);
  return true;
}

// bfloat16 cell tile of the block's tile at (col0, row0), filled by the consumer threads
// (tid < 32 kWarps3); the caller synchronises the consumer warps around it.
// A thread's positions are idx = tid + k * (32 kWarps3); the loads of a batch of KB of them
// are all issued before any value is used, so a tile start waits about one memory latency
// per batch instead of one per position (KB = 0: one position at a time, a rolled loop, for
// kernels short of registers).
template <int COLS, int KB, typename Index, int NT = 32 * kWarps3>
__device__ __forceinline__ void fill_cell_terms(const StepArgs& a, bool field_w, int col0,
                                                int row0, int tid, float* cells, int arr,
                                                Index index) {
  constexpr int kN = kCellRows * (COLS + 2);          // positions of the tile and its halo
  constexpr int kT = NT;                              // consumer threads
  constexpr int kIt = (kN + kT - 1) / kT;
  constexpr int kB = KB > 0 ? KB : 1;                 // positions per batch
#pragma unroll(KB > 0 ? kIt : 1)
  for (int h = 0; h < kIt; h += kB) {
    float ev[kB], wv[kB], rv[kB];
#pragma unroll
    for (int k = 0; k < kB; ++k) {
      const int idx = tid + (h + k) * kT;
      const int rr = idx / (COLS + 2), cc = idx - rr * (COLS + 2);
      const int row = row0 - 1 + rr, c = col0 - 1 + cc;
      ev[k] = wv[k] = rv[k] = 0.f;
      if (h + k < kIt && idx < kN && row < a.rows && c >= 0 && c < a.pitch) {
        const int64_t o = int64_t(row) * a.pitch + c;
        ev[k] = a.e_in[o];
        wv[k] = field_w ? a.wfield[o] : uniform_w(a, row, c);
        rv[k] = a.e_ref[o];
      }
    }
#pragma unroll
    for (int k = 0; k < kB; ++k) {
      const int idx = tid + (h + k) * kT;
      if (h + k < kIt && idx < kN) {
        const int rr = idx / (COLS + 2), cc = idx - rr * (COLS + 2);
        const float fv = __fmul_rn(wv[k], ev[k]), gv = __fsub_rn(1.f, wv[k]);
        const int ci = index(rr, cc);
        cells[ci] = gv;
        cells[arr + ci] = __fmul_rn(fmaf(gv, rv[k], fv), a.inv_scale);
        cells[2 * arr + ci] = __fmul_rn(fv, a.inv_scale);
      }
    }
  }
}

template <int S, bool FIELD_W, int KB = 5>
__device__ __forceinline__ void fill_cells(const StepArgs& a, int col0, int row0, int tid,
                                           const TileSmem<__nv_bfloat16, S>& m) {
  using LY = TmaLayout<__nv_bfloat16, S>;
  float* cells = reinterpret_cast<float*>(m.base + LY::off_f);
  fill_cell_terms<kTW3, KB>(a, FIELD_W, col0, row0, tid, cells, kCellArr,
                        [](int rr, int cc) { return cell_index(rr, cc); });
}

// The consumer warps' barrier (barrier 1; the producer warp never takes part).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kWarps3) : "memory");
}

// bfloat16 consumer warp with rows, cell-tile form (the tile filled and synchronised).
template <int S>
__device__ __forceinline__ bool consume_bf16c(const StepArgs& a, int col0, int row0, int ty,
                                              int lane, uint32_t g,
                                              const TileSmem<__nv_bfloat16, S>& m) {
  using LY = TmaLayout<__nv_bfloat16, S>;
  const float* cells = reinterpret_cast<const float*>(m.base + LY::off_f);
  const int r = row0 + kRPW * ty;
  const int nrw = min(kRPW, a.rmax - r + 1);
  const int c0 = col0 + 4 * lane;
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
  ctx.cells = cells + 2 * ty * kCellG + lane + 1;
  ctx.pitch = a.pitch;
  ctx.plane = a.plane;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = g;
  __nv_bfloat16* obase =
      static_cast<__nv_bfloat16*>(a.tape ? a.tape_dst : a.planes) + int64_t(r) * a.pitch + c0;
  int j = 0;
  bool ok = true;
  const int ring_off = kRPW * ty * LY::BW;
#define WLBM_KIND(K, CX, CY, P, F)                                                          \
  ok = ok && run_kind_bf16<S, CX, CY, P, F>(j, m.kind_start[K + 1], t, ctx, accw, m.table, \
                                            m.base, m.full, m.empty, obase, ring_off,      \
                                            a.status)
  if (nrw == kRPW && __all_sync(0xffffffffu, vm == 0xFu)) {
    WLBM_KINDS16(WLBM_KIND, true);
  } else {
    WLBM_KINDS16(WLBM_KIND, false);
  }
#undef WLBM_KIND
  if (!ok) return false;
  store_e_bf16(a, t, accw, r, nrw, c0, vm);
  return true;
}

// ------------------------------------------------------------------------ one tile
// One 128 x 14 tile (bx, by) of one grid; `tmap` is the generic address of the planes'
// tensor map (kernel parameter or global memory), `smem` the block's dynamic shared memory.
// Returns false when a bounded wait gave up (the status word is then set).
// PERSIST: a block that runs many tiles in turn (the persistent batched kernel).  Its
// barriers were initialised once by the caller (the empty ones for all kWarps3 consumer
// warps); g0 counts the ring uses of the block's earlier tiles (stage and phase of use g
// are g % S and (g / S) & 1) and is advanced by q; every thread returns (consumer warps
// without rows wait for and release every box) so that the caller can synchronise.
// CELLS (bfloat16): the cell terms in a block-shared tile (fewer registers: three blocks
// per SM), else in per-lane registers (two blocks per SM).
template <typename T, int S, bool FIELD_W, bool REF, bool PERSIST = false, bool CELLS = true>
__device__ __forceinline__ bool step_tma_tile(const StepArgs& a, const void* tmap, int bx,
                                              int by, unsigned char* smem, uint32_t& g0) {
  const TileSmem<T, S> m(smem);
  // warps of 32 threads, linear in (threadIdx.x, threadIdx.y): blocks of (32, 8) and of 256
  const int tid = int(threadIdx.y * blockDim.x + threadIdx.x), nthr = 32 * (kWarps3 + 1);
  const int lane = tid & 31, ty = tid >> 5;
  const int col0 = a.cbase + bx * kTW3;
  const int row0 = a.rmin + by * kRows3;
  const int nrows = min(kRows3, a.rmax - row0 + 1);     // rows row0 .. rmax are computed
  const int nwarps = (nrows + kRPW - 1) / kRPW;         // consumer warps with rows

  build_table<T, S>(a, m, tid, nthr);
  if (!PERSIST && tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&m.full[st], 1);
      mbar_init(&m.empty[st], nwarps > 0 ? nwarps : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows <= 0) return true;
  uint32_t g = PERSIST ? g0 : 0u;
  if (PERSIST) g0 += uint32_t(a.q);

  if (ty == kWarps3) {
    // ------------------------------------------------------------- producer thread
    if (lane != 0) return true;
    // persistent form: the planes may have been written by other blocks of this kernel,
    // and the ring by this block's wall chunks; order the tensor copies after those
    // generic-proxy writes
    if (PERSIST) asm volatile("fence.proxy.async;" ::: "memory");
    return produce_tile<T, S>(a, tmap, col0, row0, g, m);
  }
  // ---------------------------------------------------------------- consumer warps
  if constexpr (REF && CELLS) {
    // (the persistent kernel, three blocks per SM, has no registers to spare for batches)
    fill_cells<S, FIELD_W, PERSIST ? 0 : 5>(a, col0, row0, tid, m);
    consumers_sync();
    if (ty >= nwarps) return PERSIST ? drain_tile<T, S>(a, g, lane, m) : true;
    return consume_bf16c<S>(a, col0, row0, ty, lane, g, m);
  } else {
    if (ty >= nwarps) return PERSIST ? drain_tile<T, S>(a, g, lane, m) : true;
    if constexpr (REF) return consume_bf16r<S, FIELD_W>(a, col0, row0, ty, lane, g, m);
    else return consume_f32<T, S, FIELD_W>(a, col0, row0, ty, lane, g, m);
  }
}

// ------------------------------------------------------------------------ tile loop
// A block of resident threads that takes tiles first, first + stride, ... of one grid step
// (tiles_x per row, ntiles in all).  The direction table is the step's, built once; the
// producer thread streams the boxes of all its tiles through the ring without stopping at
// tile edges, and every consumer warp follows at its own pace (the cell-tile form
// synchronises the consumer warps around each refill of the tile).  `fail` is a shared flag;
// after a wait gives up the block stops at the next tile edge.
template <typename T, int S, bool FIELD_W, bool CELLS>
__device__ __forceinline__ void step_tma_loop(const StepArgs& a, const void* tmap, int tiles_x,
                                              int ntiles, unsigned char* smem, int* fail) {
  constexpr bool REF = sizeof(T) == 2;
  const TileSmem<T, S> m(smem);
  const int tid = int(threadIdx.y * blockDim.x + threadIdx.x), nthr = 32 * (kWarps3 + 1);
  const int lane = tid & 31, ty = tid >> 5;
  build_table<T, S>(a, m, tid, nthr);
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&m.full[st], 1);
      mbar_init(&m.empty[st], kWarps3);   // every consumer warp releases every box
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail = 0;
  }
  __syncthreads();
  uint32_t g = 0;
  const int first = int(blockIdx.x), stride = int(gridDim.x);
  if (ty == kWarps3) {
    if (lane != 0) return;
    for (int tile = first; tile < ntiles; tile += stride) {
      const int col0 = a.cbase + (tile % tiles_x) * kTW3;
      const int row0 = a.rmin + (tile / tiles_x) * kRows3;
      if (!produce_tile<T, S>(a, tmap, col0, row0, g, m)) return;
    }
    return;
  }
  for (int tile = first; tile < ntiles; tile += stride) {
    const int col0 = a.cbase + (tile % tiles_x) * kTW3;
    const int row0 = a.rmin + (tile / tiles_x) * kRows3;
    const int nrows = min(kRows3, a.rmax - row0 + 1);
    const int nwarps = (nrows + kRPW - 1) / kRPW;
    bool ok;
    if constexpr (REF && CELLS) {
      consumers_sync();                   // every warp is done with the previous tile
      if (*reinterpret_cast<volatile int*>(fail)) return;
      fill_cells<S, FIELD_W>(a, col0, row0, tid, m);
      consumers_sync();
      ok = ty >= nwarps ? drain_tile<T, S>(a, g, lane, m)
                        : consume_bf16c<S>(a, col0, row0, ty, lane, g, m);
    } else {
      if (*reinterpret_cast<volatile int*>(fail)) return;
      if (ty >= nwarps) ok = drain_tile<T, S>(a, g, lane, m);
      else if constexpr (REF) ok = consume_bf16r<S, FIELD_W>(a, col0, row0, ty, lane, g, m);
      else ok = consume_f32<T, S, FIELD_W>(a, col0, row0, ty, lane, g, m);
    }
    if (!ok) {
      *fail = 1;
      if constexpr (!(REF && CELLS)) return;   // the cell form leaves at the next edge
    }
    if (ty < nwarps) g += uint32_t(a.q);
  }
}

}  // namespace

}  // namespace wlbm
