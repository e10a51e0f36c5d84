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

template <typename T, int S>
struct TmaLayout {
  static constexpr bool REF = sizeof(T) == 2;
  static constexpr int V = 16 / int(sizeof(T));          // elements per 16 bytes
  static constexpr int BW = kTW3 + 2 * V;                // box width: columns col0-V ..
  static constexpr int kBoxElems = BW * kRows3;
  static constexpr uint32_t kBoxBytes = uint32_t(kBoxElems) * sizeof(T);
  static constexpr size_t kStage = (size_t(kBoxBytes) + 127) / 128 * 128;   // aligned stride
  // bfloat16: W E / scale of every lane's kTR x 6 register-tile cells, [warp][cell][lane]
  static constexpr size_t off_f = size_t(S) * kStage;
  static constexpr size_t f_bytes = REF ? size_t(kWarps3) * kTR * 6 * 32 * 4 : 0;
  static constexpr size_t off_bar = (off_f + f_bytes + 127) / 128 * 128;
  static constexpr size_t off_kind = off_bar + 2 * S * 8;           // 17 ints
  static constexpr size_t off_table = (off_kind + 17 * 4 + 127) / 128 * 128;
  static size_t bytes(int q) { return off_table + size_t(q) * sizeof(Dir3); }
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Register tile of one lane: rows r-1 .. r+kRPW (index 0..kTR-1) and columns c0-1 .. c0+4
// (index 0..5) around its cells (rows r, r+1; columns c0 .. c0+3).
struct Regs3 {
  float G[kTR][6];      // 1 - W
  float X[kTR][6];      // float32: W E; bfloat16: ((1 - W) E_ref + W E) / scale
  float eins[kRPW][4];  // bfloat16: E_in / scale of the own cells
  float acc[kRPW][4];   // sum over directions of the stored new values
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
  const float* fsc;    // bfloat16: this lane's W E / scale scratch (stride 32 floats)
  int64_t pitch, plane;
  float wi;
  int lane, nrw;   // nrw: computed rows of this warp (1 or 2)
  unsigned vm;     // bit j: the lane's cell j is computed
  uint32_t g0;     // ring uses before this tile (persistent blocks carry it across tiles)
};

// One direction for the lane's cells; hop (CX, CY), paused or propagating.
template <typename T, bool REF, int CX, int CY, bool PAUSED>
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
      // pairs (same rounded operations; x - y as fma(y, -1, x))
      const float2 wi2 = make_float2(c.wi, c.wi);
#pragma unroll
      for (int jp = 0; jp < 4; jp += 2) {
        const float2 g2 = make_float2(t.G[SR][SC + jp], t.G[SR][SC + jp + 1]);
        const float2 v2 = make_float2(v[jp], v[jp + 1]);
        float2 m2;
        if constexpr (REF) {
          const float2 x2 = make_float2(t.X[SR][SC + jp], t.X[SR][SC + jp + 1]);
          const float2 e2 = make_float2(t.eins[k][jp], t.eins[k][jp + 1]);
          m2 = __fmul2_rn(wi2, __ffma2_rn(e2, make_float2(-1.f, -1.f), x2));
        } else {
          m2 = __fmul2_rn(wi2, make_float2(t.X[FR][FC + jp], t.X[FR][FC + jp + 1]));
        }
        const float2 o2 = __ffma2_rn(g2, v2, m2);
        o[jp] = o2.x;
        o[jp + 1] = o2.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if constexpr (REF) {
          // stored v' = (d' - w_i E_in(y)) / scale, d' from Eq. lbm-energy with the local
          // reference R of the stored source value (see the bfloat16 storage note)
          const float tt =
              PAUSED ? __fadd_rn(__fsub_rn(t.X[1 + k][1 + j], c.fsc[((1 + k) * 6 + 1 + j) * 32]),
                                 c.fsc[(FR * 6 + FC + j) * 32])
                     : t.X[SR][SC + j];
          o[j] = fmaf(t.G[SR][SC + j], v[j], __fmul_rn(c.wi, __fsub_rn(tt, t.eins[k][j])));
        } else {
          o[j] = fmaf(t.G[SR][SC + j], v[j], __fmul_rn(c.wi, t.X[FR][FC + j]));
        }
      }
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

template <int CX, bool PAUSED, bool FULL>
__device__ __forceinline__ void dir_body_ref(Regs3& t, const DirCtx<__nv_bfloat16>& c,
                                             const float2 (&Gk)[kRPW][2],
                                             const float2 (&Dk)[kRPW][2]) {
  constexpr int BW = kTW3 + 2 * (16 / int(sizeof(__nv_bfloat16)));   // ring row length
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
// kind-sorted table.  Returns false when a bounded wait gave up.
template <typename T, int S, bool REF, int CX, int CY, bool PAUSED, bool FULL>
__device__ __forceinline__ bool run_kind(int& j, int end, Regs3& t, DirCtx<T>& c, float& accw,
                                         const Dir3* table, const unsigned char* smem,
                                         uint64_t* full, uint64_t* empty, T* obase, int ty,
                                         int* status) {
  using LY = TmaLayout<T, S>;
  // bfloat16: the per-kind parts of the update of the lane's cells, computed once per kind
  // (same float32 operations, in the same order, as computing them per direction):
  //   propagating  Gk = 1 - W(s),  D = X(s) - E_in(y) / scale
  //   paused       Gk = 1 - W(y),  D = (X(y) - W(y) E(y) / scale) + W(s) E(s) / scale
  //                                    - E_in(y) / scale
  // with s = y - c and X = ((1 - W) R + W E) / scale (R: the reference energy of the
  // stored values the step reads, E their local energy).
  float2 Gk[kRPW][2], Dk[kRPW][2];
  if constexpr (REF) {
    if (j < end) {
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
              PAUSED ? __fadd_rn(__fsub_rn(t.X[1 + k][1 + q], c.fsc[((1 + k) * 6 + 1 + q) * 32]),
                                 c.fsc[(FR * 6 + FC + q) * 32])
                     : t.X[SR][SC + q];
          d[q] = __fsub_rn(tt, t.eins[k][q]);
        }
        Gk[k][0] = make_float2(g[0], g[1]);
        Gk[k][1] = make_float2(g[2], g[3]);
        Dk[k][0] = make_float2(d[0], d[1]);
        Dk[k][1] = make_float2(d[2], d[3]);
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
    c.ring_row = reinterpret_cast<const T*>(smem + st * LY::kStage) + kRPW * ty * LY::BW;
    c.dst = obase + d.dst;
    c.wi = d.wi;
    if constexpr (REF) {
      accw += d.wi;
      if (FULL || c.vm) dir_body_ref<CX, PAUSED, FULL>(t, c, Gk, Dk);
    } else {
      if (c.vm) dir_body<T, REF, CX, CY, PAUSED>(t, c);
    }
    __syncwarp();
    mbar_arrive_if(&empty[st], c.lane == 0);
  }
  return true;
}

// One 128 x 14 tile (bx, by) of one grid; `tmap` is the generic address of the planes'
// tensor map (kernel parameter or global memory), `smem` the block's dynamic shared memory.
// Returns false when a bounded wait gave up (the status word is then set).
// PERSIST: a block that runs many tiles in turn (the persistent batched kernel).  Its
// barriers were initialised once by the caller (the empty ones for all kWarps3 consumer
// warps); g0 counts the ring uses of the block's earlier tiles (stage and phase of use g
// are g % S and (g / S) & 1) and is advanced by q; every thread returns (consumer warps
// without rows wait for and release every box) so that the caller can synchronise.
template <typename T, int S, bool FIELD_W, bool REF, bool PERSIST = false>
__device__ __forceinline__ bool step_tma_tile(const StepArgs& a, const void* tmap, int bx,
                                              int by, unsigned char* smem, uint32_t& g0) {
  using LY = TmaLayout<T, S>;
  constexpr int V = LY::V;
  // smem: S ring stages of [kRows3][BW] elements (stride kStage), the bfloat16 W E
  // scratch, the barriers, the direction table
  float* fscr = reinterpret_cast<float*>(smem + LY::off_f);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);      // [S]
  uint64_t* empty = full + S;                                            // [S]
  Dir3* table = reinterpret_cast<Dir3*>(smem + LY::off_table);           // [q]

  // warps of 32 threads, linear in (threadIdx.x, threadIdx.y): blocks of (32, 8) and of 256
  const int tid = int(threadIdx.y * blockDim.x + threadIdx.x), nthr = 32 * (kWarps3 + 1);
  const int lane = tid & 31, ty = tid >> 5;
  const int col0 = a.cbase + bx * kTW3;
  const int row0 = a.rmin + by * kRows3;
  const int nrows = min(kRows3, a.rmax - row0 + 1);     // rows row0 .. rmax are computed
  const int nwarps = (nrows + kRPW - 1) / kRPW;         // consumer warps with rows

  int* kind_start = reinterpret_cast<int*>(smem + LY::off_kind);         // [17]
  for (int k = tid; k <= 16; k += nthr) kind_start[k] = a.order[a.q + k];
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
    table[j] = d;
  }
  if (!PERSIST && tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], nwarps > 0 ? nwarps : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows <= 0) return true;
  const uint32_t gbase = PERSIST ? g0 : 0u;
  if (PERSIST) g0 += uint32_t(a.q);

  if (ty == kWarps3) {
    // ------------------------------------------------------------- producer thread
    if (lane != 0) return true;
    // the planes may have been written by other blocks of this kernel (persistent form):
    // order the tensor copies after those generic-proxy writes
    if (PERSIST) asm volatile("fence.proxy.async.global;" ::: "memory");
    for (int i = 0; i < a.q; ++i) {
      const uint32_t g = gbase + uint32_t(i);
      const int st = int(g % S);
      const uint32_t k = g / S;
      if (k > 0 && !mbar_wait(&empty[st], (k - 1) & 1u, kWaitCycles)) {
        atomicOr(a.status, 1);
        for (int j = (i > S ? i - S : 0); j < i; ++j) {   // copies still in flight
          const uint32_t gj = gbase + uint32_t(j);
          mbar_wait(&full[gj % S], (gj / S) & 1u, kWaitCycles);
        }
        return false;
      }
      const Dir3 d = table[i];
      mbar_expect(&full[st], LY::kBoxBytes);
      tma_load_3d(smem + st * LY::kStage, tmap, col0 - V, row0 + (d.zdy & 3) - 1, d.zdy >> 2,
                  &full[st]);
    }
    return true;
  }

  // ---------------------------------------------------------------- consumer warps
  if (ty >= nwarps) {
    if (!PERSIST) return true;
    // no rows here: wait for every box and release it, so that the block's barriers
    // keep one phase per ring use
    for (int i = 0; i < a.q; ++i) {
      const uint32_t g = gbase + uint32_t(i);
      if (!mbar_wait(&full[g % S], (g / S) & 1u, kWaitCycles)) {
        if (lane == 0) atomicOr(a.status, 1);
        return false;
      }
      __syncwarp();
      mbar_arrive_if(&empty[g % S], lane == 0);
    }
    return true;
  }
  const int r = row0 + kRPW * ty;                      // first row of this warp
  const int nrw = min(kRPW, a.rmax - r + 1);           // 1 or 2 computed rows
  const int c0 = col0 + 4 * lane;
  unsigned vm = 0;                                     // computed cells of the lane
#pragma unroll
  for (int j = 0; j < 4; ++j) vm |= (c0 + j >= a.cmin && c0 + j <= a.cmax) ? 1u << j : 0u;
  float* fsc = fscr + size_t(ty) * kTR * 6 * 32 + lane;
  Regs3 t;
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
        if (REF) rv = a.e_ref[o];
      }
      const float fv = __fmul_rn(wv, ev), gv = __fsub_rn(1.f, wv);
      t.G[rr][cc] = gv;
      if (REF) {
        const float fs = __fmul_rn(fv, a.inv_scale);
        const float xs = __fmul_rn(fmaf(gv, rv, fv), a.inv_scale);
        t.X[rr][cc] = xs;
        fsc[(rr * 6 + cc) * 32] = fs;
        if (rr >= 1 && rr <= kRPW && cc >= 1 && cc <= 4)
          t.eins[rr - 1][cc - 1] = ((vm >> (cc - 1)) & 1u) ? __fmul_rn(ev, a.inv_scale) : 0.f;
      } else {
        t.X[rr][cc] = fv;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kRPW; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) t.acc[k][j] = 0.f;
  float accw = 0.f;
  DirCtx<T> ctx;
  ctx.fsc = fsc;
  ctx.pitch = a.pitch;
  ctx.plane = a.plane;
  ctx.lane = lane;
  ctx.vm = vm;
  ctx.nrw = nrw;
  ctx.g0 = gbase;
  T* obase = static_cast<T*>(a.tape ? a.tape_dst : a.planes) + int64_t(r) * a.pitch + c0;

  // kind = hop | paused << 3; hop numbering of the host lattice:
  // (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P, F)                                                           \
  ok = ok && run_kind<T, S, REF, CX, CY, P, F>(j, kind_start[K + 1], t, ctx, accw, table, smem, \
                                               full, empty, obase, ty, a.status)
#define WLBM_KINDS(F)                \
  WLBM_KIND(0, 1, 0, false, F);      \
  WLBM_KIND(1, 0, 1, false, F);      \
  WLBM_KIND(2, -1, 0, false, F);     \
  WLBM_KIND(3, 0, -1, false, F);     \
  WLBM_KIND(4, 1, 1, false, F);      \
  WLBM_KIND(5, -1, 1, false, F);     \
  WLBM_KIND(6, -1, -1, false, F);    \
  WLBM_KIND(7, 1, -1, false, F);     \
  WLBM_KIND(8, 1, 0, true, F);       \
  WLBM_KIND(9, 0, 1, true, F);       \
  WLBM_KIND(10, -1, 0, true, F);     \
  WLBM_KIND(11, 0, -1, true, F);     \
  WLBM_KIND(12, 1, 1, true, F);      \
  WLBM_KIND(13, -1, 1, true, F);     \
  WLBM_KIND(14, -1, -1, true, F);    \
  WLBM_KIND(15, 1, -1, true, F)
  // bfloat16: warps whose lanes all compute 4 cells of 2 rows take loops without the
  // row and edge checks
  const bool wfull = REF && nrw == kRPW && __all_sync(0xffffffffu, vm == 0xFu);
  if (wfull) {
    WLBM_KINDS(true);
  } else {
    WLBM_KINDS(false);
  }
#undef WLBM_KINDS
#undef WLBM_KIND
  if (!ok) return false;
  // E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density); bfloat16: d' = scale v' + w_i E_in(y)
#pragma unroll
  for (int k = 0; k < kRPW; ++k) {
    if (k >= nrw) break;
    const int64_t own = int64_t(r + k) * a.pitch + c0;
    float eo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float ein = REF && ((vm >> j) & 1u) ? a.e_in[own + j] : 0.f;
      eo[j] = REF ? fmaf(t.acc[k][j], a.scale, __fmul_rn(ein, accw)) : t.acc[k][j];
    }
    float* e_out = a.e_out + own;
    if (vm == 0xFu) {
      *reinterpret_cast<float4*>(e_out) = make_float4(eo[0], eo[1], eo[2], eo[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((vm >> j) & 1u) e_out[j] = eo[j];
    }
  }
  return true;
}

}  // namespace

}  // namespace wlbm
