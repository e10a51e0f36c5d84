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
  int32_t dst;       // destination plane index (from the output base)
  float wi;          // angular weight w_i
  int32_t z;         // source plane index (tensor-map z coordinate)
  uint8_t kase;      // hop | paused << 3
  int8_t dy;         // source row shift of the box (0 when paused)
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

// All directions of one kind (hop (CX, CY), paused or not): entries j .. end-1 of the
// kind-sorted table.  Returns false when a bounded wait gave up.
template <typename T, int S, bool REF, int CX, int CY, bool PAUSED>
__device__ __forceinline__ bool run_kind(int& j, int end, Regs3& t, DirCtx<T>& c, float& accw,
                                         const Dir3* table, const unsigned char* smem,
                                         uint64_t* full, uint64_t* empty, T* obase, int ty,
                                         int* status) {
  using LY = TmaLayout<T, S>;
  for (; j < end; ++j) {
    const int st = j % S;
    if (!mbar_wait(&full[st], uint32_t(j / S) & 1u, kWaitCycles)) {
      if (c.lane == 0) atomicOr(status, 1);
      return false;
    }
    const Dir3 d = table[j];
    c.ring_row = reinterpret_cast<const T*>(smem + st * LY::kStage) + kRPW * ty * LY::BW;
    c.dst = obase + int64_t(d.dst) * c.plane;
    c.wi = d.wi;
    if (REF) accw += d.wi;
    if (c.vm) dir_body<T, REF, CX, CY, PAUSED>(t, c);
    __syncwarp();
    if (c.lane == 0) mbar_arrive(&empty[st]);
  }
  return true;
}

// One 128 x 14 tile (bx, by) of one grid; `tmap` is the generic address of the planes'
// tensor map (kernel parameter or global memory), `smem` the block's dynamic shared memory.
template <typename T, int S, bool FIELD_W, bool REF>
__device__ __forceinline__ void step_tma_tile(const StepArgs& a, const void* tmap, int bx,
                                              int by, unsigned char* smem) {
  using LY = TmaLayout<T, S>;
  constexpr int V = LY::V;
  // smem: S ring stages of [kRows3][BW] elements (stride kStage), the bfloat16 W E
  // scratch, the barriers, the direction table
  float* fscr = reinterpret_cast<float*>(smem + LY::off_f);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);      // [S]
  uint64_t* empty = full + S;                                            // [S]
  Dir3* table = reinterpret_cast<Dir3*>(smem + LY::off_table);           // [q]

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane, nthr = 32 * (kWarps3 + 1);
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
    d.dst = a.tape ? i : (paused ? par : 1 - par) * a.q + i;
    d.wi = a.w[i];
    d.z = a.tape ? a.tape_z0 + i : par * a.q + i;
    d.kase = uint8_t(hop | (paused << 3));
    d.dy = int8_t(paused ? 0 : -c_hop_y[hop]);
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
    // ------------------------------------------------------------- producer thread
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
      tma_load_3d(smem + st * LY::kStage, tmap, col0 - V, row0 + d.dy, int(d.z), &full[st]);
    }
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  if (ty >= nwarps) return;
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
  T* obase = static_cast<T*>(a.tape ? a.tape_dst : a.planes) + int64_t(r) * a.pitch + c0;

  // kind = hop | paused << 3; hop numbering of the host lattice:
  // (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
  int j = 0;
  bool ok = true;
#define WLBM_KIND(K, CX, CY, P)                                                            \
  ok = ok && run_kind<T, S, REF, CX, CY, P>(j, kind_start[K + 1], t, ctx, accw, table, smem, \
                                            full, empty, obase, ty, a.status)
  WLBM_KIND(0, 1, 0, false);
  WLBM_KIND(1, 0, 1, false);
  WLBM_KIND(2, -1, 0, false);
  WLBM_KIND(3, 0, -1, false);
  WLBM_KIND(4, 1, 1, false);
  WLBM_KIND(5, -1, 1, false);
  WLBM_KIND(6, -1, -1, false);
  WLBM_KIND(7, 1, -1, false);
  WLBM_KIND(8, 1, 0, true);
  WLBM_KIND(9, 0, 1, true);
  WLBM_KIND(10, -1, 0, true);
  WLBM_KIND(11, 0, -1, true);
  WLBM_KIND(12, 1, 1, true);
  WLBM_KIND(13, -1, 1, true);
  WLBM_KIND(14, -1, -1, true);
  WLBM_KIND(15, 1, -1, true);
#undef WLBM_KIND
  if (!ok) return;
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
}

template <typename T, int S, bool FIELD_W, bool REF>
__global__ void __maxnreg__(128)
    k_step_tma(const StepArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem[];
  step_tma_tile<T, S, FIELD_W, REF>(a, &tmap, int(blockIdx.x), int(blockIdx.y), smem);
}

// Batched form: block b belongs to the instance whose first_tile is the largest one <= b;
// the instance's tensor map sits in global memory.
template <typename T, int S, bool REF>
__global__ void __maxnreg__(128) k_step_tma_batch(const BatchInst* insts, int n, int t) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ const void* tm;
  __shared__ int tile[2];
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int lo = 0, hi = n - 1;
    const int b = int(blockIdx.x);
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (insts[mid].first_tile <= b) lo = mid;
      else hi = mid - 1;
    }
    const BatchInst& I = insts[lo];
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
  if (sa.wfield) step_tma_tile<T, S, true, REF>(sa, tm, tile[0], tile[1], smem);
  else step_tma_tile<T, S, false, REF>(sa, tm, tile[0], tile[1], smem);
}

// BATCH: also the batched form of the same storage and ring depth.
template <typename T, int S, bool BATCH>
cudaError_t configure_tma_t() {
  const int bytes = int(TmaLayout<T, S>::bytes(kMaxQ));
  const void* fns[3] = {(const void*)k_step_tma<T, S, false, sizeof(T) == 2>,
                        (const void*)k_step_tma<T, S, true, sizeof(T) == 2>,
                        BATCH ? (const void*)k_step_tma_batch<T, S, sizeof(T) == 2> : nullptr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && fns[k] && e == cudaSuccess; ++k) {
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
  if (a.wfield) k_step_tma<T, S, true, REF><<<grid, block, bytes, s>>>(a, tm);
  else k_step_tma<T, S, false, REF><<<grid, block, bytes, s>>>(a, tm);
  return cudaGetLastError();
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

}  // namespace

cudaError_t configure_step_tma() {
  cudaError_t e = configure_tma_t<float, kStagesF32, true>();
  if (e == cudaSuccess) e = configure_tma_t<__nv_bfloat16, kStagesBF16, true>();
  if (e == cudaSuccess) e = configure_tma_t<__nv_bfloat16, kStagesBF16Deep, false>();
  if (e == cudaSuccess) e = configure_tma_t<float, kStagesF32Shallow, false>();
  return e;
}

cudaError_t launch_step_tma_batch(int storage, const BatchInst* insts, int n, int max_q,
                                  int total_tiles, int t, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  const dim3 block(32, kWarps3 + 1);
  if (storage == WLBM_STORE_BF16_DEV) {
    using LY = TmaLayout<__nv_bfloat16, kStagesBF16>;
    k_step_tma_batch<__nv_bfloat16, kStagesBF16, true>
        <<<total_tiles, block, LY::bytes(max_q), s>>>(insts, n, t);
  } else {
    using LY = TmaLayout<float, kStagesF32>;
    k_step_tma_batch<float, kStagesF32, false><<<total_tiles, block, LY::bytes(max_q), s>>>(insts, n, t);
  }
  return cudaGetLastError();
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

cudaError_t launch_step_tma(int storage, const StepArgs& a, cudaStream_t s) {
  const CUtensorMap& tm = *static_cast<const CUtensorMap*>(a.tmap);
  if (storage == WLBM_STORE_BF16_DEV)
    return a.q <= kDeepMaxQ ? launch_tma_t<__nv_bfloat16, kStagesBF16Deep>(a, tm, s)
                            : launch_tma_t<__nv_bfloat16, kStagesBF16>(a, tm, s);
  return a.q <= kDeepMaxQ ? launch_tma_t<float, kStagesF32>(a, tm, s)
                          : launch_tma_t<float, kStagesF32Shallow>(a, tm, s);
}

// Tensor map of the 2q direction planes as a 3-D tensor (columns, rows, planes) with the
// box of one TMA stage.  The encoder comes from the driver through the runtime's entry
// point query, so the library does not link the driver library directly.
bool make_plane_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                           std::string* why) {
  return make_box_tensor_map(out, planes, storage, g, nplanes, kRows3, why);
}

bool make_box_tensor_map(void* out, void* planes, int storage, const Geom& g, int nplanes,
                         int box_rows, std::string* why) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      *why = "cuTensorMapEncodeTiled is not available from the driver";
      return false;
    }
    encode = reinterpret_cast<Encode>(fn);
  }
  const bool bf = storage == WLBM_STORE_BF16_DEV;
  const cuuint64_t es = bf ? 2 : 4;
  const cuuint32_t V = cuuint32_t(16 / es);
  const cuuint64_t dims[3] = {cuuint64_t(g.pitch), cuuint64_t(g.rows), cuuint64_t(nplanes)};
  const cuuint64_t strides[2] = {cuuint64_t(g.pitch) * es, cuuint64_t(g.plane) * es};
  const cuuint32_t box[3] = {cuuint32_t(kTW3) + 2 * V, cuuint32_t(box_rows), 1};
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
