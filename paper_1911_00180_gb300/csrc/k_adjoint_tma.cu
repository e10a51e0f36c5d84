// Reverse step with TMA tiles (float32 storage): the transpose of one forward step, as
// k_adj_step computes it (see k_adjoint.cu for the algebra), organised like the forward
// step kernel k_step_tma:
//   * one producer thread per block issues, for direction k, a tensor box of the output
//     adjoint's plane k and a 14 x 128 box (no column halo) of plane k of the recorded step
//     input d~, into one stage of a 6-stage ring (full/empty mbarriers, bounded waits).  A
//     propagating direction reads only l'(x + c_k): its adjoint box is the tile's 14 rows
//     shifted by c_k's row; a paused one also reads l'(x): its box is the tile's 14 rows
//     and, for a hop with a vertical component, the one row beyond them on c_k's side (15
//     rows).  So the halo rows are fetched only where they are needed;
//   * 7 consumer warps own 2 rows each, a lane 4 consecutive cells; the shared part s' of
//     the 4 x 6 cells around them sits in registers;
//   * the step's directions run sorted by kind (hop, paused), as 16 loops with
//     compile-time neighbour offsets; every direction's new lh_k = (1 - W) a_k leaves with
//     one 16-byte streaming store per lane and row.
// Tiles cover the whole frame (the boundary transposes need the ghost cells' adjoint),
// from the 16-byte aligned column at or below the left ghost column.
#include <cuda.h>

#include "elem.cuh"
#include "mbar.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kAW = 7;                     // consumer warps per block; + 1 producer warp
constexpr int kARPW = 2;                   // rows per consumer warp
constexpr int kARows = kAW * kARPW;        // rows per tile
constexpr int kATW = 128;                  // columns per tile
constexpr int kAV = 4;                     // floats per 16 bytes
constexpr int kABW = kATW + 2 * kAV;       // box width
constexpr int kAC0 = kGhostCol & ~3;       // first column of the first tile
constexpr int kAS = 6;                     // ring stages (swept: 4, 6, 8 stages took the
                                           // 1000-step backward pass 283.7, 278.7, 288.1 ms)
constexpr uint32_t kBoxL = uint32_t(kAdjTmaBoxRows) * kABW * 4;   // adjoint box (paused)
constexpr uint32_t kBoxL14 = uint32_t(kAdjTmaRows) * kABW * 4;    // adjoint box (14 rows)
constexpr uint32_t kBoxLSlot = (kBoxL + 127) / 128 * 128;         // tape box offset
constexpr uint32_t kBoxD = uint32_t(kARows) * kATW * 4;           // tape box bytes
constexpr size_t kAStage = (size_t(kBoxLSlot) + kBoxD + 127) / 128 * 128;
constexpr size_t kAOffBar = kAS * kAStage;
constexpr size_t kAOffKind = kAOffBar + 2 * kAS * 8;          // 17 ints
constexpr size_t kAOffWall = kAOffKind + 17 * 4;              // 4 floats
constexpr size_t kAOffTable = (kAOffWall + 4 * 4 + 127) / 128 * 128;
static_assert(kAdjTmaBoxRows == kARows + 1, "one halo row on the side of c_k");
static_assert(kAdjTmaRows == kARows && kAdjTmaCols == kATW, "tile-sized boxes");

struct alignas(16) AdjDir3 {
  int32_t k;        // direction index
  float wk;         // w_k
  int32_t z_tape;   // tape plane of direction k
  int32_t kind;     // hop | paused << 3
};

size_t adj_tma_bytes(int q) { return kAOffTable + size_t(q) * sizeof(AdjDir3); }

struct AdjRegs {
  float sr[kARPW + 2][6];                  // s' of rows r-1 .. r+2, columns c0-1 .. c0+4
  float keep[kARPW][4];                    // 1 - W (0 on isothermal wall cells)
  float sigma[kARPW][4], a0[kARPW][4], ed[kARPW][4], pd[kARPW][4], h[kARPW][4];
};

// 4 consecutive floats of a box row at column offset kAV + 4 lane + DX (DX = -1, 0, +1).
template <int DX>
__device__ __forceinline__ void row_vals(const float* row, int lane, float (&v)[4]) {
  const float* p = row + kAV + 4 * lane;   // 16-byte aligned
  const float4 q = *reinterpret_cast<const float4*>(p);
  if constexpr (DX == 0) {
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (DX < 0) {
    v[0] = p[-1]; v[1] = q.x; v[2] = q.y; v[3] = q.z;
  } else {
    v[0] = q.y; v[1] = q.z; v[2] = q.w; v[3] = p[4];
  }
}

struct AdjCtx {
  const float* boxl;    // adjoint box of the stage, row 0 = tile row -1
  const float* boxd;    // tape box of the stage, row 0 = tile row 0
  float* dst;           // lh_out of the lane's first cell (warp's first row, plane k)
  int64_t pitch;
  float wk;
  int lane, ty, nrw;
  unsigned vm;
  bool first, harvest;
};

template <int CX, int CY, bool PAUSED>
__device__ __forceinline__ void adj_body(AdjRegs& t, const AdjCtx& c) {
#pragma unroll
  // a paused direction's box starts at tile row OFF (one row above the tile for a hop
  // downwards), a propagating direction's at c_k's row
  constexpr int OFF = CY < 0 ? -1 : 0;
#pragma unroll
  for (int k = 0; k < kARPW; ++k) {
    if (k >= c.nrw) break;
    const int tr = kARPW * c.ty + k;               // tile row of cell row r + k
    float b[4], av[4], dv[4], o[4];
    // l'(x + c_k): row tr - OFF + CY of a paused direction's box, row tr of a propagating
    // direction's box
    row_vals<CX>(c.boxl + (PAUSED ? tr - OFF + CY : tr) * kABW, c.lane, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] += t.sr[1 + k + CY][1 + j + CX];
    if constexpr (PAUSED) {
      row_vals<0>(c.boxl + (tr - OFF) * kABW, c.lane, av);
#pragma unroll
      for (int j = 0; j < 4; ++j) av[j] += t.sr[1 + k][1 + j];
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) av[j] = b[j];
    }
    {
      const float4 q = *reinterpret_cast<const float4*>(c.boxd + tr * kATW + 4 * c.lane);
      dv[0] = q.x; dv[1] = q.y; dv[2] = q.z; dv[3] = q.w;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t.sigma[k][j] = fmaf(c.wk, b[j], t.sigma[k][j]);
      if (c.first) t.a0[k][j] = av[j];
      t.ed[k][j] += dv[j];
      t.pd[k][j] = fmaf(dv[j], av[j] - t.a0[k][j], t.pd[k][j]);
      if (c.harvest) t.h[k][j] = fmaf(c.wk, av[j], t.h[k][j]);
      o[j] = t.keep[k][j] * av[j];
    }
    float* po = c.dst + k * c.pitch;
    if (c.vm == 0xFu) {
      __stcs(reinterpret_cast<float4*>(po), make_float4(o[0], o[1], o[2], o[3]));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if ((c.vm >> j) & 1u) po[j] = o[j];
    }
  }
}

template <int CX, int CY, bool PAUSED>
__device__ __forceinline__ bool adj_kind(int& j, int end, AdjRegs& t, AdjCtx& c,
                                         const AdjDir3* table, const unsigned char* smem,
                                         uint64_t* full, uint64_t* empty, float* obase,
                                         int64_t plane, int* status) {
  for (; j < end; ++j) {
    const int st = j % kAS;
    if (!mbar_wait(&full[st], uint32_t(j / kAS) & 1u, kWaitCycles)) {
      if (c.lane == 0) atomicOr(status, 1);
      return false;
    }
    const AdjDir3 d = table[j];
    c.boxl = reinterpret_cast<const float*>(smem + st * kAStage);
    c.boxd = reinterpret_cast<const float*>(smem + st * kAStage + kBoxLSlot);
    c.dst = obase + int64_t(d.k) * plane;
    c.wk = d.wk;
    c.first = j == 0;
    if (c.vm) adj_body<CX, CY, PAUSED>(t, c);
    __syncwarp();
    if (c.lane == 0) mbar_arrive(&empty[st]);
  }
  return true;
}

__global__ void __maxnreg__(128)
    k_adj_tma(const AdjArgs a, const __grid_constant__ CUtensorMap lam_map,
              const __grid_constant__ CUtensorMap lam_map14,
              const __grid_constant__ CUtensorMap tape_map, int tape_z0, const uint16_t* order,
              int* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kAOffBar);
  uint64_t* empty = full + kAS;
  int* kind_start = reinterpret_cast<int*>(smem + kAOffKind);
  AdjDir3* table = reinterpret_cast<AdjDir3*>(smem + kAOffTable);
  float* hwall = reinterpret_cast<float*>(smem + kAOffWall);   // isothermal harvest per wall

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane, nthr = 32 * (kAW + 1);
  const int col0 = kAC0 + int(blockIdx.x) * kATW;
  const int row0 = 1 + int(blockIdx.y) * kARows;
  const int nrows = min(kARows, a.ny + 2 - row0 + 1);
  const int nwarps = (nrows + kARPW - 1) / kARPW;

  for (int k = tid; k <= 16; k += nthr) kind_start[k] = order[a.q + k];
  for (int j = tid; j < a.q; j += nthr) {
    const int k = order[j];
    AdjDir3 d;
    d.k = k;
    d.wk = a.w[k];
    d.z_tape = tape_z0 + k;
    d.kind = a.codes[k] & 15;
    table[j] = d;
  }
  if (tid < 4) hwall[tid] = 0.f;
  if (tid == 0) {
    for (int st = 0; st < kAS; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], nwarps > 0 ? nwarps : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows <= 0) return;

  if (ty == kAW) {
    // ------------------------------------------------------------- producer thread
    if (lane != 0) return;
    for (int j = 0; j < a.q; ++j) {
      const int st = j % kAS, k = j / kAS;
      if (k > 0 && !mbar_wait(&empty[st], uint32_t(k - 1) & 1u, kWaitCycles)) {
        atomicOr(status, 1);
        for (int i = (j > kAS ? j - kAS : 0); i < j; ++i)   // copies still in flight
          mbar_wait(&full[i % kAS], uint32_t(i / kAS) & 1u, kWaitCycles);
        return;
      }
      const AdjDir3 d = table[j];
      unsigned char* stage = smem + st * kAStage;
      const int cy = c_hop_y[d.kind & 7];
      if ((d.kind & 8) && cy != 0) {   // paused, vertical component: l'(x) and l'(x + c_k)
        mbar_expect(&full[st], kBoxL + kBoxD);
        tma_load_3d(stage, &lam_map, col0 - kAV, row0 + (cy < 0 ? -1 : 0), d.k, &full[st]);
      } else {   // propagating: l'(x + c_k) only; paused horizontal: the tile's rows
        mbar_expect(&full[st], kBoxL14 + kBoxD);
        tma_load_3d(stage, &lam_map14, col0 - kAV, row0 + ((d.kind & 8) ? 0 : cy), d.k,
                    &full[st]);
      }
      tma_load_3d(stage + kBoxLSlot, &tape_map, col0, row0, d.z_tape, &full[st]);
    }
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  if (ty >= nwarps) return;
  const int r = row0 + kARPW * ty;
  const int nrw = min(kARPW, a.ny + 2 - r + 1);
  const int c0 = col0 + 4 * lane;
  const int clast = kX0 + a.nx;
  unsigned vm = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) vm |= (c0 + j >= kGhostCol && c0 + j <= clast) ? 1u << j : 0u;
  const int rows = a.ny + 4;
  AdjRegs t;
#pragma unroll
  for (int rr = 0; rr < kARPW + 2; ++rr)
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const int rw = r - 1 + rr, c = c0 - 1 + cc;
      t.sr[rr][cc] = (rw < rows && c >= 0 && c < a.pitch) ? a.s_in[int64_t(rw) * a.pitch + c]
                                                          : 0.f;
    }
  bool any_iso = false;
#pragma unroll
  for (int k = 0; k < kARPW; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool on = k < nrw && ((vm >> j) & 1u);
      const int iso = on ? iso_wall_of(a, r + k, c0 + j) : -1;
      any_iso = any_iso || iso >= 0;
      t.keep[k][j] = iso >= 0 ? 0.f : 1.f - (on ? w_at(a, r + k, c0 + j) : 0.f);
      t.sigma[k][j] = 0.f; t.a0[k][j] = 0.f; t.ed[k][j] = 0.f; t.pd[k][j] = 0.f;
      t.h[k][j] = 0.f;
    }
  AdjCtx ctx;
  ctx.pitch = a.pitch;
  ctx.lane = lane;
  ctx.ty = ty;
  ctx.nrw = nrw;
  ctx.vm = vm;
  ctx.harvest = any_iso;
  float* obase = a.lam_out + int64_t(r) * a.pitch + c0;

  int j = 0;
  bool ok = true;
#define WLBM_AKIND(K, CX, CY, P)                                                               \
  ok = ok && adj_kind<CX, CY, P>(j, kind_start[K + 1], t, ctx, table, smem, full, empty, obase, \
                                 a.plane, status)
  // kind = hop | paused << 3; hop numbering of the host lattice
  WLBM_AKIND(0, 1, 0, false);
  WLBM_AKIND(1, 0, 1, false);
  WLBM_AKIND(2, -1, 0, false);
  WLBM_AKIND(3, 0, -1, false);
  WLBM_AKIND(4, 1, 1, false);
  WLBM_AKIND(5, -1, 1, false);
  WLBM_AKIND(6, -1, -1, false);
  WLBM_AKIND(7, 1, -1, false);
  WLBM_AKIND(8, 1, 0, true);
  WLBM_AKIND(9, 0, 1, true);
  WLBM_AKIND(10, -1, 0, true);
  WLBM_AKIND(11, 0, -1, true);
  WLBM_AKIND(12, 1, 1, true);
  WLBM_AKIND(13, -1, 1, true);
  WLBM_AKIND(14, -1, -1, true);
  WLBM_AKIND(15, 1, -1, true);
#undef WLBM_AKIND
  if (ok) {
#pragma unroll
    for (int k = 0; k < kARPW; ++k)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        if (k >= nrw || !((vm >> jj) & 1u)) continue;
        const int64_t off = int64_t(r + k) * a.pitch + c0 + jj;
        a.s_out[off] = w_at(a, r + k, c0 + jj) * t.sigma[k][jj];
        a.gw[off] += fmaf(t.sigma[k][jj] - t.a0[k][jj], t.ed[k][jj], -t.pd[k][jj]);
        const int iso = iso_wall_of(a, r + k, c0 + jj);
        if (iso >= 0) atomicAdd(&hwall[iso], t.h[k][jj]);
      }
  }
  // one global atomic per wall and block (named barrier over the consumer warps with rows)
  asm volatile("bar.sync 1, %0;" ::"r"(nwarps * 32) : "memory");
  if (ty == 0 && lane < 4 && hwall[lane] != 0.f) atomicAdd(a.gtw + lane, double(hwall[lane]));
}

}  // namespace

cudaError_t configure_adj_tma() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(adj_tma_bytes(kMaxQ)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_tma, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
  return e;
}

cudaError_t launch_adj_tma(const AdjArgs& a, const void* lam_map, const void* lam_map14,
                           const void* tape_map, int tape_z0, const uint16_t* order,
                           int* status, cudaStream_t s) {
  const dim3 block(32, kAW + 1);
  const dim3 grid((kX0 + a.nx - kAC0) / kATW + 1, (a.ny + 2 + kARows - 1) / kARows);
  k_adj_tma<<<grid, block, adj_tma_bytes(a.q), s>>>(
      a, *static_cast<const CUtensorMap*>(lam_map), *static_cast<const CUtensorMap*>(lam_map14),
      *static_cast<const CUtensorMap*>(tape_map), tape_z0, order, status);
  return cudaGetLastError();
}

}  // namespace wlbm
