// Boundary, initialisation, moment and reduction kernels of libwlbm.
//
//  k_walls     ghost cells of non-periodic walls (Sec. 2.6): isotropic blackbody walls
//              overwrite d_i = w_i (e_eq(T_w) - e_ref) (Eq. isotropic); adiabatic diffuse
//              walls collect the components that do not point into the domain and
//              re-emit them into the inward ones with fractions w_i (s_i.n) / sum
//              (Eq. adiabatic-diffuse, normalised so that energy is conserved).
//  k_periodic  periodic links (Sec. 2.6): ghost rows copy the opposite interior rows,
//              then ghost columns copy the opposite columns (corners via the diagonal);
//              before a step, per plane only the side that step's hop pulls from.
//  k_sources   internal temperature / radiation sources (Sec. 2.6): listed cells take fixed
//              values every step.
//  k_init      local equilibrium start e_i = w_i e_eq(T) (Sec. 2.4) in float64.
//  k_moments   T - T_ref by Eq. pseudo-T in a cancellation-free form, q by Eq. q_corr.
//  k_reduce    float64 sums: energy (interior, + adiabatic-wall ghost cells), heat flux
//              (all cells and the central band of columns), band energy moment for the
//              conductivity fit, and the largest temperature change since the previous
//              reduction (and between window means, for the steady-state run).
#include <algorithm>

#include "elem.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

__device__ __forceinline__ int parity_of(const ParityMask& m, int i) {
  return (m.bits[i >> 5] >> (i & 31)) & 1;
}

// Deviation d_i of a stored value (float32: the value itself; bfloat16: scale * v +
// w_i R at a cell whose reference energy is R, see wlbm_internal.hpp).
template <typename T>
__device__ __forceinline__ float dev_load(const T* p, float wi, const float* ref, int64_t off,
                                          float scale) {
  const float v = Elem<T>::ld(p);
  return ref ? fmaf(v, scale, __fmul_rn(wi, ref[off])) : v;
}

// Store deviation d; returns the deviation the stored value represents.
template <typename T>
__device__ __forceinline__ float dev_store(T* p, float d, float wi, const float* ref,
                                           int64_t off, float scale, float inv_scale) {
  if (!ref) return Elem<T>::st(p, d);
  // explicitly rounded operations: the same bits in every kernel that inlines this
  const float r = __fmul_rn(wi, ref[off]);
  return fmaf(Elem<T>::st(p, __fmul_rn(__fsub_rn(d, r), inv_scale)), scale, r);
}

// Wall pass.  Horizontal walls: a block of kWallWarps warps takes a chunk of 128
// consecutive ghost cells, lane l the four cells 4l .. 4l+3 of it (one 16-byte float32 or
// 8-byte bfloat16 access per direction: a warp moves 512 or 256 contiguous bytes of a row
// at once), and warp w the directions w, w + kWallWarps, ...; diffuse walls add the
// collected directions per warp, then over the warps in a fixed order, and re-read the
// values (from L2) to store them.  Vertical walls and corners: one warp per cell
// (walls_cell), which keeps many warps busy on the few, strided cells.
constexpr int kWallWarps = 8;
constexpr int kHoldCell = 8;     // values per lane held at once by a warp on one cell
static_assert(kWallChunk == 128, "four consecutive ghost cells per lane of a chunk");
static_assert(kWallCellsPerBlock == kWallWarps, "one warp per cell of a block");

// Per-direction data of a wall block in shared memory: plane parity of the step, w_i and
// the segment's re-emission fractions, staged once so that no value load waits on them.
struct WallSmem {
  float part[kWallWarps * 32 * 4];   // per warp, lane and lane cell: collected energy
  float w[kMaxQ];
  float rho[kMaxQ];
  int16_t src[kMaxQ];    // mirror direction at this wall (specular segments)
  uint8_t par[kMaxQ];
};

// Deviation of a stored value (bfloat16: scale * v + w_i R with the cell's reference R) and
// its inverse for a store; the same rounded operations as dev_load / dev_store.
template <typename T>
__device__ __forceinline__ float wall_load(const T* p, float wi, bool ref, float R, float scale) {
  const float v = Elem<T>::ld(p);
  return ref ? fmaf(v, scale, __fmul_rn(wi, R)) : v;
}
template <typename T>
__device__ __forceinline__ void wall_store(T* p, float d, float wi, bool ref, float R,
                                           float inv_scale) {
  if (!ref) {
    Elem<T>::st(p, d);
    return;
  }
  Elem<T>::st(p, __fmul_rn(__fsub_rn(d, __fmul_rn(wi, R)), inv_scale));
}

// Four consecutive stored values of a horizontal wall (one 16-byte float32 or 8-byte
// bfloat16 access; the frame's pitch keeps such groups aligned and inside the row).
__device__ __forceinline__ void ld4_raw(const float* p, float (&v)[4]) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void ld4_raw(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
  v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
}
// Store the first nv of four raw values (all four in one access when nv == 4).
__device__ __forceinline__ void st4_raw(float* p, const float (&v)[4], int nv) {
  if (nv == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    for (int j = 0; j < nv; ++j) p[j] = v[j];
  }
}
__device__ __forceinline__ void st4_raw(__nv_bfloat16* p, const float (&v)[4], int nv) {
  if (nv == 4) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&a),
                                              *reinterpret_cast<const uint32_t*>(&b));
  } else {
    for (int j = 0; j < nv; ++j) Elem<__nv_bfloat16>::st(p + j, v[j]);
  }
}
// Deviations of four cells (cell references R) and the raw values that store deviations d:
// the same rounded operations as wall_load / wall_store.
template <typename T>
__device__ __forceinline__ void ld4_dev(const T* p, float wi, bool ref, const float (&R)[4],
                                        float scale, float (&d)[4]) {
  ld4_raw(p, d);
  if (ref) {
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = fmaf(d[j], scale, __fmul_rn(wi, R[j]));
  }
}
template <typename T>
__device__ __forceinline__ void st4_dev(T* p, const float (&d)[4], float wi, bool ref,
                                        const float (&R)[4], float inv_scale, int nv) {
  float v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
    v[j] = ref ? __fmul_rn(__fsub_rn(d[j], __fmul_rn(wi, R[j])), inv_scale) : d[j];
  st4_raw(p, v, nv);
}

// One ghost cell by one warp, lanes over the directions (vertical walls and corners).
// SPEC: the launch has a segment with specularity > 0 (else that code is not compiled in).
template <typename T, bool SPEC>
__device__ __forceinline__ void walls_cell(const WallArgs& a, const WallSmem& sm,
                                           float* e_ref, const WallSeg& g, int idx, int lane) {
  const int64_t off = int64_t(g.r0 + idx * g.dr) * a.pitch + (g.c0 + idx * g.dc);
  T* planes = static_cast<T*>(a.planes);
  auto ptr = [&](int i) { return planes + int64_t(sm.par[i] * a.q + i) * a.plane + off; };
  if (g.action == WLBM_BC_ISOTHERMAL) {
    if (e_ref) {
      for (int i = lane; i < a.q; i += 32) Elem<T>::st(ptr(i), 0.f);
      if (lane == 0) e_ref[off] = g.iso;
    } else {
      for (int i = lane; i < a.q; i += 32) Elem<T>::st(ptr(i), sm.w[i] * g.iso);
    }
    return;
  }
  const bool ref = e_ref != nullptr;
  const float R = ref ? e_ref[off] : 0.f;
  if (a.q <= 32 * kHoldCell) {
    // every value of the cell in flight at once: one load round, one store round
    float val[kHoldCell];
#pragma unroll
    for (int u = 0; u < kHoldCell; ++u) {
      const int i = lane + 32 * u;
      val[u] = i < a.q ? wall_load(ptr(i), sm.w[i], ref, R, a.scale) : 0.f;
    }
    float part = 0.f;
#pragma unroll
    for (int u = 0; u < kHoldCell; ++u) {
      const int i = lane + 32 * u;
      if (i < a.q && sm.rho[i] == 0.f) part += val[u];
    }
    const float A = warp_sum(part);
    if (SPEC && g.spec > 0.f) {
      // inward directions first (they read their mirrors' outward values), then the rest
      const float p = g.spec, Ad = (1.f - g.spec) * A;
#pragma unroll
      for (int u = 0; u < kHoldCell; ++u) {
        const int i = lane + 32 * u;
        if (i >= a.q || sm.rho[i] == 0.f) continue;
        const int j = sm.src[i];
        const float m = wall_load(ptr(j), sm.w[j], ref, R, a.scale);
        wall_store(ptr(i), fmaf(Ad, sm.rho[i], fmaf(p, m, val[u])), sm.w[i], ref, R,
                   a.inv_scale);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kHoldCell; ++u) {
        const int i = lane + 32 * u;
        if (i >= a.q || sm.rho[i] != 0.f) continue;
        wall_store(ptr(i), sm.src[i] == i ? p * val[u] : 0.f, sm.w[i], ref, R, a.inv_scale);
      }
      return;
    }
#pragma unroll
    for (int u = 0; u < kHoldCell; ++u) {
      const int i = lane + 32 * u;
      if (i >= a.q) continue;
      const float d = sm.rho[i] == 0.f ? 0.f : fmaf(A, sm.rho[i], val[u]);
      wall_store(ptr(i), d, sm.w[i], ref, R, a.inv_scale);
    }
    return;
  }
  float part = 0.f;
  for (int i = lane; i < a.q; i += 32)
    if (sm.rho[i] == 0.f) part += wall_load(ptr(i), sm.w[i], ref, R, a.scale);
  const float A = warp_sum(part);
  if (SPEC && g.spec > 0.f) {
    const float p = g.spec, Ad = (1.f - g.spec) * A;
    for (int i = lane; i < a.q; i += 32) {
      if (sm.rho[i] == 0.f) continue;
      const int j = sm.src[i];
      const float m = wall_load(ptr(j), sm.w[j], ref, R, a.scale);
      const float v = wall_load(ptr(i), sm.w[i], ref, R, a.scale);
      wall_store(ptr(i), fmaf(Ad, sm.rho[i], fmaf(p, m, v)), sm.w[i], ref, R, a.inv_scale);
    }
    __syncwarp();
    for (int i = lane; i < a.q; i += 32) {
      if (sm.rho[i] != 0.f) continue;
      const float d = sm.src[i] == i ? p * wall_load(ptr(i), sm.w[i], ref, R, a.scale) : 0.f;
      wall_store(ptr(i), d, sm.w[i], ref, R, a.inv_scale);
    }
    return;
  }
  for (int i = lane; i < a.q; i += 32) {
    const float d = sm.rho[i] == 0.f
                        ? 0.f : fmaf(A, sm.rho[i], wall_load(ptr(i), sm.w[i], ref, R, a.scale));
    wall_store(ptr(i), d, sm.w[i], ref, R, a.inv_scale);
  }
}

// Diffuse (or specular-diffuse) horizontal chunk with every value staged in shared memory
// (vals[i][lane] = the deviations of the lane's four cells in direction i): the block's
// warps load all directions at once (nw warps, directions warp, warp + nw, ...), then
// warps 0 .. kWallWarps-1 add the collected directions in exactly the order of the
// streaming path below (group g: directions g, g + kWallWarps, ... in turn; then the
// groups in turn), so both paths give the same bits, and every output is computed from
// the staged values: one global load and one store per value.
template <typename T, bool SPEC>
__device__ __forceinline__ void walls_staged(const WallArgs& a, const WallSeg& g,
                                             WallSmem& sm, float4* vals, T* const planes,
                                             int64_t off, bool on, int nv, bool ref,
                                             const float (&R)[4], int lane, int warp, int nw) {
  auto ptr = [&](int i) { return planes + int64_t(sm.par[i] * a.q + i) * a.plane + off; };
#pragma unroll 4
  for (int i = warp; i < a.q; i += nw) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    if (on) ld4_dev(ptr(i), sm.w[i], ref, R, a.scale, d);
    vals[i * 32 + lane] = make_float4(d[0], d[1], d[2], d[3]);
  }
  __syncthreads();
  if (warp < kWallWarps) {
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = warp; i < a.q; i += kWallWarps) {
      if (sm.rho[i] != 0.f) continue;
      const float4 v = vals[i * 32 + lane];
      part[0] += v.x; part[1] += v.y; part[2] += v.z; part[3] += v.w;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) sm.part[(warp * 32 + lane) * 4 + j] = part[j];
  }
  __syncthreads();
  if (!on) return;
  float A[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWallWarps; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) A[j] += sm.part[(k * 32 + lane) * 4 + j];
  const float p = SPEC ? g.spec : 0.f;
#pragma unroll 4
  for (int i = warp; i < a.q; i += nw) {
    const float4 f = vals[i * 32 + lane];
    const float v[4] = {f.x, f.y, f.z, f.w};
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    if (SPEC && p > 0.f) {       // uniform over the block (one segment)
      if (sm.rho[i] != 0.f) {
        const float4 mf = vals[sm.src[i] * 32 + lane];
        const float m[4] = {mf.x, mf.y, mf.z, mf.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = fmaf((1.f - p) * A[j], sm.rho[i], fmaf(p, m[j], v[j]));
      } else if (sm.src[i] == i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = p * v[j];
      }
    } else if (sm.rho[i] != 0.f) {
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = fmaf(A[j], sm.rho[i], v[j]);
    }
    st4_dev(ptr(i), d, sm.w[i], ref, R, a.inv_scale, nv);
  }
}

// One block of a wall pass.  vals: the staging buffer of walls_staged (q * 32 float4 of
// dynamic shared memory), or nullptr for the streaming path, which keeps no values
// between its passes and runs with kWallWarps warps.
template <typename T, bool SPEC>
__device__ __forceinline__ void walls_chunk(const WallArgs& a, const uint8_t* codes,
                                            float* e_ref, int chunk, WallSmem& sm,
                                            float4* vals) {
  int c = 0;
  const int s = wall_chunk_segment(a.nseg, a.seg, chunk, &c);
  if (s >= a.nseg) return;                     // uniform over the block
  const WallSeg g = a.seg[s];
  const int lane = int(threadIdx.x) & 31, warp = int(threadIdx.x) >> 5;
  const int nw = int(blockDim.x) >> 5;
  const bool diffuse = g.action != WLBM_BC_ISOTHERMAL;
  const float* rho = a.rho + int64_t(g.table) * a.q;
  const int16_t* mir = a.mirror + int64_t(g.mirror) * a.q;
  for (int i = int(threadIdx.x); i < a.q; i += int(blockDim.x)) {
    sm.par[i] = uint8_t(a.tape ? 0 : (codes[i] >> 4) & 1);
    sm.w[i] = a.w[i];
    sm.rho[i] = diffuse ? rho[i] : 0.f;
    if (SPEC) sm.src[i] = diffuse && g.spec > 0.f ? mir[i] : int16_t(i);
  }
  __syncthreads();
  if (!wall_seg_rowwise(g)) {                  // one warp per cell, lanes over directions
    const int cell = c * kWallCellsPerBlock + warp;
    if (warp < kWallCellsPerBlock && cell < g.count)
      walls_cell<T, SPEC>(a, sm, e_ref, g, cell, lane);
    return;
  }
  // horizontal wall (dr = 0, dc = 1): the block takes cells c*128 .. c*128+127 of the
  // segment; lane owns four consecutive cells, warp w the directions w, w + nw, ...
  const int idx0 = c * kWallChunk + 4 * lane;
  const int nv = min(4, g.count - idx0);          // this lane's valid cells (<= 0: none)
  const bool on = nv > 0;
  const int64_t off = on ? int64_t(g.r0) * a.pitch + (g.c0 + idx0) : 0;
  T* planes = static_cast<T*>(a.planes);
  auto ptr = [&](int i) { return planes + int64_t(sm.par[i] * a.q + i) * a.plane + off; };
  const bool ref = e_ref != nullptr;
  float R[4] = {0.f, 0.f, 0.f, 0.f};
  if (!diffuse) {
    if (!on) return;
    float v[4];
    if (ref) {
      // bfloat16: make the wall's own equilibrium the reference of the cell, so the
      // stored values are exactly zero and decode to w_i (e_eq(T_w) - e_ref) unrounded
      const float z[4] = {0.f, 0.f, 0.f, 0.f};
      for (int i = warp; i < a.q; i += nw) st4_raw(ptr(i), z, nv);
      if (warp == 0)
        for (int j = 0; j < nv; ++j) e_ref[off + j] = g.iso;
    } else {
      for (int i = warp; i < a.q; i += nw) {
        const float x = sm.w[i] * g.iso;
        v[0] = x; v[1] = x; v[2] = x; v[3] = x;
        st4_raw(ptr(i), v, nv);
      }
    }
    return;
  }
  if (ref && on) {
    const float4 r = *reinterpret_cast<const float4*>(e_ref + off);
    R[0] = r.x; R[1] = r.y; R[2] = r.z; R[3] = r.w;
  }
  if (vals) {
    walls_staged<T, SPEC>(a, g, sm, vals, planes, off, on, nv, ref, R, lane, warp, nw);
    return;
  }
  // streaming path (nw == kWallWarps)
  // collected energy per cell: the non-inward directions of this warp, then all warps
  float part[4] = {0.f, 0.f, 0.f, 0.f};
  if (on) {
#pragma unroll 4
    for (int i = warp; i < a.q; i += kWallWarps) {
      if (sm.rho[i] != 0.f) continue;
      float d[4];
      ld4_dev(ptr(i), sm.w[i], ref, R, a.scale, d);
#pragma unroll
      for (int j = 0; j < 4; ++j) part[j] += d[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sm.part[(warp * 32 + lane) * 4 + j] = part[j];
  __syncthreads();
  float A[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWallWarps; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) A[j] += sm.part[(k * 32 + lane) * 4 + j];
  if (SPEC && g.spec > 0.f) {      // uniform over the block (one segment)
    // inward directions first (they read their mirrors' outward values), then the rest
    const float p = g.spec;
    if (on) {
      for (int i = warp; i < a.q; i += kWallWarps) {
        if (sm.rho[i] == 0.f) continue;
        float v[4], m[4], d[4];
        ld4_dev(ptr(i), sm.w[i], ref, R, a.scale, v);
        ld4_dev(ptr(sm.src[i]), sm.w[sm.src[i]], ref, R, a.scale, m);
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = fmaf((1.f - p) * A[j], sm.rho[i], fmaf(p, m[j], v[j]));
        st4_dev(ptr(i), d, sm.w[i], ref, R, a.inv_scale, nv);
      }
    }
    __syncthreads();
    if (!on) return;
    for (int i = warp; i < a.q; i += kWallWarps) {
      if (sm.rho[i] != 0.f) continue;
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      if (sm.src[i] == i) {
        ld4_dev(ptr(i), sm.w[i], ref, R, a.scale, d);
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = p * d[j];
      }
      st4_dev(ptr(i), d, sm.w[i], ref, R, a.inv_scale, nv);
    }
    return;
  }
  if (!on) return;
#pragma unroll 4
  for (int i = warp; i < a.q; i += kWallWarps) {
    // collected directions are absorbed (0); the others receive their share of A
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    if (sm.rho[i] != 0.f) {
      ld4_dev(ptr(i), sm.w[i], ref, R, a.scale, d);
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = fmaf(A[j], sm.rho[i], d[j]);
    }
    st4_dev(ptr(i), d, sm.w[i], ref, R, a.inv_scale, nv);
  }
}

// Single-grid wall pass: kStagedWarps(q) warps and staged values for q <= kStagedMaxQ,
// else the streaming path with kWallWarps warps.
constexpr int kStagedMaxQ = 256;
constexpr int kMaxWallWarps = 32;
inline int staged_warps(int q) { return std::min(kMaxWallWarps, std::max(kWallWarps, q / 4)); }

template <typename T, bool SPEC>
__global__ void __launch_bounds__(32 * kMaxWallWarps) k_walls(const WallArgs a) {
  __shared__ WallSmem sm;
  extern __shared__ float4 wall_vals[];
  walls_chunk<T, SPEC>(a, a.codes, a.e_ref, int(blockIdx.x), sm,
                       a.q <= kStagedMaxQ ? wall_vals : nullptr);
}

// Batched wall pass: block b belongs to instance block_inst[b] (a host-built table: one
// load instead of a search); the instance's wall arguments are copied to shared memory
// once, so the segment lookup and the per-direction staging read no global memory chain.
// Codes and the reference-energy plane of step t come from the instance record.
template <typename T, bool SPEC>
__global__ void __launch_bounds__(32 * kWallWarps) k_walls_batch(const BatchWalls* B,
                                                                  const int* block_inst, int t) {
  __shared__ WallSmem sm;
  __shared__ __align__(16) WallArgs wa;
  const int b = int(blockIdx.x);
  const BatchWalls& I = B[block_inst[b]];
  static_assert(sizeof(WallArgs) % 4 == 0, "copied as 32-bit words");
  const int* src = reinterpret_cast<const int*>(&I.w);
  int* dst = reinterpret_cast<int*>(&wa);
  for (int i = int(threadIdx.x); i < int(sizeof(WallArgs) / 4); i += int(blockDim.x))
    dst[i] = src[i];
  const int cur = (I.phase + t) % I.n_e;
  float* e_ref = I.n_e == 3 ? I.e[(cur + 2) % 3] : nullptr;
  const uint8_t* codes = I.codes + size_t(t) * I.w.q;
  const int chunk = b - I.first_block;
  __syncthreads();
  walls_chunk<T, SPEC>(wa, codes, e_ref, chunk, sm, nullptr);
}

// Internal sources / radiation cells: one warp per cell, lanes over the directions.  With
// bfloat16 storage the cell's reference energy becomes the imposed total, so the stored
// values are the imposed ones relative to it (as for isothermal walls).
template <typename T>
__global__ void __launch_bounds__(256) k_sources(const SourceArgs a) {
  const int s = int(blockIdx.x) * 8 + (int(threadIdx.x) >> 5);
  const int lane = int(threadIdx.x) & 31;
  if (s >= a.n) return;
  const int64_t off = a.off[s];
  const float R = a.esum[s];
  T* planes = static_cast<T*>(a.planes);
  for (int i = lane; i < a.q; i += 32) {
    T* p = planes + int64_t(((a.codes[i] >> 4) & 1) * a.q + i) * a.plane + off;
    wall_store(p, a.val[int64_t(s) * a.q + i], a.w[i], a.e_ref != nullptr, R, a.inv_scale);
  }
  if (lane == 0) {
    a.e_cur[off] = R;
    if (a.e_ref) a.e_ref[off] = R;
  }
}

template <typename T>
__global__ void k_periodic(const PeriodicArgs a) {
  const int ncy = a.yper ? (a.xper ? a.nx : a.nx + 2) : 0;
  const int cy0 = a.xper ? kX0 : kGhostCol;
  const int ncx = a.xper ? 2 * (a.ny + 2) : 0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * ncy + ncx) return;
  const int p = blockIdx.y;
  // Before a step with known codes, a direction plane gets only the ghost cells that step
  // pulls from: the bottom (top) ghost row if its hop has c_y = +1 (-1), the left (right)
  // ghost column if c_x = +1 (-1), nothing if it pauses.  Energy planes, the adjoint's tape
  // and refreshes outside the step loop (a parity mask, no codes) copy everything.
  const bool partial = p < a.q && !a.tape && !a.par && a.codes;
  int hx = 0, hy = 0;
  if (partial) {
    const int code = a.codes[p];
    if (code & 8) return;
    hx = c_hop_x[code & 7];
    hy = c_hop_y[code & 7];
  }
  int rd, cd, rs, cs;
  if (t < 2 * ncy) {
    const int side = t / ncy, k = t - side * ncy;
    if (partial && hy != (side == 0 ? 1 : -1)) return;
    cd = cs = cy0 + k;
    rd = side == 0 ? 1 : a.ny + 2;
    rs = side == 0 ? a.ny + 1 : 2;
  } else {
    const int k = t - 2 * ncy;
    const int side = k / (a.ny + 2);
    if (partial && hx != (side == 0 ? 1 : -1)) return;
    rd = 1 + (k - side * (a.ny + 2));
    rs = rd;
    if (a.yper) {
      if (rd == 1) rs = a.ny + 1;
      else if (rd == a.ny + 2) rs = 2;
    }
    cd = side == 0 ? kGhostCol : kX0 + a.nx;
    cs = side == 0 ? kX0 + a.nx - 1 : kX0;
  }
  const int64_t od = int64_t(rd) * a.pitch + cd, os = int64_t(rs) * a.pitch + cs;
  if (p == a.q) {
    a.e_cur[od] = a.e_cur[os];
  } else if (p == a.q + 1) {
    a.e_ref[od] = a.e_ref[os];
  } else {
    const int par = a.tape ? 0 : a.par ? parity_of(*a.par, p) : (a.codes[p] >> 4) & 1;
    T* base = static_cast<T*>(a.planes) + int64_t(par * a.q + p) * a.plane;
    base[od] = base[os];
  }
}

template <typename T>
__global__ void k_init(const InitArgs a) {
  const int fw = a.nx + 2, fh = a.ny + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= fw * fh) return;
  const int fy = t / fw, fx = t - fy * fw;            // framed coordinates
  const int x = min(max(fx - 1, 0), a.nx - 1), y = min(max(fy - 1, 0), a.ny - 1);
  const double temp = a.t_ref + double(a.dT[int64_t(y) * a.nx + x]);
  const double de = 1.0 / expm1(a.theta / temp) - a.e_ref;
  const int64_t off = int64_t(fy + 1) * a.pitch + (kGhostCol + fx);
  T* planes = static_cast<T*>(a.planes);
  if (a.e_refp) {   // reference energy = the equilibrium energy of this cell
    float e0 = 0.f;
    for (int i = 0; i < a.q; ++i) e0 += float(double(a.w[i]) * de);
    a.e_refp[off] = e0;
  }
  float e = 0.f;
  for (int i = 0; i < a.q; ++i)
    e += dev_store(planes + int64_t(i) * a.plane + off, float(double(a.w[i]) * de), a.w[i],
                   a.e_refp, off, a.scale, a.inv_scale);
  a.e_cur[off] = e;
}

template <typename T>
__global__ void k_moments(const MomentArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nx * a.ny) return;
  const int y = t / a.nx, x = t - y * a.nx;
  const int64_t off = int64_t(y + 2) * a.pitch + (x + kX0);
  if (a.dT) {
    // L = ln(1 + 1/e) = L_ref + log1p(dE/(e_ref+1)) - log1p(dE/e_ref);
    // T - T_ref = theta/L - theta/L_ref = -theta dL / (L_ref (L_ref + dL)).
    const float de = a.e_cur[off];
    const float dl = log1pf(de / a.e_ref1) - log1pf(de / a.e_ref);
    const float v = a.weight * (-a.theta * dl / (a.l_ref * (a.l_ref + dl)));
    a.dT[t] = a.accumulate ? a.dT[t] + v : v;
  }
  if (a.qx || a.qy) {
    const T* planes = static_cast<const T*>(a.planes);
    float qx = 0.f, qy = 0.f;
    for (int i = 0; i < a.q; ++i) {
      const float v = dev_load(planes + int64_t(parity_of(a.par, i) * a.q + i) * a.plane + off,
                               a.w[i], a.e_refp, off, a.scale);
      qx = fmaf(v, a.sx[i], qx);
      qy = fmaf(v, a.sy[i], qy);
    }
    const float wx = a.weight * (qx * a.vg), wy = a.weight * (qy * a.vg);
    if (a.qx) a.qx[t] = a.accumulate ? a.qx[t] + wx : wx;
    if (a.qy) a.qy[t] = a.accumulate ? a.qy[t] + wy : wy;
  }
}

// T - T_ref of a cell's float32 local-energy deviation (Eq. pseudo-T in the same
// cancellation-free float32 form as k_moments; float64 per cell would cost more than the
// rest of the reduction on this GPU's float64 rate).  The reductions over cells that use
// it stay in float64.
__device__ __forceinline__ float temperature_dev32(float de, float e_ref, float e_ref1,
                                                   float l_ref, float theta) {
  const float dl = log1pf(de / e_ref1) - log1pf(de / e_ref);
  return -theta * dl / (l_ref * (l_ref + dl));
}

// max that keeps NaN (a NaN temperature must show in the residual)
__device__ __forceinline__ double fmax_nan(double a, double b) {
  return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000ll) : (a > b ? a : b);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Per-direction data of a reduction block, staged once in shared memory.
struct ReduceSmem {
  float w[kMaxQ], sx[kMaxQ], sy[kMaxQ];
  uint8_t par[kMaxQ];
};

// Per-cell contributions of k_reduce at framed index t: the sums v[] and the residual.
template <typename T>
__device__ __forceinline__ void reduce_cell(const ReduceArgs& a, const ReduceSmem& sm, int t,
                                            double* v, double* res, double* resw) {
  const int fw = a.nx + 2, fh = a.ny + 2;
  const int fy = t / fw, fx = t - fy * fw;
  const bool gx = fx == 0 || fx == fw - 1, gy = fy == 0 || fy == fh - 1;
  const int64_t off = int64_t(fy + 1) * a.pitch + (kGhostCol + fx);
  const T* planes = static_cast<const T*>(a.planes);
  if (!gx && !gy) {
    const double e = double(a.e_cur[off]);
    v[0] += e;
    v[1] += e;
    // a cell's flux over its Q directions in float32 (as in k_moments: the stored values
    // are float32 or coarser), the sums over cells in float64
    float qx = 0.f, qy = 0.f;
#pragma unroll 8
    for (int i = 0; i < a.q; ++i) {
      const float u = dev_load(planes + int64_t(sm.par[i] * a.q + i) * a.plane + off, sm.w[i],
                               a.e_refp, off, float(a.scale));
      qx = fmaf(u, sm.sx[i], qx);
      qy = fmaf(u, sm.sy[i], qy);
    }
    v[2] += qx;
    v[3] += qy;
    const int x = fx - 1;
    if (x >= a.band_x0 && x < a.band_x0 + a.band_w) {
      v[4] += qx;
      v[5] += (double(x) - a.band_xbar) * e;
    }
    const int64_t c = int64_t(fy - 1) * a.nx + x;
    const double tn = double(temperature_dev32(a.e_cur[off], float(a.e_ref), float(a.e_ref1),
                                               float(a.l_ref), float(a.theta)));
    if (a.has_snap) *res = fmax_nan(*res, fabs(tn - a.snap[c]));
    a.snap[c] = tn;
    if (a.win) {
      const double acc = a.win_first ? tn : a.win[c] + tn;
      if (a.win_last) {
        const double mean = acc * a.win_inv;
        if (a.win_has_prev) *resw = fmax_nan(*resw, fabs(mean - a.win_prev[c]));
        a.win_prev[c] = mean;
      } else {
        a.win[c] = acc;
      }
    }
  } else if (wall_energy_cell(fx, fy, fw, fh, a.diff_mask)) {
    double e = 0.0;            // wall cells are few: float64 over the directions
    for (int i = 0; i < a.q; ++i)
      e += dev_load(planes + int64_t(sm.par[i] * a.q + i) * a.plane + off, sm.w[i], a.e_refp,
                    off, float(a.scale));
    v[1] += e;
  }
}

// Stage 1: a grid-stride pass; block b writes its kReduceOut partial results to
// a.part[b] (no atomics: a second kernel combines the blocks in a fixed order).
template <typename T>
__global__ void __launch_bounds__(256) k_reduce(const ReduceArgs a) {
  const int cells = (a.nx + 2) * (a.ny + 2);
  __shared__ ReduceSmem sm;
  for (int i = int(threadIdx.x); i < a.q; i += 256) {
    sm.w[i] = a.w[i];
    sm.sx[i] = a.sx[i];
    sm.sy[i] = a.sy[i];
    sm.par[i] = uint8_t(parity_of(a.par, i));
  }
  __syncthreads();
  double v[kReduceSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double res = 0.0, resw = 0.0;   // largest |T - T_snap| and window change (>= 0 or NaN)
  for (int t = int(blockIdx.x) * 256 + int(threadIdx.x); t < cells; t += int(gridDim.x) * 256)
    reduce_cell<T>(a, sm, t, v, &res, &resw);
  __shared__ double red[kReduceSums][8];
  __shared__ unsigned long long redm[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kReduceSums; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[k][wid] = s;
  }
  // |.| is non-negative, so its bit pattern orders like its value (NaN above all)
  const unsigned long long m0 = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(res)));
  const unsigned long long m1 = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(resw)));
  if (lane == 0) {
    redm[0][wid] = m0;
    redm[1][wid] = m1;
  }
  __syncthreads();
  if (threadIdx.x < kReduceSums) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    a.part[int64_t(blockIdx.x) * kReduceOut + threadIdx.x] = s;
  } else if (threadIdx.x < kReduceOut) {
    unsigned long long m = 0ull;
    for (int w = 0; w < 8; ++w) m = redm[threadIdx.x - kReduceSums][w] > m
                                        ? redm[threadIdx.x - kReduceSums][w] : m;
    a.part[int64_t(blockIdx.x) * kReduceOut + threadIdx.x] = __longlong_as_double(
        static_cast<long long>(m));
  }
}

// Stage 2, one block: the blocks' partials combined in a fixed order into a.out.
__global__ void __launch_bounds__(256) k_reduce_finish(const ReduceArgs a, int nblocks) {
  double v[kReduceSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  unsigned long long m[2] = {0ull, 0ull};
  for (int b = int(threadIdx.x); b < nblocks; b += 256) {
    const double* p = a.part + int64_t(b) * kReduceOut;
#pragma unroll
    for (int k = 0; k < kReduceSums; ++k) v[k] += p[k];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned long long u =
          static_cast<unsigned long long>(__double_as_longlong(p[kReduceSums + k]));
      m[k] = u > m[k] ? u : m[k];
    }
  }
  __shared__ double red[kReduceSums][8];
  __shared__ unsigned long long redm[2][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kReduceSums; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[k][wid] = s;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const unsigned long long u = warp_max_u64(m[k]);
    if (lane == 0) redm[k][wid] = u;
  }
  __syncthreads();
  if (threadIdx.x < kReduceSums) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    a.out[threadIdx.x] = s;
  } else if (threadIdx.x < kReduceOut) {
    unsigned long long u = 0ull;
    for (int w = 0; w < 8; ++w) u = redm[threadIdx.x - kReduceSums][w] > u
                                        ? redm[threadIdx.x - kReduceSums][w] : u;
    a.out[threadIdx.x] = __longlong_as_double(static_cast<long long>(u));
  }
}

template <typename T>
__global__ void k_get_state(const StateArgs a) {
  const int fw = a.nx + 2, fh = a.ny + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (t >= fw * fh) return;
  const int fy = t / fw, fx = t - fy * fw;
  const int64_t off = int64_t(fy + 1) * a.pitch + (kGhostCol + fx);
  const T* p = static_cast<const T*>(a.planes) + int64_t(parity_of(a.par, i) * a.q + i) * a.plane;
  a.framed[int64_t(i) * fw * fh + t] = dev_load(p + off, a.w[i], a.e_refp, off, a.scale);
}

template <typename T>
__global__ void k_set_state(const StateArgs a) {
  const int fw = a.nx + 2, fh = a.ny + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (t >= fw * fh) return;
  const int fy = t / fw, fx = t - fy * fw;
  const int64_t off = int64_t(fy + 1) * a.pitch + (kGhostCol + fx);
  T* p = static_cast<T*>(a.planes) + int64_t(parity_of(a.par, i) * a.q + i) * a.plane;
  dev_store(p + off, a.framed[int64_t(i) * fw * fh + t], a.w[i], a.e_refp, off, a.scale,
            a.inv_scale);
}

template <typename T>
__global__ void k_energy(const StateArgs a) {
  const int fw = a.nx + 2, fh = a.ny + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= fw * fh) return;
  const int fy = t / fw, fx = t - fy * fw;
  const int64_t off = int64_t(fy + 1) * a.pitch + (kGhostCol + fx);
  const T* planes = static_cast<const T*>(a.planes);
  float e = 0.f;
  for (int i = 0; i < a.q; ++i)
    e += dev_load(planes + int64_t(parity_of(a.par, i) * a.q + i) * a.plane + off, a.w[i],
                  a.e_refp, off, a.scale);
  a.e_cur[off] = e;
}

inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

template <typename T>
cudaError_t walls_t(const WallArgs& a, cudaStream_t s) {
  const int chunks = wall_chunk_count(a.nseg, a.seg);
  if (chunks == 0) return cudaSuccess;
  const bool staged = a.q <= kStagedMaxQ;
  const int warps = staged ? staged_warps(a.q) : kWallWarps;
  const size_t bytes = staged ? size_t(a.q) * 32 * sizeof(float4) : 0;
  if (a.any_spec)
    k_walls<T, true><<<chunks, 32 * warps, bytes, s>>>(a);
  else
    k_walls<T, false><<<chunks, 32 * warps, bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t periodic_t(const PeriodicArgs& a, cudaStream_t s) {
  const int ncy = a.yper ? (a.xper ? a.nx : a.nx + 2) : 0;
  const int ncx = a.xper ? 2 * (a.ny + 2) : 0;
  const int total = 2 * ncy + ncx;
  if (total == 0) return cudaSuccess;
  k_periodic<T><<<dim3(blocks_for(total, 256), a.q + (a.e_ref ? 2 : 1)), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walls_batch(int storage, const BatchWalls* b, const int* block_inst,
                               int total_blocks, int t, bool any_spec, cudaStream_t s) {
  if (total_blocks <= 0) return cudaSuccess;
  const dim3 g{unsigned(total_blocks)}, blk{32 * kWallWarps};
  if (storage == WLBM_STORE_BF16_DEV) {
    if (any_spec) k_walls_batch<__nv_bfloat16, true><<<g, blk, 0, s>>>(b, block_inst, t);
    else k_walls_batch<__nv_bfloat16, false><<<g, blk, 0, s>>>(b, block_inst, t);
  } else {
    if (any_spec) k_walls_batch<float, true><<<g, blk, 0, s>>>(b, block_inst, t);
    else k_walls_batch<float, false><<<g, blk, 0, s>>>(b, block_inst, t);
  }
  return cudaGetLastError();
}

int wall_blocks(const WallArgs& a) { return wall_chunk_count(a.nseg, a.seg); }

cudaError_t configure_walls() {
  const int bytes = kStagedMaxQ * 32 * int(sizeof(float4));
  const void* fns[4] = {(const void*)k_walls<float, false>, (const void*)k_walls<float, true>,
                        (const void*)k_walls<__nv_bfloat16, false>,
                        (const void*)k_walls<__nv_bfloat16, true>};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_walls(int storage, const WallArgs& a, cudaStream_t s) {
  return storage == WLBM_STORE_BF16_DEV ? walls_t<__nv_bfloat16>(a, s) : walls_t<float>(a, s);
}

cudaError_t launch_periodic(int storage, const PeriodicArgs& a, cudaStream_t s) {
  return storage == WLBM_STORE_BF16_DEV ? periodic_t<__nv_bfloat16>(a, s)
                                        : periodic_t<float>(a, s);
}

cudaError_t launch_init(int storage, const InitArgs& a, cudaStream_t s) {
  const unsigned g = blocks_for(int64_t(a.nx + 2) * (a.ny + 2), 256);
  if (storage == WLBM_STORE_BF16_DEV)
    k_init<__nv_bfloat16><<<g, 256, 0, s>>>(a);
  else
    k_init<float><<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const MomentArgs& a, cudaStream_t s) {
  const unsigned g = blocks_for(int64_t(a.nx) * a.ny, 256);
  if (storage == WLBM_STORE_BF16_DEV)
    k_moments<__nv_bfloat16><<<g, 256, 0, s>>>(a);
  else
    k_moments<float><<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sources(int storage, const SourceArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const unsigned g = unsigned((a.n + 7) / 8);
  if (storage == WLBM_STORE_BF16_DEV)
    k_sources<__nv_bfloat16><<<g, 256, 0, s>>>(a);
  else
    k_sources<float><<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(int storage, const ReduceArgs& a, cudaStream_t s) {
  const int cells = (a.nx + 2) * (a.ny + 2);
  const int nb = std::max(1, std::min(kReduceBlocks, (cells + 255) / 256));
  if (storage == WLBM_STORE_BF16_DEV)
    k_reduce<__nv_bfloat16><<<nb, 256, 0, s>>>(a);
  else
    k_reduce<float><<<nb, 256, 0, s>>>(a);
  k_reduce_finish<<<1, 256, 0, s>>>(a, nb);
  return cudaGetLastError();
}

cudaError_t launch_get_state(int storage, const StateArgs& a, cudaStream_t s) {
  const dim3 g(blocks_for(int64_t(a.nx + 2) * (a.ny + 2), 256), a.q);
  if (storage == WLBM_STORE_BF16_DEV)
    k_get_state<__nv_bfloat16><<<g, 256, 0, s>>>(a);
  else
    k_get_state<float><<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_set_state(int storage, const StateArgs& a, cudaStream_t s) {
  const dim3 g(blocks_for(int64_t(a.nx + 2) * (a.ny + 2), 256), a.q);
  const unsigned g1 = blocks_for(int64_t(a.nx + 2) * (a.ny + 2), 256);
  if (storage == WLBM_STORE_BF16_DEV) {
    k_set_state<__nv_bfloat16><<<g, 256, 0, s>>>(a);
    k_energy<__nv_bfloat16><<<g1, 256, 0, s>>>(a);
  } else {
    k_set_state<float><<<g, 256, 0, s>>>(a);
    k_energy<float><<<g1, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace wlbm
