// Device code of the wall pass (Sec. 2.6) shared by the wall kernels (k_aux.cu) and the
// persistent batched kernel (k_batch_persistent.cu): stored-value access with the
// bfloat16 reference energy, and walls_chunk, one block's chunk of ghost cells.
//
// Isotropic blackbody walls overwrite d_i = w_i (e_eq(T_w) - e_ref) (Eq. isotropic);
// adiabatic diffuse walls collect the components that do not point into the domain and
// re-emit them into the inward ones with fractions w_i (s_i.n) / sum (Eq.
// adiabatic-diffuse, normalised so that energy is conserved); specular and
// specular-diffusive walls give a fraction p of each outward component to its mirror
// direction (Eq. adiabatic-specular and the linear combination the paper names).
#pragma once
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

}  // namespace

}  // namespace wlbm
