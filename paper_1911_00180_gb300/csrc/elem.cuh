// Storage element access for the direction planes: float32 deviations, or bfloat16
// deviations (round-to-nearest-even on store).  All arithmetic is float32.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace wlbm {

// Basic D2Q8 hops on the device (same numbering as the host lattice).
static __constant__ int c_hop_x[8] = {1, 0, -1, 0, 1, -1, -1, 1};
static __constant__ int c_hop_y[8] = {0, 1, 0, -1, 1, 1, -1, -1};

template <typename T>
struct Elem;

template <>
struct Elem<float> {
  // streaming (evict-first) forms for the once-per-step plane traffic
  static __device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
  static __device__ __forceinline__ float st_stream(float* p, float v) {
    __stcs(p, v);
    return v;
  }
  static __device__ __forceinline__ float ld(const float* p) { return *p; }
  static __device__ __forceinline__ float st(float* p, float v) {
    *p = v;
    return v;
  }
  static __device__ __forceinline__ float round(float v) { return v; }
  static __device__ __forceinline__ float ld_shared(const float* p) { return *p; }
};

template <>
struct Elem<__nv_bfloat16> {
  static __device__ __forceinline__ float widen(unsigned short b) {
    return __uint_as_float(uint32_t(b) << 16);
  }
  static __device__ __forceinline__ unsigned short narrow(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
  static __device__ __forceinline__ float ld_stream(const __nv_bfloat16* p) {
    return widen(__ldcs(reinterpret_cast<const unsigned short*>(p)));
  }
  static __device__ __forceinline__ float st_stream(__nv_bfloat16* p, float v) {
    const unsigned short b = narrow(v);
    __stcs(reinterpret_cast<unsigned short*>(p), b);
    return widen(b);
  }
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
    return widen(*reinterpret_cast<const unsigned short*>(p));
  }
  static __device__ __forceinline__ float st(__nv_bfloat16* p, float v) {
    const unsigned short b = narrow(v);
    *reinterpret_cast<unsigned short*>(p) = b;
    return widen(b);
  }
  static __device__ __forceinline__ float round(float v) { return widen(narrow(v)); }
  static __device__ __forceinline__ float ld_shared(const __nv_bfloat16* p) {
    return widen(*reinterpret_cast<const unsigned short*>(p));
  }
};

// Whether framed cell (fx, fy) of an fw x fh frame counts towards the energy held by the
// walls: interior cells do not; a ghost cell does when every side it lies on is an
// adiabatic wall (bit k of diff_mask for side k = x-, x+, y-, y+).  Periodic
// ghosts are copies and isothermal ghosts a reservoir reset by every wall pass.
__device__ __forceinline__ bool wall_energy_cell(int fx, int fy, int fw, int fh, int diff_mask) {
  const int sx = fx == 0 ? 0 : (fx == fw - 1 ? 1 : -1);
  const int sy = fy == 0 ? 2 : (fy == fh - 1 ? 3 : -1);
  if (sx < 0 && sy < 0) return false;
  return (sx < 0 || ((diff_mask >> sx) & 1)) && (sy < 0 || ((diff_mask >> sy) & 1));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace wlbm
