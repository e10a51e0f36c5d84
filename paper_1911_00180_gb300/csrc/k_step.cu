// Fused worm-LBM collide-and-stream kernel (pull form), one launch per time step.
//
// For every frame cell y and direction i with due worm hop c (Eq. worm-paths) the kernel
// computes, with F = W E staged in shared memory and s = y - c:
//    propagating:  d_i'(y) = (1 - W(s)) d_i(s) + w_i F(s)        (Eq. lbm-energy)
//    paused:       d_i'(y) = (1 - W(y)) d_i(y) + w_i F(s)        (Eq. algorithm)
// and accumulates E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density) for the next step, so
// the local energy costs one plane read and one plane write per step instead of a
// separate pass over the Q planes.
//
// Layout: direction-major planes [buffer][i][row][col].  A direction's hop is uniform
// over the grid at a given step, so each source plane is one shifted, coalesced stream.
// A warp owns one row; lane l owns the columns col0 + l + 32 e (e < CPT), so every
// warp-wide access is 32 consecutive elements and the shared-memory tiles are read
// without bank conflicts.  A paused plane is updated in place (its source is its own
// cell), which is why every plane carries its own buffer parity in the step code.
#include "elem.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kTY = 8;   // rows (warps) per block

__device__ __forceinline__ float uniform_w(const StepArgs& a, int r, int c) {
  if (r < 1 || r > a.ny + 2 || c < kGhostCol || c > kX0 + a.nx) return 0.f;  // pads
  const bool gx = (c == kGhostCol) || (c == kX0 + a.nx);
  const bool gy = (r == 1) || (r == a.ny + 2);
  if (gx && !a.xper) return 0.f;   // wall cells do not scatter
  if (gy && !a.yper) return 0.f;
  return a.w0;
}

template <typename T, int CPT, int U, bool FIELD_W, bool REF>
__global__ void __launch_bounds__(32 * kTY) k_step(const StepArgs a) {
  constexpr int TW = 32 * CPT;   // tile width in cells
  constexpr int SW = TW + 2;     // staged width (one halo column each side)
  constexpr int SR = REF ? (kTY + 2) * SW : 1;
  __shared__ float sF[(kTY + 2) * SW];   // W E (scattered energy at each cell)
  __shared__ float sG[(kTY + 2) * SW];   // 1 - W
  __shared__ float sR[SR];               // reference energy of stored values (bf16)
  __shared__ float sw[kMaxQ];
  __shared__ uint8_t scode[kMaxQ];

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  const int col0 = kGhostCol + blockIdx.x * TW;
  const int row0 = 1 + blockIdx.y * kTY;

  // Stage F = W E, G = 1 - W (and R) for the tile plus a one-cell halo.
  for (int idx = tid; idx < (kTY + 2) * SW; idx += 32 * kTY) {
    const int rr = idx / SW, cc = idx - rr * SW;
    const int r = row0 - 1 + rr, c = col0 - 1 + cc;
    float wv = 0.f, ev = 0.f, rv = 0.f;
    if (r < a.rows && c < a.pitch) {
      const int64_t o = int64_t(r) * a.pitch + c;
      ev = a.e_in[o];
      wv = FIELD_W ? a.wfield[o] : uniform_w(a, r, c);
      if (REF) rv = a.e_ref[o];
    }
    sF[idx] = wv * ev;
    sG[idx] = 1.f - wv;
    if (REF) sR[idx] = rv;
  }
  for (int i = tid; i < a.q; i += 32 * kTY) {
    sw[i] = a.w[i];
    scode[i] = a.codes[i];
  }
  __syncthreads();

  const int r = row0 + ty;
  if (r > a.ny + 2) return;          // whole warp: one row per warp
  const int clast = kX0 + a.nx;      // right ghost column
  bool valid[CPT];
#pragma unroll
  for (int e = 0; e < CPT; ++e) valid[e] = col0 + lane + 32 * e <= clast;

  T* planes = static_cast<T*>(a.planes);
  const int64_t rowoff = int64_t(r) * a.pitch + col0 + lane;
  float acc[CPT], ein[CPT];
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    acc[e] = 0.f;
    ein[e] = 0.f;
    if (REF && valid[e]) ein[e] = a.e_in[rowoff + 32 * e];   // write reference
  }

  for (int i0 = 0; i0 < a.q; i0 += U) {
    float v[U][CPT];
    int meta[U];
    // issue the loads of U directions before any store (memory-level parallelism)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u;
      const int code = scode[i];
      const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
      const int dx = paused ? 0 : -c_hop_x[hop];
      const int dy = paused ? 0 : -c_hop_y[hop];
      meta[u] = code;
      const T* src = planes + int64_t(par * a.q + i) * a.plane + rowoff +
                     int64_t(dy) * a.pitch + dx;
#pragma unroll
      for (int e = 0; e < CPT; ++e)
        v[u][e] = valid[e] ? Elem<T>::ld_stream(src + 32 * e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u;
      const int code = meta[u];
      const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
      const int cx = c_hop_x[hop], cy = c_hop_y[hop];
      const int dx = paused ? 0 : -cx, dy = paused ? 0 : -cy;
      T* dst = planes + int64_t((paused ? par : 1 - par) * a.q + i) * a.plane + rowoff;
      const int so = (ty + 1 + dy) * SW + lane + 1 + dx;      // DDED source cell
      const float* gs = sG + so;
      const float* fs = sF + (ty + 1 - cy) * SW + lane + 1 - cx;   // EED source cell
      const float wi = sw[i];
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        if (valid[e]) {
          float d = v[u][e];
          if (REF) d = fmaf(d, a.scale, wi * sR[so + 32 * e]);
          const float out = fmaf(gs[32 * e], d, wi * fs[32 * e]);
          if (REF)
            acc[e] += Elem<T>::st_stream(dst + 32 * e, (out - wi * ein[e]) * a.inv_scale);
          else
            acc[e] += Elem<T>::st_stream(dst + 32 * e, out);
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    if (valid[e])
      a.e_out[rowoff + 32 * e] = REF ? fmaf(acc[e], a.scale, ein[e] * a.wsum) : acc[e];
  }
}

template <typename T, int CPT, int U, bool REF>
cudaError_t launch_t(const StepArgs& a, cudaStream_t s) {
  const dim3 block(32, kTY);
  const dim3 grid((a.nx + 2 + 32 * CPT - 1) / (32 * CPT), (a.ny + 2 + kTY - 1) / kTY);
  if (a.wfield)
    k_step<T, CPT, U, true, REF><<<grid, block, 0, s>>>(a);
  else
    k_step<T, CPT, U, false, REF><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(int storage, const StepArgs& a, cudaStream_t s) {
  if (storage == WLBM_STORE_BF16_DEV) return launch_t<__nv_bfloat16, 8, 2, true>(a, s);
  return launch_t<float, 4, 4, false>(a, s);
}

}  // namespace wlbm
