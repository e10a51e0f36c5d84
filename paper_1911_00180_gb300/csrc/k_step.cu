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
      const T* src = planes + int64_t(a.tape ? i : par * a.q + i) * a.plane + rowoff +
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
      T* dst = a.tape ? static_cast<T*>(a.tape_dst) + int64_t(i) * a.plane + rowoff
                      : planes + int64_t((paused ? par : 1 - par) * a.q + i) * a.plane + rowoff;
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
          if (REF) {   // accumulate the deviation the stored value will decode to
            const float r = wi * ein[e];
            acc[e] += fmaf(Elem<T>::st_stream(dst + 32 * e, (out - r) * a.inv_scale), a.scale, r);
          } else {
            acc[e] += Elem<T>::st_stream(dst + 32 * e, out);
          }
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    if (valid[e])
      a.e_out[rowoff + 32 * e] = acc[e];
  }
}

// ---------------------------------------------------------------------------------
// Variant 1: per-warp bulk-copy ring.  Each warp owns one destination row of the tile
// and a ring of S shared-memory stages.  Lane 0 fetches the (shifted) source row segment
// of direction i + S with one cp.async.bulk copy completing on the stage's mbarrier
// while the warp computes direction i from shared memory, so the bytes in flight do not
// depend on registers.  The segment starts at the 16-byte boundary at or below the
// shifted first column and is V elements longer than the tile, which covers shifts of
// -1, 0, +1.  Every mbarrier wait is bounded in time; on expiry the kernel sets bit 0 of
// the status word, waits (bounded) for its own copies still in flight and returns.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete, at most ~`limit` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

constexpr long long kWaitCycles = 4000000000LL;   // about two seconds at GB300 clocks

// Shared-memory layout of the bulk variant (dynamic shared memory, 128-byte aligned).
template <typename T, int CPT, int S, bool REF>
struct BulkLayout {
  static constexpr int TW = 32 * CPT;              // tile width in cells
  static constexpr int V = 16 / int(sizeof(T));    // elements per 16 bytes
  static constexpr int BW = TW + V;                // elements copied per direction and row
  static constexpr uint32_t kBytes = BW * sizeof(T);
  static constexpr int SW = TW + 2;                // staged width (one halo column each side)
  static constexpr int TILE = (kTY + 2) * SW;      // floats per staged tile
  static constexpr size_t off_f = 0;
  static constexpr size_t off_g = off_f + TILE * 4;
  static constexpr size_t off_r = off_g + TILE * 4;
  static constexpr size_t off_w = off_r + (REF ? TILE * 4 : 0);
  static constexpr size_t off_code = off_w + kMaxQ * 4;
  static constexpr size_t off_bar = (off_code + kMaxQ + 127) / 128 * 128;
  static constexpr size_t off_ring = off_bar + ((kTY * S * 8 + 127) / 128) * 128;
  static constexpr size_t bytes = off_ring + size_t(kTY) * S * kBytes;
  static_assert(kBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};

template <typename T, int CPT, int S, bool FIELD_W, bool REF>
__global__ void __launch_bounds__(32 * kTY) k_step_bulk(const StepArgs a) {
  using LY = BulkLayout<T, CPT, S, REF>;
  constexpr int TW = LY::TW, V = LY::V, BW = LY::BW, SW = LY::SW;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sF = reinterpret_cast<float*>(smem + LY::off_f);
  float* sG = reinterpret_cast<float*>(smem + LY::off_g);
  float* sR = reinterpret_cast<float*>(smem + LY::off_r);
  float* sw = reinterpret_cast<float*>(smem + LY::off_w);
  uint8_t* scode = smem + LY::off_code;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + LY::off_bar);     // [kTY][S]
  T* ring = reinterpret_cast<T*>(smem + LY::off_ring);                 // [kTY][S][BW]

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  const int col0 = kGhostCol + blockIdx.x * TW;
  const int row0 = 1 + blockIdx.y * kTY;

  for (int idx = tid; idx < LY::TILE; idx += 32 * kTY) {
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
  uint64_t* mybar = bar + ty * S;
  T* myring = ring + size_t(ty) * S * BW;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&mybar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int r = row0 + ty;
  if (r > a.ny + 2) return;          // whole warp: one row per warp, nothing issued
  const int clast = kX0 + a.nx;
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
    if (REF && valid[e]) ein[e] = a.e_in[rowoff + 32 * e];
  }

  auto issue = [&](int i, int s) {   // lane 0 only
    const int code = scode[i];
    const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
    const int dx = paused ? 0 : -c_hop_x[hop];
    const int dy = paused ? 0 : -c_hop_y[hop];
    const int start = (col0 + dx) & ~(V - 1);
    const T* src = planes + int64_t(a.tape ? i : par * a.q + i) * a.plane +
                   int64_t(r + dy) * a.pitch + start;
    bulk_load(myring + size_t(s) * BW, src, LY::kBytes, &mybar[s]);
  };
  if (lane == 0)
    for (int s = 0; s < S && s < a.q; ++s) issue(s, s);

  for (int i = 0; i < a.q; ++i) {
    const int s = i % S;
    if (!mbar_wait(&mybar[s], uint32_t(i / S) & 1u, kWaitCycles)) {
      if (lane == 0) {
        atomicOr(a.status, 1);
        // wait (bounded) for this warp's copies still in flight, then leave
        for (int j = i; j < a.q && j < i + S; ++j)
          mbar_wait(&mybar[j % S], uint32_t(j / S) & 1u, kWaitCycles);
      }
      return;
    }
    const int code = scode[i];
    const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
    const int cx = c_hop_x[hop], cy = c_hop_y[hop];
    const int dx = paused ? 0 : -cx, dy = paused ? 0 : -cy;
    const int start = (col0 + dx) & ~(V - 1);
    const T* seg = myring + size_t(s) * BW + (col0 + dx - start + lane);
    float v[CPT];
#pragma unroll
    for (int e = 0; e < CPT; ++e) v[e] = valid[e] ? Elem<T>::ld_shared(seg + 32 * e) : 0.f;
    __syncwarp();
    if (lane == 0 && i + S < a.q) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(i + S, s);
    }
    T* dst = a.tape ? static_cast<T*>(a.tape_dst) + int64_t(i) * a.plane + rowoff
                    : planes + int64_t((paused ? par : 1 - par) * a.q + i) * a.plane + rowoff;
    const int so = (ty + 1 + dy) * SW + lane + 1 + dx;
    const float* gs = sG + so;
    const float* fs = sF + (ty + 1 - cy) * SW + lane + 1 - cx;
    const float wi = sw[i];
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      if (valid[e]) {
        float d = v[e];
        if (REF) d = fmaf(d, a.scale, wi * sR[so + 32 * e]);
        const float out = fmaf(gs[32 * e], d, wi * fs[32 * e]);
        if (REF) {
          const float rr = wi * ein[e];
          acc[e] += fmaf(Elem<T>::st_stream(dst + 32 * e, (out - rr) * a.inv_scale), a.scale, rr);
        } else {
          acc[e] += Elem<T>::st_stream(dst + 32 * e, out);
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < CPT; ++e)
    if (valid[e]) a.e_out[rowoff + 32 * e] = acc[e];
}

template <typename T, int CPT, int S, bool FIELD_W, bool REF>
cudaError_t launch_bulk_one(const StepArgs& a, cudaStream_t s) {
  using LY = BulkLayout<T, CPT, S, REF>;
  static bool configured = false;     // opt in to more than 48 KB of shared memory once
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(k_step_bulk<T, CPT, S, FIELD_W, REF>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               int(LY::bytes));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const dim3 block(32, kTY);
  const dim3 grid((a.nx + 2 + LY::TW - 1) / LY::TW, (a.ny + 2 + kTY - 1) / kTY);
  k_step_bulk<T, CPT, S, FIELD_W, REF><<<grid, block, LY::bytes, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int CPT, int S, bool REF>
cudaError_t launch_bulk(const StepArgs& a, cudaStream_t s) {
  return a.wfield ? launch_bulk_one<T, CPT, S, true, REF>(a, s)
                  : launch_bulk_one<T, CPT, S, false, REF>(a, s);
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
  if (a.variant == 1) {
    if (storage == WLBM_STORE_BF16_DEV) return launch_bulk<__nv_bfloat16, 8, 6, true>(a, s);
    return launch_bulk<float, 4, 6, false>(a, s);
  }
  if (storage == WLBM_STORE_BF16_DEV) return launch_t<__nv_bfloat16, 8, 2, true>(a, s);
  return launch_t<float, 4, 4, false>(a, s);
}

}  // namespace wlbm
