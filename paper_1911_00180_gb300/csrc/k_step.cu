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
#include "mbar.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kTY = kStepRows;   // rows (warps) per block


// Shared-memory layout of the register-pipelined variant (one static buffer per kernel).
template <int CPT, bool REF>
struct RegLayout {
  static constexpr int SW = 32 * CPT + 2;
  static constexpr int TILE = (kTY + 2) * SW;
  static constexpr size_t bytes = size_t(TILE) * 4 * (REF ? 3 : 2) + kMaxQ * 4 + kMaxQ;
};

template <typename T, int CPT, int U, bool FIELD_W, bool REF, bool WRAP>
__device__ __forceinline__ void step_reg_tile(const StepArgs& a, int bx, int by,
                                              unsigned char* smem) {
  constexpr int TW = 32 * CPT;   // tile width in cells
  constexpr int SW = TW + 2;     // staged width (one halo column each side)
  constexpr int TILE = RegLayout<CPT, REF>::TILE;
  float* sF = reinterpret_cast<float*>(smem);            // W E (scattered energy)
  float* sG = sF + TILE;                                 // 1 - W
  float* sR = sG + TILE;                                 // bf16: reference terms
  float* sw = sR + (REF ? TILE : 0);
  uint8_t* scode = reinterpret_cast<uint8_t*>(sw + kMaxQ);

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  const int col0 = kGhostCol + bx * TW;
  const int row0 = 1 + by * kTY;

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
    const float fv = __fmul_rn(wv, ev), gv = __fsub_rn(1.f, wv);
    sG[idx] = gv;
    if (REF) {   // bfloat16: F/scale and (G R + F)/scale, see the update below
      sF[idx] = __fmul_rn(fv, a.inv_scale);
      sR[idx] = __fmul_rn(fmaf(gv, rv, fv), a.inv_scale);
    } else {
      sF[idx] = fv;
    }
  }
  for (int i = tid; i < a.q; i += 32 * kTY) {
    sw[i] = a.w[i];
    scode[i] = a.codes[i];
  }
  __syncthreads();

  const int r = row0 + ty;
  // whole warp: one row per warp (ghost rows are mirrors when both axes are periodic)
  if (r > a.ny + 2 || (WRAP && (r == 1 || r == a.ny + 2))) return;
  const int clast = kX0 + a.nx;      // right ghost column
  bool valid[CPT];
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    const int c = col0 + lane + 32 * e;
    valid[e] = WRAP ? (c >= kX0 && c < clast) : c <= clast;
  }
  // Both axes periodic (nx, ny >= 2): edge cells also store into the ghost cells that
  // mirror them, at offsets that are the same in every plane.
  const int64_t mrow = !WRAP ? 0 : r == 2 ? int64_t(a.ny) * a.pitch
                                   : r == a.ny + 1 ? -int64_t(a.ny) * a.pitch : 0;
  unsigned mcol_l = 0, mcol_r = 0;   // cells at x = 0 (mirror +nx) / x = nx-1 (mirror -nx)
  if (WRAP) {
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      const int c = col0 + lane + 32 * e;
      if (valid[e] && c == kX0) mcol_l |= 1u << e;
      if (valid[e] && c == kX0 + a.nx - 1) mcol_r |= 1u << e;
    }
  }
  const bool mirrors = mrow != 0 || (mcol_l | mcol_r) != 0;

  T* planes = static_cast<T*>(a.planes);
  const int64_t rowoff = int64_t(r) * a.pitch + col0 + lane;
  float acc[CPT], ein[CPT], eins[CPT], accw = 0.f;
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    acc[e] = 0.f;
    ein[e] = 0.f;
    if (REF && valid[e]) ein[e] = a.e_in[rowoff + 32 * e];   // write reference
    eins[e] = REF ? __fmul_rn(ein[e], a.inv_scale) : 0.f;
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
      const int fo = (ty + 1 - cy) * SW + lane + 1 - cx;   // EED source cell
      const float wi = sw[i];
      if (REF) accw += wi;
      float sv[CPT];
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        if (valid[e]) {
          float out;
          if (REF) {
            // stored v' = (d' - w_i E_in(y)) / scale with d' from Eq. lbm-energy:
            // propagating (so = fo): G(s) v + w_i ((G R + F)(s)/scale - E_in(y)/scale)
            // paused (so = y): G(y) v + w_i (G R(y)/scale + F(s)/scale - E_in(y)/scale)
            const float t = paused ? __fadd_rn(__fsub_rn(sR[so + 32 * e], sF[so + 32 * e]),
                                                      sF[fo + 32 * e])
                                   : sR[so + 32 * e];
            out = fmaf(gs[32 * e], v[u][e], __fmul_rn(wi, __fsub_rn(t, eins[e])));
          } else {
            out = fmaf(gs[32 * e], v[u][e], wi * sF[fo + 32 * e]);
          }
          sv[e] = Elem<T>::st_stream(dst + 32 * e, out);
          acc[e] += sv[e];
        }
      }
      if (mirrors) {   // periodic edge cells: also store the ghost cells mirroring them
#pragma unroll
        for (int e = 0; e < CPT; ++e) {
          if (!valid[e]) continue;
          T* p = dst + 32 * e;
          if (mrow) Elem<T>::st_stream(p + mrow, sv[e]);
          if (((mcol_l | mcol_r) >> e) & 1u) {
            const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
            Elem<T>::st_stream(p + mc, sv[e]);
            if (mrow) Elem<T>::st_stream(p + mc + mrow, sv[e]);
          }
        }
      }
    }
  }
  // E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density); bfloat16: d' = scale v' + w_i E_in(y)
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    if (valid[e]) {
      const float eo = REF ? fmaf(acc[e], a.scale, __fmul_rn(ein[e], accw)) : acc[e];
      a.e_out[rowoff + 32 * e] = eo;
      if (mirrors) {
        float* p = a.e_out + rowoff + 32 * e;
        if (mrow) p[mrow] = eo;
        if (((mcol_l | mcol_r) >> e) & 1u) {
          const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
          p[mc] = eo;
          if (mrow) p[mc + mrow] = eo;
        }
      }
    }
  }
}

template <typename T, int CPT, int U, bool FIELD_W, bool REF, bool WRAP>
__global__ void __launch_bounds__(32 * kTY, 4) k_step(const StepArgs a) {
  __shared__ __align__(16) unsigned char smem[RegLayout<CPT, REF>::bytes];
  step_reg_tile<T, CPT, U, FIELD_W, REF, WRAP>(a, blockIdx.x, blockIdx.y, smem);
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

template <typename T, int CPT, int S, bool FIELD_W, bool REF, bool WRAP>
__device__ __forceinline__ void step_bulk_tile(const StepArgs& a, int bx, int by,
                                               unsigned char* smem) {
  using LY = BulkLayout<T, CPT, S, REF>;
  constexpr int TW = LY::TW, V = LY::V, BW = LY::BW, SW = LY::SW;
  float* sF = reinterpret_cast<float*>(smem + LY::off_f);
  float* sG = reinterpret_cast<float*>(smem + LY::off_g);
  float* sR = reinterpret_cast<float*>(smem + LY::off_r);
  float* sw = reinterpret_cast<float*>(smem + LY::off_w);
  uint8_t* scode = smem + LY::off_code;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + LY::off_bar);     // [kTY][S]
  T* ring = reinterpret_cast<T*>(smem + LY::off_ring);                 // [kTY][S][BW]

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane;
  const int col0 = kGhostCol + bx * TW;
  const int row0 = 1 + by * kTY;

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
    const float fv = __fmul_rn(wv, ev), gv = __fsub_rn(1.f, wv);
    sG[idx] = gv;
    if (REF) {   // bfloat16: F/scale and (G R + F)/scale, see the update below
      sF[idx] = __fmul_rn(fv, a.inv_scale);
      sR[idx] = __fmul_rn(fmaf(gv, rv, fv), a.inv_scale);
    } else {
      sF[idx] = fv;
    }
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
  // whole warp: one row per warp (ghost rows are mirrors when both axes are periodic)
  if (r > a.ny + 2 || (WRAP && (r == 1 || r == a.ny + 2))) return;
  const int clast = kX0 + a.nx;      // right ghost column
  bool valid[CPT];
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    const int c = col0 + lane + 32 * e;
    valid[e] = WRAP ? (c >= kX0 && c < clast) : c <= clast;
  }
  // Both axes periodic (nx, ny >= 2): edge cells also store into the ghost cells that
  // mirror them, at offsets that are the same in every plane.
  const int64_t mrow = !WRAP ? 0 : r == 2 ? int64_t(a.ny) * a.pitch
                                   : r == a.ny + 1 ? -int64_t(a.ny) * a.pitch : 0;
  unsigned mcol_l = 0, mcol_r = 0;   // cells at x = 0 (mirror +nx) / x = nx-1 (mirror -nx)
  if (WRAP) {
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      const int c = col0 + lane + 32 * e;
      if (valid[e] && c == kX0) mcol_l |= 1u << e;
      if (valid[e] && c == kX0 + a.nx - 1) mcol_r |= 1u << e;
    }
  }
  const bool mirrors = mrow != 0 || (mcol_l | mcol_r) != 0;

  T* planes = static_cast<T*>(a.planes);
  const int64_t rowoff = int64_t(r) * a.pitch + col0 + lane;
  float acc[CPT], ein[CPT], eins[CPT], accw = 0.f;
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    acc[e] = 0.f;
    ein[e] = 0.f;
    if (REF && valid[e]) ein[e] = a.e_in[rowoff + 32 * e];
    eins[e] = REF ? __fmul_rn(ein[e], a.inv_scale) : 0.f;
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
      const int fo = (ty + 1 - cy) * SW + lane + 1 - cx;   // EED source cell
    const float wi = sw[i];
    if (REF) accw += wi;
    float sv[CPT];
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      if (valid[e]) {
        float out;
        if (REF) {
          // stored v' = (d' - w_i E_in(y)) / scale with d' from Eq. lbm-energy:
          // propagating (so = fo): G(s) v + w_i ((G R + F)(s)/scale - E_in(y)/scale)
          // paused (so = y): G(y) v + w_i (G R(y)/scale + F(s)/scale - E_in(y)/scale)
          const float t = paused ? __fadd_rn(__fsub_rn(sR[so + 32 * e], sF[so + 32 * e]),
                                                    sF[fo + 32 * e])
                                 : sR[so + 32 * e];
          out = fmaf(gs[32 * e], v[e], __fmul_rn(wi, __fsub_rn(t, eins[e])));
        } else {
          out = fmaf(gs[32 * e], v[e], wi * sF[fo + 32 * e]);
        }
        sv[e] = Elem<T>::st_stream(dst + 32 * e, out);
        acc[e] += sv[e];
      }
    }
    if (mirrors) {   // periodic edge cells: also store the ghost cells mirroring them
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        if (!valid[e]) continue;
        T* p = dst + 32 * e;
        if (mrow) Elem<T>::st_stream(p + mrow, sv[e]);
        if (((mcol_l | mcol_r) >> e) & 1u) {
          const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
          Elem<T>::st_stream(p + mc, sv[e]);
          if (mrow) Elem<T>::st_stream(p + mc + mrow, sv[e]);
        }
      }
    }
  }
  // E'(y) = sum_i d_i'(y) (Eq. lbm-energy-density); bfloat16: d' = scale v' + w_i E_in(y)
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    if (valid[e]) {
      const float eo = REF ? fmaf(acc[e], a.scale, __fmul_rn(ein[e], accw)) : acc[e];
      a.e_out[rowoff + 32 * e] = eo;
      if (mirrors) {
        float* p = a.e_out + rowoff + 32 * e;
        if (mrow) p[mrow] = eo;
        if (((mcol_l | mcol_r) >> e) & 1u) {
          const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
          p[mc] = eo;
          if (mrow) p[mc + mrow] = eo;
        }
      }
    }
  }
}

template <typename T, int CPT, int S, bool FIELD_W, bool REF, bool WRAP>
__global__ void __launch_bounds__(32 * kTY) k_step_bulk(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  step_bulk_tile<T, CPT, S, FIELD_W, REF, WRAP>(a, blockIdx.x, blockIdx.y, smem);
}

// Opt in to more than 48 KB of dynamic shared memory (per device; done by
// prepare_step_kernels() when a handle is created, outside any stream capture).
template <typename T, int CPT, int S, bool FIELD_W, bool REF>
cudaError_t configure_bulk() {
  using LY = BulkLayout<T, CPT, S, REF>;
  cudaError_t e = cudaFuncSetAttribute(k_step_bulk<T, CPT, S, FIELD_W, REF, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(LY::bytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_bulk<T, CPT, S, FIELD_W, REF, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(LY::bytes));
  return e;
}

template <typename T, int CPT, int S, bool FIELD_W, bool REF>
cudaError_t launch_bulk_one(const StepArgs& a, cudaStream_t s) {
  using LY = BulkLayout<T, CPT, S, REF>;
  const dim3 block(32, kTY);
  const dim3 grid((a.nx + 2 + LY::TW - 1) / LY::TW, (a.ny + 2 + kTY - 1) / kTY);
  if (a.wrap)
    k_step_bulk<T, CPT, S, FIELD_W, REF, true><<<grid, block, LY::bytes, s>>>(a);
  else
    k_step_bulk<T, CPT, S, FIELD_W, REF, false><<<grid, block, LY::bytes, s>>>(a);
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
  if (a.wfield) {
    if (a.wrap) k_step<T, CPT, U, true, REF, true><<<grid, block, 0, s>>>(a);
    else k_step<T, CPT, U, true, REF, false><<<grid, block, 0, s>>>(a);
  } else {
    if (a.wrap) k_step<T, CPT, U, false, REF, true><<<grid, block, 0, s>>>(a);
    else k_step<T, CPT, U, false, REF, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Variant 2: warp-specialised.  A block has kTY consumer warps (one destination row each)
// and one producer warp.  The producer's lane r issues the bulk copy of row r's shifted
// source segment for direction i + S while the consumers work on direction i; a stage's
// "full" barrier completes when all its row copies have landed, its "empty" barrier when
// every consumer warp has read its row.  Consumers read the per-direction quantities
// (destination plane, shared-memory source offsets, weight) from a table the block builds
// once, so their loop is loads from shared memory, the update and the stores.
struct DirEntry {
  int64_t dst_off;     // element offset of the destination plane from the output base
  int16_t so, fo;      // staged-tile offsets of the DDED and EED source cells
  int8_t ring_off;     // first element of the lane's cells in the copied row segment
  uint8_t paused;
  float wi;
};

template <typename T, int CPT, int S, bool REF>
struct WsLayout {
  static constexpr int TW = 32 * CPT;
  static constexpr int V = 16 / int(sizeof(T));
  static constexpr int BW = TW + V;
  static constexpr uint32_t kBytes = BW * sizeof(T);
  static constexpr int SW = TW + 2;
  static constexpr int TILE = (kTY + 2) * SW;
  static constexpr size_t off_f = 0;
  static constexpr size_t off_g = off_f + TILE * 4;
  static constexpr size_t off_r = off_g + TILE * 4;
  static constexpr size_t off_bar = (off_r + (REF ? TILE * 4 : 0) + 127) / 128 * 128;
  static constexpr size_t off_ring = off_bar + ((2 * S * 8 + 127) / 128) * 128;
  static constexpr size_t off_table = off_ring + size_t(S) * kTY * kBytes;
  static size_t bytes(int q) { return off_table + size_t(q) * sizeof(DirEntry); }
  static_assert(kBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
};




template <typename T, int CPT, int S, bool FIELD_W, bool REF, bool WRAP>
__device__ __forceinline__ void step_ws_tile(const StepArgs& a, int bx, int by,
                                             unsigned char* smem) {
  using LY = WsLayout<T, CPT, S, REF>;
  constexpr int TW = LY::TW, V = LY::V, BW = LY::BW, SW = LY::SW;
  float* sF = reinterpret_cast<float*>(smem + LY::off_f);
  float* sG = reinterpret_cast<float*>(smem + LY::off_g);
  float* sR = reinterpret_cast<float*>(smem + LY::off_r);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);   // [S]
  uint64_t* empty = full + S;                                          // [S]
  T* ring = reinterpret_cast<T*>(smem + LY::off_ring);                 // [S][kTY][BW]
  DirEntry* table = reinterpret_cast<DirEntry*>(smem + LY::off_table);

  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + lane, nthr = 32 * (kTY + 1);
  const int col0 = kGhostCol + bx * TW;
  const int row0 = 1 + by * kTY;
  T* planes = static_cast<T*>(a.planes);

  // rows of this block that are computed (ghost rows of a fully periodic grid are mirrors)
  int nrows = 0;
#pragma unroll
  for (int t = 0; t < kTY; ++t) {
    const int r = row0 + t;
    nrows += (r <= a.ny + 2 && !(WRAP && (r == 1 || r == a.ny + 2))) ? 1 : 0;
  }
  auto row_ok = [&](int r) { return r <= a.ny + 2 && !(WRAP && (r == 1 || r == a.ny + 2)); };

  for (int idx = tid; idx < LY::TILE; idx += nthr) {
    const int rr = idx / SW, cc = idx - rr * SW;
    const int r = row0 - 1 + rr, c = col0 - 1 + cc;
    float wv = 0.f, ev = 0.f, rv = 0.f;
    if (r < a.rows && c < a.pitch) {
      const int64_t o = int64_t(r) * a.pitch + c;
      ev = a.e_in[o];
      wv = FIELD_W ? a.wfield[o] : uniform_w(a, r, c);
      if (REF) rv = a.e_ref[o];
    }
    const float fv = __fmul_rn(wv, ev), gv = __fsub_rn(1.f, wv);
    sG[idx] = gv;
    if (REF) {
      sF[idx] = __fmul_rn(fv, a.inv_scale);
      sR[idx] = __fmul_rn(fmaf(gv, rv, fv), a.inv_scale);
    } else {
      sF[idx] = fv;
    }
  }
  for (int i = tid; i < a.q; i += nthr) {
    const int code = a.codes[i];
    const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
    const int cx = c_hop_x[hop], cy = c_hop_y[hop];
    const int dx = paused ? 0 : -cx, dy = paused ? 0 : -cy;
    DirEntry d;
    d.dst_off = int64_t(a.tape ? i : (paused ? par : 1 - par) * a.q + i) * a.plane;
    d.so = int16_t((1 + dy) * SW + 1 + dx);
    d.fo = int16_t((1 - cy) * SW + 1 - cx);
    d.ring_off = int8_t((col0 + dx) - ((col0 + dx) & ~(V - 1)));
    d.paused = uint8_t(paused);
    d.wi = a.w[i];
    table[i] = d;
  }
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], nrows > 0 ? nrows : 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (nrows == 0) return;

  if (ty == kTY) {
    // ------------------------------------------------------------- producer warp
    const int r = row0 + lane;
    const bool mine = lane < kTY && row_ok(r);
    const uint32_t stage_bytes = uint32_t(nrows) * LY::kBytes;
    for (int i = 0; i < a.q; ++i) {
      const int st = i % S, k = i / S;
      if (k > 0) {
        bool ok = true;
        if (lane == 0) ok = mbar_wait(&empty[st], uint32_t(k - 1) & 1u, kWaitCycles);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
          if (lane == 0) {
            atomicOr(a.status, 1);
            for (int j = (i > S ? i - S : 0); j < i; ++j)   // copies still in flight
              mbar_wait(&full[j % S], uint32_t(j / S) & 1u, kWaitCycles);
          }
          return;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (lane == 0) mbar_expect(&full[st], stage_bytes);
      __syncwarp();
      if (mine) {
        const int code = a.codes[i];
        const int hop = code & 7, paused = (code >> 3) & 1, par = (code >> 4) & 1;
        const int dx = paused ? 0 : -c_hop_x[hop];
        const int dy = paused ? 0 : -c_hop_y[hop];
        const int start = (col0 + dx) & ~(V - 1);
        const T* src = planes + int64_t(a.tape ? i : par * a.q + i) * a.plane +
                       int64_t(r + dy) * a.pitch + start;
        bulk_copy(ring + (size_t(st) * kTY + lane) * BW, src, LY::kBytes, &full[st]);
      }
    }
    return;
  }

  // ---------------------------------------------------------------- consumer warps
  const int r = row0 + ty;
  if (!row_ok(r)) return;
  const int clast = kX0 + a.nx;
  bool valid[CPT];
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    const int c = col0 + lane + 32 * e;
    valid[e] = WRAP ? (c >= kX0 && c < clast) : c <= clast;
  }
  const int64_t mrow = !WRAP ? 0 : r == 2 ? int64_t(a.ny) * a.pitch
                                 : r == a.ny + 1 ? -int64_t(a.ny) * a.pitch : 0;
  unsigned mcol_l = 0, mcol_r = 0;
  if (WRAP) {
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      const int c = col0 + lane + 32 * e;
      if (valid[e] && c == kX0) mcol_l |= 1u << e;
      if (valid[e] && c == kX0 + a.nx - 1) mcol_r |= 1u << e;
    }
  }
  const bool mirrors = mrow != 0 || (mcol_l | mcol_r) != 0;
  const int64_t rowoff = int64_t(r) * a.pitch + col0 + lane;
  T* obase = (a.tape ? static_cast<T*>(a.tape_dst) : planes) + rowoff;
  const int tb = ty * SW + lane;                 // this lane's origin in the staged tiles
  float acc[CPT], ein[CPT], eins[CPT], accw = 0.f;
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    acc[e] = 0.f;
    ein[e] = 0.f;
    if (REF && valid[e]) ein[e] = a.e_in[rowoff + 32 * e];
    eins[e] = REF ? __fmul_rn(ein[e], a.inv_scale) : 0.f;
  }
  for (int i = 0; i < a.q; ++i) {
    const int st = i % S;
    if (!mbar_wait(&full[st], uint32_t(i / S) & 1u, kWaitCycles)) {
      if (lane == 0) atomicOr(a.status, 1);
      return;
    }
    const DirEntry d = table[i];
    const T* seg = ring + (size_t(st) * kTY + ty) * BW + d.ring_off + lane;
    float v[CPT];
#pragma unroll
    for (int e = 0; e < CPT; ++e) v[e] = valid[e] ? Elem<T>::ld_shared(seg + 32 * e) : 0.f;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    T* dst = obase + d.dst_off;
    const float* gs = sG + tb + d.so;
    const float wi = d.wi;
    if (REF) accw += wi;
    float sv[CPT];
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      if (valid[e]) {
        float out;
        if (REF) {
          const float t = d.paused ? __fadd_rn(__fsub_rn(sR[tb + d.so + 32 * e],
                                                         sF[tb + d.so + 32 * e]),
                                               sF[tb + d.fo + 32 * e])
                                   : sR[tb + d.so + 32 * e];
          out = fmaf(gs[32 * e], v[e], __fmul_rn(wi, __fsub_rn(t, eins[e])));
        } else {
          out = fmaf(gs[32 * e], v[e], wi * sF[tb + d.fo + 32 * e]);
        }
        sv[e] = Elem<T>::st_stream(dst + 32 * e, out);
        acc[e] += sv[e];
      }
    }
    if (WRAP && mirrors) {
#pragma unroll
      for (int e = 0; e < CPT; ++e) {
        if (!valid[e]) continue;
        T* p = dst + 32 * e;
        if (mrow) Elem<T>::st_stream(p + mrow, sv[e]);
        if (((mcol_l | mcol_r) >> e) & 1u) {
          const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
          Elem<T>::st_stream(p + mc, sv[e]);
          if (mrow) Elem<T>::st_stream(p + mc + mrow, sv[e]);
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < CPT; ++e) {
    if (valid[e]) {
      const float eo = REF ? fmaf(acc[e], a.scale, __fmul_rn(ein[e], accw)) : acc[e];
      a.e_out[rowoff + 32 * e] = eo;
      if (WRAP && mirrors) {
        float* p = a.e_out + rowoff + 32 * e;
        if (mrow) p[mrow] = eo;
        if (((mcol_l | mcol_r) >> e) & 1u) {
          const int64_t mc = ((mcol_l >> e) & 1u) ? a.nx : -a.nx;
          p[mc] = eo;
          if (mrow) p[mc + mrow] = eo;
        }
      }
    }
  }
}

template <typename T, int CPT, int S, bool FIELD_W, bool REF, bool WRAP>
__global__ void __launch_bounds__(32 * (kTY + 1)) k_step_ws(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  step_ws_tile<T, CPT, S, FIELD_W, REF, WRAP>(a, blockIdx.x, blockIdx.y, smem);
}

template <typename T, int CPT, int S, bool REF>
cudaError_t configure_ws() {
  const int bytes = int(WsLayout<T, CPT, S, REF>::bytes(kMaxQ));
  cudaError_t e = cudaSuccess;
  const void* fns[4] = {(const void*)k_step_ws<T, CPT, S, false, REF, false>,
                        (const void*)k_step_ws<T, CPT, S, false, REF, true>,
                        (const void*)k_step_ws<T, CPT, S, true, REF, false>,
                        (const void*)k_step_ws<T, CPT, S, true, REF, true>};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

template <typename T, int CPT, int S, bool REF>
cudaError_t launch_ws(const StepArgs& a, cudaStream_t s) {
  using LY = WsLayout<T, CPT, S, REF>;
  const dim3 block(32, kTY + 1);
  const dim3 grid((a.nx + 2 + LY::TW - 1) / LY::TW, (a.ny + 2 + kTY - 1) / kTY);
  const size_t bytes = LY::bytes(a.q);
  if (a.wfield) {
    if (a.wrap) k_step_ws<T, CPT, S, true, REF, true><<<grid, block, bytes, s>>>(a);
    else k_step_ws<T, CPT, S, true, REF, false><<<grid, block, bytes, s>>>(a);
  } else {
    if (a.wrap) k_step_ws<T, CPT, S, false, REF, true><<<grid, block, bytes, s>>>(a);
    else k_step_ws<T, CPT, S, false, REF, false><<<grid, block, bytes, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Batched step: block b of the grid belongs to the instance whose first_tile is the
// largest one <= b.  Thread 0 completes that instance's arguments for step t (codes of
// the step, the roles of the energy planes) in shared memory; the tile body is the same
// code as the single-grid kernels.
__device__ __forceinline__ void batch_setup(const BatchInst* insts, int n, int t, StepArgs* sa,
                                            int* tile) {
  int lo = 0, hi = n - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (insts[mid].first_tile <= b) lo = mid;
    else hi = mid - 1;
  }
  const BatchInst& I = insts[lo];
  *sa = I.a;
  sa->codes = I.codes + size_t(t) * I.a.q;
  const int cur = (I.phase + t) % I.n_e;
  sa->e_in = I.e[cur];
  sa->e_out = I.e[(cur + 1) % I.n_e];
  sa->e_ref = I.n_e == 3 ? I.e[(cur + 2) % 3] : nullptr;
  const int local = b - I.first_tile;
  tile[0] = local % I.tiles_x;
  tile[1] = local / I.tiles_x;
}

template <typename T, int CPT, int S, bool REF>
__global__ void __launch_bounds__(32 * kTY) k_step_bulk_batch(const BatchInst* insts, int n,
                                                               int t) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ int tile[2];
  if (threadIdx.x == 0 && threadIdx.y == 0) batch_setup(insts, n, t, &sa, tile);
  __syncthreads();
  if (sa.wfield) {
    if (sa.wrap) step_bulk_tile<T, CPT, S, true, REF, true>(sa, tile[0], tile[1], smem);
    else step_bulk_tile<T, CPT, S, true, REF, false>(sa, tile[0], tile[1], smem);
  } else {
    if (sa.wrap) step_bulk_tile<T, CPT, S, false, REF, true>(sa, tile[0], tile[1], smem);
    else step_bulk_tile<T, CPT, S, false, REF, false>(sa, tile[0], tile[1], smem);
  }
}

template <typename T, int CPT, int U, bool REF>
__global__ void __launch_bounds__(32 * kTY, 4) k_step_reg_batch(const BatchInst* insts, int n,
                                                                 int t) {
  __shared__ StepArgs sa;
  __shared__ int tile[2];
  __shared__ __align__(16) unsigned char smem[RegLayout<CPT, REF>::bytes];
  if (threadIdx.x == 0 && threadIdx.y == 0) batch_setup(insts, n, t, &sa, tile);
  __syncthreads();
  if (sa.wfield) {
    if (sa.wrap) step_reg_tile<T, CPT, U, true, REF, true>(sa, tile[0], tile[1], smem);
    else step_reg_tile<T, CPT, U, true, REF, false>(sa, tile[0], tile[1], smem);
  } else {
    if (sa.wrap) step_reg_tile<T, CPT, U, false, REF, true>(sa, tile[0], tile[1], smem);
    else step_reg_tile<T, CPT, U, false, REF, false>(sa, tile[0], tile[1], smem);
  }
}

template <typename T, int CPT, int S, bool REF>
cudaError_t configure_bulk_batch() {
  using LY = BulkLayout<T, CPT, S, REF>;
  return cudaFuncSetAttribute(k_step_bulk_batch<T, CPT, S, REF>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, int(LY::bytes));
}

}  // namespace

int step_tile_width(int storage, int variant) {
  if (variant == 1) return storage == WLBM_STORE_BF16_DEV ? 32 * 8 : 32 * 4;
  return storage == WLBM_STORE_BF16_DEV ? 32 * 8 : 32 * 4;
}

cudaError_t launch_step_batch(int storage, int variant, const BatchInst* insts, int n,
                              int total_tiles, int t, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  const dim3 block(32, kTY);
  if (variant == 1) {
    if (storage == WLBM_STORE_BF16_DEV)
      k_step_bulk_batch<__nv_bfloat16, 8, 6, true>
          <<<total_tiles, block, BulkLayout<__nv_bfloat16, 8, 6, true>::bytes, s>>>(insts, n, t);
    else
      k_step_bulk_batch<float, 4, 6, false>
          <<<total_tiles, block, BulkLayout<float, 4, 6, false>::bytes, s>>>(insts, n, t);
  } else {
    if (storage == WLBM_STORE_BF16_DEV)
      k_step_reg_batch<__nv_bfloat16, 8, 2, true><<<total_tiles, block, 0, s>>>(insts, n, t);
    else
      k_step_reg_batch<float, 4, 4, false><<<total_tiles, block, 0, s>>>(insts, n, t);
  }
  return cudaGetLastError();
}

cudaError_t prepare_step_kernels() {
  cudaError_t e = configure_bulk<__nv_bfloat16, 8, 6, false, true>();
  if (e == cudaSuccess) e = configure_bulk<__nv_bfloat16, 8, 6, true, true>();
  if (e == cudaSuccess) e = configure_bulk<float, 4, 6, false, false>();
  if (e == cudaSuccess) e = configure_bulk<float, 4, 6, true, false>();
  if (e == cudaSuccess) e = configure_bulk_batch<__nv_bfloat16, 8, 6, true>();
  if (e == cudaSuccess) e = configure_bulk_batch<float, 4, 6, false>();
  if (e == cudaSuccess) e = configure_ws<__nv_bfloat16, 8, 8, true>();
  if (e == cudaSuccess) e = configure_ws<float, 4, 8, false>();
  if (e == cudaSuccess) e = configure_step_tma();
  if (e == cudaSuccess) e = configure_adj_tma();
  if (e == cudaSuccess) e = configure_batch_persistent();
  return e;
}

cudaError_t launch_step(int storage, const StepArgs& a, cudaStream_t s) {
  // variant 3 covers steps without fused periodic mirrors of grids (or adjoint tapes) that
  // have a tensor map; the others run variant 1
  if (a.variant == 3 && !a.wrap && a.tmap && a.order) return launch_step_tma(storage, a, s);
  if (a.variant == 2) {
    if (storage == WLBM_STORE_BF16_DEV) return launch_ws<__nv_bfloat16, 8, 8, true>(a, s);
    return launch_ws<float, 4, 8, false>(a, s);
  }
  if (a.variant == 1 || a.variant == 3) {
    if (storage == WLBM_STORE_BF16_DEV) return launch_bulk<__nv_bfloat16, 8, 6, true>(a, s);
    return launch_bulk<float, 4, 6, false>(a, s);
  }
  if (storage == WLBM_STORE_BF16_DEV) return launch_t<__nv_bfloat16, 8, 2, true>(a, s);
  return launch_t<float, 4, 4, false>(a, s);
}

}  // namespace wlbm
