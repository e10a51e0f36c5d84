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
#include "walls.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

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

// e_i - e_j of one cell from their stored values: float32 deviations subtract directly;
// bfloat16 ones subtract before the scaling, and the reference parts w R leave only
// (w_i - w_j) R.
template <typename T>
__device__ __forceinline__ float dev_diff(const T* pi, const T* pj, float wi, float wj,
                                          const float* ref, int64_t off, float scale) {
  const float d = Elem<T>::ld(pi) - Elem<T>::ld(pj);
  return ref ? fmaf(d, scale, __fmul_rn(wi - wj, ref[off])) : d;
}

// Heat flux of one cell, q = sum_i e_i s_i (Eq. heat-flux, v = 1 here), taken over the
// pairs of opposite directions i and i + Q/2 (the ring order puts them Q/2 apart, with
// s_{i+Q/2} = -s_i exactly): q = sum_{i < Q/2} (e_i - e_{i+Q/2}) s_i, summed with Kahan's
// compensation (the product's rounding folded into the compensated term by one fma).  So
// the float32 result is within a few roundings of |q| for any Q, where a plain float32 sum
// of Q products errs by about Q roundings of the summands' magnitude (at Q = 1024 more than
// 1e-5 of a direction's amplitude).
template <typename T, typename Par>
__device__ __forceinline__ void cell_flux(const T* planes, int64_t plane, int q, Par par,
                                          const float* w, const float* sx, const float* sy,
                                          const float* ref, int64_t off, float scale,
                                          float& qx, float& qy) {
  const int h = q / 2;
  float cx = 0.f, cy = 0.f;   // compensations: what the running sums lost
  qx = 0.f;
  qy = 0.f;
#pragma unroll 4
  for (int i = 0; i < h; ++i) {
    const int j = i + h;
    const float d = dev_diff(planes + int64_t(par(i) * q + i) * plane + off,
                             planes + int64_t(par(j) * q + j) * plane + off, w[i], w[j], ref,
                             off, scale);
    const float yx = fmaf(d, sx[i], -cx), yy = fmaf(d, sy[i], -cy);
    const float tx = qx + yx, ty = qy + yy;
    cx = (tx - qx) - yx;
    cy = (ty - qy) - yy;
    qx = tx;
    qy = ty;
  }
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
    float qx, qy;
    cell_flux(static_cast<const T*>(a.planes), a.plane, a.q,
              [&](int i) { return parity_of(a.par, i); }, a.w, a.sx, a.sy, a.e_refp, off,
              a.scale, qx, qy);
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
    float qx, qy;
    cell_flux(planes, a.plane, a.q, [&](int i) { return int(sm.par[i]); }, sm.w, sm.sx, sm.sy,
              a.e_refp, off, float(a.scale), qx, qy);
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
