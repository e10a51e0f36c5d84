// Reverse-mode (adjoint) kernels of the worm-LBM run.  The paper has no adjoint; these
// are the exact transposes of the forward kernels (k_step.cu, k_aux.cu) for float32
// storage.  For step n with recorded input d~ (state after the boundary pass), due hops
// c_k, pause flags and weight W, the forward update is
//    propagating:  d_k'(y) = (1 - W(s)) d~_k(s) + w_k W(s) E~(s),   s = y - c_k
//    paused:       d_k'(y) = (1 - W(y)) d~_k(y) + w_k W(s) E~(s),   E~ = sum_k d~_k,
// so with l' the adjoint of d', a_k(x) = l'_k(x + c_k) (propagating) or l'_k(x)
// (paused) and sigma(x) = sum_k w_k l'_k(x + c_k):
//    l~_k(x)   = (1 - W(x)) a_k(x) + W(x) sigma(x)
//    dJ/dW(x) += sum_k d~_k(x) (sigma(x) - a_k(x)).
// The boundary passes are transposed afterwards in reverse order: periodic links add the
// ghost adjoint to the cell they copy, isothermal overwrites zero it and harvest
// sum_i w_i l~_i (times de_eq/dT_w) for the wall temperature, diffuse collections send
// sum_k rho_k l~_k (inward k) to every collected direction.
#include "elem.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kAdjTY = 8;   // rows (warps) per block, one cell per lane

__device__ __forceinline__ float w_at(const AdjArgs& a, int r, int c) {
  if (a.wfield) return a.wfield[int64_t(r) * a.pitch + c];
  if (r < 1 || r > a.ny + 2 || c < kGhostCol || c > kX0 + a.nx) return 0.f;
  const bool gx = (c == kGhostCol) || (c == kX0 + a.nx);
  const bool gy = (r == 1) || (r == a.ny + 2);
  if ((gx && !a.xper) || (gy && !a.yper)) return 0.f;
  return a.w0;
}

// Two passes over the Q adjoint planes per cell: sigma first, then l~ and dJ/dW.  The
// second pass re-reads what the first one read moments earlier (an L2 hit for a tile of
// 32 x 8 cells).
__global__ void __launch_bounds__(32 * kAdjTY) k_adj_step(const AdjArgs a) {
  __shared__ float sw[kMaxQ];
  __shared__ uint8_t scode[kMaxQ];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int i = tid; i < a.q; i += 32 * kAdjTY) {
    sw[i] = a.w[i];
    scode[i] = a.codes[i];
  }
  __syncthreads();
  const int c = kGhostCol + blockIdx.x * 32 + threadIdx.x;
  const int r = 1 + blockIdx.y * kAdjTY + threadIdx.y;
  if (r > a.ny + 2 || c > kX0 + a.nx) return;
  const int64_t off = int64_t(r) * a.pitch + c;
  const float W = w_at(a, r, c);
  constexpr int U = 8;
  float sigma = 0.f;
  for (int k0 = 0; k0 < a.q; k0 += U) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u, hop = scode[k] & 7;
      v[u] = a.lam_in[int64_t(k) * a.plane + off + int64_t(c_hop_y[hop]) * a.pitch + c_hop_x[hop]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) sigma = fmaf(sw[k0 + u], v[u], sigma);
  }
  float g = 0.f;
  const float keep = 1.f - W, ws = W * sigma;
  for (int k0 = 0; k0 < a.q; k0 += U) {
    float av[U], dv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u, code = scode[k], hop = code & 7;
      const int64_t sh = (code & 8) ? 0 : int64_t(c_hop_y[hop]) * a.pitch + c_hop_x[hop];
      av[u] = a.lam_in[int64_t(k) * a.plane + off + sh];
      dv[u] = a.dtil[int64_t(k) * a.plane + off];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a.lam_out[int64_t(k0 + u) * a.plane + off] = fmaf(keep, av[u], ws);
      g = fmaf(dv[u], sigma - av[u], g);
    }
  }
  a.gw[off] += g;
}

// Transpose of the periodic x link (all frame rows), then of the y link.
__global__ void k_periodic_T_x(float* planes, int64_t plane, int pitch, int nx, int ny,
                               int nplanes) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (ny + 2) * nplanes) return;
  const int p = t / (ny + 2), r = 1 + (t - p * (ny + 2));
  float* row = planes + int64_t(p) * plane + int64_t(r) * pitch;
  const float gl = row[kGhostCol], gr = row[kX0 + nx];
  row[kX0 + nx - 1] += gl;
  row[kX0] += gr;
  row[kGhostCol] = 0.f;
  row[kX0 + nx] = 0.f;
}

__global__ void k_periodic_T_y(float* planes, int64_t plane, int pitch, int nx, int ny,
                               int nplanes, int xper) {
  const int ncol = xper ? nx : nx + 2, c0 = xper ? kX0 : kGhostCol;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncol * nplanes) return;
  const int p = t / ncol, c = c0 + (t - p * ncol);
  float* base = planes + int64_t(p) * plane + c;
  const float gb = base[int64_t(1) * pitch], gt = base[int64_t(ny + 2) * pitch];
  base[int64_t(ny + 1) * pitch] += gb;
  base[int64_t(2) * pitch] += gt;
  base[int64_t(1) * pitch] = 0.f;
  base[int64_t(ny + 2) * pitch] = 0.f;
}

// Transpose of the wall pass: one warp per ghost cell, same segments as k_walls.
__global__ void k_walls_T(const WallArgs wa, float* lam, double* gtw) {
  const int warp = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  int s = 0, idx = warp;
  while (s < wa.nseg && idx >= wa.seg[s].count) {
    idx -= wa.seg[s].count;
    ++s;
  }
  if (s >= wa.nseg) return;
  const WallSeg g = wa.seg[s];
  const int64_t off = int64_t(g.r0 + idx * g.dr) * wa.pitch + (g.c0 + idx * g.dc);
  if (g.action == WLBM_BC_ISOTHERMAL) {
    float part = 0.f;
    for (int i = lane; i < wa.q; i += 32) {
      float* p = lam + int64_t(i) * wa.plane + off;
      part = fmaf(wa.w[i], *p, part);
      *p = 0.f;
    }
    const float S = warp_sum(part);
    if (lane == 0) atomicAdd(gtw + g.wall, double(S));
    return;
  }
  const float* rho = wa.rho + int64_t(g.table) * wa.q;
  float part = 0.f;
  for (int i = lane; i < wa.q; i += 32)
    if (rho[i] != 0.f) part = fmaf(rho[i], lam[int64_t(i) * wa.plane + off], part);
  const float S = warp_sum(part);
  for (int i = lane; i < wa.q; i += 32)
    if (rho[i] == 0.f) lam[int64_t(i) * wa.plane + off] = S;
}

// l^N: dJ/dT(x) * dT/dE at the final local energy, for every direction (E = sum_i d_i).
__global__ void k_adj_seed(const AdjArgs a, const float* dJ_dT, const float* e_final,
                           double e_ref, double theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nx * a.ny) return;
  const int y = t / a.nx, x = t - y * a.nx;
  const int64_t off = int64_t(y + 2) * a.pitch + (x + kX0);
  const double e = e_ref + double(e_final[off]);
  const double lg = log1p(1.0 / e);
  const float g = float(double(dJ_dT[t]) * theta / (lg * lg * e * (1.0 + e)));
  for (int i = 0; i < a.q; ++i) a.lam_out[int64_t(i) * a.plane + off] = g;
}

// dJ/dMFP = dJ/dW_corr * dW_corr/dMFP on interior cells; dJ/d(dT0) from l^0 through the
// initial condition e_i = w_i e_eq(T_ref + dT0) (ghost cells copy the nearest cell).
__global__ void k_adj_final(const AdjArgs a, const float* dwc, float* dJ_dmfp,
                            const float* lam0, const float* dT0, float* dJ_ddT0,
                            double t_ref, double theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nx * a.ny) return;
  const int y = t / a.nx, x = t - y * a.nx;
  if (dJ_dmfp) dJ_dmfp[t] = a.gw[int64_t(y + 2) * a.pitch + (x + kX0)] * dwc[t];
  if (dJ_ddT0) {
    const int fx[3] = {x, x == 0 ? -1 : x, x == a.nx - 1 ? a.nx : x};
    const int fy[3] = {y, y == 0 ? -1 : y, y == a.ny - 1 ? a.ny : y};
    double acc = 0.0;
    for (int jy = 0; jy < 3; ++jy) {
      if (jy > 0 && fy[jy] == y) continue;
      for (int jx = 0; jx < 3; ++jx) {
        if (jx > 0 && fx[jx] == x) continue;
        const int64_t off = int64_t(fy[jy] + 2) * a.pitch + (fx[jx] + kX0);
        double s = 0.0;
        for (int i = 0; i < a.q; ++i) s += double(a.w[i]) * lam0[int64_t(i) * a.plane + off];
        acc += s;
      }
    }
    const double T = t_ref + double(dT0[t]);
    const double xx = theta / T, e = 1.0 / expm1(xx);
    dJ_ddT0[t] = float(acc * e * (1.0 + e) * xx / T);
  }
}

inline unsigned nblk(int64_t n, int per) { return unsigned((n + per - 1) / per); }

}  // namespace

cudaError_t launch_adj_step(const AdjArgs& a, cudaStream_t s) {
  const dim3 block(32, kAdjTY);
  const dim3 grid((a.nx + 2 + 31) / 32, (a.ny + 2 + kAdjTY - 1) / kAdjTY);
  k_adj_step<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_periodic_T(float* planes, int64_t plane, int pitch, int nx, int ny,
                              int nplanes, int xper, int yper, cudaStream_t s) {
  if (xper)
    k_periodic_T_x<<<nblk(int64_t(ny + 2) * nplanes, 256), 256, 0, s>>>(planes, plane, pitch,
                                                                         nx, ny, nplanes);
  if (yper)
    k_periodic_T_y<<<nblk(int64_t(xper ? nx : nx + 2) * nplanes, 256), 256, 0, s>>>(
        planes, plane, pitch, nx, ny, nplanes, xper);
  return cudaGetLastError();
}

cudaError_t launch_walls_T(const WallArgs& wa, float* lam, double* gtw, cudaStream_t s) {
  int cells = 0;
  for (int k = 0; k < wa.nseg; ++k) cells += wa.seg[k].count;
  if (cells == 0) return cudaSuccess;
  k_walls_T<<<nblk(int64_t(cells) * 32, 256), 256, 0, s>>>(wa, lam, gtw);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(const AdjArgs& a, const float* dJ_dT, const float* e_final,
                            double e_ref, double theta, cudaStream_t s) {
  k_adj_seed<<<nblk(int64_t(a.nx) * a.ny, 256), 256, 0, s>>>(a, dJ_dT, e_final, e_ref, theta);
  return cudaGetLastError();
}

cudaError_t launch_adj_final(const AdjArgs& a, const float* dwc, float* dJ_dmfp,
                             const float* lam0, const float* dT0, float* dJ_ddT0,
                             double t_ref, double theta, cudaStream_t s) {
  k_adj_final<<<nblk(int64_t(a.nx) * a.ny, 256), 256, 0, s>>>(a, dwc, dJ_dmfp, lam0, dT0,
                                                               dJ_ddT0, t_ref, theta);
  return cudaGetLastError();
}

}  // namespace wlbm
