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



// One pass over the Q adjoint planes.  A thread owns 4 consecutive cells of a row (a warp
// 128 cells, a block 8 rows).  With the output adjoint l' = lh' + s' (s' of the 3 x 6 cells
// around the thread's cells in registers) it reads b_k = l'_k(x + c_k), u_k = l'_k(x) for
// paused k and d~_k(x) with 16-byte loads (a shifted row piece from two aligned ones), writes
// lh_k = (1 - W) a_k at once and, after the directions, s = W sigma: no plane is read
// twice and nothing waits for sigma.  dJ/dW = sum_k d~_k (sigma - a_k) is accumulated
// shifted by a_0 (the first direction's a), as (sigma - a_0) sum_k d~_k -
// sum_k d~_k (a_k - a_0): near an isotropic adjoint every a_k is close to sigma and to a_0,
// so neither term is much larger than the result.  Cells past the right ghost column are
// neither read for output nor written (their pads stay zero).
constexpr int kAdjRows = 8;
constexpr int kAdjTW = 128;                 // cells of a row per warp
constexpr int kAdjC0 = kGhostCol & ~3;      // first column of the first group

__device__ __forceinline__ float4 ld4(const float* p) {
  return __ldcs(reinterpret_cast<const float4*>(p));
}

// l'_k at the 4 cells shifted by DX (-1, 0, +1) from a 16-byte aligned row position p.
template <int DX>
__device__ __forceinline__ void row4(const float* p, float (&v)[4]) {
  if constexpr (DX == 0) {
    const float4 m = ld4(p);
    v[0] = m.x; v[1] = m.y; v[2] = m.z; v[3] = m.w;
  } else if constexpr (DX < 0) {
    const float4 l = ld4(p - 4), m = ld4(p);
    v[0] = l.w; v[1] = m.x; v[2] = m.y; v[3] = m.z;
  } else {
    const float4 m = ld4(p), r = ld4(p + 4);
    v[0] = m.y; v[1] = m.z; v[2] = m.w; v[3] = r.x;
  }
}

struct AdjAcc {
  float sigma[4], a0[4], ed[4], pd[4], h[4];
};


// One direction with hop (CX, CY) for the thread's 4 cells.
template <int CX, int CY>
__device__ __forceinline__ void adj_dir(AdjAcc& t, const float (&sr)[3][6], const float (&keep)[4],
                                        const float* pl, const float* pdt, float* po,
                                        int pitch, float wk, bool paused, bool first,
                                        unsigned vm, bool harvest) {
  float b[4], av[4];
  row4<CX>(pl + int64_t(CY) * pitch, b);
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] += sr[1 + CY][1 + CX + j];
  if (paused) {
    row4<0>(pl, av);
#pragma unroll
    for (int j = 0; j < 4; ++j) av[j] += sr[1][1 + j];
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) av[j] = b[j];
  }
  const float4 d = ld4(pdt);
  const float dv[4] = {d.x, d.y, d.z, d.w};
  float o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    t.sigma[j] = fmaf(wk, b[j], t.sigma[j]);
    if (first) t.a0[j] = av[j];
    t.ed[j] += dv[j];
    t.pd[j] = fmaf(dv[j], av[j] - t.a0[j], t.pd[j]);
    o[j] = keep[j] * av[j];
    if (harvest) t.h[j] = fmaf(wk, av[j], t.h[j]);   // isothermal wall cells: W = 0, l = a
  }
  if (vm == 0xFu) {
    __stcs(reinterpret_cast<float4*>(po), make_float4(o[0], o[1], o[2], o[3]));
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((vm >> j) & 1u) po[j] = o[j];
  }
}

__global__ void __launch_bounds__(32 * kAdjRows) k_adj_step(const AdjArgs a) {
  __shared__ float sw[kMaxQ];
  __shared__ uint8_t scode[kMaxQ];
  __shared__ float hwall[4];   // isothermal harvest of this block per wall
  const int tid = threadIdx.y * 32 + threadIdx.x, nthr = 32 * kAdjRows;
  for (int i = tid; i < a.q; i += nthr) {
    sw[i] = a.w[i];
    scode[i] = a.codes[i];
  }
  if (tid < 4) hwall[tid] = 0.f;
  __syncthreads();
  // 16-byte aligned groups of 4 from the aligned column at or below the left ghost
  const int c0 = kAdjC0 + blockIdx.x * kAdjTW + 4 * threadIdx.x;
  const int r = 1 + blockIdx.y * kAdjRows + threadIdx.y;
  const int clast = kX0 + a.nx;
  bool any_iso = false;
  if (r <= a.ny + 2 && c0 <= clast) {
    unsigned vm = 0;   // frame cells of the group
#pragma unroll
    for (int j = 0; j < 4; ++j) vm |= (c0 + j >= kGhostCol && c0 + j <= clast) ? 1u << j : 0u;
    const int rows = a.ny + 4;
    // s' around the cells (pads and past-the-frame cells read 0)
    float sr[3][6];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        const int rw = r - 1 + rr, c = c0 - 1 + cc;
        sr[rr][cc] = (rw < rows && c < a.pitch) ? a.s_in[int64_t(rw) * a.pitch + c] : 0.f;
      }
    // isothermal wall cells are transposed here: their new adjoint is 0 (keep = 0) and
    // sum_k w_k a_k is harvested for the wall temperature
    float W[4], keep[4];
    int iso[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      W[j] = ((vm >> j) & 1u) ? w_at(a, r, c0 + j) : 0.f;
      iso[j] = ((vm >> j) & 1u) ? iso_wall_of(a, r, c0 + j) : -1;
      any_iso = any_iso || iso[j] >= 0;
      keep[j] = iso[j] >= 0 ? 0.f : 1.f - W[j];
    }
    const int64_t off = int64_t(r) * a.pitch + c0;
    AdjAcc t;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t.sigma[j] = 0.f; t.a0[j] = 0.f; t.ed[j] = 0.f; t.pd[j] = 0.f; t.h[j] = 0.f;
    }
    for (int k = 0; k < a.q; ++k) {
      const int code = scode[k];
      const bool paused = code & 8;
      const float* pl = a.lam_in + int64_t(k) * a.plane + off;
      const float* pdt = a.dtil + int64_t(k) * a.plane + off;
      float* po = a.lam_out + int64_t(k) * a.plane + off;
      const float wk = sw[k];
      const bool f = k == 0;
      switch (code & 7) {   // hop numbering of the host lattice
        case 0: adj_dir<1, 0>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 1: adj_dir<0, 1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 2: adj_dir<-1, 0>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 3: adj_dir<0, -1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 4: adj_dir<1, 1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 5: adj_dir<-1, 1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        case 6: adj_dir<-1, -1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
        default: adj_dir<1, -1>(t, sr, keep, pl, pdt, po, a.pitch, wk, paused, f, vm, any_iso); break;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((vm >> j) & 1u)) continue;
      a.s_out[off + j] = W[j] * t.sigma[j];
      a.gw[off + j] += fmaf(t.sigma[j] - t.a0[j], t.ed[j], -t.pd[j]);
      if (iso[j] >= 0) atomicAdd(&hwall[iso[j]], t.h[j]);
    }
  }
  // one global atomic per wall and block
  if (__syncthreads_or(any_iso) && tid < 4 && hwall[tid] != 0.f)
    atomicAdd(a.gtw + tid, double(hwall[tid]));
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

// Transpose of the wall pass, on the same blocks as k_walls: along horizontal walls lane l =
// ghost cells 4l .. 4l+3 of a 128-cell chunk and warp w = directions w, w + kWallWarpsT,
// ..., per-cell sums combining over the warps in a fixed order; vertical walls and corners one warp per cell.  Isothermal
// cells send sum_i w_i l_i to the wall temperature and zero l; diffuse cells give every
// collected direction sum_k rho_k l_k.
constexpr int kWallWarpsT = 8;
static_assert(kWallCellsPerBlock == kWallWarpsT, "one warp per cell of a block");

// New adjoint of a collected (outward or parallel) direction i of an adiabatic ghost cell
// with specularity p: p l_mirror(i) + (1 - p) S (a parallel direction is its own mirror);
// S = sum_k rho_k l_k over the inward directions.  Mirrors of collected directions are
// inward, so no value read here is written by the same pass.
__device__ __forceinline__ float collected_T(const WallArgs& wa, const WallSeg& g,
                                             const int16_t* mir, const float* lam, int64_t off,
                                             int i, float S) {
  if (g.spec == 0.f) return S;
  const float own = lam[int64_t(mir[i]) * wa.plane + off];
  return fmaf(g.spec, own, (1.f - g.spec) * S);
}

// One ghost cell by one warp, lanes over the directions; returns sum_i w_i l_i of an
// isothermal cell (0 for diffuse cells) for the wall-temperature gradient.
__device__ __forceinline__ float walls_T_cell(const WallArgs& wa, const WallSeg& g, int idx,
                                              int lane, float* lam) {
  const int64_t off = int64_t(g.r0 + idx * g.dr) * wa.pitch + (g.c0 + idx * g.dc);
  if (g.action == WLBM_BC_ISOTHERMAL) {
    float part = 0.f;
    for (int i = lane; i < wa.q; i += 32) {
      float* p = lam + int64_t(i) * wa.plane + off;
      part = fmaf(wa.w[i], *p, part);
      *p = 0.f;
    }
    return warp_sum(part);
  }
  const float* rho = wa.rho + int64_t(g.table) * wa.q;
  float part = 0.f;
  for (int i = lane; i < wa.q; i += 32)
    if (rho[i] != 0.f) part = fmaf(rho[i], lam[int64_t(i) * wa.plane + off], part);
  const float S = warp_sum(part);
  const int16_t* mir = wa.mirror + int64_t(g.mirror) * wa.q;
  for (int i = lane; i < wa.q; i += 32)
    if (rho[i] == 0.f) lam[int64_t(i) * wa.plane + off] = collected_T(wa, g, mir, lam, off, i, S);
  return 0.f;
}

__global__ void __launch_bounds__(32 * kWallWarpsT) k_walls_T(const WallArgs wa, float* lam,
                                                               double* gtw) {
  __shared__ float part_s[kWallWarpsT * 32 * 4];
  int c = 0;
  const int s = wall_chunk_segment(wa.nseg, wa.seg, int(blockIdx.x), &c);
  if (s >= wa.nseg) return;
  const WallSeg g = wa.seg[s];
  const int lane = int(threadIdx.x) & 31, warp = int(threadIdx.x) >> 5;
  const bool iso = g.action == WLBM_BC_ISOTHERMAL;
  // isothermal cells were transposed by the reverse step; only the segment's end cells
  // may have received corner images from the periodic transpose since
  auto wanted = [&](int cell) {
    return cell < g.count && (!iso || cell == 0 || cell == g.count - 1);
  };
  if (!wall_seg_rowwise(g)) {   // vertical walls and corners: one warp per cell
    const int cell = c * kWallCellsPerBlock + warp;
    const float S = wanted(cell) ? walls_T_cell(wa, g, cell, lane, lam) : 0.f;
    if (g.action != WLBM_BC_ISOTHERMAL) return;
    // one atomic per block: the wall temperature's accumulator is a single address
    if (lane == 0) part_s[warp] = S;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.f;
      for (int k = 0; k < kWallWarpsT; ++k) tot += part_s[k];
      atomicAdd(gtw + g.wall, double(tot));
    }
    return;
  }
  // horizontal walls: four consecutive cells per lane (the blocks of k_walls)
  const int idx0 = c * kWallChunk + 4 * lane;
  bool on[4];
  int64_t off[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int idx = idx0 + j;
    on[j] = wanted(idx);
    off[j] = on[j] ? int64_t(g.r0 + idx * g.dr) * wa.pitch + (g.c0 + idx * g.dc) : 0;
  }
  const float* rho = wa.rho + int64_t(g.table) * wa.q;
  float part[4] = {0.f, 0.f, 0.f, 0.f};
  if (on[0] || on[1] || on[2] || on[3]) {
    for (int i = warp; i < wa.q; i += kWallWarpsT) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!on[j]) continue;
        float* p = lam + int64_t(i) * wa.plane + off[j];
        if (iso) {
          part[j] = fmaf(wa.w[i], *p, part[j]);
          *p = 0.f;
        } else if (rho[i] != 0.f) {
          part[j] = fmaf(rho[i], *p, part[j]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) part_s[(warp * 32 + lane) * 4 + j] = part[j];
  __syncthreads();
  float S[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWallWarpsT; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) S[j] += part_s[(k * 32 + lane) * 4 + j];
  if (iso) {
    if (warp == 0) {
      float mine = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) mine += on[j] ? S[j] : 0.f;
      const float tot = warp_sum(mine);
      if (lane == 0) atomicAdd(gtw + g.wall, double(tot));
    }
    return;
  }
  const int16_t* mir = wa.mirror + int64_t(g.mirror) * wa.q;
  for (int i = warp; i < wa.q; i += kWallWarpsT) {
    if (rho[i] != 0.f) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (on[j]) lam[int64_t(i) * wa.plane + off[j]] = collected_T(wa, g, mir, lam, off[j], i, S[j]);
  }
}

// l^N_i(x) = dJ/dT(x) * dT/dE at the final local energy (E = sum_i d_i, Eq. pseudo-T)
// + v (dJ/dq_x(x) s_ix + dJ/dq_y(x) s_iy) (q = v sum_i d_i s_i, Eq. q_corr); NULL seeds are 0.
__global__ void k_adj_seed(const AdjArgs a, const float* dJ_dT, const float* dJ_dqx,
                           const float* dJ_dqy, const float* sx, const float* sy, float vg,
                           const float* e_final, double e_ref, double theta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nx * a.ny) return;
  const int y = t / a.nx, x = t - y * a.nx;
  const int64_t off = int64_t(y + 2) * a.pitch + (x + kX0);
  float g = 0.f;
  if (dJ_dT) {
    const double e = e_ref + double(e_final[off]);
    const double lg = log1p(1.0 / e);
    g = float(double(dJ_dT[t]) * theta / (lg * lg * e * (1.0 + e)));
  }
  // q = v_g sum_i d_i s_i (Eq. q_corr)
  const float gx = dJ_dqx ? dJ_dqx[t] * vg : 0.f, gy = dJ_dqy ? dJ_dqy[t] * vg : 0.f;
  for (int i = 0; i < a.q; ++i)
    a.lam_out[int64_t(i) * a.plane + off] = fmaf(gy, sy[i], fmaf(gx, sx[i], g));
}

// dJ/dMFP = dJ/dW_corr * dW_corr/dMFP on interior cells; dJ/d(dT0) from l^0 through the
// initial condition e_i = w_i e_eq(T_ref + dT0) (ghost cells copy the nearest cell).
__global__ void k_adj_final(const AdjArgs a, const float* dwc, float* dJ_dmfp,
                            const float* lam0, const float* s0, const float* dT0,
                            float* dJ_ddT0, double t_ref, double theta) {
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
        // l^0_i = lh_i + s, so sum_i w_i l^0_i = sum_i w_i lh_i + s sum_i w_i
        double s = 0.0, wsum = 0.0;
        for (int i = 0; i < a.q; ++i) {
          s += double(a.w[i]) * lam0[int64_t(i) * a.plane + off];
          wsum += double(a.w[i]);
        }
        acc += s + wsum * double(s0[off]);
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
  const dim3 block(32, kAdjRows);
  const dim3 grid((kX0 + a.nx - kAdjC0) / kAdjTW + 1, (a.ny + 2 + kAdjRows - 1) / kAdjRows);
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
  const int chunks = wall_chunk_count(wa.nseg, wa.seg);
  if (chunks == 0) return cudaSuccess;
  k_walls_T<<<chunks, 32 * kWallWarpsT, 0, s>>>(wa, lam, gtw);
  return cudaGetLastError();
}

cudaError_t launch_adj_seed(const AdjArgs& a, const float* dJ_dT, const float* dJ_dqx,
                            const float* dJ_dqy, const float* sx, const float* sy, float vg,
                            const float* e_final, double e_ref, double theta, cudaStream_t s) {
  k_adj_seed<<<nblk(int64_t(a.nx) * a.ny, 256), 256, 0, s>>>(a, dJ_dT, dJ_dqx, dJ_dqy, sx, sy,
                                                              vg, e_final, e_ref, theta);
  return cudaGetLastError();
}

cudaError_t launch_adj_final(const AdjArgs& a, const float* dwc, float* dJ_dmfp,
                             const float* lam0, const float* s0, const float* dT0,
                             float* dJ_ddT0, double t_ref, double theta, cudaStream_t s) {
  k_adj_final<<<nblk(int64_t(a.nx) * a.ny, 256), 256, 0, s>>>(a, dwc, dJ_dmfp, lam0, s0, dT0,
                                                               dJ_ddT0, t_ref, theta);
  return cudaGetLastError();
}

}  // namespace wlbm
