// wlbm_reduce_state_noalloc: the float64 reductions of wlbm_reduce for callers that may
// not allocate device memory.  Its scratch (per-block partial sums) lives in a file-scope
// device array, so the call path contains no cudaMalloc / cudaFree.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include <string>

#include "elem.cuh"
#include "wlbm_internal.hpp"

namespace {

constexpr int kThreads = 256;
// Partial sums of at most kMaxBlocks blocks of kThreads framed cells: 32768 * 256 cells
// = 8,388,608 cells of the (nx+2) x (ny+2) frame (for example 2894 x 2894 interior).
constexpr int kMaxBlocks = 32768;
constexpr int kOut = 4;

// 1 MiB of scratch held by every device that loads the library, until process exit.
// Host code must not use this name as an address: use the pointer from set_up().
static __device__ __align__(256) double g_partials[kMaxBlocks * kOut];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {nullptr};

// Direction i of the Q = 8M ring (counter-clockwise from +x), as unit vector.
__device__ __forceinline__ void ring_unit(int i, int m, double* sx, double* sy) {
  int x, y;
  if (i < m) { x = m; y = i; }
  else if (i < 3 * m) { x = 2 * m - i; y = m; }
  else if (i < 5 * m) { x = -m; y = 4 * m - i; }
  else if (i < 7 * m) { x = i - 6 * m; y = -m; }
  else { x = m; y = i - 8 * m; }
  const double len = sqrt(double(x) * x + double(y) * y);
  *sx = x / len;
  *sy = y / len;
}

// One block per kThreads framed cells: (sum E interior, sum E interior + adiabatic-wall
// ghost cells, sum q_x, sum q_y) of its cells into partials[block].
__global__ void k_partials(const float* framed, int nx, int ny, int q, int diff_mask,
                           double* partials) {
  const int fw = nx + 2, fh = ny + 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double v[kOut] = {0.0, 0.0, 0.0, 0.0};
  if (t < fw * fh) {
    const int fy = t / fw, fx = t - fy * fw;
    const bool gx = fx == 0 || fx == fw - 1, gy = fy == 0 || fy == fh - 1;
    const int64_t plane = int64_t(fw) * fh;
    if (!gx && !gy) {
      double e = 0.0, qx = 0.0, qy = 0.0;
      for (int i = 0; i < q; ++i) {
        const double d = framed[int64_t(i) * plane + t];
        double sx, sy;
        ring_unit(i, q / 8, &sx, &sy);
        e += d;
        qx += d * double(float(sx));
        qy += d * double(float(sy));
      }
      v[0] = e;
      v[1] = e;
      v[2] = qx;
      v[3] = qy;
    } else if (wlbm::wall_energy_cell(fx, fy, fw, fh, diff_mask)) {
      double e = 0.0;
      for (int i = 0; i < q; ++i) e += framed[int64_t(i) * plane + t];
      v[1] = e;
    }
  }
  __shared__ double red[kOut][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    const double s = wlbm::warp_sum(v[k]);
    if (lane == 0) red[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[int64_t(blockIdx.x) * kOut + threadIdx.x] = s;   // every slot used is written
  }
}

// One block: fixed-order sum of the partials, means of q over the interior.
__global__ void k_finish(const double* partials, int nblocks, double inv_cells, double speed,
                         double* out) {
  __shared__ double red[kOut][kThreads / 32];
  double v[kOut] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int k = 0; k < kOut; ++k) v[k] += partials[int64_t(b) * kOut + k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kOut; ++k) {
    const double s = wlbm::warp_sum(v[k]);
    if (lane == 0) red[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < kOut) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    // heat flux (Eq. q_corr): v_g sum_i e_i s_i, v_g = the band's speed in cells per step
    out[threadIdx.x] = threadIdx.x >= 2 ? s * inv_cells * speed : s;
  }
}

// Once per device, with that device current: the device address of the scratch array.
cudaError_t set_up(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" wlbm_status wlbm_reduce_state_noalloc(const float* framed, int32_t nx, int32_t ny,
                                                 int32_t q, double speed,
                                                 const int32_t* bc_kind, double* out,
                                                 void* stream) {
  if (!framed || !out || !bc_kind || nx < 1 || ny < 1 || q < 8 || q > 1024 || q % 8) {
    wlbm::set_global_error_msg("wlbm_reduce_state_noalloc: invalid pointer, size or Q");
    return WLBM_ERR_INVALID_ARG;
  }
  if (!(speed > 0.0 && speed <= 1.0)) {
    wlbm::set_global_error_msg("wlbm_reduce_state_noalloc: speed must lie in (0, 1]");
    return WLBM_ERR_INVALID_ARG;
  }
  const int64_t cells = (int64_t(nx) + 2) * (int64_t(ny) + 2);
  const int64_t nblocks = (cells + kThreads - 1) / kThreads;
  if (nblocks > kMaxBlocks) {
    wlbm::set_global_error_msg(
        "wlbm_reduce_state_noalloc: the framed grid has " + std::to_string(cells) +
        " cells, more than the " + std::to_string(int64_t(kMaxBlocks) * kThreads) +
        " its fixed scratch covers");
    return WLBM_ERR_INVALID_ARG;
  }
  double* partials = nullptr;
  const cudaError_t se = set_up(&partials);
  if (se != cudaSuccess) {
    wlbm::set_global_error_msg(std::string("wlbm_reduce_state_noalloc: set-up failed: ") +
                               cudaGetErrorString(se));
    return WLBM_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int diff_mask = 0;
  for (int k = 0; k < 4; ++k)
    if (bc_kind[k] == WLBM_BC_ADIABATIC_DIFFUSE || bc_kind[k] == WLBM_BC_ADIABATIC_SPECULAR)
      diff_mask |= 1 << k;
  // a launch error of earlier, unrelated work must not be reported as this call's
  cudaGetLastError();
  k_partials<<<unsigned(nblocks), kThreads, 0, s>>>(framed, nx, ny, q, diff_mask, partials);
  k_finish<<<1, kThreads, 0, s>>>(partials, int(nblocks), 1.0 / (double(nx) * ny), speed, out);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    wlbm::set_global_error_msg(std::string("wlbm_reduce_state_noalloc: ") + cudaGetErrorString(le));
    return WLBM_ERR_CUDA;
  }
  return WLBM_OK;
}
