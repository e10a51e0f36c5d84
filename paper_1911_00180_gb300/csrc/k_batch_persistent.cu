// Persistent batched kernel: the wall pass and the TMA-tile step of every instance of a
// batch, for a whole chunk of steps, in one launch of a fixed grid (a few blocks per SM).
//
// Many uncoupled gray problems (Sec. 2.1: the multigray approach solves one gray BTE per
// band; a batch also holds films of other sizes, Knudsen numbers and Q) share the GPU.
// A block takes work items from a queue in a fixed order: for every step t of the chunk,
// the wall chunks of every instance (Sec. 2.6 on the ghost frame of state t), then the
// step tiles of every instance (Eq. lbm-energy / Eq. algorithm, the same tile code as
// the other variant-3 kernels, so results are bit for bit those of the launch-per-step
// form).  Instead of a grid-wide barrier between the passes, every item waits only for
// what it reads: a wall chunk of instance k at step t for all of k's tiles of step t - 1,
// a tile for all of k's wall chunks of step t and all of k's tiles of step t - 1 (the
// energy planes rotate, so a tile also overwrites what those tiles read).  A tile's wall
// chunks were queued a whole wall pass earlier, and a wall chunk's tiles of the previous
// step a whole tile pass earlier, so waits are rare.  Items are claimed in queue order and
// depend only on earlier items, which running blocks hold, so the waits always end; each
// is still bounded in time, and a wait that gives up sets the instance's status word and an
// abort flag that makes every block leave.  Waits happen only between items, when no
// tensor copy of the block is in flight.
#include <cuda.h>

#include "elem.cuh"
#include "mbar.cuh"
#include "step_tile.cuh"
#include "walls.cuh"
#include "wlbm_internal.hpp"

namespace wlbm {

namespace {

constexpr int kPersistThreads = 32 * (kWarps3 + 1);   // 8 warps: the wall pass's kWallWarps
static_assert(kPersistThreads == 32 * kWallWarps, "wall chunks and tiles use the same block");

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until *ctr >= target; false when the abort flag is raised or `limit` cycles pass.
__device__ bool wait_count(const unsigned* ctr, unsigned target, const int* abort_flag,
                           long long limit) {
  if (ld_acquire(ctr) >= target) return true;
  const long long t0 = clock64();
  while (true) {
    __nanosleep(64);
    if (ld_acquire(ctr) >= target) return true;
    if (*reinterpret_cast<const volatile int*>(abort_flag) != 0) return false;
    if (clock64() - t0 > limit) return false;
  }
}

// Wall chunks and step tiles never run at the same time in a block, and a tile leaves no
// tensor copy in flight, so a wall chunk's shared data overlays the ring of the tiles.
struct WallOverlay {
  WallSmem wsm;
  WallArgs wa;
};

struct PersistShared {
  StepArgs sa;
  const void* tm;
  const uint8_t* wcodes;
  float* we_ref;
  int kind;     // -1: leave, 0: wall chunk, 1: step tile
  int inst, local;
  int fail;
};

// Resident blocks per SM the register budget aims at: the bfloat16 tile keeps its cell
// terms in shared memory and fits three blocks; float32 keeps them in registers (two).
template <typename T>
constexpr int persist_min_blocks() { return sizeof(T) == 2 ? 3 : 2; }

template <typename T, int S, bool SPEC>
__global__ void __launch_bounds__(kPersistThreads, persist_min_blocks<T>())
    k_batch_persistent(const PersistArgs p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ PersistShared ps;
  using LY = TmaLayout<T, S>;
  static_assert(sizeof(WallOverlay) <= LY::off_bar, "the wall data fits in the ring");
  WallOverlay& wo = *reinterpret_cast<WallOverlay*>(smem);
  constexpr bool REF = sizeof(T) == 2;
  const int tid = int(threadIdx.x);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY::off_bar);
  uint64_t* empty = full + S;
  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kWarps3);      // every consumer warp releases every box
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ps.fail = 0;
  }
  __syncthreads();
  uint32_t g0 = 0;   // ring uses of this block so far
  const int per_step = p.wall_items + p.tile_items;
  const int total = p.steps * per_step;
  unsigned* queue = p.ctr;
  unsigned* done_w = p.ctr + 1;
  unsigned* done_t = p.ctr + 1 + p.n;
  while (true) {
    if (tid == 0) {
      int kind = -1;
      const int item = int(atomicAdd(queue, 1u));
      if (item < total && *reinterpret_cast<const volatile int*>(p.abort_flag) == 0) {
        const int t = item / per_step;
        const int r = item - t * per_step;
        // a step's items: the wall chunks of every instance, then the tiles of every
        // instance (their instances from host-built tables: one load each)
        const bool wall = r < p.wall_items;
        const int rr = wall ? r : r - p.wall_items;
        const int k = wall ? p.wall_inst[rr] : p.tile_inst[rr];
        const int local = rr - (wall ? p.walls[k].first_block : p.insts[k].first_tile);
        const int nwall = p.walls[k].n_blocks;
        bool ok;
        if (wall) {
          ok = wait_count(done_t + k, unsigned(t) * unsigned(p.insts[k].n_tiles), p.abort_flag,
                          p.wait_limit);
          kind = 0;
          ps.local = local;
        } else {
          const unsigned need_w = unsigned(t + 1) * unsigned(nwall) +
                                  (p.stall_test && k == 0 ? 1u : 0u);
          ok = wait_count(done_w + k, need_w, p.abort_flag, p.wait_limit) &&
               wait_count(done_t + k, unsigned(t) * unsigned(p.insts[k].n_tiles), p.abort_flag,
                          p.wait_limit);
          kind = 1;
          ps.local = local;
        }
        if (!ok) {
          atomicOr(p.insts[k].a.status, 1);
          atomicExch(p.abort_flag, 1);
          kind = -1;
        } else if (kind == 0) {
          const BatchWalls& B = p.walls[k];
          const int cur = (B.phase + t) % B.n_e;
          ps.we_ref = B.n_e == 3 ? B.e[(cur + 2) % 3] : nullptr;
          ps.wcodes = B.codes + size_t(t) * B.w.q;
        } else {
          const BatchInst& I = p.insts[k];
          ps.sa = I.a;
          ps.sa.codes = I.codes + size_t(t) * I.a.q;
          ps.sa.order = I.order + size_t(t) * (I.a.q + 17);
          const int cur = (I.phase + t) % I.n_e;
          ps.sa.e_in = I.e[cur];
          ps.sa.e_out = I.e[(cur + 1) % I.n_e];
          ps.sa.e_ref = I.n_e == 3 ? I.e[(cur + 2) % 3] : nullptr;
          ps.tm = I.tmap;
        }
        ps.inst = k;
      }
      ps.kind = kind;
    }
    __syncthreads();
    const int kind = ps.kind;
    if (kind < 0) break;
    const int k = ps.inst;
    if (kind == 0) {
      static_assert(sizeof(WallArgs) % 4 == 0, "copied as 32-bit words");
      const int* src = reinterpret_cast<const int*>(&p.walls[k].w);
      int* dst = reinterpret_cast<int*>(&wo.wa);
      for (int i = tid; i < int(sizeof(WallArgs) / 4); i += kPersistThreads) dst[i] = src[i];
      __syncthreads();
      walls_chunk<T, SPEC>(wo.wa, ps.wcodes, ps.we_ref, ps.local, wo.wsm, nullptr);
    } else {
      const int tx = p.insts[k].tiles_x;
      const int bx = ps.local % tx, by = ps.local / tx;
      const bool ok = ps.sa.wfield
                          ? step_tma_tile<T, S, true, REF, true>(ps.sa, ps.tm, bx, by, smem, g0)
                          : step_tma_tile<T, S, false, REF, true>(ps.sa, ps.tm, bx, by, smem, g0);
      if (!ok) ps.fail = 1;
    }
    __syncthreads();
    if (tid == 0) {
      if (ps.fail) {
        atomicExch(p.abort_flag, 1);   // this block's ring phases are no longer in step
      } else {
        __threadfence();               // the item's stores before its completion count
        atomicAdd(kind == 0 ? done_w + k : done_t + k, 1u);
      }
    }
    if (ps.fail) break;                // uniform: set before the last barrier
  }
}

template <typename T, int S>
cudaError_t configure_t() {
  const int bytes = int(TmaLayout<T, S>::bytes(kMaxQ));
  const void* fns[2] = {(const void*)k_batch_persistent<T, S, false>,
                        (const void*)k_batch_persistent<T, S, true>};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fns[i], cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
  }
  return e;
}

template <typename T, int S>
int blocks_per_sm_t(int max_q) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, k_batch_persistent<T, S, true>, kPersistThreads,
          TmaLayout<T, S>::bytes(max_q)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T, int S>
cudaError_t launch_t(const PersistArgs& p, int max_q, int grid, bool any_spec, cudaStream_t s) {
  const size_t bytes = TmaLayout<T, S>::bytes(max_q);
  if (any_spec)
    k_batch_persistent<T, S, true><<<grid, kPersistThreads, bytes, s>>>(p);
  else
    k_batch_persistent<T, S, false><<<grid, kPersistThreads, bytes, s>>>(p);
  return cudaGetLastError();
}

// Ring depths compiled for the persistent kernel (the first is the default).
constexpr int kF32Stages[2] = {6, 4};
constexpr int kBF16Stages[2] = {8, 16};

}  // namespace

bool batch_persistent_stages_ok(int storage, int stages) {
  const int* list = storage == WLBM_STORE_BF16_DEV ? kBF16Stages : kF32Stages;
  return stages == 0 || stages == list[0] || stages == list[1];
}

cudaError_t configure_batch_persistent() {
  cudaError_t e = configure_t<float, kF32Stages[0]>();
  if (e == cudaSuccess) e = configure_t<float, kF32Stages[1]>();
  if (e == cudaSuccess) e = configure_t<__nv_bfloat16, kBF16Stages[0]>();
  if (e == cudaSuccess) e = configure_t<__nv_bfloat16, kBF16Stages[1]>();
  return e;
}

int batch_persistent_blocks_per_sm(int storage, int stages, int max_q) {
  if (storage == WLBM_STORE_BF16_DEV)
    return stages == kBF16Stages[1] ? blocks_per_sm_t<__nv_bfloat16, kBF16Stages[1]>(max_q)
                                    : blocks_per_sm_t<__nv_bfloat16, kBF16Stages[0]>(max_q);
  return stages == kF32Stages[1] ? blocks_per_sm_t<float, kF32Stages[1]>(max_q)
                                 : blocks_per_sm_t<float, kF32Stages[0]>(max_q);
}

cudaError_t launch_batch_persistent(int storage, int stages, const PersistArgs& p, int max_q,
                                    int grid, bool any_spec, cudaStream_t s) {
  if (grid <= 0 || p.steps <= 0) return cudaSuccess;
  if (storage == WLBM_STORE_BF16_DEV)
    return stages == kBF16Stages[1]
               ? launch_t<__nv_bfloat16, kBF16Stages[1]>(p, max_q, grid, any_spec, s)
               : launch_t<__nv_bfloat16, kBF16Stages[0]>(p, max_q, grid, any_spec, s);
  return stages == kF32Stages[1] ? launch_t<float, kF32Stages[1]>(p, max_q, grid, any_spec, s)
                                 : launch_t<float, kF32Stages[0]>(p, max_q, grid, any_spec, s);
}

}  // namespace wlbm
