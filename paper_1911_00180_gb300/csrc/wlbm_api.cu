// C ABI of libwlbm: handle lifecycle, boundary tables, the per-step launch sequence.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "wlbm_internal.hpp"

using namespace wlbm;

namespace {

constexpr int kChunk = 1024;   // steps whose codes are uploaded per host->device copy

std::mutex g_err_mu;
std::string g_err;             // errors before a handle exists

void set_global_error(const std::string& m) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = m;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// An event record on stream s; `node`: the stream is being captured and the record becomes
// an event node of the graph (timed each time the graph replays).
cudaError_t record_event(cudaEvent_t e, cudaStream_t s, bool node) {
  return node ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// One instantiated CUDA graph of a chunk of steps.  Captured while profiling, its timed
// step-kernel launches record event pairs through event nodes; a replay overwrites them,
// so they are read (waiting for that replay) before the graph replays again.
struct TimedGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;   // (start, stop) pairs
  int weight = 1;                // steps one pair times (a persistent launch: its steps)
  cudaEvent_t done = nullptr;    // recorded after every replay when there are pairs
  bool pending = false;          // replayed since the pairs were last read

  // Events for `pairs` timed launches (before the capture).
  cudaError_t make_events(int pairs) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 * pairs && e == cudaSuccess; ++k) {
      cudaEvent_t x = nullptr;
      e = cudaEventCreate(&x);
      if (e == cudaSuccess) ev.push_back(x);
    }
    if (pairs > 0 && e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    return e;
  }
  // Adds the latest replay's durations (ms) and pair count to *ms and *n.
  cudaError_t harvest(double* ms, int64_t* n) {
    if (!pending) return cudaSuccess;
    pending = false;
    cudaError_t e = cudaEventSynchronize(done);
    for (size_t k = 0; e == cudaSuccess && k + 1 < ev.size(); k += 2) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      *ms += t;
      *n += weight;
    }
    return e;
  }
  cudaError_t launch(cudaStream_t s) {
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e == cudaSuccess && done) {
      e = cudaEventRecord(done, s);
      pending = e == cudaSuccess;
    }
    return e;
  }
  void destroy() {
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t x : ev) cudaEventDestroy(x);
    if (done) cudaEventDestroy(done);
    exec = nullptr;
    ev.clear();
    done = nullptr;
    pending = false;
  }
};

}  // namespace

void wlbm::set_global_error_msg(const std::string& m) { set_global_error(m); }

struct wlbm_handle {
  Geom g;
  int storage = 0, emulate_3d = 0, relax_mode = 0;
  double t_ref = 300.0, theta = 624.8, e_eq_ref = 0.0;
  float scale = 1.f, inv_scale = 1.f;
  int bc_kind[4] = {0, 0, 0, 0};
  double t_wall[4] = {0, 0, 0, 0};
  float spec[4] = {0.f, 0.f, 0.f, 0.f};   // specularity of adiabatic walls
  int xper = 1, yper = 1;
  Lattice lat;
  TasState tas;
  bool field_w = false;
  float w0 = 0.f;
  wlbm_allocator alloc{nullptr, nullptr, nullptr};
  cudaStream_t stream = nullptr;
  // device memory
  void* planes = nullptr;     // [2][q][plane] storage elements
  float* e[3] = {nullptr, nullptr, nullptr};   // local-energy planes (3 for bfloat16)
  int e_cur = 0, e_ref = -1, e_spare = 1;      // roles of the energy planes
  float* wfield = nullptr;    // framed W_corr (per-cell MFP only)
  float* consts = nullptr;    // w[q], sx[q], sy[q], rho[8][q]
  int16_t* mirror = nullptr;  // [2][q] mirror directions (c_x flipped, c_y flipped)
  uint8_t* d_codes = nullptr; // [kChunk][q]
  uint16_t* d_order = nullptr; // [kChunk][q + 17] kind-sorted directions (variant 3)
  double* d_red = nullptr;    // [kReduceOut]
  double* d_red_part = nullptr;   // [kReduceBlocks][kReduceOut] reduction partials
  double* d_snap = nullptr;   // nx*ny float64 T - T_ref at the last reduction
  int64_t snap_step = -1;     // step of that snapshot (-1: none since the state was set)
  bool batch_owned = false;   // instance of a wlbm_batch (its records cache plane roles)
  // internal sources / radiation cells (wlbm_set_sources)
  int n_src = 0;
  int64_t* d_src_off = nullptr;
  float* d_src_val = nullptr;   // [n_src][q] deviations
  float* d_src_e = nullptr;     // [n_src] sums
  double* d_win = nullptr;    // nx*ny float64 window sum and previous window mean of
  double* d_win_prev = nullptr;   // T - T_ref (wlbm_run_steady; allocated on first use)
  int* d_status = nullptr;    // bit 0: a bounded device wait gave up
  int step_variant = 1;       // 0 register-pipelined, 1 per-warp bulk-copy ring,
                              // 2 warp-specialised ring, 3 TMA tiles
  alignas(64) unsigned char tmap[128] = {};   // CUtensorMap of the planes (variant 3)
  bool has_tmap = false;
  std::string tmap_why;       // why there is no tensor map
  alignas(64) unsigned char tmap_w[128] = {};  // bfloat16 planes as 32-bit words (wide tiles)
  bool has_tmap_w = false;
  int bf16_wide = 0;          // variant 3, bfloat16: 1 = 256-column tiles (the default
                              // where the planes have a 32-bit-word tensor map)
  int graph_steps = 0;        // >0: replay chunks of this many steps as one CUDA graph
  int ring_stages = 0;        // variant 3 ring depth (0: by Q)
  int tile_loop = 0;          // variant 3: 1 = resident blocks loop over the tiles
  int loop_blocks = 0;        // blocks of that grid (set with the options)
  int fuse_periodic = 0;      // 1: both axes periodic, the step kernel mirrors the edges
  // per energy-plane role and replay parity (consecutive replays alternate, so a graph's
  // event pairs are read while the other one runs)
  TimedGraph graphs[3][2];
  int graph_parity = 0;
  int64_t graph_replays = 0;  // chunks run as graph replays (WLBM_OPT_GRAPH_REPLAYS)
  int64_t graph_launches = 0; // kernels per graph replay
  std::vector<void*> owned;
  // host staging
  uint8_t* h_codes[2] = {nullptr, nullptr};
  uint16_t* h_order[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int slot = 0;
  WallArgs walls{};
  std::string err;
  // MFP kept on the host for the adjoint's dW_corr/dMFP
  std::vector<float> mfp_host;
  double mfp_uniform = 0.0;
  // adjoint (checkpointed forward + reverse sweep), float32 storage only
  struct Adj {
    int64_t n = 0;
    int k = 0, nck = 0;
    bool ready = false;
    float* ckpt = nullptr;     // [nck][q][plane] states before the boundary pass
    float* ckpt_e = nullptr;   // [nck][plane] their local energy
    float* tape = nullptr;     // [k][q][plane] recomputed step inputs of one segment
    float* lam[2] = {nullptr, nullptr};   // per-direction part lh of the adjoint
    float* sh[2] = {nullptr, nullptr};    // shared part s (one plane)
    float* erec[2] = {nullptr, nullptr};
    float* gw = nullptr;       // framed dJ/dW_corr
    float* dwc = nullptr;      // nx*ny dW_corr/dMFP
    float* dT0 = nullptr;      // nx*ny start field
    double* gtw = nullptr;     // [4] sum_i w_i lambda_i at isothermal ghosts
    uint8_t* codes = nullptr;  // [n][q] schedule of the run
    uint16_t* order = nullptr; // [n][q + 17] kind-sorted directions of every step
    alignas(64) unsigned char tape_tmap[128] = {};   // CUtensorMap of the k x q tape planes
    bool has_tape_tmap = false;
    alignas(64) unsigned char lam_tmap[2][128] = {}; // CUtensorMaps of the lh planes (16 rows)
    alignas(64) unsigned char lam14_tmap[2][128] = {};   // the same planes, 14-row boxes
    alignas(64) unsigned char tape_adj_tmap[128] = {};   // the tape, 14 x 128 boxes
    bool has_lam_tmap = false;
    std::vector<void*> bufs;
  } adj;
  // launch accounting and optional per-launch timing of the step kernel
  int64_t launches = 0;
  int prof_every = 0;                 // time every prof_every-th step launch (0: none)
  int64_t prof_tick = 0;              // step launches seen while profiling
  std::vector<cudaEvent_t> prof_ev;   // pairs (start, stop)
  size_t prof_used = 0;
  double prof_graph_ms = 0.0;         // read from replayed graphs, not yet reported
  int64_t prof_graph_n = 0;

  size_t elem() const { return storage == WLBM_STORE_BF16_DEV ? 2 : 4; }
  float* w_dev() const { return consts; }
  float* sx_dev() const { return consts + g.q; }
  float* sy_dev() const { return consts + 2 * g.q; }
  float* rho_dev() const { return consts + 3 * g.q; }

  wlbm_status fail(wlbm_status s, const std::string& m) {
    err = m;
    return s;
  }
  wlbm_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return WLBM_OK;
    return fail(WLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  void* dev_alloc(size_t bytes) {
    bytes = size_t(round_up(int64_t(bytes), 256));
    void* p = nullptr;
    if (alloc.alloc) {
      p = alloc.alloc(bytes, alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void dev_free(void* p) {
    for (size_t k = 0; k < owned.size(); ++k) {
      if (owned[k] != p) continue;
      if (alloc.alloc) {
        if (alloc.free) alloc.free(p, alloc.ctx);
      } else {
        cudaFree(p);
      }
      owned.erase(owned.begin() + long(k));
      return;
    }
  }
  // Destroys the graphs, keeping the timings of their latest replays for the next read.
  void drop_graphs() {
    for (auto& role : graphs)
      for (TimedGraph& tg : role) {
        tg.harvest(&prof_graph_ms, &prof_graph_n);
        tg.destroy();
      }
  }
  void release() {
    drop_graphs();
    for (void* p : owned) {
      if (alloc.alloc) {
        if (alloc.free) alloc.free(p, alloc.ctx);
      } else {
        cudaFree(p);
      }
    }
    owned.clear();
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
    for (int k = 0; k < 2; ++k) {
      if (h_codes[k]) cudaFreeHost(h_codes[k]);
      if (h_order[k]) cudaFreeHost(h_order[k]);
      h_order[k] = nullptr;
      if (ev[k]) cudaEventDestroy(ev[k]);
      h_codes[k] = nullptr;
      ev[k] = nullptr;
    }
  }
  ParityMask parity_mask() const {
    ParityMask m{};
    for (int i = 0; i < g.q; ++i)
      if (tas.parity[i]) m.bits[i >> 5] |= 1u << (i & 31);
    return m;
  }
  double delta_e(double t) const { return 1.0 / std::expm1(theta / t) - e_eq_ref; }
  bool bf16() const { return storage == WLBM_STORE_BF16_DEV; }
  float* ref_plane() const { return e_ref >= 0 ? e[e_ref] : nullptr; }
  void rotate_energy() {      // after a step: new state's E becomes current
    if (e_ref >= 0) {
      const int old_ref = e_ref;
      e_ref = e_cur;
      e_cur = e_spare;
      e_spare = old_ref;
    } else {
      std::swap(e_cur, e_spare);
    }
  }
  void build_wall_segments();
};

// Ghost-cell segments handled by the wall kernel: non-periodic edges and the corners
// that touch no periodic wall.  Corners: an isothermal x-wall decides, then an
// isothermal y-wall, else two diffuse walls use the quadrant-diagonal rule.
void wlbm_handle::build_wall_segments() {
  WallArgs& a = walls;
  a.nseg = 0;
  const int nx = g.nx, ny = g.ny;
  const int gl = kGhostCol, gr = kX0 + nx;
  struct Edge { int count, r0, c0, dr, dc; };
  const Edge edges[4] = {{ny, 2, gl, 1, 0}, {ny, 2, gr, 1, 0},
                         {nx, 1, kX0, 0, 1}, {nx, ny + 2, kX0, 0, 1}};
  auto push = [&](int count, int r0, int c0, int dr, int dc, int kind, int table, int wall) {
    WallSeg& s = a.seg[a.nseg++];
    s.count = count; s.r0 = r0; s.c0 = c0; s.dr = dr; s.dc = dc;
    s.action = kind;
    s.table = table;
    s.wall = wall;
    s.iso = kind == WLBM_BC_ISOTHERMAL ? float(delta_e(t_wall[wall])) : 0.f;
    // edges of adiabatic walls: specularity and mirror table (x walls flip c_x, y walls
    // c_y); corners keep the diffuse rule
    s.spec = kind == WLBM_BC_ADIABATIC_DIFFUSE && table < 4 ? spec[wall] : 0.f;
    s.mirror = table < 2 ? 0 : 1;
  };
  for (int k = 0; k < 4; ++k) {
    if (bc_kind[k] == WLBM_BC_PERIODIC) continue;
    push(edges[k].count, edges[k].r0, edges[k].c0, edges[k].dr, edges[k].dc, bc_kind[k], k, k);
  }
  const int cr[4] = {1, 1, ny + 2, ny + 2}, cc[4] = {gl, gr, gl, gr};
  const int cxw[4] = {0, 1, 0, 1}, cyw[4] = {2, 2, 3, 3};
  for (int k = 0; k < 4; ++k) {
    const int xw = cxw[k], yw = cyw[k];
    if (bc_kind[xw] == WLBM_BC_PERIODIC || bc_kind[yw] == WLBM_BC_PERIODIC) continue;
    if (bc_kind[xw] == WLBM_BC_ISOTHERMAL)
      push(1, cr[k], cc[k], 0, 0, WLBM_BC_ISOTHERMAL, 0, xw);
    else if (bc_kind[yw] == WLBM_BC_ISOTHERMAL)
      push(1, cr[k], cc[k], 0, 0, WLBM_BC_ISOTHERMAL, 0, yw);
    else
      push(1, cr[k], cc[k], 0, 0, WLBM_BC_ADIABATIC_DIFFUSE, 4 + k, xw);
  }
  a.any_spec = 0;
  for (int k = 0; k < a.nseg; ++k)
    if (a.seg[k].spec > 0.f) a.any_spec = 1;
  a.planes = planes;
  a.plane = g.plane;
  a.pitch = g.pitch;
  a.q = g.q;
  a.w = w_dev();
  a.rho = rho_dev();
  a.mirror = mirror;
  a.scale = scale;
  a.inv_scale = inv_scale;
}

// Fill the periodic ghost cells (and their energies) from the current state, with plane
// parities from the host mask.  Used after the state is set from outside the step loop.
static wlbm_status refresh_periodic(wlbm_handle* h) {
  if (!h->xper && !h->yper) return WLBM_OK;
  const Geom& g = h->g;
  const ParityMask m = h->parity_mask();
  PeriodicArgs pa{};
  pa.planes = h->planes; pa.plane = g.plane; pa.pitch = g.pitch; pa.nx = g.nx; pa.ny = g.ny;
  pa.q = g.q; pa.codes = nullptr; pa.e_cur = h->e[h->e_cur]; pa.e_ref = h->ref_plane();
  pa.xper = h->xper; pa.yper = h->yper;
  // the mask goes to the device through the schedule buffer (stream-ordered)
  wlbm_status st = h->cuda(cudaMemcpyAsync(h->d_codes, m.bits, sizeof(m.bits),
                                           cudaMemcpyHostToDevice, h->stream), "periodic refresh");
  if (st != WLBM_OK) return st;
  st = h->cuda(cudaStreamSynchronize(h->stream), "periodic refresh");   // m is on the stack
  if (st != WLBM_OK) return st;
  pa.par = reinterpret_cast<const ParityMask*>(h->d_codes);
  ++h->launches;
  return h->cuda(launch_periodic(h->storage, pa, h->stream), "periodic refresh");
}

// Diffuse re-emission fractions: tables 0-3 for the walls (inward normals +x, -x, +y,
// -y), 4-7 for the corners (quadrant diagonal, strictly inward directions only).
static std::vector<float> rho_tables(const Lattice& L) {
  const int q = L.q;
  std::vector<float> rho(size_t(8) * q, 0.f);
  const int nrm[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
  for (int t = 0; t < 8; ++t) {
    const int nx = nrm[t][0], ny = nrm[t][1];
    const double len = std::sqrt(double(nx * nx + ny * ny));
    std::vector<double> r(q, 0.0);
    double sum = 0.0;
    for (int i = 0; i < q; ++i) {
      const bool inward = t < 4 ? (L.dx[i] * nx + L.dy[i] * ny > 0)
                                : (L.dx[i] * nx > 0 && L.dy[i] * ny > 0);
      if (!inward) continue;
      r[i] = L.w[i] * (L.sx[i] * nx + L.sy[i] * ny) / len;
      sum += r[i];
    }
    for (int i = 0; i < q; ++i) rho[size_t(t) * q + i] = float(r[i] / sum);
  }
  return rho;
}

// Index of every direction with c_x flipped (row 0) and with c_y flipped (row 1): the
// mirror images at x and y walls (Eq. adiabatic-specular).
static std::vector<int16_t> mirror_tables(const Lattice& L) {
  const int q = L.q;
  std::vector<int16_t> m(size_t(2) * q, 0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      if (L.dx[j] == -L.dx[i] && L.dy[j] == L.dy[i]) m[i] = int16_t(j);
      if (L.dx[j] == L.dx[i] && L.dy[j] == -L.dy[i]) m[size_t(q) + i] = int16_t(j);
    }
  return m;
}

extern "C" {

const char* wlbm_last_error(const wlbm_handle* h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err.c_str();
}

wlbm_status wlbm_lattice(int32_t q, int32_t* dirs, double* weights, int8_t* worm,
                         double* lam_corr) {
  Lattice L;
  if (!build_lattice(q, &L)) {
    set_global_error("wlbm_lattice: Q must be a multiple of 8 in [8, 1024]");
    return WLBM_ERR_INVALID_ARG;
  }
  for (int i = 0; i < q; ++i) {
    if (dirs) { dirs[2 * i] = L.dx[i]; dirs[2 * i + 1] = L.dy[i]; }
    if (weights) weights[i] = L.w[i];
  }
  if (worm) std::memcpy(worm, L.worm.data(), L.worm.size());
  if (lam_corr) *lam_corr = L.lam_corr;
  return WLBM_OK;
}

wlbm_status wlbm_schedule(int32_t q, int64_t n_steps, double speed, uint8_t* codes) {
  Lattice L;
  if (speed == 0.0) speed = 1.0;
  if (!build_lattice(q, &L) || n_steps < 0 || (n_steps > 0 && !codes) ||
      !(speed > 0.0 && speed <= 1.0)) {
    set_global_error("wlbm_schedule: invalid Q, step count, speed or output");
    return WLBM_ERR_INVALID_ARG;
  }
  L.speed = speed;
  TasState st;
  st.reset(q);
  for (int64_t t = 0; t < n_steps; ++t) {
    tas_advance(L, &st, codes + t * q);
    for (int i = 0; i < q; ++i) codes[t * q + i] &= 0x0f;   // drop buffer parity
  }
  return WLBM_OK;
}

wlbm_status wlbm_create(const wlbm_grid* grid, const float* mfp_cells, double mfp_uniform,
                        const wlbm_boundary* bc, const wlbm_allocator* alloc, void* stream,
                        wlbm_handle** out) {
  if (!grid || !bc || !out) {
    set_global_error("wlbm_create: NULL grid, boundary or output pointer");
    return WLBM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const wlbm_grid& G = *grid;
  // sizes: the framed cell count indexes 32-bit thread ids of the per-cell kernels, and the
  // step kernels put 14-row tile rows in grid.y (at most 65535 of them)
  if (G.nx < 1 || G.ny < 1 || (int64_t(G.nx) + 2) * (int64_t(G.ny) + 2) > INT32_MAX ||
      int64_t(G.ny) + 2 > int64_t(65535) * 14 ||
      (G.storage != WLBM_STORE_FP32_DEV && G.storage != WLBM_STORE_BF16_DEV) ||
      (G.relax_mode != 0 && G.relax_mode != 1) || !(G.t_ref > 0) || !(G.theta > 0) ||
      !(G.speed == 0.0 || (G.speed > 0.0 && G.speed <= 1.0))) {
    set_global_error("wlbm_create: invalid grid (sizes, storage, relax_mode, t_ref, theta, "
                     "speed)");
    return WLBM_ERR_INVALID_ARG;
  }
  const double speed = G.speed == 0.0 ? 1.0 : G.speed;
  for (int k = 0; k < 4; ++k) {
    if (bc->kind[k] < 0 || bc->kind[k] > 3 ||
        (bc->kind[k] == WLBM_BC_ISOTHERMAL && !(bc->t_wall[k] > 0)) ||
        (bc->kind[k] == WLBM_BC_ADIABATIC_DIFFUSE &&
         !(bc->specularity[k] >= 0.0 && bc->specularity[k] <= 1.0))) {
      set_global_error("wlbm_create: invalid boundary kind or wall temperature");
      return WLBM_ERR_INVALID_ARG;
    }
  }
  if ((bc->kind[0] == WLBM_BC_PERIODIC) != (bc->kind[1] == WLBM_BC_PERIODIC) ||
      (bc->kind[2] == WLBM_BC_PERIODIC) != (bc->kind[3] == WLBM_BC_PERIODIC)) {
    set_global_error("wlbm_create: periodic walls must come in opposite pairs");
    return WLBM_ERR_INVALID_ARG;
  }
  auto* h = new wlbm_handle();
  h->storage = G.storage;
  h->emulate_3d = G.emulate_3d ? 1 : 0;
  h->relax_mode = G.relax_mode;
  h->t_ref = G.t_ref;
  h->theta = G.theta;
  h->e_eq_ref = 1.0 / std::expm1(G.theta / G.t_ref);
  for (int k = 0; k < 4; ++k) {
    // a specular wall is the adiabatic wall with specularity 1 (one wall path for both)
    h->bc_kind[k] = bc->kind[k] == WLBM_BC_ADIABATIC_SPECULAR ? WLBM_BC_ADIABATIC_DIFFUSE
                                                              : bc->kind[k];
    h->spec[k] = bc->kind[k] == WLBM_BC_ADIABATIC_SPECULAR ? 1.f
                 : bc->kind[k] == WLBM_BC_ADIABATIC_DIFFUSE ? float(bc->specularity[k]) : 0.f;
    h->t_wall[k] = bc->t_wall[k];
  }
  h->xper = bc->kind[0] == WLBM_BC_PERIODIC;
  h->yper = bc->kind[2] == WLBM_BC_PERIODIC;
  if (!build_lattice(G.q, &h->lat)) {
    delete h;
    set_global_error("wlbm_create: Q must be a multiple of 8 in [8, 1024]");
    return WLBM_ERR_INVALID_ARG;
  }
  h->lat.speed = speed;
  h->tas.reset(G.q);
  Geom& g = h->g;
  g.nx = G.nx; g.ny = G.ny; g.q = G.q;
  g.pitch = int(round_up(kX0 + G.nx + 2, 32));
  g.rows = G.ny + 4;
  g.plane = int64_t(g.pitch) * g.rows;
  if (alloc) h->alloc = *alloc;
  h->stream = static_cast<cudaStream_t>(stream);

  // relaxation weight (Eq. W-Kn, Eq. W-correction), stability (Appendix A: W <= 1)
  std::vector<float> wframe;
  auto bad = [&](wlbm_status s, const std::string& m) {
    h->release();
    delete h;
    set_global_error(m);
    return s;
  };
  if (mfp_cells) {
    std::vector<float> mfp(size_t(G.nx) * G.ny);
    if (cudaMemcpy(mfp.data(), mfp_cells, mfp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return bad(WLBM_ERR_CUDA, "wlbm_create: cannot read the MFP field");
    }
    h->field_w = true;
    h->mfp_host = mfp;
    wframe.assign(size_t(g.plane), 0.f);
    double wmax = 0.0;
    for (int y = 0; y < G.ny; ++y)
      for (int x = 0; x < G.nx; ++x) {
        const double m = mfp[size_t(y) * G.nx + x];
        if (!(m > 0)) return bad(WLBM_ERR_INVALID_ARG, "wlbm_create: MFP must be positive");
        const double wc = corrected_weight(m / speed, h->lat.lam_corr, h->emulate_3d,
                                           h->relax_mode);
        wmax = std::max(wmax, wc);
        wframe[size_t(g.cell(x, y))] = float(wc);
      }
    if (wmax > 1.0)
      return bad(WLBM_ERR_UNSTABLE, "wlbm_create: max W_corr > 1, unstable (use a larger MFP)");
    // periodic ghost cells carry W across the link (walls keep 0)
    auto at = [&](int r, int c) -> float& { return wframe[size_t(r) * g.pitch + c]; };
    if (h->yper) {
      const int c0 = h->xper ? kX0 : kGhostCol, c1 = h->xper ? kX0 + G.nx - 1 : kX0 + G.nx;
      for (int c = c0; c <= c1; ++c) { at(1, c) = at(G.ny + 1, c); at(G.ny + 2, c) = at(2, c); }
    }
    if (h->xper) {
      for (int r = 1; r <= G.ny + 2; ++r) {
        at(r, kGhostCol) = at(r, kX0 + G.nx - 1);
        at(r, kX0 + G.nx) = at(r, kX0);
      }
    }
  } else {
    if (!(mfp_uniform > 0))
      return bad(WLBM_ERR_INVALID_ARG, "wlbm_create: MFP must be positive");
    const double wc = corrected_weight(mfp_uniform / speed, h->lat.lam_corr, h->emulate_3d,
                                       h->relax_mode);
    if (wc > 1.0)
      return bad(WLBM_ERR_UNSTABLE, "wlbm_create: W_corr > 1, unstable (use a larger MFP)");
    h->w0 = float(wc);
    h->mfp_uniform = mfp_uniform;
  }

  // device memory through the caller's allocator
  const size_t plane_bytes = size_t(g.plane) * h->elem();
  // slack after the last plane: bulk row copies of the last tile may read past the row
  h->planes = h->dev_alloc(2 * size_t(G.q) * plane_bytes + 1024);
  const int n_e = h->bf16() ? 3 : 2;
  for (int k = 0; k < n_e; ++k) h->e[k] = static_cast<float*>(h->dev_alloc(size_t(g.plane) * 4));
  h->e_cur = 0;
  h->e_spare = 1;
  h->e_ref = h->bf16() ? 2 : -1;
  h->consts = static_cast<float*>(h->dev_alloc(size_t(11) * G.q * 4));
  h->mirror = static_cast<int16_t*>(h->dev_alloc(size_t(2) * G.q * 2));
  h->d_codes = static_cast<uint8_t*>(h->dev_alloc(size_t(kChunk) * G.q));
  h->d_order = static_cast<uint16_t*>(h->dev_alloc(size_t(kChunk) * (G.q + 17) * 2));
  h->d_red = static_cast<double*>(h->dev_alloc(8 * sizeof(double)));
  h->d_red_part = static_cast<double*>(
      h->dev_alloc(size_t(kReduceBlocks) * kReduceOut * sizeof(double)));
  h->d_snap = static_cast<double*>(h->dev_alloc(size_t(g.nx) * g.ny * sizeof(double)));
  h->d_status = static_cast<int*>(h->dev_alloc(256));
  if (h->planes)
    h->has_tmap = make_plane_tensor_map(h->tmap, h->planes, h->storage, g, 2 * G.q, &h->tmap_why);
  if (h->has_tmap) h->step_variant = 3;   // the fastest step kernel where it applies
  std::string why_w;
  if (h->has_tmap && h->bf16())
    h->has_tmap_w = make_word_tensor_map(h->tmap_w, h->planes, g, 2 * G.q, &why_w);
  h->bf16_wide = h->has_tmap_w ? 1 : 0;
  if (h->field_w) h->wfield = static_cast<float*>(h->dev_alloc(size_t(g.plane) * 4));
  if (!h->planes || !h->e[0] || !h->e[1] || (n_e == 3 && !h->e[2]) || !h->consts ||
      !h->d_codes || !h->d_order || !h->d_red || !h->d_red_part || !h->d_snap || !h->d_status ||
      !h->mirror ||
      (h->field_w && !h->wfield))
    return bad(WLBM_ERR_OOM, "wlbm_create: device allocation failed");

  std::vector<float> consts(size_t(11) * G.q);
  for (int i = 0; i < G.q; ++i) {
    consts[i] = float(h->lat.w[i]);
    consts[G.q + i] = float(h->lat.sx[i]);
    consts[2 * G.q + i] = float(h->lat.sy[i]);
  }
  const std::vector<float> rho = rho_tables(h->lat);
  std::memcpy(consts.data() + 3 * G.q, rho.data(), rho.size() * 4);
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(h->planes, 0, 2 * size_t(G.q) * plane_bytes + 1024, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, 256, s);
  for (int k = 0; k < n_e && e == cudaSuccess; ++k)
    e = cudaMemsetAsync(h->e[k], 0, size_t(g.plane) * 4, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->consts, consts.data(), consts.size() * 4, cudaMemcpyHostToDevice, s);
  const std::vector<int16_t> mirror = mirror_tables(h->lat);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->mirror, mirror.data(), mirror.size() * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h->field_w)
    e = cudaMemcpyAsync(h->wfield, wframe.data(), wframe.size() * 4, cudaMemcpyHostToDevice, s);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaHostAlloc(reinterpret_cast<void**>(&h->h_codes[k]), size_t(kChunk) * G.q,
                      cudaHostAllocDefault);
    if (e == cudaSuccess)
      e = cudaHostAlloc(reinterpret_cast<void**>(&h->h_order[k]),
                        size_t(kChunk) * (G.q + 17) * 2, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = prepare_step_kernels();
  if (e == cudaSuccess) e = configure_walls();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors die here
  if (e != cudaSuccess) {
    const std::string m = std::string("wlbm_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return bad(WLBM_ERR_CUDA, m);
  }
  h->build_wall_segments();
  *out = h;
  return WLBM_OK;
}

void wlbm_destroy(wlbm_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  h->release();
  delete h;
}

wlbm_status wlbm_set_stream(wlbm_handle* h, void* stream) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return WLBM_OK;
}

int64_t wlbm_step_count(const wlbm_handle* h) { return h ? h->tas.n : -1; }

wlbm_status wlbm_init_temperature(wlbm_handle* h, const float* dT) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (!dT) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_init_temperature: NULL dT");
  const Geom& g = h->g;
  h->scale = 1.f;
  if (h->storage == WLBM_STORE_BF16_DEV) {
    // per-run scale: the largest |e_eq(T) - e_ref| of the start field and the walls
    std::vector<float> host(size_t(g.nx) * g.ny);
    wlbm_status st = h->cuda(cudaMemcpyAsync(host.data(), dT, host.size() * 4,
                                             cudaMemcpyDeviceToHost, h->stream), "init");
    if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(h->stream), "init");
    if (st != WLBM_OK) return st;
    double m = 0.0;
    for (float v : host) m = std::max(m, std::fabs(h->delta_e(h->t_ref + double(v))));
    // values are stored relative to the local energy, so a fraction of the largest
    // deviation keeps them of order one
    for (int k = 0; k < 4; ++k)
      if (h->bc_kind[k] == WLBM_BC_ISOTHERMAL) m = std::max(m, std::fabs(h->delta_e(h->t_wall[k])));
    h->scale = m > 0 ? float(m) : 1.f;
  }
  h->inv_scale = 1.f / h->scale;
  h->build_wall_segments();
  h->drop_graphs();
  h->tas.reset(g.q);
  h->snap_step = -1;
  InitArgs a{};
  a.planes = h->planes; a.plane = g.plane; a.pitch = g.pitch; a.nx = g.nx; a.ny = g.ny; a.q = g.q;
  a.dT = dT; a.w = h->w_dev(); a.e_cur = h->e[h->e_cur]; a.e_refp = h->ref_plane();
  a.t_ref = h->t_ref; a.theta = h->theta; a.e_ref = h->e_eq_ref;
  a.scale = h->scale; a.inv_scale = h->inv_scale;
  ++h->launches;
  const wlbm_status st = h->cuda(launch_init(h->storage, a, h->stream), "wlbm_init_temperature");
  return st == WLBM_OK ? refresh_periodic(h) : st;
}

// Launch the kernels of `count` steps whose codes sit at d_codes[t][q], t < count.
// every > 0: an event pair around every every-th step-kernel launch (counted across calls;
// while capturing a graph, `cap` holds the graph's pairs and the steps t with t % every == 0
// of the chunk are timed)
static wlbm_status enqueue_steps(wlbm_handle* h, int count, int every,
                                 const std::vector<cudaEvent_t>* cap = nullptr) {
  size_t cap_used = 0;
  const Geom& g = h->g;
  const bool any_wall = h->walls.nseg > 0;
  // both axes periodic: the step kernel mirrors the edges itself (grids of 2+ cells)
  // (variant 3 has no mirror stores: there the separate periodic pass runs)
  // (sources must reach the ghost copies through the periodic pass: no mirrors with them)
  const bool wrap = h->fuse_periodic && h->step_variant != 3 && h->xper && h->yper &&
                    g.nx >= 2 && g.ny >= 2 && h->n_src == 0;
  const bool any_per = (h->xper || h->yper) && !wrap;
  wlbm_status st = WLBM_OK;
  for (int t = 0; t < count; ++t) {
    const uint8_t* codes = h->d_codes + size_t(t) * g.q;
    if (any_wall) {
      WallArgs wa = h->walls;
      wa.codes = codes;
      wa.e_ref = h->ref_plane();
      st = h->cuda(launch_walls(h->storage, wa, h->stream), "wlbm_step: walls");
      if (st != WLBM_OK) return st;
      ++h->launches;
    }
    if (h->n_src > 0) {
      SourceArgs ca{};
      ca.planes = h->planes; ca.plane = g.plane; ca.q = g.q; ca.n = h->n_src;
      ca.off = h->d_src_off; ca.val = h->d_src_val; ca.esum = h->d_src_e;
      ca.e_cur = h->e[h->e_cur]; ca.e_ref = h->ref_plane(); ca.w = h->w_dev();
      ca.codes = codes; ca.inv_scale = h->inv_scale;
      st = h->cuda(launch_sources(h->storage, ca, h->stream), "wlbm_step: sources");
      if (st != WLBM_OK) return st;
      ++h->launches;
    }
    if (any_per) {
      PeriodicArgs pa{};
      pa.planes = h->planes; pa.plane = g.plane; pa.pitch = g.pitch; pa.nx = g.nx;
      pa.ny = g.ny; pa.q = g.q; pa.codes = codes; pa.e_cur = h->e[h->e_cur];
      pa.e_ref = h->ref_plane();
      pa.xper = h->xper; pa.yper = h->yper;
      st = h->cuda(launch_periodic(h->storage, pa, h->stream), "wlbm_step: periodic");
      if (st != WLBM_OK) return st;
      ++h->launches;
    }
    StepArgs sa{};
    sa.planes = h->planes; sa.plane = g.plane; sa.pitch = g.pitch; sa.rows = g.rows;
    sa.nx = g.nx; sa.ny = g.ny; sa.q = g.q; sa.codes = codes; sa.w = h->w_dev();
    sa.e_in = h->e[h->e_cur]; sa.e_out = h->e[h->e_spare]; sa.e_ref = h->ref_plane();
    sa.wfield = h->field_w ? h->wfield : nullptr; sa.w0 = h->w0;
    sa.scale = h->scale; sa.inv_scale = h->inv_scale;
    sa.variant = h->step_variant; sa.status = h->d_status;
    sa.xper = h->xper; sa.yper = h->yper; sa.wrap = wrap;
    sa.tmap = h->has_tmap ? h->tmap : nullptr;
    sa.ring_stages = h->ring_stages;
    sa.loop_blocks = h->tile_loop ? h->loop_blocks : 0;
    sa.wide = h->bf16_wide;
    sa.tmap_w = h->has_tmap_w ? h->tmap_w : nullptr;
    sa.order = h->d_order + size_t(t) * (g.q + 17);
    int tx_unused = 0, ty_unused = 0;
    tma_cover(h->bc_kind, g.nx, g.ny, &sa, &tx_unused, &ty_unused);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (every > 0 && (cap ? t % every == 0 : h->prof_tick++ % every == 0)) {
      if (cap) {
        e0 = (*cap)[cap_used];
        e1 = (*cap)[cap_used + 1];
        cap_used += 2;
      } else {
        if (h->prof_used + 2 > h->prof_ev.size()) {
          for (int k = 0; k < 2; ++k) {
            cudaEvent_t ev;
            st = h->cuda(cudaEventCreate(&ev), "wlbm_step: profiling event");
            if (st != WLBM_OK) return st;
            h->prof_ev.push_back(ev);
          }
        }
        e0 = h->prof_ev[h->prof_used];
        e1 = h->prof_ev[h->prof_used + 1];
        h->prof_used += 2;
      }
      st = h->cuda(record_event(e0, h->stream, cap != nullptr), "wlbm_step: profiling");
      if (st != WLBM_OK) return st;
    }
    st = h->cuda(launch_step(h->storage, sa, h->stream), "wlbm_step: step");
    if (st != WLBM_OK) return st;
    ++h->launches;
    if (e1) {
      st = h->cuda(record_event(e1, h->stream, cap != nullptr), "wlbm_step: profiling");
      if (st != WLBM_OK) return st;
    }
    h->rotate_energy();
  }
  return WLBM_OK;
}

// Replay (capturing on first use) a CUDA graph of graph_steps steps.  The energy-plane
// roles return to the same state after a multiple of 6 steps, so one graph per starting
// role (and replay parity) serves every chunk.  While profiling, the graph times the steps
// t % prof_every == 0 of its chunk; the pairs of its previous replay, two chunks back, are
// read before it replays again.
static wlbm_status run_graph(wlbm_handle* h) {
  const int G = h->graph_steps;
  TimedGraph& tg = h->graphs[h->e_cur][h->graph_parity];
  h->graph_parity ^= 1;
  if (!tg.exec) {
    const int every = h->prof_every;
    wlbm_status st = h->cuda(tg.make_events(every > 0 ? (G + every - 1) / every : 0),
                             "wlbm_step: graph events");
    if (st != WLBM_OK) {
      tg.destroy();
      return st;
    }
    const int64_t launches0 = h->launches;
    st = h->cuda(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
                 "wlbm_step: graph capture");
    if (st != WLBM_OK) {
      tg.destroy();
      return st;
    }
    const wlbm_status est = enqueue_steps(h, G, every, &tg.ev);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (est != WLBM_OK) {
      if (graph) cudaGraphDestroy(graph);
      tg.destroy();
      return est;
    }
    st = h->cuda(ce, "wlbm_step: graph capture");
    if (st == WLBM_OK)
      st = h->cuda(cudaGraphInstantiate(&tg.exec, graph, 0), "wlbm_step: graph");
    if (graph) cudaGraphDestroy(graph);
    if (st != WLBM_OK) {
      tg.destroy();
      return st;
    }
    h->graph_launches = h->launches - launches0;
    h->launches = launches0;
  } else {
    const wlbm_status st =
        h->cuda(tg.harvest(&h->prof_graph_ms, &h->prof_graph_n), "wlbm_step: graph timing");
    if (st != WLBM_OK) return st;
  }
  h->launches += h->graph_launches;
  ++h->graph_replays;
  return h->cuda(tg.launch(h->stream), "wlbm_step: graph launch");
}

wlbm_status wlbm_step(wlbm_handle* h, int64_t n) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (n < 0) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_step: negative step count");
  const Geom& g = h->g;
  const bool graphs = h->graph_steps > 0 && h->stream != nullptr;
  while (n > 0) {
    const int ch = int(std::min<int64_t>(n, graphs ? h->graph_steps : kChunk));
    const int slot = h->slot;
    wlbm_status st = h->cuda(cudaEventSynchronize(h->ev[slot]), "wlbm_step");
    if (st != WLBM_OK) return st;
    uint8_t* hc = h->h_codes[slot];
    uint16_t* ho = h->h_order[slot];
    for (int t = 0; t < ch; ++t) {
      tas_advance(h->lat, &h->tas, hc + size_t(t) * g.q);
      sort_by_kind(hc + size_t(t) * g.q, g.q, ho + size_t(t) * (g.q + 17));
    }
    st = h->cuda(cudaMemcpyAsync(h->d_codes, hc, size_t(ch) * g.q, cudaMemcpyHostToDevice,
                                 h->stream), "wlbm_step: schedule upload");
    if (st == WLBM_OK)
      st = h->cuda(cudaMemcpyAsync(h->d_order, ho, size_t(ch) * (g.q + 17) * 2,
                                   cudaMemcpyHostToDevice, h->stream), "wlbm_step: order upload");
    if (st == WLBM_OK) st = h->cuda(cudaEventRecord(h->ev[slot], h->stream), "wlbm_step");
    if (st != WLBM_OK) return st;
    if (graphs && ch == h->graph_steps)
      st = run_graph(h);
    else
      st = enqueue_steps(h, ch, h->prof_every);
    if (st != WLBM_OK) return st;
    h->slot ^= 1;
    n -= ch;
  }
  return WLBM_OK;
}

wlbm_status wlbm_get_option(const wlbm_handle* h, int32_t key, int64_t* value) {
  if (!h || !value) return WLBM_ERR_INVALID_ARG;
  if (key == WLBM_OPT_STEP_VARIANT) *value = h->step_variant;
  else if (key == WLBM_OPT_GRAPH_STEPS) *value = h->graph_steps;
  else if (key == WLBM_OPT_FUSE_PERIODIC) *value = h->fuse_periodic;
  else if (key == WLBM_OPT_GRAPH_REPLAYS) *value = h->graph_replays;
  else if (key == WLBM_OPT_RING_STAGES) *value = h->ring_stages;
  else if (key == WLBM_OPT_TILE_LOOP) *value = h->tile_loop;
  else if (key == WLBM_OPT_BF16_WIDE) *value = h->bf16_wide;
  else return WLBM_ERR_INVALID_ARG;
  return WLBM_OK;
}

wlbm_status wlbm_set_option(wlbm_handle* h, int32_t key, int64_t value) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (key == WLBM_OPT_STEP_VARIANT && value == 3 && !h->has_tmap)
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_option: step variant 3 needs a tensor map of "
                                         "the planes: " + h->tmap_why);
  if (key == WLBM_OPT_STEP_VARIANT && value >= 0 && value <= 3) {
    h->step_variant = int(value);
    h->drop_graphs();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_GRAPH_STEPS && value >= 0 && value <= kChunk && value % 6 == 0) {
    h->graph_steps = int(value);
    h->drop_graphs();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_FUSE_PERIODIC && (value == 0 || value == 1)) {
    h->fuse_periodic = int(value);
    h->drop_graphs();
    return WLBM_OK;
  }
  if ((key == WLBM_OPT_RING_STAGES && step_tma_stages_ok(h->storage, int(value)) &&
       value >= 0 && value <= 64) ||
      (key == WLBM_OPT_TILE_LOOP && (value == 0 || value == 1))) {
    const int stages = key == WLBM_OPT_RING_STAGES ? int(value) : h->ring_stages;
    const int loop = key == WLBM_OPT_TILE_LOOP ? int(value) : h->tile_loop;
    int blocks = 0;
    if (loop) {
      blocks = step_tma_loop_blocks(h->storage, stages, h->field_w, h->g.q);
      if (blocks <= 0)
        return h->fail(WLBM_ERR_CUDA, "wlbm_set_option: occupancy of the tile-looping kernel");
    }
    h->ring_stages = stages;
    h->tile_loop = loop;
    h->loop_blocks = blocks;
    h->drop_graphs();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_BF16_WIDE && (value == 0 || value == 1)) {
    if (value == 1 && !h->has_tmap_w)
      return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_option: wide tiles need bfloat16 storage "
                                           "and a tensor map of the planes");
    h->bf16_wide = int(value);
    h->drop_graphs();
    return WLBM_OK;
  }
  return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_option: unknown key or value");
}

wlbm_status wlbm_check(wlbm_handle* h) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  int st = 0;
  wlbm_status r = h->cuda(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                          h->stream), "wlbm_check");
  if (r == WLBM_OK) r = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_check");
  if (r != WLBM_OK) return r;
  if (st != 0) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
    return h->fail(WLBM_ERR_TIMEOUT, "a bounded wait in the step kernel gave up");
  }
  return WLBM_OK;
}

wlbm_status wlbm_profile(wlbm_handle* h, int32_t every) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (every < 0) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_profile: negative stride");
  if (every != h->prof_every) h->drop_graphs();   // their event nodes follow the stride
  h->prof_every = every;
  h->prof_tick = 0;
  return WLBM_OK;
}

wlbm_status wlbm_profile_read(wlbm_handle* h, double* step_ms, int64_t* step_launches,
                              int64_t* all_launches) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  wlbm_status st = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_profile_read");
  if (st != WLBM_OK) return st;
  for (auto& role : h->graphs)
    for (TimedGraph& tg : role) {
      st = h->cuda(tg.harvest(&h->prof_graph_ms, &h->prof_graph_n), "wlbm_profile_read");
      if (st != WLBM_OK) return st;
    }
  double total = h->prof_graph_ms;
  for (size_t k = 0; k + 1 < h->prof_used; k += 2) {
    float ms = 0.f;
    st = h->cuda(cudaEventElapsedTime(&ms, h->prof_ev[k], h->prof_ev[k + 1]), "wlbm_profile_read");
    if (st != WLBM_OK) return st;
    total += ms;
  }
  if (step_ms) *step_ms = total;
  if (step_launches) *step_launches = h->prof_graph_n + int64_t(h->prof_used / 2);
  if (all_launches) *all_launches = h->launches;
  h->prof_used = 0;
  h->prof_graph_ms = 0.0;
  h->prof_graph_n = 0;
  return WLBM_OK;
}

static wlbm_status moments_impl(wlbm_handle* h, float* dT, float* qx, float* qy, float weight,
                                int accumulate) {
  const Geom& g = h->g;
  MomentArgs a{};
  a.planes = h->planes; a.plane = g.plane; a.pitch = g.pitch; a.nx = g.nx; a.ny = g.ny;
  a.q = g.q; a.par = h->parity_mask(); a.e_cur = h->e[h->e_cur]; a.e_refp = h->ref_plane();
  a.w = h->w_dev(); a.sx = h->sx_dev(); a.sy = h->sy_dev(); a.dT = dT; a.qx = qx; a.qy = qy;
  a.scale = h->scale;
  a.vg = float(h->lat.speed);
  a.e_ref = float(h->e_eq_ref);
  a.e_ref1 = float(h->e_eq_ref + 1.0);
  a.l_ref = float(std::log1p(1.0 / h->e_eq_ref));
  a.theta = float(h->theta);
  a.weight = weight;
  a.accumulate = accumulate;
  ++h->launches;
  return h->cuda(launch_moments(h->storage, a, h->stream), "wlbm_moments");
}

wlbm_status wlbm_moments(wlbm_handle* h, float* dT, float* qx, float* qy) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (!dT && !qx && !qy) return WLBM_OK;
  return moments_impl(h, dT, qx, qy, 1.f, 0);
}

wlbm_status wlbm_moments_mean(wlbm_handle* h, int32_t n, float* dT, float* qx, float* qy) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (n < 1) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_moments_mean: need n >= 1 steps");
  wlbm_status st = WLBM_OK;
  const float weight = 1.f / float(n);
  for (int32_t k = 0; k < n && st == WLBM_OK; ++k) {
    st = wlbm_step(h, 1);
    if (st == WLBM_OK && (dT || qx || qy)) st = moments_impl(h, dT, qx, qy, weight, k > 0);
  }
  return st;
}

// Derived outputs 6 and 7 of wlbm_reduce from outputs 2, 4 and 5.
static void reduce_conductivities(const wlbm_handle* h, double* out) {
  const double nan = std::numeric_limits<double>::quiet_NaN();
  // bulk diffusivity v_g Lambda / 3 (3D emulation) or / 2; defined for a uniform MFP only
  const double D =
      h->field_w ? nan : h->lat.speed * h->mfp_uniform / (h->emulate_3d ? 3.0 : 2.0);
  const bool iso_x = h->bc_kind[0] == WLBM_BC_ISOTHERMAL && h->bc_kind[1] == WLBM_BC_ISOTHERMAL &&
                     h->t_wall[0] != h->t_wall[1];
  out[6] = iso_x ? out[2] * h->g.nx / (D * (h->delta_e(h->t_wall[0]) - h->delta_e(h->t_wall[1])))
                 : nan;
  out[7] = out[5] != 0.0 ? out[4] / (-D * out[5]) : nan;
}

// Window control of one reduction inside wlbm_run_steady.
struct WindowCtl {
  bool first, last, has_prev;
  int32_t count;
};

static wlbm_status reduce_impl(wlbm_handle* h, double* out, const WindowCtl* win,
                               double* win_res) {
  const Geom& g = h->g;
  wlbm_status st = WLBM_OK;
  ReduceArgs a{};
  a.planes = h->planes; a.plane = g.plane; a.pitch = g.pitch; a.nx = g.nx; a.ny = g.ny;
  a.q = g.q; a.par = h->parity_mask(); a.e_cur = h->e[h->e_cur]; a.e_refp = h->ref_plane();
  a.w = h->w_dev(); a.sx = h->sx_dev(); a.sy = h->sy_dev(); a.out = h->d_red; a.scale = h->scale;
  a.part = h->d_red_part;
  a.diff_mask = 0;
  for (int k = 0; k < 4; ++k)
    if (h->bc_kind[k] == WLBM_BC_ADIABATIC_DIFFUSE) a.diff_mask |= 1 << k;
  a.band_x0 = g.nx / 4;
  a.band_w = g.nx / 2;
  a.band_xbar = a.band_x0 + 0.5 * (a.band_w - 1);
  a.snap = h->d_snap;
  a.has_snap = h->snap_step >= 0 ? 1 : 0;
  a.e_ref = h->e_eq_ref;
  a.e_ref1 = h->e_eq_ref + 1.0;
  a.l_ref = std::log1p(1.0 / h->e_eq_ref);
  a.theta = h->theta;
  if (win) {
    a.win = h->d_win;
    a.win_prev = h->d_win_prev;
    a.win_first = win->first ? 1 : 0;
    a.win_last = win->last ? 1 : 0;
    a.win_has_prev = win->has_prev ? 1 : 0;
    a.win_inv = 1.0 / win->count;
  }
  h->launches += 2;
  st = h->cuda(launch_reduce(h->storage, a, h->stream), "wlbm_reduce");
  double tmp[kReduceOut];
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(tmp, h->d_red, sizeof(tmp), cudaMemcpyDeviceToHost, h->stream),
                 "wlbm_reduce");
  if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_reduce");
  if (st != WLBM_OK) return st;
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const double cells = double(g.nx) * g.ny;
  const double bw = a.band_w;
  const double vg = h->lat.speed;        // Eq. q_corr: q = v_g sum_i e_i s_i
  out[0] = tmp[0];
  out[1] = tmp[1];
  out[2] = vg * tmp[2] / cells;
  out[3] = vg * tmp[3] / cells;
  out[4] = a.band_w >= 1 ? vg * tmp[4] / (bw * g.ny) : nan;
  // least-squares slope of the y-averaged E over the band: sum (x - xbar)^2 = w (w^2 - 1) / 12
  out[5] = a.band_w >= 2 ? tmp[5] / (double(g.ny) * bw * (bw * bw - 1.0) / 12.0) : nan;
  reduce_conductivities(h, out);
  double rmax;
  std::memcpy(&rmax, &tmp[6], sizeof(rmax));
  const int64_t n = h->tas.n;
  out[8] = h->snap_step >= 0 && n > h->snap_step ? rmax / double(n - h->snap_step) : nan;
  h->snap_step = n;
  if (win_res) std::memcpy(win_res, &tmp[7], sizeof(double));
  return WLBM_OK;
}

wlbm_status wlbm_reduce(wlbm_handle* h, double* out) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (!out) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_reduce: NULL output");
  return reduce_impl(h, out, nullptr, nullptr);
}

wlbm_status wlbm_run_steady(wlbm_handle* h, int64_t max_steps, int64_t check_every, double tol,
                            int32_t avg_steps, int64_t* steps_run, int32_t* converged,
                            double* out) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (avg_steps < 1 || check_every < avg_steps || max_steps < check_every || !(tol >= 0.0))
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_run_steady: need max_steps >= check_every >= "
                                         "avg_steps >= 1 and tol >= 0");
  const size_t cells = size_t(h->g.nx) * h->g.ny;
  if (!h->d_win) h->d_win = static_cast<double*>(h->dev_alloc(cells * sizeof(double)));
  if (!h->d_win_prev) h->d_win_prev = static_cast<double*>(h->dev_alloc(cells * sizeof(double)));
  if (!h->d_win || !h->d_win_prev)
    return h->fail(WLBM_ERR_OOM, "wlbm_run_steady: device allocation failed");
  double r[WLBM_REDUCE_N];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  double residual = std::numeric_limits<double>::quiet_NaN();
  int64_t done = 0;
  int32_t conv = 0;
  bool has_prev = false;
  wlbm_status st = WLBM_OK;
  while (st == WLBM_OK && done + check_every <= max_steps && !conv) {
    st = wlbm_step(h, check_every - avg_steps);
    for (int k = 0; k < 4; ++k) acc[k] = 0.0;
    double wres = 0.0;
    for (int32_t t = 0; t < avg_steps && st == WLBM_OK; ++t) {
      st = wlbm_step(h, 1);
      const WindowCtl w{t == 0, t == avg_steps - 1, has_prev, avg_steps};
      if (st == WLBM_OK) st = reduce_impl(h, r, &w, &wres);
      if (st == WLBM_OK)
        for (int k = 0; k < 4; ++k) acc[k] += r[2 + k];
    }
    if (st != WLBM_OK) break;
    done += check_every;
    // window centres are check_every steps apart
    residual = has_prev ? wres / double(check_every) : std::numeric_limits<double>::quiet_NaN();
    has_prev = true;
    conv = residual <= tol ? 1 : 0;
  }
  if (steps_run) *steps_run = done;
  if (converged) *converged = conv;
  if (st != WLBM_OK) return st;
  for (int k = 0; k < 4; ++k) r[2 + k] = acc[k] / avg_steps;
  reduce_conductivities(h, r);
  r[8] = residual;
  if (out) std::memcpy(out, r, sizeof(r));
  return WLBM_OK;
}

static StateArgs state_args(wlbm_handle* h, float* framed) {
  const Geom& g = h->g;
  StateArgs a{};
  a.planes = h->planes; a.plane = g.plane; a.pitch = g.pitch; a.nx = g.nx; a.ny = g.ny;
  a.q = g.q; a.par = h->parity_mask(); a.framed = framed; a.e_cur = h->e[h->e_cur];
  a.e_refp = h->ref_plane(); a.w = h->w_dev();
  a.scale = h->scale; a.inv_scale = h->inv_scale;
  return a;
}

wlbm_status wlbm_get_state(wlbm_handle* h, float* framed) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (!framed) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_get_state: NULL output");
  return h->cuda(launch_get_state(h->storage, state_args(h, framed), h->stream), "wlbm_get_state");
}

wlbm_status wlbm_set_state(wlbm_handle* h, const float* framed) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (!framed) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_state: NULL input");
  h->snap_step = -1;
  const wlbm_status st = h->cuda(
      launch_set_state(h->storage, state_args(h, const_cast<float*>(framed)), h->stream),
      "wlbm_set_state");
  return st == WLBM_OK ? refresh_periodic(h) : st;
}

wlbm_status wlbm_set_sources(wlbm_handle* h, int32_t n, const int32_t* xy, const double* t,
                             const double* e_imposed) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (h->batch_owned)
    return h->fail(WLBM_ERR_STATE, "wlbm_set_sources: handles owned by a batch are not supported");
  if (n < 0 || (n > 0 && (!xy || (!t && !e_imposed))))
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_sources: need cells and temperatures or "
                                         "imposed values");
  const Geom& g = h->g;
  const size_t ns = static_cast<size_t>(n);
  std::vector<int64_t> off(ns);
  std::vector<float> val(ns * g.q), esum(ns);
  for (int k = 0; k < n; ++k) {
    const int x = xy[2 * k], y = xy[2 * k + 1];
    if (x < -1 || x > g.nx || y < -1 || y > g.ny)
      return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_sources: cell outside the frame");
    const bool per = ((x == -1 || x == g.nx) && h->xper) || ((y == -1 || y == g.ny) && h->yper);
    if (per)
      return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_sources: cell on a periodic ghost frame");
    off[size_t(k)] = int64_t(y + 2) * g.pitch + (kX0 + x);
    double sum = 0.0;
    for (int i = 0; i < g.q; ++i) {
      double d;
      if (e_imposed) {
        d = e_imposed[size_t(k) * g.q + i] - h->lat.w[i] * h->e_eq_ref;
      } else {
        if (!(t[k] > 0))
          return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_set_sources: temperatures must be > 0");
        d = h->lat.w[i] * h->delta_e(t[k]);
      }
      val[size_t(k) * g.q + i] = float(d);
      sum += double(float(d));
    }
    esum[size_t(k)] = float(sum);
  }
  for (void* p : {static_cast<void*>(h->d_src_off), static_cast<void*>(h->d_src_val),
                  static_cast<void*>(h->d_src_e)})
    if (p) h->dev_free(p);
  h->d_src_off = nullptr; h->d_src_val = nullptr; h->d_src_e = nullptr;
  h->n_src = 0;
  h->drop_graphs();
  if (n == 0) return WLBM_OK;
  h->d_src_off = static_cast<int64_t*>(h->dev_alloc(off.size() * 8));
  h->d_src_val = static_cast<float*>(h->dev_alloc(val.size() * 4));
  h->d_src_e = static_cast<float*>(h->dev_alloc(esum.size() * 4));
  if (!h->d_src_off || !h->d_src_val || !h->d_src_e)
    return h->fail(WLBM_ERR_OOM, "wlbm_set_sources: device allocation failed");
  wlbm_status st = h->cuda(cudaMemcpyAsync(h->d_src_off, off.data(), off.size() * 8,
                                           cudaMemcpyHostToDevice, h->stream), "wlbm_set_sources");
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(h->d_src_val, val.data(), val.size() * 4,
                                 cudaMemcpyHostToDevice, h->stream), "wlbm_set_sources");
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(h->d_src_e, esum.data(), esum.size() * 4,
                                 cudaMemcpyHostToDevice, h->stream), "wlbm_set_sources");
  if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_set_sources");
  if (st == WLBM_OK) h->n_src = n;
  return st;
}

// ---------------------------------------------------------------- checkpoint / resume
// Blob: CkptHeader, the schedule cursor (px, py, h as int64[q] each, parity as uint8[q]
// padded to 8 bytes), the q current state planes as stored (framed, pitch included), the
// current local-energy plane and, with bfloat16 storage, the reference-energy plane.
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, nx, ny, q, storage, pitch;
  int32_t bc_kind[4];
  int32_t e_cur, e_ref, e_spare, n_energy;
  int64_t n, plane_bytes, energy_bytes, total;
  float scale, inv_scale;
};
constexpr char kCkptMagic[8] = {'W', 'L', 'B', 'M', 'C', 'K', 'P', 'T'};
constexpr int32_t kCkptVersion = 1;

size_t ckpt_cursor_bytes(int q) { return size_t(q) * 24 + ((size_t(q) + 7) & ~size_t(7)); }
}  // namespace

static size_t ckpt_size(const wlbm_handle* h) {
  const Geom& g = h->g;
  const size_t plane_bytes = size_t(g.plane) * h->elem();
  const size_t energy_bytes = size_t(g.plane) * 4;
  return sizeof(CkptHeader) + ckpt_cursor_bytes(g.q) + size_t(g.q) * plane_bytes +
         (h->e_ref >= 0 ? 2 : 1) * energy_bytes;
}

wlbm_status wlbm_save(wlbm_handle* h, void* dst, size_t capacity, size_t* written) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  const size_t total = ckpt_size(h);
  if (written) *written = total;
  if (!dst) return WLBM_OK;
  if (capacity < total) return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_save: buffer too small");
  const Geom& g = h->g;
  CkptHeader hd{};
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.nx = g.nx; hd.ny = g.ny; hd.q = g.q; hd.storage = h->storage; hd.pitch = g.pitch;
  for (int k = 0; k < 4; ++k) hd.bc_kind[k] = h->bc_kind[k];
  hd.e_cur = h->e_cur; hd.e_ref = h->e_ref; hd.e_spare = h->e_spare;
  hd.n_energy = h->e_ref >= 0 ? 2 : 1;
  hd.n = h->tas.n;
  hd.plane_bytes = int64_t(g.plane) * int64_t(h->elem());
  hd.energy_bytes = int64_t(g.plane) * 4;
  hd.total = int64_t(total);
  hd.scale = h->scale; hd.inv_scale = h->inv_scale;
  unsigned char* out = static_cast<unsigned char*>(dst);
  std::memcpy(out, &hd, sizeof(hd));
  unsigned char* cur = out + sizeof(hd);
  std::memcpy(cur, h->tas.px.data(), size_t(g.q) * 8);
  std::memcpy(cur + size_t(g.q) * 8, h->tas.py.data(), size_t(g.q) * 8);
  std::memcpy(cur + size_t(g.q) * 16, h->tas.h.data(), size_t(g.q) * 8);
  std::memset(cur + size_t(g.q) * 24, 0, ckpt_cursor_bytes(g.q) - size_t(g.q) * 24);
  std::memcpy(cur + size_t(g.q) * 24, h->tas.parity.data(), size_t(g.q));
  unsigned char* p = cur + ckpt_cursor_bytes(g.q);
  const unsigned char* planes = static_cast<const unsigned char*>(h->planes);
  wlbm_status st = WLBM_OK;
  for (int i = 0; i < g.q && st == WLBM_OK; ++i) {
    const size_t src = (size_t(h->tas.parity[i]) * g.q + i) * size_t(hd.plane_bytes);
    st = h->cuda(cudaMemcpyAsync(p, planes + src, size_t(hd.plane_bytes), cudaMemcpyDeviceToHost,
                                 h->stream), "wlbm_save");
    p += hd.plane_bytes;
  }
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(p, h->e[h->e_cur], size_t(hd.energy_bytes),
                                 cudaMemcpyDeviceToHost, h->stream), "wlbm_save");
  p += hd.energy_bytes;
  if (st == WLBM_OK && h->e_ref >= 0)
    st = h->cuda(cudaMemcpyAsync(p, h->e[h->e_ref], size_t(hd.energy_bytes),
                                 cudaMemcpyDeviceToHost, h->stream), "wlbm_save");
  if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_save");
  return st;
}

wlbm_status wlbm_load(wlbm_handle* h, const void* src, size_t size) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (h->batch_owned)
    return h->fail(WLBM_ERR_STATE, "wlbm_load: handles owned by a batch are not supported");
  if (!src || size < sizeof(CkptHeader))
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_load: NULL or truncated checkpoint");
  const Geom& g = h->g;
  CkptHeader hd;
  std::memcpy(&hd, src, sizeof(hd));
  bool same_walls = true;
  for (int k = 0; k < 4; ++k) same_walls = same_walls && hd.bc_kind[k] == h->bc_kind[k];
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion)
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_load: not a checkpoint of this library version");
  if (hd.nx != g.nx || hd.ny != g.ny || hd.q != g.q || hd.storage != h->storage ||
      hd.pitch != g.pitch || !same_walls)
    return h->fail(WLBM_ERR_INVALID_ARG,
                   "wlbm_load: checkpoint of another grid, Q, storage or wall set");
  if (hd.total != int64_t(ckpt_size(h)) || size < ckpt_size(h) || hd.n < 0 ||
      hd.n_energy != (h->e_ref >= 0 ? 2 : 1))
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_load: checkpoint size does not match");
  const int n_e = h->bf16() ? 3 : 2;
  const bool roles_ok = hd.e_cur >= 0 && hd.e_cur < n_e && hd.e_spare >= 0 && hd.e_spare < n_e &&
                        hd.e_cur != hd.e_spare &&
                        (h->bf16() ? (hd.e_ref >= 0 && hd.e_ref < n_e && hd.e_ref != hd.e_cur &&
                                      hd.e_ref != hd.e_spare)
                                   : hd.e_ref == -1);
  const unsigned char* in = static_cast<const unsigned char*>(src) + sizeof(hd);
  const uint8_t* parity = in + size_t(g.q) * 24;
  bool parity_ok = true;
  for (int i = 0; i < g.q; ++i) parity_ok = parity_ok && parity[i] <= 1;
  if (!roles_ok || !parity_ok || !(hd.scale > 0.f))
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_load: corrupt checkpoint header");
  h->tas.reset(g.q);
  h->tas.n = hd.n;
  std::memcpy(h->tas.px.data(), in, size_t(g.q) * 8);
  std::memcpy(h->tas.py.data(), in + size_t(g.q) * 8, size_t(g.q) * 8);
  std::memcpy(h->tas.h.data(), in + size_t(g.q) * 16, size_t(g.q) * 8);
  std::memcpy(h->tas.parity.data(), parity, size_t(g.q));
  h->e_cur = hd.e_cur; h->e_ref = hd.e_ref; h->e_spare = hd.e_spare;
  h->scale = hd.scale; h->inv_scale = hd.inv_scale;
  h->build_wall_segments();
  h->drop_graphs();
  h->snap_step = -1;
  h->adj.ready = false;
  const unsigned char* p = in + ckpt_cursor_bytes(g.q);
  unsigned char* planes = static_cast<unsigned char*>(h->planes);
  // Only the frame of each plane (rows 1 .. ny + 2, columns kGhostCol .. kX0 + nx) is
  // copied: the pads stay zero whatever the buffer holds there (the kernels that read a
  // pad from memory, instead of a tensor copy's zero fill, rely on that).
  auto copy_frame = [&](void* dst, const unsigned char* src, size_t elem) {
    const size_t pitch = size_t(g.pitch) * elem, off = pitch + size_t(kGhostCol) * elem;
    return h->cuda(cudaMemcpy2DAsync(static_cast<unsigned char*>(dst) + off, pitch, src + off,
                                     pitch, size_t(g.nx + 2) * elem, size_t(g.ny + 2),
                                     cudaMemcpyHostToDevice, h->stream),
                   "wlbm_load");
  };
  wlbm_status st = WLBM_OK;
  for (int i = 0; i < g.q && st == WLBM_OK; ++i) {
    const size_t dst = (size_t(h->tas.parity[i]) * g.q + i) * size_t(hd.plane_bytes);
    st = copy_frame(planes + dst, p, h->elem());
    p += hd.plane_bytes;
  }
  if (st == WLBM_OK) st = copy_frame(h->e[h->e_cur], p, 4);
  p += hd.energy_bytes;
  if (st == WLBM_OK && h->e_ref >= 0) st = copy_frame(h->e[h->e_ref], p, 4);
  if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(h->stream), "wlbm_load");
  return st;
}


// ------------------------------------------------------------------------- adjoint
static wlbm_status adj_alloc(wlbm_handle* h, int64_t n, int k) {
  auto& A = h->adj;
  for (void* p : A.bufs) h->dev_free(p);
  A.bufs.clear();
  A = wlbm_handle::Adj{};
  const Geom& g = h->g;
  const size_t state = size_t(g.q) * size_t(g.plane) * 4;
  const size_t cells = size_t(g.nx) * g.ny * 4;
  const int nck = int((n + k - 1) / k);
  auto get = [&](size_t bytes) {
    void* p = h->dev_alloc(bytes);
    if (p) A.bufs.push_back(p);
    return p;
  };
  A.ckpt = static_cast<float*>(get(size_t(nck) * state));
  A.ckpt_e = static_cast<float*>(get(size_t(nck) * size_t(g.plane) * 4));
  // The tape and the adjoint planes start 16 and 32 bytes into their allocations, so that
  // the reverse step's tape boxes (from the first tile column, 4 columns left of the
  // interior) and adjoint boxes (4 columns further left) begin on 128-byte lines (measured
  // DRAM reads of one reverse step at 1024^2 x Q64: 595 MB unshifted, 586 MB with both
  // shifted by 16 bytes, 578 MB with these shifts).
  constexpr int kTapeShift = 4, kLamShift = 8;   // floats
  float* tape_raw = static_cast<float*>(get(size_t(k) * state + 1024));
  A.tape = tape_raw ? tape_raw + kTapeShift : nullptr;
  // slack after the adjoint planes: the reverse step's shifted 16-byte row reads of the
  // last tile may run a few elements past the last row
  for (int b = 0; b < 2; ++b) {
    float* raw = static_cast<float*>(get(state + 1024));
    A.lam[b] = raw ? raw + kLamShift : nullptr;
  }
  A.sh[0] = static_cast<float*>(get(size_t(g.plane) * 4));
  A.sh[1] = static_cast<float*>(get(size_t(g.plane) * 4));
  A.erec[0] = static_cast<float*>(get(size_t(g.plane) * 4));
  A.erec[1] = static_cast<float*>(get(size_t(g.plane) * 4));
  A.gw = static_cast<float*>(get(size_t(g.plane) * 4));
  A.dwc = static_cast<float*>(get(cells));
  A.dT0 = static_cast<float*>(get(cells));
  A.gtw = static_cast<double*>(get(4 * sizeof(double)));
  A.codes = static_cast<uint8_t*>(get(size_t(n) * g.q));
  A.order = static_cast<uint16_t*>(get(size_t(n) * (g.q + 17) * 2));
  if (!A.ckpt || !A.ckpt_e || !A.tape || !A.lam[0] || !A.lam[1] || !A.sh[0] || !A.sh[1] ||
      !A.erec[0] || !A.erec[1] ||
      !A.gw || !A.dwc || !A.dT0 || !A.gtw || !A.codes || !A.order)
    return h->fail(WLBM_ERR_OOM, "wlbm_adjoint_forward: device allocation failed");
  A.n = n;
  A.k = k;
  A.nck = nck;
  std::string why;
  A.has_tape_tmap = make_plane_tensor_map(A.tape_tmap, A.tape, WLBM_STORE_FP32_DEV, g, k * g.q,
                                          &why);
  A.has_lam_tmap = true;
  for (int b = 0; b < 2; ++b)
    A.has_lam_tmap = A.has_lam_tmap &&
                     make_box_tensor_map(A.lam_tmap[b], A.lam[b], WLBM_STORE_FP32_DEV, g, g.q,
                                         kAdjTmaBoxRows, &why) &&
                     make_box_tensor_map(A.lam14_tmap[b], A.lam[b], WLBM_STORE_FP32_DEV, g, g.q,
                                         kAdjTmaRows, &why);
  A.has_lam_tmap = A.has_lam_tmap &&
                   make_box_tensor_map(A.tape_adj_tmap, A.tape, WLBM_STORE_FP32_DEV, g, k * g.q,
                                       kAdjTmaRows, &why, kAdjTmaCols);
  // tape slots and energy planes: pads must read zero
  cudaError_t e = cudaMemsetAsync(tape_raw, 0, size_t(k) * state + 1024, h->stream);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j)
    e = cudaMemsetAsync(A.erec[j], 0, size_t(g.plane) * 4, h->stream);
  return h->cuda(e, "wlbm_adjoint_forward");
}

wlbm_status wlbm_adjoint_forward(wlbm_handle* h, const float* dT0, int64_t n_steps,
                                 int32_t ckpt_every) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  if (h->bf16())
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_adjoint_forward: needs float32 storage");
  if (h->n_src > 0)
    return h->fail(WLBM_ERR_STATE, "wlbm_adjoint_forward: internal sources are not supported");
  if (!dT0 || n_steps < 1 || ckpt_every < 1)
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_adjoint_forward: bad start field or counts");
  const Geom& g = h->g;
  auto& A = h->adj;
  wlbm_status st = WLBM_OK;
  if (!(A.n == n_steps && A.k == ckpt_every && A.ckpt)) st = adj_alloc(h, n_steps, ckpt_every);
  if (st != WLBM_OK) return st;
  A.ready = false;
  // dW_corr/dMFP per interior cell (Eq. W-correction with W = v/MFP: a function of
  // m = MFP/v, so dW_corr/dMFP = (dW_corr/dm) / v)
  std::vector<float> dwc(size_t(g.nx) * g.ny);
  const double f = h->emulate_3d ? 1.5 : 1.0, lc = h->lat.lam_corr, v = h->lat.speed;
  for (size_t c = 0; c < dwc.size(); ++c) {
    const double m = (h->field_w ? double(h->mfp_host[c]) : h->mfp_uniform) / v;
    if (std::isinf(m)) { dwc[c] = 0.f; continue; }
    const double W = 1.0 / m;
    double d = -f * (1.0 + 2.0 * W * (lc - 1.0)) / (m * m);
    if (h->relax_mode == 1) d *= std::exp(-f * (W + W * W * (lc - 1.0)));
    dwc[c] = float(d / v);
  }
  std::vector<uint8_t> codes(size_t(n_steps) * g.q);
  std::vector<uint16_t> order(size_t(n_steps) * (g.q + 17));
  TasState ts;
  ts.reset(g.q);
  for (int64_t t = 0; t < n_steps; ++t) {
    tas_advance(h->lat, &ts, codes.data() + t * g.q);
    sort_by_kind(codes.data() + t * g.q, g.q, order.data() + t * (g.q + 17));
  }
  cudaStream_t s = h->stream;
  st = h->cuda(cudaMemcpyAsync(A.dwc, dwc.data(), dwc.size() * 4, cudaMemcpyHostToDevice, s),
               "wlbm_adjoint_forward");
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(A.codes, codes.data(), codes.size(), cudaMemcpyHostToDevice, s),
                 "wlbm_adjoint_forward");
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(A.order, order.data(), order.size() * 2, cudaMemcpyHostToDevice,
                                 s), "wlbm_adjoint_forward");
  if (st == WLBM_OK)
    st = h->cuda(cudaMemcpyAsync(A.dT0, dT0, size_t(g.nx) * g.ny * 4, cudaMemcpyDeviceToDevice, s),
                 "wlbm_adjoint_forward");
  if (st == WLBM_OK) st = wlbm_init_temperature(h, dT0);
  for (int c = 0; c < A.nck && st == WLBM_OK; ++c) {
    // checkpoint: the state before the boundary pass of step c*k + 1, gathered by parity
    for (int i = 0; i < g.q && st == WLBM_OK; ++i) {
      const float* src = static_cast<const float*>(h->planes) +
                         (size_t(h->tas.parity[i]) * g.q + i) * size_t(g.plane);
      st = h->cuda(cudaMemcpyAsync(A.ckpt + (size_t(c) * g.q + i) * g.plane, src,
                                   size_t(g.plane) * 4, cudaMemcpyDeviceToDevice, s),
                   "wlbm_adjoint_forward: checkpoint");
    }
    if (st == WLBM_OK)
      st = h->cuda(cudaMemcpyAsync(A.ckpt_e + size_t(c) * g.plane, h->e[h->e_cur],
                                   size_t(g.plane) * 4, cudaMemcpyDeviceToDevice, s),
                   "wlbm_adjoint_forward: checkpoint");
    if (st == WLBM_OK) st = wlbm_step(h, std::min<int64_t>(A.k, n_steps - int64_t(c) * A.k));
  }
  if (st == WLBM_OK) st = h->cuda(cudaStreamSynchronize(s), "wlbm_adjoint_forward");
  if (st == WLBM_OK) A.ready = true;
  return st;
}

wlbm_status wlbm_adjoint_backward(wlbm_handle* h, const float* dJ_dT, const float* dJ_dqx,
                                  const float* dJ_dqy, float* dJ_dmfp,
                                  double* dJ_dTwall, float* dJ_ddT0) {
  if (!h) return WLBM_ERR_INVALID_ARG;
  auto& A = h->adj;
  if (!A.ready || h->tas.n != A.n)
    return h->fail(WLBM_ERR_STATE, "wlbm_adjoint_backward: no checkpointed forward run ends "
                                   "at the current state");
  if (!dJ_dT && !dJ_dqx && !dJ_dqy)
    return h->fail(WLBM_ERR_INVALID_ARG, "wlbm_adjoint_backward: no seed (dJ_dT, dJ_dqx, dJ_dqy)");
  h->snap_step = -1;   // the sweep reuses the state buffers
  const Geom& g = h->g;
  cudaStream_t s = h->stream;
  const size_t state = size_t(g.q) * size_t(g.plane);
  wlbm_status st = WLBM_OK;
  auto ok = [&](cudaError_t e, const char* what) {
    if (st == WLBM_OK) st = h->cuda(e, what);
    return st == WLBM_OK;
  };
  ok(cudaMemsetAsync(A.lam[0], 0, state * 4, s), "adjoint");
  ok(cudaMemsetAsync(A.lam[1], 0, state * 4, s), "adjoint");
  ok(cudaMemsetAsync(A.sh[0], 0, size_t(g.plane) * 4, s), "adjoint");   // pads stay zero
  ok(cudaMemsetAsync(A.sh[1], 0, size_t(g.plane) * 4, s), "adjoint");
  ok(cudaMemsetAsync(A.gw, 0, size_t(g.plane) * 4, s), "adjoint");
  ok(cudaMemsetAsync(A.gtw, 0, 4 * sizeof(double), s), "adjoint");
  AdjArgs aa{};
  aa.w = h->w_dev(); aa.wfield = h->field_w ? h->wfield : nullptr; aa.w0 = h->w0;
  aa.xper = h->xper; aa.yper = h->yper; aa.gw = A.gw;
  aa.nx = g.nx; aa.ny = g.ny; aa.q = g.q; aa.pitch = g.pitch; aa.plane = g.plane;
  aa.gtw = A.gtw;
  // isothermal wall cells, by side and corner, from the wall segments
  for (int k = 0; k < 4; ++k) aa.iso_side[k] = aa.iso_corner[k] = -1;
  for (int k = 0; k < h->walls.nseg; ++k) {
    const WallSeg& sg = h->walls.seg[k];
    if (sg.action != WLBM_BC_ISOTHERMAL) continue;
    const bool right = sg.c0 == kX0 + g.nx, top = sg.r0 == g.ny + 2;
    if (sg.count == 1 && sg.dr == 0 && sg.dc == 0)
      aa.iso_corner[(top ? 2 : 0) + (right ? 1 : 0)] = sg.wall;
    else if (sg.dr != 0)
      aa.iso_side[right ? 1 : 0] = sg.wall;
    else aa.iso_side[top ? 3 : 2] = sg.wall;
  }
  aa.lam_out = A.lam[0];
  ok(launch_adj_seed(aa, dJ_dT, dJ_dqx, dJ_dqy, h->sx_dev(), h->sy_dev(), float(h->lat.speed),
                     h->e[h->e_cur], h->e_eq_ref, h->theta, s),
     "adjoint: seed");
  int cur = 0;
  for (int c = A.nck - 1; c >= 0 && st == WLBM_OK; --c) {
    const int64_t s0 = int64_t(c) * A.k;
    const int kc = int(std::min<int64_t>(A.k, A.n - s0));
    // recompute the segment: tape slot j = input of step s0 + j + 1 (after the boundary pass)
    ok(cudaMemcpyAsync(A.tape, A.ckpt + size_t(c) * state, state * 4, cudaMemcpyDeviceToDevice, s),
       "adjoint: restore");
    ok(cudaMemcpyAsync(A.erec[0], A.ckpt_e + size_t(c) * g.plane, size_t(g.plane) * 4,
                       cudaMemcpyDeviceToDevice, s), "adjoint: restore");
    int ec = 0;
    for (int j = 0; j < kc && st == WLBM_OK; ++j) {
      const uint8_t* codes = A.codes + size_t(s0 + j) * g.q;
      float* slot = A.tape + size_t(j) * state;
      if (h->walls.nseg > 0) {
        WallArgs wa = h->walls;
        wa.planes = slot; wa.codes = codes; wa.tape = 1; wa.e_ref = nullptr;
        ok(launch_walls(h->storage, wa, s), "adjoint: walls");
      }
      if (h->xper || h->yper) {
        PeriodicArgs pa{};
        pa.planes = slot; pa.plane = g.plane; pa.pitch = g.pitch; pa.nx = g.nx; pa.ny = g.ny;
        pa.q = g.q; pa.codes = codes; pa.e_cur = A.erec[ec]; pa.e_ref = nullptr;
        pa.xper = h->xper; pa.yper = h->yper; pa.tape = 1;
        ok(launch_periodic(h->storage, pa, s), "adjoint: periodic");
      }
      if (j + 1 < kc) {
        StepArgs sa{};
        sa.planes = slot; sa.plane = g.plane; sa.pitch = g.pitch; sa.rows = g.rows;
        sa.nx = g.nx; sa.ny = g.ny; sa.q = g.q; sa.codes = codes; sa.w = h->w_dev();
        sa.e_in = A.erec[ec]; sa.e_out = A.erec[ec ^ 1]; sa.e_ref = nullptr;
        sa.wfield = h->field_w ? h->wfield : nullptr; sa.w0 = h->w0;
        sa.scale = 1.f; sa.inv_scale = 1.f; sa.xper = h->xper; sa.yper = h->yper;
        sa.variant = h->step_variant; sa.status = h->d_status;
        sa.tape = 1; sa.tape_dst = slot + state;
        sa.wrap = h->xper && h->yper && g.nx >= 2 && g.ny >= 2;
        if (h->step_variant == 3 && A.has_tape_tmap) {   // TMA tiles read the tape's slots
          sa.wrap = 0;                                     // (the periodic pass ran above)
          sa.tmap = A.tape_tmap;
          sa.order = A.order + size_t(s0 + j) * (g.q + 17);
          sa.tape_z0 = j * g.q;
          int tx_unused = 0, ty_unused = 0;
          tma_cover(h->bc_kind, g.nx, g.ny, &sa, &tx_unused, &ty_unused);
        }
        ok(launch_step(h->storage, sa, s), "adjoint: recompute");
        ec ^= 1;
      }
    }
    // reverse sweep over the segment
    for (int j = kc - 1; j >= 0 && st == WLBM_OK; --j) {
      aa.lam_in = A.lam[cur];
      aa.lam_out = A.lam[cur ^ 1];
      aa.s_in = A.sh[cur];
      aa.s_out = A.sh[cur ^ 1];
      aa.dtil = A.tape + size_t(j) * state;
      aa.codes = A.codes + size_t(s0 + j) * g.q;
      if (h->step_variant == 3 && A.has_tape_tmap && A.has_lam_tmap)
        ok(launch_adj_tma(aa, A.lam_tmap[cur], A.lam14_tmap[cur], A.tape_adj_tmap, j * g.q,
                          A.order + size_t(s0 + j) * (g.q + 17), h->d_status, s),
           "adjoint: reverse step");
      else
        ok(launch_adj_step(aa, s), "adjoint: reverse step");
      // the periodic transpose is the same on every direction: it acts on lh and on s
      ok(launch_periodic_T(A.lam[cur ^ 1], g.plane, g.pitch, g.nx, g.ny, g.q, h->xper, h->yper, s),
         "adjoint: periodic transpose");
      ok(launch_periodic_T(A.sh[cur ^ 1], g.plane, g.pitch, g.nx, g.ny, 1, h->xper, h->yper, s),
         "adjoint: periodic transpose");
      // s is zero on wall ghost cells (W = 0 there), so the wall transpose sees l = lh
      if (h->walls.nseg > 0) {
        WallArgs wa = h->walls;
        wa.codes = aa.codes;
        ok(launch_walls_T(wa, A.lam[cur ^ 1], A.gtw, s), "adjoint: wall transpose");
      }
      cur ^= 1;
    }
  }
  // periodic ghosts of W_corr copy interior cells: send their gradient back
  ok(launch_periodic_T(A.gw, g.plane, g.pitch, g.nx, g.ny, 1, h->xper, h->yper, s),
     "adjoint: W transpose");
  ok(launch_adj_final(aa, A.dwc, dJ_dmfp, A.lam[cur], A.sh[cur], A.dT0, dJ_ddT0, h->t_ref,
                      h->theta, s),
     "adjoint: final");
  double gt[4] = {0, 0, 0, 0};
  ok(cudaMemcpyAsync(gt, A.gtw, sizeof(gt), cudaMemcpyDeviceToHost, s), "adjoint");
  ok(cudaStreamSynchronize(s), "adjoint");
  if (st != WLBM_OK) return st;
  if (dJ_dTwall) {
    for (int k = 0; k < 4; ++k) {
      dJ_dTwall[k] = 0.0;
      if (h->bc_kind[k] != WLBM_BC_ISOTHERMAL) continue;
      const double x = h->theta / h->t_wall[k], e = 1.0 / std::expm1(x);
      dJ_dTwall[k] = gt[k] * e * (1.0 + e) * x / h->t_wall[k];
    }
  }
  return WLBM_OK;
}

}  // extern "C"

// ============================================================================ batches
// Many independent grids (instances) advanced together: one wall launch and one step
// launch per step for the whole batch.  Each instance is a full wlbm_handle; the batch
// adds the per-chunk instance records the batched kernels read.
namespace {
constexpr int kBatchChunk = 64;   // steps per schedule upload of a batch
// default limit of a dependency wait in the persistent kernel: about two seconds of clock
constexpr long long kPersistWaitCycles = 4000000000LL;
}

struct wlbm_batch {
  std::vector<wlbm_handle*> h;
  int storage = 0, variant = 1, graph_steps = 0, fuse_periodic = 0;
  // persistent kernel (WLBM_OPT_PERSISTENT): one launch per chunk of steps, its ring depth
  // (0: default), the dependency-wait limit in clock cycles (0: the default of about two
  // seconds) and the failure-detection test hook
  int persistent = 0, ring_stages = 0, stall_test = 0;
  long long wait_limit = 0;
  unsigned* d_ctr = nullptr;   // [1 + 2n] item queue and per-instance completion counts
  int* d_abort = nullptr;
  int persist_grid = 0;        // blocks of the persistent launch (resident blocks x SMs)
  std::vector<int> prof_w;     // steps timed by each direct event pair
  cudaStream_t stream = nullptr;
  wlbm_allocator alloc{nullptr, nullptr, nullptr};
  std::vector<void*> owned;
  BatchInst* d_inst = nullptr;
  BatchWalls* d_walls = nullptr;
  int* d_wall_inst = nullptr;   // [total_wall_blocks] instance of every wall block
  int* d_tile_inst = nullptr;   // [total_tiles] instance of every variant-3 step tile
  int* d_tile_inst_w = nullptr; // [total_tiles_w] the same for 256-column tiles
  int tile_inst_cap = 0, tile_inst_w_cap = 0;
  bool tables_ok = true;        // the tables match the layout (uploaded by layout())
  uint8_t* d_codes = nullptr;
  uint16_t* d_order = nullptr;      // [instance][t][q + 17] kind-sorted directions
  unsigned char* d_tmaps = nullptr; // [instance] 128-byte CUtensorMaps (variant 3)
  bool all_tmap = false;            // every instance has a tensor map
  unsigned char* d_tmaps_w = nullptr;  // [instance] 32-bit-word maps (bfloat16 wide tiles)
  bool all_tmap_w = false;          // every instance has one
  int wide = 0;                     // per-step launches in 256-column bfloat16 tiles
  int total_tiles_w = 0;
  int max_q = 0;
  BatchInst* h_inst = nullptr;      // pinned staging
  BatchWalls* h_walls = nullptr;
  uint8_t* h_codes = nullptr;
  uint16_t* h_order = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<size_t> code_off, order_off;   // order_off in uint16 elements
  size_t code_bytes = 0, order_elems = 0;
  int total_tiles = 0, total_wall_blocks = 0;
  std::vector<int> per;             // instances whose periodic edges need their own launch
  // Captured chunks, keyed by the energy-plane phases of the instances in `per` (their
  // periodic launches bake plane pointers; the batched kernels read phases at run time).
  // Two per key (replay parity), as for a single grid.
  struct Graph {
    std::vector<int> key;
    int parity = 0;
    TimedGraph tg;
  };
  std::vector<Graph> graphs;
  int graph_parity = 0;
  int64_t graph_replays = 0;
  int64_t graph_launches = 0, launches = 0;
  int prof_every = 0;
  int64_t prof_tick = 0;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
  double prof_graph_ms = 0.0;
  int64_t prof_graph_n = 0;
  std::string err;

  wlbm_status fail(wlbm_status s, const std::string& m) {
    err = m;
    return s;
  }
  wlbm_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return WLBM_OK;
    return fail(WLBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  void* dev_alloc(size_t bytes) {
    bytes = size_t(round_up(int64_t(bytes), 256));
    void* p = nullptr;
    if (alloc.alloc) {
      p = alloc.alloc(bytes, alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void drop_graph() {
    for (Graph& gr : graphs) {
      gr.tg.harvest(&prof_graph_ms, &prof_graph_n);
      gr.tg.destroy();
    }
    graphs.clear();
  }
  std::vector<int> phase_key() const {
    std::vector<int> key;
    for (int k : per) key.push_back(h[k]->e_cur);
    return key;
  }
  void release() {
    drop_graph();
    for (void* p : owned) {
      if (alloc.alloc) {
        if (alloc.free) alloc.free(p, alloc.ctx);
      } else {
        cudaFree(p);
      }
    }
    owned.clear();
    if (h_inst) cudaFreeHost(h_inst);
    if (h_walls) cudaFreeHost(h_walls);
    if (h_codes) cudaFreeHost(h_codes);
    if (h_order) cudaFreeHost(h_order);
    h_order = nullptr;
    if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    h_inst = nullptr; h_walls = nullptr; h_codes = nullptr; ev = nullptr;
    prof_ev.clear();
    for (wlbm_handle* x : h) wlbm_destroy(x);
    h.clear();
  }
  // The persistent kernel covers the wall pass and variant-3 tiles, not periodic links.
  bool persistent_ok(std::string* why) const {
    if (variant != 3) {
      *why = "the persistent kernel runs variant 3 (TMA tiles)";
      return false;
    }
    for (const wlbm_handle* x : h)
      if (x->xper || x->yper) {
        *why = "the persistent kernel takes no instance with a periodic axis";
        return false;
      }
    return true;
  }
  // Both axes periodic and fused: the step kernel mirrors the edges of that instance
  // (not in variant 3, which has no mirror stores).
  bool wraps(const wlbm_handle* x) const {
    return fuse_periodic && variant != 3 && x->xper && x->yper && x->g.nx >= 2 && x->g.ny >= 2;
  }
  void classify() {
    per.clear();
    for (size_t k = 0; k < h.size(); ++k)
      if ((h[k]->xper || h[k]->yper) && !wraps(h[k])) per.push_back(int(k));
  }
  // Block and warp offsets of every instance in the batched grids.
  void layout() {
    total_tiles = 0;
    total_tiles_w = 0;
    total_wall_blocks = 0;
    const int tw = step_tile_width(storage, variant);
    for (size_t k = 0; k < h.size(); ++k) {
      const Geom& g = h[k]->g;
      int tx = (g.nx + 2 + tw - 1) / tw, ty = (g.ny + 2 + kStepRows - 1) / kStepRows;
      if (variant == 3) {   // tiles of the cells variant 3 computes
        StepArgs cover{};
        tma_cover(h[k]->bc_kind, g.nx, g.ny, &cover, &tx, &ty);
        int cb = 0, txw = 0;
        tma_cover_wide(cover, &cb, &txw);
        h_inst[k].cbase_w = cb;
        h_inst[k].tiles_x_w = txw;
        h_inst[k].first_tile_w = total_tiles_w;
        total_tiles_w += txw * ty;
      }
      h_inst[k].tiles_x = tx;
      h_inst[k].first_tile = total_tiles;
      h_inst[k].n_tiles = tx * ty;
      total_tiles += tx * ty;
      h_walls[k].first_block = total_wall_blocks;
      h_walls[k].n_blocks = wall_blocks(h[k]->walls);
      total_wall_blocks += h_walls[k].n_blocks;
    }
    if (variant == 3) upload_tile_tables();
  }
  // Block -> instance tables of the variant-3 batched step kernels (both tilings); the
  // device buffers are sized on the first call and the stream is drained before they are
  // rewritten.
  void upload_tile_tables() {
    std::vector<int> ti(static_cast<size_t>(total_tiles)), tw(static_cast<size_t>(total_tiles_w));
    for (size_t k = 0; k < h.size(); ++k) {
      const int n1 = h_inst[k].n_tiles;
      for (int j = 0; j < n1; ++j) ti[size_t(h_inst[k].first_tile + j)] = int(k);
      const int n2 = (k + 1 < h.size() ? h_inst[k + 1].first_tile_w : total_tiles_w) -
                     h_inst[k].first_tile_w;
      for (int j = 0; j < n2; ++j) tw[size_t(h_inst[k].first_tile_w + j)] = int(k);
    }
    tables_ok = false;
    if (total_tiles > tile_inst_cap) {
      d_tile_inst = static_cast<int*>(dev_alloc(ti.size() * sizeof(int)));
      tile_inst_cap = d_tile_inst ? total_tiles : 0;
    }
    if (total_tiles_w > tile_inst_w_cap) {
      d_tile_inst_w = static_cast<int*>(dev_alloc(tw.size() * sizeof(int)));
      tile_inst_w_cap = d_tile_inst_w ? total_tiles_w : 0;
    }
    if (!d_tile_inst || (total_tiles_w > 0 && !d_tile_inst_w)) return;
    if (stream && cudaStreamSynchronize(stream) != cudaSuccess) return;
    if (cudaMemcpy(d_tile_inst, ti.data(), ti.size() * sizeof(int), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return;
    if (!tw.empty() && cudaMemcpy(d_tile_inst_w, tw.data(), tw.size() * sizeof(int),
                                  cudaMemcpyHostToDevice) != cudaSuccess)
      return;
    tables_ok = true;
  }
};

extern "C" {

wlbm_status wlbm_batch_create(int32_t n, const wlbm_grid* grids, const float* const* mfp_cells,
                              const double* mfp_uniform, const wlbm_boundary* bcs,
                              const wlbm_allocator* alloc, void* stream, wlbm_batch** out) {
  if (n < 1 || !grids || !bcs || !out || (!mfp_cells && !mfp_uniform)) {
    set_global_error("wlbm_batch_create: bad count or NULL argument");
    return WLBM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  auto* b = new wlbm_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  if (alloc) b->alloc = *alloc;
  auto bad = [&](wlbm_status st, const std::string& m) {
    b->release();
    delete b;
    if (!m.empty()) set_global_error(m);
    return st;
  };
  for (int k = 0; k < n; ++k) {
    wlbm_handle* x = nullptr;
    const wlbm_status st = wlbm_create(&grids[k], mfp_cells ? mfp_cells[k] : nullptr,
                                       mfp_uniform ? mfp_uniform[k] : 0.0, &bcs[k], alloc, stream,
                                       &x);
    if (st != WLBM_OK) return bad(st, "");   // message of wlbm_create stays in place
    x->batch_owned = true;
    b->h.push_back(x);
    if (grids[k].storage != grids[0].storage)
      return bad(WLBM_ERR_INVALID_ARG, "wlbm_batch_create: all instances need one storage type");
  }
  b->storage = grids[0].storage;
  b->classify();
  b->code_off.resize(n);
  b->order_off.resize(n);
  b->all_tmap = true;
  b->all_tmap_w = true;
  for (int k = 0; k < n; ++k) {
    b->code_off[k] = b->code_bytes;
    b->code_bytes += size_t(kBatchChunk) * grids[k].q;
    b->order_off[k] = b->order_elems;
    b->order_elems += size_t(kBatchChunk) * (grids[k].q + 17);
    b->max_q = std::max(b->max_q, int(grids[k].q));
    b->all_tmap = b->all_tmap && b->h[k]->has_tmap;
    b->all_tmap_w = b->all_tmap_w && b->h[k]->has_tmap_w;
  }
  b->d_codes = static_cast<uint8_t*>(b->dev_alloc(b->code_bytes));
  b->d_order = static_cast<uint16_t*>(b->dev_alloc(b->order_elems * 2));
  b->d_tmaps = static_cast<unsigned char*>(b->dev_alloc(size_t(n) * 128));
  if (b->all_tmap_w) b->d_tmaps_w = static_cast<unsigned char*>(b->dev_alloc(size_t(n) * 128));
  b->d_inst = static_cast<BatchInst*>(b->dev_alloc(sizeof(BatchInst) * n));
  b->d_walls = static_cast<BatchWalls*>(b->dev_alloc(sizeof(BatchWalls) * n));
  b->d_ctr = static_cast<unsigned*>(b->dev_alloc(sizeof(unsigned) * (1 + 2 * size_t(n))));
  b->d_abort = static_cast<int*>(b->dev_alloc(sizeof(int)));
  // the wall segments of every instance are fixed: the block -> instance table once
  std::vector<int> wall_inst;
  for (int k = 0; k < n; ++k)
    wall_inst.insert(wall_inst.end(), size_t(wall_blocks(b->h[k]->walls)), k);
  if (!wall_inst.empty())
    b->d_wall_inst = static_cast<int*>(b->dev_alloc(wall_inst.size() * sizeof(int)));
  if (!b->d_codes || !b->d_order || !b->d_tmaps || !b->d_inst || !b->d_walls || !b->d_ctr ||
      !b->d_abort || (!wall_inst.empty() && !b->d_wall_inst) || (b->all_tmap_w && !b->d_tmaps_w))
    return bad(WLBM_ERR_OOM, "wlbm_batch_create: device allocation failed");
  if (!wall_inst.empty() &&
      cudaMemcpy(b->d_wall_inst, wall_inst.data(), wall_inst.size() * sizeof(int),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return bad(WLBM_ERR_CUDA, "wlbm_batch_create: upload of the wall block table failed");
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_codes), b->code_bytes,
                                cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_order), b->order_elems * 2,
                      cudaHostAllocDefault);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_inst), sizeof(BatchInst) * n,
                      cudaHostAllocDefault);
  for (int k = 0; k < n && e == cudaSuccess && b->all_tmap; ++k)
    e = cudaMemcpy(b->d_tmaps + size_t(k) * 128, b->h[k]->tmap, 128, cudaMemcpyHostToDevice);
  for (int k = 0; k < n && e == cudaSuccess && b->all_tmap_w; ++k)
    e = cudaMemcpy(b->d_tmaps_w + size_t(k) * 128, b->h[k]->tmap_w, 128, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&b->h_walls), sizeof(BatchWalls) * n,
                      cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bad(WLBM_ERR_CUDA, std::string("wlbm_batch_create: ") + cudaGetErrorString(e));
  }
  std::memset(b->h_inst, 0, sizeof(BatchInst) * n);
  if (b->all_tmap) {
    b->variant = 3;
    b->classify();
  }
  b->wide = b->all_tmap_w ? 1 : 0;
  std::memset(b->h_walls, 0, sizeof(BatchWalls) * n);
  b->layout();
  if (!b->tables_ok) {
    cudaGetLastError();
    return bad(WLBM_ERR_CUDA, "wlbm_batch_create: upload of the tile tables failed");
  }
  *out = b;
  return WLBM_OK;
}

void wlbm_batch_destroy(wlbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  b->release();
  delete b;
}

const char* wlbm_batch_last_error(const wlbm_batch* b) {
  return b ? b->err.c_str() : wlbm_last_error(nullptr);
}

int32_t wlbm_batch_size(const wlbm_batch* b) { return b ? int32_t(b->h.size()) : -1; }

wlbm_handle* wlbm_batch_instance(wlbm_batch* b, int32_t k) {
  return (b && k >= 0 && k < int32_t(b->h.size())) ? b->h[k] : nullptr;
}

wlbm_status wlbm_batch_init_temperature(wlbm_batch* b, const float* const* dT) {
  if (!b || !dT) return WLBM_ERR_INVALID_ARG;
  for (size_t k = 0; k < b->h.size(); ++k) {
    const wlbm_status st = wlbm_init_temperature(b->h[k], dT[k]);
    if (st != WLBM_OK) return b->fail(st, "instance " + std::to_string(k) + ": " + b->h[k]->err);
  }
  b->drop_graph();   // wall values may have changed
  return WLBM_OK;
}

wlbm_status wlbm_batch_get_option(const wlbm_batch* b, int32_t key, int64_t* value) {
  if (!b || !value) return WLBM_ERR_INVALID_ARG;
  if (key == WLBM_OPT_STEP_VARIANT) *value = b->variant;
  else if (key == WLBM_OPT_GRAPH_STEPS) *value = b->graph_steps;
  else if (key == WLBM_OPT_FUSE_PERIODIC) *value = b->fuse_periodic;
  else if (key == WLBM_OPT_GRAPH_REPLAYS) *value = b->graph_replays;
  else if (key == WLBM_OPT_PERSISTENT) *value = b->persistent;
  else if (key == WLBM_OPT_RING_STAGES) *value = b->ring_stages;
  else if (key == WLBM_OPT_WAIT_LIMIT) *value = b->wait_limit;
  else if (key == WLBM_OPT_STALL_TEST) *value = b->stall_test;
  else if (key == WLBM_OPT_BF16_WIDE) *value = b->wide;
  else return WLBM_ERR_INVALID_ARG;
  return WLBM_OK;
}

wlbm_status wlbm_batch_set_option(wlbm_batch* b, int32_t key, int64_t value) {
  if (!b) return WLBM_ERR_INVALID_ARG;
  if (key == WLBM_OPT_STEP_VARIANT && value == 3 && !b->all_tmap)
    return b->fail(WLBM_ERR_INVALID_ARG,
                   "wlbm_batch_set_option: step variant 3 needs a tensor map of every instance");
  if (key == WLBM_OPT_STEP_VARIANT && (value == 0 || value == 1 || value == 3)) {
    if (b->persistent && value != 3)
      return b->fail(WLBM_ERR_INVALID_ARG,
                     "wlbm_batch_set_option: the persistent kernel runs variant 3");
    b->variant = int(value);
    b->layout();
    b->classify();
    b->drop_graph();
    if (!b->tables_ok) {
      cudaGetLastError();
      return b->fail(WLBM_ERR_CUDA, "wlbm_batch_set_option: upload of the tile tables failed");
    }
    return WLBM_OK;
  }
  if (key == WLBM_OPT_PERSISTENT && (value == 0 || value == 1)) {
    std::string why;
    if (value == 1 && !b->persistent_ok(&why))
      return b->fail(WLBM_ERR_INVALID_ARG, "wlbm_batch_set_option: " + why);
    b->persistent = int(value);
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_RING_STAGES && value >= 0 && value <= 64 &&
      batch_persistent_stages_ok(b->storage, int(value))) {
    b->ring_stages = int(value);
    b->persist_grid = 0;
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_WAIT_LIMIT && value >= 0) {
    b->wait_limit = value;
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_STALL_TEST && (value == 0 || value == 1)) {
    b->stall_test = int(value);
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_GRAPH_STEPS && value >= 0 && value <= kBatchChunk && value % 6 == 0) {
    b->graph_steps = int(value);
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_FUSE_PERIODIC && (value == 0 || value == 1)) {
    b->fuse_periodic = int(value);
    b->classify();
    b->drop_graph();
    return WLBM_OK;
  }
  if (key == WLBM_OPT_BF16_WIDE && (value == 0 || value == 1)) {
    if (value == 1 && !b->all_tmap_w)
      return b->fail(WLBM_ERR_INVALID_ARG, "wlbm_batch_set_option: wide tiles need bfloat16 "
                                           "storage and a word tensor map of every instance");
    b->wide = int(value);
    b->drop_graph();
    return WLBM_OK;
  }
  return b->fail(WLBM_ERR_INVALID_ARG, "wlbm_batch_set_option: unknown key or value");
}

}  // extern "C"

// Kernels of `count` steps for the whole batch, instance records already on the device.
static wlbm_status batch_enqueue(wlbm_batch* b, int count, int every,
                                 const std::vector<cudaEvent_t>* cap = nullptr) {
  size_t cap_used = 0;
  const int n = int(b->h.size());
  wlbm_status st = WLBM_OK;
  bool any_spec = false;
  for (const wlbm_handle* x : b->h) any_spec = any_spec || x->walls.any_spec;
  if (b->persistent) {
    // one launch for the chunk: the wall pass and the tiles of every step
    if (b->persist_grid == 0) {
      int dev = 0, sms = 0;
      st = b->cuda(cudaGetDevice(&dev), "wlbm_batch_step: device");
      if (st == WLBM_OK)
        st = b->cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                     "wlbm_batch_step: device");
      if (st != WLBM_OK) return st;
      const int per_sm = batch_persistent_blocks_per_sm(b->storage, b->ring_stages, b->max_q);
      if (per_sm <= 0)
        return b->fail(WLBM_ERR_CUDA, "wlbm_batch_step: the persistent kernel does not fit an SM");
      b->persist_grid = per_sm * sms;
    }
    PersistArgs p{};
    p.insts = b->d_inst;
    p.walls = b->d_walls;
    p.wall_inst = b->d_wall_inst;
    p.tile_inst = b->d_tile_inst;
    p.n = n;
    p.wall_items = b->total_wall_blocks;
    p.tile_items = b->total_tiles;
    p.steps = count;
    p.ctr = b->d_ctr;
    p.abort_flag = b->d_abort;
    p.wait_limit = b->wait_limit > 0 ? b->wait_limit : kPersistWaitCycles;
    p.stall_test = b->stall_test;
    st = b->cuda(cudaMemsetAsync(b->d_ctr, 0, sizeof(unsigned) * (1 + 2 * size_t(n)), b->stream),
                 "wlbm_batch_step: counters");
    if (st == WLBM_OK)
      st = b->cuda(cudaMemsetAsync(b->d_abort, 0, sizeof(int), b->stream),
                   "wlbm_batch_step: counters");
    if (st != WLBM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (every > 0) {
      if (cap) {
        e0 = (*cap)[0];
        e1 = (*cap)[1];
      } else {
        if (b->prof_used + 2 > b->prof_ev.size()) {
          for (int j = 0; j < 2; ++j) {
            cudaEvent_t ev;
            st = b->cuda(cudaEventCreate(&ev), "wlbm_batch_step: profiling");
            if (st != WLBM_OK) return st;
            b->prof_ev.push_back(ev);
          }
        }
        e0 = b->prof_ev[b->prof_used];
        e1 = b->prof_ev[b->prof_used + 1];
        b->prof_used += 2;
        b->prof_w.push_back(count);
      }
      st = b->cuda(record_event(e0, b->stream, cap != nullptr), "profiling");
    }
    if (st == WLBM_OK)
      st = b->cuda(launch_batch_persistent(b->storage, b->ring_stages, p, b->max_q,
                                           b->persist_grid, any_spec, b->stream),
                   "wlbm_batch_step: persistent kernel");
    ++b->launches;
    if (st == WLBM_OK && e1) st = b->cuda(record_event(e1, b->stream, cap != nullptr), "profiling");
    return st;
  }
  for (int t = 0; t < count && st == WLBM_OK; ++t) {
    if (b->total_wall_blocks > 0) {
      st = b->cuda(launch_walls_batch(b->storage, b->d_walls, b->d_wall_inst,
                                      b->total_wall_blocks, t, any_spec, b->stream),
                   "wlbm_batch_step: walls");
      ++b->launches;
    }
    for (int k : b->per) {
      if (st != WLBM_OK) break;
      wlbm_handle* x = b->h[k];
      const Geom& g = x->g;
      const BatchInst& I = b->h_inst[k];
      const int cur = (I.phase + t) % I.n_e;
      PeriodicArgs pa{};
      pa.planes = x->planes; pa.plane = g.plane; pa.pitch = g.pitch; pa.nx = g.nx; pa.ny = g.ny;
      pa.q = g.q; pa.codes = b->d_codes + b->code_off[k] + size_t(t) * g.q;
      pa.e_cur = I.e[cur]; pa.e_ref = I.n_e == 3 ? I.e[(cur + 2) % 3] : nullptr;
      pa.xper = x->xper; pa.yper = x->yper;
      st = b->cuda(launch_periodic(b->storage, pa, b->stream), "wlbm_batch_step: periodic");
      ++b->launches;
    }
    if (st != WLBM_OK) break;
    cudaEvent_t e1 = nullptr;
    if (every > 0 && (cap ? t % every == 0 : b->prof_tick++ % every == 0)) {
      cudaEvent_t e0 = nullptr;
      if (cap) {
        e0 = (*cap)[cap_used];
        e1 = (*cap)[cap_used + 1];
        cap_used += 2;
      } else {
        if (b->prof_used + 2 > b->prof_ev.size()) {
          for (int j = 0; j < 2; ++j) {
            cudaEvent_t ev;
            st = b->cuda(cudaEventCreate(&ev), "wlbm_batch_step: profiling");
            if (st != WLBM_OK) return st;
            b->prof_ev.push_back(ev);
          }
        }
        e0 = b->prof_ev[b->prof_used];
        e1 = b->prof_ev[b->prof_used + 1];
        b->prof_used += 2;
        b->prof_w.push_back(1);
      }
      st = b->cuda(record_event(e0, b->stream, cap != nullptr), "profiling");
    }
    if (st == WLBM_OK)
      st = b->cuda(b->variant == 3 && b->wide
                       ? launch_step_tma_batch_wide(b->d_inst, b->d_tile_inst_w, n, b->max_q,
                                                    b->total_tiles_w, t, b->stream)
                   : b->variant == 3
                       ? launch_step_tma_batch(b->storage, b->d_inst, b->d_tile_inst, n,
                                               b->max_q, b->total_tiles, t, b->stream)
                       : launch_step_batch(b->storage, b->variant, b->d_inst, n, b->total_tiles,
                                           t, b->stream),
                   "wlbm_batch_step: step");
    ++b->launches;
    if (st == WLBM_OK && e1) st = b->cuda(record_event(e1, b->stream, cap != nullptr), "profiling");
  }
  return st;
}

extern "C" {

wlbm_status wlbm_batch_step(wlbm_batch* b, int64_t n) {
  if (!b) return WLBM_ERR_INVALID_ARG;
  if (n < 0) return b->fail(WLBM_ERR_INVALID_ARG, "wlbm_batch_step: negative step count");
  const int ni = int(b->h.size());
  const bool graphs = b->graph_steps > 0 && b->stream;
  while (n > 0) {
    const int ch = int(std::min<int64_t>(n, graphs ? b->graph_steps : kBatchChunk));
    wlbm_status st = b->cuda(cudaEventSynchronize(b->ev), "wlbm_batch_step");
    if (st != WLBM_OK) return st;
    for (int k = 0; k < ni; ++k) {
      wlbm_handle* x = b->h[k];
      const Geom& g = x->g;
      uint8_t* hc = b->h_codes + b->code_off[k];
      uint16_t* ho = b->h_order + b->order_off[k];
      for (int t = 0; t < ch; ++t) {
        tas_advance(x->lat, &x->tas, hc + size_t(t) * g.q);
        sort_by_kind(hc + size_t(t) * g.q, g.q, ho + size_t(t) * (g.q + 17));
      }
      BatchInst& I = b->h_inst[k];
      StepArgs& a = I.a;
      a = StepArgs{};
      a.planes = x->planes; a.plane = g.plane; a.pitch = g.pitch; a.rows = g.rows;
      a.nx = g.nx; a.ny = g.ny; a.q = g.q; a.w = x->w_dev();
      a.wfield = x->field_w ? x->wfield : nullptr; a.w0 = x->w0;
      a.scale = x->scale; a.inv_scale = x->inv_scale;
      a.variant = b->variant; a.status = x->d_status;
      a.xper = x->xper; a.yper = x->yper;
      a.wrap = b->wraps(x);
      int tx_unused = 0, ty_unused = 0;
      tma_cover(x->bc_kind, g.nx, g.ny, &a, &tx_unused, &ty_unused);
      for (int j = 0; j < 3; ++j) I.e[j] = x->e[j];
      I.codes = b->d_codes + b->code_off[k];
      I.order = b->d_order + b->order_off[k];
      I.tmap = b->d_tmaps + size_t(k) * 128;
      I.tmap_w = b->d_tmaps_w ? b->d_tmaps_w + size_t(k) * 128 : nullptr;
      I.n_e = x->bf16() ? 3 : 2;
      I.phase = x->e_cur;
      BatchWalls& Wk = b->h_walls[k];
      Wk.w = x->walls;
      for (int j = 0; j < 3; ++j) Wk.e[j] = x->e[j];
      Wk.codes = I.codes;
      Wk.n_e = I.n_e;
      Wk.phase = I.phase;
    }
    st = b->cuda(cudaMemcpyAsync(b->d_codes, b->h_codes, b->code_bytes, cudaMemcpyHostToDevice,
                                 b->stream), "wlbm_batch_step: upload");
    if (st == WLBM_OK)
      st = b->cuda(cudaMemcpyAsync(b->d_order, b->h_order, b->order_elems * 2,
                                   cudaMemcpyHostToDevice, b->stream), "wlbm_batch_step: upload");
    if (st == WLBM_OK)
      st = b->cuda(cudaMemcpyAsync(b->d_inst, b->h_inst, sizeof(BatchInst) * ni,
                                   cudaMemcpyHostToDevice, b->stream), "wlbm_batch_step: upload");
    if (st == WLBM_OK)
      st = b->cuda(cudaMemcpyAsync(b->d_walls, b->h_walls, sizeof(BatchWalls) * ni,
                                   cudaMemcpyHostToDevice, b->stream), "wlbm_batch_step: upload");
    if (st == WLBM_OK) st = b->cuda(cudaEventRecord(b->ev, b->stream), "wlbm_batch_step");
    if (st != WLBM_OK) return st;
    if (graphs && ch == b->graph_steps) {
      const std::vector<int> key = b->phase_key();
      const int parity = b->graph_parity;
      b->graph_parity ^= 1;
      TimedGraph* tg = nullptr;
      for (wlbm_batch::Graph& gr : b->graphs)
        if (gr.key == key && gr.parity == parity) tg = &gr.tg;
      if (!tg) {
        if (b->graphs.size() >= 6) b->drop_graph();
        TimedGraph fresh;
        const int every = b->prof_every;
        // a persistent chunk is one launch: one timed pair covering its ch steps
        const int pairs = every > 0 ? (b->persistent ? 1 : (ch + every - 1) / every) : 0;
        fresh.weight = b->persistent ? ch : 1;
        st = b->cuda(fresh.make_events(pairs), "wlbm_batch_step: graph events");
        const int64_t l0 = b->launches;
        if (st == WLBM_OK)
          st = b->cuda(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal),
                       "wlbm_batch_step: capture");
        if (st != WLBM_OK) {
          fresh.destroy();
          return st;
        }
        const wlbm_status est = batch_enqueue(b, ch, every, &fresh.ev);
        cudaGraph_t gr = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &gr);
        if (est == WLBM_OK) st = b->cuda(ce, "wlbm_batch_step: capture");
        else st = est;
        if (st == WLBM_OK)
          st = b->cuda(cudaGraphInstantiate(&fresh.exec, gr, 0), "wlbm_batch_step: graph");
        if (gr) cudaGraphDestroy(gr);
        if (st != WLBM_OK) {
          fresh.destroy();
          return st;
        }
        b->graphs.push_back({key, parity, fresh});
        tg = &b->graphs.back().tg;
        b->graph_launches = b->launches - l0;
        b->launches = l0;
      } else {
        st = b->cuda(tg->harvest(&b->prof_graph_ms, &b->prof_graph_n), "wlbm_batch_step: timing");
        if (st != WLBM_OK) return st;
      }
      b->launches += b->graph_launches;
      ++b->graph_replays;
      st = b->cuda(tg->launch(b->stream), "wlbm_batch_step: graph launch");
    } else {
      st = batch_enqueue(b, ch, b->prof_every);
    }
    if (st != WLBM_OK) return st;
    for (wlbm_handle* x : b->h)
      for (int t = 0; t < ch; ++t) x->rotate_energy();
    n -= ch;
  }
  return WLBM_OK;
}

wlbm_status wlbm_batch_check(wlbm_batch* b) {
  if (!b) return WLBM_ERR_INVALID_ARG;
  wlbm_status r = b->cuda(cudaStreamSynchronize(b->stream), "wlbm_batch_check");
  if (r != WLBM_OK) return r;
  int bad = -1;
  for (size_t k = 0; k < b->h.size(); ++k) {
    const wlbm_status st = wlbm_check(b->h[k]);
    if (st == WLBM_ERR_TIMEOUT && bad < 0) bad = int(k);
    else if (st != WLBM_OK && st != WLBM_ERR_TIMEOUT) return b->fail(st, b->h[k]->err);
  }
  if (bad >= 0)
    return b->fail(WLBM_ERR_TIMEOUT,
                   "a bounded wait gave up (first instance with its status set: " +
                       std::to_string(bad) + ")");
  return WLBM_OK;
}

wlbm_status wlbm_batch_profile(wlbm_batch* b, int32_t every) {
  if (!b) return WLBM_ERR_INVALID_ARG;
  if (every < 0) return b->fail(WLBM_ERR_INVALID_ARG, "wlbm_batch_profile: negative stride");
  if (every != b->prof_every) b->drop_graph();   // their event nodes follow the stride
  b->prof_every = every;
  b->prof_tick = 0;
  return WLBM_OK;
}

wlbm_status wlbm_batch_profile_read(wlbm_batch* b, double* step_ms, int64_t* step_launches,
                                    int64_t* all_launches) {
  if (!b) return WLBM_ERR_INVALID_ARG;
  wlbm_status st = b->cuda(cudaStreamSynchronize(b->stream), "wlbm_batch_profile_read");
  if (st != WLBM_OK) return st;
  for (wlbm_batch::Graph& gr : b->graphs) {
    st = b->cuda(gr.tg.harvest(&b->prof_graph_ms, &b->prof_graph_n), "profile_read");
    if (st != WLBM_OK) return st;
  }
  double total = b->prof_graph_ms;
  for (size_t k = 0; k + 1 < b->prof_used; k += 2) {
    float ms = 0.f;
    st = b->cuda(cudaEventElapsedTime(&ms, b->prof_ev[k], b->prof_ev[k + 1]), "profile_read");
    if (st != WLBM_OK) return st;
    total += ms;
  }
  int64_t timed = b->prof_graph_n;
  for (int w : b->prof_w) timed += w;
  if (step_ms) *step_ms = total;
  if (step_launches) *step_launches = timed;
  if (all_launches) *all_launches = b->launches;
  b->prof_used = 0;
  b->prof_w.clear();
  b->prof_graph_ms = 0.0;
  b->prof_graph_n = 0;
  return WLBM_OK;
}

// Native autotuner: times `trial_steps` steps for every candidate (step-kernel variant x
// graph replay with per-step launches; the persistent kernel at both ring depths x graph
// replay, where the batch allows it) after one warm-up run of each, keeps the fastest, and
// reports it.  The trial steps advance the instances: call it before
// wlbm_batch_init_temperature.
wlbm_status wlbm_batch_autotune(wlbm_batch* b, int32_t trial_steps, int32_t* variant,
                                int32_t* graph_steps, double* ms_per_step) {
  if (!b || trial_steps < 6) return WLBM_ERR_INVALID_ARG;
  const int g = std::min(kBatchChunk, (trial_steps / 6) * 6);
  const int alt = b->storage == WLBM_STORE_BF16_DEV ? 16 : 4;   // the other ring depth
  // variant, graph steps, persistent, ring stages
  const int cand[10][4] = {{1, 0, 0, 0}, {0, 0, 0, 0}, {3, 0, 0, 0}, {1, g, 0, 0},
                           {0, g, 0, 0}, {3, g, 0, 0}, {3, 0, 1, 0}, {3, g, 1, 0},
                           {3, 0, 1, alt}, {3, g, 1, alt}};
  double best = 1e300;
  int bv = 1, bg = 0, bp = 0, bs = 0;
  std::string why;
  cudaEvent_t e0, e1;
  wlbm_status st = b->cuda(cudaEventCreate(&e0), "autotune");
  if (st != WLBM_OK) return st;
  st = b->cuda(cudaEventCreate(&e1), "autotune");
  for (int c = 0; c < 10 && st == WLBM_OK; ++c) {
    if (cand[c][0] == 3 && !b->all_tmap) continue;
    st = wlbm_batch_set_option(b, WLBM_OPT_PERSISTENT, 0);
    if (st == WLBM_OK) st = wlbm_batch_set_option(b, WLBM_OPT_STEP_VARIANT, cand[c][0]);
    if (st == WLBM_OK && cand[c][2]) {
      if (!b->persistent_ok(&why)) continue;
      st = wlbm_batch_set_option(b, WLBM_OPT_PERSISTENT, 1);
    }
    if (st == WLBM_OK) st = wlbm_batch_set_option(b, WLBM_OPT_RING_STAGES, cand[c][3]);
    if (st == WLBM_OK) st = wlbm_batch_set_option(b, WLBM_OPT_GRAPH_STEPS, cand[c][1]);
    if (st == WLBM_OK) st = wlbm_batch_step(b, g > 0 ? g : 6);           // warm-up / capture
    if (st == WLBM_OK) st = b->cuda(cudaEventRecord(e0, b->stream), "autotune");
    if (st == WLBM_OK) st = wlbm_batch_step(b, trial_steps);
    if (st == WLBM_OK) st = b->cuda(cudaEventRecord(e1, b->stream), "autotune");
    if (st == WLBM_OK) st = b->cuda(cudaEventSynchronize(e1), "autotune");
    float ms = 0.f;
    if (st == WLBM_OK) st = b->cuda(cudaEventElapsedTime(&ms, e0, e1), "autotune");
    if (st == WLBM_OK && ms / trial_steps < best) {
      best = ms / trial_steps;
      bv = cand[c][0];
      bg = cand[c][1];
      bp = cand[c][2];
      bs = cand[c][3];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WLBM_OK) return st;
  wlbm_batch_set_option(b, WLBM_OPT_PERSISTENT, 0);
  wlbm_batch_set_option(b, WLBM_OPT_STEP_VARIANT, bv);
  wlbm_batch_set_option(b, WLBM_OPT_PERSISTENT, bp);
  wlbm_batch_set_option(b, WLBM_OPT_RING_STAGES, bs);
  wlbm_batch_set_option(b, WLBM_OPT_GRAPH_STEPS, bg);
  if (variant) *variant = bv;
  if (graph_steps) *graph_steps = bg;
  if (ms_per_step) *ms_per_step = best;
  return WLBM_OK;
}

// The same search for one grid.
wlbm_status wlbm_autotune(wlbm_handle* h, int32_t trial_steps, int32_t* variant,
                          int32_t* graph_steps, double* ms_per_step) {
  if (!h || trial_steps < 6) return WLBM_ERR_INVALID_ARG;
  const int g = std::min(kChunk, (trial_steps / 6) * 6);
  const int cand[8][2] = {{1, 0}, {0, 0}, {2, 0}, {3, 0}, {1, g}, {0, g}, {2, g}, {3, g}};
  double best = 1e300;
  int bv = 1, bg = 0;
  cudaEvent_t e0, e1;
  wlbm_status st = h->cuda(cudaEventCreate(&e0), "autotune");
  if (st != WLBM_OK) return st;
  st = h->cuda(cudaEventCreate(&e1), "autotune");
  for (int c = 0; c < 8 && st == WLBM_OK; ++c) {
    if (cand[c][1] > 0 && !h->stream) continue;     // graphs need a capturable stream
    if (cand[c][0] == 3 && !h->has_tmap) continue;
    st = wlbm_set_option(h, WLBM_OPT_STEP_VARIANT, cand[c][0]);
    if (st == WLBM_OK) st = wlbm_set_option(h, WLBM_OPT_GRAPH_STEPS, cand[c][1]);
    if (st == WLBM_OK) st = wlbm_step(h, g > 0 ? g : 6);
    if (st == WLBM_OK) st = h->cuda(cudaEventRecord(e0, h->stream), "autotune");
    if (st == WLBM_OK) st = wlbm_step(h, trial_steps);
    if (st == WLBM_OK) st = h->cuda(cudaEventRecord(e1, h->stream), "autotune");
    if (st == WLBM_OK) st = h->cuda(cudaEventSynchronize(e1), "autotune");
    float ms = 0.f;
    if (st == WLBM_OK) st = h->cuda(cudaEventElapsedTime(&ms, e0, e1), "autotune");
    if (st == WLBM_OK && ms / trial_steps < best) {
      best = ms / trial_steps;
      bv = cand[c][0];
      bg = cand[c][1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WLBM_OK) return st;
  wlbm_set_option(h, WLBM_OPT_STEP_VARIANT, bv);
  wlbm_set_option(h, WLBM_OPT_GRAPH_STEPS, bg);
  if (variant) *variant = bv;
  if (graph_steps) *graph_steps = bg;
  if (ms_per_step) *ms_per_step = best;
  return WLBM_OK;
}

}  // extern "C"
