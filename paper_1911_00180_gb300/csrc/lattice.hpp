// Host-side angular lattice and TAS schedule of the worm-LBM (Sec. 2.3-2.5 of the paper).
#pragma once
#include <cstdint>
#include <vector>

namespace wlbm {

// Basic D2Q8 hops, paper numbering 1-4 axial then 5-8 diagonal (Sec. 2.4, Fig. 1).
constexpr int kHopX[8] = {1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kHopY[8] = {0, 1, 0, -1, 1, 1, -1, -1};

struct Lattice {
  int q = 0, m = 0;
  std::vector<int> dx, dy;            // ring direction vectors, Chebyshev radius m
  std::vector<double> sx, sy;         // unit vectors s_i
  std::vector<double> w;              // angular weights, Eq. weight
  std::vector<int8_t> worm;           // [q][m] basic-hop index per worm sub-step
  double lam_corr = 0.0;              // Eq. W-correction-factor-generalized
  double speed = 1.0;                 // propagation speed v in (0, 1], cells per step
};

// Returns false if q is not a multiple of 8 in [8, 1024].
bool build_lattice(int q, Lattice* out);

// Corrected relaxation weight, Eq. W-correction (+ optional exponential mode).
double corrected_weight(double mfp_cells, double lam_corr, bool emulate_3d, int relax_mode);

// TAS state per direction: displacement p_i and executed-hop counter h_i (Eq. algorithm).
struct TasState {
  int64_t n = 0;                       // steps taken
  std::vector<int64_t> px, py, h;
  std::vector<uint8_t> parity;         // which buffer holds plane i (GPU bookkeeping)
  void reset(int q);
};

// Advance one step (n -> n+1).  Writes per direction: hop index | paused << 3 |
// parity-of-current-buffer << 4, then updates the state (a hopping plane switches buffer,
// a paused plane is updated in place).
void tas_advance(const Lattice& lat, TasState* st, uint8_t* codes);

}  // namespace wlbm
