// Host-side angular lattice and TAS schedule (Sec. 2.3-2.5 of the paper).
//
// Directions (Sec. 2.4): the 8M lattice points on the square ring of Chebyshev radius M,
// ordered counter-clockwise from +x.  Weights (Eq. weight, garbled in print; read as the
// sum of the two angular gaps to the neighbouring directions over 4 pi).  Worm paths
// (Eq. worm-paths): M greedy basic hops towards the ray points (n/M) s, a later hop index
// winning ties, compared exactly in integers.  TAS (Eq. algorithm): a direction hops at
// step n only if |p + c|^2 <= (n + 1)^2; its worm index advances per executed hop.
#include "lattice.hpp"

#include <cmath>

namespace wlbm {

bool build_lattice(int q, Lattice* L) {
  if (q < 8 || q > 1024 || q % 8 != 0) return false;
  const int m = q / 8;
  L->q = q;
  L->m = m;
  L->dx.clear();
  L->dy.clear();
  // Walk the ring: right edge upwards (angles [0, 45)), top edge leftwards, left edge
  // downwards, bottom edge rightwards, right edge below the axis.
  for (int j = 0; j < m; ++j) { L->dx.push_back(m); L->dy.push_back(j); }
  for (int j = m; j > -m; --j) { L->dx.push_back(j); L->dy.push_back(m); }
  for (int j = m; j > -m; --j) { L->dx.push_back(-m); L->dy.push_back(j); }
  for (int j = -m; j < m; ++j) { L->dx.push_back(j); L->dy.push_back(-m); }
  for (int j = -m; j < 0; ++j) { L->dx.push_back(m); L->dy.push_back(j); }

  const double two_pi = 2.0 * M_PI;
  std::vector<double> ang(q);
  L->sx.assign(q, 0.0);
  L->sy.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    const double len = std::sqrt(double(L->dx[i]) * L->dx[i] + double(L->dy[i]) * L->dy[i]);
    L->sx[i] = L->dx[i] / len;
    L->sy[i] = L->dy[i] / len;
    ang[i] = std::atan2(double(L->dy[i]), double(L->dx[i]));
  }
  L->w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    const int ip = (i + q - 1) % q, in = (i + 1) % q;
    double gp = std::fmod(ang[i] - ang[ip], two_pi);
    if (gp < 0) gp += two_pi;
    double gn = std::fmod(ang[in] - ang[i], two_pi);
    if (gn < 0) gn += two_pi;
    L->w[i] = (gp + gn) / (4.0 * M_PI);
  }

  L->worm.assign(size_t(q) * m, 0);
  double sum_c = 0.0;
  for (int i = 0; i < q; ++i) {
    const int64_t a = L->dx[i], b = L->dy[i];
    int64_t px = 0, py = 0;
    double len = 0.0;
    for (int n = 1; n <= m; ++n) {
      // distance^2 to the ray point, scaled by m^2; the search starts at distance 1.
      int64_t best = int64_t(m) * m;
      int pick = -1;
      for (int k = 0; k < 8; ++k) {
        const int64_t ex = int64_t(m) * (px + kHopX[k]) - n * a;
        const int64_t ey = int64_t(m) * (py + kHopY[k]) - n * b;
        const int64_t d2 = ex * ex + ey * ey;
        if (d2 <= best) { best = d2; pick = k; }
      }
      if (pick < 0) return false;
      L->worm[size_t(i) * m + (n - 1)] = int8_t(pick);
      px += kHopX[pick];
      py += kHopY[pick];
      len += (pick < 4) ? 1.0 : std::sqrt(2.0);
    }
    if (px != a || py != b) return false;
    sum_c += len / m;   // c_i: mean basic-hop length along the worm
  }
  L->lam_corr = q / sum_c;
  return true;
}

double corrected_weight(double mfp_cells, double lam_corr, bool emulate_3d, int relax_mode) {
  const double W = std::isinf(mfp_cells) ? 0.0 : 1.0 / mfp_cells;
  const double f = emulate_3d ? 1.5 : 1.0;
  double wc = f * ((1.0 - W) * W + W * (W * lam_corr));
  if (relax_mode == 1) wc = -std::expm1(-wc);
  return wc;
}

void TasState::reset(int q) {
  n = 0;
  px.assign(q, 0);
  py.assign(q, 0);
  h.assign(q, 0);
  parity.assign(q, 0);
}

void tas_advance(const Lattice& L, TasState* st, uint8_t* codes) {
  const int64_t n = st->n + 1;
  const int64_t lim = (n + 1) * (n + 1);
  // below the unit speed the reference distance is v n: |p + c|^2 <= (v n + 1)^2 in
  // float64, two roundings (v n, + 1) and the square (host code is built without
  // contraction into fused multiply-adds)
  const bool unit = L.speed == 1.0;
  const double r = L.speed * double(n) + 1.0;
  const double r2 = r * r;
  for (int i = 0; i < L.q; ++i) {
    const int k = L.worm[size_t(i) * L.m + size_t(st->h[i] % L.m)];
    const int64_t x = st->px[i] + kHopX[k], y = st->py[i] + kHopY[k];
    const bool hop = unit ? x * x + y * y <= lim : double(x * x + y * y) <= r2;
    codes[i] = uint8_t(k | (hop ? 0 : 8) | (st->parity[i] << 4));
    if (hop) {
      st->px[i] = x;
      st->py[i] = y;
      st->h[i] += 1;
      st->parity[i] ^= 1;
    }
  }
  st->n = n;
}

}  // namespace wlbm
