"""Oracle, part 1: the angular lattice of the worm-LBM, written from the paper in plain
Python / numpy float64.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Everything here follows Sec. 2.3-2.5 of the paper:

* ring_directions   the 8M propagation directions of a D2Q[M x 8] scheme (Sec. 2.4,
                    "next-next neighbour" directions; the lattice points on the square ring
                    of Chebyshev radius M, ordered counter-clockwise from +x).
* angular_weights   Eq. weight.  The printed formula is garbled; it is read as: the weight
                    of a direction is the sum of the two angular gaps to its circular
                    neighbours, divided by 4 pi (so the weights sum to one and equal 1/8 on
                    D2Q8, as Sec. 2.2 requires).
* worm_path         Eq. worm-paths (Sec. 2.5): greedy choice, at each of the M sub-steps,
                    of the basic D2Q8 hop whose end point lies nearest to the ray point
                    (n/M) * s; a later hop index wins a tie (the comparison is "<="), and
                    the running best starts at distance 1.  Distances are compared exactly
                    in integers (squared distance scaled by M^2).
* lambda_corr       Eq. W-correction-factor-generalized: Q / sum_i c_i, where c_i is the
                    mean length of one basic hop along direction i's worm path (the speed
                    of the always-propagating EED of direction i).
* w_corr            Eq. W-correction.
* TasSchedule       Eq. algorithm: the time adaptive scheme.  A direction executes its due
                    worm hop at step n only if the distance it has propagated after the hop
                    stays within the axial distance n plus one lattice spacing, i.e.
                    |p + c|^2 <= (n + 1)^2, evaluated exactly in integers.  The worm index
                    advances per executed hop.

Pins (tests/test_oracle_lattice.py): the printed D2Q8 hop pattern of Sec. 2.3 (diagonal
hops at n = 1, 2, 4, 5, pause at n = 3); Lambda_corr(D2Q8) = 2/(1+sqrt 2) (Eq.
W-correction-factor); w = 1/8 on D2Q8 (Sec. 2.2); the equal-angle pattern of Fig. 3;
worm end points and the one-grid-spacing propagation-error bound of Sec. 3.1.
"""
import math

import numpy as np

# Basic D2Q8 hops in the paper's numbering: axial directions 1-4, then diagonal 5-8
# (Sec. 2.4 and Fig. 1).  Index k here is the paper's k+1.
BASIC_HOPS = (
    (1, 0), (0, 1), (-1, 0), (0, -1),
    (1, 1), (-1, 1), (-1, -1), (1, -1),
)

HBAR = 1.054571817e-34     # J s
K_B = 1.380649e-23         # J / K
OMEGA0 = 81.8e12           # rad / s, phonon frequency of the property table (Sec. 3)
THETA_DEFAULT = HBAR * OMEGA0 / K_B   # hbar omega0 / k_B, about 624.8 K


def ring_directions(q):
    """The Q = 8M lattice vectors (integer pairs) of the D2Q[M x 8] scheme, ordered by
    angle from +x counter-clockwise.  For Q = 8 these are the eight D2Q8 hops."""
    if q < 8 or q % 8:
        raise ValueError("Q must be a positive multiple of 8")
    m = q // 8
    pts = [(m, j) for j in range(0, m)]
    pts += [(j, m) for j in range(m, -m, -1)]
    pts += [(-m, j) for j in range(m, -m, -1)]
    pts += [(j, -m) for j in range(-m, m)]
    pts += [(m, j) for j in range(-m, 0)]
    assert len(pts) == q
    return pts


def unit_vectors(dirs):
    """s_hat_i = d_i / |d_i| as a (Q, 2) float64 array (x, y)."""
    d = np.array(dirs, dtype=np.float64)
    return d / np.sqrt((d * d).sum(axis=1, keepdims=True))


def direction_angles(dirs):
    return np.array([math.atan2(y, x) for (x, y) in dirs], dtype=np.float64)


def angular_weights(dirs):
    """Eq. weight, read as w_j = (gap to previous direction + gap to next) / (4 pi)."""
    th = direction_angles(dirs)
    q = len(dirs)
    w = np.empty(q)
    for j in range(q):
        prev_gap = (th[j] - th[j - 1]) % (2 * math.pi)
        next_gap = (th[(j + 1) % q] - th[j]) % (2 * math.pi)
        w[j] = (prev_gap + next_gap) / (4 * math.pi)
    return w


def worm_path(direction):
    """Eq. worm-paths for one direction s = (a, b) with Chebyshev length M: the M basic
    hop indices K_{s,1..M}.  Squared distances are scaled by M^2 so that the comparison
    with the ray point (n/M) s is exact."""
    a, b = direction
    m = max(abs(a), abs(b))
    px, py = 0, 0
    path = []
    for n in range(1, m + 1):
        best = m * m          # the running best starts at distance 1 (scaled: M^2)
        choice = None
        for k, (cx, cy) in enumerate(BASIC_HOPS):
            dx = m * (px + cx) - n * a
            dy = m * (py + cy) - n * b
            d2 = dx * dx + dy * dy
            if d2 <= best:     # "<=": a later index wins a tie
                best = d2
                choice = k
        if choice is None:
            raise AssertionError("no basic hop within one spacing of the ray point")
        path.append(choice)
        px += BASIC_HOPS[choice][0]
        py += BASIC_HOPS[choice][1]
    return path


def worm_table(dirs):
    return [worm_path(d) for d in dirs]


def mean_hop_length(path):
    """c_i of Eq. W-correction-factor-generalized: average length of one basic hop."""
    total = 0.0
    for k in path:
        cx, cy = BASIC_HOPS[k]
        total += math.sqrt(cx * cx + cy * cy)
    return total / len(path)


def lambda_corr(dirs):
    """Eq. W-correction-factor-generalized: Q / sum_i c_i."""
    paths = worm_table(dirs)
    return len(dirs) / sum(mean_hop_length(p) for p in paths)


def w_corr(w, lam_corr, emulate_3d):
    """Eq. W-correction.  The 3/2 factor is applied only when a 2D run emulates 3D."""
    f = 1.5 if emulate_3d else 1.0
    return f * ((1.0 - w) * w + w * (w * lam_corr))


def relax_weight(mfp_cells, lam_corr, emulate_3d, relax_mode=0):
    """Per-cell relaxation weight used in the update.  W = dt/tau = 1/MFP (Eq. W-Kn, in
    lattice units), then Eq. W-correction.  relax_mode 1 is an opt-in extension outside
    the paper (W_eff = 1 - exp(-W_corr)) that stays stable for MFP < 1 cell."""
    w = 1.0 / np.asarray(mfp_cells, dtype=np.float64)
    wc = w_corr(w, lam_corr, emulate_3d)
    if relax_mode == 1:
        wc = 1.0 - np.exp(-wc)
    return wc


def e_eq(t, theta):
    """Gray equilibrium energy density, Eq. gray-energy-density, with the prefactor
    3 N hbar omega0 / V set to one (it cancels from every temperature)."""
    return 1.0 / np.expm1(theta / np.asarray(t, dtype=np.float64))


def temperature(e, theta):
    """Eq. pseudo-T with the same unit prefactor: T = theta / ln(1 + 1/e)."""
    return theta / np.log1p(1.0 / np.asarray(e, dtype=np.float64))


class TasSchedule:
    """Eq. algorithm + worm paths: per-direction displacement p_i, executed-hop counter
    h_i.  ``advance(n)`` performs step n (n = 1, 2, ...) and returns, for every direction,
    the due basic hop index and whether the DDED is paused at this step.

    speed v in (0, 1]: the propagation speed in cells per step (the TAS extended to other
    speeds, Sec. 1): the axial reference distance after step n is v n, so the hop test
    reads |p + c|^2 <= (v n + 1)^2, evaluated in float64 as written (v = 1 gives the exact
    integer test of the unit speed)."""

    def __init__(self, q, speed=1.0):
        self.dirs = ring_directions(q)
        self.paths = worm_table(self.dirs)
        self.m = q // 8
        self.p = [[0, 0] for _ in range(q)]
        self.h = [0] * q
        self.n = 0
        self.speed = float(speed)
        if not (0.0 < self.speed <= 1.0):
            raise ValueError("speed must lie in (0, 1]")

    def advance(self, n=None):
        n = self.n + 1 if n is None else n
        assert n == self.n + 1, "steps must be taken in order"
        hops, paused = [], []
        for i in range(len(self.dirs)):
            k = self.paths[i][self.h[i] % self.m]
            cx, cy = BASIC_HOPS[k]
            nx_, ny_ = self.p[i][0] + cx, self.p[i][1] + cy
            r = self.speed * n + 1.0
            if nx_ * nx_ + ny_ * ny_ <= r * r:
                self.p[i] = [nx_, ny_]
                self.h[i] += 1
                paused.append(False)
            else:
                paused.append(True)
            hops.append(k)
        self.n = n
        return hops, paused

    def displacement(self):
        return np.array(self.p, dtype=np.int64)
