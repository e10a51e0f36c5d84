"""Oracle, part 5: analytic reference solutions of the paper's validation cases, numpy
float64.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  cross_plane_fourier   transient 1D heat conduction between walls at T_h (x = 0) and T_c
                        (x = L), start at T_c (Sec. 4.4, Eq. 1DT): Fourier sine series of
                        Theta = (T - T_c)/(T_h - T_c) in X = x/L and the diffusion time
                        s = D t / L^2 (the paper's Kn xi / 3).
  ballistic_cross_plane_2d   2D ballistic front from a wall (Sec. 4.4, Eq. 1D-ball-2D): a
                        point at distance x from the wall at time t sees the wall's energy
                        over the angles |theta| < arccos(x / (v t)) and the initial
                        energy elsewhere; returns the local energy.
  ballistic_cross_plane_worm  the same for the discrete directions of the worm lattice
                        (W = 0): direction i carries the wall's w_i e(T_w) to x once its
                        worm displacement along x exceeds x (a pure function of the TAS
                        schedule of Eq. algorithm).
  one_pixel_worm        the "one-pixel source" of Sec. 4.2 at W = 0 on a periodic grid: a
                        direction carries the source's value at x exactly when its path
                        back in time passes the source cell at a step before n, i.e.
                        x - s = p_i(n) - p_i(k) (mod the grid) for some 0 <= k < n.
  disk_ballistic_2d     2D ballistic spreading of a uniform disk (Sec. 4.2, the circular
                        initial condition): the angular fraction of the circle of radius
                        v t around a point that lies inside the disk.
  one_hot_three_cold    2D steady heat conduction on the unit square, Theta = 1 on the hot
                        edge Y = 1 and 0 on the other three (Sec. 4.6, Eq. 2DT): Fourier
                        sine series in X with sinh profiles in Y.

Pins: tests/test_oracle_analytic.py (boundary values, steady limits, harmonicity by finite
differences, the discrete ballistic and one-pixel profiles against the oracle stepper at
W = 0, the small-disk limit of the disk front).
"""
import math

import numpy as np

from . import lattice as L


def cross_plane_fourier(X, s, terms=2000):
    """Theta(X, s) = 1 - X - (2/pi) sum_l sin(l pi X) exp(-l^2 pi^2 s) / l."""
    X = np.asarray(X, np.float64)
    out = 1.0 - X
    for l in range(1, terms + 1):
        decay = math.exp(-(l * math.pi) ** 2 * s)
        if decay < 1e-18:
            break
        out = out - (2.0 / math.pi) * np.sin(l * math.pi * X) * decay / l
    return out


def ballistic_cross_plane_2d(x, t, e_wall, e_init, v=1.0):
    """Local energy e_init + (theta_W / pi)(e_wall - e_init), theta_W = arccos(x / (v t))
    where v t > x, else e_init (the angle average of the paper's expression)."""
    x = np.asarray(x, np.float64)
    r = v * t
    theta = np.where(r > x, np.arccos(np.clip(x / max(r, 1e-300), -1.0, 1.0)), 0.0)
    return e_init + theta / math.pi * (e_wall - e_init)


def ballistic_cross_plane_worm(q, n, nx, de_wall):
    """E(x) - e_init after n steps, x = 0..nx-1, for walls at x = -1 (energy deviation
    de_wall) and x = nx (at the initial energy), W = 0: direction i contributes
    w_i de_wall where its x displacement p_ix(n) > x."""
    dirs = L.ring_directions(q)
    w = L.angular_weights(dirs)
    sched = L.TasSchedule(q)
    for _ in range(n):
        sched.advance()
    px = sched.displacement()[:, 0]
    x = np.arange(nx)
    return (w[:, None] * (px[:, None] > x[None, :])).sum(axis=0) * de_wall


def one_hot_three_cold(X, Y, terms=400):
    """Theta(X, Y) = sum_l 2 (1 - cos(l pi)) / (l pi sinh(l pi)) sin(l pi X) sinh(l pi Y),
    summed with sinh(l pi Y)/sinh(l pi) = exp(-l pi (1 - Y)) (1 - exp(-2 l pi Y)) /
    (1 - exp(-2 l pi)) to avoid overflow."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    out = np.zeros(np.broadcast(X, Y).shape)
    for l in range(1, terms + 1, 2):            # 1 - cos(l pi) = 2 for odd l, 0 for even
        k = l * math.pi
        ratio = np.exp(-k * (1.0 - Y)) * (-np.expm1(-2.0 * k * Y)) / (-math.expm1(-2.0 * k))
        out = out + 4.0 / k * np.sin(k * X) * ratio
    return out


def one_pixel_worm(q, n, nx, ny, src, de_src, de_init=0.0):
    """E(x, y) - e_ref after n steps, array (ny, nx): source cell src = (x, y) kept at the
    isotropic deviation de_src, the rest starting at de_init, W = 0, periodic grid."""
    dirs = L.ring_directions(q)
    w = L.angular_weights(dirs)
    sched = L.TasSchedule(q)
    path = [sched.displacement().copy()]
    for _ in range(n):
        sched.advance()
        path.append(sched.displacement().copy())
    pn = path[-1]
    e = np.zeros((ny, nx))
    for i in range(q):
        hit = np.zeros((ny, nx), bool)
        for k in range(n):
            dx, dy = pn[i] - path[k][i]
            hit[(src[1] + dy) % ny, (src[0] + dx) % nx] = True
        e += w[i] * np.where(hit, de_src, de_init)
    return e


def disk_ballistic_2d(r, t, radius, v=1.0):
    """Fraction of the directions from a point at distance r from the disk centre whose
    point at distance v t lies inside the disk of the given radius (the ballistic
    temperature rise over the disk's, as a fraction)."""
    r = np.asarray(r, np.float64)
    s = v * t
    if s == 0:
        return (r < radius).astype(np.float64)
    full = (r + s <= radius)
    part = (np.abs(r - s) < radius) & ~full
    with np.errstate(invalid="ignore", divide="ignore"):
        c = (r * r + s * s - radius * radius) / (2.0 * r * s)
    out = np.where(full, 1.0, np.where(part, np.arccos(np.clip(c, -1.0, 1.0)) / math.pi, 0.0))
    return out
