"""Oracle, part 4: effective conductivity and steady-state residual, plain numpy float64.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper reports the in-plane thermal conductivity of films relative to the bulk value
and compares it with the Fuchs-Sondheimer ratio (Sec. 4.5); it calls its conductivity
"apparent" (Sec. 1) and does not print how it extracts it, nor a steady-state test.
These functions fix one reading each, in lattice units (cell = step = v_g = 1):

  bulk diffusivity     D = Lambda / 3 for a 2D run that emulates 3D (the factor 3/2 of
                       Eq. W-correction), D = Lambda / 2 otherwise; the bulk
                       conductivity is C D, and with e = energy density C dT = de.
  apparent kappa       kappa_app / kappa_bulk = <q_x> N_x / (D (e(T_x-) - e(T_x+))):
                       mean heat flux over the interior (Eq. q_corr) against the
                       temperatures imposed by isothermal walls at x = -1 and x = N_x
                       (the wall faces are N_x cells apart).
  band kappa           kappa_band / kappa_bulk = <q_x>_band / (-D dE/dx): flux and
                       least-squares slope of the y-averaged local energy, both over the
                       central band of columns x0 <= x < x0 + m, x0 = floor(N_x/4),
                       m = floor(N_x/2); free of the wall jumps of the apparent value.
  residual             max over interior cells of |T^n(x) - T^m(x)| / (n - m), K/step.
  steady run           the TAS pauses make the field fluctuate from step to step (Sec.
                       4.3), so a steady-state check compares window means: every check
                       runs C steps, the last K of them averaged; the residual is the
                       largest change of the window-mean temperature per step between
                       consecutive checks, and the flux outputs are window means.

Reference ratios (Sec. 4.5):
  fuchs_sondheimer_3d  the textbook diffuse-wall (specularity 0) film ratio
                       1 - (3 Kn / 2) int_1^inf (t^-3 - t^-5)(1 - exp(-t/Kn)) dt.
  fuchs_sondheimer_2d  the same ratio for the discrete directions of the lattice in a 2D
                       film: direction i at angle theta_i carries w_i cos^2 theta_i of the
                       bulk conductivity, reduced by the thickness average of
                       1 - exp(-distance to its emitting wall / (Kn |sin theta_i|)).

Pins: tests/test_oracle_transport.py (closed-form first-moment state, exact ballistic
conductance sum_{cos > 0} w_i cos theta_i, diffusive bulk band kappa = 1, the oracle film
converging under grid refinement to fuchs_sondheimer_2d, the asymptotes of both ratios).
"""
import math

import numpy as np
from scipy import integrate

from . import lattice as L
from .stepper import ISOTHERMAL, XM, XP


def bulk_diffusivity(mfp, emulate_3d=True, speed=1.0):
    """D = v_g Lambda / 3 (3D) or v_g Lambda / 2 (2D), lattice units (v_g = speed)."""
    return float(speed) * float(mfp) / (3.0 if emulate_3d else 2.0)


def band_columns(nx):
    """(x0, m): the central band of columns x0 <= x < x0 + m."""
    return nx // 4, nx // 2


def band_flux_and_slope(m):
    """(<q_x> over the band, least-squares slope of the y-averaged E - e_ref over the
    band) of a WormLBM model; NaN slope for a band of fewer than two columns."""
    x0, w = band_columns(m.nx)
    qx, _ = m.heat_flux()
    if w < 1:
        return float("nan"), float("nan")
    q_band = float(qx[:, x0:x0 + w].mean())
    if w < 2:
        return q_band, float("nan")
    e_bar = m.energy_dev()[:, x0:x0 + w].mean(axis=0)      # y-averaged E per column
    xc = np.arange(x0, x0 + w, dtype=np.float64) - (x0 + (w - 1) / 2.0)
    slope = (xc * (e_bar - e_bar.mean())).sum() / (xc * xc).sum()
    return q_band, float(slope)


def kappa_apparent(m, mfp, emulate_3d=True):
    """kappa_app / kappa_bulk, or NaN unless both x walls are isothermal at different
    temperatures."""
    k = m.bc_kind
    if k[XM] != ISOTHERMAL or k[XP] != ISOTHERMAL or m.t_wall[XM] == m.t_wall[XP]:
        return float("nan")
    de = float(L.e_eq(m.t_wall[XM], m.theta) - L.e_eq(m.t_wall[XP], m.theta))
    qx, _ = m.heat_flux()
    return float(qx.mean()) * m.nx / (bulk_diffusivity(mfp, emulate_3d, m.speed) * de)


def kappa_band(m, mfp, emulate_3d=True):
    """kappa_band / kappa_bulk, NaN where the band slope is zero or undefined."""
    q_band, slope = band_flux_and_slope(m)
    if not (slope != 0.0):
        return float("nan")
    return q_band / (-bulk_diffusivity(mfp, emulate_3d, m.speed) * slope)


def temperature_residual(dT_now, dT_then, steps):
    """max |T^n - T^m| / (n - m) over the cells, in K per step."""
    if steps <= 0:
        return float("nan")
    return float(np.abs(np.asarray(dT_now) - np.asarray(dT_then)).max()) / steps


def fuchs_sondheimer_3d(kn):
    """Diffuse-wall Fuchs-Sondheimer in-plane ratio kappa_film / kappa_bulk, Kn =
    Lambda / thickness.  With u = 1/t the integral is int_0^1 (u - u^3)(1 - exp(-1/(Kn u)))
    du, smooth on [0, 1]."""
    kn = float(kn)
    f = lambda u: (u - u ** 3) * (-math.expm1(-1.0 / (kn * u))) if u > 0 else 0.0
    val, _ = integrate.quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=200)
    return 1.0 - 1.5 * kn * val


def fuchs_sondheimer_2d(q, kn, p=0.0):
    """Fuchs-Sondheimer ratio of a 2D film for the Q lattice directions and weights:
    sum_i w_i c_i^2 g(Kn |s_i|) / sum_i w_i c_i^2 with (c_i, s_i) = (cos, sin) of
    direction i and, for walls of specularity p,
    g(a) = 1 - a (1 - p)(1 - exp(-1/a)) / (1 - p exp(-1/a)), g(0) = 1 (directions along
    the film never meet a wall): the deviation carried across the film by a direction
    restarts from p times its mirror image at each wall."""
    dirs = L.ring_directions(q)
    u = L.unit_vectors(dirs)
    w = L.angular_weights(dirs)
    c2, s = u[:, 0] ** 2, np.abs(u[:, 1])
    g = np.ones(q)
    for i in range(q):
        a = kn * s[i]
        if a > 0:
            u = -math.expm1(-1.0 / a)             # 1 - exp(-1/a), also for large a
            g[i] = 1.0 - a * (1.0 - p) * u / ((1.0 - p) + p * u)
    return float((w * c2 * g).sum() / (w * c2).sum())


def run_steady(m, max_steps, check_every, tol, avg_steps, mfp, emulate_3d=True):
    """Steady-state run of a WormLBM model by window means (reading above).  Returns
    (steps, converged, residual, means) with means = (<q_x>, <q_y>, <q_x>_band, slope,
    kappa_app, kappa_band) from the window means of the last check."""
    steps, conv, residual, prev = 0, False, float("nan"), None
    means = None
    while steps + check_every <= max_steps and not conv:
        m.step(check_every - avg_steps)
        t_sum, vals = 0.0, []
        for _ in range(avg_steps):
            m.step(1)
            t_sum = t_sum + m.temperature_dev()
            qx, qy = m.heat_flux()
            vals.append((float(qx.mean()), float(qy.mean())) + band_flux_and_slope(m))
        steps += check_every
        t_mean = t_sum / avg_steps
        residual = temperature_residual(t_mean, prev, check_every) if prev is not None \
            else float("nan")
        prev = t_mean
        conv = residual <= tol
        means = tuple(float(np.mean([v[k] for v in vals])) for k in range(4))
    qx_m, qy_m, qb, slope = means
    d = bulk_diffusivity(mfp, emulate_3d, m.speed)
    k = m.bc_kind
    if k[XM] == ISOTHERMAL and k[XP] == ISOTHERMAL and m.t_wall[XM] != m.t_wall[XP]:
        de = float(L.e_eq(m.t_wall[XM], m.theta) - L.e_eq(m.t_wall[XP], m.theta))
        k_app = qx_m * m.nx / (d * de)
    else:
        k_app = float("nan")
    k_band = qb / (-d * slope) if slope != 0.0 else float("nan")
    return steps, conv, residual, (qx_m, qy_m, qb, slope, k_app, k_band)
