"""Pins of the analytic reference solutions of the paper's validation cases (CPU only):
boundary values, limits, an independent closed form (the short-time erfc profile), the
exact centre value of the one-hot square, harmonicity by finite differences, and the
discrete ballistic profile against the oracle stepper."""
import math

import numpy as np
import pytest

from oracle import analytic as AN
from oracle import lattice as L
from oracle.stepper import WormLBM, PERIODIC as P, ISOTHERMAL as I


def test_cross_plane_fourier_limits_and_short_time():
    X = np.linspace(0.05, 0.95, 19)
    np.testing.assert_allclose(AN.cross_plane_fourier(X, 5.0), 1 - X, atol=1e-14)
    assert AN.cross_plane_fourier(0.0, 0.3) == pytest.approx(1.0, abs=1e-14)
    # short times: the semi-infinite solution erfc(X / (2 sqrt(s))) near the hot wall
    s = 1e-4
    for x in (0.005, 0.01, 0.02):
        assert AN.cross_plane_fourier(x, s) == pytest.approx(math.erfc(x / (2 * math.sqrt(s))),
                                                             abs=2e-4)


def test_ballistic_2d_limits():
    assert AN.ballistic_cross_plane_2d(10.0, 5.0, 1.0, 0.0) == 0.0       # front not there
    assert AN.ballistic_cross_plane_2d(1e-9, 5.0, 1.0, 0.0) == pytest.approx(0.5, abs=1e-9)
    assert AN.ballistic_cross_plane_2d(2.5, 5.0, 1.0, 0.0) == pytest.approx(1 / 3, abs=1e-12)


def test_ballistic_worm_profile_equals_oracle_stepper():
    """W = 0 between isothermal walls, periodic y: the oracle's field equals the profile
    computed from the TAS displacements alone."""
    nx, q, n = 40, 32, 30
    m = WormLBM(nx, 1, q, 1.0, bc_kind=(I, I, P, P), t_wall=(300.5, 300.0, 300.0, 300.0),
                w_field=0.0)
    m.init_temperature(np.zeros((1, nx)))
    m.step(n)
    want = AN.ballistic_cross_plane_worm(q, n, nx, m.delta_e(300.5))
    np.testing.assert_allclose(m.energy_dev()[0], want, rtol=0, atol=1e-15)


def test_one_hot_three_cold():
    X = np.linspace(0.1, 0.9, 9)
    np.testing.assert_allclose(AN.one_hot_three_cold(X, 0.0), 0.0, atol=1e-15)
    np.testing.assert_allclose(AN.one_hot_three_cold(0.0, X), 0.0, atol=1e-12)
    # on the hot edge the series is a square wave's partial sum (slow near the corners)
    np.testing.assert_allclose(AN.one_hot_three_cold(X[2:-2], 1.0), 1.0, atol=5e-3)
    # by superposition of the four rotated problems the centre is exactly 1/4
    assert AN.one_hot_three_cold(0.5, 0.5) == pytest.approx(0.25, abs=1e-12)
    assert AN.one_hot_three_cold(0.3, 0.6) == pytest.approx(AN.one_hot_three_cold(0.7, 0.6),
                                                            abs=1e-14)
    h = 1e-3
    for (x, y) in [(0.3, 0.4), (0.6, 0.8), (0.5, 0.2)]:
        lap = (AN.one_hot_three_cold(x + h, y) + AN.one_hot_three_cold(x - h, y)
               + AN.one_hot_three_cold(x, y + h) + AN.one_hot_three_cold(x, y - h)
               - 4 * AN.one_hot_three_cold(x, y)) / h ** 2
        assert abs(lap) < 1e-4


def test_one_pixel_exact_profile_equals_oracle_stepper():
    """Sec. 4.2: a pixel kept at a higher temperature in a periodic grid; at W = 0 the
    oracle's field equals the profile built from the TAS displacements alone."""
    nx = ny = 21
    q, n, src = 16, 15, (10, 10)
    m = WormLBM(nx, ny, q, 1.0, w_field=0.0)
    m.init_temperature(np.zeros((ny, nx)))
    m.set_sources([src], temps=[301.0])
    m.step(n)
    want = AN.one_pixel_worm(q, n, nx, ny, src, m.delta_e(301.0))
    np.testing.assert_allclose(m.energy_dev(), want, rtol=0, atol=1e-15)


def test_radiation_cells_on_a_wall_equal_an_isothermal_wall():
    """Sources on the ghost cells of a wall with imposed e_i = w_i e_eq(T_w) (Eq.
    anisotropic with isotropic values) reproduce the isothermal wall (Eq. isotropic)."""
    nx, ny, q = 14, 9, 24
    dT = np.random.default_rng(2).standard_normal((ny, nx)) * 0.3
    a = WormLBM(nx, ny, q, 3.0, bc_kind=(I, I, P, P), t_wall=(300.7, 300.0, 300.0, 300.0))
    b = WormLBM(nx, ny, q, 3.0, bc_kind=(2, I, P, P), t_wall=(300.0, 300.0, 300.0, 300.0))
    e_w = L.e_eq(300.7, a.theta)
    b.set_sources([(-1, y) for y in range(ny)], imposed=[a.w * e_w] * ny)
    for m in (a, b):
        m.init_temperature(dT)
        m.step(40)
    np.testing.assert_allclose(b.d[:, 1:-1, 1:-1], a.d[:, 1:-1, 1:-1], rtol=0, atol=1e-15)


def test_sources_refuse_periodic_ghosts_and_outside_cells():
    m = WormLBM(6, 5, 8, 2.0, bc_kind=(P, P, I, I))
    with pytest.raises(ValueError):
        m.set_sources([(-1, 2)], temps=[301.0])
    with pytest.raises(ValueError):
        m.set_sources([(3, 7)], temps=[301.0])
    m.set_sources([(2, -1), (3, 5)], temps=[301.0, 299.0])     # isothermal ghosts: fine


def test_disk_ballistic_limits():
    assert AN.disk_ballistic_2d(0.0, 5.0, 10.0) == pytest.approx(1.0)   # still inside
    assert AN.disk_ballistic_2d(0.0, 15.0, 10.0) == pytest.approx(0.0)  # centre emptied
    # a point at r = v t far from a small disk: an arc of length ~ 2R of the circle of
    # radius v t lies in the disk, the fraction R / (pi v t)
    r, R = 2000.0, 5.0
    assert AN.disk_ballistic_2d(r, r, R) == pytest.approx(R / (math.pi * r), rel=1e-4)
