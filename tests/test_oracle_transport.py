"""Pins of the oracle's conductivity and steady-state functions (CPU only).  Each checks
a value fixed another way: a closed-form state, the exact ballistic steady state, the
diffusive limit, the Fuchs-Sondheimer limit of the film under grid refinement, textbook
asymptotes and the percentages the paper prints (Sec. 4.5)."""
import math
import pathlib

import numpy as np
import pytest

from oracle import lattice as L
from oracle import transport as T
from oracle.stepper import WormLBM, PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR

P, I, A = PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE
GOLDEN = pathlib.Path(__file__).parent / "golden"
EULER_GAMMA = 0.5772156649015329


def _bose(t, theta=L.THETA_DEFAULT):
    return 1.0 / math.expm1(theta / t)


def _linear_start(m):
    """Warm start: T falls linearly from +0.5 K to -0.5 K across the x extent."""
    xs = (np.arange(m.nx) + 0.5) / m.nx
    m.init_temperature(np.tile(0.5 - xs, (m.ny, 1)))


def _band_kappa_mean(m, mfp, steps, every):
    vals = []
    for _ in range(steps // every):
        m.step(every)
        vals.append(T.kappa_band(m, mfp))
    return float(np.mean(vals))


def test_first_moment_state_closed_form():
    """d_i = w_i (a + b x) + alpha w_i s_ix: by the quarter-turn symmetry of the ring,
    sum_i w_i s_ix = 0 and sum_i w_i s_ix^2 = 1/2, so E = a + b x and q_x = alpha / 2
    everywhere; the band slope is b and both conductivities follow in closed form."""
    nx, ny, q, mfp = 20, 6, 16, 6.0
    tw = (300.5, 299.5, 300.0, 300.0)
    m = WormLBM(nx, ny, q, mfp, bc_kind=(I, I, P, P), t_wall=tw)
    a, b, alpha = 3e-3, -2e-4, 5e-4
    x = np.arange(-1, nx + 1, dtype=np.float64)[None, None, :]
    d = m.w[:, None, None] * (a + b * x) + alpha * (m.w * m.s_hat[:, 0])[:, None, None]
    m.set_state(np.broadcast_to(d, (q, ny + 2, nx + 2)))
    qx, _ = m.heat_flux()
    np.testing.assert_allclose(qx, alpha / 2, rtol=1e-13)
    q_band, slope = T.band_flux_and_slope(m)
    assert q_band == pytest.approx(alpha / 2, rel=1e-13)
    assert slope == pytest.approx(b, rel=1e-11)
    dd = mfp / 3.0
    assert T.kappa_band(m, mfp) == pytest.approx((alpha / 2) / (-dd * b), rel=1e-11)
    de = _bose(tw[0]) - _bose(tw[1])
    assert T.kappa_apparent(m, mfp) == pytest.approx((alpha / 2) * nx / (dd * de), rel=1e-12)
    # 2D diffusivity without the 3D emulation factor
    assert T.kappa_band(m, mfp, emulate_3d=False) == pytest.approx(
        (alpha / 2) / (-(mfp / 2.0) * b), rel=1e-11)


def test_band_columns_are_the_central_half():
    assert T.band_columns(4096) == (1024, 2048)
    assert T.band_columns(7) == (1, 3)


def test_ballistic_conductance_is_exact():
    """W = 0 between isothermal walls, periodic y: once every direction that moves in x
    has crossed the grid, it carries its emitting wall's w_i e(T_w) everywhere, so
    <q_x> = (e(T_h) - e(T_c)) sum over cos > 0 of w_i cos(theta_i)."""
    nx, ny, q = 12, 4, 16
    tw = (301.0, 299.0, 300.0, 300.0)
    m = WormLBM(nx, ny, q, 1.0, bc_kind=(I, I, P, P), t_wall=tw, w_field=0.0)
    m.init_temperature(np.zeros((ny, nx)))
    m.step(80)
    c = m.s_hat[:, 0]
    g = float((m.w * c)[c > 0].sum())
    de = _bose(tw[0]) - _bose(tw[1])
    qx, _ = m.heat_flux()
    np.testing.assert_allclose(qx, g * de, rtol=1e-12)
    mfp = 3.0                                   # D = 1: kappa_app = G N_x
    assert T.kappa_apparent(m, mfp) == pytest.approx(g * nx, rel=1e-12)
    _, slope = T.band_flux_and_slope(m)         # uniform E: no band slope
    assert abs(slope) <= 1e-14 * abs(m.energy_dev()).max()


def test_apparent_kappa_needs_two_isothermal_x_walls():
    m = WormLBM(8, 4, 8, 2.0)
    m.init_temperature(np.zeros((4, 8)))
    assert math.isnan(T.kappa_apparent(m, 2.0))
    m = WormLBM(8, 4, 8, 2.0, bc_kind=(I, I, A, A), t_wall=(300.0,) * 4)
    assert math.isnan(T.kappa_apparent(m, 2.0))


def test_diffusive_bulk_band_kappa_extrapolates_to_one():
    """Bulk (periodic y) between isothermal ends: the band conductivity approaches the
    Fourier value C Lambda / 3 with first-order error in 1/Lambda (the grid-MFP
    correction of Eq. W-correction; Sec. 4.1); Richardson extrapolation over Lambda =
    8, 16 lands on 1."""
    k = {}
    for mfp in (8.0, 16.0):
        nx = int(8 * mfp)
        m = WormLBM(nx, 2, 16, mfp, bc_kind=(I, I, P, P), t_wall=(300.5, 299.5, 300, 300))
        _linear_start(m)
        m.step(400)
        k[mfp] = _band_kappa_mean(m, mfp, 200, 1)
    assert abs(k[16.0] - 1) < abs(k[8.0] - 1)
    assert 2 * k[16.0] - k[8.0] == pytest.approx(1.0, abs=0.01)


def test_film_converges_to_discrete_fuchs_sondheimer():
    """Adiabatic-diffuse walls at y = 0 and y = N_y (Sec. 2.6), Kn = Lambda / N_y = 1,
    3D emulation (effective 2D MFP 2 Lambda / 3): the film-to-bulk ratio of the band
    conductivity converges to first order in 1/N_y (Sec. 4.5 observes first-order grid
    convergence) towards the discrete-ordinate Fuchs-Sondheimer ratio of the same
    directions and weights."""
    q, kn = 32, 1.0
    ratio = {}
    for ny in (8, 16):
        mfp, nx = kn * ny, 8 * ny
        k = {}
        for name, bc in (("bulk", (I, I, P, P)), ("film", (I, I, A, A))):
            m = WormLBM(nx, ny, q, mfp, bc_kind=bc, t_wall=(300.5, 299.5, 300, 300))
            _linear_start(m)
            m.step(600)
            k[name] = _band_kappa_mean(m, mfp, 400, 10)
        ratio[ny] = k["film"] / k["bulk"]
    fs = T.fuchs_sondheimer_2d(q, kn * 2.0 / 3.0)
    assert abs(ratio[16] - fs) < abs(ratio[8] - fs)
    assert 2 * ratio[16] - ratio[8] == pytest.approx(fs, rel=0.01)


def test_fuchs_sondheimer_3d_asymptotes():
    """Textbook limits of the diffuse-wall FS ratio: 1 - 3 Kn / 8 for thick films and
    (3 / (4 Kn)) (ln Kn + 1 - gamma) for thin ones."""
    for kn in (1e-3, 1e-2):
        assert T.fuchs_sondheimer_3d(kn) == pytest.approx(1 - 3 * kn / 8, abs=1e-12)
    for kn in (1e4, 1e5):
        want = 3 / (4 * kn) * (math.log(kn) + 1 - EULER_GAMMA)
        assert T.fuchs_sondheimer_3d(kn) == pytest.approx(want, rel=2e-5)
    vals = [T.fuchs_sondheimer_3d(kn) for kn in (0.1, 1.0, 5.0, 20.0)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_fuchs_sondheimer_2d_limits():
    """Thick film: 1 - Kn int cos^2 |sin| / int cos^2 = 1 - 4 Kn / (3 pi) as the
    directions fill the circle.  Thin film: only directions along the film survive, so
    D2Q8 tends to 4 w_axial = 1/2 (Sec. 4.5: the axial direction never meets a wall)."""
    for q in (256, 1024):
        slope = (1 - T.fuchs_sondheimer_2d(q, 1e-3)) / 1e-3
        assert slope == pytest.approx(4 / (3 * math.pi), rel=2.0 / q)
    assert T.fuchs_sondheimer_2d(8, 1e9) == pytest.approx(0.5, abs=1e-8)
    assert T.fuchs_sondheimer_2d(64, 1e-12) == pytest.approx(1.0, abs=1e-11)


def test_fuchs_sondheimer_matches_printed_percentages():
    """Sec. 4.5 prints the D2Q8 overestimate of the FS value at Kn = 20 and the remaining
    Q = 128 vs Q = 256 difference there; the discrete-ordinate ratio of the 3D-emulating
    lattice (Kn' = 2 Kn / 3) against the 3D FS ratio reproduces both."""
    rows = {}
    for line in (GOLDEN / "fs_inplane_paper.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, kn, val, tol = line.split()
            rows[name] = (float(kn), float(val), float(tol))
    kn, val, tol = rows["d2q8_over_fs_percent"]
    got = 100 * (T.fuchs_sondheimer_2d(8, 2 * kn / 3) / T.fuchs_sondheimer_3d(kn) - 1)
    assert abs(got - val) <= tol
    kn, val, tol = rows["q128_vs_q256_percent"]
    got = 100 * (T.fuchs_sondheimer_2d(128, 2 * kn / 3) / T.fuchs_sondheimer_2d(256, 2 * kn / 3) - 1)
    assert abs(got - val) <= tol


def test_temperature_residual():
    """Residual of a uniform equilibrium is exactly zero; for a ballistic (W = 0) periodic
    run it equals the largest change of the exactly translated temperature field
    E(n) = sum_i w_i e0(x - p_i(n)) per step."""
    m = WormLBM(10, 10, 16, 4.0)
    m.init_temperature(np.full((10, 10), 0.3))
    t0 = m.temperature_dev()
    m.step(7)
    assert T.temperature_residual(m.temperature_dev(), t0, 7) == 0.0
    assert math.isnan(T.temperature_residual(t0, t0, 0))

    nx = ny = 24
    q = 16
    yy, xx = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((xx - 11.3) ** 2 + (yy - 12.6) ** 2) / (2 * 3.0 ** 2))
    m = WormLBM(nx, ny, q, 1.0, w_field=0.0)
    m.init_temperature(dT0)
    e0 = L.e_eq(300.0 + dT0, m.theta) - m.e_ref
    sched = L.TasSchedule(q)

    def exact_temperature(disp):
        e = sum(m.w[i] * np.roll(e0, (disp[i][1], disp[i][0]), axis=(0, 1)) for i in range(q))
        return L.temperature(m.e_ref + e, m.theta) - 300.0

    for _ in range(5):
        sched.advance()
    t5 = exact_temperature(sched.displacement())
    for _ in range(4):
        sched.advance()
    t9 = exact_temperature(sched.displacement())
    m.step(5)
    a = m.temperature_dev()
    m.step(4)
    b = m.temperature_dev()
    want = np.abs(t9 - t5).max() / 4
    assert T.temperature_residual(b, a, 4) == pytest.approx(want, rel=1e-9)


def test_run_steady_windows():
    """Window means: a uniform equilibrium is steady at the second check (residual 0);
    for a ballistic periodic run the residual of the second check is the largest change
    per step of the exactly translated temperature averaged over steps 10-12 against
    steps 4-6 (checks of 6 steps, windows of 3)."""
    m = WormLBM(12, 10, 16, 4.0)
    m.init_temperature(np.full((10, 12), -0.2))
    steps, conv, res, _ = T.run_steady(m, 400, 100, 0.0, 10, 4.0)
    assert (steps, conv, res) == (200, True, 0.0)

    nx = ny = 20
    q = 16
    yy, xx = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((xx - 9.4) ** 2 + (yy - 10.2) ** 2) / (2 * 2.5 ** 2))
    m = WormLBM(nx, ny, q, 1.0, w_field=0.0)
    m.init_temperature(dT0)
    e0 = L.e_eq(300.0 + dT0, m.theta) - m.e_ref
    sched = L.TasSchedule(q)
    temps = []
    for _ in range(12):
        sched.advance()
        disp = sched.displacement()
        e = sum(m.w[i] * np.roll(e0, (disp[i][1], disp[i][0]), axis=(0, 1)) for i in range(q))
        temps.append(L.temperature(m.e_ref + e, m.theta) - 300.0)
    w1 = (temps[3] + temps[4] + temps[5]) / 3.0
    w2 = (temps[9] + temps[10] + temps[11]) / 3.0
    steps, conv, res, _ = T.run_steady(m, 12, 6, 0.0, 3, 1.0)
    assert steps == 12 and not conv
    assert res == pytest.approx(np.abs(w2 - w1).max() / 6, rel=1e-9)


@pytest.mark.parametrize("p,kind", [(0.5, ADIABATIC_DIFFUSE), (1.0, ADIABATIC_SPECULAR)])
def test_specular_film_converges_to_fuchs_sondheimer(p, kind):
    """Partly specular walls (Sec. 2.6, the linear combination of the diffuse and specular
    rules) with specularity p: the film-to-bulk band conductivity converges to first order
    in 1/N_y to the discrete-ordinate ratio with specularity p; fully specular walls do
    not reduce the in-plane conductivity (ratio 1)."""
    q, kn = 32, 1.0
    ratio = {}
    for ny in (8, 16):
        mfp, nx = kn * ny, 8 * ny
        k = {}
        for name, bc in (("bulk", (I, I, P, P)), ("film", (I, I, kind, kind))):
            m = WormLBM(nx, ny, q, mfp, bc_kind=bc, t_wall=(300.5, 299.5, 300, 300),
                        specularity=(0.0, 0.0, p, p))
            _linear_start(m)
            m.step(600)
            k[name] = _band_kappa_mean(m, mfp, 400, 10)
        ratio[ny] = k["film"] / k["bulk"]
    fs = T.fuchs_sondheimer_2d(q, kn * 2.0 / 3.0, p)
    assert abs(ratio[16] - fs) < abs(ratio[8] - fs)
    assert 2 * ratio[16] - ratio[8] == pytest.approx(fs, rel=0.01)


def test_fuchs_sondheimer_2d_specularity_limits():
    """Specular walls leave every direction's conductivity intact (ratio 1); the
    thick-film slope scales with 1 - p."""
    for kn in (0.1, 1.0, 20.0):
        assert T.fuchs_sondheimer_2d(64, kn, 1.0) == pytest.approx(1.0, abs=1e-14)
    base = 1 - T.fuchs_sondheimer_2d(256, 1e-3)
    for p in (0.25, 0.5, 0.9):
        assert (1 - T.fuchs_sondheimer_2d(256, 1e-3, p)) == pytest.approx((1 - p) * base, rel=1e-6)
