"""Pins of the oracle's time step against what the paper and the mathematics fix
(CPU only).  None of these retypes the step: each checks a consequence computed another
way (a lattice translation, a convolution, moment recursions, conservation)."""
import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle.stepper import WormLBM, PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR

P, I, A, S = PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR


def _rand(ny, nx, seed):
    return np.random.default_rng(seed).standard_normal((ny, nx))


def test_energy_conserved_on_periodic_grid():
    """Eq. lbm-energy-density: scattering conserves energy; with periodic links the
    grid total is constant to round-off."""
    m = WormLBM(23, 19, 16, 3.0)
    m.init_temperature(_rand(19, 23, 1))
    e0 = m.total_energy()
    scale = np.abs(m.d).sum()
    for _ in range(60):
        m.step()
        assert abs(m.total_energy() - e0) <= 1e-13 * scale


@pytest.mark.parametrize("kinds,spec", [((A, A, A, A), (0, 0, 0, 0)),
                                       ((P, P, A, A), (0, 0, 0, 0)),
                                       ((A, A, P, P), (0, 0, 0, 0)),
                                       ((S, S, S, S), (0, 0, 0, 0)),
                                       ((A, S, A, A), (0.3, 0, 0.7, 1.0)),
                                       ((P, P, S, A), (0, 0, 0, 0.5))])
def test_energy_conserved_with_adiabatic_walls(kinds, spec):
    """Adiabatic walls (Sec. 2.6: diffuse, specular and their linear combinations) neither
    add nor remove energy: the total over the interior plus the wall cells stays
    constant."""
    m = WormLBM(21, 17, 32, 2.5, bc_kind=kinds, specularity=spec)
    m.init_temperature(_rand(17, 21, 2))
    m.apply_bc()
    e0 = m.total_energy(include_frame=True)
    scale = np.abs(m.d).sum()
    m.step(150)
    assert abs(m.total_energy(include_frame=True) - e0) <= 1e-13 * scale


@pytest.mark.parametrize("kinds", [(P, P, P, P), (I, I, A, A), (A, A, A, A),
                                   (I, I, P, P), (P, P, I, A), (A, I, I, A)])
def test_reference_equilibrium_is_a_fixed_point(kinds):
    """A uniform state at T_ref with all walls at T_ref stays exactly uniform: the
    update maps w_i e_ref to itself (sum w = 1)."""
    m = WormLBM(12, 10, 16, 2.0, bc_kind=kinds, t_wall=(300.0,) * 4)
    m.init_temperature(np.zeros((10, 12)))
    m.step(40)
    assert np.abs(m.d).max() == 0.0


@pytest.mark.parametrize("q", [8, 16, 32])
def test_ballistic_limit_translates_each_plane_exactly(q):
    """W = 0 (MFP -> infinity): each DDED only advects, so plane i after n steps is the
    initial plane translated by the cumulative worm displacement p_i(n) (Sec. 2.3-2.5);
    checked against np.roll on a periodic grid, bit for bit."""
    nx, ny = 29, 26
    m = WormLBM(nx, ny, q, None, w_field=0.0)
    rng = np.random.default_rng(q)
    d0 = np.zeros((q, ny + 2, nx + 2))
    d0[:, 1:-1, 1:-1] = rng.standard_normal((q, ny, nx))
    m.set_state(d0)
    ref = L.TasSchedule(q)
    for n in range(1, 41):
        m.step()
        ref.advance(n)
        p = ref.displacement()
        for i in range(q):
            want = np.roll(d0[i, 1:-1, 1:-1], shift=(p[i, 1], p[i, 0]), axis=(0, 1))
            assert np.array_equal(m.d[i, 1:-1, 1:-1], want)


def test_w_equal_one_reduces_to_standard_d2q8():
    """Sec. 2.3: at W = 1 only the EED evolves and the scheme is the standard D2Q8, i.e.
    E(n+1)(y) = 1/8 sum_k E(n)(y - c_k) over the 8 basic hops (pauses included, since
    the EED always hops)."""
    nx, ny = 20, 18
    m = WormLBM(nx, ny, 8, None, w_field=1.0)
    m.init_temperature(_rand(ny, nx, 3) * 0.3)
    e = m.energy_dev().copy()
    for _ in range(12):
        m.step()
        e = sum(np.roll(e, shift=(cy, cx), axis=(0, 1)) for (cx, cy) in L.BASIC_HOPS) / 8
        assert np.allclose(m.energy_dev(), e, rtol=0, atol=1e-15)


def _moment_recursion(q, w_uniform, steps, m0, m1x, m1y, m2x, speed=1.0):
    """Per-direction spatial moments propagated in moment space: sum_x d_i, sum_x x d_i,
    sum_x y d_i, sum_x x^2 d_i.  Translation by c shifts moments; scattering mixes
    directions through the totals.  Independent of the field code."""
    dirs = L.ring_directions(q)
    w = L.angular_weights(dirs)
    W = w_uniform
    sched = L.TasSchedule(q, speed)
    out = []
    for n in range(1, steps + 1):
        hops, paused = sched.advance(n)
        T0, T1x, T1y, T2x = m0.sum(), m1x.sum(), m1y.sum(), m2x.sum()
        g0 = (1 - W) * m0 + w * W * T0
        g1x = (1 - W) * m1x + w * W * T1x
        g1y = (1 - W) * m1y + w * W * T1y
        g2x = (1 - W) * m2x + w * W * T2x
        n0, n1x, n1y, n2x = g0.copy(), g1x.copy(), g1y.copy(), g2x.copy()
        for i in range(q):
            cx, cy = L.BASIC_HOPS[hops[i]]
            if paused[i]:    # only the scattered part moves
                n1x[i] = g1x[i] + cx * w[i] * W * T0
                n1y[i] = g1y[i] + cy * w[i] * W * T0
                n2x[i] = g2x[i] + w[i] * W * (2 * cx * T1x + cx * cx * T0)
            else:            # everything moves by c
                n1x[i] = g1x[i] + cx * g0[i]
                n1y[i] = g1y[i] + cy * g0[i]
                n2x[i] = g2x[i] + 2 * cx * g1x[i] + cx * cx * g0[i]
        m0, m1x, m1y, m2x = n0, n1x, n1y, n2x
        out.append((m0.copy(), m1x.copy(), m1y.copy(), m2x.copy()))
    return out


def test_field_step_matches_moment_recursion():
    """The field oracle and the moment-space recursion agree exactly while the support
    stays away from the periodic seam."""
    q, nx, ny, steps = 16, 90, 90, 30
    mfp = 3.0
    m = WormLBM(nx, ny, q, mfp, emulate_3d=True)
    W = float(m.w_int[0, 0])
    rng = np.random.default_rng(7)
    d0 = np.zeros((q, ny + 2, nx + 2))
    d0[:, 44:49, 43:48] = rng.standard_normal((q, 5, 5))
    m.set_state(d0)
    y, x = np.mgrid[0:ny + 2, 0:nx + 2].astype(np.float64)
    mom = lambda d: (d.sum((1, 2)), (d * x).sum((1, 2)), (d * y).sum((1, 2)),
                     (d * x * x).sum((1, 2)))
    ref = _moment_recursion(q, W, steps, *mom(d0))
    for n in range(steps):
        m.step()
        got = mom(m.d)
        for a, b in zip(got, ref[n]):
            assert np.allclose(a, b, rtol=1e-11, atol=1e-9)


def _diffusivity(q, mfp, emulate_3d, steps, speed=1.0):
    dirs = L.ring_directions(q)
    W = float(L.relax_weight(mfp / speed, L.lambda_corr(dirs), emulate_3d))
    w = L.angular_weights(dirs)
    z = np.zeros(q)
    hist = _moment_recursion(q, W, steps, w.copy(), z.copy(), z.copy(), z.copy(), speed)

    def var(t):
        m0, m1x, _, m2x = hist[t]
        return m2x.sum() / m0.sum() - (m1x.sum() / m0.sum()) ** 2
    t1, t2 = steps // 2, steps - 1
    return (var(t2) - var(t1)) / (2.0 * (t2 - t1))


@pytest.mark.parametrize("emulate_3d,target", [(True, 1.0 / 3.0), (False, 0.5)])
def test_diffusive_limit_grid_mfp_correction(emulate_3d, target):
    """Sec. 2.3 / Eq. W-correction and Sec. 4.3: in the Fourier limit the corrected
    scheme diffuses with D = v_g Lambda / 3 when a 2D run emulates 3D (D = Lambda / 2
    for plain 2D), up to a first-order lattice error in 1/Lambda."""
    d16 = _diffusivity(8, 16.0, emulate_3d, 1400)
    d32 = _diffusivity(8, 32.0, emulate_3d, 2400)
    slope = (d32 - d16) / 16.0
    assert slope == pytest.approx(target, rel=0.01)
    e16 = 1 - d16 / (16 * target)
    e32 = 1 - d32 / (32 * target)
    assert 0 < e32 < e16 and 0.3 < e32 / e16 < 0.7          # first order in 1/Lambda


def test_heat_flux_of_equilibrium_is_zero_and_single_beam_is_exact():
    """Eq. q_corr: an isotropic equilibrium carries no flux; a single populated
    direction carries exactly e_i s_i."""
    m = WormLBM(8, 8, 32, 4.0)
    m.init_temperature(np.full((8, 8), 0.7))
    qx, qy = m.heat_flux()
    assert np.abs(qx).max() < 1e-17 and np.abs(qy).max() < 1e-17
    d = np.zeros_like(m.d)
    d[5, 1:-1, 1:-1] = 2.0
    m.set_state(d)
    qx, qy = m.heat_flux()
    assert np.allclose(qx, 2.0 * m.s_hat[5, 0]) and np.allclose(qy, 2.0 * m.s_hat[5, 1])


def test_cross_plane_fourier_steady_profile_is_linear():
    """Sec. 4.4 (cross-plane, Fourier limit): isothermal walls at T_h and T_c and
    periodic y give, once steady and averaged over TAS fluctuations (Sec. 4.4 averages
    the flux over steps), a linear energy profile away from the wall layers and a
    uniform heat flux."""
    nx = 40
    m = WormLBM(nx, 1, 16, 1.5, bc_kind=(I, I, P, P), t_wall=(301.0, 300.0, 0, 0))
    m.init_temperature(np.zeros((1, nx)))
    m.step(5000)
    e_acc = np.zeros(nx)
    q_acc = np.zeros(nx)
    for _ in range(400):
        m.step()
        e_acc += m.energy_dev()[0]
        q_acc += m.heat_flux()[0][0]
    e, q = e_acc / 400, q_acc / 400
    x = np.arange(nx)
    fit = np.polyfit(x[6:-6], e[6:-6], 1)
    assert np.abs(np.polyval(fit, x) - e)[6:-6].max() < 1e-4 * np.ptp(e)
    assert fit[0] < 0 and q.mean() > 0
    assert np.ptp(q[2:-2]) < 0.03 * q.mean()


def test_specular_mirror_and_zero_specularity():
    """The mirror of a direction at a wall flips the normal component and is an
    involution; a specularity of 0 gives the diffuse wall exactly (same arithmetic, so
    bit for bit)."""
    m = WormLBM(9, 7, 24, 3.0)
    for normal in ((1, 0), (0, 1)):
        mi = m.mirror_index(normal)
        assert np.array_equal(mi[mi], np.arange(24))
        for i, (a, b) in enumerate(m.dirs):
            assert m.dirs[mi[i]] == ((-a, b) if normal[0] else (a, -b))
    x = WormLBM(13, 9, 16, 2.0, bc_kind=(A, A, A, A))
    y = WormLBM(13, 9, 16, 2.0, bc_kind=(A, A, A, A), specularity=(0.0,) * 4)
    for z in (x, y):
        z.init_temperature(_rand(9, 13, 4))
        z.step(30)
    assert np.array_equal(x.d, y.d)


@pytest.mark.parametrize("speed", [0.5, 0.3])
def test_tas_at_lower_speed_keeps_every_direction_within_one_cell(speed):
    """TAS beyond the unit speed (Sec. 1): with the reference distance v n every direction
    stays within one cell of v n along its ray (the unit-speed bound of Sec. 3.1 carried
    over), and now the axial directions pause too, at the rate 1 - v."""
    q = 32
    sched = L.TasSchedule(q, speed)
    dirs = np.array(L.ring_directions(q), np.float64)
    u = dirs / np.linalg.norm(dirs, axis=1)[:, None]
    axial_pauses = 0
    steps = 400
    for n in range(1, steps + 1):
        _, paused = sched.advance(n)
        axial_pauses += sum(paused[i] for i in (0, q // 4, q // 2, 3 * q // 4))
        p = sched.displacement().astype(np.float64)
        along = (p * u).sum(axis=1)
        across = p[:, 0] * u[:, 1] - p[:, 1] * u[:, 0]
        assert np.all(np.abs(along - speed * n) <= 1.0 + 1e-12)
        assert np.all(np.abs(across) <= 1.0 + 1e-12)
    assert axial_pauses / (4 * steps) == pytest.approx(1 - speed, abs=0.01)


@pytest.mark.parametrize("speed", [0.5, 0.25])
def test_diffusive_limit_at_lower_speed(speed):
    """A band with speed v relaxes with W = v / Lambda per step and diffuses with
    D = v Lambda / 3 (3D emulation), up to a first-order error in 1/Lambda."""
    d16 = _diffusivity(16, 16.0, True, int(1400 / speed), speed)
    d32 = _diffusivity(16, 32.0, True, int(2400 / speed), speed)
    assert (d32 - d16) / 16.0 == pytest.approx(speed / 3.0, rel=0.01)
    e16 = d16 / (16 * speed / 3) - 1
    e32 = d32 / (32 * speed / 3) - 1
    assert 0.3 < e32 / e16 < 0.7                       # first order in 1/Lambda


def test_mean_moments_of_a_ballistic_run():
    """Sec. 4.3 averages the flux over 10 steps: at W = 0 on a periodic grid the mean over
    the next n states equals the mean of the exactly translated fields."""
    nx = ny = 18
    q, n0, n = 16, 3, 10
    yy, xx = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((xx - 8.3) ** 2 + (yy - 9.1) ** 2) / 8.0)
    m = WormLBM(nx, ny, q, 1.0, w_field=0.0)
    m.init_temperature(dT0)
    m.step(n0)
    mt, mqx, mqy = m.mean_moments(n)
    e0 = L.e_eq(300.0 + dT0, m.theta) - m.e_ref
    sched = L.TasSchedule(q)
    u = L.unit_vectors(L.ring_directions(q))
    st = sx = sy = 0.0
    for k in range(1, n0 + n + 1):
        sched.advance()
        if k <= n0:
            continue
        p = sched.displacement()
        planes = [m.w[i] * np.roll(e0, (p[i][1], p[i][0]), axis=(0, 1)) for i in range(q)]
        st = st + L.temperature(m.e_ref + sum(planes), m.theta) - 300.0
        sx = sx + sum(u[i, 0] * planes[i] for i in range(q))
        sy = sy + sum(u[i, 1] * planes[i] for i in range(q))
    np.testing.assert_allclose(mt, st / n, rtol=0, atol=1e-12)
    np.testing.assert_allclose(mqx, sx / n, rtol=0, atol=1e-15)
    np.testing.assert_allclose(mqy, sy / n, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------------------
# Per-cell relaxation weight.  Eq. lbm-energy and Eq. algorithm print one W; with a field
# W(x) the oracle takes the loss of a paused DDED at its own cell y and every gain (the
# EED, which always hops) at the source cell s = y - c.  The pins below fix that reading
# from outside the step: global conservation (which any other placement of W breaks), one
# step written out by hand, and the uniform field.

def _lognormal_w(ny, nx, seed):
    """A rough log-normal MFP field (cells), every W_corr well inside (0, 1)."""
    g = np.random.default_rng(seed).standard_normal((ny, nx))
    return np.maximum(np.exp(math.log(4.0) + 0.6 * g), 1.5)


def test_energy_conserved_with_per_cell_mfp_field():
    """Eq. lbm-energy-density with a non-uniform W: the loss (1 - W(y)) d_i(y) of a paused
    DDED and the gains w_i W(s) E(s) sum to the scattered energy of every cell, so a
    periodic grid keeps its total to round-off through propagating and paused steps."""
    ny, nx, q = 19, 23, 16
    m = WormLBM(nx, ny, q, _lognormal_w(ny, nx, 11))
    assert np.ptp(m.w_int) > 0.2                       # the field really varies
    m.init_temperature(_rand(ny, nx, 12))
    e0 = m.total_energy()
    scale = np.abs(m.d).sum()
    sched = L.TasSchedule(q)
    n_paused = 0
    for n in range(1, 61):
        _, paused = sched.advance(n)
        n_paused += int(np.sum(paused))
        m.step()
        assert abs(m.total_energy() - e0) <= 1e-13 * scale
    assert n_paused > 0                                # paused steps were exercised


@pytest.mark.parametrize("q", [8, 16])
def test_one_step_with_per_cell_w_written_out_by_hand(q):
    """Two populated directions of one cell y0 (one paused, one propagating at the first
    step that pauses anything), a distinct W in every cell, one update.  Expected values
    from Eq. algorithm with the loss of a paused DDED at its own cell and every gain at the
    source cell, written out term by term:
        every direction i:      d_i'(y0 + c_i)  gains w_i W(y0) E(y0);
        propagating b:          d_b'(y0 + c_b) += (1 - W(y0)) b;
        paused a:               d_a'(y0)        = (1 - W(y0)) a."""
    nx = ny = 7
    rng = np.random.default_rng(5 + q)
    wf = 0.05 + 0.9 * rng.random((ny, nx))             # distinct W in every cell
    m = WormLBM(nx, ny, q, None, w_field=wf, bc_kind=(P, P, P, P))
    sched = L.TasSchedule(q)
    for n in range(1, 200):
        hops, paused = sched.advance(n)
        if any(paused):
            break
    assert any(paused) and not all(paused)
    ia = int(np.flatnonzero(paused)[0])
    ib = int(np.flatnonzero(~np.asarray(paused, bool))[0])
    Y0, X0 = 4, 3                                       # framed indices of y0
    a, b = 0.7, -1.3
    d = np.zeros((q, ny + 2, nx + 2))
    d[ia, Y0, X0] = a
    d[ib, Y0, X0] = b
    E0 = a + b
    W0 = wf[Y0 - 1, X0 - 1]
    want = np.zeros_like(d)
    for i in range(q):
        cx, cy = L.BASIC_HOPS[hops[i]]
        want[i, Y0 + cy, X0 + cx] += m.w[i] * W0 * E0
    cbx, cby = L.BASIC_HOPS[hops[ib]]
    want[ib, Y0 + cby, X0 + cbx] += (1.0 - W0) * b
    want[ia, Y0, X0] += (1.0 - W0) * a
    got = m.collide_stream(d, hops, paused)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    # the two placements of W the reading rules out give other values here
    cax, cay = L.BASIC_HOPS[hops[ia]]
    assert abs(wf[Y0 - 1 - cay, X0 - 1 - cax] - W0) > 1e-3     # W(s) of the paused loss
    assert abs(wf[Y0 - 1 + cby, X0 - 1 + cbx] - W0) > 1e-3     # W(y) of the propagating one


def test_uniform_w_field_equals_scalar_mfp():
    """A field whose every cell carries the same MFP is the scalar-MFP run, bit for bit."""
    ny, nx, q = 13, 17, 16
    dT = _rand(ny, nx, 21)
    runs = []
    for mfp in (3.5, np.full((ny, nx), 3.5)):
        m = WormLBM(nx, ny, q, mfp, bc_kind=(I, I, A, A), t_wall=(301.0, 300.0, 0, 0))
        m.init_temperature(dT)
        m.step(25)
        runs.append(m.d.copy())
    assert np.array_equal(runs[0], runs[1])
