"""Pins of the oracle's angular lattice against what the paper fixes (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import lattice as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_constants():
    out = {}
    for line in open(os.path.join(GOLDEN, "lattice_constants.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_tas_printed_d2q8_pattern():
    """Sec. 2.3: the diagonal hops at n = 1, 2, 4, 5 and pauses at n = 3."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tas_d2q8_first_steps.txt"))
            if l.strip() and not l.startswith("#")]
    sched = L.TasSchedule(8)
    dirs = sched.dirs
    diag = [i for i, d in enumerate(dirs) if abs(d[0]) == abs(d[1])]
    axial = [i for i, d in enumerate(dirs) if 0 in d]
    for n, dstate, astate in rows:
        hops, paused = sched.advance(int(n))
        for i in diag:
            assert paused[i] == (dstate == "P"), (n, i)
        for i in axial:
            assert paused[i] == (astate == "P"), (n, i)


@pytest.mark.parametrize("q", [8, 16, 32, 64, 128, 256])
def test_axial_directions_never_pause(q):
    """Eq. algorithm: for axial directions the propagation condition always holds."""
    sched = L.TasSchedule(q)
    axial = [i for i, d in enumerate(sched.dirs) if 0 in d]
    for n in range(1, 600):
        _, paused = sched.advance(n)
        assert not any(paused[i] for i in axial)


@pytest.mark.parametrize("q", [8, 16, 64, 256])
def test_propagation_error_at_most_one_spacing(q):
    """Sec. 3.1: the propagated distance never differs from the axial one (n) by more
    than one grid spacing, and the perpendicular deviation from the ray stays within
    one spacing."""
    sched = L.TasSchedule(q)
    s_hat = L.unit_vectors(sched.dirs)
    perp = np.stack([-s_hat[:, 1], s_hat[:, 0]], axis=1)
    for n in range(1, 1500):
        sched.advance(n)
        p = sched.displacement().astype(np.float64)
        r = np.sqrt((p * p).sum(axis=1))
        assert np.all(np.abs(r - n) <= 1.0 + 1e-12)
        assert np.all(np.abs((p * perp).sum(axis=1)) <= 1.0 + 1e-12)


def test_lambda_corr_d2q8_printed():
    """Eq. W-correction-factor: Lambda_corr = 2/(1+sqrt 2) for D2Q8, and the general
    formula Q / sum c_i reduces to it at Q = 8."""
    g = _golden_constants()
    assert L.lambda_corr(L.ring_directions(8)) == pytest.approx(g["lambda_corr_d2q8"],
                                                                rel=0, abs=1e-15)


def test_weights_d2q8_uniform_and_normalised():
    """Sec. 2.2: uniform intervals give e_i^eq = e^eq / Q, i.e. w = 1/8 on D2Q8; the
    weights of every scheme sum to one."""
    g = _golden_constants()
    w8 = L.angular_weights(L.ring_directions(8))
    assert np.allclose(w8, g["weight_d2q8"], rtol=0, atol=1e-15)
    for q in (16, 24, 32, 64, 128, 256):
        w = L.angular_weights(L.ring_directions(q))
        assert abs(w.sum() - 1.0) < 1e-13
        assert np.all(w > 0)


def test_weights_d2q16_follow_fig3_angle_pattern():
    """Fig. 3 caption: on D2Q16 the angular intervals satisfy theta1 = theta4 = theta5 =
    theta8 = ... and theta2 = theta3 = theta6 = theta7 = ..., with theta1 != theta2."""
    dirs = L.ring_directions(16)
    th = L.direction_angles(dirs)
    gaps = [(th[(j + 1) % 16] - th[j]) % (2 * math.pi) for j in range(16)]
    a = [gaps[j] for j in (0, 3, 4, 7, 8, 11, 12, 15)]
    b = [gaps[j] for j in (1, 2, 5, 6, 9, 10, 13, 14)]
    assert np.ptp(a) < 1e-14 and np.ptp(b) < 1e-14
    assert abs(a[0] - b[0]) > 0.1
    # with the weight read as (left gap + right gap) / (4 pi)
    w = L.angular_weights(dirs)
    assert w[0] == pytest.approx((a[0] + a[0]) / (4 * math.pi), abs=1e-15)
    assert w[1] == pytest.approx((a[0] + b[0]) / (4 * math.pi), abs=1e-15)
    assert w[2] == pytest.approx((b[0] + b[0]) / (4 * math.pi), abs=1e-15)


@pytest.mark.parametrize("q", [16, 24, 32, 40, 64, 128, 256])
def test_worm_paths_reach_their_direction(q):
    """Eq. worm-paths: M basic hops, repeated every M steps, follow direction s; after
    one period the path ends exactly on the lattice point s (so c_i is consistent)."""
    dirs = L.ring_directions(q)
    m = q // 8
    for d, path in zip(dirs, L.worm_table(dirs)):
        assert len(path) == m
        px = sum(L.BASIC_HOPS[k][0] for k in path)
        py = sum(L.BASIC_HOPS[k][1] for k in path)
        assert (px, py) == tuple(d)
        # every hop moves forward along the direction
        for k in path:
            assert L.BASIC_HOPS[k][0] * d[0] + L.BASIC_HOPS[k][1] * d[1] > 0


@pytest.mark.parametrize("q", [16, 64, 256])
def test_worm_paths_share_the_lattice_symmetry(q):
    """Mirroring a direction mirrors its worm path (the diagonal wins every tie, so the
    greedy rule of Eq. worm-paths commutes with the 8 lattice symmetries)."""
    dirs = L.ring_directions(q)
    table = dict(zip(dirs, L.worm_table(dirs)))
    hop_index = {h: k for k, h in enumerate(L.BASIC_HOPS)}
    for sym in [lambda x, y: (y, x), lambda x, y: (-x, y), lambda x, y: (x, -y)]:
        for d, path in table.items():
            md = sym(*d)
            mpath = [hop_index[sym(*L.BASIC_HOPS[k])] for k in path]
            assert table[md] == mpath


def test_w_corr_limits():
    """Eq. W-correction: W_corr / W -> 3/2 as W -> 0 and W_corr = 3/2 Lambda_corr at
    W = 1 (the two limits the paper quotes, read for the ratio and the value)."""
    lc = 2.0 / (1.0 + math.sqrt(2.0))
    assert L.w_corr(1e-9, lc, True) / 1e-9 == pytest.approx(1.5, rel=1e-8)
    assert L.w_corr(1.0, lc, True) == pytest.approx(1.5 * lc, rel=1e-15)
    assert L.w_corr(1.0, lc, False) == pytest.approx(lc, rel=1e-15)


def test_theta_from_property_table():
    """Sec. 3 property table: omega = 81.8e12 /s gives hbar omega / k_B ~ 624.8 K."""
    g = _golden_constants()
    theta = L.HBAR * g["omega0_rad_per_s"] / L.K_B
    assert theta == pytest.approx(L.THETA_DEFAULT, rel=1e-15)
    assert theta == pytest.approx(624.807, abs=1e-3)


def test_pseudo_temperature_inverts_gray_energy():
    """Eq. pseudo-T is the inverse of Eq. gray-energy-density."""
    t = np.linspace(50.0, 1000.0, 97)
    assert np.allclose(L.temperature(L.e_eq(t, 624.8), 624.8), t, rtol=1e-14)
