"""Pins of the oracle's adjoint (CPU only): the reverse step is the exact transpose of the
forward one-step map (built column by column from unit vectors), and full-run gradients
equal central finite differences of the forward oracle."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle.stepper import (WormLBM, PERIODIC as P, ISOTHERMAL as I, ADIABATIC_DIFFUSE as D,
                            ADIABATIC_SPECULAR as S)

NO_SPEC = (0.0,) * 4
BC_CASES = [((P, P, P, P), (300.0,) * 4, NO_SPEC),
            ((I, I, D, D), (300.7, 299.6, 300.0, 300.0), NO_SPEC),
            ((D, D, D, D), (300.0,) * 4, NO_SPEC),
            ((P, P, I, D), (300.0, 300.0, 300.4, 300.0), NO_SPEC),
            ((D, I, P, P), (300.0, 300.3, 300.0, 300.0), NO_SPEC),
            ((I, I, S, S), (300.7, 299.6, 300.0, 300.0), NO_SPEC),
            ((D, S, D, D), (300.0,) * 4, (0.35, 0.0, 0.6, 0.0))]


def _model(kinds, tw, mfp, q=16, nx=5, ny=4, spec=NO_SPEC):
    return WormLBM(nx, ny, q, mfp, bc_kind=kinds, t_wall=tw, emulate_3d=True,
                   specularity=spec)


def _one_step(m, d, hops, paused):
    m.d = d.copy()
    m.apply_bc()
    return m.collide_stream(m.d, hops, paused)


@pytest.mark.parametrize("kinds,tw,spec", BC_CASES)
def test_reverse_step_is_exact_transpose(kinds, tw, spec):
    rng = np.random.default_rng(3)
    nx, ny, q = 5, 4, 16
    mfp = 1.6 + 3 * rng.random((ny, nx))
    m = _model(kinds, tw, mfp, q, nx, ny, spec)
    for n in range(1, 4):                  # step 3 has paused diagonals
        hops, paused = m.sched.advance(n)
    assert any(paused)
    shape = m.d.shape
    zero = np.zeros(shape)
    f0 = _one_step(m, zero, hops, paused)
    cols = []
    for j in range(zero.size):
        e = np.zeros(zero.size)
        e[j] = 1.0
        cols.append((_one_step(m, e.reshape(shape), hops, paused) - f0).ravel())
    M = np.array(cols).T                   # d_out = M d_in + f0
    lam_p = rng.standard_normal(shape)
    d_in = rng.standard_normal(shape)
    # recorded input of the step = state after the boundary pass
    m.d = d_in.copy()
    m.apply_bc()
    d_bc = m.d.copy()
    lam, gW = A.reverse_step(m, lam_p, d_bc, hops, paused)
    A.bc_transpose(m, lam)
    assert np.allclose(lam.ravel(), M.T @ lam_p.ravel(), rtol=1e-12, atol=1e-12)
    # W gradient: the step is affine in W, so a unit change of W(x) is exact
    A._periodic_links_T(m, gW[None])
    base = float((lam_p * _one_step(m, d_in, hops, paused)).sum())
    for (y, x) in [(0, 0), (1, 3), (3, 4), (2, 2)]:
        m2 = _model(kinds, tw, mfp, q, nx, ny, spec)
        wi = m.w_int.copy()
        wi[y, x] += 1.0
        m2.wf = m2._frame_scalar(wi)
        got = float((lam_p * _one_step(m2, d_in, hops, paused)).sum()) - base
        assert gW[y + 1, x + 1] == pytest.approx(got, rel=1e-10, abs=1e-12)


def _fd(fun, h):
    return (fun(h) - fun(-h)) / (2 * h)


@pytest.mark.parametrize("kinds,objective,spec,speed", [
    ((I, I, P, P), "temperature", NO_SPEC, 1.0),
    ((I, I, D, D), "temperature", NO_SPEC, 1.0),
    ((I, I, D, D), "flux_x", NO_SPEC, 1.0),
    ((I, I, D, S), "flux_x", (0, 0, 0.5, 0), 1.0),
    ((I, I, D, D), "flux_x", NO_SPEC, 0.6)])
def test_gradients_match_central_differences(kinds, objective, spec, speed):
    """Gradients of J (mean T - T_ref, or mean q_x, on a probe column) with respect to the
    per-cell MFP, the wall temperatures and the start field, against central differences
    of the forward oracle."""
    nx, ny, q, steps = 20, 14, 16, 40
    rng = np.random.default_rng(11)
    mfp = np.exp(np.log(3.0) + 0.3 * rng.standard_normal((ny, nx)))
    y, x = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((x - 8.0) ** 2 + (y - 7.0) ** 2) / 18.0)
    probe = np.zeros((ny, nx), bool)
    probe[:, 14] = True
    tw = (300.5, 299.8, 300.0, 300.0)
    kw = dict(nx=nx, ny=ny, q=q, mfp=mfp, bc_kind=kinds, t_wall=tw, emulate_3d=True,
              specularity=spec, speed=speed)
    run = A.AdjointRun(kw, dT0, steps, probe, objective)
    g = run.gradients()
    assert g["J"] == pytest.approx(run.forward(), rel=1e-14)
    for (cy, cx) in [(7, 10), (3, 13), (12, 2), (7, 14)]:
        def f(h, cy=cy, cx=cx):
            mm = mfp.copy()
            mm[cy, cx] *= 1.0 + h
            return run.forward(mfp=mm)
        fd = _fd(f, 1e-4) / mfp[cy, cx]
        assert g["dJ_dmfp"][cy, cx] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    for wall in (0, 1):
        def f(h, wall=wall):
            t = list(tw)
            t[wall] += h
            return run.forward(t_wall=tuple(t))
        assert g["dJ_dTwall"][wall] == pytest.approx(_fd(f, 1e-3), rel=1e-6)
    for (cy, cx) in [(7, 8), (0, 0)]:
        def f(h, cy=cy, cx=cx):
            d2 = dT0.copy()
            d2[cy, cx] += h
            r2 = A.AdjointRun(kw, d2, steps, probe, objective)
            return r2.forward()
        assert g["dJ_ddT0"][cy, cx] == pytest.approx(_fd(f, 1e-3), rel=1e-6, abs=1e-14)
