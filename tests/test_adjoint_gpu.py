"""GPU adjoint (through the C ABI) against the oracle's exact transpose (itself pinned to
the one-step matrix transpose and to central differences, tests/test_oracle_adjoint.py).

J = mean of T - T_ref over a probe column of the final state.  Tolerance: 1e-4 of the
largest gradient entry (float32 forward and reverse sweeps against float64)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A

pytestmark = pytest.mark.gpu
P, I, D = W.PERIODIC, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE
TOL = 1e-4
THETA = 624.8074248458514


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401


def _case(kinds, nx=26, ny=18, q=16, steps=60, seed=3, field=True):
    rng = np.random.default_rng(seed)
    # log-normal MFP around 4 cells, kept above the W_corr <= 1 limit (1.37 cells)
    mfp = (np.maximum(np.exp(np.log(4.0) + 0.25 * rng.standard_normal((ny, nx))), 1.6)
           .astype(np.float32) if field else None)
    y, x = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((x - nx / 3.0) ** 2 + (y - ny / 2.0) ** 2) / 20.0).astype(np.float32)
    probe = np.zeros((ny, nx), bool)
    probe[:, (3 * nx) // 4] = True
    tw = (300.6, 299.7, 300.2, 299.9)
    return mfp, dT0, probe, tw


def _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q, mfp_uniform=3.0, variant=None,
         objective="temperature", spec=(0.0,) * 4, speed=1.0):
    import torch
    import paper_1911_00180_gb300 as wl
    ny, nx = dT0.shape
    h = wl.WormLBM(nx, ny, q, mfp=mfp_uniform if mfp is None else None, mfp_field=mfp,
                   bc=kinds, t_wall=tw, emulate_3d=True, theta=THETA, specularity=spec,
                   speed=speed)
    if variant is not None:
        h.wlbm_set_option(wl.wlbm.OPT_STEP_VARIANT, variant)
    h.wlbm_adjoint_forward(dT0, steps, ckpt)
    dT, qx, _ = h.wlbm_moments()
    g = torch.as_tensor(probe.astype(np.float32) / probe.sum(), device="cuda")
    if objective == "flux_x":
        g_mfp, g_tw, g_dT0 = h.wlbm_adjoint_backward(None, dJ_dqx=g)
        J = float(qx.cpu().numpy().astype(np.float64)[probe].mean())
    else:
        g_mfp, g_tw, g_dT0 = h.wlbm_adjoint_backward(g)
        J = float(dT.cpu().numpy()[probe].mean())
    h.wlbm_check()
    torch.cuda.synchronize()
    out = (J, g_mfp.cpu().numpy().astype(np.float64), np.array(g_tw),
           g_dT0.cpu().numpy().astype(np.float64))
    h.close()
    return out


def _oracle(kinds, mfp, dT0, probe, tw, steps, q, mfp_uniform=3.0, objective="temperature",
            spec=(0.0,) * 4, speed=1.0):
    ny, nx = dT0.shape
    kw = dict(nx=nx, ny=ny, q=q,
              mfp=(np.full((ny, nx), mfp_uniform) if mfp is None else mfp.astype(np.float64)),
              bc_kind=kinds, t_wall=tw, emulate_3d=True, theta=THETA, specularity=spec,
              speed=speed)
    return A.AdjointRun(kw, dT0.astype(np.float64), steps, probe, objective).gradients()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("kinds", [(I, I, P, P), (I, I, D, D), (P, P, P, P), (D, D, D, D),
                                   (P, P, I, D), (D, I, I, D)])
def test_adjoint_gradients_match_oracle(kinds):
    steps, ckpt, q = 60, 7, 16              # ragged last segment (60 = 8*7 + 4)
    mfp, dT0, probe, tw = _case(kinds)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q)
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q)
    assert abs(J - ref["J"]) <= 1e-5
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    iso = [k for k in range(4) if kinds[k] == I]
    if iso:
        assert _rel(g_tw[iso], ref["dJ_dTwall"][iso]) <= TOL
    assert np.all(g_tw[[k for k in range(4) if kinds[k] != I]] == 0.0)


@pytest.mark.parametrize("q", [256, 1024])
def test_adjoint_largest_direction_sets_match_oracle(q):
    """Q = 256 and the largest Q the library takes (1024): the reverse step's direction
    table and ring at their largest, with walls of every kind, against the oracle."""
    kinds = (D, I, P, P)                   # the isothermal wall 7 cells from the probe
    steps, ckpt = 20, 6
    mfp, dT0, probe, tw = _case(kinds, nx=30, ny=16, seed=7)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q)
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q)
    assert abs(J - ref["J"]) <= 1e-5
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    assert abs(ref["dJ_dTwall"][1]) > 0
    assert _rel(g_tw[1:2], ref["dJ_dTwall"][1:2]) <= TOL


@pytest.mark.parametrize("kinds,spec", [((I, I, 3, D), (0.0, 0.0, 0.0, 0.45)),
                                       ((D, 3, I, D), (0.7, 0.0, 0.0, 0.0))])
def test_adjoint_specular_walls_match_oracle(kinds, spec):
    """Specular and partly specular walls: the transposed wall pass (an outward direction
    takes p l_mirror + (1 - p) S) against the oracle's transpose."""
    steps, ckpt, q = 50, 9, 16
    mfp, dT0, probe, tw = _case(kinds)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q, spec=spec)
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q, spec=spec)
    assert abs(J - ref["J"]) <= 1e-5
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    iso = [k for k in range(4) if kinds[k] == I]
    assert _rel(g_tw[iso], ref["dJ_dTwall"][iso]) <= TOL


@pytest.mark.parametrize("objective,kinds,spec", [
    ("temperature", (I, I, D, D), (0.0,) * 4),
    ("flux_x", (I, I, D, 3), (0.0, 0.0, 0.0, 0.6))])
def test_adjoint_band_speed_matches_oracle(objective, kinds, spec):
    """A band of speed v = 0.6 cells/step (W = v / MFP, the hop test against (v n + 1)^2,
    the flux seed scaled by v): the GPU reverse sweep against the oracle's transpose."""
    steps, ckpt, q, v = 56, 9, 16, 0.6
    mfp, dT0, probe, tw = _case(kinds, seed=5)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q,
                                 objective=objective, spec=spec, speed=v)
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q, objective=objective, spec=spec,
                  speed=v)
    assert abs(J - ref["J"]) <= (1e-5 * 1.2e-3 * q if objective == "flux_x" else 1e-5)
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    assert _rel(g_tw[:2], ref["dJ_dTwall"][:2]) <= TOL


@pytest.mark.parametrize("kinds", [(I, I, D, D), (I, I, P, P)])
def test_adjoint_flux_objective_matches_oracle(kinds):
    """J = mean q_x over the probe column (the numerator of the film conductivity): the
    flux seed of the reverse sweep against the oracle's gradients."""
    steps, ckpt, q = 60, 7, 16
    mfp, dT0, probe, tw = _case(kinds)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q,
                                 objective="flux_x")
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q, objective="flux_x")
    # a stored deviation within 1e-5 of its scale (|d| < e(301 K) - e(300 K) < 1.2e-3)
    # and sum_i |s_ix| < Q bound the float32 flux error
    assert abs(J - ref["J"]) <= 1e-5 * 1.2e-3 * q
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    assert _rel(g_tw[:2], ref["dJ_dTwall"][:2]) <= TOL


def test_autograd_conductivity_gradient():
    """kappa_app = mean q_x * nx / (D (e(T_h) - e(T_c))) built in torch on the autograd
    run's flux: its gradient is the oracle's flux gradient scaled, plus the explicit
    dependence on the wall temperatures through e(T_h) - e(T_c)."""
    import math
    import torch
    from paper_1911_00180_gb300.autograd import wlbm_run_moments
    kinds = (I, I, D, D)
    mfp, dT0, probe, tw = _case(kinds, nx=24, ny=12)
    spec = dict(nx=24, ny=12, q=16, bc=kinds, steps=40, ckpt=9)
    m = torch.tensor(mfp, device="cuda", requires_grad=True)
    t = torch.tensor(tw, dtype=torch.float64, device="cuda", requires_grad=True)
    d0 = torch.tensor(dT0, device="cuda", requires_grad=True)
    _, qx, _ = wlbm_run_moments(m, t, d0, spec)
    d_bulk = 4.0 / 3.0                             # reference MFP of 4 cells
    e = lambda tt: 1.0 / torch.expm1(THETA / tt)
    de = e(t[0]) - e(t[1])
    kappa = qx.double().mean() * spec["nx"] / (d_bulk * de)
    kappa.backward()
    everywhere = np.ones((12, 24), bool)
    ref = _oracle(kinds, mfp, dT0, everywhere, tw, 40, 16, objective="flux_x")
    de0 = 1.0 / math.expm1(THETA / tw[0]) - 1.0 / math.expm1(THETA / tw[1])
    scale = spec["nx"] / (d_bulk * de0)
    assert _rel(m.grad.double().cpu().numpy(), scale * ref["dJ_dmfp"]) <= TOL
    assert _rel(d0.grad.double().cpu().numpy(), scale * ref["dJ_ddT0"]) <= TOL
    dede = [math.exp(THETA / tt) / math.expm1(THETA / tt) ** 2 * THETA / tt ** 2 for tt in tw[:2]]
    k0 = ref["J"] * scale
    want = [scale * ref["dJ_dTwall"][0] - k0 / de0 * dede[0],
            scale * ref["dJ_dTwall"][1] + k0 / de0 * dede[1]]
    assert _rel(t.grad.cpu().numpy()[:2], np.array(want)) <= TOL


def test_adjoint_uniform_mfp_and_register_variant():
    kinds = (I, I, P, P)
    _, dT0, probe, tw = _case(kinds, nx=33, ny=12, q=24)
    J, g_mfp, g_tw, g_dT0 = _gpu(kinds, None, dT0, probe, tw, 45, 10, 24, mfp_uniform=2.2,
                                 variant=0)
    ref = _oracle(kinds, None, dT0, probe, tw, 45, 24, mfp_uniform=2.2)
    assert _rel(g_mfp, ref["dJ_dmfp"]) <= TOL
    assert _rel(g_dT0, ref["dJ_ddT0"]) <= TOL
    assert _rel(g_tw[:2], ref["dJ_dTwall"][:2]) <= TOL


@pytest.mark.parametrize("kinds,p,v", [((I, I, P, P), (0.0,) * 4, 1.0),
                                       ((I, I, 3, D), (0.0, 0.0, 0.8, 0.0), 0.7)])
def test_autograd_function_matches_direct_backward(kinds, p, v):
    import torch
    from paper_1911_00180_gb300.autograd import wlbm_run
    mfp, dT0, probe, tw = _case(kinds, nx=20, ny=14)
    spec = dict(nx=20, ny=14, q=16, bc=kinds, steps=30, ckpt=8, specularity=p, speed=v)
    m = torch.tensor(mfp, device="cuda", requires_grad=True)
    t = torch.tensor(tw, dtype=torch.float64, device="cuda", requires_grad=True)
    d0 = torch.tensor(dT0, device="cuda", requires_grad=True)
    out = wlbm_run(m, t, d0, spec)
    J = out[torch.as_tensor(probe, device="cuda")].mean()
    J.backward()
    ref = _oracle(kinds, mfp, dT0, probe, tw, 30, 16, spec=p, speed=v)
    assert _rel(m.grad.double().cpu().numpy(), ref["dJ_dmfp"]) <= TOL
    assert _rel(d0.grad.double().cpu().numpy(), ref["dJ_ddT0"]) <= TOL
    assert _rel(t.grad.cpu().numpy()[:2], ref["dJ_dTwall"][:2]) <= TOL


def test_adjoint_directional_derivative_mid_size():
    """256 x 192, Q = 32, 200 steps: <dJ/d dT0, v> against a central difference of the GPU
    forward along a smooth direction v (a property that holds at any size)."""
    import torch
    import paper_1911_00180_gb300 as wl
    nx, ny, q, steps = 256, 192, 32, 200
    kinds = (I, I, P, P)
    mfp = W.lognormal_mfp(nx, ny, seed=7, corr=16.0)
    dT0 = W.gaussian_field(nx, ny, [(128.0, 96.0)], [24.0], [1.0], periodic=False).astype(np.float32)
    v = W.gaussian_field(nx, ny, [(100.0, 80.0)], [30.0], [1.0], periodic=False).astype(np.float32)
    probe = np.zeros((ny, nx), bool)
    probe[:, 192] = True
    tw = (300.0,) * 4

    def J_of(d):
        h = wl.WormLBM(nx, ny, q, mfp_field=mfp, bc=kinds, t_wall=tw, theta=THETA)
        h.wlbm_init_temperature(d)
        h.wlbm_step(steps)
        dT, _, _ = h.wlbm_moments(want_q=False)
        val = float(dT.double().cpu().numpy()[probe].mean())
        h.close()
        return val
    h = wl.WormLBM(nx, ny, q, mfp_field=mfp, bc=kinds, t_wall=tw, theta=THETA)
    h.wlbm_adjoint_forward(dT0, steps, 25)
    g = torch.as_tensor(probe.astype(np.float32) / probe.sum(), device="cuda")
    _, _, g_dT0 = h.wlbm_adjoint_backward(g, want_mfp=False)
    ad = float((g_dT0.double().cpu().numpy() * v).sum())
    h.close()
    eps = 0.05
    fd = (J_of(dT0 + eps * v) - J_of(dT0 - eps * v)) / (2 * eps)
    assert ad == pytest.approx(fd, rel=2e-3)


def test_adjoint_multi_tile_c5_recipe_matches_oracle():
    """The adjoint workload's recipe beyond one tile: 260 x 30 (three 128-column tiles and
    three 14-row tile rows of the TMA kernels), Q = 64, log-normal MFP field, isothermal x
    walls at 300 K, periodic y, central Gaussian pulse, checkpoints every 50 steps over 110
    steps (three checkpoints, a ragged last segment), on a stream of its own as the
    benchmark runs it.  J = mean T over the column at 3 nx / 4; dJ/dMFP, dJ/dT_wall and
    dJ/d(dT0) against the oracle's transpose at 1e-4."""
    import torch
    nx, ny, q, steps, ckpt = 260, 30, 64, 110, 50
    kinds = (I, I, P, P)
    mfp = np.maximum(W.lognormal_mfp(nx, ny, seed=9, corr=8.0), 1.6).astype(np.float32)
    dT0 = W.gaussian_field(nx, ny, [(nx / 2.0, ny / 2.0)], [8.0], [1.0],
                           periodic=False).astype(np.float32)
    probe = np.zeros((ny, nx), bool)
    probe[:, (3 * nx) // 4] = True
    tw = (300.0,) * 4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        J, g_mfp, g_tw, g_dT0 = _gpu(kinds, mfp, dT0, probe, tw, steps, ckpt, q)
    ref = _oracle(kinds, mfp, dT0, probe, tw, steps, q)
    assert abs(J - ref["J"]) <= 1e-5
    e = (_rel(g_mfp, ref["dJ_dmfp"]), _rel(g_dT0, ref["dJ_ddT0"]),
         _rel(g_tw[:2], ref["dJ_dTwall"][:2]))
    print("adjoint 260x30 Q64: dJ/dMFP %.3g  dJ/ddT0 %.3g  dJ/dTwall %.3g" % e)
    assert max(e) <= TOL
    assert np.all(g_tw[2:] == 0.0)


def test_adjoint_full_size_c5_directional_derivatives():
    """The adjoint workload at full size: 1024^2, Q = 64, its log-normal MFP field,
    isothermal x walls, periodic y, checkpoints every 50, on a stream of its own as the
    benchmark runs it; 160 steps (a ragged last segment).  The adjoint's directional
    derivatives of J (mean T over the column x = 560, 48 cells from the pulse centre) along
    a start-field direction v and along a relative MFP-field direction u, against central
    differences of the GPU forward run: a property that holds at any size, so it reaches
    the configuration the oracle is too slow for (the oracle's own gradients are checked on
    the smaller grids above)."""
    import torch
    import paper_1911_00180_gb300 as wl
    cfg = W.adjoint_c5()
    nx, ny, q = cfg["nx"], cfg["ny"], cfg["q"]
    steps, ckpt, px = 160, 50, 560
    probe = np.zeros((ny, nx), bool)
    probe[:, px] = True
    v = W.gaussian_field(nx, ny, [(540.0, 480.0)], [40.0], [1.0],
                         periodic=False).astype(np.float32)
    u = W.gaussian_field(nx, ny, [(550.0, 520.0)], [60.0], [1.0], periodic=False)
    mfp = cfg["mfp_field"].astype(np.float64)
    stream = torch.cuda.Stream()

    def handle(mfp_field):
        return wl.WormLBM(nx, ny, q, mfp_field=np.asarray(mfp_field, np.float32), bc=cfg["bc"],
                          t_wall=cfg["t_wall"], emulate_3d=True, theta=THETA, stream=stream)

    def J_of(dT, mfp_field):
        with torch.cuda.stream(stream):
            h = handle(mfp_field)
            h.wlbm_init_temperature(dT)
            h.wlbm_step(steps)
            dTo, _, _ = h.wlbm_moments(want_q=False)
            val = float(dTo.double().cpu().numpy()[probe].mean())
            h.wlbm_check()
            h.close()
        return val

    with torch.cuda.stream(stream):
        h = handle(mfp)
        h.wlbm_adjoint_forward(cfg["dT"], steps, ckpt)
        g = torch.as_tensor(probe.astype(np.float32) / probe.sum(), device="cuda")
        g_mfp, _, g_dT0 = h.wlbm_adjoint_backward(g)
        h.wlbm_check()
        gm = g_mfp.double().cpu().numpy()
        gd = g_dT0.double().cpu().numpy()
        h.close()
    ad_v = float((gd * v).sum())
    ad_u = float((gm * mfp * u).sum())          # d/de J(mfp (1 + e u)) at e = 0
    eps_v, eps_u = 0.05, 1e-2
    fd_v = (J_of(cfg["dT"] + eps_v * v, mfp) - J_of(cfg["dT"] - eps_v * v, mfp)) / (2 * eps_v)
    fd_u = (J_of(cfg["dT"], mfp * (1 + eps_u * u)) -
            J_of(cfg["dT"], mfp * (1 - eps_u * u))) / (2 * eps_u)
    print("adjoint 1024^2 Q64: <dJ/ddT0, v> %.6g (fd %.6g)  <dJ/dMFP, MFP u> %.6g (fd %.6g)"
          % (ad_v, fd_v, ad_u, fd_u))
    assert abs(ad_v) > 0 and abs(ad_u) > 0
    # J is linear in the start field up to T(E)'s curvature: the adjoint's bar, 1e-4.  J is
    # nonlinear in the MFP: the central difference's O(eps^2) truncation at a 1 % step
    # (measured 6e-5) sets 5e-4
    assert ad_v == pytest.approx(fd_v, rel=1e-4)
    assert ad_u == pytest.approx(fd_u, rel=5e-4)

