"""Bands slower than one cell per step (the TAS beyond the unit speed, Sec. 1; the bands of
a multigray run, Sec. 2.1) on the GPU: parity with the oracle, the conductivity
reductions (D = v Lambda / 3, q = v sum_i e_i s_i), a batch of bands with different
speeds and MFPs equal to the bands run one by one, and the adjoint."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from oracle import transport as T
from tests._pair import THETA, gpu_handle, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu
P, I, D = W.PERIODIC, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE
TOL32, TOL16, TOL16_STATE = 1e-5, 2e-3, 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401  (fails loudly if the library is missing)


def _pulses(speed, n=80, q=32, mfp=6.0):
    cfg = W.pulses_c2(seed=3, n=n, q=q, mfp=mfp, npulse=4)
    cfg["speed"] = speed
    return cfg


def _film(speed, nx=120, ny=24, q=32, kn=0.8):
    cfg = W.film_c3(kn=kn, nx=nx, ny=ny, q=q)
    cfg["speed"] = speed
    return cfg


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("cfg", [_pulses(0.5), _pulses(0.23, q=16), _film(0.7)],
                         ids=["pulses_v0.5", "pulses_v0.23", "film_v0.7"])
def test_lower_speed_matches_oracle(cfg, storage):
    steps = 90
    orc = oracle_run(cfg, steps)
    gpu = gpu_run(cfg, steps, storage)
    amp = cfg["amp"]
    dscale = float(np.abs(oracle_run(cfg, 0).d).max())
    tol, stol = (TOL32, TOL32) if storage == 0 else (TOL16, TOL16_STATE)
    assert rel_linf(gpu["dT"], orc.temperature_dev(), amp) <= tol
    assert rel_linf(gpu["state"][:, 1:-1, 1:-1], orc.d[:, 1:-1, 1:-1], dscale) <= stol
    qx, qy = orc.heat_flux()
    qscale = dscale * float(np.abs(orc.s_hat[:, 0]).sum()) * cfg["speed"]
    assert rel_linf(gpu["qx"], qx, qscale) <= stol
    assert rel_linf(gpu["qy"], qy, qscale) <= stol
    # mean flux and conductivities of wlbm_reduce with v_g = v and D = v Lambda / 3
    eps_q = stol * qscale
    assert abs(gpu["red"][2] - float(qx.mean())) <= eps_q
    if cfg["bc"][0] == I:
        de = 1 / math.expm1(THETA / cfg["t_wall"][0]) - 1 / math.expm1(THETA / cfg["t_wall"][1])
        dd = T.bulk_diffusivity(cfg["mfp"], True, cfg["speed"])
        assert abs(gpu["red"][6] - T.kappa_apparent(orc, cfg["mfp"])) <= eps_q * cfg["nx"] / (dd * de)


def test_multigray_batch_equals_bands_one_by_one():
    """Three bands of one film (different speed and MFP, one grid shape), stepped as one
    batch: each band bit for bit as when stepped alone; their heat fluxes superpose."""
    import paper_1911_00180_gb300 as wl
    base = _film(1.0, nx=96, ny=20, q=32)
    bands = [dict(speed=1.0, mfp=20.0), dict(speed=0.6, mfp=8.0), dict(speed=0.3, mfp=3.0)]
    specs = [dict(nx=base["nx"], ny=base["ny"], q=base["q"], bc=base["bc"],
                  t_wall=base["t_wall"], mfp=b["mfp"], speed=b["speed"]) for b in bands]
    bt = wl.WormLBMBatch(specs)
    bt.wlbm_batch_init_temperature([base["dT"]] * len(bands))
    bt.wlbm_batch_step(45)
    got = [v.wlbm_get_state().cpu().numpy() for v in bt.instances]
    q_b = [v.wlbm_reduce()[2] for v in bt.instances]
    bt.close()
    for k, sp in enumerate(specs):
        h = wl.WormLBM(sp["nx"], sp["ny"], sp["q"], mfp=sp["mfp"], bc=sp["bc"],
                       t_wall=sp["t_wall"], speed=sp["speed"])
        h.wlbm_init_temperature(base["dT"])
        h.wlbm_step(45)
        want = h.wlbm_get_state().cpu().numpy()
        h.close()
        assert np.array_equal(got[k][:, 1:-1, 1:-1], want[:, 1:-1, 1:-1]), k
    # the bands are uncoupled: the total flux is the sum of the bands' fluxes
    orc = [oracle_run(dict(base, mfp=b["mfp"], speed=b["speed"]), 45) for b in bands]
    total = sum(float(o.heat_flux()[0].mean()) for o in orc)
    assert sum(q_b) == pytest.approx(total, rel=1e-4)


def test_adjoint_at_lower_speed_matches_oracle():
    kinds = (I, I, D, D)
    ny, nx, q, steps, ckpt, speed = 14, 22, 16, 48, 10, 0.6
    rng = np.random.default_rng(9)
    mfp = np.maximum(np.exp(np.log(4.0) + 0.25 * rng.standard_normal((ny, nx))), 1.6).astype(np.float32)
    yy, xx = np.mgrid[0:ny, 0:nx]
    dT0 = np.exp(-((xx - 8.0) ** 2 + (yy - 7.0) ** 2) / 20.0).astype(np.float32)
    tw = (300.6, 299.7, 300.0, 300.0)
    probe = np.zeros((ny, nx), bool)
    probe[:, 16] = True
    import torch
    import paper_1911_00180_gb300 as wl
    h = wl.WormLBM(nx, ny, q, mfp_field=mfp, bc=kinds, t_wall=tw, theta=THETA, speed=speed)
    h.wlbm_adjoint_forward(dT0, steps, ckpt)
    g = torch.as_tensor(probe.astype(np.float32) / probe.sum(), device="cuda")
    g_mfp, g_tw, g_dT0 = h.wlbm_adjoint_backward(None, dJ_dqx=g)
    torch.cuda.synchronize()
    h.close()
    kw = dict(nx=nx, ny=ny, q=q, mfp=mfp.astype(np.float64), bc_kind=kinds, t_wall=tw,
              emulate_3d=True, theta=THETA, speed=speed)
    ref = A.AdjointRun(kw, dT0.astype(np.float64), steps, probe, "flux_x").gradients()
    rel = lambda a, b: float(np.abs(np.asarray(a) - b).max() / np.abs(b).max())
    assert rel(g_mfp.double().cpu().numpy(), ref["dJ_dmfp"]) <= 1e-4
    assert rel(g_dT0.double().cpu().numpy(), ref["dJ_ddT0"]) <= 1e-4
    assert rel(np.array(g_tw)[:2], ref["dJ_dTwall"][:2]) <= 1e-4
