"""Helpers that run one workload through the oracle and through the CUDA library on the
same seeded inputs (tests only)."""
import numpy as np

from oracle.stepper import WormLBM as OracleLBM

THETA = 624.8074248458514


def oracle_run(cfg, steps, state=None, flux_peak=False):
    """The oracle after `steps` steps; with flux_peak the largest |q_x|, |q_y| of any cell
    over the start state and every step is kept as m.flux_peak (the run's flux
    amplitude)."""
    m = OracleLBM(cfg["nx"], cfg["ny"], cfg["q"],
                  cfg["mfp"] if cfg.get("mfp_field") is None else cfg["mfp_field"],
                  bc_kind=cfg["bc"], t_wall=cfg["t_wall"], emulate_3d=cfg["emulate_3d"],
                  relax_mode=cfg.get("relax_mode", 0), theta=THETA,
                  w_field=cfg.get("w_field"), specularity=cfg.get("specularity", (0.0,) * 4),
                  speed=cfg.get("speed", 1.0))
    if state is None:
        m.init_temperature(cfg["dT"].astype(np.float64))
    else:
        m.set_state(state)
    if not flux_peak:
        m.step(steps)
        return m
    peak = 0.0
    for n in range(steps + 1):
        if n:
            m.step()
        qx, qy = m.heat_flux()
        peak = max(peak, float(np.abs(qx).max()), float(np.abs(qy).max()))
    m.flux_peak = peak
    return m


def gpu_handle(cfg, storage=0, variant=None, options=None):
    import paper_1911_00180_gb300 as wl
    mfp = cfg.get("mfp")
    if mfp is None:
        mfp = 0.0
    h = wl.WormLBM(cfg["nx"], cfg["ny"], cfg["q"], mfp=mfp,
                   mfp_field=cfg.get("mfp_field"), bc=cfg["bc"], t_wall=cfg["t_wall"],
                   storage=storage, emulate_3d=cfg["emulate_3d"],
                   relax_mode=cfg.get("relax_mode", 0), theta=THETA,
                   specularity=cfg.get("specularity", (0.0,) * 4),
                   speed=cfg.get("speed", 1.0))
    if variant is not None:
        h.wlbm_set_option(wl.wlbm.OPT_STEP_VARIANT, variant)
    for key, value in (options or {}).items():
        h.wlbm_set_option(key, value)
    return h


def gpu_run(cfg, steps, storage=0, state=None, variant=None, options=None):
    import torch
    h = gpu_handle(cfg, storage, variant, options)
    if state is None:
        h.wlbm_init_temperature(cfg["dT"])
    else:
        h.wlbm_init_temperature(np.zeros((cfg["ny"], cfg["nx"]), np.float32))
        h.wlbm_set_state(torch.as_tensor(state, dtype=torch.float32))
    h.wlbm_step(steps)
    h.wlbm_check()
    dT, qx, qy = h.wlbm_moments()
    st = h.wlbm_get_state()
    torch.cuda.synchronize()
    out = dict(dT=dT.cpu().numpy().astype(np.float64), qx=qx.cpu().numpy().astype(np.float64),
               qy=qy.cpu().numpy().astype(np.float64),
               state=st.cpu().numpy().astype(np.float64), red=h.wlbm_reduce())
    h.close()
    return out


def rel_linf(a, b, scale):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / scale)
