"""torch.autograd wrapper of a checkpointed worm-LBM run.

`wlbm_run(mfp_field, t_wall, dT0, spec)` runs `spec["steps"]` steps from the start field
dT0 (K above T_ref) with per-cell mean free paths `mfp_field` (cells) and wall
temperatures `t_wall` (4, K) and returns the final temperature deviation field.  `spec`
holds nx, ny, q, bc, steps, ckpt and optionally emulate_3d, relax_mode, specularity (4)
and speed (the band's propagation speed, cells per step).
`wlbm_run_moments(...)` returns the final (dT, q_x, q_y) fields instead, so that an
objective can use the heat flux (Eq. q_corr), e.g. the apparent conductivity of a film
mean(q_x) * nx / (D (e(T_h) - e(T_c))), whose explicit dependence on t_wall torch then
differentiates itself.  The backward pass calls the library's adjoint (checkpoints every
`spec["ckpt"]` steps, recompute in between) and returns dJ/dMFP, dJ/dT_wall and
dJ/d(dT0).  All arithmetic runs in libwlbm's kernels; this module only moves tensors.
"""
import torch

from .wlbm import WormLBM


class _WormLBMRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mfp_field, t_wall, dT0, spec):
        h = WormLBM(spec["nx"], spec["ny"], spec["q"], mfp_field=mfp_field.detach(),
                    bc=spec["bc"], t_wall=tuple(float(t) for t in t_wall.detach().cpu()),
                    emulate_3d=spec.get("emulate_3d", True),
                    relax_mode=spec.get("relax_mode", 0),
                    specularity=spec.get("specularity", (0.0,) * 4),
                    speed=spec.get("speed", 1.0))
        h.wlbm_adjoint_forward(dT0.detach(), spec["steps"], spec["ckpt"])
        dT, qx, qy = h.wlbm_moments()
        ctx.h = h
        ctx.t_wall_device = t_wall.device
        return dT.clone(), qx.clone(), qy.clone()

    @staticmethod
    def backward(ctx, grad_dT, grad_qx, grad_qy):
        h = ctx.h
        seed = lambda g: None if g is None else g.contiguous()
        g_mfp, g_tw, g_dT0 = h.wlbm_adjoint_backward(seed(grad_dT), dJ_dqx=seed(grad_qx),
                                                     dJ_dqy=seed(grad_qy))
        h.close()
        ctx.h = None
        return (g_mfp, torch.tensor(g_tw, dtype=torch.float64, device=ctx.t_wall_device),
                g_dT0, None)


def wlbm_run(mfp_field, t_wall, dT0, spec):
    return _WormLBMRun.apply(mfp_field, t_wall, dT0, spec)[0]


def wlbm_run_moments(mfp_field, t_wall, dT0, spec):
    return _WormLBMRun.apply(mfp_field, t_wall, dT0, spec)
