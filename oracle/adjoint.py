"""Oracle, part 3: the exact adjoint (reverse mode) of the worm-LBM run, plain numpy
float64.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no adjoint; this is the transpose of the linear map the oracle's forward
step applies (oracle/stepper.py), written out term by term.  For step n with recorded
input state d~ (ghost frame already set by the boundary conditions), hops c_k, pause
flags and the framed weight W, the forward update is, for every cell y and s = y - c_k,
    propagating:  d_k'(y) = (1 - W(s)) d~_k(s) + w_k W(s) E~(s)
    paused:       d_k'(y) = (1 - W(y)) d~_k(y) + w_k W(s) E~(s),     E~ = sum_k d~_k.
With lam' the adjoint of d' and a_k(x) = lam'_k(x + c_k) if k propagates, lam'_k(x) if
it pauses, and sigma(x) = sum_k w_k lam'_k(x + c_k):
    lam~_k(x) = (1 - W(x)) a_k(x) + W(x) sigma(x)
    dJ/dW(x) += sum_k [ -d~_k(x) a_k(x) ] + E~(x) sigma(x).
The boundary passes (diffuse, isothermal, periodic) are then transposed in reverse order:
periodic copies add the ghost adjoint to the source cell; isothermal overwrites zero the
adjoint and harvest dJ/dT_wall = sum_i lam~_i w_i de_eq/dT; the diffuse collection sends
sum_k rho_k lam~_k (over inward k) to every collected direction.

Objective (the adjoint workload): J = mean of T - T_ref over a set of interior probe cells
of the final state, T from Eq. pseudo-T.

Pins (tests/test_oracle_adjoint.py): the reverse step equals the transpose of the forward
one-step matrix built column by column on small grids with every wall kind, and the
gradients equal central finite differences of the forward oracle.
"""
import numpy as np

from . import lattice as L
from .stepper import (WormLBM, shift, PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC,
                      XM, XP, YM, YP, INWARD_NORMAL)


def de_dT(t, theta):
    """d e_eq / dT of Eq. gray-energy-density (unit prefactor)."""
    x = theta / t
    e = 1.0 / np.expm1(x)
    return e * (1.0 + e) * x / t


def dT_dE(e, theta):
    """d T / d E of Eq. pseudo-T: T = theta / ln(1 + 1/E)."""
    lg = np.log1p(1.0 / e)
    return theta / (lg * lg * e * (1.0 + e))


def dwcorr_dmfp(mfp, lam_corr, emulate_3d, relax_mode=0):
    """Derivative of the per-cell relaxation weight with respect to the MFP."""
    f = 1.5 if emulate_3d else 1.0
    w = 1.0 / mfp
    wc = f * (w + w * w * (lam_corr - 1.0))
    d = -f * (1.0 + 2.0 * w * (lam_corr - 1.0)) / (mfp * mfp)
    if relax_mode == 1:
        d = d * np.exp(-wc)
    return d


def reverse_step(m, lam_p, d_in, hops, paused):
    """Adjoint of collide_stream: returns (lam~, dJ/dW framed) for the recorded input."""
    W = m.wf
    sigma = np.zeros_like(W)
    a = np.empty_like(lam_p)
    for k in range(m.q):
        c = L.BASIC_HOPS[hops[k]]
        back = shift(lam_p[k], (-c[0], -c[1]))          # lam'_k(x + c_k)
        sigma += m.w[k] * back
        a[k] = lam_p[k] if paused[k] else back
    lam_t = (1.0 - W)[None] * a + (W * sigma)[None]
    gW = -(d_in * a).sum(axis=0) + d_in.sum(axis=0) * sigma
    return lam_t, gW


def _periodic_links_T(m, a):
    """Transpose of WormLBM._periodic_links on (..., Ny+2, Nx+2), in place."""
    nx, ny = m.nx, m.ny
    xper = m.bc_kind[XM] == PERIODIC
    yper = m.bc_kind[YM] == PERIODIC
    if xper:                                     # forward: col 0 <- col nx, nx+1 <- 1
        a[..., :, nx] += a[..., :, 0]
        a[..., :, 1] += a[..., :, nx + 1]
        a[..., :, 0] = 0.0
        a[..., :, nx + 1] = 0.0
    if yper:
        xs = slice(1, nx + 1) if xper else slice(0, nx + 2)
        a[..., ny, xs] += a[..., 0, xs]
        a[..., 1, xs] += a[..., ny + 1, xs]
        a[..., 0, xs] = 0.0
        a[..., ny + 1, xs] = 0.0


def bc_transpose(m, lam):
    """Transpose of WormLBM.apply_bc (linear part) on an adjoint state, in place.
    Returns dJ/dT_wall[4] harvested from the isothermal overwrites."""
    k = m.bc_kind
    g_t = np.zeros(4)
    _periodic_links_T(m, lam)
    # isothermal overwrites (forward pass 2): harvest, then zero
    for (yy, xx, xw, yw) in reversed(m._corners()):
        if k[xw] == PERIODIC or k[yw] == PERIODIC:
            continue
        wall = xw if k[xw] == ISOTHERMAL else (yw if k[yw] == ISOTHERMAL else None)
        if wall is None:
            continue
        g_t[wall] += float((lam[:, yy, xx] * m.w).sum()) * de_dT(m.t_wall[wall], m.theta)
        lam[:, yy, xx] = 0.0
    for wall in (YP, YM, XP, XM):
        if k[wall] == ISOTHERMAL:
            dd = de_dT(m.t_wall[wall], m.theta)
            for (yy, xx) in m._edge_cells(wall):
                g_t[wall] += float((lam[:, yy, xx] * m.w).sum()) * dd
                lam[:, yy, xx] = 0.0
    # diffuse walls (forward pass 1): collected directions receive sum rho_k lam_k
    for (yy, xx, xw, yw) in reversed(m._corners()):
        if k[xw] in ADIABATIC and k[yw] in ADIABATIC:
            n = (INWARD_NORMAL[xw][0], INWARD_NORMAL[yw][1])
            _diffuse_T(m, lam, yy, xx, n, True)
    for wall in (YP, YM, XP, XM):
        if k[wall] in ADIABATIC:
            for (yy, xx) in m._edge_cells(wall):
                _diffuse_T(m, lam, yy, xx, INWARD_NORMAL[wall], False, m.spec[wall])
    return g_t


def _diffuse_T(m, lam, yy, xx, normal, strict, p=0.0):
    """Transpose of the adiabatic ghost-cell rule: inward components keep their adjoint;
    an outward one takes p lam_mirror + (1 - p) S, a parallel one p lam + (1 - p) S, with
    S = sum over inward of rho_i lam_i."""
    inward, rho = m.diffuse_split(normal, strict)
    s = float((lam[inward, yy, xx] * rho[inward]).sum())
    if p == 0.0:
        lam[~inward, yy, xx] = s
        return
    mirror = m.mirror_index(normal)
    dots = np.array(m.dirs) @ np.array(normal)
    old = lam[:, yy, xx].copy()
    for j in np.flatnonzero(~inward):
        own = old[mirror[j]] if dots[j] < 0 else old[j]
        lam[j, yy, xx] = p * own + (1.0 - p) * s


class AdjointRun:
    """Forward run with recording, then the reverse sweep.

    probe: boolean (ny, nx) mask of the interior cells averaged in J.
    objective: "temperature" (J = mean of T - T_ref over the probe) or "flux_x" (J = mean
    of q_x over the probe, Eq. q_corr; the effective conductivity of a film is this mean
    over the interior times N_x / (D (e(T_h) - e(T_c))))."""

    def __init__(self, model_kwargs, dT0, steps, probe, objective="temperature"):
        self.kw = dict(model_kwargs)
        self.dT0 = np.asarray(dT0, np.float64)
        self.steps = steps
        self.probe = np.asarray(probe, bool)
        if objective not in ("temperature", "flux_x"):
            raise ValueError("objective is 'temperature' or 'flux_x'")
        self.objective_kind = objective

    def model(self, **over):
        kw = dict(self.kw)
        kw.update(over)
        return WormLBM(**kw)

    def objective(self, m):
        if self.objective_kind == "flux_x":
            return float(m.heat_flux()[0][self.probe].mean())
        t = m.temperature_dev()
        return float(t[self.probe].mean())

    def forward(self, **over):
        m = self.model(**over)
        m.init_temperature(self.dT0)
        m.step(self.steps)
        return self.objective(m)

    def gradients(self):
        m = self.model()
        m.init_temperature(self.dT0)
        rec = []
        for n in range(1, self.steps + 1):
            m.apply_bc()
            hops, paused = m.sched.advance(n)
            rec.append((m.d.copy(), hops, paused))
            m.d = m.collide_stream(m.d, hops, paused)
            m.n = n
        J = self.objective(m)
        lam = np.zeros_like(m.d)
        if self.objective_kind == "flux_x":
            # q_x(x) = v sum_i s_ix d_i(x): dJ/dd_i(x) = v s_ix over the probe cells
            g = self.probe / self.probe.sum()
            lam[:, 1:-1, 1:-1] = m.speed * m.s_hat[:, 0][:, None, None] * g[None]
        else:
            e_abs = m.e_ref + m.energy_dev()
            g = np.where(self.probe, dT_dE(e_abs, m.theta), 0.0) / self.probe.sum()
            lam[:, 1:-1, 1:-1] = g[None]
        gW = np.zeros_like(m.wf)
        g_t = np.zeros(4)
        for d_in, hops, paused in reversed(rec):
            lam, gw = reverse_step(m, lam, d_in, hops, paused)
            gW += gw
            g_t += bc_transpose(m, lam)
        _periodic_links_T(m, gW[None])
        g_wc = gW[1:-1, 1:-1]
        # initial condition: interior cells plus the frame copies of their neighbours
        lam0 = lam.copy()
        g_e0 = np.zeros((m.ny, m.nx))
        sw = (lam0 * m.w[:, None, None]).sum(axis=0)
        yi = np.clip(np.arange(m.ny + 2) - 1, 0, m.ny - 1)
        xi = np.clip(np.arange(m.nx + 2) - 1, 0, m.nx - 1)
        np.add.at(g_e0, (yi[:, None], xi[None, :]), sw)
        g_dT0 = g_e0 * de_dT(m.t_ref + self.dT0, m.theta)
        out = dict(J=J, dJ_dWcorr=g_wc, dJ_dTwall=g_t, dJ_ddT0=g_dT0)
        if self.kw.get("w_field") is None:
            mfp = np.broadcast_to(np.asarray(self.kw["mfp"], np.float64), (m.ny, m.nx))
            # W = speed / MFP: the weight is a function of MFP / speed
            v = m.speed
            out["dJ_dmfp"] = g_wc * dwcorr_dmfp(mfp / v, m.lam_corr,
                                                self.kw.get("emulate_3d", True),
                                                self.kw.get("relax_mode", 0)) / v
        return out
