"""Oracle, part 2: the worm-LBM time step on a framed 2D grid, plain numpy float64.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State.  For each direction i the oracle stores the deviation
    d_i(x) = e_i(x) - w_i e_ref,   e_ref = e_eq(T_ref)
of the discrete directional energy density (DDED) e_i from the reference equilibrium.
The update of Eq. lbm-energy / Eq. algorithm is linear and maps w_i e_ref to itself
(sum_i w_i = 1), so d obeys the same update; only temperatures (Eq. pseudo-T) add e_ref
back.  Arrays have shape (Q, Ny + 2, Nx + 2): a one-cell ghost frame holds the boundary
(Sec. 2.6); anything outside the frame reads as zero.

One step n (n = 1, 2, ...), in the order the paper applies it:
  1. boundary conditions on the ghost frame of state n-1 (Sec. 2.6, "at every time
     step"): adiabatic-diffuse walls, then isotropic blackbody (isothermal) walls, then
     periodic links;
  2. local energy E(x) = sum_i d_i(x)   (Eq. lbm-energy-density);
  3. for every direction i with due worm hop c_i and every cell y (frame included),
     with F = W E and the source cell s = y - c_i:
        propagating:  d_i'(y) = (1 - W(s)) d_i(s) + w_i F(s)
        paused:       d_i'(y) = (1 - W(y)) d_i(y) + w_i F(s)
     (Eq. lbm-energy with e_i^eq = w_i E, read from the garbled Eq.
     lbm-energy-weighting; Eq. algorithm for the paused DDED whose EED still hops).
     W is the corrected weight W_corr of Eq. W-correction; ghost cells of walls have
     W = 0 (no scattering inside a wall), periodic ghost cells copy W across the link.

Readings of passages the paper leaves open:
  * per-cell W in the paused branch: the loss uses W(y), the gain uses W(s);
  * adiabatic diffuse wall (Eq. adiabatic-diffuse, normalisation garbled): a ghost cell
    collects A = sum of its components that do not point into the domain, zeroes them,
    and adds A * w_i (s_i . n) / sum_k w_k (s_k . n) to each inward component i;
    a corner between two diffuse walls uses n = the quadrant diagonal and counts as
    inward only directions strictly inside the quadrant;
  * adiabatic specular and specular-diffusive walls (Eq. adiabatic-specular and the
    linear combination the paper names): with specularity p (1 for a specular wall,
    the wall's `specularity` for a diffuse one, 0 by default), each outward component j
    (s_j . n < 0) gives p d_j to its mirror direction (the normal component flipped) and
    (1 - p) d_j to the diffuse collection; a component parallel to the wall keeps p of
    its value and gives the rest to the collection; inward components receive
    p d_mirror + (1 - p) rho_i A on top of what they hold.  Exactly conserving; p = 0 is
    the diffuse rule;
  * internal sources (Sec. 2.6: isotropic blackbody and anisotropic radiation conditions
    "or, equivalently", internal temperature and radiation sources): listed cells of the
    interior or of a non-periodic wall's ghost frame whose DDEDs are overwritten at every
    step, after the wall conditions and before the periodic links, with w_i e_eq(T_s)
    (Eq. isotropic) or imposed values (Eq. anisotropic); on a wall's ghost cells they make
    an anisotropic radiation wall;
  * corner ghost cells: a periodic link fills them; otherwise an isothermal x-wall,
    then an isothermal y-wall, decides; two adiabatic walls (diffuse or specular) use the
    diffuse corner rule above (a specular corner would map up to three directions onto
    one);
  * heat flux (Eq. q_corr) uses the nominal unit vector s_i of each direction and
    v_g = the propagation speed (1 cell per step unless a band is slower);
  * propagation speed v <= 1 (TAS beyond the unit speed, Sec. 1; one band of a multigray
    run, Sec. 2.1): the hop test compares with v n instead of n, and the relaxation per
    step is W = v / MFP before Eq. W-correction.

Pins: tests/test_oracle_stepper.py (energy conservation on periodic and adiabatic
grids, exact ballistic translation, reduction to standard D2Q8 at W = 1, the moment
recursion, the diffusive Gaussian limit, isothermal steady profile; for a per-cell W
field: conservation through paused steps, which every other placement of W(y) and W(s)
breaks, one step written out term by term, and the uniform field equal to the scalar).
"""
import math

import numpy as np

from . import lattice as L

PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR = 0, 1, 2, 3
ADIABATIC = (ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR)
XM, XP, YM, YP = 0, 1, 2, 3           # wall order: x-, x+, y-, y+
INWARD_NORMAL = {XM: (1, 0), XP: (-1, 0), YM: (0, 1), YP: (0, -1)}


def shift(a, c):
    """b(y) = a(y - c) over the last two axes (y, x), zero where y - c leaves the array."""
    cx, cy = c
    b = np.zeros_like(a)
    ny, nx = a.shape[-2], a.shape[-1]
    ys_dst = slice(max(cy, 0), ny + min(cy, 0))
    ys_src = slice(max(-cy, 0), ny + min(-cy, 0))
    xs_dst = slice(max(cx, 0), nx + min(cx, 0))
    xs_src = slice(max(-cx, 0), nx + min(-cx, 0))
    b[..., ys_dst, xs_dst] = a[..., ys_src, xs_src]
    return b


class WormLBM:
    """Plain FP64 worm-LBM on an nx x ny grid with Q directions."""

    def __init__(self, nx, ny, q, mfp, bc_kind=(0, 0, 0, 0), t_wall=(300.0,) * 4,
                 emulate_3d=True, relax_mode=0, t_ref=300.0, theta=L.THETA_DEFAULT,
                 w_field=None, specularity=(0.0,) * 4, speed=1.0):
        self.nx, self.ny, self.q = nx, ny, q
        # propagation speed in cells per step (TAS beyond the unit speed, Sec. 1): one
        # band of a multigray run; its relaxation per step is W = speed / MFP
        self.speed = float(speed)
        self.bc_kind = tuple(int(k) for k in bc_kind)
        self.t_wall = tuple(float(t) for t in t_wall)
        # specularity of each adiabatic wall: 1 for specular walls, the given fraction
        # for diffuse ones
        self.spec = tuple(1.0 if k == ADIABATIC_SPECULAR else
                          (float(p) if k == ADIABATIC_DIFFUSE else 0.0)
                          for k, p in zip(self.bc_kind, specularity))
        if any(not (0.0 <= p <= 1.0) for p in self.spec):
            raise ValueError("specularity must lie in [0, 1]")
        if (self.bc_kind[XM] == PERIODIC) != (self.bc_kind[XP] == PERIODIC) or \
           (self.bc_kind[YM] == PERIODIC) != (self.bc_kind[YP] == PERIODIC):
            raise ValueError("periodic walls come in opposite pairs")
        self.t_ref, self.theta = float(t_ref), float(theta)
        self.dirs = L.ring_directions(q)
        self.s_hat = L.unit_vectors(self.dirs)
        self.w = L.angular_weights(self.dirs)
        self.lam_corr = L.lambda_corr(self.dirs)
        self.sched = L.TasSchedule(q, self.speed)
        self.e_ref = float(L.e_eq(self.t_ref, self.theta))
        if w_field is not None:            # direct W (tests of the W = 1 limit, adjoint)
            wc = np.broadcast_to(np.asarray(w_field, np.float64), (ny, nx)).copy()
        else:
            mfp = np.broadcast_to(np.asarray(mfp, np.float64), (ny, nx))
            if np.any(mfp <= 0):
                raise ValueError("MFP must be positive")
            wc = L.relax_weight(mfp / self.speed, self.lam_corr, emulate_3d, relax_mode)
        if wc.max() > 1.0:
            # Appendix A: the paused step is stable only for W <= 1.
            raise ValueError("unstable: max W_corr = %g > 1" % wc.max())
        self.w_int = wc
        self.wf = self._frame_scalar(wc)
        self.d = np.zeros((q, ny + 2, nx + 2))
        self.n = 0
        self.sources = []                  # (Y, X, deviations (q,)) in framed indices

    # ----------------------------------------------------------------- geometry
    def _frame_scalar(self, interior):
        """Embed an interior field in the frame: walls 0, periodic links copied."""
        f = np.zeros((self.ny + 2, self.nx + 2))
        f[1:-1, 1:-1] = interior
        self._periodic_links(f[None])
        return f

    def _periodic_links(self, a):
        """Periodic boundary of Sec. 2.6 on arrays (..., Ny+2, Nx+2): the y link first
        (over all columns unless x is periodic too), then the x link over all rows."""
        nx, ny = self.nx, self.ny
        xper = self.bc_kind[XM] == PERIODIC
        yper = self.bc_kind[YM] == PERIODIC
        if yper:
            xs = slice(1, nx + 1) if xper else slice(0, nx + 2)
            a[..., 0, xs] = a[..., ny, xs]
            a[..., ny + 1, xs] = a[..., 1, xs]
        if xper:
            a[..., :, 0] = a[..., :, nx]
            a[..., :, nx + 1] = a[..., :, 1]

    def _edge_cells(self, wall):
        """Framed (Y, X) indices of a wall's ghost cells, corners excluded."""
        nx, ny = self.nx, self.ny
        if wall == XM:
            return [(y, 0) for y in range(1, ny + 1)]
        if wall == XP:
            return [(y, nx + 1) for y in range(1, ny + 1)]
        if wall == YM:
            return [(0, x) for x in range(1, nx + 1)]
        return [(ny + 1, x) for x in range(1, nx + 1)]

    def _corners(self):
        """(Y, X, x-wall, y-wall) for the four corner ghost cells."""
        nx, ny = self.nx, self.ny
        return [(0, 0, XM, YM), (0, nx + 1, XP, YM),
                (ny + 1, 0, XM, YP), (ny + 1, nx + 1, XP, YP)]

    # -------------------------------------------------------- boundary conditions
    def diffuse_split(self, normal, strict_quadrant=False):
        """Inward mask and re-emission fractions rho_i = w_i (s_i.n) / sum over inward."""
        nxn, nyn = normal
        dirs = np.array(self.dirs)
        if strict_quadrant:
            inward = (dirs[:, 0] * nxn > 0) & (dirs[:, 1] * nyn > 0)
        else:
            inward = (dirs[:, 0] * nxn + dirs[:, 1] * nyn) > 0
        nrm = np.array([nxn, nyn], np.float64)
        nrm /= np.linalg.norm(nrm)
        cosn = self.s_hat @ nrm
        rho = np.where(inward, self.w * cosn, 0.0)
        rho /= rho.sum()
        return inward, rho

    def mirror_index(self, normal):
        """Index of each direction reflected at a wall with an axis-aligned normal."""
        index = {tuple(v): i for i, v in enumerate(self.dirs)}
        fx, fy = (-1, 1) if normal[0] != 0 else (1, -1)
        return np.array([index[(fx * a, fy * b)] for (a, b) in self.dirs])

    def _diffuse_cell(self, yy, xx, normal, strict, p=0.0):
        """One adiabatic ghost cell, or (yy, xx) index arrays of a wall's ghost cells
        that share the normal; each cell is handled on its own.  p: specularity (edges
        only)."""
        inward, rho = self.diffuse_split(normal, strict)
        yy, xx = np.atleast_1d(yy)[None, :], np.atleast_1d(xx)[None, :]
        out_i, in_i = np.flatnonzero(~inward)[:, None], np.flatnonzero(inward)[:, None]
        a = self.d[out_i, yy, xx].sum(axis=0)           # collected energy per cell
        if p == 0.0:
            self.d[out_i, yy, xx] = 0.0
            self.d[in_i, yy, xx] += rho[in_i] * a[None, :]
            return
        mirror = self.mirror_index(normal)
        old = self.d[:, yy[0], xx[0]]                   # (q, cells), a copy
        dots = np.array(self.dirs) @ np.array(normal)
        o, i = out_i[:, 0], in_i[:, 0]
        self.d[out_i, yy, xx] = np.where((dots[o] == 0)[:, None], p * old[o], 0.0)
        self.d[in_i, yy, xx] = old[i] + p * old[mirror[i]] + (1.0 - p) * rho[i][:, None] * a[None, :]

    def delta_e(self, t):
        """e_eq(T) - e_ref in float64."""
        return float(L.e_eq(t, self.theta)) - self.e_ref

    def apply_bc(self):
        k = self.bc_kind
        # 1. adiabatic diffuse walls (edges), then diffuse-diffuse corners
        for wall in (XM, XP, YM, YP):
            if k[wall] in ADIABATIC:
                cells = np.array(self._edge_cells(wall))
                self._diffuse_cell(cells[:, 0], cells[:, 1], INWARD_NORMAL[wall], False,
                                   self.spec[wall])
        for (yy, xx, xw, yw) in self._corners():
            if k[xw] in ADIABATIC and k[yw] in ADIABATIC:
                n = (INWARD_NORMAL[xw][0], INWARD_NORMAL[yw][1])
                self._diffuse_cell(yy, xx, n, True)
        # 2. isotropic blackbody walls (Eq. isotropic): d_i = w_i (e_eq(T_w) - e_ref)
        for wall in (XM, XP, YM, YP):
            if k[wall] == ISOTHERMAL:
                de = self.delta_e(self.t_wall[wall])
                for (yy, xx) in self._edge_cells(wall):
                    self.d[:, yy, xx] = self.w * de
        for (yy, xx, xw, yw) in self._corners():
            if k[xw] == PERIODIC or k[yw] == PERIODIC:
                continue
            if k[xw] == ISOTHERMAL:
                self.d[:, yy, xx] = self.w * self.delta_e(self.t_wall[xw])
            elif k[yw] == ISOTHERMAL:
                self.d[:, yy, xx] = self.w * self.delta_e(self.t_wall[yw])
        # 3. internal sources and radiation cells (Eq. isotropic / Eq. anisotropic)
        for (yy, xx, v) in self.sources:
            self.d[:, yy, xx] = v
        # 4. periodic links
        self._periodic_links(self.d)

    def set_sources(self, cells, temps=None, imposed=None):
        """Cells (x, y) with -1 <= x <= nx, -1 <= y <= ny (not on a periodic side's ghost
        frame) kept at temperature temps[k] (isotropic: e_i = w_i e_eq(T)) or at the
        imposed absolute DDEDs imposed[k] (Q values each).  An empty list removes them."""
        per = [self.bc_kind[s] == PERIODIC for s in (XM, XP, YM, YP)]
        out = []
        for k, (x, y) in enumerate(cells):
            if not (-1 <= x <= self.nx and -1 <= y <= self.ny):
                raise ValueError("source outside the frame")
            sides = [s for s, hit in ((XM, x == -1), (XP, x == self.nx), (YM, y == -1),
                                      (YP, y == self.ny)) if hit]
            if any(per[s] for s in sides):
                raise ValueError("source on a periodic ghost cell")
            if imposed is not None:
                v = np.asarray(imposed[k], np.float64) - self.w * self.e_ref
            else:
                v = self.w * self.delta_e(float(temps[k]))
            out.append((y + 1, x + 1, v))
        self.sources = out

    # ------------------------------------------------------------------- state
    def init_temperature(self, dT):
        """Equilibrium start (Sec. 2.4: the weights set the initial conditions):
        e_i = w_i e_eq(T_ref + dT).  Frame cells copy their nearest interior cell."""
        dT = np.asarray(dT, np.float64).reshape(self.ny, self.nx)
        de = L.e_eq(self.t_ref + dT, self.theta) - self.e_ref
        de_f = np.pad(de, 1, mode="edge")
        self.d = self.w[:, None, None] * de_f[None]
        self.n = 0

    def set_state(self, d_framed):
        self.d = np.array(d_framed, dtype=np.float64, copy=True)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self._one_step()

    def _one_step(self):
        n = self.n + 1
        self.apply_bc()
        hops, paused = self.sched.advance(n)
        self.d = self.collide_stream(self.d, hops, paused)
        self.n = n

    def collide_stream(self, d, hops, paused):
        """One update of Eq. lbm-energy / Eq. algorithm on a framed state d whose ghost
        frame already holds the boundary values."""
        e_loc = d.sum(axis=0)                        # Eq. lbm-energy-density
        f = self.wf * e_loc                          # scattered energy W E at each cell
        keep = 1.0 - self.wf                         # (1 - W)
        new = np.empty_like(d)
        for i in range(self.q):
            c = L.BASIC_HOPS[hops[i]]
            gain = self.w[i] * shift(f, c)           # EED always hops: w_i W(s) E(s)
            if paused[i]:
                new[i] = keep * d[i] + gain
            else:
                new[i] = shift(keep * d[i], c) + gain
        return new

    # ---------------------------------------------------------------- moments
    def energy_dev(self):
        """E(x) - e_ref on the interior (Eq. lbm-energy-density)."""
        return self.d[:, 1:-1, 1:-1].sum(axis=0)

    def temperature_dev(self):
        """T(x) - T_ref by Eq. pseudo-T, float64."""
        e = self.e_ref + self.energy_dev()
        return L.temperature(e, self.theta) - self.t_ref

    def heat_flux(self):
        """(q_x, q_y) by Eq. q_corr with v_g = speed (1 by default) and c_i/|c_i| = s_i."""
        di = self.d[:, 1:-1, 1:-1]
        qx = np.tensordot(self.s_hat[:, 0], di, axes=(0, 0))
        qy = np.tensordot(self.s_hat[:, 1], di, axes=(0, 0))
        if self.speed != 1.0:
            qx, qy = self.speed * qx, self.speed * qy
        return qx, qy

    def mean_moments(self, nsteps):
        """Advance nsteps steps and return the means of T - T_ref, q_x and q_y over the
        nsteps states reached (the running average of the flux over 10 steps of Sec. 4.3,
        which smooths the TAS fluctuations)."""
        acc_t = acc_x = acc_y = 0.0
        for _ in range(nsteps):
            self.step()
            qx, qy = self.heat_flux()
            acc_t = acc_t + self.temperature_dev()
            acc_x = acc_x + qx
            acc_y = acc_y + qy
        return acc_t / nsteps, acc_x / nsteps, acc_y / nsteps

    def total_energy(self, include_frame=False):
        """Sum of E - e_ref over the interior, or over the interior plus the ghost cells
        that hold energy of the system: those of adiabatic (diffuse or specular) walls (a
        corner only between two of them).  Periodic ghosts are copies; isothermal ghosts are the
        imposed reservoir, reset by every boundary pass (Sec. 2.6)."""
        if not include_frame:
            return float(self.d[:, 1:-1, 1:-1].sum())
        k = self.bc_kind
        fh, fw = self.ny + 2, self.nx + 2
        side_x = np.full(fw, -1)
        side_x[0], side_x[-1] = XM, XP
        side_y = np.full(fh, -1)
        side_y[0], side_y[-1] = YM, YP
        total = float(self.d[:, 1:-1, 1:-1].sum())
        for yy in range(fh):
            for xx in range(fw):
                sides = [s for s in (side_x[xx], side_y[yy]) if s >= 0]
                if sides and all(k[s] in ADIABATIC for s in sides):
                    total += float(self.d[:, yy, xx].sum())
        return total
