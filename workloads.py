"""Seeded synthetic inputs for the worm-LBM workloads (shared by the tests, the bench and
the smoke check).

This module holds input generation only: temperature-deviation fields, mean-free-path
fields and run descriptions.  It contains none of the method's arithmetic (no weights,
no equilibrium energies, no schedule); the oracle and the CUDA library each turn these
inputs into lattice state on their own.  Every array is float32 (the dtype the C-ABI
takes) and is produced by numpy's PCG64 generator from an integer seed, so both sides
receive bit-identical inputs on any host.

Workloads (lattice units: one cell = one MFP grid spacing, one step = one time step):

  gaussian_c1   64 x 64 periodic, Q = 16, MFP = 8 cells, 3D emulation on, one Gaussian
                pulse (sigma0 = 4 cells, 1 K over 300 K) at a seed-drawn centre, 500 steps.
  pulses_c2     2048 x 2048 periodic, Q = 64, uniform MFP drawn log-uniform in
                [1, 1000] cells, 16 Gaussian pulses (sigma0 log-uniform in [4, 32],
                1 K each), 2000 steps; limits MFP = inf (ballistic) and MFP = 0.5.
  film_c3       4096 x 256 in-plane film, Q = 128, isothermal x walls 301 / 300 K,
                adiabatic-diffuse y walls, MFP = Kn * 256, linear initial profile.
  batch_c4      96 films, thickness log-uniform [16, 512], aspect uniform [8, 32],
                Kn log-uniform [0.01, 100], Q from {16, 32, 64, 128, 256}.
  adjoint_c5    1024 x 1024, Q = 64, log-normal MFP field exp(ln 8 + 0.5 g) with g a
                unit-variance Gaussian random field of correlation length 32 cells,
                isothermal x walls at 300 K, periodic y, central pulse sigma0 = 32.
Each generator takes size overrides so the tests can run reduced versions of the same
recipe.
"""
import math

import numpy as np

PERIODIC, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_SPECULAR = 0, 1, 2, 3


def _rng(seed):
    return np.random.default_rng(np.uint64(seed))


def gaussian_field(nx, ny, centres, sigmas, amps, periodic=True):
    """Sum of Gaussian bumps amp * exp(-r^2 / (2 sigma^2)) (minimum-image distance when
    periodic), float64; callers cast."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = np.zeros((ny, nx))
    for (cx, cy), s, a in zip(centres, sigmas, amps):
        dx = x - cx
        dy = y - cy
        if periodic:
            dx = dx - nx * np.round(dx / nx)
            dy = dy - ny * np.round(dy / ny)
        out += a * np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
    return out


def gaussian_c1(seed=1, n=64, q=16, mfp=8.0, sigma0=4.0, amp=1.0, steps=500):
    rng = _rng(seed)
    cx, cy = rng.integers(0, n, size=2)
    dT = gaussian_field(n, n, [(float(cx), float(cy))], [sigma0], [amp]).astype(np.float32)
    return dict(name="gaussian_c1", nx=n, ny=n, q=q, mfp=float(mfp), mfp_field=None,
                bc=(PERIODIC,) * 4, t_wall=(300.0,) * 4, emulate_3d=True, relax_mode=0,
                dT=dT, steps=steps, amp=amp)


def pulses_c2(seed=2, n=2048, q=64, mfp=None, npulse=16, steps=2000, relax_mode=0):
    rng = _rng(seed)
    if mfp is None:
        mfp = float(math.exp(rng.uniform(math.log(1.0), math.log(1000.0))))
    else:
        rng.uniform()                      # keep the stream aligned with the default
    centres = [tuple(map(float, rng.uniform(0, n, size=2))) for _ in range(npulse)]
    sigmas = [float(math.exp(rng.uniform(math.log(4.0), math.log(32.0))))
              for _ in range(npulse)]
    dT = gaussian_field(n, n, centres, sigmas, [1.0] * npulse).astype(np.float32)
    return dict(name="pulses_c2", nx=n, ny=n, q=q, mfp=float(mfp), mfp_field=None,
                bc=(PERIODIC,) * 4, t_wall=(300.0,) * 4, emulate_3d=False,
                relax_mode=relax_mode, dT=dT, steps=steps, amp=1.0)


def film_c3(kn=1.0, nx=4096, ny=256, q=128, t_hot=301.0, t_cold=300.0, steps=2000):
    x = (np.arange(nx, dtype=np.float64) + 1.0) / (nx + 1.0)
    prof = (t_hot - 300.0) + (t_cold - t_hot) * x
    dT = np.broadcast_to(prof[None, :], (ny, nx)).astype(np.float32)
    return dict(name="film_c3", nx=nx, ny=ny, q=q, mfp=float(kn * ny), mfp_field=None,
                bc=(ISOTHERMAL, ISOTHERMAL, ADIABATIC_DIFFUSE, ADIABATIC_DIFFUSE),
                t_wall=(t_hot, t_cold, 300.0, 300.0), emulate_3d=True, relax_mode=0,
                dT=np.ascontiguousarray(dT), steps=steps, amp=t_hot - t_cold, kn=kn)


def batch_c4(seed=4, count=96, thick=(16, 512), aspect=(8, 32), kn=(0.01, 100.0),
             qs=(16, 32, 64, 128, 256), steps=200):
    rng = _rng(seed)
    out = []
    for k in range(count):
        ny = int(round(math.exp(rng.uniform(math.log(thick[0]), math.log(thick[1])))))
        nx = int(round(ny * rng.uniform(*aspect)))
        knk = float(math.exp(rng.uniform(math.log(kn[0]), math.log(kn[1]))))
        q = int(qs[int(rng.integers(0, len(qs)))])
        inst = film_c3(kn=knk, nx=nx, ny=ny, q=q, steps=steps)
        inst["name"] = "batch_c4[%d]" % k
        out.append(inst)
    return out


def lognormal_mfp(nx, ny, seed, corr=32.0, mu=math.log(8.0), sigma=0.5):
    """exp(mu + sigma g), g = white noise blurred by a periodic Gaussian of standard
    deviation `corr` cells and rescaled to unit variance."""
    rng = _rng(seed)
    noise = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    kern = np.exp(-2.0 * (math.pi * corr) ** 2 * (kx * kx + ky * ky))
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * kern))
    g = (g - g.mean()) / g.std()
    return np.exp(mu + sigma * g).astype(np.float32)


def adjoint_c5(seed=5, n=1024, q=64, sigma0=32.0, steps=1000, ckpt=50):
    mfp = lognormal_mfp(n, n, seed)
    dT = gaussian_field(n, n, [(n / 2.0, n / 2.0)], [sigma0], [1.0],
                        periodic=False).astype(np.float32)
    return dict(name="adjoint_c5", nx=n, ny=n, q=q, mfp=None, mfp_field=mfp,
                bc=(ISOTHERMAL, ISOTHERMAL, PERIODIC, PERIODIC), t_wall=(300.0,) * 4,
                emulate_3d=True, relax_mode=0, dT=dT, steps=steps, ckpt=ckpt, amp=1.0,
                probe_x=(3 * n) // 4)


def random_dT(nx, ny, seed, scale=1.0):
    """Unstructured test field (normal deviates), for parity cases with no physics."""
    return (_rng(seed).standard_normal((ny, nx)) * scale).astype(np.float32)
