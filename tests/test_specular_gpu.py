"""Specular and specular-diffusive walls (Sec. 2.6, Eq. adiabatic-specular and its linear
combination with Eq. adiabatic-diffuse) on the GPU: parity with the oracle element by
element on ragged grids, through the wall kernels' register-held and looped paths (Q up
to 264), in float32 and bfloat16; and the film conductivity against the discrete-ordinate
Fuchs-Sondheimer ratio with specularity p at sizes the oracle cannot reach."""
import numpy as np
import pytest

import workloads as W
from oracle import transport as T
from tests._pair import gpu_handle, gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu
P, I, A, S = W.PERIODIC, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE, W.ADIABATIC_SPECULAR
TOL32, TOL16, TOL16_STATE = 1e-5, 2e-3, 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401  (fails loudly if the library is missing)


def _cfg(nx, ny, q, bc, spec, mfp, seed, t_wall=(300.6, 299.7, 300.3, 299.9)):
    return dict(nx=nx, ny=ny, q=q, mfp=mfp, bc=bc, t_wall=t_wall, emulate_3d=True,
                specularity=spec, dT=W.random_dT(nx, ny, seed=seed, scale=0.5))


CASES = [
    ("film_specular", _cfg(83, 29, 32, (I, I, S, S), (0, 0, 0, 0), 6.0, 1)),
    ("box_mixed", _cfg(45, 37, 24, (A, S, A, A), (0.3, 0, 0.7, 1.0), 3.0, 2)),
    ("periodic_x", _cfg(40, 51, 48, (P, P, S, A), (0, 0, 0, 0.5), 9.0, 3)),
    ("q264_loops", _cfg(12, 10, 264, (S, A, A, S), (0, 0.4, 0.8, 0), 4.0, 4)),
    ("q136_chunk_loop", _cfg(70, 9, 136, (I, I, A, A), (0, 0, 0.5, 0.5), 5.0, 5)),
]


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("name,cfg", CASES)
def test_specular_walls_match_oracle(name, cfg, storage):
    steps = 60
    orc = oracle_run(cfg, steps)
    gpu = gpu_run(cfg, steps, storage)
    amp = max(float(np.abs(cfg["dT"]).max()), 0.6)
    dscale = float(np.abs(oracle_run(cfg, 0).d).max())
    tol, stol = (TOL32, TOL32) if storage == 0 else (TOL16, TOL16_STATE)
    assert rel_linf(gpu["dT"], orc.temperature_dev(), amp) <= tol
    assert rel_linf(gpu["state"][:, 1:-1, 1:-1], orc.d[:, 1:-1, 1:-1], dscale) <= stol
    # energy including the adiabatic walls' ghost cells: every stored value within the
    # state bound, so the sum within that bound times the values summed
    frame_values = cfg["q"] * (cfg["nx"] + 2) * (cfg["ny"] + 2)
    assert abs(gpu["red"][1] - orc.total_energy(include_frame=True)) <= \
        stol * dscale * frame_values


def _band_kappa(nx, ny, q, mfp, bc, spec, warm, avg_steps, every):
    cfg = dict(nx=nx, ny=ny, q=q, mfp=mfp, bc=bc, t_wall=(300.5, 299.5, 300.0, 300.0),
               emulate_3d=True, specularity=spec)
    xs = (np.arange(nx) + 0.5) / nx
    dT = np.ascontiguousarray(np.tile(0.5 - xs, (ny, 1)).astype(np.float32))
    h = gpu_handle(cfg)
    h.wlbm_init_temperature(dT)
    h.wlbm_step(warm)
    vals = []
    for _ in range(avg_steps // every):
        h.wlbm_step(every)
        vals.append(h.wlbm_reduce()[7])
    h.close()
    return float(np.mean(vals))


@pytest.mark.parametrize("p,kind", [(0.5, A), (1.0, S)])
def test_specular_film_conductivity_converges(p, kind):
    """Kn = 1, Q = 64: film-to-bulk band conductivity with walls of specularity p,
    Richardson over N_y = 32, 64 against the discrete-ordinate ratio (1 for p = 1)."""
    q, kn = 64, 1.0
    ratio = {}
    for ny in (32, 64):
        mfp, nx = kn * ny, 8 * ny
        kb = _band_kappa(nx, ny, q, mfp, (I, I, P, P), (0,) * 4, 20 * ny, 20 * ny, 10)
        kf = _band_kappa(nx, ny, q, mfp, (I, I, kind, kind), (0, 0, p, p), 20 * ny, 20 * ny, 10)
        ratio[ny] = kf / kb
    fs = T.fuchs_sondheimer_2d(q, kn * 2.0 / 3.0, p)
    assert abs(ratio[64] - fs) < abs(ratio[32] - fs)
    assert 2 * ratio[64] - ratio[32] == pytest.approx(fs, rel=0.005)
