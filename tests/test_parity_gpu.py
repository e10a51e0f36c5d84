"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances.  Temperature: relative L-inf of the pulse (or wall) amplitude, 1e-5 for
float32 storage and 2e-3 for bfloat16 storage.  Per-direction state and heat flux:
relative to the largest initial per-direction deviation, 1e-5 for float32 storage.
With bfloat16 storage every stored value carries a rounding of up to 2^-9 of its
non-equilibrium part, several times over near walls (ghost values are re-stored by the
wall pass and by the step), so the state is held to 1e-2 of the largest initial
per-direction deviation.  The heat flux with bfloat16 storage is held to TOL16_Q of the
oracle's flux amplitude (the largest |q_x|, |q_y| of the oracle's field); separately, the
flux the library returns must equal the oracle's formula applied to the library's own
state to 1e-5 of the state scale (the moment kernel, free of the storage rounding).  The
ballistic limit is exact (no arithmetic happens there)."""
import math

import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_run, oracle_run, rel_linf

pytestmark = pytest.mark.gpu
P, I, A = W.PERIODIC, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE
TOL32, TOL16 = 1e-5, 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401  (fails loudly if the library is missing)


TOL16_STATE = 1e-2
# bfloat16 heat flux: the benchmark spec's bfloat16 bar, relative to the oracle's flux
# amplitude (the largest |q_x|, |q_y| of any cell at any step of the run: a decaying
# pulse's flux falls by orders of magnitude while the rounding of the stored values does
# not fall with it).
TOL16_Q = 2e-3
# bfloat16 per-direction values of the full-size film and batch runs, relative to the
# largest per-direction wall deviation: next to an isothermal wall of a near-ballistic film
# (W ~ 1/170 at Kn = 1 on 256 rows) the stored non-equilibrium part is of the wall's order
# and round-to-nearest repeats nearly the same rounding every step, so the error of a
# stored value grows towards several of its rounding steps (2^-9 each); the temperature
# there stays within TOL16.
TOL16_STATE_WALL = 2e-2


def _compare(cfg, steps, storage=0, tol=TOL32, state_tol=None, variant=None, options=None,
             q_of_flux=False):
    orc = oracle_run(cfg, steps, flux_peak=storage == 1)
    gpu = gpu_run(cfg, steps, storage, variant=variant, options=options)
    amp = max(float(np.abs(cfg["dT"]).max()),
              max(abs(t - 300.0) for k, t in zip(cfg["bc"], cfg["t_wall"]) if k == I)
              if I in cfg["bc"] else 0.0)
    ref0 = oracle_run(cfg, 0).d
    dscale = float(np.abs(ref0).max())
    e_t = rel_linf(gpu["dT"], orc.temperature_dev(), amp)
    e_s = rel_linf(gpu["state"][:, 1:-1, 1:-1], orc.d[:, 1:-1, 1:-1], dscale)
    qx, qy = orc.heat_flux()
    qscale, qtol = dscale, tol
    if q_of_flux:   # float32 q against the oracle's flux amplitude at the compared step
        qscale = float(max(np.abs(qx).max(), np.abs(qy).max()))
    if storage == 1:
        own = gpu["state"][:, 1:-1, 1:-1]
        e_m = max(rel_linf(gpu["qx"], np.tensordot(orc.s_hat[:, 0], own, axes=(0, 0)), dscale),
                  rel_linf(gpu["qy"], np.tensordot(orc.s_hat[:, 1], own, axes=(0, 0)), dscale))
        assert e_m <= TOL32, ("q of own state", e_m)
        qscale = orc.flux_peak
        qtol = TOL16_Q
    e_q = max(rel_linf(gpu["qx"], qx, qscale), rel_linf(gpu["qy"], qy, qscale))
    where = np.unravel_index(np.argmax(np.abs(gpu["state"][:, 1:-1, 1:-1] - orc.d[:, 1:-1, 1:-1])),
                             orc.d[:, 1:-1, 1:-1].shape)
    print("parity %s %dx%d Q%d %s %d steps: T %.3g  state %.3g at %s  q %.3g (of %s)"
          % ("bf16" if storage == 1 else "fp32", cfg["nx"], cfg["ny"], cfg["q"], cfg["bc"],
             steps, e_t, e_s, where, e_q,
             "flux amplitude" if storage == 1 or q_of_flux else "state scale"))
    assert e_t <= tol, ("T", e_t)
    assert e_s <= (state_tol or tol), ("state", e_s)
    assert e_q <= qtol, ("q", e_q)
    return orc, gpu


def test_c1_gaussian_fp32_full_run():
    """Gaussian pulse, 64 x 64 periodic, Q = 16, MFP = 8 cells, 500 steps."""
    _compare(W.gaussian_c1(seed=1), 500)


def test_c1_gaussian_bf16_full_run():
    _compare(W.gaussian_c1(seed=1), 500, storage=1, tol=TOL16, state_tol=TOL16_STATE)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("storage,tol,stol", [(0, TOL32, None), (1, TOL16, TOL16_STATE)])
@pytest.mark.parametrize("kinds", [(P,) * 4, (I, I, A, A), (A, A, P, P)])
def test_step_kernel_variants(variant, storage, tol, stol, kinds):
    """Every step-kernel variant (0 register-pipelined, 1 per-warp bulk rings, 2
    warp-specialised, 3 TMA tiles) meets the parity tolerances."""
    nx, ny, q = 141, 23, 32
    cfg = dict(nx=nx, ny=ny, q=q, mfp=2.5, bc=kinds, t_wall=(300.8, 300.0, 300.0, 300.0),
               emulate_3d=True, dT=W.gaussian_field(nx, ny, [(70.0, 11.0)], [6.0], [1.0])
               .astype(np.float32))
    _compare(cfg, 90, storage=storage, tol=tol, state_tol=stol, variant=variant)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("fuse", [0, 1])
def test_step_kernel_variants_bitwise_equal(storage, fuse):
    """Variants 0-2 (and the fused periodic mirrors) compute the same arithmetic in the
    same order: equal states bit for bit.  Variant 3 sums E' over the directions in
    kind-sorted order, so it agrees up to float rounding: 1e-5 of the state scale in
    float32, one bfloat16 rounding step (the bfloat16 state tolerance) in bfloat16."""
    import paper_1911_00180_gb300 as wl
    from tests._pair import gpu_handle
    cfg = W.pulses_c2(seed=2, n=157, q=32, npulse=4)
    cfg["mfp"] = 5.0
    out = []
    for variant in (0, 1, 2, 3):
        h = gpu_handle(cfg, storage, variant)
        h.wlbm_set_option(wl.wlbm.OPT_FUSE_PERIODIC, fuse)
        h.wlbm_init_temperature(cfg["dT"])
        h.wlbm_step(33)
        h.wlbm_check()
        out.append(h.wlbm_get_state().cpu().numpy())
        h.close()
    for k in (1, 2):
        assert np.array_equal(out[0], out[k]), k
    # Variant 3 computes ghost cells only where a diffuse wall reads them; ghost cells of
    # periodic axes are copies that the periodic pass rewrites before the next step (and
    # the fused variants mirror instead), not state: compare the interior.
    sl = (slice(None), slice(1, -1), slice(1, -1))
    scale = float(np.abs(out[0]).max())
    tol = (TOL32 if storage == 0 else TOL16_STATE) * scale
    assert np.abs(out[3][sl] - out[0][sl]).max() <= tol


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("kinds", [(P,) * 4, (I, I, A, A)])
def test_tile_loop_and_ring_depths_bitwise_equal(storage, kinds):
    """Variant 3 with one block per tile, with resident blocks looping over the tiles, with
    either ring depth, and (bfloat16) with the cell terms in shared memory: the same
    arithmetic in another schedule, so the same states bit for bit (grids of several tiles
    in both directions, a per-cell MFP field)."""
    import paper_1911_00180_gb300 as wl
    from tests._pair import gpu_handle
    nx, ny, q = 301, 47, 32
    cfg = dict(nx=nx, ny=ny, q=q, mfp=None, mfp_field=np.maximum(
               W.lognormal_mfp(nx, ny, seed=4, corr=6.0), 1.6).astype(np.float32),
               bc=kinds, t_wall=(300.8, 300.0, 300.0, 300.0), emulate_3d=True,
               dT=W.random_dT(nx, ny, seed=8, scale=0.5))
    alt = 8 if storage else 4
    out = []
    runs = [(0, 0, 0), (1, 0, 0), (1, alt, 0), (0, alt, 0)]
    if storage:
        runs += [(0, 6, 0), (0, 0, 1)]   # cell-tile form; 256-column tiles
    for loop, ring, wide in runs:
        h = gpu_handle(cfg, storage, 3)
        h.wlbm_set_option(wl.wlbm.OPT_RING_STAGES, ring)
        h.wlbm_set_option(wl.wlbm.OPT_TILE_LOOP, loop)
        if storage:
            h.wlbm_set_option(wl.wlbm.OPT_BF16_WIDE, wide)
        h.wlbm_init_temperature(cfg["dT"])
        h.wlbm_step(29)
        h.wlbm_check()
        out.append(h.wlbm_get_state().cpu().numpy())
        h.close()
    sl = (slice(None), slice(1, -1), slice(1, -1))
    for k in range(1, len(runs)):
        assert np.array_equal(out[0][sl], out[k][sl]), runs[k]


@pytest.mark.parametrize("storage,tol,stol", [(0, TOL32, None), (1, TOL16, TOL16_STATE)])
@pytest.mark.parametrize("nx,ny,q", [(1, 1, 8), (1, 7, 16), (5, 1, 8), (2, 3, 24), (126, 9, 16),
                                     (127, 17, 8), (258, 41, 40)])
def test_tma_variant_edges_and_field(storage, tol, stol, nx, ny, q):
    """Variant 3 on degenerate grids, on widths around its 128-column tile (126 + 2 ghost
    columns fill one tile exactly, 127 spills one column into a second tile), with a
    per-cell MFP field and mixed walls."""
    # log-normal MFP (a constant field on 1 x 1), kept above the W_corr <= 1 limit
    mfp = (np.full((1, 1), 6.0, np.float32) if nx * ny == 1 else
           np.maximum(W.lognormal_mfp(nx, ny, seed=nx + ny, corr=3.0), 1.6).astype(np.float32))
    cfg = dict(nx=nx, ny=ny, q=q, mfp=None, mfp_field=mfp, bc=(I, A, P, P),
               t_wall=(300.6, 300.0, 300.0, 300.0), emulate_3d=True,
               dT=W.random_dT(nx, ny, seed=nx * ny + q, scale=0.5))
    _compare(cfg, 40, storage=storage, tol=tol, state_tol=stol, variant=3)


@pytest.mark.parametrize("nx,ny,q,bc", [(1, 1, 8, (I, A, P, P)), (7, 3, 16, (A, A, A, A)),
                                        (256, 15, 24, (P, P, I, I)), (257, 14, 16, (P, P, A, A)),
                                        (247, 29, 8, (A, A, P, P)), (248, 9, 40, (A, A, I, I)),
                                        (600, 31, 64, (P, P, P, P)), (520, 43, 32, (A, I, I, A))])
def test_wide_tiles_edges_and_field(nx, ny, q, bc):
    """bfloat16 256-column tiles: widths around one and two tiles (256 interior columns fill
    one tile, 257 spill one into a second; with diffuse walls on both sides the first tile
    starts 8 columns left of the interior and covers the ghost columns of 247, while 248
    spill the right ghost), rows around the 14-row tile, every wall kind, a per-cell MFP
    field; against the oracle."""
    import paper_1911_00180_gb300 as wl
    mfp = (np.full((1, 1), 6.0, np.float32) if nx * ny == 1 else
           np.maximum(W.lognormal_mfp(nx, ny, seed=nx + ny, corr=3.0), 1.6).astype(np.float32))
    cfg = dict(nx=nx, ny=ny, q=q, mfp=None, mfp_field=mfp, bc=bc,
               t_wall=(300.6, 300.0, 300.3, 300.0), emulate_3d=True,
               dT=W.random_dT(nx, ny, seed=nx * ny + q, scale=0.5))
    _compare(cfg, 40, storage=1, tol=TOL16, state_tol=TOL16_STATE, variant=3,
             options={wl.wlbm.OPT_BF16_WIDE: 1})


@pytest.mark.parametrize("storage,tol,stol", [(0, TOL32, None), (1, TOL16, TOL16_STATE)])
@pytest.mark.parametrize("q", [256, 1024])
def test_largest_direction_sets(storage, tol, stol, q):
    """Q = 256 and the largest Q the library takes (1024, M = 128 hops a worm): the
    direction table and the ring of every step kernel at their largest, on a grid of two
    tiles and a ragged tail in x (three 128-column tiles, two 256-column ones) and a
    ragged tile row in y, with mixed walls and a per-cell MFP field; against the oracle.
    The float32 flux is held to 1e-5 of the flux amplitude (the pulse amplitude of q): q
    sums Q directions, at Q = 1024 some 60 times one direction's amplitude, and each
    float32 state value carries about 2e-7 of that amplitude after 24 steps, so the flux
    measured against one direction's amplitude (1.5e-5 at Q = 1024) reflects the size of
    the sum, not an error of the method (2.5e-7 of the flux amplitude)."""
    nx, ny = 300, 17
    cfg = dict(nx=nx, ny=ny, q=q, mfp=None,
               mfp_field=np.maximum(W.lognormal_mfp(nx, ny, seed=q, corr=4.0), 1.6)
               .astype(np.float32),
               bc=(I, A, P, P), t_wall=(300.7, 300.0, 300.0, 300.0),
               emulate_3d=True, dT=W.random_dT(nx, ny, seed=q + 1, scale=0.5))
    _compare(cfg, 24, storage=storage, tol=tol, state_tol=stol, variant=3, q_of_flux=True)


def test_wide_tiles_refused_for_float32():
    import paper_1911_00180_gb300 as wl
    from tests._pair import gpu_handle
    cfg = W.gaussian_c1(seed=1)
    h = gpu_handle(cfg, 0, 3)
    with pytest.raises(Exception):
        h.wlbm_set_option(wl.wlbm.OPT_BF16_WIDE, 1)
    assert h.wlbm_get_option(wl.wlbm.OPT_BF16_WIDE) == 0
    h.close()


def test_init_roundtrip_temperature():
    cfg = W.gaussian_c1(seed=3)
    gpu = gpu_run(cfg, 0)
    assert rel_linf(gpu["dT"], cfg["dT"], 1.0) <= TOL32


@pytest.mark.parametrize("q", [8, 16, 64])
def test_ballistic_limit_bitwise(q):
    """MFP = inf (W = 0): pure advection, so GPU and oracle agree bit for bit."""
    nx, ny = 45, 38
    rng = np.random.default_rng(q)
    state = np.zeros((q, ny + 2, nx + 2))
    state[:, 1:-1, 1:-1] = rng.standard_normal((q, ny, nx)).astype(np.float32)
    cfg = dict(nx=nx, ny=ny, q=q, mfp=math.inf, bc=(P,) * 4, t_wall=(300.0,) * 4,
               emulate_3d=True, dT=np.zeros((ny, nx), np.float32))
    orc = oracle_run(dict(cfg, w_field=0.0), 47, state=state)
    gpu = gpu_run(cfg, 47, state=state)
    assert np.array_equal(gpu["state"][:, 1:-1, 1:-1], orc.d[:, 1:-1, 1:-1])


WALL_CASES = [
    ((I, I, A, A), (301.0, 300.0, 300.0, 300.0)),     # in-plane film
    ((A, A, A, A), (300.0,) * 4),                     # adiabatic box
    ((P, P, A, A), (300.0,) * 4),
    ((A, A, P, P), (300.0,) * 4),
    ((I, I, P, P), (300.6, 299.7, 300.0, 300.0)),     # cross-plane
    ((P, P, I, A), (300.0, 300.0, 300.8, 300.0)),
    ((I, A, I, A), (300.9, 300.0, 299.4, 300.0)),
]


@pytest.mark.parametrize("kinds,tw", WALL_CASES)
@pytest.mark.parametrize("nx,ny,q", [(61, 37, 16), (130, 9, 32)])
def test_walls_parity_ragged_grids(kinds, tw, nx, ny, q):
    cfg = dict(nx=nx, ny=ny, q=q, mfp=3.0, bc=kinds, t_wall=tw, emulate_3d=True,
               dT=W.random_dT(nx, ny, seed=nx * ny + q, scale=0.4))
    _compare(cfg, 120)


@pytest.mark.parametrize("kinds,tw", [WALL_CASES[1], WALL_CASES[2], WALL_CASES[4],
                                      WALL_CASES[6]])
def test_walls_parity_bf16(kinds, tw):
    """bfloat16 storage through every wall kind (values stored against the local
    reference energy in the wall pass as well as in the step)."""
    nx, ny, q = 77, 29, 16
    cfg = dict(nx=nx, ny=ny, q=q, mfp=3.0, bc=kinds, t_wall=tw, emulate_3d=True,
               dT=W.random_dT(nx, ny, seed=nx * ny + q, scale=0.4))
    _compare(cfg, 120, storage=1, tol=TOL16, state_tol=TOL16_STATE)


def test_mfp_field_parity():
    """Per-cell MFP (log-normal field) with isothermal x walls and periodic y."""
    n = 96
    mfp = W.lognormal_mfp(n, n + 7, seed=5, corr=8.0)
    cfg = dict(nx=n, ny=n + 7, q=16, mfp=None, mfp_field=mfp, bc=(I, I, P, P),
               t_wall=(300.5, 300.0, 300.0, 300.0), emulate_3d=True,
               dT=W.gaussian_field(n, n + 7, [(48.0, 50.0)], [10.0], [1.0]).astype(np.float32))
    _compare(cfg, 150)


def test_bf16_film_parity():
    cfg = W.film_c3(kn=0.5, nx=200, ny=24, q=32)
    _compare(cfg, 300, storage=1, tol=TOL16, state_tol=TOL16_STATE)


def test_exponential_relaxation_mode_parity():
    """MFP = 0.5 cell needs the opt-in exponential weight (the paper's is unstable)."""
    cfg = W.pulses_c2(seed=2, n=64, q=64, mfp=0.5, npulse=3, relax_mode=1)
    _compare(cfg, 80)


@pytest.mark.parametrize("nx,ny,kinds", [(1, 1, (P,) * 4), (1, 7, (P, P, A, A)),
                                         (5, 1, (I, I, P, P)), (2, 3, (A, A, A, A))])
def test_degenerate_grids(nx, ny, kinds):
    cfg = dict(nx=nx, ny=ny, q=8, mfp=2.0, bc=kinds, t_wall=(300.5, 300.0, 300.2, 300.0),
               emulate_3d=True, dT=W.random_dT(nx, ny, seed=11, scale=0.5))
    _compare(cfg, 40)


def test_energy_conservation_fp64_reductions():
    """Periodic grid: the FP64 total energy of the float32 state drifts by round-off
    only; an adiabatic box keeps interior + wall energy."""
    import paper_1911_00180_gb300 as wl
    for kinds in [(P,) * 4, (A,) * 4]:
        cfg = dict(nx=256, ny=200, q=32, mfp=4.0, bc=kinds, t_wall=(300.0,) * 4,
                   emulate_3d=True, dT=W.random_dT(256, 200, seed=9, scale=1.0))
        orc = oracle_run(cfg, 0)
        orc.apply_bc()
        e0 = orc.total_energy(include_frame=True)
        gpu = gpu_run(cfg, 300)
        scale = float(np.abs(orc.d).sum())
        assert abs(gpu["red"][1] - e0) <= 1e-6 * scale


def _window_oracle(cfg, cx, cy, steps, pad):
    """Oracle on a periodic window around (cx, cy): the update is local (one cell per
    step), so the centre after `steps` steps is exact when pad > steps."""
    nx, ny = cfg["nx"], cfg["ny"]
    xs = (np.arange(cx - pad, cx + pad + 1)) % nx
    ys = (np.arange(cy - pad, cy + pad + 1)) % ny
    sub = dict(cfg, nx=len(xs), ny=len(ys), dT=cfg["dT"][np.ix_(ys, xs)])
    return oracle_run(sub, steps)


BENCH_GRAPH, BENCH_PROFILE = 48, 8     # the benchmark's graph chunk and timing stride


def _sampled_full_size(cfg, steps, samples, window_fn, storage=0):
    """Run the full-size grid on the GPU in the benchmark's launch configuration (its own
    stream, 48-step CUDA-graph replays, event timing of every 8th step kernel), then
    check sampled cells one by one against the oracle on a window around each
    (temperature to TOL32 / TOL16 of the amplitude, state to TOL32 / TOL16_STATE of the
    largest per-direction pulse deviation)."""
    import torch
    import paper_1911_00180_gb300 as wl
    from oracle import lattice as L
    from tests._pair import THETA
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = wl.WormLBM(cfg["nx"], cfg["ny"], cfg["q"], mfp=cfg["mfp"], bc=cfg["bc"],
                       t_wall=cfg["t_wall"], storage=storage, emulate_3d=cfg["emulate_3d"],
                       relax_mode=cfg.get("relax_mode", 0), theta=THETA, stream=stream)
        h.wlbm_set_option(wl.wlbm.OPT_GRAPH_STEPS, BENCH_GRAPH)
        h.wlbm_profile(BENCH_PROFILE)
        h.wlbm_init_temperature(cfg["dT"])
        h.wlbm_step(steps)
        dT, _, _ = h.wlbm_moments(want_q=False)
        state = h.wlbm_get_state()
        stream.synchronize()
        assert h.wlbm_profile_read()[1] == steps // BENCH_PROFILE
        assert h.wlbm_get_option(wl.wlbm.OPT_GRAPH_REPLAYS) == steps // BENCH_GRAPH
    w = L.angular_weights(L.ring_directions(cfg["q"]))
    dscale = float(w.max() * (L.e_eq(301.0, 624.8074248458514) - L.e_eq(300.0, 624.8074248458514)))
    t_tol, s_tol = (TOL32, TOL32) if storage == 0 else (TOL16, TOL16_STATE_WALL)
    worst_t = worst_s = 0.0
    for (cx, cy) in samples:
        orc, (ox, oy) = window_fn(cfg, cx, cy, steps)
        e_t = abs(float(dT[cy, cx]) - orc.temperature_dev()[oy, ox])
        got = state[:, cy + 1, cx + 1].double().cpu().numpy()
        want = orc.d[:, oy + 1, ox + 1]
        e_s = float(np.abs(got - want).max()) / dscale
        worst_t, worst_s = max(worst_t, e_t), max(worst_s, e_s)
        assert e_t <= t_tol, ((cx, cy), e_t)
        assert e_s <= s_tol, ((cx, cy), e_s)
    print("full size %s: T %.3g  state %.3g" % ("bf16" if storage else "fp32", worst_t, worst_s))
    h.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_full_size_c2_sampled_cells(storage):
    """2048 x 2048, Q = 64, periodic, 16 pulses (the benchmark workload), one 48-step
    graph replay; float32 and bfloat16 storage (the 16-stage ring of Q <= 64)."""
    cfg = W.pulses_c2(seed=2)
    steps, pad = BENCH_GRAPH, BENCH_GRAPH + 2
    rng = np.random.default_rng(0)
    samples = [tuple(int(v) for v in rng.integers(0, 2048, size=2)) for _ in range(5)]
    # plus the hottest cell, where the pulse signal is largest
    cy, cx = np.unravel_index(np.argmax(cfg["dT"]), cfg["dT"].shape)
    samples.append((int(cx), int(cy)))

    def window(cfg, cx, cy, steps):
        return _window_oracle(cfg, cx, cy, steps, pad), (pad, pad)
    _sampled_full_size(cfg, steps, samples, window, storage)


@pytest.mark.parametrize("storage", [0, 1])
def test_full_size_c3_film_sampled_cells(storage):
    """4096 x 256 film, Q = 128, isothermal x walls, diffuse y walls: sampled cells
    (including ones next to the diffuse walls) against the oracle on an x-window that
    keeps the full film thickness and its walls; one 48-step graph replay; float32 and
    bfloat16 storage (the 8-stage ring of Q > 64)."""
    cfg = W.film_c3(kn=1.0)
    steps, pad = BENCH_GRAPH, BENCH_GRAPH + 2
    samples = [(1000, 0), (2500, 255), (3100, 128), (7, 40), (4090, 200)]

    def window(cfg, cx, cy, steps):
        # x-window with the film's own walls: where the window is cut inside the film
        # the (artificial) wall is more than `steps` cells from the sample, so it cannot
        # reach it; where the window meets a real wall, that wall is exact.
        x0, x1 = max(cx - pad, 0), min(cx + pad, cfg["nx"] - 1)
        sub = dict(cfg, nx=x1 - x0 + 1, dT=cfg["dT"][:, x0:x1 + 1])
        return oracle_run(sub, steps), (cx - x0, cy)
    _sampled_full_size(cfg, steps, samples, window, storage)
