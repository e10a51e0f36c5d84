"""Checkpoint and resume through the C ABI (wlbm_save / wlbm_load): stepping a handle
loaded from a checkpoint gives bit-for-bit the states of the uninterrupted run, in a new
handle and in the same one, for both storage types, every step variant's default and
CUDA-graph replay; mismatched or damaged checkpoints are refused with an error."""
import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_handle

pytestmark = pytest.mark.gpu
P, I, A = W.PERIODIC, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401  (fails loudly if the library is missing)


def _snapshot(h):
    import torch
    dT, qx, _ = h.wlbm_moments()
    st = h.wlbm_get_state()
    torch.cuda.synchronize()
    return (st[:, 1:-1, 1:-1].cpu().numpy().copy(), dT.cpu().numpy().copy(),
            qx.cpu().numpy().copy(), h.wlbm_step_count())


def _same(a, b):
    assert a[3] == b[3]
    for x, y in zip(a[:3], b[:3]):
        assert x.shape == y.shape
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def _cases():
    film = W.film_c3(kn=0.7, nx=150, ny=37, q=32)
    pulses = W.pulses_c2(seed=2, n=96, q=16, mfp=6.0, npulse=3)
    box = dict(nx=61, ny=45, q=24, mfp=3.0, bc=(A, A, A, A), t_wall=(300.0,) * 4,
               emulate_3d=True, dT=W.random_dT(61, 45, seed=7, scale=0.5))
    return [("film", film), ("pulses", pulses), ("box", box)]


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("name,cfg", _cases())
def test_resume_is_bitwise(name, cfg, storage):
    n1, n2 = 37, 50                       # odd split: mid energy-plane rotation
    h = gpu_handle(cfg, storage)
    h.wlbm_init_temperature(cfg["dT"])
    h.wlbm_step(n1)
    blob = h.wlbm_save()
    h.wlbm_step(n2)
    want = _snapshot(h)
    # a fresh handle created with the same arguments
    g = gpu_handle(cfg, storage)
    g.wlbm_load(blob)
    assert g.wlbm_step_count() == n1
    g.wlbm_step(n2)
    _same(_snapshot(g), want)
    g.close()
    # the same handle, rewound
    h.wlbm_load(blob)
    h.wlbm_step(n2)
    _same(_snapshot(h), want)
    h.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_load_keeps_pads_zero(storage):
    """A checkpoint whose pad bytes (the columns left of the ghost column and right of the
    right ghost column, the rows outside the frame) hold garbage loads and steps bit for
    bit like the clean one: wlbm_load copies only the frame.  Diffuse x walls put computed
    ghost columns next to the pads: the first box of a row reads pad columns from memory,
    and with an even width the bfloat16 256-column tiles read the first pad right of the
    right ghost column from memory too."""
    nx, ny, q = 150, 37, 32
    cfg = dict(nx=nx, ny=ny, q=q, mfp=4.0, bc=(A, A, I, A), t_wall=(300.0, 300.0, 300.6, 300.0),
               emulate_3d=True, dT=W.random_dT(nx, ny, seed=5, scale=0.5))
    h = gpu_handle(cfg, storage)
    h.wlbm_init_temperature(cfg["dT"])
    h.wlbm_step(13)
    blob = h.wlbm_save().copy()
    h.wlbm_step(20)
    want = _snapshot(h)
    h.close()
    # blob layout: 104-byte header (pitch at byte 28, plane and energy bytes at 72 and 80),
    # the schedule cursor, then q planes and the energy planes, each (ny + 4) x pitch
    pitch = int(blob[28:32].view(np.int32)[0])
    plane_bytes, energy_bytes = (int(v) for v in blob[72:88].view(np.int64))
    elem = plane_bytes // ((ny + 4) * pitch)
    off = 104 + q * 24 + ((q + 7) // 8) * 8
    frame = np.zeros((ny + 4, pitch), bool)
    frame[1:ny + 3, 31:31 + nx + 2] = True
    rng = np.random.default_rng(3)
    bad = blob.copy()
    for size, e in [(plane_bytes, elem)] * q + [(energy_bytes, 4)] * (2 if storage else 1):
        region = bad[off:off + size].reshape(ny + 4, pitch, e)
        region[~frame] = rng.integers(1, 255, size=(int((~frame).sum()), e), dtype=np.uint8)
        off += size
    assert off == bad.size
    g = gpu_handle(cfg, storage)
    g.wlbm_load(bad)
    g.wlbm_step(20)
    _same(_snapshot(g), want)
    g.close()


def test_resume_under_graph_replay():
    """Graph replay needs a stream of its own (not the legacy default stream): both
    handles run on one, so their 12-step chunks are captured graphs."""
    import torch
    import paper_1911_00180_gb300 as wl
    from tests._pair import THETA
    cfg = W.film_c3(kn=2.0, nx=64, ny=20, q=16)

    def make(stream):
        x = wl.WormLBM(cfg["nx"], cfg["ny"], cfg["q"], mfp=cfg["mfp"], bc=cfg["bc"],
                       t_wall=cfg["t_wall"], storage=1, emulate_3d=cfg["emulate_3d"],
                       theta=THETA, stream=stream)
        x.wlbm_set_option(wl.wlbm.OPT_GRAPH_STEPS, 12)
        return x
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h = make(stream)
        h.wlbm_init_temperature(cfg["dT"])
        h.wlbm_step(29)
        blob = h.wlbm_save()
        h.wlbm_step(40)
        want = _snapshot(h)
        g = make(stream)
        g.wlbm_load(blob)
        g.wlbm_step(40)
        _same(_snapshot(g), want)
        # 29 + 40 steps = 2 + 3 whole chunks of h, 3 of g, each a graph replay
        assert h.wlbm_get_option(wl.wlbm.OPT_GRAPH_REPLAYS) == 5
        assert g.wlbm_get_option(wl.wlbm.OPT_GRAPH_REPLAYS) == 3
        g.close()
        h.close()


def test_load_refuses_mismatches():
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=1.0, nx=40, ny=12, q=16)
    h = gpu_handle(cfg)
    h.wlbm_init_temperature(cfg["dT"])
    h.wlbm_step(5)
    blob = h.wlbm_save()
    bad = [blob[:100], blob[:-8]]
    damaged = blob.copy()
    damaged[:8] = 0
    bad.append(damaged)
    for b in bad:
        with pytest.raises(wl.WlbmError) as e:
            h.wlbm_load(b)
        assert e.value.status == wl.wlbm.WLBM_ERR_INVALID_ARG
    for other in (dict(cfg, nx=41, dT=np.zeros((12, 41), np.float32)), dict(cfg, q=24)):
        g = gpu_handle(other)
        with pytest.raises(wl.WlbmError):
            g.wlbm_load(blob)
        g.close()
    g = gpu_handle(cfg, 1)                 # other storage type
    with pytest.raises(wl.WlbmError):
        g.wlbm_load(blob)
    g.close()
    h.wlbm_load(blob)                      # the good one still loads
    assert h.wlbm_step_count() == 5
    h.close()

    spec = dict(nx=40, ny=12, q=16, bc=cfg["bc"], t_wall=cfg["t_wall"], mfp=12.0,
                emulate_3d=True)
    b = wl.WormLBMBatch([spec, spec])
    b.wlbm_batch_init_temperature([cfg["dT"], cfg["dT"]])
    inst = b.instances[0]
    blob2 = inst.wlbm_save()               # saving an instance is fine
    with pytest.raises(wl.WlbmError) as e:
        inst.wlbm_load(blob2)
    assert e.value.status == wl.wlbm.WLBM_ERR_STATE
    b.close()
