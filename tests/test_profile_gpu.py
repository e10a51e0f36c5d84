"""Step-kernel timing through the C ABI (wlbm_profile / wlbm_profile_read and the batch
forms): an event pair around every S-th step-kernel launch, counted across calls, or,
under graph replay, the steps of each chunk that the stride selects, recorded by the
graph's event nodes; a negative stride is refused; profiling changes no result."""
import numpy as np
import pytest

import workloads as W
from tests._pair import gpu_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300  # noqa: F401


def _state(h):
    import torch
    st = h.wlbm_get_state()
    torch.cuda.synchronize()
    return st.cpu().numpy().view(np.uint32).copy()


def test_stride_counts_launches_across_calls():
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=1.0, nx=64, ny=16, q=16)
    h = gpu_handle(cfg)
    h.wlbm_init_temperature(cfg["dT"])
    h.wlbm_profile(3)
    h.wlbm_step(4)                      # launches 0..3: 0 and 3 timed
    h.wlbm_step(6)                      # launches 4..9: 6 and 9 timed
    ms, n, all1 = h.wlbm_profile_read()
    assert n == 4 and ms > 0.0
    ms, n, all2 = h.wlbm_profile_read()  # reset by the read
    assert n == 0 and ms == 0.0 and all2 == all1
    h.wlbm_profile(1)
    h.wlbm_step(5)
    assert h.wlbm_profile_read()[1] == 5
    h.wlbm_profile(0)
    h.wlbm_step(5)
    _, n, all3 = h.wlbm_profile_read()
    assert n == 0 and all3 > all1
    with pytest.raises(wl.WlbmError) as e:
        h.wlbm_profile(-2)
    assert e.value.status == wl.wlbm.WLBM_ERR_INVALID_ARG
    h.close()


def _streamed(cfg, storage, stream):
    import paper_1911_00180_gb300 as wl
    from tests._pair import THETA
    return wl.WormLBM(cfg["nx"], cfg["ny"], cfg["q"], mfp=cfg["mfp"], bc=cfg["bc"],
                      t_wall=cfg["t_wall"], storage=storage, emulate_3d=cfg["emulate_3d"],
                      theta=THETA, stream=stream)


def test_graph_replay_is_timed_and_changes_no_result():
    """Graph replay of 12-step chunks with stride 4: every replay times its steps 0, 4 and 8
    through event nodes of the graph, the direct steps after the last whole chunk count on
    from the stride's start; the states equal those of an untimed run launched step by
    step, bit for bit."""
    import torch
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=0.5, nx=96, ny=24, q=24)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = _streamed(cfg, 1, s)
        b = _streamed(cfg, 1, s)
        b.wlbm_set_option(wl.wlbm.OPT_GRAPH_STEPS, 12)
        b.wlbm_profile(4)
        for h in (a, b):
            h.wlbm_init_temperature(cfg["dT"])
            h.wlbm_step(24)
        ms, n, _ = b.wlbm_profile_read()
        assert n == 6 and ms > 0.0            # two replays x steps 0, 4, 8
        for h in (a, b):
            h.wlbm_step(3 * 12 + 5)
        assert b.wlbm_profile_read()[1] == 3 * 3 + 2   # + direct steps 0 and 4 of 5
        b.wlbm_profile(0)                     # drops the timed graphs; untimed replay on
        for h in (a, b):
            h.wlbm_step(24)
        assert b.wlbm_profile_read()[1] == 0
        assert b.wlbm_get_option(wl.wlbm.OPT_GRAPH_REPLAYS) == 2 + 3 + 2
        assert a.wlbm_get_option(wl.wlbm.OPT_GRAPH_REPLAYS) == 0
        assert np.array_equal(_state(a), _state(b))
        a.close()
        b.close()


@pytest.mark.parametrize("graph", [0, 6])
def test_batch_stride(graph):
    import torch
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=1.0, nx=40, ny=12, q=16)
    spec = dict(nx=40, ny=12, q=16, bc=cfg["bc"], t_wall=cfg["t_wall"], mfp=12.0,
                emulate_3d=True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = wl.WormLBMBatch([spec, dict(spec, q=24)], stream=s)
        b.wlbm_batch_set_option(wl.wlbm.OPT_GRAPH_STEPS, graph)
        b.wlbm_batch_init_temperature([cfg["dT"], cfg["dT"]])
        b.wlbm_batch_profile(2)
        b.wlbm_batch_step(6)             # launches 0, 2, 4 (directly or in one replay)
        ms, n, _ = b.wlbm_batch_profile_read()
        assert n == 3 and ms > 0.0
        b.wlbm_batch_step(18)            # three more chunks of 6
        assert b.wlbm_batch_profile_read()[1] == 9
        with pytest.raises(wl.WlbmError):
            b.wlbm_batch_profile(-1)
        b.close()
