"""Step-kernel timing through the C ABI (wlbm_profile / wlbm_profile_read and the batch
forms): an event pair around every S-th step-kernel launch, counted across calls; a
negative stride is refused; profiling changes no result, also where it turns graph replay
off."""
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


def test_profiling_changes_no_result():
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=0.5, nx=96, ny=24, q=24)
    a = gpu_handle(cfg, 1)
    b = gpu_handle(cfg, 1)
    b.wlbm_set_option(wl.wlbm.OPT_GRAPH_STEPS, 12)
    b.wlbm_profile(5)                    # graph replay is off while profiling
    for h in (a, b):
        h.wlbm_init_temperature(cfg["dT"])
        h.wlbm_step(31)
    b.wlbm_profile(0)                    # and back on for the rest
    for h in (a, b):
        h.wlbm_step(24)
    assert np.array_equal(_state(a), _state(b))
    assert b.wlbm_profile_read()[1] == 7  # launches 0, 5, ..., 30
    a.close()
    b.close()


def test_batch_stride():
    import paper_1911_00180_gb300 as wl
    cfg = W.film_c3(kn=1.0, nx=40, ny=12, q=16)
    spec = dict(nx=40, ny=12, q=16, bc=cfg["bc"], t_wall=cfg["t_wall"], mfp=12.0,
                emulate_3d=True)
    b = wl.WormLBMBatch([spec, dict(spec, q=24)])
    b.wlbm_batch_init_temperature([cfg["dT"], cfg["dT"]])
    b.wlbm_batch_profile(2)
    b.wlbm_batch_step(5)                 # launches 0, 2, 4
    ms, n, _ = b.wlbm_batch_profile_read()
    assert n == 3 and ms > 0.0
    with pytest.raises(wl.WlbmError):
        b.wlbm_batch_profile(-1)
    b.close()
