"""The no-allocation reduction entry point (wlbm_reduce_state_noalloc), checked through
the C ABI against wlbm_reduce on the same state, on two calls in a row.

It serves callers that cannot allocate device memory where they call it (a host
application that owns the device memory through its own pool, or a latency-critical
monitoring hook), so its scratch is a fixed static device array.  This file is named to
be collected last, so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5          # the float32 parity tolerance of the other GPU tests


def test_noalloc_reduction_matches_handle_reduction_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300 as wl
    nx, ny, q = 203, 77, 32
    kinds = (W.ISOTHERMAL, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE, W.ADIABATIC_DIFFUSE)
    h = wl.WormLBM(nx, ny, q, mfp=4.0, bc=kinds, t_wall=(301.0, 300.0, 300.0, 300.0))
    h.wlbm_init_temperature(W.random_dT(nx, ny, seed=5, scale=0.5))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for call in range(2):
        h.wlbm_step(25)
        want = np.array(h.wlbm_reduce())[:4]
        framed = h.wlbm_get_state()
        out.fill_(float("nan"))
        wl.wlbm_reduce_state_noalloc(framed, nx, ny, q, kinds, out, stream=h.stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = float(framed.abs().sum())
        assert np.all(np.isfinite(got)), call
        assert abs(got[0] - want[0]) <= TOL * scale, (call, got, want)
        assert abs(got[1] - want[1]) <= TOL * scale, (call, got, want)
        assert np.all(np.abs(got[2:] - want[2:]) <= TOL * scale / (nx * ny)), (call, got, want)
        assert got[1] != got[0]        # the diffuse walls hold energy of their own
    h.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_00180_gb300 as wl
    dummy = torch.zeros(1, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(wl.WlbmError) as err:
        wl.wlbm_reduce_state_noalloc(dummy, 4000, 4000, 8, (0, 0, 0, 0), out)
    assert "scratch" in str(err.value)
