"""The no-allocation reduction entry point (wlbm_reduce_state_noalloc), checked through
the C ABI against wlbm_reduce on the same state, on two calls in a row.

It serves callers that cannot allocate device memory where they call it (a host
application that owns the device memory through its own pool, or a latency-critical
monitoring hook), so its scratch is a fixed static device array.  This file is named to
be collected last, so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5          # the float32 parity tolerance of the other GPU tests


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("speed", [1.0, 0.6])
def test_noalloc_reduction_matches_handle_reduction_twice(speed):
    """Two calls in a row on a film with diffuse walls; at v = 0.6 (one slower band of a
    multigray run) the mean fluxes carry the band speed as wlbm_reduce's do."""
    torch = _cuda()
    import paper_1911_00180_gb300 as wl
    nx, ny, q = 203, 77, 32
    kinds = (W.ISOTHERMAL, W.ISOTHERMAL, W.ADIABATIC_DIFFUSE, W.ADIABATIC_DIFFUSE)
    h = wl.WormLBM(nx, ny, q, mfp=4.0, bc=kinds, t_wall=(301.0, 300.0, 300.0, 300.0),
                   speed=speed)
    h.wlbm_init_temperature(W.random_dT(nx, ny, seed=5, scale=0.5))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for call in range(2):
        h.wlbm_step(25)
        want = np.array(h.wlbm_reduce())[:4]
        framed = h.wlbm_get_state()
        out.fill_(float("nan"))
        wl.wlbm_reduce_state_noalloc(framed, nx, ny, q, kinds, out, stream=h.stream,
                                     speed=speed)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = float(framed.abs().sum())
        assert np.all(np.isfinite(got)), call
        assert abs(got[0] - want[0]) <= TOL * scale, (call, got, want)
        assert abs(got[1] - want[1]) <= TOL * scale, (call, got, want)
        assert np.all(np.abs(got[2:] - want[2:]) <= TOL * scale / (nx * ny)), (call, got, want)
        assert got[1] != got[0]        # the diffuse walls hold energy of their own
        assert abs(got[2]) > 100 * TOL * scale / (nx * ny)    # a flux that tells v apart
    h.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    """The C entry point refuses a frame larger than its fixed scratch before it touches
    any memory (so the pointer is never read)."""
    torch = _cuda()
    import paper_1911_00180_gb300 as wl
    dummy = torch.zeros(1, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    kinds = (C.c_int32 * 4)(0, 0, 0, 0)
    st = wl.lib.wlbm_reduce_state_noalloc(C.c_void_p(dummy.data_ptr()), 4000, 4000, 8, 1.0,
                                          kinds, C.c_void_p(out.data_ptr()), None)
    assert st == wl.wlbm.WLBM_ERR_INVALID_ARG
    assert b"scratch" in wl.lib.wlbm_last_error(None)


def test_noalloc_wrapper_refuses_mismatched_tensors():
    """The binding checks dtype, device, layout and size before it launches anything."""
    torch = _cuda()
    import paper_1911_00180_gb300 as wl
    nx, ny, q = 10, 6, 8
    n = q * (ny + 2) * (nx + 2)
    ok = torch.zeros(n, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    bad = [(torch.zeros(n - 1, device="cuda"), out),                      # too small
           (torch.zeros(n, dtype=torch.float64, device="cuda"), out),     # wrong dtype
           (torch.zeros(2 * n, device="cuda")[::2], out),                 # not contiguous
           (torch.zeros(n), out),                                          # host memory
           (ok, torch.zeros(3, dtype=torch.float64, device="cuda")),       # out too small
           (ok, torch.zeros(4, device="cuda"))]                            # out not float64
    for framed, o in bad:
        with pytest.raises(ValueError):
            wl.wlbm_reduce_state_noalloc(framed, nx, ny, q, (0, 0, 0, 0), o)
    wl.wlbm_reduce_state_noalloc(ok, nx, ny, q, (0, 0, 0, 0), out)     # current stream
    torch.cuda.synchronize()
    assert out.abs().max().item() == 0.0
