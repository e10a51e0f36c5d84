"""Thin ctypes binding of libwlbm (include/wlbm.h).

Functions carry the C names and only marshal arguments: every step of the worm-LBM runs
inside the library's CUDA kernels.  PyTorch supplies device memory (through the
library's allocator callback) and the CUDA stream; tensors passed in or out are plain
device buffers.  If the shared library is missing the import fails: there is no CPU or
eager fallback.
"""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libwlbm.so")

WLBM_OK, WLBM_ERR_INVALID_ARG, WLBM_ERR_UNSTABLE, WLBM_ERR_OOM = 0, 1, 2, 3
WLBM_ERR_CUDA, WLBM_ERR_TIMEOUT, WLBM_ERR_STATE = 4, 5, 6
BC_PERIODIC, BC_ISOTHERMAL, BC_ADIABATIC_DIFFUSE, BC_ADIABATIC_SPECULAR = 0, 1, 2, 3
STORE_FP32_DEV, STORE_BF16_DEV = 0, 1
OPT_STEP_VARIANT, OPT_GRAPH_STEPS, OPT_FUSE_PERIODIC, OPT_GRAPH_REPLAYS = 1, 2, 3, 4
OPT_PERSISTENT, OPT_RING_STAGES, OPT_WAIT_LIMIT, OPT_STALL_TEST = 5, 6, 7, 8
OPT_TILE_LOOP = 9
OPT_BF16_WIDE = 10
REDUCE_N = 9          # WLBM_REDUCE_N
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSTABLE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT",
                6: "STATE"}


class wlbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("q", C.c_int32),
                ("storage", C.c_int32), ("emulate_3d", C.c_int32),
                ("relax_mode", C.c_int32), ("t_ref", C.c_double), ("theta", C.c_double),
                ("speed", C.c_double)]


class wlbm_boundary(C.Structure):
    _fields_ = [("kind", C.c_int32 * 4), ("t_wall", C.c_double * 4),
                ("specularity", C.c_double * 4)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class wlbm_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class WlbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libwlbm.so is not built (%s); run "
                          "`python -m paper_1911_00180_gb300.build`" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "wlbm_create": (C.c_int, [C.POINTER(wlbm_grid), vp, dbl, C.POINTER(wlbm_boundary),
                                  C.POINTER(wlbm_allocator), vp, C.POINTER(vp)]),
        "wlbm_destroy": (None, [vp]),
        "wlbm_last_error": (C.c_char_p, [vp]),
        "wlbm_set_stream": (C.c_int, [vp, vp]),
        "wlbm_init_temperature": (C.c_int, [vp, vp]),
        "wlbm_step": (C.c_int, [vp, i64]),
        "wlbm_step_count": (i64, [vp]),
        "wlbm_moments": (C.c_int, [vp, vp, vp, vp]),
        "wlbm_reduce": (C.c_int, [vp, C.POINTER(dbl)]),
        "wlbm_moments_mean": (C.c_int, [vp, i32, vp, vp, vp]),
        "wlbm_run_steady": (C.c_int, [vp, i64, i64, dbl, i32, C.POINTER(C.c_int64),
                                      C.POINTER(i32), C.POINTER(dbl)]),
        "wlbm_get_state": (C.c_int, [vp, vp]),
        "wlbm_save": (C.c_int, [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)]),
        "wlbm_set_sources": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl)]),
        "wlbm_load": (C.c_int, [vp, vp, C.c_size_t]),
        "wlbm_set_state": (C.c_int, [vp, vp]),
        "wlbm_adjoint_forward": (C.c_int, [vp, vp, i64, i32]),
        "wlbm_adjoint_backward": (C.c_int, [vp, vp, vp, vp, vp, C.POINTER(dbl), vp]),
        "wlbm_set_option": (C.c_int, [vp, i32, i64]),
        "wlbm_get_option": (C.c_int, [vp, i32, C.POINTER(C.c_int64)]),
        "wlbm_autotune": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]),
        "wlbm_batch_create": (C.c_int, [i32, C.POINTER(wlbm_grid), C.POINTER(vp), C.POINTER(dbl),
                                        C.POINTER(wlbm_boundary), C.POINTER(wlbm_allocator), vp,
                                        C.POINTER(vp)]),
        "wlbm_batch_destroy": (None, [vp]),
        "wlbm_batch_last_error": (C.c_char_p, [vp]),
        "wlbm_batch_size": (i32, [vp]),
        "wlbm_batch_instance": (vp, [vp, i32]),
        "wlbm_batch_init_temperature": (C.c_int, [vp, C.POINTER(vp)]),
        "wlbm_batch_set_option": (C.c_int, [vp, i32, i64]),
        "wlbm_batch_get_option": (C.c_int, [vp, i32, C.POINTER(C.c_int64)]),
        "wlbm_batch_check": (C.c_int, [vp]),
        "wlbm_batch_step": (C.c_int, [vp, i64]),
        "wlbm_batch_profile": (C.c_int, [vp, i32]),
        "wlbm_batch_profile_read": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(i64),
                                              C.POINTER(i64)]),
        "wlbm_batch_autotune": (C.c_int, [vp, i32, C.POINTER(i32), C.POINTER(i32),
                                          C.POINTER(dbl)]),
        "wlbm_check": (C.c_int, [vp]),
        "wlbm_profile": (C.c_int, [vp, i32]),
        "wlbm_profile_read": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(i64), C.POINTER(i64)]),
        "wlbm_reduce_state_noalloc": (C.c_int, [vp, i32, i32, i32, C.c_double, C.POINTER(i32),
                                                vp, vp]),
        "wlbm_lattice": (C.c_int, [i32, C.POINTER(i32), C.POINTER(dbl), C.POINTER(C.c_int8),
                                   C.POINTER(dbl)]),
        "wlbm_schedule": (C.c_int, [i32, i64, dbl, C.POINTER(C.c_uint8)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status, handle=None):
    if status != WLBM_OK:
        msg = lib.wlbm_last_error(handle)
        raise WlbmError(status, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- host-only queries
def wlbm_lattice(q):
    """Ring directions (Q, 2) int32, weights (Q,) float64, worm table (Q, M) int8,
    Lambda_corr (Sec. 2.4-2.5), computed by the library's host code."""
    import numpy as np
    dirs = np.zeros(2 * q, np.int32)
    w = np.zeros(q, np.float64)
    worm = np.zeros(q * (q // 8), np.int8)
    lam = C.c_double()
    _check(lib.wlbm_lattice(q, dirs.ctypes.data_as(C.POINTER(C.c_int32)),
                            w.ctypes.data_as(C.POINTER(C.c_double)),
                            worm.ctypes.data_as(C.POINTER(C.c_int8)), C.byref(lam)))
    return dirs.reshape(q, 2), w, worm.reshape(q, q // 8), lam.value


def wlbm_schedule(q, n_steps, speed=1.0):
    """TAS codes (n_steps, Q) uint8: hop index | paused << 3 (Eq. algorithm) at the given
    propagation speed."""
    import numpy as np
    out = np.zeros(max(n_steps, 1) * q, np.uint8)
    _check(lib.wlbm_schedule(q, n_steps, float(speed),
                             out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out[:n_steps * q].reshape(n_steps, q)


def wlbm_reduce_state_noalloc(framed, nx, ny, q, bc_kind, out, stream=None, speed=1.0):
    """No-allocation reduction of a framed float32 state (contiguous CUDA tensor of at least
    q * (ny + 2) * (nx + 2) elements) into a contiguous CUDA float64 tensor `out` of at
    least 4 entries on the same device (see include/wlbm.h); `speed` is the band's v_g.
    Runs on `stream`, by default torch's current stream.  Tensors of another dtype,
    device, layout or size raise ValueError before anything is launched."""
    nx, ny, q = int(nx), int(ny), int(q)
    need = q * (ny + 2) * (nx + 2)
    for name, t, dt, n in (("framed", framed, "float32", need), ("out", out, "float64", 4)):
        if not getattr(t, "is_cuda", False):
            raise ValueError("wlbm_reduce_state_noalloc: %s must be a CUDA tensor" % name)
        if str(t.dtype) != "torch." + dt:
            raise ValueError("wlbm_reduce_state_noalloc: %s must be %s" % (name, dt))
        if not t.is_contiguous():
            raise ValueError("wlbm_reduce_state_noalloc: %s must be contiguous" % name)
        if t.numel() < n:
            raise ValueError("wlbm_reduce_state_noalloc: %s holds %d elements, needs %d"
                             % (name, t.numel(), n))
    if framed.device != out.device:
        raise ValueError("wlbm_reduce_state_noalloc: framed and out on different devices")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(framed.device)
    kinds = (C.c_int32 * 4)(*bc_kind)
    _check(lib.wlbm_reduce_state_noalloc(_ptr(framed), nx, ny, q, float(speed), kinds,
                                         _ptr(out), C.c_void_p(stream.cuda_stream)))


# ------------------------------------------------------------------ device handle
class WormLBM:
    """One worm-LBM grid on the current CUDA device (wraps a wlbm_handle*)."""

    def __init__(self, nx, ny, q, mfp=None, mfp_field=None, bc=(0, 0, 0, 0),
                 t_wall=(300.0,) * 4, storage=STORE_FP32_DEV, emulate_3d=True,
                 relax_mode=0, t_ref=300.0, theta=624.8074248458514, stream=None,
                 allocator=None, specularity=(0.0,) * 4, speed=1.0):
        import torch
        self._torch = torch
        self.nx, self.ny, self.q = nx, ny, q
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = wlbm_grid(nx, ny, q, storage, 1 if emulate_3d else 0, relax_mode, t_ref, theta,
                      float(speed))
        b = wlbm_boundary((C.c_int32 * 4)(*bc), (C.c_double * 4)(*t_wall),
                          (C.c_double * 4)(*specularity))
        if allocator is None:
            dev, strm = self.device.index, self.stream.cuda_stream

            def _alloc(n, ctx):
                return torch.cuda.caching_allocator_alloc(int(n), dev, strm)

            def _free(p, ctx):
                torch.cuda.caching_allocator_delete(p)
            allocator = (_alloc, _free)
        self._alloc_fns = (ALLOC_FN(allocator[0]), FREE_FN(allocator[1]))
        self._alloc = wlbm_allocator(self._alloc_fns[0], self._alloc_fns[1], None)
        mfp_t = None
        if mfp_field is not None:
            mfp_t = torch.as_tensor(mfp_field, dtype=torch.float32, device=self.device).contiguous()
        handle = C.c_void_p()
        st = lib.wlbm_create(C.byref(g), _ptr(mfp_t), float(mfp if mfp is not None else 0.0),
                             C.byref(b), C.byref(self._alloc),
                             C.c_void_p(self.stream.cuda_stream), C.byref(handle))
        _check(st, None)
        self.h = handle

    def close(self):
        if getattr(self, "h", None):
            lib.wlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # entry points ---------------------------------------------------------------
    def wlbm_init_temperature(self, dT):
        t = self._torch.as_tensor(dT, dtype=self._torch.float32, device=self.device).contiguous()
        _check(lib.wlbm_init_temperature(self.h, _ptr(t)), self.h)
        self._keep = t            # keep alive until the stream has consumed it

    def wlbm_step(self, n=1):
        _check(lib.wlbm_step(self.h, int(n)), self.h)

    def wlbm_step_count(self):
        return lib.wlbm_step_count(self.h)

    def wlbm_moments(self, want_t=True, want_q=True, out=None):
        torch = self._torch
        if out is None:
            mk = lambda f: torch.empty((self.ny, self.nx), dtype=torch.float32,
                                       device=self.device) if f else None
            out = (mk(want_t), mk(want_q), mk(want_q))
        dT, qx, qy = out
        _check(lib.wlbm_moments(self.h, _ptr(dT), _ptr(qx), _ptr(qy)), self.h)
        return dT, qx, qy

    def wlbm_moments_mean(self, n, want_t=True, want_q=True):
        """Advance n steps; means of (dT, q_x, q_y) over the n states reached."""
        torch = self._torch
        mk = lambda f: torch.empty((self.ny, self.nx), dtype=torch.float32,
                                   device=self.device) if f else None
        dT, qx, qy = mk(want_t), mk(want_q), mk(want_q)
        _check(lib.wlbm_moments_mean(self.h, int(n), _ptr(dT), _ptr(qx), _ptr(qy)), self.h)
        return dT, qx, qy

    def wlbm_reduce(self):
        """The WLBM_REDUCE_N float64 reductions of include/wlbm.h, as a list."""
        out = (C.c_double * REDUCE_N)()
        _check(lib.wlbm_reduce(self.h, out), self.h)
        return list(out)

    def wlbm_run_steady(self, max_steps, check_every, tol, avg_steps=10):
        """Steps until the temperature residual is <= tol K/step or max_steps ran, then
        averages the flux outputs over avg_steps steps: returns (steps_run, converged,
        reductions)."""
        out = (C.c_double * REDUCE_N)()
        steps, conv = C.c_int64(0), C.c_int32(0)
        _check(lib.wlbm_run_steady(self.h, int(max_steps), int(check_every), float(tol),
                                   int(avg_steps), C.byref(steps), C.byref(conv), out), self.h)
        return steps.value, bool(conv.value), list(out)

    def wlbm_set_sources(self, cells, temps=None, imposed=None):
        """Cells [(x, y), ...] kept at temperatures `temps` (K) or at the imposed absolute
        DDEDs `imposed` (n x Q); an empty list removes the sources."""
        import numpy as np
        n = len(cells)
        xy = np.ascontiguousarray(np.asarray(cells, np.int32).reshape(-1))
        t = None if temps is None else np.ascontiguousarray(np.asarray(temps, np.float64))
        e = None if imposed is None else np.ascontiguousarray(
            np.asarray(imposed, np.float64).reshape(n, self.q))
        ptr = lambda a, ty: None if a is None else a.ctypes.data_as(C.POINTER(ty))
        _check(lib.wlbm_set_sources(self.h, n, ptr(xy, C.c_int32) if n else None,
                                    ptr(t, C.c_double), ptr(e, C.c_double)), self.h)

    def wlbm_save(self):
        """Checkpoint of the current state and schedule cursor as a numpy uint8 array."""
        import numpy as np
        size = C.c_size_t(0)
        _check(lib.wlbm_save(self.h, None, 0, C.byref(size)), self.h)
        buf = np.empty(size.value, np.uint8)
        _check(lib.wlbm_save(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, C.byref(size)),
               self.h)
        return buf

    def wlbm_load(self, blob):
        import numpy as np
        buf = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib.wlbm_load(self.h, buf.ctypes.data_as(C.c_void_p), buf.nbytes), self.h)

    def wlbm_adjoint_forward(self, dT0, n_steps, ckpt_every):
        t = self._torch.as_tensor(dT0, dtype=self._torch.float32, device=self.device).contiguous()
        _check(lib.wlbm_adjoint_forward(self.h, _ptr(t), int(n_steps), int(ckpt_every)), self.h)

    def wlbm_adjoint_backward(self, dJ_dT=None, want_mfp=True, want_dT0=True, dJ_dqx=None,
                              dJ_dqy=None):
        """(dJ/dMFP (ny, nx), dJ/dT_wall [4], dJ/d dT0 (ny, nx)) for the checkpointed run,
        J given by its derivatives with respect to the final T, q_x and q_y (None: 0)."""
        torch = self._torch
        dev = lambda a: None if a is None else torch.as_tensor(
            a, dtype=torch.float32, device=self.device).contiguous()
        seeds = [dev(a) for a in (dJ_dT, dJ_dqx, dJ_dqy)]
        mk = lambda f: torch.empty((self.ny, self.nx), dtype=torch.float32,
                                   device=self.device) if f else None
        g_mfp, g_dT0 = mk(want_mfp), mk(want_dT0)
        g_tw = (C.c_double * 4)()
        _check(lib.wlbm_adjoint_backward(self.h, *[_ptr(a) for a in seeds], _ptr(g_mfp), g_tw,
                                         _ptr(g_dT0)), self.h)
        return g_mfp, list(g_tw), g_dT0

    def wlbm_set_option(self, key, value):
        _check(lib.wlbm_set_option(self.h, int(key), int(value)), self.h)

    def wlbm_get_option(self, key):
        v = C.c_int64()
        _check(lib.wlbm_get_option(self.h, int(key), C.byref(v)), self.h)
        return v.value

    def wlbm_autotune(self, trial_steps=48):
        """Native search over step-kernel variant x CUDA-graph replay (advances the state:
        call before wlbm_init_temperature).  Returns (variant, graph_steps, ms/step)."""
        v, g, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib.wlbm_autotune(self.h, int(trial_steps), C.byref(v), C.byref(g), C.byref(ms)),
               self.h)
        return v.value, g.value, ms.value

    def wlbm_check(self):
        _check(lib.wlbm_check(self.h), self.h)

    def wlbm_profile(self, every=1):
        """Time every `every`-th step-kernel launch (True: every launch; False or 0: off)."""
        _check(lib.wlbm_profile(self.h, int(every)), self.h)

    def wlbm_profile_read(self):
        """(summed step-kernel ms, timed step launches, all kernel launches so far)."""
        ms, n, alln = C.c_double(), C.c_int64(), C.c_int64()
        _check(lib.wlbm_profile_read(self.h, C.byref(ms), C.byref(n), C.byref(alln)), self.h)
        return ms.value, n.value, alln.value

    def wlbm_get_state(self):
        t = self._torch.empty((self.q, self.ny + 2, self.nx + 2), dtype=self._torch.float32,
                              device=self.device)
        _check(lib.wlbm_get_state(self.h, _ptr(t)), self.h)
        return t

    def wlbm_set_state(self, framed):
        t = self._torch.as_tensor(framed, dtype=self._torch.float32, device=self.device).contiguous()
        _check(lib.wlbm_set_state(self.h, _ptr(t)), self.h)
        self._keep = t


# ---------------------------------------------------------------------------------- batch
def _batch_check(status, b):
    if status != WLBM_OK:
        msg = lib.wlbm_batch_last_error(b) if b else lib.wlbm_last_error(None)
        raise WlbmError(status, msg.decode() if msg else "")


class _InstanceView(WormLBM):
    """A WormLBM facade over one instance of a batch (owned by the batch)."""

    def __init__(self, batch, k, spec):
        self._torch = batch._torch
        self.nx, self.ny, self.q = spec["nx"], spec["ny"], spec["q"]
        self.device, self.stream = batch.device, batch.stream
        self.h = lib.wlbm_batch_instance(batch.b, k)
        self._owner = batch

    def close(self):        # the batch owns the handle
        self.h = None


class WormLBMBatch:
    """Many independent grids advanced by one wall launch and one step launch per step.

    specs: list of dicts with nx, ny, q, bc, t_wall, mfp or mfp_field, emulate_3d,
    relax_mode; every instance uses the same storage."""

    def __init__(self, specs, storage=STORE_FP32_DEV, t_ref=300.0, theta=624.8074248458514,
                 stream=None):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        n = len(specs)
        grids = (wlbm_grid * n)()
        bcs = (wlbm_boundary * n)()
        mfps = (C.c_void_p * n)()
        mfpu = (C.c_double * n)()
        self._keep = []
        for k, sp in enumerate(specs):
            grids[k] = wlbm_grid(sp["nx"], sp["ny"], sp["q"], storage,
                                 1 if sp.get("emulate_3d", True) else 0, sp.get("relax_mode", 0),
                                 t_ref, theta, float(sp.get("speed", 1.0)))
            bcs[k] = wlbm_boundary((C.c_int32 * 4)(*sp["bc"]), (C.c_double * 4)(*sp["t_wall"]),
                                   (C.c_double * 4)(*sp.get("specularity", (0.0,) * 4)))
            if sp.get("mfp_field") is not None:
                t = torch.as_tensor(sp["mfp_field"], dtype=torch.float32,
                                    device=self.device).contiguous()
                self._keep.append(t)
                mfps[k] = t.data_ptr()
            else:
                mfps[k] = None
                mfpu[k] = float(sp["mfp"])
        dev, strm = self.device.index, self.stream.cuda_stream
        self._alloc_fns = (ALLOC_FN(lambda nb, ctx: torch.cuda.caching_allocator_alloc(
                               int(nb), dev, strm)),
                           FREE_FN(lambda p, ctx: torch.cuda.caching_allocator_delete(p)))
        self._alloc = wlbm_allocator(self._alloc_fns[0], self._alloc_fns[1], None)
        b = C.c_void_p()
        st = lib.wlbm_batch_create(n, grids, mfps, mfpu, bcs, C.byref(self._alloc),
                                   C.c_void_p(strm), C.byref(b))
        _batch_check(st, None)
        self.b = b
        self.specs = specs
        self.instances = [_InstanceView(self, k, sp) for k, sp in enumerate(specs)]

    def close(self):
        if getattr(self, "b", None):
            for v in self.instances:
                v.close()
            lib.wlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wlbm_batch_init_temperature(self, dTs):
        torch = self._torch
        ts = [torch.as_tensor(d, dtype=torch.float32, device=self.device).contiguous()
              for d in dTs]
        ptrs = (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
        _batch_check(lib.wlbm_batch_init_temperature(self.b, ptrs), self.b)
        self._keep_dT = ts

    def wlbm_batch_step(self, n=1):
        _batch_check(lib.wlbm_batch_step(self.b, int(n)), self.b)

    def wlbm_batch_set_option(self, key, value):
        _batch_check(lib.wlbm_batch_set_option(self.b, int(key), int(value)), self.b)

    def wlbm_batch_get_option(self, key):
        v = C.c_int64()
        _batch_check(lib.wlbm_batch_get_option(self.b, int(key), C.byref(v)), self.b)
        return v.value

    def wlbm_batch_check(self):
        """Raises WlbmError(WLBM_ERR_TIMEOUT) if a bounded wait in a kernel of any instance
        gave up since the last check (see include/wlbm.h)."""
        _batch_check(lib.wlbm_batch_check(self.b), self.b)

    def wlbm_batch_profile(self, every=1):
        _batch_check(lib.wlbm_batch_profile(self.b, int(every)), self.b)

    def wlbm_batch_profile_read(self):
        ms, n, alln = C.c_double(), C.c_int64(), C.c_int64()
        _batch_check(lib.wlbm_batch_profile_read(self.b, C.byref(ms), C.byref(n), C.byref(alln)),
                     self.b)
        return ms.value, n.value, alln.value

    def wlbm_batch_autotune(self, trial_steps=48):
        v, g, ms = C.c_int32(), C.c_int32(), C.c_double()
        _batch_check(lib.wlbm_batch_autotune(self.b, int(trial_steps), C.byref(v), C.byref(g),
                                             C.byref(ms)), self.b)
        return v.value, g.value, ms.value
