"""Autotuning cache for libwlbm.

The search itself is native (wlbm_autotune / wlbm_batch_autotune time every candidate of
step-kernel variant x CUDA-graph replay on the real grid; for batches also the persistent
kernel at two ring depths, with a chunk of 64 steps per launch or the graph's).  This module only remembers
the winner per workload signature in a JSON file, so a later run with the same shapes
skips the search.  The signature covers the GPU model, the storage type, the grids' shapes,
walls and MFP kind, and the build of libwlbm.so (its size and modification time), so a
rebuilt library searches again.  Cache file: $WLBM_AUTOTUNE_CACHE, else
_autotune_cache.json next to this module.
"""
import hashlib
import json
import os

from .wlbm import (LIB_PATH, OPT_GRAPH_STEPS, OPT_PERSISTENT, OPT_RING_STAGES,
                   OPT_STEP_VARIANT)

_HERE = os.path.dirname(os.path.abspath(__file__))


def _cache_path():
    return os.environ.get("WLBM_AUTOTUNE_CACHE", os.path.join(_HERE, "_autotune_cache.json"))


def _build_identity():
    try:
        st = os.stat(LIB_PATH)
        return [st.st_size, st.st_mtime_ns]
    except OSError:
        return None


def signature(specs, storage):
    import torch
    shapes = sorted((int(s["nx"]), int(s["ny"]), int(s["q"]), tuple(int(k) for k in s["bc"]),
                     s.get("mfp_field") is not None) for s in specs)
    key = json.dumps([torch.cuda.get_device_name(), int(storage), shapes, _build_identity()])
    return hashlib.sha1(key.encode()).hexdigest()


def _load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(sig, rec):
    cache = _load()
    cache[sig] = rec
    tmp = _cache_path() + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _cache_path())


def tune_batch(batch, storage, trial_steps=48, use_cache=True):
    """Pick variant, graph replay, persistent kernel and its ring depth for a WormLBMBatch
    (before its init).  Returns the record {variant, graph_steps, persistent, ring_stages,
    ms_per_step, cached}."""
    sig = signature(batch.specs, storage)
    if use_cache:
        rec = _load().get(sig)
        if rec and "persistent" in rec:
            batch.wlbm_batch_set_option(OPT_PERSISTENT, 0)
            batch.wlbm_batch_set_option(OPT_STEP_VARIANT, rec["variant"])
            batch.wlbm_batch_set_option(OPT_PERSISTENT, rec["persistent"])
            batch.wlbm_batch_set_option(OPT_RING_STAGES, rec["ring_stages"])
            batch.wlbm_batch_set_option(OPT_GRAPH_STEPS, rec["graph_steps"])
            return dict(rec, cached=True)
    v, g, ms = batch.wlbm_batch_autotune(trial_steps)
    rec = {"variant": v, "graph_steps": g, "ms_per_step": ms,
           "persistent": batch.wlbm_batch_get_option(OPT_PERSISTENT),
           "ring_stages": batch.wlbm_batch_get_option(OPT_RING_STAGES)}
    _store(sig, rec)
    return dict(rec, cached=False)


def tune(handle, spec, storage, trial_steps=48, use_cache=True):
    """The same for one WormLBM grid (before its init)."""
    sig = signature([spec], storage)
    if use_cache:
        rec = _load().get(sig)
        if rec:
            handle.wlbm_set_option(OPT_STEP_VARIANT, rec["variant"])
            handle.wlbm_set_option(OPT_GRAPH_STEPS, rec["graph_steps"])
            return dict(rec, cached=True)
    v, g, ms = handle.wlbm_autotune(trial_steps)
    rec = {"variant": v, "graph_steps": g, "ms_per_step": ms}
    _store(sig, rec)
    return dict(rec, cached=False)
