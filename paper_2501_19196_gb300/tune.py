"""Autotuner front end: candidate tunables, a JSON cache, and the native rs_tune sweep.

The sweep itself (rebuild + render + adjoint per candidate, CUDA-event timed) runs in
libraysplats.so (`rs_tune`); this module picks the candidates and caches the winner keyed by
(GPU name, Gaussian-count bucket, ray-count bucket, camera count, backward or not).
"""
from __future__ import annotations

import ctypes
import itertools
import json
import math
import os

import torch

from . import native

CACHE_ENV = "RAYSPLATS_TUNE_CACHE"


def default_cache_path() -> str:
    return os.environ.get(CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "raysplats_tune.json"))


def candidates(tiles=((8, 4), (4, 8)), kbufs=(16, 32), leaves=(16, 32), warps=(4,), morton=(20, 21),
               traversal=(2,), persistent=1, hit_lists=(256,), smem_nodes=256):
    """The cross product of the given tunables (all persistent launches by default)."""
    out = []
    for (tw, th), k, leaf, w, mb, tr, hl in itertools.product(tiles, kbufs, leaves, warps, morton, traversal,
                                                                hit_lists):
        out.append(native.RsTuneParams(tw, th, k, leaf, mb, persistent, w, tr, smem_nodes, hl))
    return out


def cache_key(n_gauss, n_rays, n_cams, backward, device=None) -> str:
    name = torch.cuda.get_device_name(device) if torch.cuda.is_available() else "cpu"
    b = lambda x: 2 ** int(round(math.log2(max(1, x))))  # noqa: E731
    return f"{name}|n{b(n_gauss)}|r{b(n_rays)}|c{n_cams}|{'fb' if backward else 'f'}"


def autotune(params5, cams, render_params, d_rgb=None, d_alpha=None, cands=None, reps=3, cache=True,
             cache_path=None, stream=None):
    """Run the sweep (or read the cache).  params5 = (means, quats, scales, opacities, rgb) CUDA
    tensors; cams: workloads.Cameras; render_params: renderer.RenderParams.  Returns
    (best RsTuneParams, {candidate dict as json: ms})."""
    lib = native.load()
    n = params5[0].shape[0]
    cam_arr = native.cameras_to_ctypes(cams)
    P = int(sum(c.width * c.height for c in cam_arr))
    key = cache_key(n, P, len(cam_arr), d_rgb is not None)
    path = cache_path or default_cache_path()
    if cache:
        hit = cache_load(path, key)
        if hit is not None:
            return native.RsTuneParams(**hit["best"]), hit.get("ms", {})
    cands = cands or candidates()
    arr = (native.RsTuneParams * len(cands))(*cands)
    dev = params5[0].device
    out = (torch.empty((P, 3), device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev))
    frame = native.RsFrame(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
    g = native.RsGaussians(n, *[t.data_ptr() for t in params5])
    grads = None
    dl = None
    if d_rgb is not None:
        scratch = [torch.zeros((n, w), device=dev) for w in (3, 4, 3, 1, 3)]
        grads = native.RsGaussianGrads(*[t.data_ptr() for t in scratch])
        dl = native.RsFrameGrad(d_rgb.data_ptr(), None if d_alpha is None else d_alpha.data_ptr())
    best = native.RsTuneParams()
    ms = (ctypes.c_float * len(cands))()
    rp = render_params.to_c()
    s = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    native.check(lib.rs_tune(ctypes.byref(g), float(render_params.Q), cam_arr, len(cam_arr), ctypes.byref(rp), arr,
                             len(cands), int(reps), ctypes.byref(frame), None if dl is None else ctypes.byref(dl),
                             None if grads is None else ctypes.byref(grads), ctypes.byref(best), ms, s))
    table = {json.dumps(c.as_dict(), sort_keys=True): float(m) for c, m in zip(cands, ms)}
    if cache:
        cache_store(path, key, {"best": best.as_dict(), "ms": table})
    return best, table


def cache_load(path, key):
    """The cached entry for key, or None (no file, no entry, or a file being replaced)."""
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError, AttributeError):
        return None


def cache_store(path, key, entry):
    """Add entry under key.  Best effort: several processes (one per GPU) may store at once;
    each writes its own temporary file and renames it over the cache, so a reader sees a whole
    file, and the last rename wins (an entry another process stored meanwhile may be lost and
    is then measured again)."""
    db = {}
    try:
        with open(path) as f:
            db = json.load(f)
        if not isinstance(db, dict):
            db = {}
    except (OSError, ValueError):
        db = {}
    db[key] = entry
    tmp = f"{path}.{os.getpid()}.tmp"
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        try:
            os.remove(tmp)
        except OSError:
            pass
