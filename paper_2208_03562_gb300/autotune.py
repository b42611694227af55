"""Variant selection for the interior kernel, cached per device and grid class.

The library compiles a few shapes of the TMA-staged interior kernel (tile width
and height, CTA size, CTAs per SM).  ``tune(lbm)`` picks one for a handle: it
looks up a JSON cache keyed by (GPU name, storage type, density-gradient mode,
power-of-two buckets of nx and ny, the compiled variant list) and otherwise
times every variant on the handle's own grid with ``lbm_autotune`` (the
library restores the state afterwards) and stores the winner.
"""
import json
import math
import os
import threading

from . import lbm as L

_LOCK = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("PRC_LBM_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "prc_lbm")
    return os.path.join(base, "autotune.json")


def _bucket(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(n, 1))))


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def key_of(p) -> str:
    nv = L.lbm_variant_count(p.dtype)
    variants = [L.lbm_variant_info(p.dtype, i) for i in range(nv)]
    return json.dumps([_device_name(), int(p.dtype), int(p.drho), _bucket(p.nx), _bucket(p.ny), variants])


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only costs a re-tune


def tune(lb: "L.Lbm", steps: int = 20, use_cache: bool = True) -> dict:
    """Select the variant for ``lb``; returns {"variant", "ms_per_step", "cached"}."""
    k = key_of(lb.p)
    with _LOCK:
        d = _load() if use_cache else {}
        if k in d:
            try:
                lb.variant = d[k]["variant"]
                return {"variant": d[k]["variant"], "ms_per_step": d[k]["ms_per_step"], "cached": True}
            except L.LbmError:
                pass  # e.g. the cluster engine does not fit this grid of the bucket: re-tune
        best, ms = lb.autotune(steps)
        d = _load()
        d[k] = {"variant": best, "ms_per_step": ms}
        _store(d)
        return {"variant": best, "ms_per_step": ms, "cached": False}
