"""Autotune cache: kernel variants per (device, grid, precision), kept as JSON.

HartreePlan.autotune() times every compiled tile shape of each pass on the
plan's own workspace.  tuned(plan) reuses an earlier result for the same
device name, grid and precision when the cache has one, else tunes and saves.
The cache lives in $HARTREE_AUTOTUNE_CACHE or ~/.cache/hartree_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os
import threading

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("HARTREE_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "hartree_gb300", "autotune.json"))


def _key(plan) -> str:
    import torch

    name = torch.cuda.get_device_name(plan.device)
    return f"{name}|{plan.n[0]}x{plan.n[1]}x{plan.n[2]}|{plan.precision}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tuned(plan, path: str | None = None):
    """Apply cached variants to `plan`, or autotune it and store the result; returns the picks."""
    path = path or cache_path()
    key = _key(plan)
    with _lock:
        cache = _load(path)
        if key in cache:
            try:
                plan.set_variants(cache[key])
                return list(cache[key])
            except Exception:
                pass  # stale entry (variant list changed): tune again
        choice = plan.autotune()
        cache = _load(path)
        cache[key] = choice
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = f"{path}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass
        return choice
