"""Autotuner for the engine's launch options (block size, driver, solo-episode
threshold, learned-frontier threshold and refresh period).

`tune()` times short normalisations of a representative workload for each
candidate and stores the fastest per GPU name in a JSON cache
(`_build/autotune.json` unless TRS_AUTOTUNE_CACHE is set); `choose()` returns
the cached choice, or defaults when nothing was tuned on this GPU.
"""
from __future__ import annotations

import json
import os

CACHE = os.environ.get("TRS_AUTOTUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                                    "autotune.json"))

DEFAULTS = {
    "plain": {"mode": "plain", "driver": "persistent", "block_size": 512},
    "frontier": {"mode": "frontier", "driver": "persistent", "block_size": 512, "solo_max": 512},
    "learned": {"mode": "learned", "driver": "persistent", "block_size": 512, "solo_max": 512,
                "refresh": 64, "threshold": 0.5},
}


def gpu_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:  # pragma: no cover - torch missing
        pass
    return "cpu"


def load_cache(path: str = CACHE) -> dict:
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def save_cache(cache: dict, path: str = CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(mode: str, gpu: str | None = None, path: str = CACHE) -> dict:
    gpu = gpu or gpu_name()
    entry = load_cache(path).get(gpu, {}).get(mode)
    out = dict(DEFAULTS[mode])
    if entry:
        out.update(entry["opts"])
    return out
