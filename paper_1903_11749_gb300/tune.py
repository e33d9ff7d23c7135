"""Tuning cache: the launch tuning chosen by ppr_autotune (native timing of
candidate walkers-per-CTA, queue chunk and cooperative threshold), kept in a
JSON file keyed by the graph's shape, the run parameters and the device.
Tuning never changes results; a stale entry only costs speed."""
from __future__ import annotations

import json
import os

_DEFAULT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning.json")


def cache_path() -> str:
    return os.environ.get("PPR_TUNE_CACHE", _DEFAULT)


def key(G, device_name: str, **run) -> str:
    info = G.info()
    return (f"n={info.n};m={info.m};inst={info.instances};R={run.get('R')};alpha={run.get('alpha')};"
            f"seg={int(bool(run.get('segments', False)))};sampler={run.get('sampler', 0)};topk={run.get('topk', 0)};"
            f"dev={device_name}")


def tuned(G, device_name: str, sample_sources: int = 0, refresh: bool = False, **run) -> dict:
    """Cached tuning for this graph and run; times the candidates on a miss."""
    path = cache_path()
    k = key(G, device_name, **run)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not refresh and k in cache:
        return dict(cache[k], cached=True)
    t = G.autotune(sample_sources=sample_sources, **run)
    cache[k] = t
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return dict(t, cached=False)


def launch_kwargs(t: dict) -> dict:
    return {"chunk_sources": t["chunk_sources"], "large_degree": t["large_degree"],
            "warps_per_block": t["warps_per_block"], "refill_lanes": t.get("refill_lanes", 0)}
