"""Autotuner results kept across processes.

dfb_graph_autotune times the candidate launch shapes of a batched graph and
keeps the fastest.  This module stores that choice in a JSON file keyed by
the GPU and a description of the workload (frame sizes, tile size, storage
dtype, fragment counts, ...), so a later process with the same key applies
the stored shape with dfb_graph_set_tuning instead of timing again.
"""

from __future__ import annotations

import json
import os
import tempfile

from . import dfb as D

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "dfb_tuning.json")


def gpu_name(device: int = 0) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return "%s/sm_%d%d/%d" % (p.name, p.major, p.minor, p.multi_processor_count)


def make_key(gpu: str, workload: dict) -> str:
    """Stable key of a GPU and a workload description (JSON-serialisable)."""
    return gpu + "|" + json.dumps(workload, sort_keys=True, separators=(",", ":"))


def load(path: str = DEFAULT_PATH) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key: str, shape: dict, path: str = DEFAULT_PATH) -> None:
    """Add or replace one entry; the file is replaced atomically (two
    processes storing at once keep one of the two entries)."""
    data = load(path)
    data[key] = {k: shape[k] for k in ("ring_kb", "ctas_per_sm", "groups", "ms") if k in shape}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def autotune_cached(graph, key: str, stream=None, reps: int = 3, path: str = DEFAULT_PATH,
                    lib=D) -> dict:
    """The stored shape for `key` applied to `graph`, or a fresh autotune
    (stored for next time).  Returns the shape and whether it came from the
    cache."""
    entry = load(path).get(key)
    if entry is not None:
        try:
            lib.dfb_graph_set_tuning(graph, entry["ring_kb"], entry["ctas_per_sm"],
                                     entry["groups"])
            return dict(entry, cached=True)
        except (KeyError, D.DfbError):
            pass  # stale or unusable entry: tune again
    best = lib.dfb_graph_autotune(graph, stream, reps)
    store(key, best, path)
    return dict(best, cached=False)
