"""A JSON file of batch launch choices, so that a process need not autotune a
batch shape another process has tuned on the same kind of GPU.

Key: the GPU name, the spacing (or K) asked for, the colour model, the
precision, the image count and the total pixel count in quarter-octave
buckets.  Value: the E + M pass blocks per SM, the 16-lane finalize choice,
the measured E + M times and (optional) the first pass's blocks per SM.  Writes go through a temporary file and an
atomic rename; a file that cannot be parsed reads as empty.
"""
from __future__ import annotations

import json
import math
import os
import tempfile


def batch_key(device: str, shapes, spacing: int, K: int, colour: int, precision: int) -> str:
    """shapes: (H, W) per image."""
    total = sum(int(h) * int(w) for h, w in shapes)
    bucket = round(4 * math.log2(max(total, 1))) / 4
    return f"{device}|v{int(spacing)}|K{int(K)}|c{int(colour)}|p{int(precision)}|n{len(shapes)}|px2^{bucket:g}"


def load(path: str) -> dict:
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(path: str, key: str):
    entry = load(path).get(key)
    if not isinstance(entry, dict):
        return None
    bps, f16 = entry.get("blocks_per_sm"), entry.get("finalize16")
    if not (isinstance(bps, int) and 1 <= bps <= 16 and isinstance(f16, bool)):
        return None
    first = entry.get("first_pass_blocks_per_sm", 0)  # 0: the first pass follows blocks_per_sm
    if not (isinstance(first, int) and not isinstance(first, bool) and 0 <= first <= 16):
        return None
    return entry


def store(path: str, key: str, entry: dict) -> None:
    data = load(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning", suffix=".json")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
