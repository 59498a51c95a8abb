"""Record comparison helpers shared by the tests and the golden-value script.

These only reshape records (oracle dataclasses, library ndarray rows, or
plain dicts) into one canonical tuple form; they compute nothing about p_min.
"""
from __future__ import annotations

import hashlib
import json

FIELDS = ("n_first", "n_count", "max_pmin", "argmax_n", "sum_pmin", "wsum_pmin", "n_slow",
          "counterexample_n")


def canon(rec) -> tuple:
    """Canonical tuple of a record given as dict, oracle record or numpy row."""
    if isinstance(rec, tuple):
        return rec
    if isinstance(rec, dict):
        get = rec.__getitem__
    elif hasattr(rec, "dtype"):
        get = lambda f: rec[f]  # noqa: E731
    else:
        get = lambda f: getattr(rec, f)  # noqa: E731
    head = tuple(int(get(f)) for f in FIELDS)
    hist = tuple(int(x) for x in list(get("hist"))[:64])
    hist = hist + (0,) * (64 - len(hist))
    return head + hist


def to_dict(t: tuple) -> dict:
    d = dict(zip(FIELDS, t[:len(FIELDS)]))
    d["hist"] = list(t[len(FIELDS):])
    return d


def digest(records) -> str:
    h = hashlib.sha256()
    for r in records:
        h.update(json.dumps(canon(r), separators=(",", ":")).encode())
        h.update(b"\n")
    return h.hexdigest()


def diff(a, b, limit: int = 5) -> list[str]:
    """Human-readable differences between two record sequences."""
    out = []
    if len(a) != len(b):
        out.append(f"length {len(a)} != {len(b)}")
    for i, (x, y) in enumerate(zip(a, b)):
        cx, cy = canon(x), canon(y)
        if cx != cy:
            dx, dy = to_dict(cx), to_dict(cy)
            fields = [k for k in dx if dx[k] != dy[k]]
            out.append(f"record {i} (n_first {cx[0]}): " +
                       ", ".join(f"{k}: {dx[k]} vs {dy[k]}" for k in fields if k != "hist") +
                       (" hist differs" if "hist" in fields else ""))
            if len(out) >= limit:
                break
    return out
