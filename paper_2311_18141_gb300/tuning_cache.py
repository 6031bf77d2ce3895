"""Persisted autotuner results for batched products.

spmm_batch_autotune times candidate tile and chunk shapes for every size class
of a batch.  The shapes it keeps depend on the problems' sizes and storage types
and on the GPU, so they are stored as JSON keyed by a signature of exactly
those; a later run over a batch with the same signature sets the stored shapes
instead of tuning again.  The sparsity patterns themselves are not part of the
signature: two batches of the same sizes share their tuned shapes.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile


def batch_signature(problems, device_name: str) -> str:
    """Signature of a batch: the GPU name and, per problem in order, M, K, N,
    nnz and the storage types of A's values and of B."""
    h = hashlib.sha256(device_name.encode())
    for q in problems:
        h.update(f"{int(q['M'])},{int(q['K'])},{int(q['N'])},{int(q['colind'].numel())},"
                 f"{q['vals'].dtype},{q['B'].dtype};".encode())
    return h.hexdigest()[:32]


def _read(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def load(path: str, signature: str, count: int) -> dict | None:
    """The entry stored for `signature` if it is well formed for `count`
    problems: {"tile_rows", "tile_cols", "chunk_items": lists, "ms": float}."""
    e = _read(path).get(signature)
    if not isinstance(e, dict):
        return None
    try:
        shapes = {k: [int(x) for x in e[k]] for k in ("tile_rows", "tile_cols", "chunk_items")}
        ms = float(e["ms"])
    except (KeyError, TypeError, ValueError):
        return None
    if any(len(v) != count for v in shapes.values()):
        return None
    return {**shapes, "ms": ms}


def store(path: str, signature: str, tile_rows, tile_cols, chunk_items, ms: float) -> None:
    """Add or replace the entry for `signature`; the file is replaced atomically."""
    data = _read(path)
    data[signature] = {"tile_rows": [int(x) for x in tile_rows],
                       "tile_cols": [int(x) for x in tile_cols],
                       "chunk_items": [int(x) for x in chunk_items], "ms": float(ms)}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning-", suffix=".json")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
