"""The autotuner cache on the host: signatures separate batches that differ in
any size or storage type (and GPU), entries round-trip, malformed or
mismatched entries are ignored, and writes replace the file whole."""
import json

import torch

from paper_2311_18141_gb300 import tuning_cache


def _problem(M, K, N, nnz, vdt=torch.bfloat16, bdt=torch.bfloat16):
    return {"M": M, "K": K, "N": N, "colind": torch.zeros(nnz, dtype=torch.int32),
            "vals": torch.zeros(1, dtype=vdt), "B": torch.zeros(1, dtype=bdt)}


def test_signature_depends_on_every_size_type_and_order():
    base = [_problem(100, 100, 16, 500), _problem(2000, 2000, 64, 9000)]
    sig = tuning_cache.batch_signature(base, "GPU-A")
    assert sig == tuning_cache.batch_signature([dict(q) for q in base], "GPU-A")
    variants = [
        [_problem(101, 100, 16, 500), base[1]],
        [_problem(100, 101, 16, 500), base[1]],
        [_problem(100, 100, 32, 500), base[1]],
        [_problem(100, 100, 16, 501), base[1]],
        [_problem(100, 100, 16, 500, vdt=torch.float32), base[1]],
        [_problem(100, 100, 16, 500, bdt=torch.float32), base[1]],
        [base[1], base[0]],
        base[:1],
    ]
    sigs = {tuning_cache.batch_signature(v, "GPU-A") for v in variants}
    assert sig not in sigs and len(sigs) == len(variants)
    assert tuning_cache.batch_signature(base, "GPU-B") != sig


def test_store_load_round_trip_and_replace(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert tuning_cache.load(path, "abc", 2) is None
    tuning_cache.store(path, "abc", [4, 8], [1, 2], [256, 512], 1.25)
    tuning_cache.store(path, "def", [1], [1], [128], 0.5)
    assert tuning_cache.load(path, "abc", 2) == {"tile_rows": [4, 8], "tile_cols": [1, 2],
                                                 "chunk_items": [256, 512], "ms": 1.25}
    assert tuning_cache.load(path, "def", 1)["ms"] == 0.5
    tuning_cache.store(path, "abc", [2, 2], [1, 1], [1024, 1024], 0.75)
    assert tuning_cache.load(path, "abc", 2)["tile_rows"] == [2, 2]
    assert sorted(json.load(open(path))) == ["abc", "def"]
    assert not [p for p in (tmp_path / "sub").iterdir() if p.name.startswith(".tuning-")]


def test_malformed_or_mismatched_entries_are_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tuning_cache.load(str(path), "abc", 1) is None
    path.write_text(json.dumps({"abc": {"tile_rows": [1], "tile_cols": [1]}}))
    assert tuning_cache.load(str(path), "abc", 1) is None
    path.write_text(json.dumps({"abc": {"tile_rows": [1, 2], "tile_cols": [1, 1],
                                        "chunk_items": [256, 256], "ms": 1.0}}))
    assert tuning_cache.load(str(path), "abc", 3) is None          # another batch length
    path.write_text(json.dumps(["abc"]))
    assert tuning_cache.load(str(path), "abc", 1) is None
