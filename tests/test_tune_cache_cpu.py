"""The autotuner's cache (tune.cache_load / cache_store) when several processes store at once,
as the ranks of a multi-GPU run do on a fresh machine: no process fails, and the file stays
whole JSON that cache_load reads."""
import json
import multiprocessing as mp
import os

from paper_2501_19196_gb300 import tune


def _writer(args):
    path, rank = args
    for i in range(25):
        tune.cache_store(path, f"gpu{rank}|n{i}", {"best": {"kbuf": 32, "rank": rank}, "ms": {"c": float(i)}})
    return rank


def test_concurrent_stores_leave_a_whole_file(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    ctx = mp.get_context("spawn")
    with ctx.Pool(8) as pool:
        assert sorted(pool.map(_writer, [(path, r) for r in range(8)])) == list(range(8))
    with open(path) as f:
        db = json.load(f)
    assert isinstance(db, dict) and len(db) >= 1
    key = next(iter(db))
    assert tune.cache_load(path, key) == db[key]
    # no temporary file is left behind
    assert [p for p in os.listdir(os.path.dirname(path)) if p.endswith(".tmp")] == []


def test_missing_or_corrupt_cache_reads_as_empty(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tune.cache_load(path, "k") is None
    with open(path, "w") as f:
        f.write('{"k": {"best": ')  # cut short, as if another process were writing it in place
    assert tune.cache_load(path, "k") is None
    tune.cache_store(path, "k", {"best": {"kbuf": 16}})
    assert tune.cache_load(path, "k") == {"best": {"kbuf": 16}}
