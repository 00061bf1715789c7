"""Host logic of the autotuner (no GPU): the choice among measured configurations and
the tuning cache file."""
import math
import os

import pytest

from paper_2411_09982_gb300 import magnus as M


def entry(p, s, t, a, err, us, tu=0.0):
    return dict(precision=p, slices=s, taylor=t, action=a, error=err, us_per_interval=us, taylor_target=tu)


TABLE = [entry(0, 0, 1, 0, 1e-12, 900.0),      # FP64: accurate, slow
         entry(1, 4, 0, 0, 2e-4, 200.0),       # fastest, too inaccurate
         entry(1, 5, 0, 0, 4e-7, 300.0),       # within 1e-6 only without the safety factor
         entry(1, 6, 0, 0, 8e-9, 350.0),       # the answer for 1e-6 with safety 4
         entry(1, 6, 1, 0, 5e-9, 380.0),
         entry(0, 0, 1, 1, math.nan, math.nan)]  # a candidate that could not run


def test_select_takes_the_fastest_entry_within_tolerance():
    assert M.mg_tune_select(TABLE, 1e-6, 4.0) == 3
    assert M.mg_tune_select(TABLE, 1e-6, 1.0) == 2
    assert M.mg_tune_select(TABLE, 1e-3, 4.0) == 1
    assert M.mg_tune_select(TABLE, 1e-11, 4.0) == 0
    # brute force over every tolerance: the choice is the minimum time among qualifying entries
    for tol in (1e-13, 1e-10, 1e-8, 1e-6, 1e-4, 1.0):
        for safety in (1.0, 2.0, 4.0, 10.0):
            ok = [i for i, e in enumerate(TABLE) if e["error"] * safety <= tol]
            if not ok:
                with pytest.raises(M.MagnusError) as ex:
                    M.mg_tune_select(TABLE, tol, safety)
                assert ex.value.code == M.MG_EUNSUPPORTED
            else:
                assert M.mg_tune_select(TABLE, tol, safety) == min(ok, key=lambda i: TABLE[i]["us_per_interval"])


def test_select_rejects_bad_arguments():
    for tol, safety in ((0.0, 4.0), (-1.0, 4.0), (1e-6, 0.5)):
        with pytest.raises(M.MagnusError) as ex:
            M.mg_tune_select(TABLE, tol, safety)
        assert ex.value.code == M.MG_EINVAL


def test_cache_round_trip_latest_wins_and_prefix_lookup(tmp_path):
    path = str(tmp_path / "tune.txt")
    key = "gpu=GB300|d=30|K=1|out=0|tol=1e-06|nu=5|N=1024"
    assert M.mg_tune_cache_lookup(path, key) is None          # no file yet
    M.mg_tune_cache_store(path, key, TABLE, 3)
    got = M.mg_tune_cache_lookup(path, key)
    assert got == TABLE[3]
    M.mg_tune_cache_store(path, key, TABLE, 4)                # a later tuning of the same key wins
    assert M.mg_tune_cache_lookup(path, key) == TABLE[4]
    other = "gpu=GB300|d=30|K=1|out=0|tol=1e-06|nu=6|N=2048"
    M.mg_tune_cache_store(path, other, TABLE, 2)
    assert M.mg_tune_cache_lookup(path, key) == TABLE[4]
    # the leading fields of a key find the latest tuning of that family
    assert M.mg_tune_cache_lookup(path, "gpu=GB300|d=30|K=1|out=0|tol=1e-06") == TABLE[2]
    # a prefix that ends inside a field does not match
    assert M.mg_tune_cache_lookup(path, "gpu=GB300|d=3") is None
    assert M.mg_tune_cache_lookup(path, "gpu=GB300|d=30|K=1|out=1") is None
    lines = open(path).read().splitlines()
    assert len(lines) == 3 and all(line.count("\t") == 2 for line in lines)


def test_cache_rejects_keys_that_would_break_the_format(tmp_path):
    path = str(tmp_path / "tune.txt")
    for key in ("a\tb", "a;b", "a\nb", ""):
        with pytest.raises(M.MagnusError) as ex:
            M.mg_tune_cache_store(path, key, TABLE, 0)
        assert ex.value.code == M.MG_EINVAL
    with pytest.raises(M.MagnusError):
        M.mg_tune_cache_store(path, "k", TABLE, len(TABLE))
    assert not os.path.exists(path)


def test_cache_keeps_the_taylor_target_and_reads_six_field_entries(tmp_path):
    """An entry's Taylor truncation target survives the round trip bit for bit; lines
    written with six fields per entry (no target) read back with target 0."""
    path = str(tmp_path / "tune.txt")
    key = "gpu=GB300|d=729|K=6|out=1|tol=1e-06|nu=3|N=2048"
    table = [entry(1, 6, 0, 0, 1.5e-8, 310.0, 2.0 ** -34), entry(1, 6, 0, 0, 7.6e-9, 350.0)]
    M.mg_tune_cache_store(path, key, table, 0)
    got = M.mg_tune_cache_lookup(path, key)
    assert got == table[0] and got["taylor_target"] == 2.0 ** -34
    with open(path, "a") as f:
        f.write("gpu=GB300|d=30|K=1|out=0|tol=1e-06|nu=5|N=1024\t1\t0 0 1 0 1e-12 900;1 6 0 0 8e-09 350\n")
    old = M.mg_tune_cache_lookup(path, "gpu=GB300|d=30|K=1|out=0|tol=1e-06|nu=5|N=1024")
    assert old == entry(1, 6, 0, 0, 8e-9, 350.0)
