"""The autotuner's cache file (host only, no GPU): a text file with one line per layer shape,
key<TAB>qr<TAB>k2<TAB>timings. Lookups are deterministic, the last valid line of a key wins,
malformed lines and out-of-range choices are ignored, and keys that would break the format are
rejected."""
import os

import pytest


@pytest.fixture(scope="module")
def capi():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2201_05529_gb300 as pkg
    pkg.build()
    return pkg.load()


KEY = "NVIDIA_GB300|drv13000|sm103|p4|n10|k2048|m2048|c10240|b2048"


def test_round_trip_and_last_line_wins(capi, tmp_path):
    path = str(tmp_path / "tune.tsv")
    assert capi.tune_cache_lookup(path, KEY) is None            # no file yet
    capi.tune_cache_store(path, KEY, 2, 0)
    assert capi.tune_cache_lookup(path, KEY) == (2, 0)
    capi.tune_cache_store(path, KEY, 1, 1)
    assert capi.tune_cache_lookup(path, KEY) == (1, 1)
    assert capi.tune_cache_lookup(path, KEY.replace("p4", "p0")) is None   # precision is part of the key
    # the same file read twice gives the same answer
    assert capi.tune_cache_lookup(path, KEY) == capi.tune_cache_lookup(path, KEY)


def test_malformed_and_out_of_range_lines_are_ignored(capi, tmp_path):
    path = str(tmp_path / "tune.tsv")
    capi.tune_cache_store(path, KEY, 0, 0)
    with open(path, "a") as f:
        f.write("garbage without a tab\n")
        f.write(KEY + "\t7\t0\n")                  # qr out of range
        f.write(KEY + "\tx\ty\n")                  # not numbers
    assert capi.tune_cache_lookup(path, KEY) == (0, 0)


def test_bad_keys_and_choices_are_rejected(capi, tmp_path):
    path = str(tmp_path / "tune.tsv")
    with pytest.raises(capi.PTError):
        capi.tune_cache_store(path, "a\tb", 0, 0)
    with pytest.raises(capi.PTError):
        capi.tune_cache_store(path, KEY, 3, 0)
    assert not os.path.exists(path)
