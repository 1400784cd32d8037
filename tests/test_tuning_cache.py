"""The JSON tuning cache (host logic, CPU)."""
import json

from paper_1612_08792_gb300 import tuning_cache as tc


def test_key_buckets_and_fields():
    a = tc.batch_key("NVIDIA GB300", [(321, 481)] * 256, 15, 0, 0, 0)
    b = tc.batch_key("NVIDIA GB300", [(321, 481)] * 255 + [(320, 481)], 15, 0, 0, 0)  # same bucket
    c = tc.batch_key("NVIDIA GB300", [(321, 481)] * 256, 15, 0, 1, 0)                  # another colour model
    d = tc.batch_key("NVIDIA GB300", [(642, 962)] * 256, 15, 0, 0, 0)                  # 4x the pixels
    assert a == b and a != c and a != d
    assert a.startswith("NVIDIA GB300|v15|K0|c0|p0|n256|px2^")


def test_round_trip_and_bad_files(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert tc.lookup(path, "k") is None                       # no file
    tc.store(path, "k", {"blocks_per_sm": 7, "finalize16": False, "em_pass_ms": {"7": 1.06}})
    tc.store(path, "j", {"blocks_per_sm": 6, "finalize16": True})
    assert tc.lookup(path, "k")["blocks_per_sm"] == 7 and tc.lookup(path, "j")["finalize16"] is True
    assert set(json.load(open(path))) == {"j", "k"}
    tc.store(path, "bad", {"blocks_per_sm": 99, "finalize16": False})
    assert tc.lookup(path, "bad") is None                     # out of range entries are ignored
    tc.store(path, "f", {"blocks_per_sm": 7, "finalize16": False, "first_pass_blocks_per_sm": 6})
    assert tc.lookup(path, "f")["first_pass_blocks_per_sm"] == 6
    for bad in (17, -1, "6", True):
        tc.store(path, "fb", {"blocks_per_sm": 7, "finalize16": False, "first_pass_blocks_per_sm": bad})
        assert tc.lookup(path, "fb") is None
    with open(path, "w") as fh:
        fh.write("{not json")
    assert tc.lookup(path, "k") is None and tc.load(path) == {}
