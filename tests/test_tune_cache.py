"""The batched-launch tuning cache (host only, no GPU): a JSON file mapping
keys (GPU, kernel family, size class) to launch configurations, written by
batch_autotune and read by batch_create."""
import json
import os

import pytest

from paper_2302_10736_gb300 import pfgrid

CFG_A = {"window": 256, "terminals_per_thread": 2, "ctas_per_sm": 4, "adjoint_form": 0, "ybus_lanes": 4,
         "ybus_block": 256}
CFG_B = {"window": 128, "terminals_per_thread": 3, "ctas_per_sm": 0, "adjoint_form": 1, "ybus_lanes": 32,
         "ybus_block": 512}
KEY_A = "NVIDIA GB300|batched|nb<=2^14|S<=2^10|n-1"
KEY_B = "NVIDIA GB300|batched|nb<=2^18|S<=2^4|no-outage"


def test_missing_file_is_an_empty_cache(tmp_path):
    assert pfgrid.tune_cache_lookup(str(tmp_path / "none.json"), KEY_A) is None


def test_store_and_lookup_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    pfgrid.tune_cache_store(path, KEY_A, CFG_A)
    pfgrid.tune_cache_store(path, KEY_B, CFG_B)
    assert pfgrid.tune_cache_lookup(path, KEY_A) == CFG_A
    assert pfgrid.tune_cache_lookup(path, KEY_B) == CFG_B
    # replacing one entry keeps the other
    pfgrid.tune_cache_store(path, KEY_A, CFG_B)
    assert pfgrid.tune_cache_lookup(path, KEY_A) == CFG_B
    assert pfgrid.tune_cache_lookup(path, KEY_B) == CFG_B
    # the file is plain JSON, and no temporary file is left behind
    doc = json.load(open(path))
    assert set(doc["entries"]) == {KEY_A, KEY_B}
    assert os.listdir(str(tmp_path)) == ["tune.json"]
    assert pfgrid.tune_cache_lookup(path, "other key") is None


def test_reader_skips_unknown_members(tmp_path):
    path = str(tmp_path / "tune.json")
    doc = {"pfgrid_tune_cache": 1, "note": ["written", "by", "hand"], "flags": {"x": True, "y": None},
           "entries": {KEY_A: dict(CFG_A, ms=1.25, origin="bench")}}
    json.dump(doc, open(path, "w"))
    assert pfgrid.tune_cache_lookup(path, KEY_A) == CFG_A


@pytest.mark.parametrize("text", ["", "{", "not json", '{"entries": {"k": 3}}', '{"entries": {"k": {"window": }}}'])
def test_malformed_file_is_reported(tmp_path, text):
    path = str(tmp_path / "tune.json")
    open(path, "w").write(text)
    with pytest.raises(pfgrid.PfError):
        pfgrid.tune_cache_lookup(path, KEY_A)


def test_incomplete_entry_is_reported(tmp_path):
    path = str(tmp_path / "tune.json")
    json.dump({"entries": {KEY_A: {"window": 256}}}, open(path, "w"))
    with pytest.raises(pfgrid.PfError):
        pfgrid.tune_cache_lookup(path, KEY_A)


@pytest.mark.parametrize("key", ['with "quote"', "back\\slash", ""])
def test_invalid_keys_are_rejected(tmp_path, key):
    with pytest.raises(pfgrid.PfError):
        pfgrid.tune_cache_store(str(tmp_path / "tune.json"), key, CFG_A)
