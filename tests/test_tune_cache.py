"""The autotuner's JSON cache file (tsnnls_tune_cache_get / _put): host
code only, no device needed."""
import json
import os

import pytest

import paper_cs_0408029_gb300 as ts


def test_round_trip_keeps_other_entries(tmp_path):
    path = str(tmp_path / "widths.json")
    assert ts.tune_cache_get(path, "dev|mixed") is None  # no file yet
    ts.tune_cache_put(path, "dev|mixed", [8, 16, 32, 32, 48])
    ts.tune_cache_put(path, "dev|fp64", [8, 8, 16, 16, 16])
    ts.tune_cache_put(path, "dev|mixed", [16, 16, 32, 48, 48])  # replaces
    assert list(ts.tune_cache_get(path, "dev|mixed")) == [16, 16, 32, 48, 48]
    assert list(ts.tune_cache_get(path, "dev|fp64")) == [8, 8, 16, 16, 16]
    assert ts.tune_cache_get(path, "other") is None
    doc = json.load(open(path))  # a standard JSON reader agrees
    assert doc["format"] == "tsnnls-batch-panel-widths/1"
    assert doc["entries"] == {"dev|mixed": [16, 16, 32, 48, 48], "dev|fp64": [8, 8, 16, 16, 16]}
    assert [p for p in os.listdir(tmp_path) if p != "widths.json"] == []  # no temporary left


def test_reads_a_file_written_by_another_json_writer(tmp_path):
    path = str(tmp_path / "w.json")
    key = 'NVIDIA "X" \\ GPU|sm_103|152 SMs'
    with open(path, "w") as f:
        json.dump({"entries": {key: [4, 8, 16, 32, 64], "b/c": [8, 8, 8, 8, 8]},
                   "format": "tsnnls-batch-panel-widths/1"}, f, indent=3)
    assert list(ts.tune_cache_get(path, key)) == [4, 8, 16, 32, 64]
    ts.tune_cache_put(path, "new", [32] * 5)
    doc = json.load(open(path))
    assert doc["entries"][key] == [4, 8, 16, 32, 64] and doc["entries"]["b/c"] == [8] * 5


@pytest.mark.parametrize("text", ["not json", "{}", '{"format": "other/1", "entries": {}}',
                                  '{"format": "tsnnls-batch-panel-widths/1", "entries": {"k": [1, 2]}}',
                                  '{"format": "tsnnls-batch-panel-widths/1", "entries": {}} trailing',
                                  '{"format": "tsnnls-batch-panel-widths/1", "entries": {}, "x": 1}'])
def test_foreign_or_malformed_file_is_refused_and_left_alone(tmp_path, text):
    path = str(tmp_path / "w.json")
    with open(path, "w") as f:
        f.write(text)
    with pytest.raises(ts.TsnnlsError) as e:
        ts.tune_cache_get(path, "k")
    assert e.value.status == ts.EINVAL
    with pytest.raises(ts.TsnnlsError):
        ts.tune_cache_put(path, "k", [8] * 5)
    assert open(path).read() == text


def test_bad_keys_are_refused(tmp_path):
    path = str(tmp_path / "w.json")
    for key in ("", "a\nb", "tab\there"):
        with pytest.raises(ts.TsnnlsError):
            ts.tune_cache_put(path, key, [8] * 5)
    assert not os.path.exists(path)
