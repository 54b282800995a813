"""The autotuner's cache on the host (no GPU): key composition, the JSON file
round trip, tolerant parsing, and refusal of files of another format.  (The
GPU tests check that a tuned solve equals the untuned one bit for bit and that
a reloaded cache skips the timing.)"""

import json

import pytest


@pytest.fixture()
def tuner():
    import paper_2502_03249_gb300 as stag
    stag.load()
    stag.tuner.clear()
    yield stag.tuner
    stag.tuner.clear()


def test_key_names_kernel_shape_storage_and_gpu(tuner):
    k = tuner.make_key("cg_hop", (48, 48, 48, 12), 3, 18, 1, "NVIDIA GB300")
    assert k == "cg_hop|48x48x48x12|p3|r18|n1|NVIDIA_GB300"
    # every field matters
    assert len({k, tuner.make_key("cg_hop", (48, 48, 48, 14), 3, 18, 1, "NVIDIA GB300"),
                tuner.make_key("cg_hop", (48, 48, 48, 12), 1, 18, 1, "NVIDIA GB300"),
                tuner.make_key("cg_hop", (48, 48, 48, 12), 3, 12, 1, "NVIDIA GB300"),
                tuner.make_key("cg_hop", (48, 48, 48, 12), 3, 18, 16, "NVIDIA GB300"),
                tuner.make_key("cg_upd", (48, 48, 48, 12), 3, 18, 1, "NVIDIA GB300"),
                tuner.make_key("cg_hop", (48, 48, 48, 12), 3, 18, 1, "NVIDIA B200")}) == 7
    # characters that would break the file are replaced
    assert tuner.make_key("x", (2, 2, 2, 2), 0, 18, 1, 'a"b\\c d') == "x|2x2x2x2|p0|r18|n1|a_b_c_d"


def test_file_round_trip(tuner, tmp_path):
    p = tmp_path / "sub" / "tune.json"
    tuner.insert("multi_dslash|32x32x32x16|p1|r12|n16|GPU", (8 << 8) | 2)
    tuner.insert("cg_hop|4x4x4x4|p0|r18|n1|GPU", 128)
    tuner.save(p)
    d = json.loads(p.read_text())             # a real JSON document
    assert d["format"] == "stag-tune-1"
    assert d["entries"]["cg_hop|4x4x4x4|p0|r18|n1|GPU"]["choice"] == 128
    tuner.clear()
    assert tuner.lookup("cg_hop|4x4x4x4|p0|r18|n1|GPU") is None
    assert tuner.load(p) == 2
    assert tuner.lookup("cg_hop|4x4x4x4|p0|r18|n1|GPU") == 128
    assert tuner.lookup("multi_dslash|32x32x32x16|p1|r12|n16|GPU") == (8 << 8) | 2
    assert tuner.stats() == {"timed": 0, "from_cache": 0}


def test_parser_tolerates_layout_and_keeps_candidates(tuner, tmp_path):
    p = tmp_path / "t.json"
    p.write_text('{"entries":{"a|1":{"ms":[0.5,0.25],"candidates":[64,128],"choice":128},\n'
                 '  "b|2" : { "choice" : -3 }},"format":"stag-tune-1"}')
    assert tuner.load(p) == 2
    assert tuner.lookup("a|1") == 128 and tuner.lookup("b|2") == -3


@pytest.mark.parametrize("text", ['{"format": "other", "entries": {}}', "not json", ""])
def test_foreign_files_are_refused(tuner, tmp_path, text):
    import paper_2502_03249_gb300 as stag
    p = tmp_path / "t.json"
    p.write_text(text)
    with pytest.raises(stag.StagError):
        tuner.load(p)
    with pytest.raises(stag.StagError):
        tuner.load(tmp_path / "missing.json")
