"""CPU checks of the autotuner's table file (no GPU: kohler_tune_save, _load,
_clear and _count never touch the device).  A file written by tune_save reads
back to the same entries; a file that does not parse, or holds an entry that is
not valid for its pass (a route that is not one of the pass's alternatives, a
block size or pixel count the uint16 pass does not have), is refused whole and
leaves the table unchanged."""
import ctypes
import json
import os
import shutil

import pytest


@pytest.fixture()
def L():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1707_05062_gb300 import build

    lib = ctypes.CDLL(build.build())
    for name in ("kohler_tune_save", "kohler_tune_load"):
        getattr(lib, name).argtypes = [ctypes.c_char_p]
        getattr(lib, name).restype = ctypes.c_int
    lib.kohler_tune_clear.restype = ctypes.c_int
    lib.kohler_tune_count.restype = ctypes.c_int32
    assert lib.kohler_tune_clear() == 0
    yield lib
    lib.kohler_tune_clear()


def entry(**kw):
    e = {"pass": "u16_fast", "M": 4096, "px_class": 26, "route": "u16_fast", "warps": 16, "px": 8, "per_sm": 1,
         "upw": 64, "us": 12.5}
    e.update(kw)
    return e


def write(tmp_path, entries, name="t.json", head=None):
    path = tmp_path / name
    doc = head if head is not None else {"kohler_tune": 1, "entries": entries}
    path.write_text(json.dumps(doc))
    return str(path).encode()


def test_round_trip(L, tmp_path):
    entries = [entry(), entry(px_class=20, route="u16_generic", warps=8, px=4, per_sm=0, upw=16),
               entry(**{"pass": "u8_strip", "M": 256, "px_class": 24, "route": "u8_row", "warps": 8, "px": 4,
                        "per_sm": 0, "upw": 1}),
               entry(**{"pass": "u8_generic_n8", "M": 256, "px_class": 16, "route": "u8_generic_n8", "warps": 8,
                        "px": 4, "per_sm": 1, "upw": 4})]
    assert L.kohler_tune_load(write(tmp_path, entries)) == 0
    assert L.kohler_tune_count() == 4
    out = str(tmp_path / "saved.json").encode()
    assert L.kohler_tune_save(out) == 0
    saved = json.loads(open(out).read())
    assert saved["kohler_tune"] == 1
    key = lambda e: (e["pass"], e["M"], e["px_class"])
    got = sorted(saved["entries"], key=key)
    want = sorted(entries, key=key)
    assert [{k: v for k, v in e.items()} for e in got] == want
    # reading the saved file again replaces entries of the same kind, adds none
    assert L.kohler_tune_load(out) == 0 and L.kohler_tune_count() == 4
    assert L.kohler_tune_clear() == 0 and L.kohler_tune_count() == 0


def test_empty_and_missing_files(L, tmp_path):
    assert L.kohler_tune_load(write(tmp_path, [])) == 0 and L.kohler_tune_count() == 0
    assert L.kohler_tune_load(str(tmp_path / "absent.json").encode()) == -1
    assert L.kohler_tune_load(None) == -1 and L.kohler_tune_save(None) == -1
    assert L.kohler_tune_save(str(tmp_path / "no_dir" / "x.json").encode()) == -1


@pytest.mark.parametrize("bad", [
    entry(route="u8_row"),                      # not an alternative of the uint16 pass
    entry(warps=5),                             # no such block size
    entry(px=6),                                # no such pixel count
    entry(per_sm=-1),
    entry(upw=0),
    entry(M=1),
    entry(**{"pass": "u8_generic", "route": "u8_strip"}),  # the strip pass needs 16-byte rows
    entry(**{"pass": "u8_generic_n8", "route": "u8_generic"}),  # another neighbourhood
    entry(**{"pass": "no_such_pass"}),
])
def test_invalid_entries_refuse_the_whole_file(L, tmp_path, bad):
    assert L.kohler_tune_load(write(tmp_path, [entry(px_class=3)])) == 0
    assert L.kohler_tune_load(write(tmp_path, [entry(px_class=4), bad], name="bad.json")) == -1
    assert L.kohler_tune_count() == 1


@pytest.mark.parametrize("text", ["", "{}", "[1, 2]", '{"kohler_tune": 2, "entries": []}',
                                  '{"kohler_tune": 1, "entries": [{"pass": "u16_fast"', "not json at all",
                                  '{"kohler_tune": 1, "entries": [{"pass": "u16_fast", "M": }]}'])
def test_malformed_files(L, tmp_path, text):
    path = tmp_path / "m.json"
    path.write_text(text)
    assert L.kohler_tune_load(str(path).encode()) == -1
    assert L.kohler_tune_count() == 0
