"""The C-ABI library builds, loads without a GPU and exports every entry point
include/lh.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lh_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(lhlib):
    L = ctypes.CDLL(lhlib.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lhlib):
    bound = set(lhlib.EXPORTS) | {"lh_last_error", "lh_version"}
    assert set(declared_functions()) <= bound


def test_version_and_error_string_without_gpu(lhlib):
    L = lhlib.lib()
    assert b"sm_103a" in L.lh_version()
    assert L.lh_last_error(None) == b"null context"


def test_struct_sizes_match_header_layout(lhlib):
    # ctypes mirrors of the header structs; sizes follow natural alignment
    assert ctypes.sizeof(lhlib.Set) == 24
    assert ctypes.sizeof(lhlib.Edge) == 4 + 4 + 24 + 4 + 4 + 8 + 8 + 8
    assert ctypes.sizeof(lhlib.Group) == 16


def test_committed_dram_traffic_matches_the_kernel_source():
    """The DRAM traffic the bench reports for its dominant kernel comes from a
    committed ncu capture keyed by a hash of the kernel's source: the bench
    reports the captured bytes (scaled by rows when the capture ran a smaller
    case) while the source is unchanged, and null once it has changed."""
    import hashlib
    import json
    import bench
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        recs = json.load(f)
    assert recs
    for name, rec in recs.items():
        text = open(os.path.join(ROOT, "paper_1708_07859_b300", "csrc", rec["source"])).read()
        a = text.find(rec["begin"])
        b = text.find(rec["end"], a + 1)
        current = a >= 0 and b >= 0 and hashlib.sha256(text[a:b].encode()).hexdigest() == rec["source_sha256"]
        got = bench.dram_traffic(name, 2 * rec.get("rows", 1))
        if current:
            scale = 2 if rec.get("scales_with_rows") else 1
            assert got == scale * rec["bytes_per_launch"]
        else:
            assert got is None
        assert "--clock-control none" in rec["capture"]
