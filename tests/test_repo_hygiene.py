"""Repository rules checked on the CPU: every ncu command in the committed
profile summaries leaves the GPU clocks alone, every profile named in the
design notes exists, and no source names the batched memory-copy entry
points (the library issues one copy per buffer instead)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_every_ncu_command_keeps_clock_control_off():
    seen = 0
    for fn in sorted(os.listdir(PROFILES)):
        text = open(os.path.join(PROFILES, fn)).read()
        for line in text.splitlines():
            if re.search(r"\bncu\b", line) and ("--set" in line or "--metrics" in line):
                seen += 1
                assert "--clock-control none" in line, (fn, line)
    assert seen >= 10


def test_profiles_named_in_the_design_notes_exist():
    text = open(os.path.join(ROOT, "DESIGN.md")).read()
    names = set(re.findall(r"`(?:profiles/)?([A-Za-z0-9_]+\.md)`", text))
    names = {n for n in names if n not in ("DESIGN.md", "README.md")}
    assert names, "no profile references found"
    missing = sorted(n for n in names if not os.path.exists(os.path.join(PROFILES, n)))
    assert not missing, missing


def test_no_source_names_the_batched_copy_calls():
    closed = ["cudaMemcpy" + "BatchAsync", "cudaMemcpy3D" + "BatchAsync", "cuMemcpy" + "BatchAsync",
              "cuMemcpy3D" + "BatchAsync"]
    hits = []
    for base in ("paper_1708_07859_b300", "include", "oracle", "tests"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, base)):
            for fn in files:
                if fn.endswith((".cu", ".cuh", ".h", ".c", ".py", ".cpp")):
                    text = open(os.path.join(dirpath, fn), errors="replace").read()
                    hits += [(fn, c) for c in closed if c in text]
    for fn in ("bench.py", "__graft_entry__.py"):
        text = open(os.path.join(ROOT, fn)).read()
        hits += [(fn, c) for c in closed if c in text]
    assert not hits, hits
