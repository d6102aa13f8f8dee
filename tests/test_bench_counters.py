"""bench.py's stored ncu counters of the fused kernel belong to the capture that
profiles/ summarises: the same kernel-source hash and the same counts."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counters_match_the_profile_summary():
    sys.path.insert(0, ROOT)
    import bench
    text = open(os.path.join(ROOT, "profiles", "k_fused_step_channel_4096x512.md")).read()
    assert f"`{bench.FUSED_COUNTERS_SOURCE}`" in text
    m = re.search(r"dram__bytes_write\.sum \| ([\d.]+) \+ ([\d.]+) = ", text)
    assert m, "DRAM line missing from the summary"
    mb = float(m.group(1)) + float(m.group(2))
    assert abs(bench.FUSED_F32_4096x512_DRAM_BYTES / 1e6 - mb) < 0.011
    m = re.search(r"warp instructions executed \| ([\d.]+) M", text)
    assert m and abs(bench.FUSED_F32_4096x512_WARP_INSTR / 1e6 - float(m.group(1))) < 0.006


def test_source_hash_covers_existing_files():
    sys.path.insert(0, ROOT)
    import bench
    for rel in bench.FUSED_SOURCES:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    assert len(bench.fused_source_hash()) == 16
