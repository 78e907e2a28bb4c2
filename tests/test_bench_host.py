"""Host logic of bench.py that needs no GPU: the source fingerprint that
keys the recorded DRAM traffic of a kernel to the code it was measured on."""
import os

import bench


def test_comments_and_layout_do_not_change_the_tokens():
    src = open(os.path.join(bench.ROOT, "paper_2309_14311_gb300", "csrc", "grid_kernels.cu")).read()
    base = bench.source_tokens(src)
    assert "//" not in base.replace('"//', "")          # no comment survives (literals aside)
    moved = src.replace("\n", "\n   // a note\n", 5).replace("{", "{ /* inline */ ", 3)
    assert bench.source_tokens(moved) == base
    assert bench.source_tokens(src.replace("kK1Words = 3", "kK1Words = 4")) != base


def test_literals_are_kept():
    t = 'const char *s = "// not a comment /* nor this */"; char q = \'"\'; // gone\nint x;'
    assert bench.source_tokens(t) == 'const char *s = "// not a comment /* nor this */"; char q = \'"\'; int x;'


def test_recorded_traffic_is_current():
    """Every recorded capture belongs to the kernel as it is; after a change
    to a kernel its record is taken again or dropped."""
    for k in bench.NCU_TRAFFIC:
        assert bench.traffic_for(k) == bench.NCU_TRAFFIC[k]["bytes_per_launch"] > 0, k


def test_both_arms_name_the_same_workload():
    """The reference arm prints workload_config as it is and the GPU arm
    with its layout, which defaults to the agent layout: the two configs are
    equal at every world size, one replica road per rank."""
    spec = bench.WL.LARGE_ROAD
    for world in (1, 2, 8):
        ref = bench.workload_config(spec, world)
        assert dict(ref, layout="agent") == ref
        assert (ref["L"], ref["N"], ref["vmax"], ref["p"]) == (2**31, 2**27, 5, 0.13)
        assert len(ref["road_ids"]) == world and len(set(ref["road_ids"])) == world
        assert ref["parallelism"] == f"replicas{world}"
