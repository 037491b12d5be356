"""Host logic of bench.py that needs no GPU: the hub-count factorisation for
hierarchical balanced k-means, the kernel-source digest's insensitivity to
comments and prototypes, and the mode names."""
import os
import re
import shutil

import pytest

import bench


def test_hbkm_shape():
    assert bench.hbkm_shape(1024) == (32, 2)
    assert bench.hbkm_shape(4096) == (16, 3)
    assert bench.hbkm_shape(16384) == (4, 7)
    assert bench.hbkm_shape(27) == (27, 1)
    for H in (1024, 4096, 16384, 27, 512):
        k, levels = bench.hbkm_shape(H)
        assert k ** levels == H and 2 <= k <= 32
    assert bench.hbkm_shape(1000) == (10, 3)
    with pytest.raises(SystemExit):
        bench.hbkm_shape(1001)  # 7 * 11 * 13: no power of one branching factor


def test_kernel_digest_ignores_comments_and_prototypes(tmp_path, monkeypatch):
    root = tmp_path / "r"
    for rel in ("paper_2506_15986_gb300/csrc", "include"):
        (root / rel).mkdir(parents=True)
    for rel in ("paper_2506_15986_gb300/csrc/search.cu", "paper_2506_15986_gb300/csrc/device_util.cuh",
                "paper_2506_15986_gb300/csrc/internal.h", "include/ann.h"):
        shutil.copy(os.path.join(bench.ROOT, rel), root / rel)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.kernel_digest()
    hdr = root / "include/ann.h"
    text = hdr.read_text()
    hdr.write_text(text.replace("#endif", "/* a note */\nann_status ann_new_call(ann_index *idx, int32_t x);\n#endif", 1))
    assert bench.kernel_digest() == d0  # a comment and a new prototype
    hdr.write_text(re.sub(r"#define ANN_MAX_L \d+", "#define ANN_MAX_L 12345", text))
    assert bench.kernel_digest() != d0  # a constant the kernel compiles against
    hdr.write_text(text)
    cu = root / "paper_2506_15986_gb300/csrc/search.cu"
    cu.write_text(cu.read_text() + "\n// trailing note\n")
    assert bench.kernel_digest() == d0


def test_mode_names():
    class A:
        ENTRY_MEDOID, ENTRY_LEARNED_NAV, ENTRY_LEARNED_EXHAUSTIVE = 0, 1, 2
    assert bench.mode_info(A, "medoid") == (0, 1)
    assert bench.mode_info(A, "learned") == (1, 1)
    assert bench.mode_info(A, "exhaustive_s8") == (2, 8)


def test_batch10m_spec(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py", "--workload", "batch10m"])
    args = bench.parse()
    spec = args.spec
    assert spec["n"] == 10_000_000 and spec["dim"] == 96 and spec["nq"] == 100_000
    assert spec["insert"] == (1_000_000, 1_000_000) and spec["gt_rows"] == 5_000
    assert spec["batching"] and spec["hubs"] == 16384


def test_capture_and_knob_options(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py", "--capture", "--fixed-L", "93", "--knobs=-1,8,4,12,0,1,1",
                                     "--modes", "exhaustive"])
    args = bench.parse()
    assert args.capture and args.knobs == "-1,8,4,12,0,1,1" and args.spec["fixed_L"] == 93
    # the stored headline traffic names every speed knob the bench matches on
    for mt in bench.MEASURED_TRAFFIC["shift"]:
        for key in ("digest", "entry", "L", "nq", "hash_bits", "stage_rows", "team", "spill_bits", "gather",
                    "visited_l2", "group_entries", "bytes"):
            assert key in mt, key


def test_hub_graph_options(monkeypatch):
    # the hub-graph mode's defaults: the undirected s = 8 graph capped at 16
    # neighbours, a pool of 32, no start sample
    monkeypatch.setattr("sys.argv", ["bench.py"])
    args = bench.parse()
    assert args.hub_graph == "8:16" and args.l_hub == 32 and args.hub_seeds == 0 and args.nav_sweep == ""
    monkeypatch.setattr("sys.argv", ["bench.py", "--hub-graph", "16:0", "--l-hub", "16", "--hub-seeds", "32",
                                     "--nav-sweep", "16:0:16:32,32:32"])
    args = bench.parse()
    assert args.hub_graph == "16:0" and args.l_hub == 16 and args.hub_seeds == 32
    assert [item.split(":") for item in args.nav_sweep.split(",")] == [["16", "0", "16", "32"], ["32", "32"]]
