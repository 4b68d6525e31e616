"""Host helpers of bench.py without a GPU: extraction of a function's source
text, the source hash that ties a recorded ncu traffic figure to the kernel
it was measured on, and the lookup that drops a figure taken on other
sources, another sweep layout or another precision."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SRC = """#include <x>
// k_demo( in a comment before the definition is not the definition
int other(int a) { return a; }

template <class T, int G>
__global__ void __launch_bounds__(256) k_demo(T* x, int n) {
  if (n > 0) {
    for (int i = 0; i < n; ++i) { x[i] = T(G); }
  }
}

void tail() {}
"""


def test_definition_extracts_the_whole_body(tmp_path):
    f = tmp_path / "demo.cuh"
    f.write_text(SRC)
    d = bench._definition(str(f), "k_demo")
    assert d.startswith("template <class T, int G>")
    assert d.endswith("x[i] = T(G); }\n  }\n}")
    assert "tail" not in d and "other" not in d
    assert bench._definition(str(f), "missing") == ""
    assert bench._definition(str(f), "other") == "int other(int a) { return a; }"


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and profiles under a temporary root."""
    csrc = tmp_path / "paper_1309_5048_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fname in {f for srcs in bench.TRAFFIC_SOURCES.values() for f, _ in srcs}:
        shutil.copy(os.path.join(ROOT, "paper_1309_5048_gb300", "csrc", fname), csrc / fname)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _record(tree, **entry):
    e = {"dram_bytes_per_launch": 123456, "src_hash": bench.source_hash("ic0_apply", "packed32"), "trsv": "packed32",
         "precision": "fp64"}
    e.update(entry)
    (tree / "profiles" / "traffic.json").write_text(json.dumps({"2d256": {"ic0_apply": e}}))


def test_source_hash_follows_the_kernel_text(tree):
    h0 = bench.source_hash("ic0_apply", "packed32")
    assert h0 == bench.source_hash("ic0_apply", "packed12") and len(h0) == 16
    hs = bench.source_hash("ic0_apply", "split32")
    assert hs != h0  # each layout family hashes its own kernel
    assert bench.source_hash("ic0_apply", "csr") is None and bench.source_hash("cg_spmv", "packed32") is None
    fname, func = bench.TRAFFIC_SOURCES[("ic0_apply", "packed")][0]
    path = tree / "paper_1309_5048_gb300" / "csrc" / fname
    text = path.read_text()
    # an edit outside the recorded functions keeps the hash
    path.write_text(text + "\n// trailing comment\n")
    assert bench.source_hash("ic0_apply", "packed32") == h0
    # an edit inside one changes it, and only for the layout that uses it
    i = text.index(" " + func + "(")
    j = text.index("{", i)
    path.write_text(text[: j + 1] + "\n  int unused_marker = 0;" + text[j + 1:])
    assert bench.source_hash("ic0_apply", "packed32") != h0
    assert bench.source_hash("ic0_apply", "split32") == hs


def test_traffic_lookup_matches_sources_layout_and_precision(tree):
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "fp64") is None  # no record yet
    _record(tree)
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "fp64") == 123456
    assert bench.traffic_for("ic0_apply", "2d256", "split32", "fp64") is None
    assert bench.traffic_for("ic0_apply", "2d256", None, "fp64") is None
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "mixed") is None
    assert bench.traffic_for("ic0_apply", "3d32", "packed32", "fp64") is None
    assert bench.traffic_for("cg_spmv", "2d256", "packed32", "fp64") is None
    _record(tree, src_hash="0000000000000000")
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "fp64") is None
    (tree / "profiles" / "traffic.json").write_text("not json")
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "fp64") is None


def test_a_record_may_name_several_layouts_of_one_kernel(tree):
    """The light SELL-W sweep on a grid covering every slice group and on a
    grid of the resident blocks reads the same data; one record serves both
    names, and only those."""
    h = bench.source_hash("ic0_apply", "sellwl")
    assert h == bench.source_hash("ic0_apply", "sellwlr")
    _record(tree, src_hash=h, trsv=["sellwl", "sellwlr"])
    assert bench.traffic_for("ic0_apply", "2d256", "sellwl", "fp64") == 123456
    assert bench.traffic_for("ic0_apply", "2d256", "sellwlr", "fp64") == 123456
    assert bench.traffic_for("ic0_apply", "2d256", "sellwl8", "fp64") is None
    assert bench.traffic_for("ic0_apply", "2d256", "packed32", "fp64") is None
