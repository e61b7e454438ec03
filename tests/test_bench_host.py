"""Host logic of bench.py that needs no GPU: the key under which the ncu figures of the tile
kernels are carried into the roofline, and the algorithmic byte counts behind it."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
pytest.importorskip("torch")

import bench  # noqa: E402


def _tag_of(text, tmp_path, monkeypatch, common="__device__ int g(int x) { return x; }\n"):
    csrc = tmp_path / "paper_2506_20513_gb300" / "csrc"
    csrc.mkdir(parents=True, exist_ok=True)
    (csrc / "gf_tile_kernels.cu").write_text(text)
    (csrc / "gf_tile_common.cuh").write_text(common)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench.kernel_source_tag()


def test_code_tag_ignores_comments_and_blank_lines(tmp_path, monkeypatch):
    src = "// header\nint f(int x) {\n    return x + 1;  // add one\n}\n"
    base = _tag_of(src, tmp_path, monkeypatch)
    edited = "// a longer header\n// over two lines\n\nint f(int x) {\n\n    return x + 1;\n}\n"
    assert _tag_of(edited, tmp_path, monkeypatch) == base
    changed = "// header\nint f(int x) {\n    return x + 2;  // add one\n}\n"
    assert _tag_of(changed, tmp_path, monkeypatch) != base
    # the shared device code counts too
    other = "__device__ int g(int x) { return x + 1; }\n"
    assert _tag_of(src, tmp_path, monkeypatch, common=other) != base


def test_real_sources_have_a_tag():
    tag = bench.kernel_source_tag()
    assert len(tag) == 12 and int(tag, 16) >= 0


def test_algorithmic_bytes_per_cell_step():
    """Forward: fields read and written (24 B) and the model (8 B) once per launch, the history
    4 B per step; adjoint: state, gradient pair read and written (16 B) once per launch, the
    history K + 1 slots; strips add their CPML memories.  At K = 7 on the 540x290 workload:
    about 8.0 and 10.8 B per cell-step."""
    wl = bench.workload(0, nshots=32, nt=2000)
    cells = wl.nshots * wl.grid.ncells * 7
    fwd = bench.algorithmic_bytes_per_launch("fwd", wl, 7) / cells
    adj = bench.algorithmic_bytes_per_launch("adj", wl, 7) / cells
    assert 7.5 < fwd < 8.5
    assert 10.3 < adj < 11.3
    assert adj > fwd
    # a misfit-only forward stores no history: 4 B per step less
    nohist = bench.algorithmic_bytes_per_launch("fwd", wl, 7, 0.0) / cells
    assert fwd - nohist == pytest.approx(4.0)


def test_cpu_sample_is_bounded_by_shots_and_cores():
    n = bench.cpu_sample_shots(0, 32)
    assert 1 <= n <= min(32, bench.host_cores())
    assert bench.cpu_sample_shots(0, 2) <= 2
    assert bench.cpu_sample_shots(5, 3) == 3


def test_blocks_per_pass_counts_segment_ends():
    assert bench.blocks_per_pass(2000, 7, 0) == 286
    assert bench.blocks_per_pass(2000, 7, 100) == 20 * 15      # 100 = 14 x 7 + 2
    assert bench.blocks_per_pass(250, 7, 100) == 15 + 15 + 8   # segments 100, 100, 50
    assert bench.blocks_per_pass(8000, 7, 200) == 40 * 29


def test_kernel_roofline_counts_lane_launches():
    """Two lanes double the launches of a pass and halve the shots of each: the bytes per
    launch halve and the steps per launch stay K, so the same busy time per pass gives the
    same achieved bandwidth as one lane."""
    wl = bench.workload(0, nshots=32, nt=2000)
    clk = {"sm_mhz": 2070.0}
    one = {"fwd": (40.0, 286, 40.0), "adj": (50.0, 286, 50.0), "aux": (0.1, 5, 0.1)}
    two = {"fwd": (40.0, 572, 40.0), "adj": (50.0, 572, 50.0), "aux": (0.1, 6, 0.1)}
    r1 = bench.tile_roofline(one, wl, 1, 1.0, "x", clk, 152, 7, 0)
    r2 = bench.tile_roofline(two, wl, 1, 1.0, "x", clk, 152, 7, 0)
    assert r1["shot_lanes"] == 1 and r2["shot_lanes"] == 2
    assert r2["algorithmic_bytes_per_launch"] == pytest.approx(
        r1["algorithmic_bytes_per_launch"] / 2, rel=0.01)
    assert r2["achieved"] == pytest.approx(r1["achieved"], rel=0.01)
    assert r1["kernel"] == "adj_tile_kernel"


def test_path_roofline_adds_both_kernels():
    wl = bench.workload(0, nshots=32, nt=2000)
    r = bench.path_roofline(100.0, wl, 1, 7, 0)
    cells = wl.nshots * wl.grid.ncells * 2000
    # about 8.0 (forward) + 10.8 (adjoint) algorithmic bytes per cell-step
    assert 18.0 < r["algorithmic_bytes_per_step"] / cells < 19.6
    assert r["achieved"] == pytest.approx(r["algorithmic_bytes_per_step"] / 0.1 / 1e9)
