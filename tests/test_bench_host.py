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
