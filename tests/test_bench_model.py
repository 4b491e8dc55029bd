"""Host-side pieces of the benchmark's byte model: the fraction of (y, z) rows the stars' CIC
stencils touch (the density pass reads and clears the deposit only there), checked against a
brute-force enumeration of the stencil nodes, and the comment-insensitive source hash."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def brute_fraction(pos, shape, L=1.0):
    nz, ny, nx = shape
    rows = set()
    for p in pos:
        j0 = int(np.floor((p[1] + 0.5 * L) / L * ny)) % ny
        k0 = int(np.floor((p[2] + 0.5 * L) / L * nz)) % nz
        for dy in (0, 1):
            for dz in (0, 1):
                rows.add(((k0 + dz) % nz, (j0 + dy) % ny))
    return len(rows) / (ny * nz)


def test_deposit_row_fraction_matches_brute_force():
    rng = np.random.default_rng(5)
    for shape in ((8, 8, 8), (6, 12, 4), (16, 4, 8)):
        pos = rng.uniform(-0.5, 0.5, (40, 3))
        assert bench.deposit_row_fraction(pos, shape) == brute_fraction(pos, shape)


def test_deposit_row_fraction_special_cases():
    shape = (8, 8, 8)
    assert bench.deposit_row_fraction(np.zeros((0, 3)), shape) == 0.0
    # one star on a node: its stencil spans nodes (j0, j0 + 1) x (k0, k0 + 1), 4 of 64 rows
    assert bench.deposit_row_fraction(np.zeros((1, 3)), shape) == 4 / 64
    # the periodic wrap: a star in the last cell touches row 0 as well
    p = np.array([[0.0, 0.5 - 1e-3, 0.5 - 1e-3]])
    assert bench.deposit_row_fraction(p, shape) == 4 / 64
    # stars on every node touch every row
    g = (np.arange(8) + 0.5) / 8 - 0.5
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    assert bench.deposit_row_fraction(pos, shape) == 1.0


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2606_25026_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("int f() { return 1; }  // one\n/* block */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash()
    (csrc / "a.cu").write_text("// a comment\nint f() {   return 1; }\n")
    assert bench.source_hash() == h0
    (csrc / "a.cu").write_text("int f() { return 2; }\n")
    assert bench.source_hash() != h0
