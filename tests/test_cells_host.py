"""Host side of the 2D P2 cell-major order (no GPU).

The cell kernels hard-code which lattice points an interior row of each dof type
couples to (``PFC_CELL2D_ENTRIES`` in ``csrc/cell2d.h``).  These tests pin that table
against the oracle's own assembled P2 mass and stiffness matrices (Section 3), which
share no code with the library, and check the host builder's row classes."""
import os
import re

import numpy as np
import pytest

from oracle import assembly, mesh as omesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CELL_DX = [-1, 0, -1, 0, 1, 0, 1]
CELL_DY = [-1, -1, 0, 0, 0, 1, 1]


def _cell_entries():
    text = open(os.path.join(ROOT, "paper_1501_06852_gb300", "csrc", "cell2d.h")).read()
    body = text[text.index("#define PFC_CELL2D_ENTRIES"):]
    body = body[:body.index("// clang-format on")]
    ents = [tuple(int(v) for v in m) for m in re.findall(r"X\((\d+), (\d+), (\d+)\)", body)]
    dx = [int(v) for v in re.search(r"#define PFC_CELL2D_DX \{([^}]*)\}", text).group(1).split(",")]
    dy = [int(v) for v in re.search(r"#define PFC_CELL2D_DY \{([^}]*)\}", text).group(1).split(",")]
    return ents, dx, dy


def _lattice_offsets(ents, dx, dy):
    """{type: set of (ox, oy) lattice offsets} implied by the table."""
    out = {t: set() for t in range(4)}
    for t, q, sub in ents:
        tx, ty = t & 1, t >> 1
        sx, sy = 2 * dx[q] + (sub & 1), 2 * dy[q] + (sub >> 1)
        out[t].add((sx - tx, sy - ty))
    return out


def test_cell_table_shape():
    ents, dx, dy = _cell_entries()
    assert dx == CELL_DX and dy == CELL_DY
    assert len(ents) == 46
    # no coupling listed twice, every entry reads one of the seven source cells
    assert len(set(ents)) == len(ents)
    assert all(0 <= q < 7 and 0 <= t < 4 and 0 <= s < 4 for t, q, s in ents)
    counts = [sum(1 for e in ents if e[0] == t) for t in range(4)]
    assert counts == [19, 9, 9, 9]


@pytest.mark.parametrize("side", [4, 7])
def test_cell_table_matches_oracle_pattern(side):
    """Every interior row of the oracle's M and K couples exactly to the lattice
    offsets the table lists for its dof type (and M has no other nonzeros)."""
    ents, dx, dy = _cell_entries()
    table = _lattice_offsets(ents, dx, dy)
    m = omesh.structured_mesh(2, side, float(side))
    M = assembly.mass_matrix(m).tocsr()
    K = assembly.stiffness_matrix(m).tocsr()
    lat = 2 * side + 1
    checked = 0
    for y in range(2, lat - 2):
        for x in range(2, lat - 2):
            i = y * lat + x
            t = (x & 1) | ((y & 1) << 1)
            cols = M.indices[M.indptr[i]:M.indptr[i + 1]]
            offs = {(c % lat - x, c // lat - y) for c in cols}
            assert offs == table[t], (x, y, t)
            kcols = set(K.indices[K.indptr[i]:K.indptr[i + 1]])
            assert kcols <= set(cols)
            checked += 1
    assert checked == (lat - 4) ** 2


@pytest.mark.parametrize("side", [2, 3, 5, 32, 512])
def test_host_cells(side):
    from paper_1501_06852_gb300 import host_cells
    h = host_cells(side, float(side))
    assert h["rows"] == (2 * side + 1) ** 2
    assert h["pattern_ok"]
    # four interior stencils, the empty one, and the boundary stencils of a uniform
    # mesh, whose number does not grow with the mesh
    assert h["classes"] == host_cells(64, 64.0)["classes"]
    assert h["entries"] == host_cells(64, 64.0)["entries"]
    assert 5 < h["classes"] <= 255
    # cell classes: the interior cell and the cells along the sides and corners
    assert 1 < h["cell_classes"] <= 16


def test_host_cells_single_cell_mesh_keeps_cell_kernels_off():
    """side 1 has no interior row, so the extracted stencils are not the interior ones."""
    from paper_1501_06852_gb300 import host_cells
    h = host_cells(1, 1.0)
    assert h["rows"] == 9
    assert not h["pattern_ok"]


def test_host_cells_weights_translation_invariant():
    """Boundary classes: their count is that of the distinct (side, corner, type)
    stencils, the same at h = 1 and h = 0.5 (scaled weights, same structure)."""
    from paper_1501_06852_gb300 import host_cells
    a = host_cells(16, 16.0)
    b = host_cells(16, 8.0)
    assert a["classes"] == b["classes"] and a["entries"] == b["entries"]


# ---------------------------------------------------------------------------- 3D
def _cell3d_entries():
    text = open(os.path.join(ROOT, "paper_1501_06852_gb300", "csrc", "cell3d.h")).read()
    body = text[text.index("#define PFC_CELL3D_ENTRIES"):]
    body = body[:body.index("// clang-format on")]
    ents = [tuple(int(v) for v in m) for m in re.findall(r"X\((\d+), (\d+), (\d+)\)", body)]
    loads = [int(v) for v in re.findall(r"L\((\d+)\)", body)]
    d = {}
    for axis in "XYZ":
        d[axis] = [int(v) for v in re.search(rf"#define PFC_CELL3D_D{axis} \{{([^}}]*)\}}", text).group(1).split(",")]
    return ents, loads, d["X"], d["Y"], d["Z"]


def test_cell3d_table_shape():
    ents, loads, dx, dy, dz = _cell3d_entries()
    assert len(ents) == 230 and len(set(ents)) == 230
    # every source cell is loaded once, before its couplings, in order
    assert loads == list(range(15))
    assert [e[1] for e in ents] == sorted(e[1] for e in ents)
    # the fifteen cells whose offsets have no two components of opposite sign
    cells = list(zip(dx, dy, dz))
    assert len(set(cells)) == 15 and (0, 0, 0) in cells
    assert all(not (min(c) < 0 < max(c)) for c in cells)
    counts = [sum(1 for e in ents if e[0] == t) for t in range(8)]
    assert counts == [65, 27, 27, 19, 27, 19, 19, 27]


@pytest.mark.parametrize("side", [4, 5])
def test_cell3d_table_matches_oracle_pattern(side):
    """Every interior row of the oracle's 3D M couples exactly to the lattice offsets the
    table lists for its dof type (Kuhn tetrahedra, Section 7's 3D meshes)."""
    ents, _, dx, dy, dz = _cell3d_entries()
    table = {t: set() for t in range(8)}
    for t, q, sub in ents:
        tx, ty, tz = t & 1, (t >> 1) & 1, t >> 2
        sx = 2 * dx[q] + (sub & 1) - tx
        sy = 2 * dy[q] + ((sub >> 1) & 1) - ty
        sz = 2 * dz[q] + (sub >> 2) - tz
        table[t].add((sx, sy, sz))
    m = omesh.structured_mesh(3, side, float(side))
    M = assembly.mass_matrix(m).tocsr()
    K = assembly.stiffness_matrix(m).tocsr()
    lat = 2 * side + 1
    checked = 0
    for z in range(2, lat - 2):
        for y in range(2, lat - 2):
            for x in range(2, lat - 2):
                i = (z * lat + y) * lat + x
                t = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2)
                cols = M.indices[M.indptr[i]:M.indptr[i + 1]]
                offs = {(c % lat - x, (c // lat) % lat - y, c // (lat * lat) - z) for c in cols}
                assert offs == table[t], (x, y, z, t)
                assert set(K.indices[K.indptr[i]:K.indptr[i + 1]]) <= set(cols)
                checked += 1
    assert checked == (lat - 4) ** 3


@pytest.mark.parametrize("side", [2, 3, 16, 64])
def test_host_cells_3d(side):
    from paper_1501_06852_gb300 import host_cells
    h = host_cells(side, float(side), dim=3)
    assert h["rows"] == (2 * side + 1) ** 3
    assert h["pattern_ok"]
    ref = host_cells(16, 16.0, dim=3)
    assert h["classes"] == ref["classes"] and h["entries"] == ref["entries"]
    assert 9 < h["classes"] <= 255
    assert 1 < h["cell_classes"] <= 64
