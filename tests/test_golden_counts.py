"""DOF counts the paper prints, reproduced by the voxel-boundary mesher (tests/golden)."""
import json
import os

import pytest

import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def test_printed_dof_counts():
    n = GOLD["cantilever_N"]
    V, T = W.cube_mesh(n)
    assert len(T) == GOLD["cube_triangles_per_N2"] * n * n
    surf = GOLD["source_dofs_per_triangle"] * len(T)
    vol = GOLD["volume_dofs_per_cell"] * n ** 3
    assert surf == pytest.approx(GOLD["cantilever_surface_dofs_printed"], rel=0.005)
    assert vol == pytest.approx(GOLD["cantilever_volume_dofs_printed"], rel=0.005)
    npc = GOLD["periodic_N"]
    assert GOLD["volume_dofs_per_cell"] * npc ** 3 == pytest.approx(GOLD["periodic_volume_dofs_printed"], rel=1e-12)
