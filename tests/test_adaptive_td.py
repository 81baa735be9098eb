"""Two-scale sampling of the topological derivative (Sec. "Discussion and future work": a
coarse grid, refined where the threshold function differs between neighbouring cells and on
the material's boundary), on synthetic D^T fields: the voxels the hard-kill update removes
(D^T below D_C = D_min + C (D_max - D_min)) are the same as with D^T at every voxel, with fewer
evaluations (the saving grows with the ratio of volume to surface voxels, as the paper notes:
here 48 x 24 x 24 voxels)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def field(p):
    """A smooth D^T-like field on [0,2]x[0,1]^2: large at the clamped face and the load,
    smallest in a band away from them, plus a ridge along the cantilever's neutral plane."""
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return (np.exp(-3 * x) * 4 + 2 * np.exp(-((x - 2) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / 0.02)
            + 0.4 * (z - 0.5) ** 2 + 0.05 * np.sin(7 * y) + 0.02 * x)


@pytest.mark.parametrize("C,holes,frac", [(0.02, 0, 0.7), (0.05, 40, 0.8), (0.1, 120, 0.9), (0.02, 300, 0.8)])
def test_adaptive_removal_set_matches_full(C, holes, frac):
    from paper_1612_04082_gb300.driver import adaptive_td
    n = 24
    h = 1.0 / n
    mask = np.ones((2 * n, n, n), np.uint8)
    rng = np.random.default_rng(holes)
    for _ in range(holes):  # voids of one voxel, as earlier iterations leave them
        i, j, k = rng.integers(1, 2 * n - 1), rng.integers(1, n - 1), rng.integers(1, n - 1)
        mask[i, j, k] = 0
    calls = []

    def evaluate(pts):
        calls.append(len(pts))
        return field(pts.astype(np.float64)).astype(np.float32)

    ii = np.argwhere(mask > 0)
    full = np.zeros(mask.shape, np.float32)
    full[tuple(ii.T)] = field(((ii + 0.5) * h).astype(np.float32).astype(np.float64)).astype(np.float32)
    td, exact, nev = adaptive_td(mask, h, evaluate, C)
    assert nev == sum(calls) and len(calls) <= 2
    v_full, v_ad = full[tuple(ii.T)], td[tuple(ii.T)]
    dc_full = v_full.min() + C * (v_full.max() - v_full.min())
    dc_ad = v_ad.min() + C * (v_ad.max() - v_ad.min())
    removed_full = set(map(tuple, ii[v_full < dc_full]))
    removed_ad = set(map(tuple, ii[v_ad < dc_ad]))
    assert removed_full == removed_ad
    assert np.all(td[exact] == full[exact])      # evaluated values are exact
    assert nev < frac * len(ii), (nev, len(ii))  # fewer evaluations than one per voxel
