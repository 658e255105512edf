"""Pins of the oracle's brute-force neighbour pairs (CPU only).

The neighbour set is N(i) = {j != i : |r_ij|^2 < rc^2} (strict), r_ij the
minimum-image vector in a cubic periodic box (the 3.5 A / 5.0 A cutoffs of
the two models). Checked against an independent formulation: the minimum over
the 27 nearest periodic images by explicit loops.
"""
import itertools

import numpy as np
import pytest

from oracle import model as M


def _pairs_by_images(x, L, rc):
    """Pure-Python brute force: min over the 27 image shifts (small N only)."""
    n = len(x)
    out = set()
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            best = None
            for s in itertools.product((-1, 0, 1), repeat=3):
                dv = [x[j][k] + s[k] * L - x[i][k] for k in range(3)]
                d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]
                best = d2 if best is None else min(best, d2)
            if best < rc * rc:
                out.add((i, j))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pairs_match_image_brute_force(seed):
    rng = np.random.default_rng(seed)
    L, rc = 11.0, 3.5
    x = rng.uniform(0, L, size=(60, 3))
    i, j = M.pair_list(x, [0, 60], [L], rc)
    assert set(zip(i.tolist(), j.tolist())) == _pairs_by_images(x.tolist(), L, rc)
    # rows sorted by i then j, symmetric, no self pairs
    assert np.all(np.diff(i) >= 0)
    for a in range(60):
        row = j[i == a]
        assert np.all(np.diff(row) > 0)
    assert set(zip(i.tolist(), j.tolist())) == set(zip(j.tolist(), i.tolist()))


def test_exact_cutoff_distance_excluded():
    # distance exactly rc (representable): strict '<' excludes it
    x = np.array([[1.0, 1.0, 1.0], [6.0, 1.0, 1.0], [1.0, 4.5, 1.0], [1.0, 1.0, 5.999999]])
    i, j = M.pair_list(x, [0, 4], [0.0], 5.0)
    pairs = set(zip(i.tolist(), j.tolist()))
    assert (0, 1) not in pairs and (1, 0) not in pairs
    assert (0, 2) in pairs and (0, 3) in pairs
    # across the periodic boundary: 0.5 and 10.5 in a box of 15 are 5.0 apart
    xp = np.array([[0.5, 1.0, 1.0], [10.5, 1.0, 1.0], [10.49, 1.0, 1.0]])
    i, j = M.pair_list(xp, [0, 3], [15.0], 5.0)
    pairs = set(zip(i.tolist(), j.tolist()))
    assert (0, 1) not in pairs and (0, 2) not in pairs
    xp[2, 0] = 10.51
    i, j = M.pair_list(xp, [0, 3], [15.0], 5.0)
    assert (0, 2) in set(zip(i.tolist(), j.tolist()))


def test_systems_do_not_interact_and_small_box_rejected():
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, 0, 0], [1.5, 0, 0]])
    i, j = M.pair_list(x, [0, 2, 4], [0.0, 0.0], 5.0)
    assert set(zip(i.tolist(), j.tolist())) == {(0, 1), (1, 0), (2, 3), (3, 2)}
    with pytest.raises(ValueError):
        M.pair_list(x[:2], [0, 2], [9.9], 5.0)


def test_empty_and_single_atom():
    i, j = M.pair_list(np.zeros((1, 3)), [0, 1], [0.0], 5.0)
    assert len(i) == 0 and len(j) == 0


def test_pair_row_equals_rows_of_pair_list():
    rng = np.random.default_rng(4)
    L, rc = 12.0, 5.0
    x = rng.uniform(0, L, size=(80, 3))
    i, j = M.pair_list(x, [0, 80], [L], rc)
    for a in (0, 17, 79):
        np.testing.assert_array_equal(M.pair_row(x, a, [0, 80], [L], rc), j[i == a])
