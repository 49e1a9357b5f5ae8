"""The seeded input recipe: every workload is what its description states
(counts, radii, non-overlap under the periodic distance, pattern shapes,
contrast ranges, volume fractions) and is reproducible from its seed."""
import math

import numpy as np
import pytest

import workloads as W


def _no_overlap(c, r):
    for i in range(len(r)):
        for j in range(i):
            assert np.linalg.norm(W.periodic_delta(c[i], c[j])) > r[i] + r[j]


def test_dlvp_sheared_recipe():
    w = W.dlvp_sheared()
    assert w["M"] == [[128, 32], [0, 128]] and w["generator"] == {"kind": "dlvp", "alpha": [0.25, 0.25]}
    c, r = w["centres"], w["radii"]
    assert c.shape == (20, 2) and np.all((r >= 0.03) & (r <= 0.08))
    assert np.all((c >= -0.5) & (c < 0.5))
    _no_overlap(c, r)
    assert w["phases"][1][0] / w["phases"][0][0] == 100.0
    w2 = W.dlvp_sheared()
    assert np.array_equal(w2["centres"], c) and np.array_equal(w2["radii"], r)


def test_box3d_recipe_and_realised_fraction():
    w = W.box3d()
    c, r = w["centres"], w["radii"]
    assert c.shape == (50, 3) and np.all((r >= 0.05) & (r <= 0.1))
    _no_overlap(c, r)
    vf = 4.0 / 3.0 * math.pi * np.sum(r ** 3)
    assert 0.07 < vf < 0.13          # the stated count and radii give about 0.10, not 0.25


@pytest.mark.parametrize("i", [0, 1, 2, 3, 101, 510, 511])
def test_batch2d_item_recipe(i):
    w = W.batch2d_item(i)
    M = w["M"]
    N = M[0][0]
    assert N in (64, 96, 128, 192, 256) and M[1][1] == N and M[1][0] == 0
    if i % 2 == 0:
        assert M[0][1] == 0
    else:
        assert M[0][1] in (N // 8, N // 4, N // 2)
    c, r = w["centres"], w["radii"]
    assert 5 <= len(r) <= 30 and np.all((r >= 0.03) & (r <= 0.1))
    _no_overlap(c, r)
    assert 5.0 <= w["phases"][1][0] <= 200.0


@pytest.mark.parametrize("seed", [0, 7, 100000])
def test_fno3d_item_recipe(seed):
    w = W.fno3d_item(seed, n=16)
    c, r = w["centres"], w["radii"]
    assert np.all((r >= 0.06) & (r <= 0.12))
    _no_overlap(c, r)
    vf = 4.0 / 3.0 * math.pi * np.sum(r ** 3)
    assert 0.1 <= vf <= 0.35 + 4.0 / 3.0 * math.pi * 0.12 ** 3   # stops at the first ball past the target
    assert 10.0 <= w["phases"][1][0] <= 100.0


def test_phase_ids_use_the_periodic_distance():
    """A ball centred near a corner wraps around the cell; the boundary is strict."""
    c = np.array([[0.4375, 0.4375]])                       # binary fractions: exact distances
    pts = np.array([[-0.46875, 0.4375], [0.0, 0.0], [0.3125, 0.4375], [0.4375, -0.4375]])
    ids = W.phase_ids(pts, c, np.array([0.125]))
    assert ids.tolist() == [1, 0, 0, 0]                     # wrapped inside; at distance r: outside
    assert ids.dtype == np.uint8


def test_laminate_ids():
    y = np.array([[0.0, -0.2], [0.0, 0.19], [0.0, 0.2], [0.3, 0.0]])
    assert W.laminate_ids(y, 1, 0.4).tolist() == [1, 1, 0, 1]
