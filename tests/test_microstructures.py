"""The seeded input generators (geometry only) against brute force and their
stated recipes: the workloads both the CUDA path and the oracle receive."""
import itertools
import math

import numpy as np
import pytest

from paper_1411_0330_gb300 import microstructures as ms


def _min_dist2(a, b):
    d = a - b
    d -= np.round(d)
    return np.sum(d * d, axis=-1)


def test_square_inclusion_is_the_centred_half_side_square():
    ph = ms.square_inclusion(32)
    inside = np.zeros((32, 32), np.uint8)
    inside[8:24, 8:24] = 1  # cells 8..23 x 8..23
    assert np.array_equal(ph, inside)


def test_laminate_varies_along_one_axis_with_the_given_widths():
    ph = ms.laminate((6, 10), 0, [(0, 3), (1, 2)])  # axis 0 = fastest (last array axis)
    assert np.array_equal(ph[0], [0, 0, 0, 1, 1, 0, 0, 0, 1, 1])
    assert (ph == ph[0][None, :]).all()


@pytest.mark.parametrize("seed", [1, 2])
def test_rsa_spheres_do_not_overlap_and_reach_the_count(seed):
    r, f = 0.08, 0.2
    cen = ms.rsa_spheres(r, f, seed)
    assert len(cen) == int(round(f / ms.sphere_volume(r)))
    for i, j in itertools.combinations(range(len(cen)), 2):
        assert _min_dist2(cen[i], cen[j]) >= (2 * r) ** 2 - 1e-15
    assert np.array_equal(cen, ms.rsa_spheres(r, f, seed))  # seeded


def test_hard_sphere_mc_keeps_every_pair_apart():
    r = 0.06
    count = int(round(0.35 / ms.sphere_volume(r)))
    cen = ms.hard_sphere_mc(r, count, seed=5, sweeps=5)
    assert cen.shape == (count, 3) and (cen >= 0).all() and (cen < 1).all()
    for i in range(count):
        d2 = _min_dist2(cen, cen[i])
        d2[i] = np.inf
        assert d2.min() >= (2 * r) ** 2 - 1e-15


def test_voxelize_is_the_centre_rule_with_periodic_images():
    rng = np.random.default_rng(9)
    n, r = 10, 0.17
    cen = rng.random((3, 3))
    cen[0] = [0.02, 0.97, 0.5]  # crosses the cell faces
    ph = ms.voxelize_spheres(n, cen, r)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    centres = np.stack([(x + 0.5) / n, (y + 0.5) / n, (z + 0.5) / n], axis=-1)
    brute = np.zeros((n, n, n), bool)
    for c in cen:
        brute |= _min_dist2(centres, c) <= r * r + 1e-15
    assert np.array_equal(ph.astype(bool), brute)


def test_sphere_fractions_average_the_centre_rule_of_a_finer_grid():
    cen = np.array([[0.3, 0.4, 0.55], [0.8, 0.1, 0.9]])
    r = 0.15
    f = ms.sphere_fractions(8, cen, r, sub=4)
    fine = ms.voxelize_spheres(32, cen, r)
    assert f.shape == (8, 8, 8) and f.min() >= 0 and f.max() <= 1
    assert math.isclose(float(f.mean()), float(fine.mean()), rel_tol=1e-6)
    assert math.isclose(float(f.mean()), 2 * ms.sphere_volume(r), rel_tol=0.1)


def test_benchmark_packing_recipe():
    """The 128^3 workload: RSA of radius-8-voxel spheres to f = 0.3 with seed 1411 gives
    293 spheres and a voxel fraction of 0.2997 (the numbers the bench line names)."""
    ph, cen, r = ms.sphere_microstructure(128, 8.0, 0.3, seed=1411)
    assert ph.shape == (128, 128, 128) and len(cen) == 293 and r == 8.0 / 128
    assert abs(float(ph.mean()) - 0.2997) < 5e-5
