"""CPU checks of the seeded input recipes the benchmark and the serving stream use: the
same seed gives the same inputs, sizes and bands are the stated ones, and the structure
families have the geometric properties the recipes claim."""
import numpy as np
import pytest


def test_serving_mix_is_seeded_and_in_range(S):
    a = S.serving_mix(300)
    b = S.serving_mix(300)
    assert len(a["requests"]) == 300 and len(a["gaps"]) == 300
    assert np.array_equal(a["gaps"], b["gaps"])
    for (si, om, d), (sj, om2, d2) in zip(a["requests"], b["requests"]):
        assert si == sj and np.array_equal(om, om2) and np.array_equal(d, d2)
    sizes = [len(p["xyz"]) for p in a["pool"]]
    assert min(sizes) >= 1000 and max(sizes) <= 21000
    for si, om, d in a["requests"]:
        lo, hi = a["pool"][si]["band"]
        assert 1 <= len(om) <= 64 and 1 <= len(d) <= 3
        assert np.all(np.diff(om) >= 0)
        assert np.all(om >= S.ev(lo) - 1e-15) and np.all(om <= S.ev(hi) + 1e-15)
        assert np.array_equal(d, np.eye(3)[:len(d)])
    assert np.all(a["gaps"] > 0) and abs(np.mean(S.serving_mix(2000)["gaps"]) - 1.0) < 0.1


def test_sphere_jitter_moves_only_surface_atoms(S):
    a = 4.23
    R = S.fcc_sphere_radius_for(2000, a)
    plain = S.fcc_sphere(a, R)
    jit = S.fcc_sphere(a, R, 0.05, seed=20210301)
    assert plain.shape == jit.shape
    moved = np.any(plain != jit, axis=1)
    assert 0 < moved.sum() < len(plain)
    # displacements within the U(-0.05, 0.05) Angstrom box
    assert np.abs(jit - plain).max() <= 0.05 * S.BOHR_PER_ANGSTROM + 1e-12
    # interior atoms (12 neighbours at a / sqrt(2)) stay on the lattice
    r = np.linalg.norm(plain, axis=1) / S.BOHR_PER_ANGSTROM
    assert not np.any(moved[r < R - 2 * a])


@pytest.mark.parametrize("n_rings", [3, 13])
def test_flake_counts_and_bond_length(S, n_rings):
    xyz = S.honeycomb_flake(n_rings)
    assert len(xyz) == 6 * n_rings ** 2
    from scipy.spatial import cKDTree
    dmin = cKDTree(xyz).query(xyz, k=2)[0][:, 1].min() / S.BOHR_PER_ANGSTROM
    assert abs(dmin - 1.42) < 1e-9
