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


@pytest.mark.parametrize("a,b", [(40.0, 40.0), (60.0, 30.0), (25.0, 50.0)])
def test_spheroid_surface_geometry(S, a, b):
    """The BEM surface recipe: points on the spheroid, unit outward normals along the
    gradient of the implicit surface, areas summing to the exact spheroid area, and the
    mean curvature 1/R on a sphere and half the divergence of the unit normal field
    everywhere."""
    n = 4000
    s = S.spheroid_surface(n, a, b)
    x, y, z = s["xyz"].T
    assert np.abs((x * x + y * y) / b ** 2 + z * z / a ** 2 - 1.0).max() < 1e-12
    nrm = s["normal"]
    assert np.abs(np.linalg.norm(nrm, axis=1) - 1.0).max() < 1e-12
    grad = np.stack([x / b ** 2, y / b ** 2, z / a ** 2], axis=1)
    grad /= np.linalg.norm(grad, axis=1)[:, None]
    assert np.abs(nrm - grad).max() < 1e-12
    if a == b:
        exact = 4.0 * np.pi * a * a
    elif a > b:      # prolate
        e = np.sqrt(1.0 - b * b / (a * a))
        exact = 2.0 * np.pi * b * b * (1.0 + a / (b * e) * np.arcsin(e))
    else:            # oblate
        e = np.sqrt(1.0 - a * a / (b * b))
        exact = 2.0 * np.pi * b * b * (1.0 + (1.0 - e * e) / e * np.arctanh(e))
    assert abs(s["area"].sum() / exact - 1.0) < 1e-5
    assert np.all(s["area"] > 0)
    H = s["curvature"]
    if a == b:
        assert np.abs(H - 1.0 / a).max() < 1e-12
    # mean curvature = half the divergence of the unit normal field grad F / |grad F| of the
    # implicit surface F = (x^2 + y^2) / b^2 + z^2 / a^2, by central differences
    def unit_grad(p):
        g = np.stack([p[:, 0] / b ** 2, p[:, 1] / b ** 2, p[:, 2] / a ** 2], axis=1)
        return g / np.linalg.norm(g, axis=1)[:, None]
    h = 1e-4 * min(a, b)
    div = np.zeros(n)
    for k in range(3):
        dp = np.zeros(3)
        dp[k] = h
        div += (unit_grad(s["xyz"] + dp)[:, k] - unit_grad(s["xyz"] - dp)[:, k]) / (2.0 * h)
    assert np.abs(H / (0.5 * div) - 1.0).max() < 1e-6
    # the same call gives the same mesh (no seed: the lattice is deterministic)
    assert np.array_equal(S.spheroid_surface(n, a, b)["xyz"], s["xyz"])


def test_drude_metal_resonance_in_band(S):
    m = S.drude_metal_params()
    wl = S.workload("bem_spheroid30k")
    # sphere dipole resonance eps_in = -2: w = wp / sqrt(eps_inf + 2 eps_out) = 3.41 eV
    w_f = m["omega_p"] / np.sqrt(m["eps_inf"] + 2.0 * m["eps_out"]) * S.HARTREE_EV
    assert abs(w_f - 3.406) < 1e-3
    assert wl["omega"][0] < S.ev(w_f) < wl["omega"][-1]
    assert len(wl["omega"]) == 64 and wl["surface"]["xyz"].shape == (30000, 3)
