"""Pins of the FMM oracle (oracle/fmm.py: the far-field-compressed D product that the
paper's conclusions point to for systems beyond a million atoms) against the exact
product of Eq. 3, not against the FMM itself: a structure whose tree has no far field
gives the exact product; the error falls geometrically with the interpolation order p
on a flat flake (quadtree) and a nanotube (octree); the approximate operator is exactly
symmetric, as D is; and copies of the oracle with a planted mistake (an interaction list
that double counts, nodes that are not Chebyshev nodes, an untransposed L2L) miss the
convergence pin by orders of magnitude.  CPU only."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fmm():
    from oracle import fmm
    return fmm


def _case(S, name):
    if name == "flake":
        return S.honeycomb_flake(18), 0.6            # 1944 atoms, planar: quadtree of depth 3
    return S.nanotube(5, 5, 50), 0.6                 # 1000 atoms, 3D: octree of depth 4


def _err(orc, fmm_mod, xyz, eta, p, x):
    """max_i |u_i - (D x)_i| / (|D| |x|)_i of the FMM product against the exact one."""
    D = orc.d_matrix(xyz, eta)
    u = fmm_mod.d_apply(xyz, eta, x, p)
    return float(np.max(np.abs(u - D @ x) / (np.abs(D) @ np.abs(x))))


def test_no_far_field_is_exact(orc, fmm, S):
    xyz = S.random_cluster(1500, seed=3)            # too compact for a tree of depth 2
    assert fmm.build_tree(xyz, 0.6)["depth"] < 2
    x = np.random.default_rng(5).standard_normal((1500, 2))
    assert _err(orc, fmm, xyz, 0.6, 4, x) <= 1e-13


def test_tree_leaves_hold_only_exact_coulomb_pairs(fmm, S):
    # every far pair is at least one leaf side apart, and the leaf side is >= 6 max s_ij,
    # where erf(r / s_ij) = 1 in FP64
    from scipy.special import erf
    for name in ("flake", "tube"):
        xyz, eta = _case(S, name)
        t = fmm.build_tree(xyz, eta)
        assert t["depth"] >= 3 and t["h"] >= t["r_far"]
        assert erf(t["r_far"] / (t["r_far"] / 6.0)) == 1.0
        assert t["dim"] == (2 if name == "flake" else 3)


@pytest.mark.parametrize("name,orders,last", [("flake", (3, 4, 6, 8), 2e-7), ("tube", (3, 4, 6), 1e-5)])
def test_error_falls_geometrically_with_order(orc, fmm, S, name, orders, last):
    xyz, eta = _case(S, name)
    x = np.random.default_rng(11).standard_normal((len(xyz), 2))
    errs = [_err(orc, fmm, xyz, eta, p, x) for p in orders]
    for (p0, e0), (p1, e1) in zip(zip(orders, errs), zip(orders[1:], errs[1:])):
        assert e1 < e0 * 0.35 ** (p1 - p0), (name, orders, errs)
    assert errs[-1] <= last, (name, errs)


@pytest.mark.parametrize("name", ["flake", "tube"])
def test_fmm_operator_is_symmetric(fmm, S, name):
    # P2M and L2P are transposes and 1/|t - s| is symmetric: x^T (F y) = y^T (F x) for the
    # approximate operator F itself, to rounding
    xyz, eta = _case(S, name)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(len(xyz)), rng.standard_normal(len(xyz))
    a, b = x @ fmm.d_apply(xyz, eta, y, 4), y @ fmm.d_apply(xyz, eta, x, 4)
    assert abs(a - b) <= 1e-13 * abs(a)


_PLANTS = {
    "interaction list without the parent condition": (
        "if _adjacent(c, s) or not _adjacent(pc, tuple(v // 2 for v in s)):", "if _adjacent(c, s):"),
    "nodes not at the Chebyshev points": (
        "np.cos((2.0 * np.arange(1, p + 1) - 1.0) * math.pi / (2.0 * p))",
        "np.cos((2.0 * np.arange(1, p + 1)) * math.pi / (2.0 * p))"),
    "L2L not transposed": ("_node_points(tree, p, l, c)).T @ Lc[l - 1][pc]", "_node_points(tree, p, l, c)) @ Lc[l - 1][pc]"),
}


@pytest.mark.parametrize("plant", sorted(_PLANTS))
def test_convergence_pin_catches_planted_mistakes(orc, fmm, S, plant):
    src = open(os.path.join(os.path.dirname(fmm.__file__), "fmm.py")).read()
    old, new = _PLANTS[plant]
    assert src.count(old) == 1, plant
    ns = {"__name__": "oracle.fmm_planted", "__package__": "oracle"}
    exec(compile(src.replace(old, new), "fmm_planted", "exec"), ns)
    planted = type(fmm)("fmm_planted")
    planted.__dict__.update(ns)
    xyz, eta = _case(S, "flake")
    x = np.random.default_rng(11).standard_normal((len(xyz), 2))
    assert _err(orc, planted, xyz, eta, 6, x) > 1e-4, plant
