"""FP64 CPU oracle of the far-field-compressed D product (a fast multipole method).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the CPU legs of bench.py, never by the
product package.  Plain numpy in FP64, box by box, so that each step can be checked by eye.

What it computes.  u = D x for the charge kernel of Eq. 3, D_ij = erf(r_ij / s_ij) / r_ij
(i != j, s_ij = sqrt(w_i^2 + w_j^2), widths from Eq. 4) and D_ii = eta_i, with the work
split the way the paper's conclusions point to for systems far beyond a million atoms: a
fast multipole method for the far field.  The paper gives no FMM of its own; this one is
the Chebyshev-interpolation ("black-box") FMM of Fong and Darve (J. Comput. Phys. 228,
2009), written from its published description:

  * the atoms are put in a uniform tree over the bounding cube (a quadtree over the
    bounding square when every atom has the same z, as for a flat graphene disk), with
    leaves no smaller than r_far = 6 max_ij s_ij: beyond r_far, erf(r / s_ij) rounds to 1
    in FP64, so every pair the far field handles has D_ij = 1 / r_ij exactly;
  * near field: pairs in the same or adjacent leaves (box indices differing by at most 1
    in every dimension) use Eq. 3 directly;
  * far field: 1 / |t - s| interpolated at p Chebyshev nodes per dimension in the target
    box and in the source box.  With the interpolation weights
        S_p(x_m, y) = 1/p + (2/p) sum_{k=1}^{p-1} T_k(x_m) T_k(y)
    (x_m = cos((2m - 1) pi / (2p)) the Chebyshev nodes of [-1, 1], y a coordinate scaled
    to the box), the steps are P2M (sources to the nodes of their leaf), M2M (child nodes
    to parent nodes), M2L (node-to-node kernel 1 / |t - s| between the boxes of each
    interaction list), L2L (parent nodes to child nodes) and L2P (leaf nodes to targets);
  * interaction list of a box at level l >= 2: the boxes of level l whose parents are
    adjacent to (or equal to) its parent and which are not adjacent to it.  Together with
    the near field every pair (i, j) is counted exactly once.

Pins (tests/test_oracle_fmm_pins.py): everything near -> the exact product; geometric
convergence in p to the exact product; the approximate operator is exactly symmetric
(P2M and L2P are transposes, M2L kernels symmetric); planted mistakes fail.
"""
import math

import numpy as np
from scipy.special import erf as _erf

from . import oracle as _core


def cheb_nodes(p):
    """The p Chebyshev nodes of [-1, 1]: cos((2m - 1) pi / (2p)), m = 1..p."""
    return np.cos((2.0 * np.arange(1, p + 1) - 1.0) * math.pi / (2.0 * p))


def cheb_weights(p, y):
    """S_p(x_m, y) for every node x_m (rows) and every y (columns)."""
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    xm = cheb_nodes(p)
    S = np.full((p, len(y)), 1.0 / p)
    for k in range(1, p):
        S += (2.0 / p) * np.outer(np.cos(k * np.arccos(xm)), np.cos(k * np.arccos(np.clip(y, -1.0, 1.0))))
    return S


def far_radius(eta):
    """r_far = 6 max_ij s_ij with s_ij = sqrt(w_i^2 + w_j^2): erfc(6) < 2^-54, so erf(r / s_ij)
    is 1 in FP64 for every pair at r >= r_far."""
    w = _core.widths(eta)
    return 6.0 * math.sqrt(2.0) * float(np.max(w))


def build_tree(xyz, eta, min_leaf=None):
    """Uniform tree over the bounding cube (square if all z are equal).  Returns a dict with
    dim (2 or 3), depth, root origin and side, the leaf side h, and each atom's integer
    leaf coordinates.  The depth is the largest L with side / 2^L >= r_far."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = len(xyz)
    eta = np.broadcast_to(np.asarray(eta, dtype=np.float64), (n,))
    r_far = far_radius(eta) if min_leaf is None else max(float(min_leaf), far_radius(eta))
    mn, mx = xyz.min(axis=0), xyz.max(axis=0)
    dim = 2 if mx[2] == mn[2] else 3
    ext = (mx - mn)[:dim]
    side = float(ext.max()) * (1.0 + 2.0 ** -20) + 1e-300
    origin = 0.5 * (mn + mx)
    origin[:dim] -= 0.5 * side
    depth = 0
    while side / 2.0 ** (depth + 1) >= r_far:
        depth += 1
    h = side / 2.0 ** depth
    coords = np.floor((xyz[:, :dim] - origin[:dim]) / h).astype(np.int64)
    coords = np.clip(coords, 0, 2 ** depth - 1)
    return {"dim": dim, "depth": depth, "origin": origin, "side": side, "h": h, "r_far": r_far,
            "leaf": coords, "z0": float(mn[2])}


def _box_center(tree, level, c):
    dim = tree["dim"]
    hb = tree["side"] / 2.0 ** level
    ctr = tree["origin"].copy()
    ctr[:dim] = tree["origin"][:dim] + (np.asarray(c, dtype=np.float64) + 0.5) * hb
    if dim == 2:
        ctr[2] = tree["z0"]
    return ctr, 0.5 * hb


def _node_points(tree, p, level, c):
    """Chebyshev nodes of box c at `level` as points (p^dim x 3), node index m = (mx, my[, mz])
    with the last dimension fastest."""
    ctr, a = _box_center(tree, level, c)
    xm = cheb_nodes(p)
    dim = tree["dim"]
    grids = np.meshgrid(*([xm] * dim), indexing="ij")
    pts = np.tile(ctr, (p ** dim, 1))
    for d in range(dim):
        pts[:, d] = ctr[d] + a * grids[d].ravel()
    return pts


def _weights_at(tree, p, level, c, pts):
    """S(node m, point) for the p^dim nodes of box c and the given points: the product over
    dimensions of S_p(x_{m_d}, (pt_d - center_d) / a)."""
    ctr, a = _box_center(tree, level, c)
    dim = tree["dim"]
    W1 = [cheb_weights(p, (pts[:, d] - ctr[d]) / a) for d in range(dim)]
    if dim == 2:
        return np.einsum("ai,bi->abi", W1[0], W1[1]).reshape(p * p, len(pts))
    return np.einsum("ai,bi,ci->abci", W1[0], W1[1], W1[2]).reshape(p ** 3, len(pts))


def _adjacent(c1, c2):
    return np.max(np.abs(np.asarray(c1) - np.asarray(c2))) <= 1


def d_apply(xyz, eta, x, p, min_leaf=None, tree=None):
    """u = D x (x: n or n x C, real or complex) by the FMM described in the module header."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = len(xyz)
    eta = np.broadcast_to(np.asarray(eta, dtype=np.float64), (n,)).copy()
    x = np.asarray(x)
    one = x.ndim == 1
    X = x.reshape(n, -1)
    if tree is None:
        tree = build_tree(xyz, eta, min_leaf)
    dim, L = tree["dim"], tree["depth"]
    leaf = [tuple(c) for c in tree["leaf"]]
    members = {}
    for i, c in enumerate(leaf):
        members.setdefault(c, []).append(i)
    U = np.zeros_like(X, dtype=np.result_type(X.dtype, np.float64))

    # near field: Eq. 3 for pairs in the same or adjacent leaves
    w = _core.widths(eta)
    for c, idx in members.items():
        idx = np.array(idx)
        src = np.array([j for c2, js in members.items() if _adjacent(c, c2) for j in js])
        for i in idx:
            d = xyz[src] - xyz[i]
            r = np.sqrt(np.einsum("jk,jk->j", d, d))
            self_ = src == i
            r[self_] = 1.0
            row = _erf(r / np.sqrt(w[i] ** 2 + w[src] ** 2)) / r
            row[self_] = eta[i]
            U[i] += row @ X[src]
    if L < 2:
        return U[:, 0] if one else U

    # boxes per level (non-empty), bottom-up multipole coefficients
    boxes = [None] * (L + 1)
    boxes[L] = sorted(members)
    for l in range(L - 1, -1, -1):
        boxes[l] = sorted({tuple(v // 2 for v in c) for c in boxes[l + 1]})
    P = p ** dim
    M = [dict() for _ in range(L + 1)]
    for c in boxes[L]:                                                     # P2M
        idx = np.array(members[c])
        M[L][c] = _weights_at(tree, p, L, c, xyz[idx]) @ X[idx]
    for l in range(L - 1, 1, -1):                                          # M2M
        for c in boxes[l]:
            acc = np.zeros((P, X.shape[1]), dtype=U.dtype)
            for ch in boxes[l + 1]:
                if tuple(v // 2 for v in ch) == c:
                    acc += _weights_at(tree, p, l, c, _node_points(tree, p, l + 1, ch)) @ M[l + 1][ch]
            M[l][c] = acc
    Lc = [dict() for _ in range(L + 1)]
    for l in range(2, L + 1):                                              # M2L
        for c in boxes[l]:
            acc = np.zeros((P, X.shape[1]), dtype=U.dtype)
            pc = tuple(v // 2 for v in c)
            t_pts = _node_points(tree, p, l, c)
            for s in boxes[l]:
                if _adjacent(c, s) or not _adjacent(pc, tuple(v // 2 for v in s)):
                    continue
                s_pts = _node_points(tree, p, l, s)
                d = t_pts[:, None, :] - s_pts[None, :, :]
                K = 1.0 / np.sqrt(np.einsum("abk,abk->ab", d, d))
                acc += K @ M[l][s]
            Lc[l][c] = acc
    for l in range(3, L + 1):                                              # L2L
        for c in boxes[l]:
            pc = tuple(v // 2 for v in c)
            Lc[l][c] = Lc[l][c] + _weights_at(tree, p, l - 1, pc, _node_points(tree, p, l, c)).T @ Lc[l - 1][pc]
    for c in boxes[L]:                                                     # L2P
        idx = np.array(members[c])
        U[idx] += _weights_at(tree, p, L, c, xyz[idx]).T @ Lc[L][c]
    return U[:, 0] if one else U


def apply(xyz, p_params, csr, z, x, order, min_leaf=None):
    """y = (A - zI) x = (Kbar - P)(D x) - z x (Eq. 17) with D x from the FMM (one column)."""
    u = d_apply(xyz, p_params["eta"], x, order, min_leaf)
    rowptr, col, val = csr
    y = np.empty_like(u)
    for i in range(len(u)):
        js, ks = col[rowptr[i]:rowptr[i + 1]], val[rowptr[i]:rowptr[i + 1]]
        y[i] = np.sum(ks * (u[js] - u[i]))
    return y - z * np.asarray(x)
