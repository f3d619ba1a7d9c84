"""CPU checks of bench.py's oracle legs: for the BEM workload family the sampled-column
baseline solves the right columns (alpha equal to the oracle's LU to 1e-8) and reports
what it solved; the sampled-row residual estimate of the large solves' audit is unbiased in
its square and its bootstrap interval covers the true value."""
import numpy as np


def test_bem_oracle_sample_matches_lu(S):
    import bench
    from oracle import bem
    surf = S.spheroid_surface(800, 60.0, 30.0)
    wl = {"xyz": surf["xyz"], "surface": surf, "bem": S.drude_metal_params(),
          "omega": S.ev([2.5, 3.5]), "dirs": np.eye(3)}
    assert bench.is_bem(wl)
    solved, secs, alphas, cores, A = bench.oracle_sample_bem(wl, 30.0, [0, 4])
    assert solved == 2 and secs > 0 and cores >= 1 and sorted(alphas) == [0, 4]
    for c, a in alphas.items():
        f, d = divmod(c, 3)
        R = bem.rhs(surf["normal"], surf["area"], wl["dirs"][d]).astype(complex)
        ref = bem.alpha(surf["xyz"], bem.solve(A, bem.z_of_omega(wl["omega"][f], wl["bem"]), R))
        assert np.abs(a - ref).max() <= 1e-8 * np.abs(ref).max()


def _edge_heavy_case(seed):
    """R and a residual both concentrated on 2% of the rows (edges), plus a diffuse part."""
    rng = np.random.default_rng(seed)
    n = 20000
    hot = rng.choice(n, size=n // 50, replace=False)
    R = rng.normal(size=n)
    R[hot] *= 40.0
    r = 1e-9 * (0.3 * np.abs(R) * rng.normal(size=n) + 0.05 * rng.normal(size=n))
    return n, R, r


def test_sampled_residual_estimate_is_unbiased_and_covers():
    """The audit's estimator on an edge-heavy residual: its square is unbiased over many
    draws of the rows, its 95% bootstrap interval holds the true ||r|| / ||R|| in most
    draws, and it beats uniform sampling of the same number of rows."""
    import bench
    n, R, r = _edge_heavy_case(7)
    Rn = np.linalg.norm(R)
    true = np.linalg.norm(r) / Rn
    pr = bench.audit_row_probabilities(R)
    assert abs(pr.sum() - 1.0) < 1e-12 and pr.min() >= 0.5 / n
    rng = np.random.default_rng(11)
    sq, covered, err_is, err_u = [], 0, [], []
    for t in range(300):
        draws = rng.choice(n, size=48, replace=True, p=pr)
        est, lo, hi = bench.sampled_residual_estimate(r[draws], pr[draws], Rn, seed=t, nboot=400)
        assert lo <= est <= hi
        sq.append(est ** 2)
        covered += lo <= true <= hi
        err_is.append(abs(est / true - 1.0))
        u = rng.choice(n, size=48, replace=True)
        est_u, _, _ = bench.sampled_residual_estimate(r[u], np.full(48, 1.0 / n), Rn, seed=t, nboot=10)
        err_u.append(abs(est_u / true - 1.0))
    assert abs(np.mean(sq) / true ** 2 - 1.0) < 0.1
    assert covered >= 0.85 * 300
    assert np.median(err_is) < 0.5 * np.median(err_u)


def test_sampled_residual_estimate_unbiased_for_a_residual_unlike_R():
    """A residual that lives away from R's large rows: still unbiased (every row keeps at
    least half its uniform probability)."""
    import bench
    n, R, _ = _edge_heavy_case(8)
    rng = np.random.default_rng(12)
    r = 1e-9 * rng.normal(size=n)
    r[np.abs(R) > 10] = 0.0
    Rn = np.linalg.norm(R)
    true = np.linalg.norm(r) / Rn
    pr = bench.audit_row_probabilities(R)
    sq = []
    for t in range(400):
        draws = rng.choice(n, size=48, replace=True, p=pr)
        est, _, _ = bench.sampled_residual_estimate(r[draws], pr[draws], Rn, seed=t, nboot=10)
        sq.append(est ** 2)
    assert abs(np.mean(sq) / true ** 2 - 1.0) < 0.1
