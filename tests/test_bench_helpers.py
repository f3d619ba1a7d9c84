"""CPU checks of bench.py's oracle legs for the BEM workload family: the sampled-column
baseline solves the right columns (alpha equal to the oracle's LU to 1e-8) and reports
what it solved."""
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
