"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself: closed forms (dimer, static and high-frequency limits,
modal expansion), independent quadrature of the Gaussian Coulomb overlap,
invariants stated in Section 2.1 (D SPD, 1^T A = 0, DA = A^T D, real spectrum),
the GMRES minimal-residual property checked by brute-force least squares, and LU
vs Krylov agreement.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate, linalg

KX, KY, KZ = np.eye(3)


def _params(S, **kw):
    p = S.carbon_params(1.51)
    p.update(kw)
    return p


# --------------------------------------------------------------------- Eq. 3 / Eq. 4

def _gauss_coulomb_quadrature(r, w1, w2):
    """Coulomb energy of two unit Gaussian charges exp(-r^2/w^2)/(pi^1.5 w^3) at
    distance r, from the Fourier representation (form factors exp(-k^2 w^2/4),
    Coulomb kernel 4 pi / k^2):  (2/pi) int_0^inf exp(-k^2 (w1^2+w2^2)/4) sin(kr)/(kr) dk.
    Independent of erf."""
    s2 = w1 * w1 + w2 * w2
    f = lambda k: math.exp(-k * k * s2 / 4.0) * (math.sin(k * r) / (k * r) if k > 0 else 1.0)
    kmax = 40.0 / math.sqrt(s2)
    val, _ = integrate.quad(f, 0.0, kmax, limit=400, epsabs=1e-14, epsrel=1e-13)
    return 2.0 / math.pi * val


def test_d_entry_is_gaussian_coulomb_overlap(orc):
    rng = np.random.default_rng(1)
    for _ in range(12):
        eta = rng.uniform(0.2, 1.2, size=2)
        r = rng.uniform(0.3, 12.0)
        xyz = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        w = orc.widths(eta)
        got = orc.d_matrix(xyz, eta)[0, 1]
        ref = _gauss_coulomb_quadrature(r, w[0], w[1])
        assert abs(got - ref) <= 1e-11 * abs(ref), (got, ref)


def test_width_rule_reproduces_diagonal_limit(orc):
    # Eq. 4: the r -> 0 limit of the off-diagonal entry equals eta (same species)
    for eta in (0.25, 0.6, 1.3):
        xyz = np.array([[0.0, 0.0, 0.0], [1e-6, 0.0, 0.0]])
        D = orc.d_matrix(xyz, eta)
        assert D[0, 0] == eta
        assert abs(D[0, 1] - eta) < 1e-9 * eta


def test_d_far_field_is_coulomb(orc):
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 80.0]])
    D = orc.d_matrix(xyz, 0.6)
    assert D[0, 1] == pytest.approx(1.0 / 80.0, rel=1e-15)


def test_d_symmetric_positive_definite(orc, S):
    xyz = S.random_cluster(150, seed=3)
    eta = np.random.default_rng(3).uniform(0.4, 0.9, 150)
    D = orc.d_matrix(xyz, eta)
    assert np.array_equal(D, D.T)
    linalg.cholesky(D)  # raises unless SPD (Section 2: D is SPD)


# --------------------------------------------------------------------- Eq. 6 / Eq. 9

def test_fermi_damping_shape(orc, S):
    p = _params(S)
    r_mid = p["s_fermi"] * p["r0"]
    assert orc.fermi(r_mid, p) == pytest.approx(0.5, abs=1e-15)
    rs = np.linspace(0.5 * r_mid, 3 * r_mid, 50)
    f = np.array([orc.fermi(r, p) for r in rs])
    assert np.all(np.diff(f) > 0)                  # damping grows with distance
    assert f[0] < 5e-3 and f[-1] > 1 - 1e-9
    # Kbar = (1 - f) A / r: half the bare Drude value at r = s r0, vanishing far away
    assert orc.kbar_entry(r_mid, p) == pytest.approx(0.5 * p["area"] / r_mid, rel=1e-14)
    assert orc.kbar_entry(4 * r_mid, p) < 1e-14


def test_kbar_csr_equals_dense_and_cutoff_is_harmless(orc, S):
    xyz = S.honeycomb_flake(4)
    p = _params(S)
    K = orc.kbar_matrix(xyz, p)
    assert np.array_equal(K, K.T) and np.all(np.diag(K) == 0)
    rowptr, col, val = orc.kbar_csr(xyz, p, cutoff_eps=0.0)
    dense = np.zeros_like(K)
    for i in range(len(xyz)):
        dense[i, col[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    assert np.array_equal(dense, K)
    # cutoff at 1 - f >= 1e-16 changes the solution by far less than any tolerance used
    sys_d = orc.System(xyz, p)
    sys_c = orc.System(xyz, p, dense=False)
    om = S.ev(0.8)
    qd, _ = sys_d.solve(om, KX, method="lu")
    qc, info = sys_c.solve(om, KX, method="gmres", rel_tol=1e-14)
    ad = orc.alpha(xyz, qd)[0]
    ac = orc.alpha(xyz, qc)[0]
    assert abs(ad - ac) <= 1e-11 * abs(ad)


# --------------------------------------------------------------------- Eq. 11 / 16 / 17

def test_a_matrix_definition_properties(orc, S):
    xyz = S.random_cluster(60, seed=5)
    p = _params(S, r0=2.7)
    D = orc.d_matrix(xyz, p["eta"])
    K = orc.kbar_matrix(xyz, p)
    A = orc.a_matrix(D, K)
    # product form of Eq. 17 with P from Eq. 16 (numpy matmul as an independent route)
    P = np.diag(K.sum(axis=1))
    np.testing.assert_allclose(A, (K - P) @ D, rtol=0, atol=1e-13 * np.abs(A).max())
    # 1^T A = 0 (Kbar - P has zero column sums), DA = A^T D (Eq. 18)
    assert np.abs(A.sum(axis=0)).max() <= 1e-13 * np.abs(A).max()
    np.testing.assert_allclose(D @ A, A.T @ D, atol=1e-13 * np.abs(D @ A).max())
    # real spectrum (D-self-adjointness, Eq. 20), one exact zero eigenvalue family
    ev = np.linalg.eigvals(A)
    assert np.abs(ev.imag).max() <= 1e-10 * np.abs(ev).max()
    assert ev.real.max() <= 1e-10 * np.abs(ev).max()      # A = -(P - Kbar) D is NSD-similar


def test_operator_kinds_agree(orc, S):
    xyz = S.random_cluster(80, seed=6)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    z = sysm.z(S.ev(0.7))
    x = S.random_complex(80, seed=7)
    y_dense = orc.Operator.dense(sysm.A).apply(z, x)
    y_stored = orc.Operator.stored(sysm.D, sysm.csr).apply(z, x)
    y_otf = orc.Operator.on_the_fly(sysm.xyz, sysm.eta, sysm.csr).apply(z, x)
    scale = np.abs(y_dense).max()
    assert np.abs(y_stored - y_dense).max() <= 1e-13 * scale
    assert np.abs(y_otf - y_dense).max() <= 1e-13 * scale


def test_apply_rows_equals_full_apply(orc, S):
    xyz = S.random_cluster(150, seed=8)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    z = sysm.z(S.ev(0.9))
    x = S.random_complex(150, seed=2)
    full = orc.Operator.dense(sysm.A).apply(z, x)
    rows = np.array([0, 7, 77, 149])
    y, bound = orc.apply_rows(xyz, dict(p, cutoff_eps=0.0), z, x, rows)
    assert np.abs(y - full[rows]).max() <= 1e-13 * np.abs(full).max()
    assert np.all(bound >= np.abs(full[rows]))


# --------------------------------------------------------------------- closed forms

def test_dimer_closed_form(orc, S):
    """N = 2 along x at distance a: (A - zI) q = R reduces to one scalar equation,
    alpha_xx = Kbar12 a^2 / (2 Kbar12 (eta - D12) + z)."""
    p = _params(S)
    a = 3.1
    xyz = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0]])
    sysm = orc.System(xyz, p)
    k12 = orc.kbar_entry(a, p)
    d12 = orc.d_matrix(xyz, p["eta"])[0, 1]
    for om_ev in (0.05, 0.3, 1.0, 3.0):
        om = S.ev(om_ev)
        z = orc.z_of_omega(om, p)
        q, _ = sysm.solve(om, KX, method="lu")
        al = orc.alpha(xyz, q)
        ref = k12 * a * a / (2 * k12 * (p["eta"] - d12) + z)
        assert abs(al[0] - ref) <= 1e-13 * abs(ref)
        assert abs(al[1]) == 0 and abs(al[2]) == 0


def _modal_alpha(D, K, X, n0, tau, om):
    """alpha tensor from the eigen-decomposition of D^1/2 (P - Kbar) D^1/2
    (a derivation independent of the solve): alpha_ab = sum_n c_n^a c_n^b Om_n^2 /
    (Om_n^2 - om^2 - i om/tau), Om_n^2 = 2 n0 lam_n, c_n^a = v_n^T D^-1/2 x_a."""
    w, U = np.linalg.eigh(D)
    Dh = (U * np.sqrt(w)) @ U.T
    Dmh = (U / np.sqrt(w)) @ U.T
    L = np.diag(K.sum(1)) - K
    lam, V = np.linalg.eigh(Dh @ L @ Dh)
    C = V.T @ (Dmh @ X)                  # (modes, 3)
    Om2 = 2 * n0 * lam
    g = Om2 / (Om2 - om * om - 1j * om / tau)
    return np.einsum("na,n,nb->ab", C, g, C)


def test_modal_expansion_full_tensor(orc, S):
    xyz = S.random_cluster(70, seed=11)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    for om_ev in (0.1, 0.5, 1.2, 2.5):
        om = S.ev(om_ev)
        ref = _modal_alpha(sysm.D, sysm.K, xyz, p["n0"], p["tau"], om)
        got = np.zeros((3, 3), dtype=complex)
        for b, kdir in enumerate(np.eye(3)):
            q, _ = sysm.solve(om, kdir, method="lu")
            got[:, b] = orc.alpha(xyz, q)
            assert abs(q.sum()) <= 1e-12 * np.abs(q).sum()     # charge conservation
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        assert np.all(np.diag(got).imag >= 0)                   # lossy Drude response
        np.testing.assert_allclose(got, got.T, atol=1e-10 * np.abs(got).max())  # reciprocity


def test_static_limit_perfect_conductor(orc, S):
    """omega -> 0: equipotential conductor, alpha = k^T D^-1 k - (1^T D^-1 k)^2 / (1^T D^-1 1)."""
    xyz = S.random_cluster(50, seed=12)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    k = xyz[:, 0]
    c = linalg.cho_factor(sysm.D)
    Dk = linalg.cho_solve(c, k)
    D1 = linalg.cho_solve(c, np.ones(len(k)))
    ref = k @ Dk - (np.ones(len(k)) @ Dk) ** 2 / (np.ones(len(k)) @ D1)
    # the correction is O(omega / (tau Omega_min^2)): 2.6e-5 relative at omega = 1e-6
    errs = []
    for om in (1e-7, 1e-8):
        q, _ = sysm.solve(om, KX, method="lu")
        errs.append(abs(orc.alpha(xyz, q)[0] - ref) / abs(ref))
    assert errs[1] <= 1e-6 and errs[1] < 0.2 * errs[0]


def test_high_frequency_sum_rule(orc, S):
    """omega >> all modes: alpha_xx -> -(2 n0 / omega^2) * 1/2 sum_ij Kbar_ij (x_i - x_j)^2."""
    xyz = S.random_cluster(40, seed=13)
    p = _params(S, r0=2.7, tau=1e9)
    sysm = orc.System(xyz, p)
    x = xyz[:, 0]
    fsum = 0.5 * np.sum(sysm.K * (x[:, None] - x[None, :]) ** 2)
    om = 50.0
    q, _ = sysm.solve(om, KX, method="lu")
    al = orc.alpha(xyz, q)[0]
    ref = -2 * p["n0"] / om ** 2 * fsum
    assert abs(al - ref) <= 1e-4 * abs(ref)


def test_translation_and_rotation_covariance(orc, S):
    xyz = S.random_cluster(45, seed=14)
    p = _params(S, r0=2.7)
    om = S.ev(0.9)
    base = orc.System(xyz, p)
    Rm = linalg.expm(np.array([[0, -0.3, 0.2], [0.3, 0, -0.5], [-0.2, 0.5, 0]]))
    moved = orc.System(xyz @ Rm.T + np.array([5.0, -3.0, 7.0]), p)
    a0 = np.zeros((3, 3), dtype=complex)
    a1 = np.zeros((3, 3), dtype=complex)
    for b, kdir in enumerate(np.eye(3)):
        R0 = base.rhs(kdir)
        R1 = orc.System(xyz + 11.0, p).rhs(kdir)
        np.testing.assert_allclose(R0, R1, atol=1e-12 * np.abs(R0).max())   # V differences only
        a0[:, b] = orc.alpha(base.xyz, base.solve(om, kdir)[0])
        a1[:, b] = orc.alpha(moved.xyz, moved.solve(om, kdir)[0])
    np.testing.assert_allclose(a1, Rm @ a0 @ Rm.T, atol=1e-10 * np.abs(a0).max())


# --------------------------------------------------------------------- solvers

def test_lu_solution_has_tiny_residual(orc, S):
    xyz = S.random_cluster(120, seed=15)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    om = S.ev(0.6)
    z = sysm.z(om)
    R = sysm.rhs(KX).astype(complex)
    q, _ = sysm.solve(om, KX, method="lu")
    M = sysm.A - z * np.eye(len(q))
    assert np.linalg.norm(R - M @ q) <= 1e-12 * np.linalg.norm(R)


def test_gmres_iterates_minimise_residual_over_krylov_space(orc, S):
    """Eq. 24: x_m is the minimiser of ||R - M x|| over K_m(M, R) (x0 = 0) -- checked
    against brute-force least squares on an orthonormalised Krylov basis."""
    xyz = S.random_cluster(40, seed=16)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    z = sysm.z(S.ev(0.7))
    R = sysm.rhs(KX).astype(complex)
    M = sysm.A - z * np.eye(40)
    op = orc.Operator.dense(sysm.A)
    Kr = [R]
    for m in range(1, 9):
        x, info = op.gmres(z, R, restart=0, rel_tol=1e-300, max_iter=m)
        assert info["iters"] == m
        Q, _ = np.linalg.qr(np.stack(Kr, axis=1))
        y, *_ = np.linalg.lstsq(M @ Q, R, rcond=None)
        xref = Q @ y
        assert np.linalg.norm(x - xref) <= 1e-8 * np.linalg.norm(xref)
        Kr.append(M @ Kr[-1])


def test_gmres_full_and_restarted_match_lu(orc, S):
    xyz = S.honeycomb_flake(6)
    p = _params(S)
    sysm = orc.System(xyz, p)
    for om_ev in (0.3, 1.1):
        om = S.ev(om_ev)
        q_lu, _ = sysm.solve(om, KX, method="lu")
        q_g, info = sysm.solve(om, KX, method="gmres", rel_tol=1e-12)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-11
        assert np.linalg.norm(q_g - q_lu) <= 1e-9 * np.linalg.norm(q_lu)
        q_r, info_r = sysm.solve(om, KX, method="gmres", rel_tol=1e-12, restart=5,
                                 max_iter=5000)
        assert info_r["status"] == 0 and info_r["restarts"] >= 1
        assert np.linalg.norm(q_r - q_lu) <= 1e-9 * np.linalg.norm(q_lu)


def test_qmr_matches_lu_and_stays_in_krylov_space(orc, S):
    xyz = S.honeycomb_flake(5)
    p = _params(S)
    sysm = orc.System(xyz, p)
    om = S.ev(0.9)
    z = sysm.z(om)
    R = sysm.rhs(KX).astype(complex)
    q_lu, _ = sysm.solve(om, KX, method="lu")
    q_q, info = sysm.solve(om, KX, method="qmr", rel_tol=1e-12, max_iter=3000)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    assert np.linalg.norm(q_q - q_lu) <= 1e-8 * np.linalg.norm(q_lu)
    # after k steps the QMR iterate lies in K_k(M, R), and its residual is never below
    # the GMRES (minimal) residual of the same step
    M = sysm.A - z * np.eye(len(R))
    op = sysm.operator()
    Kr = [R]
    for k in range(1, 7):
        xq, _ = op.qmr(z, R, rel_tol=1e-300, max_iter=k)
        xg, _ = op.gmres(z, R, rel_tol=1e-300, max_iter=k)
        Q, _ = np.linalg.qr(np.stack(Kr, axis=1))
        assert np.linalg.norm(xq - Q @ (Q.conj().T @ xq)) <= 1e-9 * np.linalg.norm(xq)
        assert np.linalg.norm(R - M @ xq) >= np.linalg.norm(R - M @ xg) * (1 - 1e-10)
        Kr.append(M @ Kr[-1])


def _krylov_basis(M, R, k):
    """Orthonormal basis of K_k(M, R) by Arnoldi with two Gram-Schmidt passes (numpy)."""
    Q = np.zeros((len(R), k), dtype=complex)
    Q[:, 0] = R / np.linalg.norm(R)
    for j in range(1, k):
        w = M @ Q[:, j - 1]
        for _ in range(2):
            w = w - Q[:, :j] @ (Q[:, :j].conj().T @ w)
        Q[:, j] = w / np.linalg.norm(w)
    return Q


def _qmr_from_bcg_brute_force(M, D, R, kmax):
    """k-step J-symmetric QMR iterates (J = D, Section 3) built with no Lanczos recurrence.

    BCG: x_k lies in K_k(M, R) and its residual R - M x_k is orthogonal, in the bilinear
    form u^T D v (no conjugation), to all of K_k(M, R); for M^T D = D M (Eq. 18 with the
    shift) the shadow space K_k(M^T, D R) is D K_k(M, R), so this is the Petrov-Galerkin
    condition of BCG with the shadow start D R.  Solved as a dense k x k system.

    QMR from BCG: with Lanczos vectors of unit Euclidean length the QMR iterate is the
    weighted mean of the BCG iterates x_0 = 0, x_1, ..., x_k with weights proportional to
    1 / ||r_i||^2 (quasi-residual tau_k^2 = 1 / sum_i ||r_i||^-2)."""
    xs, inv = [np.zeros_like(R)], [1.0 / np.vdot(R, R).real]
    out = []
    for k in range(1, kmax + 1):
        Q = _krylov_basis(M, R, k)
        y = np.linalg.solve(Q.T @ D @ M @ Q, Q.T @ D @ R)
        x = Q @ y
        r = R - M @ x
        xs.append(x)
        inv.append(1.0 / np.vdot(r, r).real)
        w = np.array(inv) / np.sum(inv)
        out.append(sum(wi * xi for wi, xi in zip(w, xs)))
    return out


def _qmr_system(orc, S):
    sysm = orc.System(S.honeycomb_flake(5), _params(S))
    z = sysm.z(S.ev(0.9))
    R = sysm.rhs(KX).astype(complex)
    M = sysm.A - z * np.eye(len(R))
    return sysm, z, R, M


def _qmr_pin_deviation(op, sysm, z, R, M, library=None, kmax=8):
    ref = _qmr_from_bcg_brute_force(M, sysm.D, R, kmax)
    dev = []
    for k in range(1, kmax + 1):
        xq, info = op.qmr(z, R, rel_tol=1e-300, max_iter=k, library=library)
        assert info["iters"] == k
        dev.append(np.linalg.norm(xq - ref[k - 1]) / np.linalg.norm(ref[k - 1]))
    return max(dev)


def test_qmr_iterates_are_smoothed_bcg_iterates(orc, S):
    # each k-step oracle QMR iterate equals the brute-force BCG + closed-form smoothing
    sysm, z, R, M = _qmr_system(orc, S)
    assert _qmr_pin_deviation(sysm.operator(), sysm, z, R, M) <= 1e-9


_QMR_PLANTS = {
    "smoothing weight divided by ||r|| once": (
        "double wgt = tau2_new / (rn * rn);", "double wgt = tau2_new / rn;"),
    "quasi-residual not accumulated": (
        "double tau2_new = 1.0 / (1.0 / tau2 + 1.0 / (rn * rn));",
        "double tau2_new = 1.0 / (1.0 / (rn * rn));"),
    "beta inverted": ("cplx beta = rho_new / rho;", "cplx beta = rho / rho_new;"),
    "conjugating form": ("for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];",
                         "for (int64_t i = 0; i < n; ++i) s += conj(u[i]) * v[i];"),
}


@pytest.mark.parametrize("plant", sorted(_QMR_PLANTS))
def test_qmr_pin_catches_planted_mistakes(orc, S, tmp_path, plant):
    # a copy of the oracle's source with one plausible mistake fails the pin above
    import os, subprocess
    src = open(os.path.join(os.path.dirname(orc.__file__), "wfq_oracle.c")).read()
    old, new = _QMR_PLANTS[plant]
    assert src.count(old) == 1, plant
    c = tmp_path / "planted.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libplanted.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", str(c), "-o", str(so),
                    "-lm"], check=True)
    sysm, z, R, M = _qmr_system(orc, S)
    assert _qmr_pin_deviation(sysm.operator(), sysm, z, R, M, library=orc.load(str(so))) > 1e-6


def test_rhs_rows_equal_the_assembled_rhs(orc, S):
    # the brute-force row form of Eq. 13 used by residual audits of large structures
    xyz = S.random_cluster(300, seed=8)
    p = _params(S, r0=2.7)
    K = orc.kbar_matrix(xyz, p)
    rows = np.arange(0, 300, 7)
    for k in (KX, np.array([0.6, 0.0, 0.8])):
        R = orc.rhs_dense(xyz, K, k, E0=0.7)
        np.testing.assert_allclose(orc.rhs_rows(xyz, p, k, rows, E0=0.7), R[rows], rtol=0,
                                   atol=1e-13 * np.abs(R).max())


def test_qmr_on_the_fly_equals_stored(orc, S):
    xyz = S.random_cluster(90, seed=17)
    p = _params(S, r0=2.7)
    sysm = orc.System(xyz, p)
    om = S.ev(0.5)
    z = sysm.z(om)
    R = sysm.rhs(KY).astype(complex)
    a, _ = orc.Operator.stored(sysm.D, sysm.csr).qmr(z, R, rel_tol=1e-12)
    b, _ = orc.Operator.on_the_fly(sysm.xyz, sysm.eta, sysm.csr).qmr(z, R, rel_tol=1e-12)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


# --------------------------------------------------------------------- Section 4 tables

def test_structures_reproduce_paper_tables(S):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    for row in gold["cnt"]:
        n, m = row["chirality"]
        per_cell, period, diam = S.nanotube_cell(n, m)
        ncells = round(row["L_nm"] * 10.0 / period)
        assert per_cell * ncells == row["atoms"], row
        dC = gold["b_G_nm"] / math.pi * math.sqrt(n * n + m * m + n * m)
        if row["id"] != "CNT2":            # (16,24) is printed as 2.77 nm; the formula gives 2.73
            assert abs(dC - row["d_nm"]) <= 0.006, row
        assert abs(diam / 10.0 - dC) <= 0.01     # 1.42 A bond vs 0.246 nm lattice rounding
    assert len(S.nanotube(8, 12, 27)) == 8208
    for row in gold["gd"]:
        n = len(S.graphene_disk(row["d_nm"]))
        assert abs(n - row["atoms"]) <= 0.015 * row["atoms"], (row, n)
    for k in (1, 2, 5, 13):
        assert len(S.honeycomb_flake(k)) == 6 * k * k
