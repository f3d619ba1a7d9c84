"""GPU parity of the continuum BEM operator (Section 2.3, Eq. 21-22) against the BEM
oracle (oracle/bem.py), through the C ABI.

The surface is a prolate spheroid (semi-axes 60 and 30 bohr) with 1501 collocation
points: ragged against the 128-row bf16 tiles and the 4-float rows of the FP32 planes.
Tolerances, per element of y = (A - zI) x, relative to the magnitude bound
(|A| |x|)_i + |z| |x_i|:
  * FP64 products: 1e-12 (N-term FP64 sums in another order);
  * double-float products: 8 * 2^-48 * sqrt(N), as for the omega-FQ operator;
  * mixed (3 bf16 products, FP32 accumulation): 4e-5.
Solves: FP64 alpha against the oracle LU to 1e-8 relative; mixed solves to the acceptance
bar (alpha 1e-6, FP64 residual 1e-8 re-measured with the oracle's A); k-step iterates
against the oracle's own GMRES on the same A to 1e-10.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TAU_MIXED = 4e-5
N_SURF = 1501


@pytest.fixture(scope="module")
def W():
    from paper_2103_00438_gb300 import wfq
    wfq.load()
    return wfq


@pytest.fixture(scope="module")
def ctx(W):
    c = W.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def bem():
    from oracle import bem
    return bem


@pytest.fixture(scope="module")
def surf(S, bem):
    s = S.spheroid_surface(N_SURF, 60.0, 30.0)
    A = bem.a_matrix(s["xyz"], s["normal"], s["area"], s["curvature"])
    return s, A, S.drude_metal_params()


def _geom(W, ctx, s, m, store):
    return W.BemGeometry(ctx, s["xyz"], s["normal"], s["area"], s["curvature"], m, store=store)


def _bound(A, z, x):
    return np.abs(A) @ np.abs(x) + abs(z) * np.abs(x)


def test_bem_rhs_matches_oracle(W, ctx, bem, surf):
    s, A, m = surf
    g = _geom(W, ctx, s, m, W.STORE_FP64)
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0.6, 0.0, 0.8]])
    R = g.rhs(dirs, E0=0.7)
    for d in range(len(dirs)):
        ref = bem.rhs(s["normal"], s["area"], dirs[d], E0=0.7)
        assert np.abs(R[:, d] - ref).max() <= 1e-15 * np.abs(ref).max()


@pytest.mark.parametrize("prec,store,ncplx", [("fp64", "fp64", 1), ("fp64", "fp64", 3),
                                              ("df", "f32x2", 7), ("mixed", "bf16", 2), ("mixed", "bf16", 5)])
def test_bem_apply_matches_oracle(W, ctx, bem, S, surf, prec, store, ncplx):
    s, A, m = surf
    flag = W.STORE_FP64 | {"fp64": 0, "f32x2": W.STORE_F32X2, "bf16": W.STORE_BF16X2}[store]
    g = _geom(W, ctx, s, m, flag)
    om = S.ev(np.linspace(2.0, 4.5, ncplx))
    pr = {"fp64": W.PREC_FP64, "df": W.PREC_DF, "mixed": W.PREC_MIXED}[prec]
    tol = {"fp64": 1e-12, "df": 8 * 2.0 ** -48 * np.sqrt(N_SURF), "mixed": TAU_MIXED}[prec]
    x = S.random_complex((N_SURF, ncplx), seed=31 + ncplx)
    if prec == "mixed":
        x = x.astype(np.complex64)
    y = np.empty_like(x)
    g.apply(om, x, y, prec=pr)
    worst = 0.0
    for c in range(ncplx):
        z = bem.z_of_omega(om[c], m)
        xc = x[:, c].astype(np.complex128)
        ref = A @ xc - z * xc
        worst = max(worst, float(np.max(np.abs(y[:, c] - ref) / _bound(A, z, xc))))
    print(prec, "BEM apply: max |dy| / unit bound =", worst)
    assert worst <= tol


@pytest.mark.parametrize("store", ["f32x2", "fp64"])
def test_bem_shifted_gmres_columns_match_lu(W, ctx, bem, S, surf, store):
    """Every (omega, direction) column of one shifted solve -- the frequencies straddle the
    spheroid's two dipole resonances -- equals its own oracle LU solve."""
    s, A, m = surf
    g = _geom(W, ctx, s, m, W.STORE_FP64 | (W.STORE_F32X2 if store == "f32x2" else 0))
    om = S.ev([2.0, 2.6, 3.2, 3.6, 4.5])
    dirs = np.eye(3)
    q, st, status = g.solve_gmres_shifted(om, dirs, rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK"
    al = g.polarizability(q)
    for f in range(len(om)):
        z = bem.z_of_omega(om[f], m)
        for d in range(3):
            c = f * 3 + d
            R = bem.rhs(s["normal"], s["area"], dirs[d]).astype(complex)
            q_lu = bem.solve(A, z, R)
            a_ref = bem.alpha(s["xyz"], q_lu)
            assert np.abs(al[c] - a_ref).max() <= 1e-8 * np.abs(a_ref).max(), (f, d)
            rr = np.linalg.norm(R - (A @ q[:, c] - z * q[:, c])) / np.linalg.norm(R)
            assert rr <= 1.01e-10 and st[c]["rel_residual"] <= 1e-10, (f, d, rr, st[c])


def test_bem_shifted_gmres_iterates_match_oracle_gmres(W, ctx, orc, bem, S, surf):
    """After k Arnoldi steps each column holds the k-step GMRES iterate of its own system,
    computed by the oracle's GMRES on the oracle's dense A.

    Tolerance: 1e-10 relative, or, where the k-step least-squares problem is ill
    conditioned, 30 times the oracle iterate's own change when every entry of A is
    perturbed by 2^-48 relative (seeded signs) -- the rounding level of the double-float
    products.  The largest ratio measured is 10 (3.4 eV, field z, k = 10: 2.6e-10 against a
    sensitivity of 2.6e-11); the factor 30 leaves 3x for the other rounding orders (real
    Arnoldi of A with CGS2 and shifted Givens, against complex Arnoldi of A - zI with MGS)."""
    s, A, m = surf
    g = _geom(W, ctx, s, m, W.STORE_FP64 | W.STORE_F32X2)
    om = S.ev([2.2, 3.4])
    dirs = np.array([[1.0, 0, 0], [0, 0, 1.0]])
    op = orc.Operator.dense(A)
    sign = np.where(np.random.default_rng(48).random(A.shape) < 0.5, -1.0, 1.0)
    op_pert = orc.Operator.dense(A * (1.0 + 2.0 ** -48 * sign))
    for k in (1, 4, 10):
        q, st, status = g.solve_gmres_shifted(om, dirs, m_max=k, rel_tol=1e-14, max_iter=k, prec=W.PREC_FP64)
        assert status == "WFQ_ENOCONV"
        for f in range(len(om)):
            z = bem.z_of_omega(om[f], m)
            for d in range(2):
                c = f * 2 + d
                assert st[c]["iters"] == k
                R = bem.rhs(s["normal"], s["area"], dirs[d]).astype(complex)
                qo, _ = op.gmres(z, R, restart=0, rel_tol=1e-300, max_iter=k)
                qp, _ = op_pert.gmres(z, R, restart=0, rel_tol=1e-300, max_iter=k)
                sens = np.linalg.norm(qp - qo) / np.linalg.norm(qo)
                dev = np.linalg.norm(q[:, c] - qo) / np.linalg.norm(qo)
                print(f"k={k} f={f} d={d}: |q - q_oracle| / |q| = {dev:.2e}, oracle sensitivity {sens:.2e}")
                assert dev <= max(1e-10, 30.0 * sens), (k, f, d, dev, sens)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bem_block_gmres_meets_bar(W, ctx, bem, S, surf, prec):
    s, A, m = surf
    g = _geom(W, ctx, s, m, W.STORE_FP64 | W.STORE_BF16X2)
    om = S.ev([2.4, 3.5, 4.2])
    dirs = np.array([[1.0, 0, 0], [0, 0, 1.0]])
    pr = W.PREC_FP64 if prec == "fp64" else W.PREC_MIXED
    q, st, status = g.solve_gmres(om, dirs, m=30, rel_tol=1e-8, max_iter=3000, prec=pr)
    assert status == "WFQ_OK", st
    al = g.polarizability(q)
    for f in range(len(om)):
        z = bem.z_of_omega(om[f], m)
        for d in range(2):
            c = f * 2 + d
            R = bem.rhs(s["normal"], s["area"], dirs[d]).astype(complex)
            a_ref = bem.alpha(s["xyz"], bem.solve(A, z, R))
            assert np.abs(al[c] - a_ref).max() <= 1e-6 * np.abs(a_ref).max(), (f, d)
            rr = np.linalg.norm(R - (A @ q[:, c] - z * q[:, c])) / np.linalg.norm(R)
            assert rr <= 1e-8 and abs(rr - st[c]["rel_residual"]) <= 1e-10, (f, d, rr, st[c])


def test_bem_sphere_polarizability_on_gpu_tends_to_closed_form(W, ctx, S):
    """A 4000-point sphere through the library alone: alpha_zz within the collocation
    error (1.2 / sqrt(N)) of R^3 (eps_in - 1) / (eps_in + 2), at three frequencies."""
    n, Rs = 4000, 40.0
    s = S.spheroid_surface(n, Rs, Rs)
    m = S.drude_metal_params()
    g = _geom(W, ctx, s, m, W.STORE_FP64 | W.STORE_F32X2)
    om = S.ev([1.0, 2.5, 4.5])
    q, st, status = g.solve_gmres_shifted(om, [[0, 0, 1.0]], rel_tol=1e-10, max_iter=2000, prec=W.PREC_FP64)
    assert status == "WFQ_OK"
    al = g.polarizability(q)[:, 2]
    for f, w in enumerate(om):
        ei = m["eps_inf"] - m["omega_p"] ** 2 / (w * (w + 1j * m["gamma"]))
        ex = Rs ** 3 * (ei - 1.0) / (ei + 2.0)
        assert abs(al[f] / ex - 1.0) < 1.2 / np.sqrt(n), (f, al[f], ex)


def test_bem_geometry_through_the_server(W, ctx, bem, S, surf):
    """BEM requests mixed with omega-FQ requests in the request server: each BEM column
    meets the acceptance bar against its own oracle LU solve."""
    s, A, m = surf
    gb = _geom(W, ctx, s, m, W.STORE_FP64)
    gw = W.Geometry(ctx, S.honeycomb_flake(8), S.carbon_params(1.51), store=W.STORE_F32X2)
    sv = W.Server(ctx, nworkers=2, budget_bytes=8 << 30, max_columns=48)
    reqs = [(gb, S.ev([2.3, 3.3]), np.eye(3)[:2]), (gw, S.ev([0.4, 0.9]), np.eye(3)[:1]),
            (gb, S.ev([4.0]), np.eye(3)[2:]), (gb, S.ev([2.8, 3.9]), np.eye(3))]
    ids = [sv.submit(g, om, d, rel_tol=1e-8) for g, om, d in reqs]
    res = [sv.poll(i, wait=True) for i in ids]
    sv.close()
    for (g, om, d), r in zip(reqs, res):
        assert r["status"] == "WFQ_OK", r["stats"]
        if g is gw:
            continue
        al = g.polarizability(r["q"])
        for f in range(len(om)):
            z = bem.z_of_omega(om[f], m)
            for k in range(len(d)):
                c = f * len(d) + k
                R = bem.rhs(s["normal"], s["area"], d[k]).astype(complex)
                a_ref = bem.alpha(s["xyz"], bem.solve(A, z, R))
                assert np.abs(al[c] - a_ref).max() <= 1e-6 * np.abs(a_ref).max(), (f, k)
                qc = r["q"][:, c]
                assert np.linalg.norm(R - (A @ qc - z * qc)) <= 1e-8 * np.linalg.norm(R)
    gw.close()
    gb.close()


def test_bem_errors(W, ctx, S, surf):
    s, A, m = surf
    g = _geom(W, ctx, s, m, W.STORE_FP64)
    with pytest.raises(W.WfqError) as e:
        g.solve_qmr(S.ev([3.0]), [[1.0, 0, 0]])
    assert e.value.code == -8                       # J-symmetric QMR: no D factor
    with pytest.raises(W.WfqError) as e:
        g.solve_gmres(S.ev([3.0]), [[1.0, 0, 0]], prec=W.PREC_MIXED)
    assert e.value.code == -8                       # mixed needs the bf16 planes
    with pytest.raises(W.WfqError) as e:
        g.solve_gmres_shifted([0.0], [[1.0, 0, 0]])
    assert e.value.code == -2                       # omega = 0
    with pytest.raises(W.WfqError) as e:
        _geom(W, ctx, s, m, W.STORE_F32X2)
    assert e.value.code == -1                       # FP64 storage required
    with pytest.raises(W.WfqError) as e:
        _geom(W, ctx, s, m, W.STORE_FP64 | W.STORE_F32X2_SYM)
    assert e.value.code == -1                       # not symmetric
    bad = dict(s, normal=2.0 * s["normal"])
    with pytest.raises(W.WfqError) as e:
        _geom(W, ctx, bad, m, W.STORE_FP64)
    assert e.value.code == -1                       # normals must be unit vectors
    dup = {k: np.concatenate([v, v[:1]]) for k, v in s.items()}
    with pytest.raises(W.WfqError) as e:
        _geom(W, ctx, dup, m, W.STORE_FP64)
    assert e.value.code == -1                       # two elements at one point
    with pytest.raises(W.WfqError) as e:
        _geom(W, ctx, s, dict(m, omega_p=-1.0), W.STORE_FP64)
    assert e.value.code == -1
    # the allocation-free apply takes omega-FQ geometries only
    gb = _geom(W, ctx, s, m, W.STORE_FP64 | W.STORE_BF16X2)
    import torch
    x = torch.zeros((N_SURF, 1), dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(W.WfqError) as e:
        gb.apply_mixed_noalloc([0.1], x, y)
    assert e.value.code == -8
    gb.close()
    g.close()
